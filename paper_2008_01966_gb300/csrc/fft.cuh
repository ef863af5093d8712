// Shared-memory FFTs of power-of-two length for the cavity solver.
//
// All transforms of the hot path -- the Fourier-series synthesis (E123F), the
// trapezoid projections and the torus convolution of Sec. 5.2 -- are batches
// of 1-D transforms of lines held in shared memory.
//
// Two algorithms:
//  * warp transform (FP32, 64 <= n <= 1024): the line is split as n = LW x RV
//    (LW lanes, RV values per lane, RV = LW or 2 LW); each lane does an RV-point
//    DFT in registers, the twiddle w_n^{l k1}, one transpose through shared
//    memory and an LW-point DFT in registers (the "four-step" factorisation).
//    Only warp-level synchronisation inside the transform.
//  * block transform (FP64, and FP32 lines outside that range): Stockham
//    auto-sort with radix-8 passes, each thread owning 8 slots of a line per
//    pass; inputs are read from shared memory into registers, twiddled,
//    transformed and written back in place after a CTA barrier.
// Lines use a padded layout (one pad word per 16 elements, see pidx) so that
// strided accesses do not collide in the shared-memory banks.  Twiddles come
// from a table tw[k] = exp(-2 pi i k / TW) computed once in FP64 (rounded for
// the FP32 table); the block transform forms FP32 powers of the table value by
// multiplication (at most 7 products, ~5e-7 relative) and reads every FP64
// power from the table.  Forward = exp(-...), inverse = exp(+...),
// unnormalised.
//
// Contract: a CTA transforms `nlines` lines of length n = 2^logn stored at
// line_base + l * lstride (padded indices, lstride >= padded_len(n)).  Threads
// 0 .. nlines*tpl-1 do the work, tpl = fft_tpl<T>(n); all threads of the CTA
// must call (barriers).
#pragma once
#include "common.cuh"

__host__ __device__ constexpr int pidx(int i) { return i + (i >> 4); }
// line length in shared memory: room for the padded layout and for the
// transposed tile of the warp transform (n + n/8 for n >= 64)
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 3) + 2; }
// block transform: elements per thread (radix up to 8), and at most
// FFT_MAX_TPL threads per line: lines longer than 8 FFT_MAX_TPL points give
// each thread several butterflies per pass (16 points per thread at 4096)
template <typename T> struct FftE { static constexpr int E = 8, LRMAX = 3; };
#define FFT_MAX_TPL 256
// warp transform (FP32, 64 <= n <= 1024): n = LW * RV lanes x values per lane
__host__ __device__ constexpr bool warp_fft_ok(int n, int elem_bytes) {
  return elem_bytes == 8 && n >= 64 && n <= 1024;
}
__host__ __device__ constexpr int warp_lanes(int n) {
  int lg = 0;
  while ((1 << lg) < n) ++lg;
  return 1 << (lg >> 1);
}
// threads cooperating on one line (same as LineShape<T, log2 n>::TPL)
template <typename T> __host__ __device__ constexpr int fft_tpl(int n) {
  if (warp_fft_ok(n, (int)sizeof(C<T>))) return warp_lanes(n);
  return n >= FftE<T>::E ? (n / FftE<T>::E < FFT_MAX_TPL ? n / FftE<T>::E : FFT_MAX_TPL) : 1;
}

// twiddle constants (forward sign); the inverse uses the conjugates
#define FFT_C8 0.70710678118654752440
#define FFT_C16 0.92387953251128675613
#define FFT_S16 0.38268343236508977173

template <typename T, bool INV>
__device__ __forceinline__ C<T> mulw(C<T> v, T c, T s) {
  // v * (c - i s) forward, v * (c + i s) inverse
  if (!INV) return mk<T>(v.x * c + v.y * s, v.y * c - v.x * s);
  return mk<T>(v.x * c - v.y * s, v.y * c + v.x * s);
}
// v * (-i) forward / (+i) inverse
template <typename T, bool INV> __device__ __forceinline__ C<T> mulmi(C<T> v) {
  return INV ? mk<T>(-v.y, v.x) : mk<T>(v.y, -v.x);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(C<T>* v) {
  C<T> a = v[0], b = v[1];
  v[0] = cadd<T>(a, b);
  v[1] = csub<T>(a, b);
}

// in-register 4-point DFT of v[0], v[st], v[2st], v[3st]
template <typename T, bool INV>
__device__ __forceinline__ void dft4s(C<T>* v, int st) {
  C<T> a0 = v[0], a1 = v[st], a2 = v[2 * st], a3 = v[3 * st];
  C<T> s0 = cadd<T>(a0, a2), d0 = csub<T>(a0, a2);
  C<T> s1 = cadd<T>(a1, a3), d1 = csub<T>(a1, a3);
  C<T> e = mulmi<T, INV>(d1);
  v[0] = cadd<T>(s0, s1);
  v[2 * st] = csub<T>(s0, s1);
  v[st] = cadd<T>(d0, e);
  v[3 * st] = csub<T>(d0, e);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(C<T>* v) { dft4s<T, INV>(v, 1); }

template <typename T, bool INV>
__device__ __forceinline__ void dft8(C<T>* v) {
  // even / odd halves, then combine with w8^k
  C<T> e[4] = {v[0], v[2], v[4], v[6]};
  C<T> o[4] = {v[1], v[3], v[5], v[7]};
  dft4<T, INV>(e);
  dft4<T, INV>(o);
  const T c = (T)FFT_C8;
  o[1] = mulw<T, INV>(o[1], c, c);
  o[2] = mulmi<T, INV>(o[2]);
  o[3] = mulw<T, INV>(o[3], -c, c);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[k] = cadd<T>(e[k], o[k]);
    v[k + 4] = csub<T>(e[k], o[k]);
  }
}

// 16-point DFT in place, output in transposed order: on return v[4 r + s]
// holds X[r + 4 s] (dft16_out maps an output index to its slot).
template <typename T, bool INV>
__device__ __forceinline__ void dft16(C<T>* v) {
  // n = c + 4 t, k = r + 4 s:  u_c[r] = DFT4_t(v[c + 4t]);  u_c[r] *= w16^{c r};
  // X[r + 4 s] = DFT4_c(u_c[r])
#pragma unroll
  for (int c = 0; c < 4; ++c) dft4s<T, INV>(v + c, 4);   // v[c + 4 r] = u_c[r]
  const T c1 = (T)FFT_C16, s1 = (T)FFT_S16, c2 = (T)FFT_C8;
  v[5] = mulw<T, INV>(v[5], c1, s1);
  v[9] = mulw<T, INV>(v[9], c2, c2);
  v[13] = mulw<T, INV>(v[13], s1, c1);
  v[6] = mulw<T, INV>(v[6], c2, c2);
  v[10] = mulmi<T, INV>(v[10]);
  v[14] = mulw<T, INV>(v[14], -c2, c2);
  v[7] = mulw<T, INV>(v[7], s1, c1);
  v[11] = mulw<T, INV>(v[11], -c2, c2);
  v[15] = mulw<T, INV>(v[15], -c1, -s1);
#pragma unroll
  for (int r = 0; r < 4; ++r) dft4s<T, INV>(v + 4 * r, 1);  // v[4 r + s] = X[r + 4 s]
}
__host__ __device__ constexpr int dft16_slot(int k) { return 4 * (k & 3) + (k >> 2); }

// 32-point DFT in place (natural order): even/odd 16-point halves + w32^k
template <typename T, bool INV>
__device__ __forceinline__ void dft32(C<T>* v) {
  C<T> e[16], o[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    e[i] = v[2 * i];
    o[i] = v[2 * i + 1];
  }
  dft16<T, INV>(e);
  dft16<T, INV>(o);
  // cos(k pi / 16), sin(k pi / 16), k = 0..15
  const T cs[16] = {(T)1.0, (T)0.98078528040323044913, (T)0.92387953251128675613,
                    (T)0.83146961230254523708, (T)0.70710678118654752440, (T)0.55557023301960222474,
                    (T)0.38268343236508977173, (T)0.19509032201612826785, (T)0.0,
                    (T)-0.19509032201612826785, (T)-0.38268343236508977173, (T)-0.55557023301960222474,
                    (T)-0.70710678118654752440, (T)-0.83146961230254523708, (T)-0.92387953251128675613,
                    (T)-0.98078528040323044913};
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const T c = cs[k], sn = cs[k < 8 ? 8 - k : k - 8];  // sin(k pi/16) = cos((8-k) pi/16)
    const C<T> t = mulw<T, INV>(o[dft16_slot(k)], c, sn);
    const C<T> ev = e[dft16_slot(k)];
    v[k] = cadd<T>(ev, t);
    v[k + 16] = csub<T>(ev, t);
  }
}

// in-register DFT of size R with natural-order output
template <typename T, bool INV, int R>
__device__ __forceinline__ void dft_nat(C<T>* v) {
  if constexpr (R == 32) {
    dft32<T, INV>(v);
  } else if constexpr (R == 16) {
    C<T> u[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) u[i] = v[i];
    dft16<T, INV>(u);
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = u[dft16_slot(k)];
  } else if constexpr (R == 8) {
    dft8<T, INV>(v);
  } else if constexpr (R == 4) {
    dft4<T, INV>(v);
  } else {
    dft2<T, INV>(v);
  }
}

// Line access of the first read and the last write of a transform.  The
// default reads and writes the line in place; kernels pass their own to fuse
// a gather into the first read or a product / scatter into the last write.
// ld(l, line, n): input n of line l;  st(l, line, k, v): output k of line l.
template <typename T> struct LineId {
  __device__ __forceinline__ C<T> ld(int, const C<T>* line, int n) const { return line[pidx(n)]; }
  __device__ __forceinline__ void st(int, C<T>* line, int k, C<T> v) const { line[pidx(k)] = v; }
};

template <typename T, bool INV>
__device__ __forceinline__ C<T> twid(const C<T>* __restrict__ tw, int idx) {
  C<T> w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

// Barrier of the threads that transform one line (tpl consecutive threads,
// several lines per call): the warp when tpl <= 32, else a named barrier per
// group of tpl threads (ids 1..15; id 0 is __syncthreads), so the groups of a
// block do not wait for each other between passes.  Lines of different groups
// never share shared memory within a transform call, and every transform call
// ends with a block barrier.  The branch depends only on tpl and the block
// size, so all threads of a block take the same one.
__device__ __forceinline__ void line_group_sync(int tpl) {
  const int nthr = blockDim.x * blockDim.y;
  if (tpl <= 32) {
    __syncwarp();
  } else if (tpl >= nthr || (tpl & 31) != 0 || nthr % tpl != 0 || nthr / tpl > 15) {
    __syncthreads();
  } else {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    asm volatile("bar.sync %0, %1;" ::"r"(1 + tid / tpl), "r"(tpl) : "memory");
  }
}

// radix-R pass (R = 2^LR), PER butterflies per thread (PER * R = E, or 1 for n < E)
template <typename T, bool INV, int LR, int PER, bool FIRST = false, bool LAST = false,
          typename Op = LineId<T>>
__device__ __forceinline__ void fft_pass(C<T>* line, int n, int s, int t, int tpl,
                                         const C<T>* __restrict__ tw, int twlog, bool active,
                                         int lidx = 0, const Op& op = Op()) {
  constexpr int R = 1 << LR;
  const int Ns = 1 << s;
  const int nb = n >> LR;
  C<T> v[PER * R];
  if (active) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = t + q * tpl;
      const int k = j & (Ns - 1);
#pragma unroll
      for (int r = 0; r < R; ++r)
        v[q * R + r] = FIRST ? op.ld(lidx, line, j + r * nb) : line[pidx(j + r * nb)];
      if (s > 0) {
        const int shift = twlog - (s + LR);
        if constexpr (sizeof(T) == 4) {
          // FP32: one table twiddle w^k per butterfly, powers by multiplication
          const C<T> w1 = twid<T, INV>(tw, k << shift);
          C<T> wr = w1;
#pragma unroll
          for (int r = 1; r < R; ++r) {
            v[q * R + r] = cmul<T>(v[q * R + r], wr);
            if (r + 1 < R) wr = cmul<T>(wr, w1);
          }
        } else {
          // FP64: table lookups (loads are cheaper than FP64 multiplies)
#pragma unroll
          for (int r = 1; r < R; ++r)
            v[q * R + r] = cmul<T>(v[q * R + r], twid<T, INV>(tw, (k * r) << shift));
        }
      }
    }
  }
  line_group_sync(tpl);
  if (active) {
#pragma unroll
    for (int q = 0; q < PER; ++q) {
      const int j = t + q * tpl;
      const int k = j & (Ns - 1);
      C<T>* w = v + q * R;
      const int base = ((j - k) << LR) + k;
      if constexpr (LR == 4) {
        dft16<T, INV>(w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if constexpr (LAST) op.st(lidx, line, base + r * Ns, w[dft16_slot(r)]);
          else line[pidx(base + r * Ns)] = w[dft16_slot(r)];
        }
      } else {
        if constexpr (LR == 3) dft8<T, INV>(w);
        else if constexpr (LR == 2) dft4<T, INV>(w);
        else dft2<T, INV>(w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          if constexpr (LAST) op.st(lidx, line, base + r * Ns, w[r]);
          else line[pidx(base + r * Ns)] = w[r];
        }
      }
    }
  }
  line_group_sync(tpl);
}

// Core of the warp transform: lane l holds v[r] = x[l + LW r], r < RV, of a
// line of length n = LW * RV (RV = LW or 2 LW).
//   X1[k1] = DFT_RV over r;  X1[k1] *= w_n^{l k1};  transposed through the
//   tile (RV x (LW + 1) entries of shared memory);  lane l then owns
//   k1 = l + LW q and forms the LW-point DFT over the lanes.
// On return v[q LW + k2] = X[k1 + RV k2] with k1 = l + LW q.  The tile may
// overlap the line (all inputs are in registers); warp synchronisation only.
template <typename T, bool INV, int LW, int RV>
__device__ __forceinline__ void fft_warp_core(C<T>* v, C<T>* tile, int n, int logn, int l,
                                              bool active, const C<T>* __restrict__ tw,
                                              int twlog) {
  if (active) {
    dft_nat<T, INV, RV>(v);
    const int shift = twlog - logn;
    // w^{l k1} = w^{8 g l} w^{i l} for k1 = 8 g + i: 7 + RV/8 - 1 table reads
    // instead of RV - 1 (each product adds at most ~2 ulp)
    C<T> wi[8];
#pragma unroll
    for (int i = 1; i < 8 && i < RV; ++i) wi[i] = twid<T, INV>(tw, ((l * i) & (n - 1)) << shift);
#pragma unroll
    for (int i = 1; i < 8 && i < RV; ++i) v[i] = cmul<T>(v[i], wi[i]);
#pragma unroll
    for (int g = 1; g < RV / 8; ++g) {
      const C<T> wg = twid<T, INV>(tw, ((l * 8 * g) & (n - 1)) << shift);
      v[8 * g] = cmul<T>(v[8 * g], wg);
#pragma unroll
      for (int i = 1; i < 8; ++i) v[8 * g + i] = cmul<T>(v[8 * g + i], cmul<T>(wg, wi[i]));
    }
#pragma unroll
    for (int k1 = 0; k1 < RV; ++k1) tile[k1 * (LW + 1) + l] = v[k1];
  }
  __syncwarp();
  constexpr int Q = RV / LW;
  if (active) {
#pragma unroll
    for (int q = 0; q < Q; ++q)
#pragma unroll
      for (int ll = 0; ll < LW; ++ll) v[q * LW + ll] = tile[(l + LW * q) * (LW + 1) + ll];
  }
  __syncwarp();
  if (active) {
#pragma unroll
    for (int q = 0; q < Q; ++q) dft_nat<T, INV, LW>(v + q * LW);
  }
}

// Warp transform of one line of length n = LW * RV (RV = LW or 2 LW) by LW lanes
// (several lines per warp when LW < 32): the core above on the line's own
// shared memory, with op's first read and last write.
template <typename T, bool INV, int LW, int RV, typename Op = LineId<T>>
__device__ __forceinline__ void fft_warp(C<T>* line, int n, int logn, int l, bool active,
                                         const C<T>* __restrict__ tw, int twlog, int lidx = 0,
                                         const Op& op = Op()) {
  C<T> v[RV];
  if (active) {
#pragma unroll
    for (int r = 0; r < RV; ++r) v[r] = op.ld(lidx, line, l + LW * r);
  }
  __syncwarp();
  fft_warp_core<T, INV, LW, RV>(v, line, n, logn, l, active, tw, twlog);
  constexpr int Q = RV / LW;
  if (active) {
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int k1 = l + LW * q;
#pragma unroll
      for (int k2 = 0; k2 < LW; ++k2) op.st(lidx, line, k1 + RV * k2, v[q * LW + k2]);
    }
  }
  __syncwarp();
}

// Block transform of `nlines` lines of runtime length n = 2^logn (setup
// kernels only; the hot passes use the compile-time fft_lines below).
// Must be called by all threads of the CTA; ends with a CTA barrier.  Lines
// beyond what the CTA covers at once (blockDim / tpl) are done in groups.
template <typename T, bool INV>
__device__ void fft_inplace(C<T>* base, int lstride, int n, int logn, int nlines,
                            const C<T>* __restrict__ tw, int twlog) {
  constexpr int E = FftE<T>::E, LRMAX = FftE<T>::LRMAX;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int tpl = fft_tpl<T>(n);
  const int ept = n / tpl;               // points per thread: 8, or 16 at 4096
  const int lpg = nthr >= tpl ? nthr / tpl : 1;
  const int lg = tid / tpl, t = tid - lg * tpl;
  for (int l0 = 0; l0 < nlines; l0 += lpg) {
    const int l = l0 + lg;
    const bool active = lg < lpg && l < nlines;
    C<T>* line = base + (size_t)(active ? l : 0) * lstride;
    if (n < E) {
      switch (logn) {
        case 3: fft_pass<T, INV, 3, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
        case 2: fft_pass<T, INV, 2, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
        case 1: fft_pass<T, INV, 1, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
        default: break;
      }
      continue;
    }
    const int k = (logn + LRMAX - 1) / LRMAX;
    int s = 0;
    for (int p = 0; p < k; ++p) {
      const int lr = logn / k + (p < logn % k ? 1 : 0);
      if (ept == 16) {
        switch (lr) {
          case 3: fft_pass<T, INV, 3, 2>(line, n, s, t, tpl, tw, twlog, active); break;
          case 2: fft_pass<T, INV, 2, 4>(line, n, s, t, tpl, tw, twlog, active); break;
          default: fft_pass<T, INV, 1, 8>(line, n, s, t, tpl, tw, twlog, active); break;
        }
      } else {
        switch (lr) {
          case 3: fft_pass<T, INV, 3, 1>(line, n, s, t, tpl, tw, twlog, active); break;
          case 2: fft_pass<T, INV, 2, 2>(line, n, s, t, tpl, tw, twlog, active); break;
          default: fft_pass<T, INV, 1, 4>(line, n, s, t, tpl, tw, twlog, active); break;
        }
      }
      s += lr;
    }
  }
  __syncthreads();
}

// threads cooperating on one line of length 2^LOGN
template <typename T, int LOGN> struct LineShape {
  static constexpr bool WARP = sizeof(T) == 4 && LOGN >= 6 && LOGN <= 10;
  static constexpr int LW = 1 << (LOGN / 2);
  static constexpr int RV = (1 << LOGN) / LW;
  static constexpr int TPL =
      WARP ? LW : (LOGN >= 3 ? ((1 << LOGN) / 8 < FFT_MAX_TPL ? (1 << LOGN) / 8 : FFT_MAX_TPL) : 1);
};

// radix (log2) of pass P of the balanced schedule for a length 2^LOGN
template <int LOGN, int P> struct BlockRadix {
  static constexpr int K = (LOGN + 2) / 3;
  static constexpr int LR = LOGN / K + (P < LOGN % K ? 1 : 0);
  static constexpr int S = P == 0 ? 0 : BlockRadix<LOGN, (P > 0 ? P - 1 : 0)>::S + BlockRadix<LOGN, (P > 0 ? P - 1 : 0)>::LR;
};
template <int LOGN> struct BlockRadix<LOGN, 0> {
  static constexpr int K = (LOGN + 2) / 3;
  static constexpr int LR = LOGN / K + (0 < LOGN % K ? 1 : 0);
  static constexpr int S = 0;
};

template <typename T, bool INV, int LOGN, int P, typename Op>
__device__ __forceinline__ void block_passes(C<T>* line, int t, int tpl, const C<T>* __restrict__ tw,
                                             int twlog, bool active, int lidx, const Op& op) {
  constexpr int K = BlockRadix<LOGN, 0>::K;
  if constexpr (P < K) {
    constexpr int LR = BlockRadix<LOGN, P>::LR;
    constexpr int EPT = (1 << LOGN) / LineShape<T, LOGN>::TPL;   // 8, or 16 at 4096
    constexpr int PER = EPT >> LR;
    fft_pass<T, INV, LR, PER, P == 0, P == K - 1, Op>(line, 1 << LOGN, BlockRadix<LOGN, P>::S, t,
                                                      tpl, tw, twlog, active, lidx, op);
    block_passes<T, INV, LOGN, P + 1, Op>(line, t, tpl, tw, twlog, active, lidx, op);
  }
}


// In-place FFT of `nlines` padded lines (stride lstride) of the compile-time
// length 2^LOGN: the warp transform where it applies, else the block
// transform.  Called by all threads of the CTA; ends with a CTA barrier.
template <typename T, bool INV, int LOGN, typename Op = LineId<T>>
__device__ __forceinline__ void fft_lines(C<T>* base, int lstride, int nlines,
                                          const C<T>* __restrict__ tw, int twlog,
                                          const Op& op = Op()) {
  using S = LineShape<T, LOGN>;
  constexpr int n = 1 << LOGN, tpl = S::TPL;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  const int lpg = nthr >= tpl ? nthr / tpl : 1;
  const int lg = tid / tpl, t = tid - lg * tpl;
  for (int l0 = 0; l0 < nlines; l0 += lpg) {
    const int l = l0 + lg;
    const bool active = lg < lpg && l < nlines;
    C<T>* line = base + (size_t)(active ? l : 0) * lstride;
    if constexpr (S::WARP) {
      fft_warp<T, INV, S::LW, S::RV, Op>(line, n, LOGN, t, active, tw, twlog, l, op);
    } else if constexpr (LOGN <= 3) {
      if constexpr (LOGN >= 1)
        fft_pass<T, INV, LOGN, 1, true, true, Op>(line, n, 0, t, tpl, tw, twlog, active, l, op);
    } else {
      block_passes<T, INV, LOGN, 0, Op>(line, t, tpl, tw, twlog, active, l, op);
    }
  }
  __syncthreads();
}

// Warp-resident transform of the lines [first, first + cnt) that belong to the
// calling warp (FP32, LineShape<T, LOGN>::WARP): 32 / LW lines at a time, each
// on LW lanes.  Warp-level synchronisation only -- no block barrier, so the
// warps of a block can run their chains of transforms independently.
template <typename T, bool INV, int LOGN, typename Op = LineId<T>>
__device__ __forceinline__ void fft_warp_lines(C<T>* base, int lstride, int first, int cnt,
                                               const C<T>* __restrict__ tw, int twlog,
                                               const Op& op = Op()) {
  using S = LineShape<T, LOGN>;
  static_assert(S::WARP, "warp transform lengths only");
  constexpr int LW = S::LW, LPW = 32 / LW;
  const int lane = threadIdx.x & 31;
  const int sub = lane / LW, t = lane - sub * LW;
  for (int l0 = 0; l0 < cnt; l0 += LPW) {
    const int l = first + l0 + sub;
    const bool active = l0 + sub < cnt;
    C<T>* line = base + (size_t)(active ? l : first) * lstride;
    fft_warp<T, INV, LW, S::RV, Op>(line, 1 << LOGN, LOGN, t, active, tw, twlog, l, op);
  }
}

// Named barrier of the two warps of a two-warp transform (ids 1..15; 0 is
// __syncthreads).
__device__ __forceinline__ void pair_sync(int id) {
  asm volatile("bar.sync %0, 64;" ::"r"(id) : "memory");
}

// Two-warp transform of one FP32 line of length n = 2^LOGN (2048): one radix-2
// step (decimation in frequency) and a warp transform of length n/2 per warp.
// Warp h (0 or 1) forms u_h[i] = x[i] + x[i + n/2] (h = 0) or
// (x[i] - x[i + n/2]) w_n^i (h = 1) and transforms it: X[2k + h] = DFT_{n/2}(u_h)[k].
// Both warps read the whole line (op.ld) before either writes; their tiles
// lie in disjoint halves of the line (the line's padded length is at least
// n + n/8); both finish reading their tiles before either stores (op.st with
// the output index 2k + h).  bar_id: a named barrier owned by the two warps.
template <typename T, bool INV, int LOGN, typename Op = LineId<T>>
__device__ __forceinline__ void fft_warp2(C<T>* line, int h, int l, const C<T>* __restrict__ tw,
                                          int twlog, int bar_id, int lidx = 0,
                                          const Op& op = Op()) {
  constexpr int n = 1 << LOGN, nh = n / 2;
  using S = LineShape<T, LOGN - 1>;
  static_assert(S::WARP && S::LW == 32, "two-warp transform of 2 x 1024 points");
  constexpr int LW = S::LW, RV = S::RV;
  C<T> v[RV];
  const int shift = twlog - LOGN;
#pragma unroll
  for (int r = 0; r < RV; ++r) {
    const int i = l + LW * r;
    const C<T> a = op.ld(lidx, line, i), b = op.ld(lidx, line, i + nh);
    v[r] = h == 0 ? cadd<T>(a, b) : cmul<T>(csub<T>(a, b), twid<T, INV>(tw, i << shift));
  }
  pair_sync(bar_id);
  constexpr int TILE = RV * (LW + 1);
  static_assert(TILE <= nh + nh / 8, "tiles fit in the two halves of the padded line");
  fft_warp_core<T, INV, LW, RV>(v, line + h * (nh + nh / 8), nh, LOGN - 1, l, true, tw, twlog);
  pair_sync(bar_id);
  constexpr int Q = RV / LW;
#pragma unroll
  for (int q = 0; q < Q; ++q) {
    const int k1 = l + LW * q;
#pragma unroll
    for (int k2 = 0; k2 < LW; ++k2) op.st(lidx, line, 2 * (k1 + RV * k2) + h, v[q * LW + k2]);
  }
  __syncwarp();
}
