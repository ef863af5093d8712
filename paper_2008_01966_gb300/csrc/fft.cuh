// Shared-memory FFTs of power-of-two length for the cavity solver.
//
// All transforms of the hot path -- the Fourier-series synthesis (E123F), the
// trapezoid projections and the torus convolution of Sec. 5.2 -- are batches
// of 1-D transforms of lines held in shared memory.
//
// Algorithm: Stockham auto-sort in at most three passes for n <= 4096: each
// thread owns 16 consecutive "slots" of a line and, per pass, one radix-16
// butterfly (or two radix-8, four radix-4, eight radix-2), whose inputs are
// read from shared memory into registers, twiddled, transformed in registers
// and written back in place after a barrier.  Lines use a padded layout
// (one pad word per 16 elements, see pidx) so that the strided writes of the
// first pass do not collide in the shared-memory banks.  Twiddles come from a
// table tw[k] = exp(-2 pi i k / TW) computed once in FP64 (rounded for the
// FP32 table): in FP32 a butterfly reads w^k and forms its powers by
// multiplication (at most 7 products, ~5e-7 relative); in FP64 it reads every
// power from the table.  Forward = exp(-...), inverse = exp(+...),
// unnormalised.
//
// Contract: a CTA transforms `nlines` lines of length n = 2^logn stored at
// line_base + l * lstride (padded indices).  Threads 0 .. nlines*tpl-1 do the
// work, tpl = max(1, n/16); all threads of the CTA must call (barriers).
#pragma once
#include "common.cuh"

__host__ __device__ __forceinline__ int pidx(int i) { return i + (i >> 4); }
__host__ __device__ __forceinline__ int padded_len(int n) { return n + (n >> 4) + 1; }
// elements per thread: 16 (radix up to 16) in FP32, 8 (radix up to 8) in FP64,
// which keeps a butterfly's operands in registers without spilling
template <typename T> struct FftE { static constexpr int E = 8, LRMAX = 3; };
template <> struct FftE<double> { static constexpr int E = 8, LRMAX = 3; };
template <typename T> __host__ __device__ __forceinline__ int fft_tpl(int n) {
  return n >= FftE<T>::E ? n / FftE<T>::E : 1;
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

template <typename T, bool INV>
__device__ __forceinline__ C<T> twid(const C<T>* __restrict__ tw, int idx) {
  C<T> w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

// radix-R pass (R = 2^LR), PER butterflies per thread (PER * R = E, or 1 for n < E)
template <typename T, bool INV, int LR, int PER>
__device__ __forceinline__ void fft_pass(C<T>* line, int n, int s, int t, int tpl,
                                         const C<T>* __restrict__ tw, int twlog, bool active) {
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
      for (int r = 0; r < R; ++r) v[q * R + r] = line[pidx(j + r * nb)];
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
  __syncthreads();
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
        for (int r = 0; r < R; ++r) line[pidx(base + r * Ns)] = w[dft16_slot(r)];
      } else {
        if constexpr (LR == 3) dft8<T, INV>(w);
        else if constexpr (LR == 2) dft4<T, INV>(w);
        else dft2<T, INV>(w);
#pragma unroll
        for (int r = 0; r < R; ++r) line[pidx(base + r * Ns)] = w[r];
      }
    }
  }
  __syncthreads();
}

// In-place FFT of `nlines` padded lines (stride lstride) of length n = 2^logn.
template <typename T, bool INV>
__device__ void fft_inplace(C<T>* base, int lstride, int n, int logn, int nlines,
                            const C<T>* __restrict__ tw, int twlog) {
  constexpr int E = FftE<T>::E, LRMAX = FftE<T>::LRMAX;
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int tpl = fft_tpl<T>(n);
  const int l = tid / tpl, t = tid - l * tpl;
  const bool active = l < nlines;
  C<T>* line = base + (size_t)(active ? l : 0) * lstride;
  if (n < E) {
    // one pass of radix n
    switch (logn) {
      case 3: fft_pass<T, INV, 3, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
      case 2: fft_pass<T, INV, 2, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
      case 1: fft_pass<T, INV, 1, 1>(line, n, 0, t, tpl, tw, twlog, active); break;
      default: break;
    }
    return;
  }
  // pass schedule: ceil(logn / LRMAX) passes with balanced radices
  const int k = (logn + LRMAX - 1) / LRMAX;
  int s = 0;
  for (int p = 0; p < k; ++p) {
    const int lr = logn / k + (p < logn % k ? 1 : 0);
    if constexpr (E == 16) {
      switch (lr) {
        case 4: fft_pass<T, INV, 4, 1>(line, n, s, t, tpl, tw, twlog, active); break;
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
