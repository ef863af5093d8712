// The aperture operator of (EJ1)/(uT1): the cavity (local) part and the TBC
// part whose singular integrals follow Sec. 5 (discrete rule: periodised FFT
// convolution with the exact transform of the truncated basis, the kernel
// table F(G), inverse transform on the torus grid, trapezoid outer rule).
//
// For each right-hand side the TBC needs three convolution-projections,
//   U1 = <cs_mn, G*u1>,  U2 = <sc_mn, G*u2>,  W = <cc_mn, G*w>,
// u1 = sum E1 cs, u2 = sum E2 sc, w = div_Gamma(z x E) = sum (k2 pi/b) E1 cc -
// sum (k1 pi/a) E2 cc (Sec. 5.1 reduces every coefficient to I1, I2, I3).
// Each one is four passes of batched line transforms in shared memory:
//   A  (rows k1)   basis transform along x2: FFT convolution of the mirrored
//                  coefficients with the 1-D kernel E(nu) of F(F)
//   B  (cols j2)   basis transform along x1, times F(G)/(Lx Ly), inverse DFT
//                  along x1 evaluated at the nodes p = 0..Nx
//   C  (rows p)    inverse DFT along x2 at q = 0..Ny, trapezoid projection
//                  onto cos/sin(n pi q/Ny) (an extended FFT of length 2Ny)
//   D  (cols n)    trapezoid projection along x1 (extended FFT of length 2Nx)
// and a final elementwise pass adds the local part of (EJ1)/(uT1).
// Templated on the arithmetic type: FP64 for the FP64 path and the residuals,
// FP32 for the inner Krylov iterations of the mixed path.  Every pass kernel
// is instantiated per grid size so that its line transforms have compile-time
// lengths; tbc.cu instantiates the FP64 operator, tbc_f32.cu the FP32 one.
#pragma once
#include <algorithm>
#include <atomic>
#include <type_traits>

#include "common.cuh"
#include "fft.cuh"

struct TbcP {
  int nx, ny, M, N, Px, Py, lPx, lPy, lnx, lny, nap, n1, n2;
  double a, b, h, k2x2;  // k2x2 = 2 kappa0^2
  double pia, pib, ab;   // pi / a, pi / b, a b
  double wy, wx;         // trapezoid weights / 2: b / (2 ny), a / (2 nx)
  int twlog;
};

static TbcP make_params(const cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  TbcP p;
  p.nx = g.nx; p.ny = g.ny; p.M = g.M; p.N = g.N; p.Px = g.Px; p.Py = g.Py;
  p.lPx = g.lPx; p.lPy = g.lPy; p.lnx = g.lnx; p.lny = g.lny;
  p.nap = g.nap; p.n1 = g.n1; p.n2 = g.n2;
  p.a = g.a; p.b = g.b; p.h = g.h; p.k2x2 = 2.0 * ctx->kappa0 * ctx->kappa0;
  p.pia = M_PI / g.a; p.pib = M_PI / g.b; p.ab = g.a * g.b;
  p.wy = 0.5 * g.b / g.ny; p.wx = 0.5 * g.a / g.nx;
  p.twlog = ilog2(ctx->TW);
  return p;
}

template <typename T> __device__ __forceinline__ C<T> czero() { return mk<T>(0, 0); }

// Lines per CTA: enough lines that a pass of the longest transform in the
// kernel occupies LINES_THREADS threads (nlong = that length).
#define LINES_THREADS 256
template <typename T> __host__ __device__ constexpr int lines_per_cta(int nlong) {
  return fft_tpl<T>(nlong) >= LINES_THREADS ? 1 : LINES_THREADS / fft_tpl<T>(nlong);
}
// passes A and B hold two lines (parities r = 0, 1) per row / column
template <typename T> __host__ __device__ constexpr int pairs_per_cta(int n) {
  return 2 * fft_tpl<T>(n) >= LINES_THREADS ? 1 : LINES_THREADS / (2 * fft_tpl<T>(n));
}
// registers: the pass kernels run two CTAs of LINES_THREADS per SM (the
// pair-of-FP32 ones spill ~450 bytes per thread at this bound, but one CTA per
// SM without spills was slower: pass B 10.6 ms against 7.6 ms)
#define TBC_BOUNDS __launch_bounds__(LINES_THREADS, 2)
// the same per grid size: with 4096-point lines (1024-point sides) a CTA's
// lines take most of the shared memory, so one CTA per SM, with the whole
// register file for the 16 points per thread of the block transform
#define TBC_BOUNDS_LN(LN) __launch_bounds__(LINES_THREADS, (LN) >= 10 ? 1 : 2)

// The pass kernels are instantiated per grid size: LNY = log2 ny (passes A,
// C), LNX = log2 nx (passes B, D).  With the period pad = 4: Px = 4 nx,
// Py = 4 ny.

// ------------------------------------------------------------------ pass A
// grid (ceil(nx / L) row groups, 3 fields, ndir); field 0: cs (E1), 1: sc (E2),
// 2: cc (w).  Per row k1: the mirrored coefficient sequence along x2 (period
// Py) is transformed, multiplied by the transforms of the two parity kernels
// eps_r and transformed back: the linear convolutions give the basis
// transform at j2 = 2t + r of the symmetric box.  Lines: [parity][row].
// The gather of the coefficients is the forward transform's first read, the
// kernel products its last write, and the scatter to Vy the inverse
// transforms' last write: shared memory holds only the transforms.

// coefficient k2 (0 <= k2 < ny) of row k1 for field f, mirrored to the input
// n of a line of length Py
template <typename T, int LNY>
struct GatherA {
  const C<T>* E1;
  const C<T>* E2;
  int row0, nx, f;
  T pib, pia;                     // pi / b, pi / a
  __device__ __forceinline__ C<T> coef(int k1, int k2) const {
    constexpr int ny = 1 << LNY, N = ny - 1;
    C<T> c = czero<T>();
    if (f == 0) {
      if (k2 >= 1) c = E1[k1 * N + (k2 - 1)];
    } else if (f == 1) {
      if (k1 >= 1) c = E2[(k1 - 1) * ny + k2];
    } else {
      if (k2 >= 1) c = cscale<T>(E1[k1 * N + (k2 - 1)], (T)k2 * pib);
      if (k1 >= 1) c = csub<T>(c, cscale<T>(E2[(k1 - 1) * ny + k2], (T)k1 * pia));
    }
    return c;
  }
  __device__ __forceinline__ C<T> ld(int l, const C<T>*, int n) const {
    constexpr int ny = 1 << LNY, Py = 4 * ny;
    const int k1 = row0 + l;
    if (k1 >= nx) return czero<T>();
    const bool ycos = f != 0;
    if (n < ny) {
      if (n == 0) return ycos ? cscale<T>(coef(k1, 0), (T)2) : czero<T>();
      return coef(k1, n);
    }
    if (n > Py - ny) {
      const C<T> c = coef(k1, Py - n);
      return ycos ? c : mk<T>(-c.x, -c.y);
    }
    return czero<T>();
  }
};

// last write of the forward transform: the products with the two parity
// kernels, into line l (r = 0) and line L + l (r = 1)
template <typename T, typename G>
struct ParityProducts : G {
  const C<T>* eh;                 // [r][P]
  int P, L, ls;
  C<T>* buf;
  __device__ __forceinline__ void st(int l, C<T>*, int k, C<T> v) const {
    buf[(size_t)l * ls + pidx(k)] = cmul<T>(v, eh[k]);
    buf[(size_t)(L + l) * ls + pidx(k)] = cmul<T>(v, eh[P + k]);
  }
};

// last write of the forward transform when each parity line transforms its
// own copy of the column: the product with its parity's kernel, in place
template <typename T>
struct OwnParity : LineId<T> {
  const C<T>* eh;                 // [r][P]
  int P, L;
  __device__ __forceinline__ void st(int l, C<T>* line, int k, C<T> v) const {
    const int r = l >= L ? 1 : 0;
    line[pidx(k)] = cmul<T>(v, eh[r * P + k]);
  }
};

// pass A with one copy of the row per parity line: gather of row (l mod L),
// product with the kernel of parity (l >= L), in place
template <typename T, int LNY>
struct GatherOwnA : GatherA<T, LNY> {
  const C<T>* eh;                 // [r][P]
  int P, L;
  __device__ __forceinline__ C<T> ld(int l, const C<T>* line, int n) const {
    return GatherA<T, LNY>::ld(l >= L ? l - L : l, line, n);
  }
  __device__ __forceinline__ void st(int l, C<T>* line, int k, C<T> v) const {
    const int r = l >= L ? 1 : 0;
    line[pidx(k)] = cmul<T>(v, eh[r * P + k]);
  }
};

// last write of the inverse transforms of pass A: Vy(k1, j), j = 2t + r mod Py
template <typename T, int LNY>
struct ScatterA : LineId<T> {
  C<T>* Vy;                       // this field's [nx][Py] block
  int row0, nx, L;
  __device__ __forceinline__ void st(int lr, C<T>*, int k, C<T> v) const {
    constexpr int Py = 4 << LNY;
    const int r = lr >= L ? 1 : 0, l = lr - r * L;
    const int k1 = row0 + l;
    const int t = k < Py / 2 ? k : k - Py;
    if (k1 >= nx || t < -Py / 4 || t >= Py / 4) return;
    const int j2 = 2 * t + r;
    Vy[(size_t)k1 * Py + (j2 & (Py - 1))] = (j2 == -Py / 2) ? czero<T>() : v;
  }
};

template <typename T, int LNY>
__global__ void TBC_BOUNDS_LN(LNY) k_tbcA(const C<T>* __restrict__ x, C<T>* __restrict__ Vy, TbcP p,
                                  const C<T>* __restrict__ tw, const C<T>* __restrict__ eh_c,
                                  const C<T>* __restrict__ eh_s) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int LPY = LNY + 2, Py = 1 << LPY, ls = padded_len(Py);
  constexpr int L = pairs_per_cta<T>(Py);
  const int f = blockIdx.y, d = blockIdx.z;
  const int row0 = blockIdx.x * L;
  ScatterA<T, LNY> sc;
  sc.Vy = Vy + (size_t)(d * 3 + f) * p.nx * Py;
  sc.row0 = row0;
  sc.nx = p.nx;
  sc.L = L;
  if constexpr (LineShape<T, LPY>::WARP && 2 * L * LineShape<T, LPY>::TPL == LINES_THREADS) {
    // every warp transforms its own lines (parity 0 or 1 of a row) from the
    // gather to the scatter, the row's forward transform done by both of its
    // lines' warps: no idle warps and no block barrier
    GatherOwnA<T, LNY> fwd;
    fwd.E1 = x + (size_t)d * p.nap;
    fwd.E2 = fwd.E1 + p.n1;
    fwd.row0 = row0;
    fwd.nx = p.nx;
    fwd.f = f;
    fwd.pib = (T)p.pib;
    fwd.pia = (T)p.pia;
    fwd.eh = f != 0 ? eh_c : eh_s;
    fwd.P = Py;
    fwd.L = L;
    constexpr int LPW = 32 / LineShape<T, LPY>::TPL;
    const int first = (threadIdx.x >> 5) * LPW;
    fft_warp_lines<T, false, LPY>(buf, ls, first, LPW, tw, p.twlog, fwd);
    fft_warp_lines<T, true, LPY>(buf, ls, first, LPW, tw, p.twlog, sc);
  } else {
    ParityProducts<T, GatherA<T, LNY>> fwd;
    fwd.E1 = x + (size_t)d * p.nap;
    fwd.E2 = fwd.E1 + p.n1;
    fwd.row0 = row0;
    fwd.nx = p.nx;
    fwd.f = f;
    fwd.pib = (T)p.pib;
    fwd.pia = (T)p.pia;
    fwd.eh = f != 0 ? eh_c : eh_s;
    fwd.P = Py;
    fwd.L = L;
    fwd.ls = ls;
    fwd.buf = buf;
    fft_lines<T, false, LPY>(buf, ls, L, tw, p.twlog, fwd);
    fft_lines<T, true, LPY>(buf, ls, 2 * L, tw, p.twlog, sc);
  }
}

// ------------------------------------------------------------------ pass B
// grid (Py / L column groups, 3 fields, ndir).  Per column j2: the basis
// transform along x1 split by the parity of j1 = 2t + r (as in pass A), times
// F(G)(|j1|, |j2|)/(Lx Ly), then the inverse torus transform along x1 at the
// nodes p = 0..nx:  sum_j1 Y(j1) e^{2 pi i j1 p/Px} = Z_0(p) + e^{2 pi i p/Px} Z_1(p),
// Z_r = inverse transform of length Px/2 of Y(2t + r) over t.
// Fused: the parity products (last write of the forward transform), the
// kernel-table products with the move of t to slot t mod Px/2 (last write of
// the first inverse transforms).  The column gather stays a cooperative pass:
// as a per-line first read it would load one element per 32-byte sector.

// last write of the first inverse transforms of pass B: output t (k = t mod
// Px) of line (r, l), |t| < Px/4, times the kernel table at (|2t + r|, |j2|),
// written to slot t mod Px/2 (other outputs are not needed)
// STAGED: kh holds the rows of the block's columns in shared memory,
// [l][j1 < Px/2]; else kh is the whole quarter box in global memory, [j2][j1]
template <typename T, int LNX, bool STAGED = true>
struct KhatB : LineId<T> {
  const C<T>* kh;
  int j0, Py, L;
  __device__ __forceinline__ void st(int lr, C<T>* line, int k, C<T> v) const {
    constexpr int Px = 4 << LNX, hp = Px / 2, qp = Px / 4;
    int t, u;
    if (k < qp) { t = k; u = k; }
    else if (k >= Px - qp) { t = k - Px; u = k - hp; }
    else return;
    const int r = lr >= L ? 1 : 0, l = lr - r * L;
    const int j = j0 + l;
    const int j1 = 2 * t + r;
    C<T> o = czero<T>();
    if (j1 != -hp && j < Py && j != Py / 2) {
      const int j1a = j1 < 0 ? -j1 : j1;
      if constexpr (STAGED) {
        o = cmul<T>(v, kh[l * hp + j1a]);
      } else {
        const int j2a = j < Py / 2 ? j : Py - j;
        o = cmul<T>(v, kh[(size_t)j2a * hp + j1a]);
      }
    }
    line[pidx(u)] = o;
  }
};

// pass B stages the two parity kernels and the kernel-table rows of its
// columns in shared memory when lines and tables together take at most
// 100 KB (every FP32 grid; 16-byte types up to 256 points per side); else it
// reads them from global memory (they stay in L2), which leaves room for more
// CTAs per SM: at 512 points per side the pair-of-FP32 pass B of the
// four-layer 512^2 benchmark step went from 16.2 to 9.4 ms (one CTA per SM
// with the 156 KB of staging, two without), and it is the only way at 1024
template <typename T> __host__ __device__ constexpr size_t smem_b_lines(int nx) {
  return sizeof(C<T>) * 2 * (size_t)pairs_per_cta<T>(4 * nx) * (size_t)padded_len(4 * nx);
}
template <typename T> __host__ __device__ constexpr size_t smem_b_tables(int nx) {
  return sizeof(C<T>) * (2 * 4 * (size_t)nx + (size_t)pairs_per_cta<T>(4 * nx) * 2 * (size_t)nx);
}
template <typename T> __host__ __device__ constexpr bool b_staged(int nx) {
  return smem_b_lines<T>(nx) + smem_b_tables<T>(nx) <= 100 * 1024;
}

template <typename T, int LNX>
__global__ void TBC_BOUNDS_LN(LNX) k_tbcB(const C<T>* __restrict__ Vy, C<T>* __restrict__ W, TbcP p,
                                  const C<T>* __restrict__ tw, const C<T>* __restrict__ eh_c,
                                  const C<T>* __restrict__ eh_s, const C<T>* __restrict__ kh) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int LPX = LNX + 2, Px = 1 << LPX, nx = 1 << LNX, ls = padded_len(Px);
  constexpr int L = pairs_per_cta<T>(Px), lL = clog2(L);
  const int Py = p.Py;
  const int f = blockIdx.y, d = blockIdx.z;
  const int j0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xcos = (f != 1);
  // the per-warp chain (below) needs the column in both of its lines
  constexpr int NCOPY = (LineShape<T, LPX>::WARP && LineShape<T, LPX - 1>::WARP &&
                         2 * L * LineShape<T, LPX>::TPL == LINES_THREADS) ? 2 : 1;
  // shared memory: 2L lines, then the two parity kernels [2][Px], then the
  // kernel-table rows |j2| of the L columns [L][Px/2] (staged once per block,
  // so the fused products read shared memory instead of waiting on loads)
  constexpr bool STAGE = b_staged<T>(nx);
  C<T>* eh_sm = buf + (size_t)2 * L * ls;
  C<T>* kh_sm = eh_sm + 2 * Px;
  const C<T>* eh_use = xcos ? eh_c : eh_s;
  if constexpr (STAGE) {
    const C<T>* eh = xcos ? eh_c : eh_s;
    for (int t = tid; t < 2 * Px; t += nthr) eh_sm[t] = eh[t];
    for (int idx = tid; idx < L * (Px / 2); idx += nthr) {
      const int l = idx >> (LPX - 1), j1 = idx & (Px / 2 - 1);
      const int j = j0 + l;
      const int j2a = j < Py / 2 ? j : Py - j;
      kh_sm[idx] = (j < Py && j != Py / 2) ? kh[(size_t)j2a * (Px / 2) + j1] : czero<T>();
    }
    eh_use = eh_sm;
  }
  // cooperative, coalesced gather of the L columns (consecutive threads take
  // consecutive columns of a row); the mirrored lines cover every slot but
  // [nx, Px - nx], which is cleared
  {
    const C<T>* src = Vy + (size_t)(d * 3 + f) * nx * Py;
#pragma unroll 4
    for (int idx = tid; idx < L * nx; idx += nthr) {
      const int k1 = idx >> lL, l = idx & (L - 1);
      const int j = j0 + l;
      const C<T> c = j < Py ? src[(size_t)k1 * Py + j] : czero<T>();
      const C<T> c0 = k1 == 0 ? (xcos ? cscale<T>(c, (T)2) : czero<T>()) : c;
      const C<T> cm = xcos ? c : mk<T>(-c.x, -c.y);
#pragma unroll
      for (int r = 0; r < NCOPY; ++r) {
        C<T>* line = buf + (size_t)(r * L + l) * ls;
        line[pidx(k1)] = c0;
        if (k1 > 0) line[pidx(Px - k1)] = cm;
      }
    }
    for (int idx = tid; idx < NCOPY * L * (2 * nx + 1); idx += nthr) {
      const int l = idx / (2 * nx + 1), k = nx + idx - l * (2 * nx + 1);
      buf[(size_t)l * ls + pidx(k)] = czero<T>();
    }
    __syncthreads();
  }
  KhatB<T, LNX, STAGE> kb;
  kb.kh = STAGE ? kh_sm : kh;
  kb.j0 = j0;
  kb.Py = Py;
  kb.L = L;
  if constexpr (LineShape<T, LPX>::WARP && LineShape<T, LPX - 1>::WARP &&
                2 * L * LineShape<T, LPX>::TPL == LINES_THREADS) {
    // every warp runs the whole chain on its own lines (a parity-0 or a
    // parity-1 line of a column): the forward transform of the column is done
    // by both of its lines' warps, so no warp idles and no block barrier is
    // needed until the two parities are combined
    constexpr int LPW = 32 / LineShape<T, LPX>::TPL;
    const int first = (tid >> 5) * LPW;
    OwnParity<T> fwd;
    fwd.eh = eh_use;
    fwd.P = Px;
    fwd.L = L;
    fft_warp_lines<T, false, LPX>(buf, ls, first, LPW, tw, p.twlog, fwd);
    fft_warp_lines<T, true, LPX>(buf, ls, first, LPW, tw, p.twlog, kb);
    fft_warp_lines<T, true, LPX - 1>(buf, ls, first, LPW, tw, p.twlog);
    __syncthreads();
  } else {
    ParityProducts<T, LineId<T>> fwd;
    fwd.eh = eh_use;
    fwd.P = Px;
    fwd.L = L;
    fwd.ls = ls;
    fwd.buf = buf;
    fft_lines<T, false, LPX>(buf, ls, L, tw, p.twlog, fwd);
    fft_lines<T, true, LPX>(buf, ls, 2 * L, tw, p.twlog, kb);
    fft_lines<T, true, LPX - 1>(buf, ls, 2 * L, tw, p.twlog);
  }
  C<T>* dst = W + (size_t)(d * 3 + f) * (nx + 1) * Py;
  const int sh = p.twlog - LPX;
  for (int idx = tid; idx < L * (nx + 1); idx += nthr) {
    const int q = idx >> lL, l = idx & (L - 1);
    const int j = j0 + l;
    if (j >= Py) continue;
    const C<T> z0 = buf[(size_t)l * ls + pidx(q)];
    const C<T> z1 = buf[(size_t)(L + l) * ls + pidx(q)];
    dst[(size_t)q * Py + j] = cadd<T>(z0, cmul<T>(z1, twid<T, true>(tw, q << sh)));
  }
}

// ------------------------------------------------------------------ pass C
// grid (ceil((nx+1)/L) row groups, 3 fields, ndir).  Per node row p: inverse
// torus transform along x2 at q = 0..ny, then the trapezoid projection onto
// cos/sin(n pi q/ny) as an extended FFT of length 2 ny.  Fused: the row load
// (first read), the even / odd extension of U(q), q <= ny (last write of the
// inverse transform), the weighted store of Z (last write of the projection).

template <typename T, int LNY>
struct RowC {
  const C<T>* src;                // this field's [nx+1][Py] block
  int r0, nx;
  bool ycos;
  __device__ __forceinline__ C<T> ld(int l, const C<T>*, int n) const {
    constexpr int Py = 4 << LNY;
    const int row = r0 + l;
    return row <= nx ? src[(size_t)row * Py + n] : czero<T>();
  }
  __device__ __forceinline__ void st(int, C<T>* line, int k, C<T> v) const {
    constexpr int ny = 1 << LNY, n2 = 2 * ny;
    if (k > ny) return;
    if (!ycos && (k == 0 || k == ny)) {
      line[pidx(k)] = czero<T>();
      return;
    }
    line[pidx(k)] = v;
    if (k > 0 && k < ny) line[pidx(n2 - k)] = ycos ? v : mk<T>(-v.x, -v.y);
  }
};

template <typename T, int LNY>
struct StoreZ : LineId<T> {
  C<T>* Z;                        // this field's [nx+1][ny+1] block
  int r0, nx;
  bool ycos;
  T w;
  __device__ __forceinline__ void st(int l, C<T>*, int k, C<T> v) const {
    constexpr int ny = 1 << LNY;
    const int row = r0 + l;
    if (k > ny || row > nx) return;
    Z[(size_t)row * (ny + 1) + k] = ycos ? cscale<T>(v, w) : cscale<T>(cmul_i<T>(v), w);
  }
};

template <typename T, int LNY>
__global__ void TBC_BOUNDS_LN(LNY) k_tbcC(const C<T>* __restrict__ W, C<T>* __restrict__ Z, TbcP p,
                                  const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int LPY = LNY + 2, Py = 1 << LPY, ny = 1 << LNY, ls = padded_len(Py);
  constexpr int L = lines_per_cta<T>(Py);
  const int f = blockIdx.y, d = blockIdx.z;
  const int r0 = blockIdx.x * L;
  const bool ycos = (f != 0);
  RowC<T, LNY> rc;
  rc.src = W + (size_t)(d * 3 + f) * (p.nx + 1) * Py;
  rc.r0 = r0;
  rc.nx = p.nx;
  rc.ycos = ycos;
  fft_lines<T, true, LPY>(buf, ls, L, tw, p.twlog, rc);
  StoreZ<T, LNY> sz;
  sz.Z = Z + (size_t)(d * 3 + f) * (p.nx + 1) * (ny + 1);
  sz.r0 = r0;
  sz.nx = p.nx;
  sz.ycos = ycos;
  sz.w = (T)p.wy;
  fft_lines<T, false, LNY + 1>(buf, ls, L, tw, p.twlog, sz);
}

// ------------------------------------------------------------------ pass D
// grid (ceil((ny+1)/L) column groups, 3 fields, ndir).  Per column n: the
// trapezoid projection along x1 (extended FFT of length 2 nx), with the
// column gather and extension as the first read and the weighted store of O
// as the last write.
template <typename T, int LNX>
struct ColD {
  const C<T>* src;                // this field's [nx+1][ny+1] block
  C<T>* dst;                      // this field's [nx][ny+1] block
  int c0, ny;
  bool xcos;
  T w;
  __device__ __forceinline__ C<T> ld(int l, const C<T>*, int t) const {
    constexpr int nx = 1 << LNX, n2 = 2 * nx;
    const int col = c0 + l;
    if (col > ny) return czero<T>();
    if (t <= nx) {
      if (!xcos && (t == 0 || t == nx)) return czero<T>();
      return src[(size_t)t * (ny + 1) + col];
    }
    const C<T> r = src[(size_t)(n2 - t) * (ny + 1) + col];
    return xcos ? r : mk<T>(-r.x, -r.y);
  }
  __device__ __forceinline__ void st(int l, C<T>*, int m, C<T> v) const {
    constexpr int nx = 1 << LNX;
    const int col = c0 + l;
    if (m >= nx || col > ny) return;
    dst[(size_t)m * (ny + 1) + col] = xcos ? cscale<T>(v, w) : cscale<T>(cmul_i<T>(v), w);
  }
};

template <typename T, int LNX>
__global__ void TBC_BOUNDS_LN(LNX) k_tbcD(const C<T>* __restrict__ Z, C<T>* __restrict__ O, TbcP p,
                                  const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int nx = 1 << LNX, n2 = 2 * nx, ls = padded_len(n2);
  constexpr int L = lines_per_cta<T>(n2);
  const int f = blockIdx.y, d = blockIdx.z;
  ColD<T, LNX> cd;
  cd.src = Z + (size_t)(d * 3 + f) * (nx + 1) * (p.ny + 1);
  cd.dst = O + (size_t)(d * 3 + f) * nx * (p.ny + 1);
  cd.c0 = blockIdx.x * L;
  cd.ny = p.ny;
  cd.xcos = (f != 1);
  cd.w = (T)p.wx;
  fft_lines<T, false, LNX + 1>(buf, ls, L, tw, p.twlog, cd);
}

// ------------------------------------------------------------------ passes B, C at 2048 points
// FP32 lines of 2048 points (the 512 x 512 grid: Px = Py = 2048) do not fit
// one warp's registers; each line is transformed by two warps (fft_warp2:
// one radix-2 step, then a 1024-point warp transform per warp), so these
// passes keep the warp transforms of the smaller grids -- no block barrier
// inside a transform, one shared-memory round trip per 1024-point half.
// Pass B: two columns per block of eight warps, each parity line on a warp
// pair; pass C: four rows per block, each on a warp pair; the named barrier
// of pair g is 1 + g.  (Pass A keeps the block transform at this size: a
// two-warp version measured 0.46 against 0.29 ms per 8-direction launch.)
template <int N2> struct W2 {
  static constexpr int LS = padded_len(N2);
  static constexpr int L = 2;           // rows / columns per block
};

// pass B: grid (Py / 2 column pairs, 3 fields, ndir).  The parity kernels
// are read from global memory (32 KB, L1 resident); shared memory holds the
// four lines and the kernel-table rows of the two columns.
template <typename T>
struct OwnParityG : LineId<T> {
  const C<T>* __restrict__ eh;    // [r][P], global
  int P, L;
  __device__ __forceinline__ void st(int l, C<T>* line, int k, C<T> v) const {
    const int r = l >= L ? 1 : 0;
    line[pidx(k)] = cmul<T>(v, __ldg(eh + r * P + k));
  }
};

// KhatB for the two-warp pass: the lanes of a warp write outputs 2 apart, so
// they read the kernel table 4 apart in j1; the rows are staged with
// j1 -> (j1 mod 4) (Px/8 + 4) + j1 / 4 (row length KH_ROW), which makes
// those reads consecutive and the staging writes free of bank conflicts
template <int LNX>
struct KhatBPerm : LineId<float> {
  static constexpr int KH_ROW = 4 * ((4 << LNX) / 8 + 4);
  const float2* kh;               // rows |j2| of the block's columns, permuted
  int j0, Py, L;
  __device__ __forceinline__ static int perm(int j1) {
    constexpr int Px = 4 << LNX;
    return (j1 & 3) * (Px / 8 + 4) + (j1 >> 2);
  }
  __device__ __forceinline__ void st(int lr, float2* line, int k, float2 v) const {
    constexpr int Px = 4 << LNX, hp = Px / 2, qp = Px / 4;
    int t, u;
    if (k < qp) { t = k; u = k; }
    else if (k >= Px - qp) { t = k - Px; u = k - hp; }
    else return;
    const int r = lr >= L ? 1 : 0, l = lr - r * L;
    const int j = j0 + l;
    const int j1 = 2 * t + r;
    float2 o = czero<float>();
    if (j1 != -hp && j < Py && j != Py / 2) {
      const int j1a = j1 < 0 ? -j1 : j1;
      o = cmul<float>(v, kh[l * KH_ROW + perm(j1a)]);
    }
    line[pidx(u)] = o;
  }
};

template <int LNX>
__global__ void __launch_bounds__(LINES_THREADS, 2)
    k_tbcB_w2(const float2* __restrict__ Vy, float2* __restrict__ W, TbcP p,
              const float2* __restrict__ tw, const float2* __restrict__ eh_c,
              const float2* __restrict__ eh_s, const float2* __restrict__ kh) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float2* buf = (float2*)sm_raw;
  constexpr int LPX = LNX + 2, Px = 1 << LPX, nx = 1 << LNX, ls = W2<Px>::LS, L = W2<Px>::L;
  const int Py = p.Py;
  const int f = blockIdx.y, d = blockIdx.z;
  const int j0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;
  const bool xcos = (f != 1);
  float2* kh_sm = buf + (size_t)2 * L * ls;
  for (int idx = tid; idx < L * (Px / 2); idx += nthr) {
    const int l = idx >> (LPX - 1), j1 = idx & (Px / 2 - 1);
    const int j = j0 + l;
    const int j2a = j < Py / 2 ? j : Py - j;
    kh_sm[l * KhatBPerm<LNX>::KH_ROW + KhatBPerm<LNX>::perm(j1)] =
        (j < Py && j != Py / 2) ? kh[(size_t)j2a * (Px / 2) + j1] : czero<float>();
  }
  // both parity lines of each column receive the mirrored column; the slots
  // [nx, Px - nx] are cleared
  {
    const float2* src = Vy + (size_t)(d * 3 + f) * nx * Py;
    for (int idx = tid; idx < L * nx; idx += nthr) {
      const int k1 = idx >> 1, l = idx & 1;
      const int j = j0 + l;
      const float2 c = j < Py ? src[(size_t)k1 * Py + j] : czero<float>();
      const float2 c0 = k1 == 0 ? (xcos ? cscale<float>(c, 2.f) : czero<float>()) : c;
      const float2 cm = xcos ? c : mk<float>(-c.x, -c.y);
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        float2* line = buf + (size_t)(r * L + l) * ls;
        line[pidx(k1)] = c0;
        if (k1 > 0) line[pidx(Px - k1)] = cm;
      }
    }
    for (int idx = tid; idx < 2 * L * (2 * nx + 1); idx += nthr) {
      const int l = idx / (2 * nx + 1), k = nx + idx - l * (2 * nx + 1);
      buf[(size_t)l * ls + pidx(k)] = czero<float>();
    }
    __syncthreads();
  }
  const int lr = warp >> 1, h = warp & 1;
  float2* line = buf + (size_t)lr * ls;
  OwnParityG<float> fwd;
  fwd.eh = xcos ? eh_c : eh_s;
  fwd.P = Px;
  fwd.L = L;
  fft_warp2<float, false, LPX>(line, h, lane, tw, p.twlog, 1 + lr, lr, fwd);
  pair_sync(1 + lr);
  KhatBPerm<LNX> kb;
  kb.kh = kh_sm;
  kb.j0 = j0;
  kb.Py = Py;
  kb.L = L;
  fft_warp2<float, true, LPX>(line, h, lane, tw, p.twlog, 1 + lr, lr, kb);
  pair_sync(1 + lr);
  if (h == 0) fft_warp<float, true, 32, 32>(line, Px / 2, LPX - 1, lane, true, tw, p.twlog);
  __syncthreads();
  float2* dst = W + (size_t)(d * 3 + f) * (nx + 1) * Py;
  const int sh = p.twlog - LPX;
  for (int idx = tid; idx < L * (nx + 1); idx += nthr) {
    const int q = idx >> 1, l = idx & 1;
    const int j = j0 + l;
    if (j >= Py) continue;
    const float2 z0 = buf[(size_t)l * ls + pidx(q)];
    const float2 z1 = buf[(size_t)(L + l) * ls + pidx(q)];
    dst[(size_t)q * Py + j] = cadd<float>(z0, cmul<float>(z1, twid<float, true>(tw, q << sh)));
  }
}

// pass C: grid (ceil((nx+1) / 4) row groups, 3 fields, ndir); four rows per
// block, the inverse torus transform of a row (2048 points) on a warp pair,
// then its projection (1024 points) on the pair's first warp
template <int LNY>
__global__ void __launch_bounds__(LINES_THREADS, 2)
    k_tbcC_w2(const float2* __restrict__ W, float2* __restrict__ Z, TbcP p,
              const float2* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float2* buf = (float2*)sm_raw;
  constexpr int LPY = LNY + 2, Py = 1 << LPY, ny = 1 << LNY, ls = W2<Py>::LS;
  constexpr int RB = 4;   // rows per block
  const int f = blockIdx.y, d = blockIdx.z;
  const int r0 = blockIdx.x * RB;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int l = warp >> 1, h = warp & 1;
  const bool ycos = (f != 0);
  RowC<float, LNY> rc;
  rc.src = W + (size_t)(d * 3 + f) * (p.nx + 1) * Py;
  rc.r0 = r0;
  rc.nx = p.nx;
  rc.ycos = ycos;
  float2* line = buf + (size_t)l * ls;
  fft_warp2<float, true, LPY>(line, h, lane, tw, p.twlog, 1 + l, l, rc);
  pair_sync(1 + l);
  if (h == 0) {
    StoreZ<float, LNY> sz;
    sz.Z = Z + (size_t)(d * 3 + f) * (p.nx + 1) * (ny + 1);
    sz.r0 = r0;
    sz.nx = p.nx;
    sz.ycos = ycos;
    sz.w = (float)p.wy;
    fft_warp<float, false, 32, 32>(line, 2 * ny, LNY + 1, lane, true, tw, p.twlog, l, sz);
  }
}

template <typename T> __host__ __device__ constexpr bool w2_ok(int ln) {
  return sizeof(T) == 4 && ln == 9;
}
static size_t smem_b_w2(int nx) {
  return sizeof(float2) * (4 * (size_t)padded_len(4 * nx) + 2 * (size_t)(2 * nx + 16));
}
static size_t smem_c_w2(int ny) { return sizeof(float2) * 4 * (size_t)padded_len(4 * ny); }

// ------------------------------------------------------------------ combine
// y = local part of (EJ1)/(uT1) + TBC rows, with the TBC sign that makes T
// the exterior admittance z x curl E^s of (EGa2):
//  row 1: (-1+tau1)E1 + (m pi h/a + vs1)E3 + (h/q)(2k^2 U1 - 2(n pi/b) W)
//  row 2: (-1+tau2)E2 + (n pi h/b + vs2)E3 + (h/c)(2k^2 U2 + 2(m pi/a) W)
//  row 3: (m pi h/a)E1 + (n pi h/b)E2 + (-1+tau3)E3
// One thread per mode pair (m, n), m < nx, n < ny, writing the rows of the
// three components that exist for it; grid (ceil(nx ny / 256), ndir).
template <typename T>
__global__ void k_combine(const C<T>* __restrict__ x, const C<T>* __restrict__ O,
                          const C<T>* __restrict__ top, C<T>* __restrict__ y, long long ys, TbcP p) {
  const int d = blockIdx.y;
  const int mn = blockIdx.x * blockDim.x + threadIdx.x;
  if (mn >= p.nx * p.ny) return;
  const int m = mn >> p.lny, n = mn & (p.ny - 1);
  const C<T>* xd = x + (size_t)d * p.nap;
  C<T>* yd = y + (size_t)d * ys;
  const int N = p.N, nyp = p.ny + 1;
  const size_t fs = (size_t)p.nx * nyp;
  const C<T>* Od = O + (size_t)d * 3 * fs;
  const T pa = (T)p.pia, pb = (T)p.pib, h = (T)p.h, ab = (T)p.ab;
  const T k2 = (T)p.k2x2;
  const int i1 = m * N + (n - 1), i2 = p.n1 + (m - 1) * (N + 1) + n;
  const int i3 = p.n1 + p.n2 + (m - 1) * N + (n - 1);
  const bool has1 = n >= 1, has2 = m >= 1, has3 = m >= 1 && n >= 1;
  const C<T> e1 = has1 ? xd[i1] : mk<T>(0, 0);
  const C<T> e2 = has2 ? xd[i2] : mk<T>(0, 0);
  const C<T> e3 = has3 ? xd[i3] : mk<T>(0, 0);
  const size_t o = (size_t)m * nyp + n;
  if (has1) {
    C<T> r = cmul<T>(cadd<T>(mk<T>(-1, 0), top[i1]), e1);
    if (has3) r = cadd<T>(r, cmul<T>(cadd<T>(mk<T>(m * pa * h, 0), top[p.nap + i1]), e3));
    const T s = h / (m == 0 ? ab / 2 : ab / 4);
    const C<T> t = csub<T>(cscale<T>(Od[o], k2), cscale<T>(Od[2 * fs + o], 2 * n * pb));
    yd[i1] = cadd<T>(r, cscale<T>(t, s));
  }
  if (has2) {
    C<T> r = cmul<T>(cadd<T>(mk<T>(-1, 0), top[i2]), e2);
    if (has3) r = cadd<T>(r, cmul<T>(cadd<T>(mk<T>(n * pb * h, 0), top[p.nap + i2]), e3));
    const T s = h / (n == 0 ? ab / 2 : ab / 4);
    const C<T> t = cadd<T>(cscale<T>(Od[fs + o], k2), cscale<T>(Od[2 * fs + o], 2 * m * pa));
    yd[i2] = cadd<T>(r, cscale<T>(t, s));
  }
  if (has3) {
    C<T> r = cscale<T>(e1, m * pa * h);
    r = cadd<T>(r, cscale<T>(e2, n * pb * h));
    yd[i3] = cadd<T>(r, cmul<T>(cadd<T>(mk<T>(-1, 0), top[i3]), e3));
  }
}

// Explicit instantiation (EXT empty) or its declaration (EXT = extern) of the
// four pass kernels of type T at log2 size LN; lets a type's instantiations
// be compiled in several translation units (in parallel) while one unit
// launches them.
#define TBC_PASS_KERNELS(EXT, T, LN)                                                          \
  EXT template __global__ void k_tbcA<T, LN>(const C<T>*, C<T>*, TbcP, const C<T>*,           \
                                             const C<T>*, const C<T>*);                       \
  EXT template __global__ void k_tbcB<T, LN>(const C<T>*, C<T>*, TbcP, const C<T>*,           \
                                             const C<T>*, const C<T>*, const C<T>*);          \
  EXT template __global__ void k_tbcC<T, LN>(const C<T>*, C<T>*, TbcP, const C<T>*);          \
  EXT template __global__ void k_tbcD<T, LN>(const C<T>*, C<T>*, TbcP, const C<T>*);

template <typename T> struct Tabs;
template <> struct Tabs<double> {
  static const double2* tw(cavity_ctx* c) { return c->tw64; }
  static const double2* ex(cavity_ctx* c, int k) { return c->ehat_x64[k]; }
  static const double2* ey(cavity_ctx* c, int k) { return c->ehat_y64[k]; }
  static const double2* kh(cavity_ctx* c) { return c->khat64; }
  static const double2* top(cavity_ctx* c) { return c->top64; }
};
template <> struct Tabs<float> {
  static const float2* tw(cavity_ctx* c) { return c->tw32; }
  static const float2* ex(cavity_ctx* c, int k) { return c->ehat_x32[k]; }
  static const float2* ey(cavity_ctx* c, int k) { return c->ehat_y32[k]; }
  static const float2* kh(cavity_ctx* c) { return c->khat32; }
  static const float2* top(cavity_ctx* c) { return c->top32; }
};

// shared memory of each pass (bytes) for the grid sizes of g
template <typename T> static size_t smem_a(int ny) { return sizeof(C<T>) * 2 * pairs_per_cta<T>(4 * ny) * (size_t)padded_len(4 * ny); }
template <typename T> static size_t smem_b(int nx) {
  return smem_b_lines<T>(nx) + (b_staged<T>(nx) ? smem_b_tables<T>(nx) : 0);
}
template <typename T> static size_t smem_c(int ny) { return sizeof(C<T>) * lines_per_cta<T>(4 * ny) * (size_t)padded_len(4 * ny); }
template <typename T> static size_t smem_d(int nx) { return sizeof(C<T>) * lines_per_cta<T>(2 * nx) * (size_t)padded_len(2 * nx); }

// opt every instantiation of kernel K into the device's shared-memory maximum
// once per process
template <typename K> static cavity_status smem_once(cavity_ctx* ctx, K kern, std::atomic<bool>& done) {
  if (!done) {
    CK(allow_max_smem(kern));
    done = true;
  }
  return CAVITY_OK;
}

// launch-accounting class of pass `k` (0..4: A, B, C, D, combine) for type T
template <typename T> static int kclass(int k) {
  if (sizeof(C<T>) == 8) return KC_TBC_A32 + k;
  if (std::is_same<T, double>::value) return KC_TBC_A64 + k;
  return KC_TBC_AP + k;
}

// Truncated aperture expansion (Sec. 7, Table 2: the paper's runs keep the
// modes m <= ~2a/lambda): y_i = 0 for unknowns i of a mode (m, n) with
// m > mm or n > nn.  Unknown order (Appendix A): E1 over m = 0..M, n = 1..N;
// E2 over m = 1..M, n = 0..N; E3 over m = 1..M, n = 1..N.
// grid (ceil(nap / 256), ndir)
template <typename T>
__global__ void k_mode_mask(C<T>* __restrict__ y, long long ystride, int nap, int N, int n1, int n2,
                            int mm, int nn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nap) return;
  int m, n;
  if (i < n1) {
    m = i / N;
    n = i - m * N + 1;
  } else if (i < n1 + n2) {
    const int j = i - n1;
    m = j / (N + 1) + 1;
    n = j - (m - 1) * (N + 1);
  } else {
    const int j = i - n1 - n2;
    m = j / N + 1;
    n = j - (m - 1) * N + 1;
  }
  if (m > mm || n > nn) y[(size_t)blockIdx.y * ystride + i] = czero<T>();
}

template <typename T>
cavity_status launch_mode_mask_t(cavity_ctx* ctx, int ndir, C<T>* y, long long ystride, int cls) {
  const cavity_desc& d = ctx->desc;
  if (d.modes_m <= 0 && d.modes_n <= 0) return CAVITY_OK;
  const Geo& g = ctx->g;
  const int mm = d.modes_m > 0 ? d.modes_m : g.M, nn = d.modes_n > 0 ? d.modes_n : g.N;
  KScope ks_(ctx, cls);
  k_mode_mask<T><<<dim3((g.nap + 255) / 256, ndir), 256, 0, ctx->stream>>>(y, ystride, g.nap, g.N, g.n1,
                                                                          g.n2, mm, nn);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

template <typename T>
cavity_status launch_apply(cavity_ctx* ctx, int ndir, const C<T>* x, C<T>* y, void* work,
                           long long ystride) {
  if (!ctx->g.fft_ok) {
    ctx->err = "the FFT operator needs the convolution period 4 on both axes";
    return CAVITY_EINVAL;
  }
  if (ystride < 0) ystride = ctx->g.nap;
  const Geo& g = ctx->g;
  const size_t need = std::max(std::max(smem_a<T>(g.ny), smem_b<T>(g.nx)),
                               std::max(smem_c<T>(g.ny), smem_d<T>(g.nx)));
  if (need > (size_t)smem_optin()) {
    ctx->err = "grid too large for the shared-memory transforms";
    return CAVITY_EINVAL;
  }
  TbcP p = make_params(ctx);
  size_t vy = (size_t)ndir * 3 * g.nx * g.Py;
  size_t z = (size_t)ndir * 3 * (g.nx + 1) * (g.ny + 1);
  C<T>* R1 = (C<T>*)work;                      // Vy, later Z
  C<T>* R2 = R1 + std::max(vy, z);             // W, later O
  cudaStream_t st = ctx->stream;
  const C<T>* tw = Tabs<T>::tw(ctx);
  const int T_ = LINES_THREADS;
  CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lny, [&](auto c) -> cavity_status {
    constexpr int LN = decltype(c)::value;
    constexpr int L = pairs_per_cta<T>(4 << LN);
    static std::atomic<bool> done{false};  // set once; host threads may race
    CKS(smem_once(ctx, k_tbcA<T, LN>, done));
    KScope ks_(ctx, kclass<T>(0));
    k_tbcA<T, LN><<<dim3((g.nx + L - 1) / L, 3, ndir), T_, smem_a<T>(g.ny), st>>>(
        x, R1, p, tw, Tabs<T>::ey(ctx, 0), Tabs<T>::ey(ctx, 1));
    return CAVITY_OK;
  }));
  CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lnx, [&](auto c) -> cavity_status {
    constexpr int LN = decltype(c)::value;
    constexpr int L = pairs_per_cta<T>(4 << LN);
    if constexpr (w2_ok<T>(LN)) {
      if (ctx->opt[CAVITY_OPT_PASS_B_2048] == 0) {
        static std::atomic<bool> done2{false};
        CKS(smem_once(ctx, k_tbcB_w2<LN>, done2));
        KScope ks_(ctx, kclass<T>(1));
        k_tbcB_w2<LN><<<dim3(g.Py / 2, 3, ndir), T_, smem_b_w2(g.nx), st>>>(
            (const float2*)R1, (float2*)R2, p, (const float2*)tw,
            (const float2*)Tabs<T>::ex(ctx, 0), (const float2*)Tabs<T>::ex(ctx, 1),
            (const float2*)Tabs<T>::kh(ctx));
        return CAVITY_OK;
      }
    }
    {
      static std::atomic<bool> done{false};  // set once; host threads may race
      CKS(smem_once(ctx, k_tbcB<T, LN>, done));
      KScope ks_(ctx, kclass<T>(1));
      k_tbcB<T, LN><<<dim3((g.Py + L - 1) / L, 3, ndir), T_, smem_b<T>(g.nx), st>>>(
          R1, R2, p, tw, Tabs<T>::ex(ctx, 0), Tabs<T>::ex(ctx, 1), Tabs<T>::kh(ctx));
      return CAVITY_OK;
    }
  }));
  CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lny, [&](auto c) -> cavity_status {
    constexpr int LN = decltype(c)::value;
    constexpr int L = lines_per_cta<T>(4 << LN);
    if constexpr (w2_ok<T>(LN)) {
      if (ctx->opt[CAVITY_OPT_PASS_C_2048] == 0) {
        static std::atomic<bool> done2{false};
        CKS(smem_once(ctx, k_tbcC_w2<LN>, done2));
        KScope ks_(ctx, kclass<T>(2));
        k_tbcC_w2<LN><<<dim3((g.nx + 1 + 3) / 4, 3, ndir), T_, smem_c_w2(g.ny), st>>>(
            (const float2*)R2, (float2*)R1, p, (const float2*)tw);
        return CAVITY_OK;
      }
    }
    {
      static std::atomic<bool> done{false};  // set once; host threads may race
      CKS(smem_once(ctx, k_tbcC<T, LN>, done));
      KScope ks_(ctx, kclass<T>(2));
      k_tbcC<T, LN><<<dim3((g.nx + 1 + L - 1) / L, 3, ndir), T_, smem_c<T>(g.ny), st>>>(R2, R1, p,
                                                                                       tw);
      return CAVITY_OK;
    }
  }));
  CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lnx, [&](auto c) -> cavity_status {
    constexpr int LN = decltype(c)::value;
    constexpr int L = lines_per_cta<T>(2 << LN);
    static std::atomic<bool> done{false};  // set once; host threads may race
    CKS(smem_once(ctx, k_tbcD<T, LN>, done));
    KScope ks_(ctx, kclass<T>(3));
    k_tbcD<T, LN><<<dim3((g.ny + 1 + L - 1) / L, 3, ndir), T_, smem_d<T>(g.nx), st>>>(R1, R2, p, tw);
    return CAVITY_OK;
  }));
  {
    KScope ks_(ctx, kclass<T>(4));
    k_combine<T><<<dim3((g.nx * g.ny + 255) / 256, ndir), 256, 0, st>>>(x, R2, Tabs<T>::top(ctx), y,
                                                                       ystride, p);
  }
  CK(cudaGetLastError());
  // truncated expansion: the rows of the dropped modes (the operator then
  // maps the kept subspace to itself, as does the mode-wise preconditioner)
  CKS(launch_mode_mask_t<T>(ctx, ndir, y, ystride, kclass<T>(4)));
  return CAVITY_OK;
}

