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
// FP32 for the inner Krylov iterations of the mixed path.
#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "fft.cuh"

struct TbcP {
  int nx, ny, M, N, Px, Py, lPx, lPy, lnx, lny, nap, n1, n2;
  double a, b, h, k2x2;  // k2x2 = 2 kappa0^2
  int twlog;
};

static TbcP make_params(const cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  TbcP p;
  p.nx = g.nx; p.ny = g.ny; p.M = g.M; p.N = g.N; p.Px = g.Px; p.Py = g.Py;
  p.lPx = g.lPx; p.lPy = g.lPy; p.lnx = g.lnx; p.lny = g.lny;
  p.nap = g.nap; p.n1 = g.n1; p.n2 = g.n2;
  p.a = g.a; p.b = g.b; p.h = g.h; p.k2x2 = 2.0 * ctx->kappa0 * ctx->kappa0;
  p.twlog = ilog2(ctx->TW);
  return p;
}

template <typename T> __device__ __forceinline__ C<T> czero() { return mk<T>(0, 0); }

// ------------------------------------------------------------------ setup
__global__ void k_twiddles(double2* tw64, float2* tw32, int TW) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= TW) return;
  double s, c;
  sincospi(-2.0 * (double)k / (double)TW, &s, &c);
  tw64[k] = make_double2(c, s);
  tw32[k] = make_float2((float)c, (float)s);
}

cavity_status launch_twiddles(cavity_ctx* ctx) {
  int TW = ctx->TW;
  CK(cudaMalloc(&ctx->tw64, sizeof(double2) * TW));
  CK(cudaMalloc(&ctx->tw32, sizeof(float2) * TW));
  {
    KScope ks_(ctx, KC_SETUP);
    k_twiddles<<<(TW + 255) / 256, 256, 0, ctx->stream>>>(ctx->tw64, ctx->tw32, TW);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// eps(d) = E(d/L) = int_0^side exp(-2 pi i (d/L) y) dy for |d| <= P-1 (0 at d=-P),
// transformed with a length-2P FFT; the convolution scale (1/2 for the cosine
// basis, 1/(2i) for the sine basis) and the 1/(2P) of the inverse are folded in.
__global__ void k_ehat(double2* out64, float2* out32, int P, int lP, double side, int pad,
                       int kind, const double2* __restrict__ tw, int twlog) {
  extern __shared__ double2 sm_e[];
  const int Q = 2 * P;
  double2* A = sm_e;
  for (int t = threadIdx.x; t < Q; t += blockDim.x) {
    int d = t < P ? t : t - Q;
    double2 v;
    if (d == 0) {
      v = make_double2(side, 0.0);
    } else if (d == -P) {
      v = make_double2(0.0, 0.0);
    } else {
      // (1 - exp(-2 pi i d / pad)) * L / (2 pi i d),  L = pad * side
      double s, c;
      sincospi(-2.0 * (double)d / (double)pad, &s, &c);
      double2 num = make_double2(1.0 - c, -s);
      double L = pad * side;
      double f = L / (2.0 * M_PI * (double)d);
      // num / i = (num.y, -num.x)
      v = make_double2(num.y * f, -num.x * f);
    }
    A[pidx(t)] = v;
  }
  __syncthreads();
  fft_inplace<double, false>(A, padded_len(Q), Q, lP + 1, 1, tw, twlog);
  for (int t = threadIdx.x; t < Q; t += blockDim.x) {
    double2 v = A[pidx(t)];
    double sc = 1.0 / (double)Q;
    double2 r;
    if (kind == 0) r = make_double2(0.5 * sc * v.x, 0.5 * sc * v.y);   // * 1/2
    else r = make_double2(0.5 * sc * v.y, -0.5 * sc * v.x);           // * 1/(2i)
    out64[t] = r;
    out32[t] = make_float2((float)r.x, (float)r.y);
  }
}

cavity_status launch_ehat(cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  int twlog = ilog2(ctx->TW);
  for (int kind = 0; kind < 2; ++kind) {
    CK(cudaMalloc(&ctx->ehat_x64[kind], sizeof(double2) * 2 * g.Px));
    CK(cudaMalloc(&ctx->ehat_x32[kind], sizeof(float2) * 2 * g.Px));
    CK(cudaMalloc(&ctx->ehat_y64[kind], sizeof(double2) * 2 * g.Py));
    CK(cudaMalloc(&ctx->ehat_y32[kind], sizeof(float2) * 2 * g.Py));
    size_t smx = sizeof(double2) * padded_len(2 * g.Px), smy = sizeof(double2) * padded_len(2 * g.Py);
    CK(allow_max_smem(k_ehat));
    {
      KScope ks_(ctx, KC_SETUP);
      k_ehat<<<1, std::max(32, fft_tpl<double>(2 * g.Px)), smx, ctx->stream>>>(ctx->ehat_x64[kind], ctx->ehat_x32[kind], g.Px,
                                            g.lPx, g.a, g.pad, kind, ctx->tw64, twlog);
    }
    {
      KScope ks_(ctx, KC_SETUP);
      k_ehat<<<1, std::max(32, fft_tpl<double>(2 * g.Py)), smy, ctx->stream>>>(ctx->ehat_y64[kind], ctx->ehat_y32[kind], g.Py,
                                            g.lPy, g.b, g.pad, kind, ctx->tw64, twlog);
    }
    CK(cudaGetLastError());
  }
  return CAVITY_OK;
}

// Lines per CTA: enough lines that a pass of the longest transform in the
// kernel occupies LINES_THREADS threads (nlong = that length).
#define LINES_THREADS 256
template <typename T> __host__ __device__ __forceinline__ int lines_per_cta(int nlong) {
  int tl = fft_tpl<T>(nlong);
  return tl >= LINES_THREADS ? 1 : LINES_THREADS / tl;
}

// ------------------------------------------------------------------ pass A
// grid (ceil(nx / L) row groups, 3 fields, ndir); field 0: cs (E1), 1: sc (E2),
// 2: cc (w).  Per row k1: the mirrored coefficient sequence along x2 is
// transformed (length Py), multiplied by the transform of the 1-D kernel
// (length 2 Py, periodic extension) and transformed back: a linear
// convolution giving the basis transform at j2 in the symmetric box.
template <typename T>
__global__ void __launch_bounds__(LINES_THREADS, sizeof(T) == 4 ? 3 : 2) k_tbcA(const C<T>* __restrict__ x, C<T>* __restrict__ Vy,
                                                        TbcP p, const C<T>* __restrict__ tw,
                                                        const C<T>* __restrict__ eh_c,
                                                        const C<T>* __restrict__ eh_s) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  const int Py = p.Py, Q = 2 * Py, ls = padded_len(Q);
  const int L = lines_per_cta<T>(Q);
  const int f = blockIdx.y, d = blockIdx.z;
  const int row0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const C<T>* E1 = x + (size_t)d * p.nap;
  const C<T>* E2 = E1 + p.n1;
  const bool ycos = (f != 0);
  for (int t = tid; t < L * ls; t += nthr) buf[t] = czero<T>();
  __syncthreads();
  const int nk = p.N + 1;                     // = ny, a power of two
  for (int idx = tid; idx < L * nk; idx += nthr) {
    const int l = idx >> p.lny, k2 = idx & (nk - 1);
    const int k1 = row0 + l;
    if (k1 >= p.nx) continue;
    C<T> c = czero<T>();
    if (f == 0) {
      if (k2 >= 1) c = E1[k1 * p.N + (k2 - 1)];
    } else if (f == 1) {
      if (k1 >= 1) c = E2[(k1 - 1) * (p.N + 1) + k2];
    } else {
      if (k2 >= 1) c = cscale<T>(E1[k1 * p.N + (k2 - 1)], (T)(k2 * M_PI / p.b));
      if (k1 >= 1) c = csub<T>(c, cscale<T>(E2[(k1 - 1) * (p.N + 1) + k2], (T)(k1 * M_PI / p.a)));
    }
    C<T>* line = buf + (size_t)l * ls;
    if (ycos) {
      if (k2 == 0) line[0] = cscale<T>(c, (T)2);
      else { line[pidx(k2)] = c; line[pidx(Py - k2)] = c; }
    } else if (k2 >= 1) {
      line[pidx(k2)] = c;
      line[pidx(Py - k2)] = mk<T>(-c.x, -c.y);
    }
  }
  __syncthreads();
  fft_inplace<T, false>(buf, ls, Py, p.lPy, L, tw, p.twlog);
  const C<T>* eh = ycos ? eh_c : eh_s;
  for (int idx = tid; idx < L * Py; idx += nthr) {
    const int l = idx >> p.lPy, t = idx & (Py - 1);
    C<T>* line = buf + (size_t)l * ls;
    const C<T> sv = line[pidx(t)];
    line[pidx(t)] = cmul<T>(sv, eh[t]);
    line[pidx(t + Py)] = cmul<T>(sv, eh[t + Py]);
  }
  __syncthreads();
  fft_inplace<T, true>(buf, ls, Q, p.lPy + 1, L, tw, p.twlog);
  for (int idx = tid; idx < L * Py; idx += nthr) {
    const int l = idx >> p.lPy, j = idx & (Py - 1);
    const int k1 = row0 + l;
    if (k1 >= p.nx) continue;
    C<T> r = czero<T>();
    if (j != Py / 2) {
      const int j2 = j < Py / 2 ? j : j - Py;
      r = buf[(size_t)l * ls + pidx(j2 & (Q - 1))];
    }
    Vy[((size_t)(d * 3 + f) * p.nx + k1) * Py + j] = r;
  }
}

// ------------------------------------------------------------------ pass B
// grid (Py / L column groups, 3 fields, ndir).  Per column j2: the basis
// transform along x1 (as in pass A), times F(G)(|j1|, |j2|)/(Lx Ly), then the
// inverse torus transform along x1 evaluated at the nodes p = 0..nx.
template <typename T>
__global__ void __launch_bounds__(LINES_THREADS, sizeof(T) == 4 ? 3 : 2) k_tbcB(const C<T>* __restrict__ Vy, C<T>* __restrict__ W,
                                                        TbcP p, const C<T>* __restrict__ tw,
                                                        const C<T>* __restrict__ eh_c,
                                                        const C<T>* __restrict__ eh_s,
                                                        const C<T>* __restrict__ kh) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  const int Px = p.Px, Py = p.Py, Q = 2 * Px, ls = padded_len(Q);
  const int L = lines_per_cta<T>(Q);
  const int f = blockIdx.y, d = blockIdx.z;
  const int j0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xcos = (f != 1);
  const C<T>* src = Vy + (size_t)(d * 3 + f) * p.nx * Py;
  for (int t = tid; t < L * ls; t += nthr) buf[t] = czero<T>();
  __syncthreads();
  const int lL = __ffs(L) - 1;
  for (int idx = tid; idx < L * p.nx; idx += nthr) {
    const int k1 = idx >> lL, l = idx & (L - 1);
    const int j = j0 + l;
    if (j >= Py) continue;
    const C<T> c = src[(size_t)k1 * Py + j];
    C<T>* line = buf + (size_t)l * ls;
    if (xcos) {
      if (k1 == 0) line[0] = cscale<T>(c, (T)2);
      else { line[pidx(k1)] = c; line[pidx(Px - k1)] = c; }
    } else if (k1 >= 1) {
      line[pidx(k1)] = c;
      line[pidx(Px - k1)] = mk<T>(-c.x, -c.y);
    }
  }
  __syncthreads();
  fft_inplace<T, false>(buf, ls, Px, p.lPx, L, tw, p.twlog);
  const C<T>* eh = xcos ? eh_c : eh_s;
  for (int idx = tid; idx < L * Px; idx += nthr) {
    const int l = idx >> p.lPx, t = idx & (Px - 1);
    C<T>* line = buf + (size_t)l * ls;
    const C<T> sv = line[pidx(t)];
    line[pidx(t)] = cmul<T>(sv, eh[t]);
    line[pidx(t + Px)] = cmul<T>(sv, eh[t + Px]);
  }
  __syncthreads();
  fft_inplace<T, true>(buf, ls, Q, p.lPx + 1, L, tw, p.twlog);
  // K-hat line of length Px in place (sources never overlap other threads'
  // destinations: i < Px/2 reads i, i > Px/2 reads Px + i)
  const int hp = Px / 2;
  for (int idx = tid; idx < L * Px; idx += nthr) {
    const int l = idx >> p.lPx, i = idx & (Px - 1);
    const int j = j0 + l;
    C<T>* line = buf + (size_t)l * ls;
    C<T> r = czero<T>();
    if (i != Px / 2 && j < Py && j != Py / 2) {
      const int j1 = i < Px / 2 ? i : i - Px;
      const int j1a = j1 < 0 ? -j1 : j1;
      const int j2a = j < Py / 2 ? j : Py - j;
      r = cmul<T>(line[pidx(j1 & (Q - 1))], kh[(size_t)j2a * hp + j1a]);
    }
    line[pidx(i)] = r;
  }
  __syncthreads();
  fft_inplace<T, true>(buf, ls, Px, p.lPx, L, tw, p.twlog);
  C<T>* dst = W + (size_t)(d * 3 + f) * (p.nx + 1) * Py;
  for (int idx = tid; idx < L * (p.nx + 1); idx += nthr) {
    const int q = idx >> lL, l = idx & (L - 1);
    const int j = j0 + l;
    if (j >= Py) continue;
    dst[(size_t)q * Py + j] = buf[(size_t)l * ls + pidx(q)];
  }
}

// ------------------------------------------------------------------ pass C
// grid (ceil((nx+1)/L) row groups, 3 fields, ndir).  Per node row p: inverse
// torus transform along x2 at q = 0..ny, then the trapezoid projection onto
// cos/sin(n pi q/ny) as an extended FFT of length 2 ny.
template <typename T>
__global__ void __launch_bounds__(LINES_THREADS, sizeof(T) == 4 ? 3 : 2) k_tbcC(const C<T>* __restrict__ W, C<T>* __restrict__ Z,
                                                        TbcP p, const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  const int Py = p.Py, ls = padded_len(Py);
  const int L = lines_per_cta<T>(Py);
  const int f = blockIdx.y, d = blockIdx.z;
  const int r0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int ny = p.ny, n2 = 2 * ny;
  const bool ycos = (f != 0);
  const C<T>* src = W + (size_t)(d * 3 + f) * (p.nx + 1) * Py;
  for (int idx = tid; idx < L * Py; idx += nthr) {
    const int l = idx >> p.lPy, t = idx & (Py - 1);
    const int row = r0 + l;
    buf[(size_t)l * ls + pidx(t)] = row <= p.nx ? src[(size_t)row * Py + t] : czero<T>();
  }
  __syncthreads();
  fft_inplace<T, true>(buf, ls, Py, p.lPy, L, tw, p.twlog);
  // even (cos) / odd (sin) extension of U(q), q = 0..ny, to length 2 ny in place
  for (int idx = tid; idx < L * n2; idx += nthr) {
    const int l = idx >> (p.lny + 1), t = idx & (n2 - 1);
    C<T>* line = buf + (size_t)l * ls;
    if (t <= ny) {
      if (!ycos && (t == 0 || t == ny)) line[pidx(t)] = czero<T>();
    } else {
      C<T> v = line[pidx(n2 - t)];
      line[pidx(t)] = ycos ? v : mk<T>(-v.x, -v.y);
    }
  }
  __syncthreads();
  fft_inplace<T, false>(buf, ls, n2, p.lny + 1, L, tw, p.twlog);
  const T w = (T)(0.5 * p.b / ny);
  for (int l = 0; l < L; ++l) {
    const int row = r0 + l;
    if (row > p.nx) break;
    for (int n = tid; n <= ny; n += nthr) {
      const C<T> v = buf[(size_t)l * ls + pidx(n)];
      Z[((size_t)(d * 3 + f) * (p.nx + 1) + row) * (ny + 1) + n] =
          ycos ? cscale<T>(v, w) : cscale<T>(cmul_i<T>(v), w);
    }
  }
}

// ------------------------------------------------------------------ pass D
// grid (ceil((ny+1)/L) column groups, 3 fields, ndir).  Per column n: the
// trapezoid projection along x1 (extended FFT of length 2 nx).
template <typename T>
__global__ void __launch_bounds__(LINES_THREADS, sizeof(T) == 4 ? 3 : 2) k_tbcD(const C<T>* __restrict__ Z, C<T>* __restrict__ O,
                                                        TbcP p, const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  const int nx = p.nx, n2 = 2 * p.nx, ny = p.ny, ls = padded_len(n2);
  const int L = lines_per_cta<T>(n2);
  const int f = blockIdx.y, d = blockIdx.z;
  const int c0 = blockIdx.x * L;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xcos = (f != 1);
  const C<T>* src = Z + (size_t)(d * 3 + f) * (nx + 1) * (ny + 1);
  const int lL = __ffs(L) - 1;
  for (int idx = tid; idx < L * n2; idx += nthr) {
    const int t = idx >> lL, l = idx & (L - 1);
    const int col = c0 + l;
    C<T> r = czero<T>();
    if (col <= ny) {
      if (t <= nx) {
        r = src[(size_t)t * (ny + 1) + col];
        if (!xcos && (t == 0 || t == nx)) r = czero<T>();
      } else {
        r = src[(size_t)(n2 - t) * (ny + 1) + col];
        if (!xcos) r = mk<T>(-r.x, -r.y);
      }
    }
    buf[(size_t)l * ls + pidx(t)] = r;
  }
  __syncthreads();
  fft_inplace<T, false>(buf, ls, n2, p.lnx + 1, L, tw, p.twlog);
  C<T>* dst = O + (size_t)(d * 3 + f) * nx * (ny + 1);
  const T w = (T)(0.5 * p.a / nx);
  for (int idx = tid; idx < L * nx; idx += nthr) {
    const int m = idx >> lL, l = idx & (L - 1);
    const int col = c0 + l;
    if (col > ny) continue;
    const C<T> v = buf[(size_t)l * ls + pidx(m)];
    dst[(size_t)m * (ny + 1) + col] = xcos ? cscale<T>(v, w) : cscale<T>(cmul_i<T>(v), w);
  }
}

// ------------------------------------------------------------------ combine
// y = local part of (EJ1)/(uT1) + TBC rows (with the sign of the exterior
// admittance, see the design notes):
//  row 1: (-1+tau1)E1 + (m pi h/a + vs1)E3 + (h/q)(2k^2 U1 - 2(n pi/b) W)
//  row 2: (-1+tau2)E2 + (n pi h/b + vs2)E3 + (h/c)(2k^2 U2 + 2(m pi/a) W)
//  row 3: (m pi h/a)E1 + (n pi h/b)E2 + (-1+tau3)E3
template <typename T>
__global__ void k_combine(const C<T>* __restrict__ x, const C<T>* __restrict__ O,
                          const C<T>* __restrict__ top, C<T>* __restrict__ y, long long ys, TbcP p,
                          int ndir) {
  const long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= (long long)ndir * p.nap) return;
  const int d = (int)(gid / p.nap), i = (int)(gid - (long long)d * p.nap);
  const C<T>* xd = x + (size_t)d * p.nap;
  const C<T>* E1 = xd;
  const C<T>* E2 = xd + p.n1;
  const C<T>* E3 = xd + p.n1 + p.n2;
  const int N = p.N, nyp = p.ny + 1;
  const size_t fs = (size_t)p.nx * nyp;
  const C<T>* Ocs = O + (size_t)(d * 3 + 0) * fs;
  const C<T>* Osc = O + (size_t)(d * 3 + 1) * fs;
  const C<T>* Occ = O + (size_t)(d * 3 + 2) * fs;
  const T pa = (T)(M_PI / p.a), pb = (T)(M_PI / p.b), h = (T)p.h, ab = (T)(p.a * p.b);
  const T k2 = (T)p.k2x2;
  C<T> r;
  if (i < p.n1) {
    const int m = i / N, n = i - m * N + 1;
    r = cmul<T>(cadd<T>(mk<T>(-1, 0), top[i]), E1[i]);
    if (m >= 1) {
      C<T> cf = cadd<T>(mk<T>(m * pa * h, 0), top[p.nap + i]);
      r = cadd<T>(r, cmul<T>(cf, E3[(m - 1) * N + (n - 1)]));
    }
    const T s = h / (m == 0 ? ab / 2 : ab / 4);
    C<T> t = csub<T>(cscale<T>(Ocs[(size_t)m * nyp + n], k2),
                     cscale<T>(Occ[(size_t)m * nyp + n], 2 * n * pb));
    r = cadd<T>(r, cscale<T>(t, s));
  } else if (i < p.n1 + p.n2) {
    const int ii = i - p.n1;
    const int m = ii / (N + 1) + 1, n = ii - (m - 1) * (N + 1);
    r = cmul<T>(cadd<T>(mk<T>(-1, 0), top[i]), E2[ii]);
    if (n >= 1) {
      C<T> cf = cadd<T>(mk<T>(n * pb * h, 0), top[p.nap + i]);
      r = cadd<T>(r, cmul<T>(cf, E3[(m - 1) * N + (n - 1)]));
    }
    const T s = h / (n == 0 ? ab / 2 : ab / 4);
    C<T> t = cadd<T>(cscale<T>(Osc[(size_t)m * nyp + n], k2),
                     cscale<T>(Occ[(size_t)m * nyp + n], 2 * m * pa));
    r = cadd<T>(r, cscale<T>(t, s));
  } else {
    const int ii = i - p.n1 - p.n2;
    const int m = ii / N + 1, n = ii - (m - 1) * N + 1;
    r = cscale<T>(E1[m * N + (n - 1)], m * pa * h);
    r = cadd<T>(r, cscale<T>(E2[(m - 1) * (N + 1) + n], n * pb * h));
    r = cadd<T>(r, cmul<T>(cadd<T>(mk<T>(-1, 0), top[i]), E3[ii]));
  }
  y[(size_t)d * ys + i] = r;
}

size_t apply_work_bytes(const Geo& g, int ndir, int eb) {
  size_t vy = (size_t)ndir * 3 * g.nx * g.Py;
  size_t w = (size_t)ndir * 3 * (g.nx + 1) * g.Py;
  size_t z = (size_t)ndir * 3 * (g.nx + 1) * (g.ny + 1);
  size_t o = (size_t)ndir * 3 * g.nx * (g.ny + 1);
  // Vy and Z share one region, W and O another; eb = bytes of one complex
  return (std::max(vy, z) + std::max(w, o)) * (size_t)eb;
}

template <typename T> struct SmemCfg {
  size_t a, b, c, d;
  int La, Lb, Lc, Ld;
};

template <typename T> static SmemCfg<T> smem_cfg(const Geo& g) {
  SmemCfg<T> s;
  s.La = lines_per_cta<T>(2 * g.Py);
  s.Lb = lines_per_cta<T>(2 * g.Px);
  s.Lc = lines_per_cta<T>(g.Py);
  s.Ld = lines_per_cta<T>(2 * g.nx);
  s.a = sizeof(C<T>) * (size_t)s.La * padded_len(2 * g.Py);
  s.b = sizeof(C<T>) * (size_t)s.Lb * padded_len(2 * g.Px);
  s.c = sizeof(C<T>) * (size_t)s.Lc * padded_len(g.Py);
  s.d = sizeof(C<T>) * (size_t)s.Ld * padded_len(2 * g.nx);
  return s;
}

// every pass kernel may use up to the device's opt-in shared memory
template <typename T>
static cavity_status set_smem(cavity_ctx* ctx) {
  CK(allow_max_smem(k_tbcA<T>));
  CK(allow_max_smem(k_tbcB<T>));
  CK(allow_max_smem(k_tbcC<T>));
  CK(allow_max_smem(k_tbcD<T>));
  return CAVITY_OK;
}

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

template <typename T>
cavity_status launch_apply(cavity_ctx* ctx, int ndir, const C<T>* x, C<T>* y, void* work,
                           long long ystride) {
  if (ystride < 0) ystride = ctx->g.nap;
  const Geo& g = ctx->g;
  const SmemCfg<T> sc = smem_cfg<T>(g);
  static bool smem_set[2] = {false, false};
  const int ti = sizeof(T) == 8 ? 0 : 1;
  const size_t need = std::max(std::max(sc.a, sc.b), std::max(sc.c, sc.d));
  if (need > (size_t)smem_optin()) {
    ctx->err = "grid too large for the shared-memory transforms";
    return CAVITY_EINVAL;
  }
  if (!smem_set[ti]) {
    CKS(set_smem<T>(ctx));
    smem_set[ti] = true;
  }
  TbcP p = make_params(ctx);
  size_t vy = (size_t)ndir * 3 * g.nx * g.Py;
  size_t z = (size_t)ndir * 3 * (g.nx + 1) * (g.ny + 1);
  C<T>* R1 = (C<T>*)work;                      // Vy, later Z
  C<T>* R2 = R1 + std::max(vy, z);             // W, later O
  cudaStream_t st = ctx->stream;
  const C<T>* tw = Tabs<T>::tw(ctx);
  const int T_ = LINES_THREADS;
  {
    KScope ks_(ctx, (sizeof(T) == 8 ? KC_TBC_A64 : KC_TBC_A32));
    k_tbcA<T><<<dim3((g.nx + sc.La - 1) / sc.La, 3, ndir), T_, sc.a, st>>>(
        x, R1, p, tw, Tabs<T>::ey(ctx, 0), Tabs<T>::ey(ctx, 1));
  }
  {
    KScope ks_(ctx, (sizeof(T) == 8 ? KC_TBC_B64 : KC_TBC_B32));
    k_tbcB<T><<<dim3((g.Py + sc.Lb - 1) / sc.Lb, 3, ndir), T_, sc.b, st>>>(
        R1, R2, p, tw, Tabs<T>::ex(ctx, 0), Tabs<T>::ex(ctx, 1), Tabs<T>::kh(ctx));
  }
  {
    KScope ks_(ctx, (sizeof(T) == 8 ? KC_TBC_C64 : KC_TBC_C32));
    k_tbcC<T><<<dim3((g.nx + 1 + sc.Lc - 1) / sc.Lc, 3, ndir), T_, sc.c, st>>>(R2, R1, p, tw);
  }
  {
    KScope ks_(ctx, (sizeof(T) == 8 ? KC_TBC_D64 : KC_TBC_D32));
    k_tbcD<T><<<dim3((g.ny + 1 + sc.Ld - 1) / sc.Ld, 3, ndir), T_, sc.d, st>>>(R1, R2, p, tw);
  }
  long long tot = (long long)ndir * g.nap;
  {
    KScope ks_(ctx, (sizeof(T) == 8 ? KC_COMB64 : KC_COMB32));
    k_combine<T><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(x, R2, Tabs<T>::top(ctx), y, ystride,
                                                                p, ndir);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

template cavity_status launch_apply<double>(cavity_ctx*, int, const double2*, double2*, void*,
                                           long long);
template cavity_status launch_apply<float>(cavity_ctx*, int, const float2*, float2*, void*,
                                          long long);

// ------------------------------------------------------------------ no-alloc
// Variant of cavity_apply for callers that must not allocate device memory.
// The four transform passes need scratch for their intermediate grids; here it
// lives in a fixed device array compiled into the library instead of the
// context's workspace.  Every pass writes all of the scratch it later reads
// within the same call, so nothing has to be cleared between calls.
#define CAVITY_NOALLOC_SCRATCH_BYTES (4u << 20)
static __device__ __align__(256) unsigned char g_noalloc_scratch[CAVITY_NOALLOC_SCRATCH_BYTES];
static void* g_noalloc_addr[64] = {nullptr};
static std::mutex g_noalloc_mu;

extern "C" cavity_status cavity_apply_noalloc(cavity_ctx* ctx, int ndir, int precision,
                                              const void* x, void* y) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared || ndir < 1 || !x || !y ||
      (precision != CAVITY_FP64 && precision != CAVITY_MIXED)) {
    ctx->err = "cavity_apply_noalloc: not prepared or bad arguments";
    return CAVITY_EINVAL;
  }
  const size_t need = apply_work_bytes(ctx->g, ndir,
                                       precision == CAVITY_FP64 ? sizeof(double2) : sizeof(float2));
  if (need > CAVITY_NOALLOC_SCRATCH_BYTES) {
    ctx->err = "cavity_apply_noalloc: needs " + std::to_string(need) +
               " bytes of scratch, more than the fixed " +
               std::to_string(CAVITY_NOALLOC_SCRATCH_BYTES) +
               " (use fewer directions, a smaller grid, or cavity_apply)";
    return CAVITY_EINVAL;
  }
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != ctx->device || dev < 0 || dev >= 64) {
    ctx->err = "cavity_apply_noalloc: the context's device must be current";
    return CAVITY_EINVAL;
  }
  void* scratch;
  {
    // first call on this device: resolve the device address of the array
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_addr[dev]) {
      void* p = nullptr;
      CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
      g_noalloc_addr[dev] = p;
    }
    scratch = g_noalloc_addr[dev];
  }
  if (precision == CAVITY_FP64)
    CKS(launch_apply<double>(ctx, ndir, (const double2*)x, (double2*)y, scratch));
  else
    CKS(launch_apply<float>(ctx, ndir, (const float2*)x, (float2*)y, scratch));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}
