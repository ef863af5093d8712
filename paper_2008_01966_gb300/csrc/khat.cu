// Kernel table of Sec. 5.2: the 2-D Fourier transform of the truncated
// free-space Green's function,
//     F(G)(rho) = 1/2 int_0^R J0(2 pi rho r) exp(i kappa0 r) dr,
// R = sqrt(2) max(a, b), at rho = |(j1/Lx, j2/Ly)| for the quarter box
// 0 <= j1 < Px/2, 0 <= j2 < Py/2 (the table is even in j1 and in j2).
// (The paper prints 1/(4 pi) in front of the radial integral; the angular
// integral contributes 2 pi J0, hence the 1/2.)
//
// The integrand is entire, so composite Gauss-Legendre quadrature converges
// geometrically: panels no wider than pi / (2 pi rho + |kappa0|), 16 nodes
// each.  One warp per table entry, lanes striding over panels, a fixed-order
// shuffle reduction (deterministic).  FP64 throughout.  Entries of large
// argument away from the ridge 2 pi rho = kappa0 use the asymptotic evaluation
// below instead (most of the box: the quadrature's cost grows with rho).
//
// J0: CUDA's j0() for x < 8; above that its error relative to the envelope
// sqrt(2/(pi x)) grows to ~1e-12, and because it is systematic it survives
// the quadrature sum, so J0 is evaluated here from two classical methods:
//   8 <= x < 25   Miller's backward recurrence J_{k-1} = (2k/x) J_k - J_{k+1}
//                 from an order N well above x, normalised by
//                 J_0 + 2 sum_k J_{2k} = 1;
//   x >= 25       Hankel's asymptotic expansion
//                 J0(x) = sqrt(2/(pi x)) (P cos chi - Q sin chi), chi = x - pi/4,
//                 P = sum_k (-1)^k b_{2k} x^{-2k},  Q = -sum_k (-1)^k b_{2k+1} x^{-2k-1},
//                 b_k = 1^2 3^2 ... (2k-1)^2 / (k! 8^k), summed to its smallest
//                 term, with cos chi = (cos x + sin x)/sqrt 2 (no rounding of
//                 x - pi/4).
// Both stay within ~1e-15 of the envelope (checked against 40-digit values).
#include <cmath>
#include <vector>

#include "common.cuh"

#define GLN 16
__constant__ double c_gl_x[GLN];
__constant__ double c_gl_w[GLN];

// Gauss-Legendre nodes and weights on [-1, 1] by Newton's iteration on the
// three-term recurrence of the Legendre polynomials.
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

__device__ double bessel_j0(double x) {
  if (x < 8.0) return j0(x);
  if (x < 25.0) {
    const int N = 2 * (int)(0.5 * (x + 12.0 * cbrt(x) + 30.0));
    const double ix2 = 2.0 / x;
    double jp1 = 0.0, jk = 1e-30, s = 0.0;
    for (int k = N; k >= 1; --k) {
      const double jm1 = (k * ix2) * jk - jp1;   // J_{k-1}
      jp1 = jk;
      jk = jm1;
      if (((k - 1) & 1) == 0 && k > 1) s += 2.0 * jk;
      if (fabs(jk) > 1e250) {
        jk *= 1e-250;
        jp1 *= 1e-250;
        s *= 1e-250;
      }
    }
    return jk / (s + jk);
  }
  double P = 0.0, Q = 0.0, t = 1.0;
  const double i8x = 1.0 / (8.0 * x);
  for (int k = 0; k < 64; ++k) {
    // t = b_k / x^k
    if ((k & 1) == 0) P += (k & 2) ? -t : t;
    else Q += (k & 2) ? t : -t;
    const double tn = t * (double)((2 * k + 1) * (2 * k + 1)) * i8x / (double)(k + 1);
    if (tn > t || tn < 1e-18) break;
    t = tn;
  }
  double sx, cx;
  sincos(x, &sx, &cx);
  const double r2 = 0.70710678118654752440;
  const double cchi = (cx + sx) * r2, schi = (sx - cx) * r2;
  return sqrt(2.0 / (M_PI * x)) * (P * cchi - Q * schi);
}

// ---- the paper's large-frequency scheme (CAVITY_KHAT_PAPER), Sec. 5.2:
//   int_0^R J0(c r) e^{i k r} dr = int_0^inf - (1/c) int_{cR}^inf J0(z) e^{i k z/c} dz,
// int_0^inf = 1/sqrt(c^2 - k^2) (c > k) or i/sqrt(k^2 - c^2) (c < k); in the tail
// J0(z) ~ sqrt(2/(pi z)) (cos(z - pi/4) + sin(z - pi/4)/(8z)), the exponentials
// e^{+-i(z - pi/4)} combine with e^{i k z/c} into
//   A(p) = int_Z^inf e^{ipz} z^{-1/2} dz = sqrt(pi/(2|p|)) (1 + i - 2C(T) - 2iS(T)),
//   T = sqrt(2|p|Z/pi) (complex conjugate for p < 0), and
//   B(p) = int_Z^inf e^{ipz} z^{-3/2} dz = 2 e^{ipZ}/sqrt(Z) + 2ip A(p),
// p = k/c +- 1, with the Fresnel integrals C, S from their two-term asymptotic
// expansions.  (The paper prints 1/(c^2 - k^2) for the integral to infinity and
// sqrt(pi)/(2p) in front of A; the forms above are the corrected ones.)
#define KHAT_PAPER_CR (20.0 * M_PI * 1.41421356237309504880)

__device__ double2 kp_tail_half(double p, double Z) {
  const double ap = fabs(p);
  const double T = sqrt(2.0 * ap * Z / M_PI);
  const double u = M_PI * T * T;
  const double f = (1.0 - 3.0 / (u * u)) / (M_PI * T);
  const double g = (1.0 - 15.0 / (u * u)) / (M_PI * M_PI * T * T * T);
  double sp, cp;
  sincos(0.5 * u, &sp, &cp);
  const double C = 0.5 + f * sp - g * cp;
  const double S = 0.5 - f * cp - g * sp;
  const double pre = sqrt(M_PI / (2.0 * ap));
  double2 v = make_double2(pre * (1.0 - 2.0 * C), pre * (1.0 - 2.0 * S));
  if (p < 0) v.y = -v.y;
  return v;
}

__device__ double2 kp_tail_3half(double p, double Z) {
  const double2 A = kp_tail_half(p, Z);
  double s, c;
  sincos(p * Z, &s, &c);
  const double w = 2.0 / sqrt(Z);
  // 2 e^{ipZ}/sqrt(Z) + 2 i p A
  return make_double2(w * c - 2.0 * p * A.y, w * s + 2.0 * p * A.x);
}

__device__ double2 khat_paper_tail(double c, double k, double R) {
  const double d = c * c - k * k;
  const double2 inf = d > 0 ? make_double2(1.0 / sqrt(d), 0.0) : make_double2(0.0, 1.0 / sqrt(-d));
  const double Z = c * R;
  const double pp = k / c + 1.0, pm = k / c - 1.0;
  const double r2 = 0.70710678118654752440;
  const double2 e4 = make_double2(r2, -r2), e4c = make_double2(r2, r2);  // e^{-i pi/4}, e^{+i pi/4}
  const double2 ap = kp_tail_half(pp, Z), am = kp_tail_half(pm, Z);
  const double2 bp = kp_tail_3half(pp, Z), bm = kp_tail_3half(pm, Z);
  const double2 cosp = cscale<double>(cadd<double>(cmul<double>(e4, ap), cmul<double>(e4c, am)), 0.5);
  const double2 dsin = csub<double>(cmul<double>(e4, bp), cmul<double>(e4c, bm));
  const double2 sinp = make_double2(0.5 * dsin.y, -0.5 * dsin.x);     // / (2i)
  const double2 tail = cscale<double>(cadd<double>(cosp, cscale<double>(sinp, 0.125)),
                                      sqrt(2.0 / M_PI) / c);
  return cscale<double>(csub<double>(inf, tail), 0.5);
}

// ---- large-argument evaluation of the same integral (default scheme).
// Where c R >= KHAT_ASYM_CR and |c - kappa0| R >= KHAT_ASYM_GAP:
//   int_0^R = int_0^inf - int_R^inf,  int_0^inf as in the paper's scheme, and
//   int_R^inf J0(c r) e^{i k r} dr = (1/c) int_Z^inf J0(z) e^{i k z/c} dz, Z = c R,
// with the complete Hankel expansion
//   J0(z) = sqrt(2/pi) (1/2) sum_m b_m z^{-m-1/2} [(-i)^m e^{i(z - pi/4)} + i^m e^{-i(z - pi/4)}],
//   b_m = 1^2 3^2 ... (2m-1)^2 / (m! 8^m),
// and each  F_m(p) = int_Z^inf z^{-m-1/2} e^{ipz} dz  (p = 1 + k/c, k/c - 1) from
// repeated integration by parts,
//   F_m(p) = (i/p) e^{ipZ} Z^{-m-1/2} sum_j (m + 1/2)_j (-i/(pZ))^j,
// both series summed to their smallest term.  The thresholds keep every series
// far inside its range (|p| Z >= 30, Z >= 100).  Measured against a 30-digit
// evaluation the result is within ~2e-15 there, better than the quadrature,
// whose sum of ~1000 oscillating panels loses ~Z 1e-16 to the rounding of c r.
#define KHAT_ASYM_CR 100.0
#define KHAT_ASYM_GAP 30.0
#define KHAT_NB 40
__constant__ double c_hank_b[KHAT_NB];

__device__ double2 khat_f_series(double s, double p, double Z, double2 eipz, double zs) {
  // (i/p) e^{ipZ} Z^{-s} sum_j (s)_j (-i/(pZ))^j ;  zs = Z^{-s}
  const double x = -1.0 / (p * Z);         // -i/(pZ) = i x
  double2 term = make_double2(1.0, 0.0), sum = make_double2(0.0, 0.0);
  double prev = 1e300;
  for (int j = 0; j < 200; ++j) {
    const double mag = fabs(term.x) + fabs(term.y);
    if (mag > prev) break;
    sum = cadd<double>(sum, term);
    if (mag < 1e-18 * (fabs(sum.x) + fabs(sum.y))) break;
    prev = mag;
    const double f = (s + j) * x;          // term *= (s + j) * (i x)
    term = make_double2(-f * term.y, f * term.x);
  }
  const double2 a = cmul<double>(eipz, sum);
  return make_double2(-a.y * zs / p, a.x * zs / p);   // (i/p) a zs
}

__device__ double2 khat_asymptotic(double c, double k, double R) {
  const double d = c * c - k * k;
  const double2 inf = d > 0 ? make_double2(1.0 / sqrt(d), 0.0) : make_double2(0.0, 1.0 / sqrt(-d));
  const double Z = c * R;
  const double pp = 1.0 + k / c, pm = k / c - 1.0;
  double sp, cp, sm, cm;
  sincos(pp * Z, &sp, &cp);
  sincos(pm * Z, &sm, &cm);
  const double2 ep = make_double2(cp, sp), em = make_double2(cm, sm);
  const double r2 = 0.70710678118654752440;
  const double2 e4 = make_double2(r2, -r2), e4c = make_double2(r2, r2);   // e^{-i pi/4}, e^{+i pi/4}
  const double zinv = 1.0 / Z;
  double zs = 1.0 / sqrt(Z);               // Z^{-m-1/2}
  double2 T = make_double2(0.0, 0.0);
  double2 mi = make_double2(1.0, 0.0), pi_ = make_double2(1.0, 0.0);   // (-i)^m, i^m
  for (int m = 0; m < KHAT_NB; ++m) {
    const double s = m + 0.5;
    const double2 fp = khat_f_series(s, pp, Z, ep, zs);
    const double2 fm = khat_f_series(s, pm, Z, em, zs);
    const double2 t = cscale<double>(cadd<double>(cmul<double>(cmul<double>(mi, e4), fp),
                                                  cmul<double>(cmul<double>(pi_, e4c), fm)),
                                     c_hank_b[m]);
    T = cadd<double>(T, t);
    if (m >= 2 && fabs(t.x) + fabs(t.y) < 1e-18 * (fabs(T.x) + fabs(T.y))) break;
    zs *= zinv;
    mi = make_double2(mi.y, -mi.x);        // *= -i
    pi_ = make_double2(-pi_.y, pi_.x);     // *= i
  }
  T = cscale<double>(T, 0.5 * sqrt(2.0 / M_PI) / c);
  return cscale<double>(csub<double>(inf, T), 0.5);
}

__device__ __forceinline__ bool khat_use_asym(double c, double k, double R) {
  return c * R >= KHAT_ASYM_CR && fabs(c - fabs(k)) * R >= KHAT_ASYM_GAP;
}

// one thread per entry of the quarter box; entries outside the asymptotic
// range are left to the quadrature kernel
__global__ void k_khat_asym(double2* __restrict__ raw, double2* __restrict__ s64,
                            float2* __restrict__ s32, int hx, int hy, double Lx, double Ly,
                            double kappa0, double R, double scale) {
  const long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (e >= (long long)hx * hy) return;
  const int j1 = (int)(e / hy), j2 = (int)(e - (long long)j1 * hy);
  const double r1 = j1 / Lx, r2 = j2 / Ly;
  const double c = 2.0 * M_PI * sqrt(r1 * r1 + r2 * r2);
  if (!khat_use_asym(c, kappa0, R)) return;
  const double2 v = khat_asymptotic(c, kappa0, R);
  raw[(size_t)j1 * hy + j2] = v;
  const size_t o = (size_t)j2 * hx + j1;
  s64[o] = make_double2(v.x * scale, v.y * scale);
  s32[o] = make_float2((float)(v.x * scale), (float)(v.y * scale));
}

__global__ void k_khat(double2* __restrict__ raw, double2* __restrict__ s64, float2* __restrict__ s32,
                       int hx, int hy, double Lx, double Ly, double kappa0, double R, double scale,
                       int scheme) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= hx * hy) return;
  const int j1 = warp / hy, j2 = warp - j1 * hy;
  const double r1 = j1 / Lx, r2 = j2 / Ly;
  const double rho = sqrt(r1 * r1 + r2 * r2);
  const double c = 2.0 * M_PI * rho;
  if (scheme == CAVITY_KHAT_QUADRATURE && khat_use_asym(c, kappa0, R)) return;  // k_khat_asym
  if (scheme == CAVITY_KHAT_PAPER && c * R > KHAT_PAPER_CR) {
    if (lane == 0) {
      const double2 v = khat_paper_tail(c, kappa0, R);
      raw[(size_t)j1 * hy + j2] = v;
      const size_t o = (size_t)j2 * hx + j1;
      s64[o] = make_double2(v.x * scale, v.y * scale);
      s32[o] = make_float2((float)(v.x * scale), (float)(v.y * scale));
    }
    return;
  }
  const double omega = c + fabs(kappa0);
  int npan = (int)ceil(omega * R / M_PI);
  if (npan < 1) npan = 1;
  const double width = R / npan;
  double sr = 0.0, si = 0.0;
  for (int pn = lane; pn < npan; pn += 32) {
    const double r0 = pn * width;
    double pr = 0.0, pi_ = 0.0;
#pragma unroll
    for (int k = 0; k < GLN; ++k) {
      const double r = r0 + 0.5 * width * (c_gl_x[k] + 1.0);
      double s, co;
      sincos(kappa0 * r, &s, &co);
      const double jv = bessel_j0(c * r) * c_gl_w[k];
      pr += jv * co;
      pi_ += jv * s;
    }
    sr += 0.5 * width * pr;
    si += 0.5 * width * pi_;
  }
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, off);
    si += __shfl_xor_sync(0xffffffffu, si, off);
  }
  if (lane == 0) {
    double2 v = make_double2(0.5 * sr, 0.5 * si);
    raw[(size_t)j1 * hy + j2] = v;
    // scaled copies are stored transposed, [j2][j1]: the operator reads them
    // along j1 for fixed j2
    const size_t o = (size_t)j2 * hx + j1;
    s64[o] = make_double2(v.x * scale, v.y * scale);
    s32[o] = make_float2((float)(v.x * scale), (float)(v.y * scale));
  }
}

cavity_status launch_khat(cavity_ctx* ctx, double kappa0) {
  const Geo& g = ctx->g;
  static bool gl_done = false;
  if (!gl_done) {
    std::vector<double> x, w;
    gauss_legendre(GLN, x, w);
    CK(cudaMemcpyToSymbol(c_gl_x, x.data(), sizeof(double) * GLN));
    CK(cudaMemcpyToSymbol(c_gl_w, w.data(), sizeof(double) * GLN));
    double b[KHAT_NB];
    b[0] = 1.0;
    for (int m = 1; m < KHAT_NB; ++m) b[m] = b[m - 1] * (double)((2 * m - 1) * (2 * m - 1)) / (8.0 * m);
    CK(cudaMemcpyToSymbol(c_hank_b, b, sizeof(double) * KHAT_NB));
    gl_done = true;
  }
  const int hx = g.Px / 2, hy = g.Py / 2;
  size_t n = (size_t)hx * hy;
  if (!ctx->khat64) {
    CK(cudaMalloc(&ctx->khat64, sizeof(double2) * n));
    CK(cudaMalloc(&ctx->khat32, sizeof(float2) * n));
    CK(cudaMalloc(&ctx->khat_raw, sizeof(double2) * n));
  }
  const long long threads = (long long)n * 32;
  {
    KScope ks_(ctx, KC_SETUP);
    k_khat<<<(unsigned)((threads + 255) / 256), 256, 0, ctx->stream>>>(
        ctx->khat_raw, ctx->khat64, ctx->khat32, hx, hy, g.Lx, g.Ly, kappa0, g.R,
        1.0 / (g.Lx * g.Ly), ctx->desc.khat_scheme);
  }
  if (ctx->desc.khat_scheme == CAVITY_KHAT_QUADRATURE) {
    KScope ks_(ctx, KC_SETUP);
    k_khat_asym<<<(unsigned)((n + 127) / 128), 128, 0, ctx->stream>>>(
        ctx->khat_raw, ctx->khat64, ctx->khat32, hx, hy, g.Lx, g.Ly, kappa0, g.R,
        1.0 / (g.Lx * g.Ly));
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}
