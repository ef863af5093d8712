// Right-hand side of (EJ1)/(uT1) (row 2 of the design table, "forward
// transform of the excitation") and the backscatter RCS.
//
// RHS: g1 = (h/q) 2i(alpha1 p3 + beta p1) g~1, g2 = (h/c) 2i(alpha2 p3 + beta p2) g~2
// (c1mn and Appendix A), where g~ are the Galerkin tests (nosig) of the plane
// wave exp(i(alpha1 x1 + alpha2 x2)) taken with the trapezoid rule on the
// aperture nodes.  The test integral is separable, so per direction four 1-D
// sums  sum_p w_p {cos,sin}(m pi p/Nx) exp(i alpha1 x1_p)  (and the x2
// counterparts) are formed and multiplied out.
//
// RCS: L = int_Gamma (z x E) exp(-i kappa0 x_hat . y) dy with the exact 1-D
// integrals of cos/sin(m pi y/a) exp(-i g y), then
// sigma = (kappa0^2/pi) |e . (x_hat x L)|^2 (derived from (EGa2)).
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

struct DirPar {
  double a1, a2, A1r, A1i, A2r, A2i;  // alpha1, alpha2, 2i(alpha1 p3 + beta p1), 2i(...)
};

// incident wave of Sec. 7: d = -(sin t cos f, sin t sin f, cos t), q = kappa0 d,
// p = cos(alpha) theta_hat + sin(alpha) phi_hat
static DirPar dir_params(double kappa0, double t, double f, double al) {
  double st = std::sin(t), ct = std::cos(t), sf = std::sin(f), cf = std::cos(f);
  double a1 = -kappa0 * st * cf, a2 = -kappa0 * st * sf, beta = kappa0 * ct;
  double th[3] = {ct * cf, ct * sf, -st}, ph[3] = {-sf, cf, 0.0};
  double p[3];
  for (int k = 0; k < 3; ++k) p[k] = std::cos(al) * th[k] + std::sin(al) * ph[k];
  DirPar d;
  d.a1 = a1;
  d.a2 = a2;
  double s1 = a1 * p[2] + beta * p[0], s2 = a2 * p[2] + beta * p[1];
  d.A1r = 0.0; d.A1i = 2.0 * s1;
  d.A2r = 0.0; d.A2i = 2.0 * s2;
  return d;
}

// fac layout per direction: [cx (nx) | sx (nx) | cy (ny+1) | sy (ny+1)]
// cx[m] = sum_p w_p cos(m pi p/nx) e^{i a1 x_p}, m = 0..nx-1;  sx[m] likewise
// with sin (index m, m = 1..nx-1 used); cy, sy over n = 0..ny.
// With cos = (e^{+} + e^{-})/2 both reduce to the trapezoid sum of a geometric
// progression, in closed form:
//   T(th) = 1/2 + z + ... + z^{N-1} + z^N/2 = (i/2) cot(th/2) (1 - z^N),  z = e^{i th},
//   th = (alpha side +- pi m)/N,  z^N = (-1)^m e^{i alpha side};
// where |sin(th/2)| < 1e-3 the progression is summed term by term instead
// (the closed form would cancel there).
__device__ double2 trap_progression(double th, int N, double2 zN) {
  double s, c;
  sincos(0.5 * th, &s, &c);
  if (fabs(s) < 1e-3) {
    double sr = 0, si = 0;
    for (int p = 0; p <= N; ++p) {
      const double w = (p == 0 || p == N) ? 0.5 : 1.0;
      double es, ec;
      sincos(th * p, &es, &ec);
      sr += w * ec;
      si += w * es;
    }
    return make_double2(sr, si);
  }
  const double ct = 0.5 * c / s;
  return make_double2(ct * zN.y, ct * (1.0 - zN.x));
}

__global__ void k_rhs_factors(const DirPar* __restrict__ dp, double2* __restrict__ fac, int nx,
                              int ny, double a, double b) {
  const int d = blockIdx.y, which = blockIdx.z;
  const int per = 2 * nx + 2 * (ny + 1);
  const bool xdir = which < 2;
  const int nint = xdir ? nx : ny;
  const int count = xdir ? nx : ny + 1;
  const double side = xdir ? a : b;
  const double al = xdir ? dp[d].a1 : dp[d].a2;
  const bool isc = (which == 0 || which == 2);
  const int off = which == 0 ? 0 : which == 1 ? nx : which == 2 ? 2 * nx : 2 * nx + ny + 1;
  double es, ec;
  sincos(al * side, &es, &ec);
  const double w = side / nint;
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < count; m += gridDim.x * blockDim.x) {
    const double sg = (m & 1) ? -1.0 : 1.0;
    const double2 zN = make_double2(sg * ec, sg * es);
    const double2 gp = trap_progression((al * side + M_PI * m) / nint, nint, zN);
    const double2 gm = trap_progression((al * side - M_PI * m) / nint, nint, zN);
    double2 r;
    if (isc) r = make_double2(0.5 * w * (gp.x + gm.x), 0.5 * w * (gp.y + gm.y));
    else r = make_double2(0.5 * w * (gp.y - gm.y), -0.5 * w * (gp.x - gm.x));
    fac[(size_t)d * per + off + m] = r;
  }
}

__global__ void k_rhs_assemble(const DirPar* __restrict__ dp, const double2* __restrict__ fac,
                               double2* __restrict__ out, int nx, int ny, int n1, int n2, int nap,
                               int ndir, double a, double b, double h) {
  long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gid >= (long long)ndir * nap) return;
  const int d = (int)(gid / nap), i = (int)(gid - (long long)d * nap);
  const int N = ny - 1;
  const int per = 2 * nx + 2 * (ny + 1);
  const double2* f = fac + (size_t)d * per;
  const double2* cx = f;
  const double2* sx = f + nx;
  const double2* cy = f + 2 * nx;
  const double2* sy = f + 2 * nx + ny + 1;
  const double ab = a * b;
  double2 r = make_double2(0, 0);
  if (i < n1) {
    int m = i / N, n = i - m * N + 1;
    double2 g = cmul<double>(cx[m], sy[n]);
    double s = h / (m == 0 ? ab / 2 : ab / 4);
    r = cscale<double>(cmul<double>(make_double2(dp[d].A1r, dp[d].A1i), g), s);
  } else if (i < n1 + n2) {
    int ii = i - n1;
    int m = ii / (N + 1) + 1, n = ii - (m - 1) * (N + 1);
    double2 g = cmul<double>(sx[m], cy[n]);
    double s = h / (n == 0 ? ab / 2 : ab / 4);
    r = cscale<double>(cmul<double>(make_double2(dp[d].A2r, dp[d].A2i), g), s);
  }
  out[gid] = r;
}

cavity_status launch_rhs(cavity_ctx* ctx, int ndir, const double* theta, const double* phi,
                         const double* alpha, double2* out) {
  const Geo& g = ctx->g;
  std::vector<DirPar> hp(ndir);
  for (int d = 0; d < ndir; ++d) hp[d] = dir_params(ctx->kappa0, theta[d], phi[d], alpha[d]);
  const int per = 2 * g.nx + 2 * (g.ny + 1);
  size_t need = sizeof(DirPar) * ndir + sizeof(double2) * (size_t)per * ndir + 256;
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, need));
  DirPar* dp = (DirPar*)ctx->ws2;
  double2* fac = (double2*)((char*)ctx->ws2 + ((sizeof(DirPar) * ndir + 255) / 256) * 256);
  CK(cudaMemcpyAsync(dp, hp.data(), sizeof(DirPar) * ndir, cudaMemcpyHostToDevice, ctx->stream));
  int bx = (std::max(g.nx, g.ny + 1) + 127) / 128;
  {
    KScope ks_(ctx, KC_RHS);
    k_rhs_factors<<<dim3(bx, ndir, 4), 128, 0, ctx->stream>>>(dp, fac, g.nx, g.ny, g.a, g.b);
  }
  long long tot = (long long)ndir * g.nap;
  {
    KScope ks_(ctx, KC_RHS);
    k_rhs_assemble<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(
        dp, fac, out, g.nx, g.ny, g.n1, g.n2, g.nap, ndir, g.a, g.b, g.h);
  }
  CK(cudaGetLastError());
  // the host parameter array must outlive the copy
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

// ------------------------------------------------------------------ RCS
// int_0^side exp(-i s y) dy = side exp(-i s side/2) sinc(s side/2)
__device__ __forceinline__ double2 ef(double s, double side) {
  double x = 0.5 * s * side;
  double sc = fabs(x) < 1e-8 ? 1.0 - x * x / 6.0 : sin(x) / x;
  double ss, cc;
  sincos(-x, &ss, &cc);
  return make_double2(side * sc * cc, side * sc * ss);
}

struct ObsPar {
  double g1, g2;        // kappa0 x_hat1, kappa0 x_hat2
  double xh[3], e[3];   // x_hat and the polarisation vector
};

__global__ void k_rcs(const double2* __restrict__ ap, const ObsPar* __restrict__ op,
                      double* __restrict__ sigma, int nx, int ny, int n1, int n2, int nap,
                      double a, double b, double kappa0) {
  extern __shared__ double2 sm_f[];
  const int d = blockIdx.x;
  const int N = ny - 1;
  double2* C1x = sm_f;             // m = 0..M
  double2* S2x = C1x + nx;         // m = 1..M (index m)
  double2* S1y = S2x + nx;         // n = 1..N (index n)
  double2* C2y = S1y + ny;         // n = 0..N
  const ObsPar o = op[d];
  for (int m = threadIdx.x; m < nx; m += blockDim.x) {
    double k = m * M_PI / a;
    double2 fm = ef(o.g1 - k, a), fp = ef(o.g1 + k, a);
    C1x[m] = make_double2(0.5 * (fm.x + fp.x), 0.5 * (fm.y + fp.y));
    double2 df = make_double2(fm.x - fp.x, fm.y - fp.y);   // /(2i)
    S2x[m] = make_double2(0.5 * df.y, -0.5 * df.x);
  }
  for (int n = threadIdx.x; n < ny; n += blockDim.x) {
    double k = n * M_PI / b;
    double2 fm = ef(o.g2 - k, b), fp = ef(o.g2 + k, b);
    C2y[n] = make_double2(0.5 * (fm.x + fp.x), 0.5 * (fm.y + fp.y));
    double2 df = make_double2(fm.x - fp.x, fm.y - fp.y);
    S1y[n] = make_double2(0.5 * df.y, -0.5 * df.x);
  }
  __syncthreads();
  const double2* E = ap + (size_t)d * nap;
  double2 L1 = make_double2(0, 0), L2 = make_double2(0, 0);   // int E1, int E2
  for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
    if (i < n1) {
      int m = i / N, n = i - m * N + 1;
      L1 = cadd<double>(L1, cmul<double>(E[i], cmul<double>(C1x[m], S1y[n])));
    } else {
      int ii = i - n1;
      int m = ii / (N + 1) + 1, n = ii - (m - 1) * (N + 1);
      L2 = cadd<double>(L2, cmul<double>(E[i], cmul<double>(S2x[m], C2y[n])));
    }
  }
  __shared__ double2 red1[32], red2[32];
  for (int off = 16; off > 0; off >>= 1) {
    L1.x += __shfl_xor_sync(0xffffffffu, L1.x, off);
    L1.y += __shfl_xor_sync(0xffffffffu, L1.y, off);
    L2.x += __shfl_xor_sync(0xffffffffu, L2.x, off);
    L2.y += __shfl_xor_sync(0xffffffffu, L2.y, off);
  }
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { red1[wid] = L1; red2[wid] = L2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 s1 = make_double2(0, 0), s2 = make_double2(0, 0);
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      s1 = cadd<double>(s1, red1[w]);
      s2 = cadd<double>(s2, red2[w]);
    }
    // L = (-int E2, int E1, 0)
    double2 L[3] = {make_double2(-s2.x, -s2.y), s1, make_double2(0, 0)};
    // v = e . (x_hat x L)
    double2 cr[3];
    for (int k = 0; k < 3; ++k) {
      int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
      cr[k] = csub<double>(cscale<double>(L[k2], o.xh[k1]), cscale<double>(L[k1], o.xh[k2]));
    }
    double2 v = make_double2(0, 0);
    for (int k = 0; k < 3; ++k) v = cadd<double>(v, cscale<double>(cr[k], o.e[k]));
    sigma[d] = kappa0 * kappa0 / M_PI * cabs2<double>(v);
  }
}

cavity_status launch_rcs(cavity_ctx* ctx, int ndir, const double2* ap, const double* th,
                         const double* ph, int pol, double* sigma) {
  const Geo& g = ctx->g;
  std::vector<ObsPar> hp(ndir);
  for (int d = 0; d < ndir; ++d) {
    double st = std::sin(th[d]), ct = std::cos(th[d]), sf = std::sin(ph[d]), cf = std::cos(ph[d]);
    ObsPar& o = hp[d];
    o.xh[0] = st * cf; o.xh[1] = st * sf; o.xh[2] = ct;
    o.g1 = ctx->kappa0 * o.xh[0];
    o.g2 = ctx->kappa0 * o.xh[1];
    if (pol == CAVITY_POL_THETA) { o.e[0] = ct * cf; o.e[1] = ct * sf; o.e[2] = -st; }
    else { o.e[0] = -sf; o.e[1] = cf; o.e[2] = 0.0; }
  }
  size_t need = sizeof(ObsPar) * ndir + sizeof(double) * ndir + 512;
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, need));
  ObsPar* op = (ObsPar*)ctx->ws2;
  double* sg = (double*)((char*)ctx->ws2 + ((sizeof(ObsPar) * ndir + 255) / 256) * 256);
  CK(cudaMemcpyAsync(op, hp.data(), sizeof(ObsPar) * ndir, cudaMemcpyHostToDevice, ctx->stream));
  size_t sm = sizeof(double2) * (2 * g.nx + 2 * g.ny);
  CK(allow_max_smem(k_rcs));
  {
    KScope ks_(ctx, KC_RHS);
    k_rcs<<<ndir, 256, sm, ctx->stream>>>(ap, op, sg, g.nx, g.ny, g.n1, g.n2, g.nap, g.a, g.b,
                                          ctx->kappa0);
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(sigma, sg, sizeof(double) * ndir, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}
