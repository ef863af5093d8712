// Block-diagonal preconditioner of the aperture system (EJ1)/(uT1).
//
// The coefficients E1^{mn}, E2^{mn}, E3^{mn} of one mode (m, n) are coupled
// by the cavity part (row 3 and the E3 columns of rows 1, 2) and by the
// diagonal entries of the three TBC integrals I1, I2, I3 of Sec. 5.1.  Those
// diagonals are evaluated exactly under the same discrete rule as the
// operator itself:
//     I^{mn}_{mn} = sum_{j1, j2} Ax(m, j1) F(G)(j1, j2) Ay(n, j2) / (Lx Ly),
//     Ax(m, j1) = X(m, j1) Phi(j1, m),
// with X the trapezoid projection of the torus Fourier mode exp(2 pi i j1 x/Lx)
// onto cos/sin(m pi x/a) and Phi the exact basis transform of Sec. 5.2.  The
// 3x3 blocks (2x2 / 1x1 where a component is absent) are inverted once per
// (kappa0, eps) and applied as a right preconditioner in GMRES.  Only the
// iteration count depends on it, never the solution.
#include "common.cuh"

// Ax[kind][m][j], j in FFT order over the box (Nyquist slot zero)
__global__ void k_pc_ax(double2* __restrict__ out, int nint, int Pn, double side, int pad,
                        const double2* __restrict__ tw, int TW) {
  const int kind = blockIdx.z;  // 0 cos, 1 sin
  const int m = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Pn; j += gridDim.x * blockDim.x) {
    double2 r = make_double2(0, 0);
    if (j != Pn / 2 && !(kind == 1 && m == 0)) {
      const long long j1 = j < Pn / 2 ? j : j - Pn;
      double2 X = make_double2(0, 0);
      for (int p = 0; p <= nint; ++p) {
        double w = side / nint;
        if (p == 0 || p == nint) w *= 0.5;
        double2 t = tw_at(tw, TW, (long long)m * p, 2 * nint);    // exp(-i pi m p / nint)
        double tr = kind == 0 ? t.x : -t.y;
        double2 e = cconj<double>(tw_at(tw, TW, j1 * p, Pn));      // exp(2 pi i j1 p / Pn)
        X = cadd<double>(X, cscale<double>(e, w * tr));
      }
      const long long sh = (long long)(pad / 2) * m;
      double2 em = eps_d(j1 - sh, side, pad), ep = eps_d(j1 + sh, side, pad);
      double2 phi;
      if (kind == 0) phi = make_double2(0.5 * (em.x + ep.x), 0.5 * (em.y + ep.y));
      else phi = make_double2(0.5 * (em.y - ep.y), -0.5 * (em.x - ep.x));   // /(2i)
      r = cmul<double>(X, phi);
    }
    out[((size_t)kind * nint + m) * Pn + j] = r;
  }
}

// T[xk][m][j2a] = sum_j Ax[xk][m][j] khat(|j1|, j2a)   (khat stored [j2a][j1a])
__global__ void k_pc_t(const double2* __restrict__ ax, const double2* __restrict__ kh,
                       double2* __restrict__ out, int nx, int Px, int hy) {
  const int xk = blockIdx.z, m = blockIdx.y;
  const int j2a = blockIdx.x * blockDim.x + threadIdx.x;
  if (j2a >= hy) return;
  const double2* a = ax + ((size_t)xk * nx + m) * Px;
  double2 s = make_double2(0, 0);
  for (int j = 0; j < Px; ++j) {
    if (j == Px / 2) continue;
    int j1a = j < Px / 2 ? j : Px - j;
    s = cadd<double>(s, cmul<double>(a[j], kh[(size_t)j2a * (Px / 2) + j1a]));
  }
  out[((size_t)xk * nx + m) * hy + j2a] = s;
}

// d[f][m][n] = sum_j2 T[xk][m][|j2|] Ay[yk][n][j2];  f: 0 cs, 1 sc, 2 cc
__global__ void k_pc_d(const double2* __restrict__ T, const double2* __restrict__ ay,
                       double2* __restrict__ dout, int nx, int ny, int Py) {
  const int f = blockIdx.z;
  const int xk = (f == 1) ? 1 : 0, yk = (f == 0) ? 1 : 0;
  const int m = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n > ny) return;
  const int hy = Py / 2;
  const double2* t = T + ((size_t)xk * nx + m) * hy;
  double2 s = make_double2(0, 0);
  if (n < ny) {
    const double2* a = ay + ((size_t)yk * ny + n) * Py;
    for (int j = 0; j < Py; ++j) {
      if (j == Py / 2) continue;
      int j2a = j < Py / 2 ? j : Py - j;
      s = cadd<double>(s, cmul<double>(t[j2a], a[j]));
    }
  }
  dout[((size_t)f * nx + m) * (ny + 1) + n] = s;
}

__device__ void inv3(double2 A[3][3], double2 Bi[3][3]) {
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) Bi[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  for (int k = 0; k < 3; ++k) {
    int piv = k;
    double best = cabs2<double>(A[k][k]);
    for (int r = k + 1; r < 3; ++r)
      if (cabs2<double>(A[r][k]) > best) { best = cabs2<double>(A[r][k]); piv = r; }
    if (piv != k)
      for (int c = 0; c < 3; ++c) {
        double2 t = A[k][c]; A[k][c] = A[piv][c]; A[piv][c] = t;
        t = Bi[k][c]; Bi[k][c] = Bi[piv][c]; Bi[piv][c] = t;
      }
    double2 inv = cdiv<double>(make_double2(1, 0), A[k][k]);
    for (int c = 0; c < 3; ++c) { A[k][c] = cmul<double>(A[k][c], inv); Bi[k][c] = cmul<double>(Bi[k][c], inv); }
    for (int r = 0; r < 3; ++r) {
      if (r == k) continue;
      double2 f = A[r][k];
      for (int c = 0; c < 3; ++c) {
        A[r][c] = csub<double>(A[r][c], cmul<double>(f, A[k][c]));
        Bi[r][c] = csub<double>(Bi[r][c], cmul<double>(f, Bi[k][c]));
      }
    }
  }
}

__global__ void k_pc_blocks(const double2* __restrict__ dd, const double2* __restrict__ top,
                            double2* __restrict__ pinv, float2* __restrict__ pinv32, int nx, int ny,
                            int n1, int n2, int nap, double a, double b, double h, double k2) {
  const int m = blockIdx.y;
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= ny) return;
  const int N = ny - 1;
  const double2* d1 = dd + ((size_t)0 * nx + m) * (ny + 1);
  const double2* d2 = dd + ((size_t)1 * nx + m) * (ny + 1);
  const double2* d3 = dd + ((size_t)2 * nx + m) * (ny + 1);
  const double mx = m * M_PI / a, nyv = n * M_PI / b;
  const double ab = a * b;
  const double sq = h / (m == 0 ? ab / 2 : ab / 4), sc = h / (n == 0 ? ab / 2 : ab / 4);
  double2 A[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) A[r][c] = make_double2(r == c ? 1.0 : 0.0, 0.0);
  const bool has1 = n >= 1, has2 = m >= 1, has3 = m >= 1 && n >= 1;
  const int i1 = m * N + (n - 1), i2 = n1 + (m - 1) * (N + 1) + n;
  const int i3 = n1 + n2 + (m - 1) * N + (n - 1);
  if (has1) {
    double2 tb = csub<double>(cscale<double>(d1[n], k2), cscale<double>(d3[n], 2 * nyv * nyv));
    A[0][0] = cadd<double>(make_double2(-1.0 + top[i1].x, top[i1].y), cscale<double>(tb, sq));
  }
  if (has2) {
    double2 tb = csub<double>(cscale<double>(d2[n], k2), cscale<double>(d3[n], 2 * mx * mx));
    A[1][1] = cadd<double>(make_double2(-1.0 + top[i2].x, top[i2].y), cscale<double>(tb, sc));
  }
  if (has3) {
    A[0][1] = cscale<double>(d3[n], sq * 2 * nyv * mx);
    A[0][2] = make_double2(mx * h + top[nap + i1].x, top[nap + i1].y);
    A[1][0] = cscale<double>(d3[n], sc * 2 * mx * nyv);
    A[1][2] = make_double2(nyv * h + top[nap + i2].x, top[nap + i2].y);
    A[2][0] = make_double2(mx * h, 0);
    A[2][1] = make_double2(nyv * h, 0);
    A[2][2] = make_double2(-1.0 + top[i3].x, top[i3].y);
  }
  double2 Bi[3][3];
  inv3(A, Bi);
  double2* o = pinv + ((size_t)m * ny + n) * 9;
  float2* o32 = pinv32 + ((size_t)m * ny + n) * 9;
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      o[r * 3 + c] = Bi[r][c];
      o32[r * 3 + c] = make_float2((float)Bi[r][c].x, (float)Bi[r][c].y);
    }
}

cavity_status launch_precond(cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  const int hy = g.Py / 2;
  size_t nax = (size_t)2 * g.nx * g.Px, nay = (size_t)2 * g.ny * g.Py;
  size_t nT = (size_t)2 * g.nx * hy, nd = (size_t)3 * g.nx * (g.ny + 1);
  size_t need = sizeof(double2) * (nax + nay + nT + nd);
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, need));
  double2* ax = (double2*)ctx->ws2;
  double2* ay = ax + nax;
  double2* T = ay + nay;
  double2* dd = T + nT;
  if (!ctx->pinv64) {
    CK(cudaMalloc(&ctx->pinv64, sizeof(double2) * 9 * (size_t)g.nx * g.ny));
    CK(cudaMalloc(&ctx->pinv32, sizeof(float2) * 9 * (size_t)g.nx * g.ny));
  }
  cudaStream_t st = ctx->stream;
  {
    KScope ks_(ctx, KC_SETUP);
    k_pc_ax<<<dim3((g.Px + 255) / 256, g.nx, 2), 256, 0, st>>>(ax, g.nx, g.Px, g.a, g.padx, ctx->tw64,
                                                               ctx->TW);
  }
  {
    KScope ks_(ctx, KC_SETUP);
    k_pc_ax<<<dim3((g.Py + 255) / 256, g.ny, 2), 256, 0, st>>>(ay, g.ny, g.Py, g.b, g.pady, ctx->tw64,
                                                               ctx->TW);
  }
  {
    KScope ks_(ctx, KC_SETUP);
    k_pc_t<<<dim3((hy + 127) / 128, g.nx, 2), 128, 0, st>>>(ax, ctx->khat64, T, g.nx, g.Px, hy);
  }
  {
    KScope ks_(ctx, KC_SETUP);
    k_pc_d<<<dim3((g.ny + 1 + 127) / 128, g.nx, 3), 128, 0, st>>>(T, ay, dd, g.nx, g.ny, g.Py);
  }
  {
    KScope ks_(ctx, KC_SETUP);
    k_pc_blocks<<<dim3((g.ny + 127) / 128, g.nx), 128, 0, st>>>(
        dd, ctx->top64, ctx->pinv64, ctx->pinv32, g.nx, g.ny, g.n1, g.n2, g.nap, g.a, g.b, g.h,
        2.0 * ctx->kappa0 * ctx->kappa0);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// y = (block diagonal)^{-1} x for ndir vectors
template <typename T>
__global__ void k_pc_apply(const C<T>* __restrict__ x, long long xs, C<T>* __restrict__ y,
                           long long ys, const C<T>* __restrict__ pinv, int nx, int ny, int n1,
                           int n2, int nap, int ndir) {
  long long gid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long per = (long long)nx * ny;
  if (gid >= per * ndir) return;
  const int d = (int)(gid / per);
  const int mn = (int)(gid - (long long)d * per);
  const int lny = __ffs(ny) - 1;                 // ny is a power of two
  const int m = mn >> lny, n = mn & (ny - 1);
  const int N = ny - 1;
  const bool has1 = n >= 1, has2 = m >= 1, has3 = m >= 1 && n >= 1;
  const int i1 = m * N + (n - 1), i2 = n1 + (m - 1) * (N + 1) + n;
  const int i3 = n1 + n2 + (m - 1) * N + (n - 1);
  const C<T>* xd = x + (size_t)d * xs;
  C<T>* yd = y + (size_t)d * ys;
  C<T> v[3] = {mk<T>(0, 0), mk<T>(0, 0), mk<T>(0, 0)};
  if (has1) v[0] = xd[i1];
  if (has2) v[1] = xd[i2];
  if (has3) v[2] = xd[i3];
  const C<T>* B = pinv + (size_t)mn * 9;
  C<T> r[3];
  for (int a = 0; a < 3; ++a) {
    r[a] = cmul<T>(B[a * 3 + 0], v[0]);
    r[a] = cadd<T>(r[a], cmul<T>(B[a * 3 + 1], v[1]));
    r[a] = cadd<T>(r[a], cmul<T>(B[a * 3 + 2], v[2]));
  }
  if (has1) yd[i1] = r[0];
  if (has2) yd[i2] = r[1];
  if (has3) yd[i3] = r[2];
}

template <typename T>
cavity_status launch_precond_apply(cavity_ctx* ctx, int ndir, const C<T>* x, C<T>* y,
                                   long long xs, long long ys) {
  if (xs < 0) xs = ctx->g.nap;
  if (ys < 0) ys = ctx->g.nap;
  const Geo& g = ctx->g;
  const C<T>* pinv;
  if (sizeof(T) == 8) pinv = (const C<T>*)ctx->pinv64;
  else pinv = (const C<T>*)ctx->pinv32;
  long long tot = (long long)g.nx * g.ny * ndir;
  {
    KScope ks_(ctx, KC_PRECOND);
    k_pc_apply<T><<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(x, xs, y, ys, pinv, g.nx,
        g.ny, g.n1, g.n2, g.nap, ndir);
  }
  CK(cudaGetLastError());
  // two-level variant (FP32 inner solves of the mixed path): the coarse
  // unknowns take the exact solve of the coarse block instead
  if constexpr (std::is_same<T, float>::value) CKS(coarse_correct(ctx, ndir, x, xs, y, ys));
  return CAVITY_OK;
}

template cavity_status launch_precond_apply<double>(cavity_ctx*, int, const double2*, double2*,
                                                    long long, long long);
template cavity_status launch_precond_apply<float>(cavity_ctx*, int, const float2*, float2*,
                                                   long long, long long);
