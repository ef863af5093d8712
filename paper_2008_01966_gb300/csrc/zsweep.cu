// Per-mode elimination in x3 (Algorithm I/II, Step 2), one thread per mode.
//
// The tridiagonal systems (dfE1M)/(dfE3M) -- and in a layered fill the
// interface rows of Sec. 4, repeated at every interface as the remark closing
// Sec. 4 describes -- are eliminated bottom-up without pivoting.  What is
// carried is the ratio rho_{j+1} = E_j / E_{j+1}, i.e. -1 over the running
// pivot of the LU factorisation (LU1)/(LU2), so the last one is the
// -1/r_JJ of (EJJ1).  Determinants (det U4 in d_l of Sec. 4) are never formed:
// products of bounded ratios underflow to the correct zero for evanescent
// modes instead of overflowing.
//
//  tangential E1 / E2 (T_0 = 0): rho_1 = 0, eta_1 = 0
//    ordinary level j of layer l:  rho_{j+1} = 1/(2 - sigma_l - rho_j),
//                                  eta_{j+1} = rho_{j+1} eta_j
//    interface level j (from (con42-2) and the (con51) analogue):
//                                  rho_{j+1} = 1/(2 - rho_j),
//      eta_{j+1} = rho_{j+1} (eta_j - mu h (1 - eps_U/eps_D) P3_j)
//    so that T_j = rho_{j+1} T_{j+1} + eta_{j+1} E3_ap; P3_j is the E3
//    profile (upper value) of the same mode at the interface.
//  E3 (Neumann bottom E_{3,0} = E_{3,1}): rho_1 = 1
//    ordinary level: as above;
//    interface level j ((con32), (con61)): rho_{j+1} = U_j / E_{j+1}
//                                        = 1/(1 + (eps_U/eps_D)(1 - rho_j)).
//  Top-down: P_nz = 1, P_j = rho_{j+1} P_{j+1} (times eps_U/eps_D when level
//  j+1 is an interface, since the lower value there is (eps_U/eps_D) U);
//  Q_nz = 0, Q_j = rho_{j+1} Q_{j+1} + eta_{j+1}.
//  Top relations: tau = rho_nz = P_{nz-1}, varsigma = eta_nz = Q_{nz-1}.
//
// Storage: the profiles are written level-major, prof[(j-1) * nap + i] for
// j = 1..nz-1, so that consecutive threads (modes) write consecutive words; the
// bottom-up pass stores rho_{j+1} in level j's slot and the top-down pass
// overwrites it with P_j.
#include "common.cuh"

#define MAXL 16
struct LayerTab {
  int nl;
  int top[MAXL];     // level index of the upper boundary of layer l (top to bottom)
  int bot[MAXL];     // level index of the lower boundary
  double er[MAXL], ei[MAXL];
};

struct ZP {
  int nz, M, N, n1, n2, nap;
  double a, b, h, k2;  // k2 = kappa0^2
  double pivtol;
};

__device__ __forceinline__ int layer_of(const LayerTab& L, int j) {
  // interior levels of layer l are (bot, top); returns -1 for interface levels
  for (int l = 0; l < L.nl; ++l)
    if (j > L.bot[l] && j < L.top[l]) return l;
  return -1;
}

// mode i of the aperture ordering -> component (0,1,2) and (m, n)
__device__ __forceinline__ void mode_of(const ZP& p, int i, int& comp, int& m, int& n) {
  if (i < p.n1) {
    comp = 0; m = i / p.N; n = i - m * p.N + 1;
  } else if (i < p.n1 + p.n2) {
    int ii = i - p.n1;
    comp = 1; m = ii / (p.N + 1) + 1; n = ii - (m - 1) * (p.N + 1);
  } else {
    int ii = i - p.n1 - p.n2;
    comp = 2; m = ii / p.N + 1; n = ii - (m - 1) * p.N + 1;
  }
}

__device__ __forceinline__ void atomic_min_pos(double* addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMin((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// pass 1: E3 modes (or all modes when `all` is set: homogeneous fill)
// pass 2: tangential modes of a layered fill, reading P3 at the interfaces
__global__ void k_zsweep(ZP p, LayerTab L, double2* __restrict__ prof, double2* __restrict__ profq,
                         double2* __restrict__ top, double* minpiv, int pass) {
  const int nmodes = (pass == 1) ? p.nap : (p.n1 + p.n2);
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmodes) return;
  int i = t;
  int comp, m, n;
  if (pass == 1 && L.nl > 1) {
    // layered pass 1 handles only E3 modes
    i = t + p.n1 + p.n2;
    if (i >= p.nap) return;
  }
  mode_of(p, i, comp, m, n);
  const double lam = (m * M_PI / p.a) * (m * M_PI / p.a) + (n * M_PI / p.b) * (n * M_PI / p.b);
  const double h2 = p.h * p.h;
  const bool e3 = (comp == 2);
  const bool layered = L.nl > 1;
  double mu = 0.0;
  if (comp == 0) mu = m * M_PI / p.a;
  if (comp == 1) mu = n * M_PI / p.b;
  const int e3i = (m >= 1 && n >= 1) ? p.n1 + p.n2 + (m - 1) * p.N + (n - 1) : -1;
  const bool src = layered && !e3 && mu != 0.0 && e3i >= 0;
  const int nqs = p.n1 + p.n2;

  double2 rho = make_double2(e3 ? 1.0 : 0.0, 0.0);
  double2 eta = make_double2(0.0, 0.0);
  double worst = 1e300;
  for (int j = 1; j < p.nz; ++j) {
    int l = layer_of(L, j);
    double2 piv;
    if (l >= 0) {
      double2 sig = make_double2(h2 * (p.k2 * L.er[l] - lam), h2 * (p.k2 * L.ei[l]));
      piv = make_double2(2.0 - sig.x - rho.x, -sig.y - rho.y);
      double sc = fmax(1.0, sqrt(cabs2<double>(make_double2(sig.x - 2.0, sig.y))));
      worst = fmin(worst, sqrt(cabs2<double>(piv)) / sc);
    } else {
      // interface level between layer lu (above) and ld (below)
      int lu = -1, ld = -1;
      for (int q = 0; q < L.nl; ++q) {
        if (L.bot[q] == j) lu = q;
        if (L.top[q] == j) ld = q;
      }
      if (e3) {
        double2 ratio = cdiv<double>(make_double2(L.er[lu], L.ei[lu]), make_double2(L.er[ld], L.ei[ld]));
        double2 om = make_double2(1.0 - rho.x, -rho.y);
        double2 pr = cmul<double>(ratio, om);
        piv = make_double2(1.0 + pr.x, pr.y);
      } else {
        piv = make_double2(2.0 - rho.x, -rho.y);
        if (src) {
          double2 ratio = cdiv<double>(make_double2(L.er[lu], L.ei[lu]), make_double2(L.er[ld], L.ei[ld]));
          double2 cf = make_double2(mu * p.h * (1.0 - ratio.x), -mu * p.h * ratio.y);
          double2 p3 = prof[(size_t)(j - 1) * p.nap + e3i];
          eta = csub<double>(eta, cmul<double>(cf, p3));
        }
      }
      worst = fmin(worst, sqrt(cabs2<double>(piv)));
    }
    rho = cdiv<double>(make_double2(1.0, 0.0), piv);
    eta = cmul<double>(rho, eta);
    prof[(size_t)(j - 1) * p.nap + i] = rho;
    if (src) profq[(size_t)(j - 1) * nqs + i] = eta;
  }
  // top-down
  double2 P = make_double2(1.0, 0.0), Q = make_double2(0.0, 0.0);
  for (int j = p.nz - 1; j >= 1; --j) {
    double2 r = prof[(size_t)(j - 1) * p.nap + i];
    // factor eps_U/eps_D when level j+1 is an interface (E3 only)
    double2 f = make_double2(1.0, 0.0);
    if (e3 && j + 1 < p.nz && layer_of(L, j + 1) < 0) {
      int lu = -1, ld = -1;
      for (int q = 0; q < L.nl; ++q) {
        if (L.bot[q] == j + 1) lu = q;
        if (L.top[q] == j + 1) ld = q;
      }
      f = cdiv<double>(make_double2(L.er[lu], L.ei[lu]), make_double2(L.er[ld], L.ei[ld]));
    }
    if (src) {
      double2 e = profq[(size_t)(j - 1) * nqs + i];
      Q = cadd<double>(cmul<double>(r, Q), e);
      profq[(size_t)(j - 1) * nqs + i] = Q;
    } else if (!e3 && layered) {
      profq[(size_t)(j - 1) * nqs + i] = make_double2(0.0, 0.0);
    }
    P = cmul<double>(cmul<double>(r, P), f);
    prof[(size_t)(j - 1) * p.nap + i] = P;
    if (j == p.nz - 1) {
      top[i] = P;
      if (!e3) top[p.nap + i] = src ? Q : make_double2(0.0, 0.0);
    }
  }
  atomic_min_pos(minpiv, worst);
}

__global__ void k_f32_copy(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

cavity_status launch_zsweep(cavity_ctx* ctx, double kappa0) {
  const Geo& g = ctx->g;
  if ((int)ctx->layers.size() > MAXL) {
    ctx->err = "at most 16 layers are supported";
    return CAVITY_EINVAL;
  }
  ZP p;
  p.nz = g.nz; p.M = g.M; p.N = g.N; p.n1 = g.n1; p.n2 = g.n2; p.nap = g.nap;
  p.a = g.a; p.b = g.b; p.h = g.h; p.k2 = kappa0 * kappa0;
  p.pivtol = ctx->desc.pivot_tol;
  LayerTab L;
  L.nl = (int)ctx->layers.size();
  int topl = g.nz;
  for (int l = 0; l < L.nl; ++l) {
    L.top[l] = topl;
    L.bot[l] = topl - ctx->layers[l].nlev;
    L.er[l] = ctx->layers[l].eps_re;
    L.ei[l] = ctx->layers[l].eps_im;
    topl = L.bot[l];
  }
  size_t nprof = (size_t)(g.nz - 1) * g.nap;
  size_t nq = (size_t)(g.nz - 1) * (g.n1 + g.n2);
  // FP32 copies of the profiles for the complex64 field of mixed contexts:
  // records for the fused kernel where it runs, else plain copies
  const bool mixed = ctx->desc.precision == CAVITY_MIXED;
  const bool recs = mixed && field_fused_use(ctx);
  const bool plain32 = mixed && !recs;
  if (!ctx->prof) CK(cudaMalloc(&ctx->prof, sizeof(double2) * nprof));
  if (plain32 && !ctx->prof32) CK(cudaMalloc(&ctx->prof32, sizeof(float2) * nprof));
  if (!ctx->top64) CK(cudaMalloc(&ctx->top64, sizeof(double2) * (g.nap + g.n1 + g.n2)));
  if (!ctx->top32) CK(cudaMalloc(&ctx->top32, sizeof(float2) * (g.nap + g.n1 + g.n2)));
  if (!ctx->minpiv) CK(cudaMalloc(&ctx->minpiv, sizeof(double)));
  const bool layered = L.nl > 1;
  if (layered && !ctx->profq) CK(cudaMalloc(&ctx->profq, sizeof(double2) * nq));
  if (plain32 && layered && !ctx->profq32) CK(cudaMalloc(&ctx->profq32, sizeof(float2) * nq));
  double big = 1e300;
  CK(cudaMemcpyAsync(ctx->minpiv, &big, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemsetAsync(ctx->top64, 0, sizeof(double2) * (g.nap + g.n1 + g.n2), ctx->stream));
  if (!layered) {
    {
      KScope ks_(ctx, KC_SETUP);
      k_zsweep<<<(g.nap + 127) / 128, 128, 0, ctx->stream>>>(p, L, ctx->prof, ctx->profq,
                                                            ctx->top64, ctx->minpiv, 1);
    }
  } else {
    {
      KScope ks_(ctx, KC_SETUP);
      k_zsweep<<<(g.n3 + 127) / 128, 128, 0, ctx->stream>>>(p, L, ctx->prof, ctx->profq,
                                                           ctx->top64, ctx->minpiv, 1);
    }
    {
      KScope ks_(ctx, KC_SETUP);
      k_zsweep<<<(g.n1 + g.n2 + 127) / 128, 128, 0, ctx->stream>>>(p, L, ctx->prof, ctx->profq,
                                                                   ctx->top64, ctx->minpiv, 2);
    }
  }
  CK(cudaGetLastError());
  if (plain32) {
    KScope ks_(ctx, KC_SETUP);
    k_f32_copy<<<(unsigned)((nprof + 255) / 256), 256, 0, ctx->stream>>>(ctx->prof, ctx->prof32,
                                                                       (long long)nprof);
  }
  if (recs) CKS(launch_prof_records(ctx));
  long long ntop = g.nap + g.n1 + g.n2;
  {
    KScope ks_(ctx, KC_SETUP);
    k_f32_copy<<<(unsigned)((ntop + 255) / 256), 256, 0, ctx->stream>>>(ctx->top64, ctx->top32, ntop);
  }
  if (plain32 && layered) {
    KScope ks_(ctx, KC_SETUP);
    k_f32_copy<<<(unsigned)((nq + 255) / 256), 256, 0, ctx->stream>>>(ctx->profq, ctx->profq32,
                                                                    (long long)nq);
  }
  CK(cudaGetLastError());
  double worst = 0;
  CK(cudaMemcpyAsync(&worst, ctx->minpiv, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (!(worst > ctx->desc.pivot_tol)) {
    ctx->err = "a per-mode pivot vanished (|pivot| = " + std::to_string(worst) +
               "): kappa0 is a discrete cavity resonance";
    return CAVITY_ESINGULAR;
  }
  return CAVITY_OK;
}
