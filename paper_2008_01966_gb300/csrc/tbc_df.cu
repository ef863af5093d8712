// The aperture operator in pair-of-FP32 arithmetic (df64.cuh): the residual
// operator of the mixed-precision solve.  Same passes as the FP64 and FP32
// operators (tbc_apply.cuh), instantiated for the pair type; FP64 vectors in
// and out, converted at the boundary.
#include "df64.cuh"
#include "tbc_apply.cuh"

template <> struct Tabs<df> {
  static const cdf* tw(cavity_ctx* c) { return (const cdf*)c->tw_p; }
  static const cdf* ex(cavity_ctx* c, int k) { return (const cdf*)c->ehat_xp[k]; }
  static const cdf* ey(cavity_ctx* c, int k) { return (const cdf*)c->ehat_yp[k]; }
  static const cdf* kh(cavity_ctx* c) { return (const cdf*)c->khat_p; }
  static const cdf* top(cavity_ctx* c) { return (const cdf*)c->top_p; }
};

// the pass kernels of the pair type are compiled in tbc_df_k*.cu (in
// parallel: one unit with all sizes took three minutes)
TBC_PASS_KERNELS(extern, df, 2)
TBC_PASS_KERNELS(extern, df, 3)
TBC_PASS_KERNELS(extern, df, 4)
TBC_PASS_KERNELS(extern, df, 5)
TBC_PASS_KERNELS(extern, df, 6)
TBC_PASS_KERNELS(extern, df, 7)
TBC_PASS_KERNELS(extern, df, 8)
TBC_PASS_KERNELS(extern, df, 9)
TBC_PASS_KERNELS(extern, df, 10)

template cavity_status launch_apply<df>(cavity_ctx*, int, const cdf*, cdf*, void*, long long);

__global__ void k_to_pair(const double2* __restrict__ a, cdf* __restrict__ b, long long n) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = to_cdf(a[k]);
}
__global__ void k_from_pair(const cdf* __restrict__ a, double2* __restrict__ b, long long n) {
  const long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = to_d2(a[k]);
}

static cavity_status to_pair(cavity_ctx* ctx, const double2* a, void** dst, long long n) {
  if (!*dst) CK(cudaMalloc(dst, sizeof(cdf) * n));
  KScope ks_(ctx, KC_SETUP);
  k_to_pair<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(a, (cdf*)*dst, n);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// pair copies of the twiddle and basis-kernel tables (once per context) and
// of the kernel table and top relations (every prepare)
cavity_status launch_pair_tables(cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  if (!ctx->tw_p) {
    CKS(to_pair(ctx, ctx->tw64, &ctx->tw_p, ctx->TW));
    for (int k = 0; k < 2; ++k) {
      CKS(to_pair(ctx, ctx->ehat_x64[k], &ctx->ehat_xp[k], 2LL * g.Px));
      CKS(to_pair(ctx, ctx->ehat_y64[k], &ctx->ehat_yp[k], 2LL * g.Py));
    }
  }
  CKS(to_pair(ctx, ctx->khat64, &ctx->khat_p, (long long)(g.Px / 2) * (g.Py / 2)));
  CKS(to_pair(ctx, ctx->top64, &ctx->top_p, (long long)g.nap + g.n1 + g.n2));
  return CAVITY_OK;
}

size_t apply_pair_work_bytes(const Geo& g, int ndir) {
  const size_t v = ((sizeof(cdf) * (size_t)ndir * g.nap + 255) / 256) * 256;
  return apply_work_bytes(g, ndir, sizeof(cdf)) + 2 * v;
}

cavity_status launch_apply_pair(cavity_ctx* ctx, int ndir, const double2* x, double2* y,
                                void* work) {
  if (!ctx->g.fft_ok) {
    ctx->err = "the FFT operator needs the convolution period 4 on both axes";
    return CAVITY_EINVAL;
  }
  const Geo& g = ctx->g;
  const long long n = (long long)ndir * g.nap;
  const size_t v = ((sizeof(cdf) * (size_t)n + 255) / 256) * 256;
  cdf* xp = (cdf*)work;
  cdf* yp = (cdf*)((char*)work + v);
  void* w = (char*)work + 2 * v;
  {
    KScope ks_(ctx, KC_COMBP);
    k_to_pair<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(x, xp, n);
  }
  CKS(launch_apply<df>(ctx, ndir, xp, yp, w));
  {
    KScope ks_(ctx, KC_COMBP);
    k_from_pair<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(yp, y, n);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}
