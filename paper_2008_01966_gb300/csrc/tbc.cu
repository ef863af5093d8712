// Setup tables of the TBC operator, the FP64 instantiation of the aperture
// operator and its allocation-free entry point (the operator itself is in
// tbc_apply.cuh).
#include <algorithm>
#include <mutex>

#include "tbc_apply.cuh"

// the FP32 operator is instantiated in tbc_f32.cu
extern template cavity_status launch_apply<float>(cavity_ctx*, int, const float2*, float2*, void*,
                                                 long long);

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

// The 1-D kernel of F(F) on the frequency grid d/L (L = pad * side):
//   eps(d) = E(d/L) = int_0^side exp(-2 pi i (d/L) y) dy,  E(0) = side.
// The basis transform at frequency j only involves eps(j -/+ 2k) (the basis
// cos/sin(k pi y/side) has frequencies k/(2 side) = 2k/L), so the convolution
// splits by the parity r of j = 2t + r into two convolutions along t with the
// kernels eps_r(u) = eps(2u + r), u in [-P/2, P/2) (slot u = -P/2 is never
// reached and is set to 0).  Each is transformed with a length-P FFT; the
// convolution scale (1/2 for the cosine basis, 1/(2i) for the sine basis) and
// the 1/P of the inverse transform are folded in.  Output: out[r * P + t].
__global__ void k_ehat(double2* out64, float2* out32, int P, int lP, double side, int pad,
                       int kind, const double2* __restrict__ tw, int twlog) {
  extern __shared__ double2 sm_e[];
  const int r = blockIdx.x;
  double2* A = sm_e;
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    const int u = t < P / 2 ? t : t - P;
    const int d = 2 * u + r;
    double2 v;
    if (u == -P / 2) {
      v = make_double2(0.0, 0.0);
    } else if (d == 0) {
      v = make_double2(side, 0.0);
    } else {
      // (1 - exp(-2 pi i d / pad)) * L / (2 pi i d)
      double sn, cs;
      sincospi(-2.0 * (double)d / (double)pad, &sn, &cs);
      const double2 num = make_double2(1.0 - cs, -sn);
      const double f = pad * side / (2.0 * M_PI * (double)d);
      v = make_double2(num.y * f, -num.x * f);  // num / i
    }
    A[pidx(t)] = v;
  }
  __syncthreads();
  fft_inplace<double, false>(A, padded_len(P), P, lP, 1, tw, twlog);
  const double sc = 0.5 / (double)P;
  for (int t = threadIdx.x; t < P; t += blockDim.x) {
    const double2 v = A[pidx(t)];
    double2 o;
    if (kind == 0) o = make_double2(sc * v.x, sc * v.y);   // * 1/2
    else o = make_double2(sc * v.y, -sc * v.x);            // * 1/(2i)
    out64[r * P + t] = o;
    out32[r * P + t] = make_float2((float)o.x, (float)o.y);
  }
}

cavity_status launch_ehat(cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  int twlog = ilog2(ctx->TW);
  CK(allow_max_smem(k_ehat));
  for (int kind = 0; kind < 2; ++kind) {
    CK(cudaMalloc(&ctx->ehat_x64[kind], sizeof(double2) * 2 * g.Px));
    CK(cudaMalloc(&ctx->ehat_x32[kind], sizeof(float2) * 2 * g.Px));
    CK(cudaMalloc(&ctx->ehat_y64[kind], sizeof(double2) * 2 * g.Py));
    CK(cudaMalloc(&ctx->ehat_y32[kind], sizeof(float2) * 2 * g.Py));
    const size_t smx = sizeof(double2) * padded_len(g.Px), smy = sizeof(double2) * padded_len(g.Py);
    {
      KScope ks_(ctx, KC_SETUP);
      k_ehat<<<2, std::max(32, fft_tpl<double>(g.Px)), smx, ctx->stream>>>(
          ctx->ehat_x64[kind], ctx->ehat_x32[kind], g.Px, g.lPx, g.a, g.padx, kind, ctx->tw64, twlog);
    }
    {
      KScope ks_(ctx, KC_SETUP);
      k_ehat<<<2, std::max(32, fft_tpl<double>(g.Py)), smy, ctx->stream>>>(
          ctx->ehat_y64[kind], ctx->ehat_y32[kind], g.Py, g.lPy, g.b, g.pady, kind, ctx->tw64, twlog);
    }
    CK(cudaGetLastError());
  }
  return CAVITY_OK;
}

size_t apply_work_bytes(const Geo& g, int ndir, int eb) {
  size_t vy = (size_t)ndir * 3 * g.nx * g.Py;
  size_t w = (size_t)ndir * 3 * (g.nx + 1) * g.Py;
  size_t z = (size_t)ndir * 3 * (g.nx + 1) * (g.ny + 1);
  size_t o = (size_t)ndir * 3 * g.nx * (g.ny + 1);
  // Vy and Z share one region, W and O another; eb = bytes of one complex
  return (std::max(vy, z) + std::max(w, o)) * (size_t)eb;
}

template cavity_status launch_apply<double>(cavity_ctx*, int, const double2*, double2*, void*,
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

cavity_status launch_mode_mask(cavity_ctx* ctx, int ndir, double2* v) {
  return launch_mode_mask_t<double>(ctx, ndir, v, ctx->g.nap, KC_RHS);
}
