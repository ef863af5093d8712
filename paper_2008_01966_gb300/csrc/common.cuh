// Internal definitions shared by the CUDA translation units of the cavity
// solver: complex arithmetic, the context with its resident device state, and
// error plumbing.  Nothing here is part of the public ABI (include/cavity.h).
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "../../include/cavity.h"

// ------------------------------------------------------------ complex numbers
template <typename T> struct cplx_t;
template <> struct cplx_t<double> { typedef double2 type; };
template <> struct cplx_t<float> { typedef float2 type; };

template <typename T> using C = typename cplx_t<T>::type;

template <typename T> __host__ __device__ __forceinline__ C<T> mk(T x, T y) {
  C<T> r; r.x = x; r.y = y; return r;
}
template <typename T> __host__ __device__ __forceinline__ C<T> cadd(C<T> a, C<T> b) {
  return mk<T>(a.x + b.x, a.y + b.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> csub(C<T> a, C<T> b) {
  return mk<T>(a.x - b.x, a.y - b.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cconj(C<T> a) {
  return mk<T>(a.x, -a.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> cscale(C<T> a, T s) {
  return mk<T>(a.x * s, a.y * s);
}
// multiply by +i
template <typename T> __host__ __device__ __forceinline__ C<T> cmul_i(C<T> a) {
  return mk<T>(-a.y, a.x);
}
// a / b
template <typename T> __host__ __device__ __forceinline__ C<T> cdiv(C<T> a, C<T> b) {
  // scaled division (Smith) keeps the range for large |b|
  T ar = b.x < 0 ? -b.x : b.x, ai = b.y < 0 ? -b.y : b.y;
  if (ar >= ai) {
    T r = b.y / b.x, d = b.x + b.y * r;
    return mk<T>((a.x + a.y * r) / d, (a.y - a.x * r) / d);
  } else {
    T r = b.x / b.y, d = b.y + b.x * r;
    return mk<T>((a.x * r + a.y) / d, (a.y * r - a.x) / d);
  }
}
template <typename T> __host__ __device__ __forceinline__ T cabs2(C<T> a) {
  return a.x * a.x + a.y * a.y;
}
__host__ __device__ __forceinline__ float2 to_f(double2 a) {
  return make_float2((float)a.x, (float)a.y);
}
__host__ __device__ __forceinline__ double2 to_d(float2 a) {
  return make_double2((double)a.x, (double)a.y);
}
template <typename T> __host__ __device__ __forceinline__ C<T> conv(double2 a);
template <> __host__ __device__ __forceinline__ double2 conv<double>(double2 a) { return a; }
template <> __host__ __device__ __forceinline__ float2 conv<float>(double2 a) { return to_f(a); }

// ------------------------------------------------------------ geometry
struct Geo {
  double a, b, c, h;
  int nx, ny, nz, M, N;
  int n1, n2, n3, nap;     // sizes of the aperture blocks (Appendix A)
  int padx, pady, Px, Py;  // TBC torus: Px = padx*nx points, period Lx = padx*a (y alike)
  bool fft_ok;             // padx = pady = 4: the FFT operator's layout (else dense solver only)
  double Lx, Ly, R;        // R = sqrt(2) max(a,b): truncation of the kernel
  int lnx, lny, lPx, lPy;  // log2 of nx, ny, Px, Py
  long long field_per_level, field_per_dir;
};

// kernel classes for launch counting and event timing (cavity_timing_read)
enum KClass {
  KC_TBC_A64, KC_TBC_B64, KC_TBC_C64, KC_TBC_D64, KC_COMB64,
  KC_TBC_A32, KC_TBC_B32, KC_TBC_C32, KC_TBC_D32, KC_COMB32,
  KC_KRYLOV, KC_PRECOND, KC_FIELD_Y, KC_FIELD_X, KC_RHS, KC_SETUP,
  KC_TBC_AP, KC_TBC_BP, KC_TBC_CP, KC_TBC_DP, KC_COMBP,
  KC_DENSE_ASM, KC_DENSE_LU, KC_DENSE_TRS, KC_N
};

// one layer of the fill, top to bottom
struct LayerDev {
  int nlev;
  double eps_re, eps_im;
};

// kept block of the aperture system: the modes m <= mm, n <= nn
struct KeptSet {
  int mm, nn, n1, n2, n3, nk;
};

// FP32 LU factors of a kept block (row-major, leading dimension lda), the row
// permutation, the inverted 64 x 64 diagonal blocks of L and U, the map from
// kept (compact) to full unknown indices, and a work area for its solves
struct DenseLU {
  KeptSet ks{};
  int n = 0, lda = 0;
  bool ready = false;
  float2* a = nullptr;
  double2* a64 = nullptr;   // the block in FP64 (residuals of the refinement), or null
  float2* dinv = nullptr;
  int* ipiv = nullptr;
  int* perm = nullptr;
  int* map = nullptr;
  void* work = nullptr;
  size_t work_bytes = 0;
};

// The resident device state of one context.
struct cavity_ctx {
  Geo g;
  cavity_desc desc;
  cudaStream_t stream;
  int device;
  std::string err;

  // twiddle table exp(-2 pi i k / TW), k < TW, TW = max transform length
  int TW;
  double2* tw64 = nullptr;
  float2* tw32 = nullptr;
  // FFT of the 1-D Cauchy-type kernel of the basis transform (Sec. 5.2 F(F)):
  // length 2*Px (x) and 2*Py (y), for cos ('c') and sin ('s') kinds, with the
  // convolution scale folded in
  double2 *ehat_x64[2] = {nullptr, nullptr}, *ehat_y64[2] = {nullptr, nullptr};
  float2 *ehat_x32[2] = {nullptr, nullptr}, *ehat_y32[2] = {nullptr, nullptr};
  // the same tables in pair-of-FP32 form (struct cdf, 16 bytes per entry) for
  // the residual operator of the mixed solve
  void* tw_p = nullptr;
  void *ehat_xp[2] = {nullptr, nullptr}, *ehat_yp[2] = {nullptr, nullptr};

  // ---- state of the last prepare (kappa0, layers)
  bool prepared = false;
  double kappa0 = 0;
  std::vector<LayerDev> layers;
  double2* khat64 = nullptr;   // quarter box [j2][j1] (Py/2 x Px/2), scaled by 1/(Lx Ly)
  float2* khat32 = nullptr;
  double2* khat_raw = nullptr; // unscaled copy [j1][j2] for export
  double2* prof = nullptr;     // (nz-1) x nap profiles P, level-major
  double2* profq = nullptr;    // (nz-1) x (n1+n2) profiles Q (layered only)
  double2* top64 = nullptr;    // nap tau, then n1+n2 varsigma
  float2* top32 = nullptr;
  void* khat_p = nullptr;      // pair-of-FP32 copies of khat64 and top64
  void* top_p = nullptr;
  double2* pinv64 = nullptr;   // (M+1)(N+1) x 9 inverse diagonal blocks
  float2* pinv32 = nullptr;
  float2* prof32 = nullptr;    // FP32 copies of the profiles for the mixed field path
  float2* profq32 = nullptr;
  // FP32 profiles of the fused field kernel as one record per (level, m, n)
  // on the full nx x ny mode grid: {P1, P2}, {P3, Q1}, {Q2, 0} (layered, 3
  // float4) or {P1, P2}, {P3, 0} (homogeneous, 2 float4); entries outside a
  // component's index set are 0 (field_fused.cu)
  float4* prof_rec = nullptr;
  int prof_rec_w = 0;
  double* minpiv = nullptr;    // device scalar: min |pivot| / scale

  // ---- workspaces (grown on demand)
  size_t ws_bytes = 0;
  void* ws = nullptr;
  size_t ws2_bytes = 0;
  void* ws2 = nullptr;
  size_t stage_bytes = 0;   // device staging of cavity_solve (right-hand sides,
  void* stage = nullptr;    // and outputs that go to host memory)
  size_t pin_bytes = 0;     // pinned host staging of the block Krylov
  void* pin = nullptr;      // coefficient matrices (asynchronous copies)
  cudaStream_t copy_stream = nullptr;   // device-to-host copies of host outputs,
  std::vector<cudaEvent_t> copy_evs;    // overlapped with the field synthesis
  cudaStream_t copy_more[3] = {nullptr, nullptr, nullptr};  // further copy engines
  cudaEvent_t copy_join[3] = {nullptr, nullptr, nullptr};

  // ---- dense LU factors of a kept block: the direct solver's (kept set of
  // modes_m, modes_n; aperture_solver == CAVITY_SOLVER_DENSE) and the coarse
  // level of the two-level preconditioner (modes m, n <= CAVITY_OPT_COARSE_MODES)
  DenseLU dn, cs;
  void* dn_scr = nullptr;     // LU scratch (pivot candidates, barrier counters)
  size_t dn_scr_bytes = 0;

  // ---- implementation options (cavity_set_option)
  int opt[CAVITY_NUM_OPT] = {0, 0, 16, 0, 0};

  // ---- launch accounting: counts always, CUDA-event times while timing is on
  long long nlaunch[KC_N] = {0};
  bool timing = false;
  struct Ev { int cls; cudaEvent_t a, b; };
  std::vector<Ev> evs;
  std::vector<cudaEvent_t> evpool;
  double ms[KC_N] = {0};
};

// Counts one launch of class `cls`; with timing on, brackets it with events on
// the context's stream.  Use as  { KScope k_(ctx, KC_...); kernel<<<...>>>(...); }
struct KScope {
  cavity_ctx* c;
  int cls;
  cudaEvent_t a = nullptr;
  static cudaEvent_t get(cavity_ctx* c) {
    cudaEvent_t e;
    if (!c->evpool.empty()) {
      e = c->evpool.back();
      c->evpool.pop_back();
    } else {
      cudaEventCreate(&e);
    }
    return e;
  }
  KScope(cavity_ctx* c_, int k) : c(c_), cls(k) {
    c->nlaunch[k]++;
    if (c->timing) {
      a = get(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~KScope() {
    if (c->timing) {
      cudaEvent_t b = get(c);
      cudaEventRecord(b, c->stream);
      c->evs.push_back({cls, a, b});
    }
  }
};

// ------------------------------------------------------------ errors
#define CK(call)                                                                 \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      ctx->err = std::string(#call) + ": " + cudaGetErrorString(e_);             \
      return CAVITY_ECUDA;                                                       \
    }                                                                            \
  } while (0)

#define CKS(...)                                                                 \
  do {                                                                           \
    cavity_status s_ = (__VA_ARGS__);                                            \
    if (s_ != CAVITY_OK) return s_;                                              \
  } while (0)

inline int ilog2(int n) {
  int l = 0;
  while ((1 << l) < n) ++l;
  return l;
}

// opt-in shared memory limit of the current device (bytes)
inline int smem_optin() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return v > 0 ? v : 48 * 1024;
}

// allow `func` the device's opt-in dynamic shared memory (minus its static part)
template <typename F> inline cudaError_t allow_max_smem(F func) {
  cudaFuncAttributes a;
  cudaError_t e = cudaFuncGetAttributes(&a, func);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              smem_optin() - (int)a.sharedSizeBytes);
}

// grow the pinned host staging to at least `bytes`
inline cavity_status ensure_pin(cavity_ctx* ctx, size_t bytes) {
  if (ctx->pin_bytes >= bytes) return CAVITY_OK;
  if (ctx->pin) cudaFreeHost(ctx->pin);
  ctx->pin = nullptr;
  ctx->pin_bytes = 0;
  cudaError_t e = cudaMallocHost(&ctx->pin, bytes);
  if (e != cudaSuccess) {
    ctx->pin = nullptr;
    ctx->err = "pinned staging allocation of " + std::to_string(bytes) + " bytes failed: " +
               cudaGetErrorString(e);
    return CAVITY_ENOMEM;
  }
  ctx->pin_bytes = bytes;
  return CAVITY_OK;
}

// grow a workspace to at least `bytes`
inline cavity_status ensure_ws(cavity_ctx* ctx, void** p, size_t* have, size_t bytes) {
  if (*have >= bytes) return CAVITY_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    *p = nullptr;
    ctx->err = "workspace allocation of " + std::to_string(bytes) + " bytes failed: " +
               cudaGetErrorString(e);
    return CAVITY_ENOMEM;
  }
  *have = bytes;
  return CAVITY_OK;
}

// ------------------------------------------------------------ step launchers
// (defined in the individual .cu files)
cavity_status launch_twiddles(cavity_ctx* ctx);
cavity_status launch_ehat(cavity_ctx* ctx);
cavity_status launch_khat(cavity_ctx* ctx, double kappa0);
cavity_status launch_zsweep(cavity_ctx* ctx, double kappa0);
cavity_status launch_precond(cavity_ctx* ctx);
cavity_status launch_rhs(cavity_ctx* ctx, int ndir, const double* theta,
                         const double* phi, const double* alpha, double2* out);
// y = A x; direction d of y starts at y + d * ystride (ystride < 0: n_ap)
template <typename T>
cavity_status launch_apply(cavity_ctx* ctx, int ndir, const C<T>* x, C<T>* y, void* work,
                           long long ystride = -1);
size_t apply_work_bytes(const Geo& g, int ndir, int elem_bytes);
// y = A x in pair-of-FP32 arithmetic (~1e-12), FP64 vectors in and out;
// work: apply_pair_work_bytes
cavity_status launch_apply_pair(cavity_ctx* ctx, int ndir, const double2* x, double2* y,
                                void* work);
size_t apply_pair_work_bytes(const Geo& g, int ndir);
cavity_status launch_pair_tables(cavity_ctx* ctx);
// y = M^{-1} x with per-direction strides (< 0: n_ap)
template <typename T>
cavity_status launch_precond_apply(cavity_ctx* ctx, int ndir, const C<T>* x, C<T>* y,
                                   long long xs = -1, long long ys = -1);
cavity_status run_gmres64(cavity_ctx* ctx, int ndir, const double2* b, double2* x,
                          int* iters, double* resid);
cavity_status run_mixed_solve(cavity_ctx* ctx, int ndir, const double2* b, double2* x,
                              int* iters, double* resid);
// FP32 block GMRES for the inner solves of the mixed refinement (bgmres.cu):
// solves A M^{-1} y = r_d for the directions with active[d], d = M^{-1} y.
cavity_status run_block_inner(cavity_ctx* ctx, int ndir, const float2* r, float2* d,
                              const std::vector<double>& tol, const std::vector<char>& active,
                              int mb, int maxit, void* work, std::vector<int>& iters,
                              std::vector<double>& est);
size_t block_inner_work_bytes(const Geo& g, int ndir, int mb, int gw);
// zero the aperture unknowns outside the truncated mode set (modes_m, modes_n
// of the descriptor; no-op without truncation), ndir contiguous FP64 vectors
cavity_status launch_mode_mask(cavity_ctx* ctx, int ndir, double2* v);
// host_out (optional): a host buffer of the field's layout; each chunk of
// levels is copied there on ctx->copy_stream as soon as it is written (the
// caller joins the copy stream)
template <typename T>
cavity_status launch_field(cavity_ctx* ctx, int ndir, const double2* ap, C<T>* out,
                           void* host_out = nullptr);
// the fused field kernel (field_fused.cu): the grids it covers, and the
// per-(level, m, n) FP32 profile records it reads, built from the FP64
// profiles at prepare
bool field_fused_supported(const Geo& g);
// whether this context's complex64 field takes the fused kernel
// (CAVITY_OPT_FIELD_FUSED; fixed at prepare, with the profile layout)
bool field_fused_use(const cavity_ctx* ctx);
cavity_status launch_prof_records(cavity_ctx* ctx);
// the copy stream and at least n events for it (created once per context)
inline cavity_status ensure_copy_stream(cavity_ctx* ctx, size_t n) {
  if (!ctx->copy_stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      ctx->copy_stream = nullptr;
      ctx->err = cudaGetErrorString(e);
      return CAVITY_ECUDA;
    }
  }
  for (int k = 0; k < 3; ++k) {
    if (ctx->copy_more[k]) continue;
    if (cudaStreamCreateWithFlags(&ctx->copy_more[k], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->copy_join[k], cudaEventDisableTiming) != cudaSuccess) {
      ctx->err = "copy stream creation failed";
      return CAVITY_ECUDA;
    }
  }
  while (ctx->copy_evs.size() < n) {
    cudaEvent_t ev;
    cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      ctx->err = cudaGetErrorString(e);
      return CAVITY_ECUDA;
    }
    ctx->copy_evs.push_back(ev);
  }
  return CAVITY_OK;
}
// dense path (dense.cu): the kept set, the FP32 kept block assembled from the
// per-axis factors of Sec. 5.2, its LU factors, and one inner solve of the
// refinement: x += s^-1 (LU)^-1 (s r) on the kept unknowns (s[d] per direction)
KeptSet kept_set(const cavity_desc& d, const Geo& g);
KeptSet kept_set_of(int mm, int nn);
cavity_status dense_assemble(cavity_ctx* ctx, const KeptSet& ks, float2* a, int lda);
// assemble and factor the kept block ks into f (kept resident until destroy)
cavity_status dense_factor(cavity_ctx* ctx, DenseLU& f, const KeptSet& ks, bool keep64 = false);
// r = b - A x on the kept rows of the solver's block in FP64 (ndir vectors of
// length n_ap; rows outside the kept set are not written)
cavity_status dense_residual(cavity_ctx* ctx, int ndir, const double2* b, const double2* x,
                             double2* r);
void dense_free(DenseLU& f);
// the coarse level of the mixed solver's preconditioner: factors it when
// CAVITY_OPT_COARSE_MODES > 0 and it is missing; y <- A_cc^{-1} x on the
// coarse unknowns of ndir FP32 vectors (other unknowns untouched)
cavity_status coarse_prepare(cavity_ctx* ctx);
cavity_status coarse_correct(cavity_ctx* ctx, int ndir, const float2* x, long long xs, float2* y,
                             long long ys);
cavity_status dense_lu(cavity_ctx* ctx, float2* a, int n, int lda, int* ipiv, int* info);
cavity_status dense_lu_solve(cavity_ctx* ctx, const float2* lu, int n, int lda, const int* ipiv,
                             const int* perm, int nrhs, float2* y, int ldy);
cavity_status launch_dense_factor(cavity_ctx* ctx);
size_t dense_inner_work_bytes(const cavity_ctx* ctx, int ndir);
// the barrier-timeout flag inside dense_inner_solve's work area (nonzero after
// the stream: a substitution gave up)
int* dense_inner_err(const cavity_ctx* ctx, int ndir, void* work);
cavity_status dense_inner_solve(cavity_ctx* ctx, int ndir, const double2* r, const double* s,
                                double2* x, void* work);
cavity_status run_dense_solve(cavity_ctx* ctx, int ndir, const double2* b, double2* x,
                              int* iters, double* resid);
cavity_status launch_rcs(cavity_ctx* ctx, int ndir, const double2* ap,
                         const double* th, const double* ph, int pol, double* sigma);

// exp(-2 pi i k / n) from the twiddle table tw of length TW (n divides TW)
static __device__ __forceinline__ double2 tw_at(const double2* __restrict__ tw, int TW, long long k,
                                                int n) {
  long long r = k % n;
  if (r < 0) r += n;
  return tw[r * (TW / n)];
}
// E(d / L) of the basis transform (Sec. 5.2) on the torus of period
// L = pad side: (1 - exp(-2 pi i d / pad)) L / (2 pi i d), and side at d = 0
// (pad = 4: exp(-2 pi i d / 4) = (-i)^d taken exactly)
static __device__ __forceinline__ double2 eps_d(long long d, double side, int pad = 4) {
  if (d == 0) return make_double2(side, 0.0);
  double2 num;
  if (pad == 4) {
    int r = (int)(((d % 4) + 4) % 4);
    if (r == 0) num = make_double2(0.0, 0.0);
    else if (r == 1) num = make_double2(1.0, 1.0);    // 1 - (-i)
    else if (r == 2) num = make_double2(2.0, 0.0);    // 1 - (-1)
    else num = make_double2(1.0, -1.0);               // 1 - i
  } else {
    double sn, cs;
    sincospi(-2.0 * (double)(d % pad) / (double)pad, &sn, &cs);
    num = make_double2(1.0 - cs, -sn);
  }
  double f = pad * side / (2.0 * M_PI * (double)d);
  return make_double2(num.y * f, -num.x * f);       // num / i * f
}

// Kernels whose line transforms have compile-time lengths are instantiated for
// log2 sizes LO..HI; dispatch_log calls f(std::integral_constant<int, v>).
template <int LO, int HI, typename F>
inline cavity_status dispatch_log(int v, F&& f) {
  if constexpr (LO > HI) {
    (void)v;
    return CAVITY_EINVAL;
  } else {
    if (v == LO) return f(std::integral_constant<int, LO>{});
    return dispatch_log<LO + 1, HI>(v, std::forward<F>(f));
  }
}
__host__ __device__ constexpr int clog2(int v) { return v <= 1 ? 0 : 1 + clog2(v >> 1); }
// log2 of the grid sizes nx, ny accepted by cavity_setup (4 .. 1024)
#define CAV_LOG_MIN 2
#define CAV_LOG_MAX 10
