// C ABI of the cavity solver (include/cavity.h): argument checking, the
// resident state per (kappa0, layers), and the composition of the hot-path
// steps into cavity_solve.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

static thread_local std::string g_setup_err;

static bool pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }

extern "C" cavity_status cavity_setup(const cavity_desc* desc, void* cuda_stream, cavity_ctx** out) {
  if (!out) {
    g_setup_err = "out is NULL";
    return CAVITY_EINVAL;
  }
  *out = nullptr;
  if (!desc) {
    g_setup_err = "desc is NULL";
    return CAVITY_EINVAL;
  }
  const cavity_desc& d = *desc;
  auto bad = [&](const std::string& m) {
    g_setup_err = m;
    return CAVITY_EINVAL;
  };
  if (!(d.a > 0) || !(d.b > 0) || !(d.c > 0)) return bad("a, b, c must be positive");
  if (!pow2(d.nx) || !pow2(d.ny) || d.nx < 4 || d.ny < 4 || d.nx > 1024 || d.ny > 1024)
    return bad("nx, ny must be powers of two in [4, 1024]");
  if (d.nz < 2 || d.nz > 1 << 20) return bad("nz must be in [2, 2^20]");
  if (d.precision != CAVITY_FP64 && d.precision != CAVITY_MIXED) return bad("unknown precision");
  if (d.pad_factor != 0 && d.pad_factor != 4) return bad("pad_factor must be 0 or 4");
  // period of the TBC convolution per axis (Sec. 5.2): it must exceed the
  // side plus the kernel's truncation radius R; 4 sides where that suffices
  // (apertures up to about 2:1), else the next power of two (0 = automatic)
  const double R = std::sqrt(2.0) * std::max(d.a, d.b);
  auto period = [&](double side) {
    int p = 4;
    while (p <= 16 && !(p * side > side + R)) p *= 2;
    return p;
  };
  const int padx = period(d.a), pady = period(d.b);
  if (padx > 16 || pady > 16) return bad("aspect ratio too large (needs max/min < 11)");
  if (d.pad_factor == 4 && (padx != 4 || pady != 4))
    return bad("aspect ratio too large for the period 4*side (needs max/min < 2.12)");
  if (d.gmres_tol < 0 || d.gmres_restart < 0 || d.gmres_max_iter < 0 || d.pivot_tol < 0)
    return bad("negative solver parameter");
  if (d.gmres_restart > 120) return bad("gmres_restart must be at most 120");
  if (d.khat_scheme != CAVITY_KHAT_QUADRATURE && d.khat_scheme != CAVITY_KHAT_PAPER)
    return bad("khat_scheme must be CAVITY_KHAT_QUADRATURE or CAVITY_KHAT_PAPER");
  if (d.modes_m < 0 || d.modes_m > d.nx - 1 || d.modes_n < 0 || d.modes_n > d.ny - 1)
    return bad("modes_m, modes_n must be in [0, nx-1], [0, ny-1]");
  if (d.aperture_solver != CAVITY_SOLVER_KRYLOV && d.aperture_solver != CAVITY_SOLVER_DENSE)
    return bad("aperture_solver must be CAVITY_SOLVER_KRYLOV or CAVITY_SOLVER_DENSE");
  if (d.outer_rule != CAVITY_OUTER_TRAPEZOID && d.outer_rule != CAVITY_OUTER_PARSEVAL)
    return bad("outer_rule must be CAVITY_OUTER_TRAPEZOID or CAVITY_OUTER_PARSEVAL");
  if (d.outer_rule == CAVITY_OUTER_PARSEVAL && d.aperture_solver != CAVITY_SOLVER_DENSE)
    return bad("the Parseval outer rule is implemented by the dense solver only");
  if ((padx != 4 || pady != 4) && d.aperture_solver != CAVITY_SOLVER_DENSE)
    return bad("this aperture needs a convolution period of more than 4 sides (max/min >= "
               "2.12); the FFT operator has period 4, so use the dense solver");
  if (d.aperture_solver == CAVITY_SOLVER_DENSE) {
    const long long mm = d.modes_m > 0 ? d.modes_m : d.nx - 1, nn = d.modes_n > 0 ? d.modes_n : d.ny - 1;
    if (3 * mm * nn + mm + nn > CAVITY_DENSE_MAX_N)
      return bad("dense aperture solver: the kept block (3 mm nn + mm + nn unknowns) exceeds "
                 "CAVITY_DENSE_MAX_N; truncate with modes_m, modes_n");
  }
  cavity_ctx* ctx = new cavity_ctx();
  ctx->desc = d;
  if (ctx->desc.pad_factor == 0) ctx->desc.pad_factor = 4;
  if (ctx->desc.pivot_tol == 0) ctx->desc.pivot_tol = 1e-12;
  ctx->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&ctx->device);
  Geo& g = ctx->g;
  g.a = d.a; g.b = d.b; g.c = d.c; g.nx = d.nx; g.ny = d.ny; g.nz = d.nz;
  g.h = d.c / d.nz;
  g.M = d.nx - 1; g.N = d.ny - 1;
  g.n1 = (g.M + 1) * g.N; g.n2 = g.M * (g.N + 1); g.n3 = g.M * g.N;
  g.nap = g.n1 + g.n2 + g.n3;
  g.padx = padx; g.pady = pady;
  g.fft_ok = padx == 4 && pady == 4;
  g.Px = padx * d.nx; g.Py = pady * d.ny;
  g.Lx = padx * d.a; g.Ly = pady * d.b; g.R = R;
  g.lnx = ilog2(d.nx); g.lny = ilog2(d.ny); g.lPx = ilog2(g.Px); g.lPy = ilog2(g.Py);
  g.field_per_level = (long long)(d.nx + 1) * (d.ny - 1) + (long long)(d.nx - 1) * (d.ny + 1) +
                      (long long)(d.nx - 1) * (d.ny - 1);
  g.field_per_dir = g.field_per_level * d.nz;
  ctx->TW = 2 * std::max(g.Px, g.Py);
  cavity_status s = launch_twiddles(ctx);
  if (s == CAVITY_OK && g.fft_ok) s = launch_ehat(ctx);
  if (s == CAVITY_OK) {
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      ctx->err = cudaGetErrorString(e);
      s = CAVITY_ECUDA;
    }
  }
  if (s != CAVITY_OK) {
    g_setup_err = ctx->err;
    cavity_destroy(ctx);
    return s;
  }
  *out = ctx;
  return CAVITY_OK;
}

extern "C" void cavity_destroy(cavity_ctx* ctx) {
  if (!ctx) return;
  void* ptrs[] = {ctx->tw64, ctx->tw32, ctx->ehat_x64[0], ctx->ehat_x64[1], ctx->ehat_y64[0],
                  ctx->ehat_y64[1], ctx->ehat_x32[0], ctx->ehat_x32[1], ctx->ehat_y32[0],
                  ctx->ehat_y32[1], ctx->khat64, ctx->khat32, ctx->khat_raw, ctx->prof, ctx->profq,
                  ctx->top64, ctx->top32, ctx->pinv64, ctx->pinv32, ctx->prof32, ctx->profq32,
                  ctx->minpiv, ctx->ws, ctx->ws2, ctx->stage, ctx->tw_p, ctx->ehat_xp[0],
                  ctx->ehat_xp[1], ctx->ehat_yp[0], ctx->ehat_yp[1], ctx->khat_p, ctx->top_p, ctx->prof_rec,
                  ctx->dn_scr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  dense_free(ctx->dn);
  dense_free(ctx->cs);
  if (ctx->pin) cudaFreeHost(ctx->pin);
  for (auto e : ctx->copy_evs) cudaEventDestroy(e);
  if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
  for (int k = 0; k < 3; ++k) {
    if (ctx->copy_join[k]) cudaEventDestroy(ctx->copy_join[k]);
    if (ctx->copy_more[k]) cudaStreamDestroy(ctx->copy_more[k]);
  }
  for (auto& e : ctx->evs) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  for (auto e : ctx->evpool) cudaEventDestroy(e);
  delete ctx;
}

extern "C" const char* cavity_last_error(const cavity_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_setup_err.c_str();
}

extern "C" cavity_status cavity_sizes(const cavity_ctx* ctx, long long* n_ap, long long* fpd) {
  if (!ctx) return CAVITY_EINVAL;
  if (n_ap) *n_ap = ctx->g.nap;
  if (fpd) *fpd = ctx->g.field_per_dir;
  return CAVITY_OK;
}

extern "C" cavity_status cavity_periods(const cavity_ctx* ctx, int* pad_x, int* pad_y) {
  if (!ctx || !pad_x || !pad_y) return CAVITY_EINVAL;
  *pad_x = ctx->g.padx;
  *pad_y = ctx->g.pady;
  return CAVITY_OK;
}

static cavity_status check_layers(cavity_ctx* ctx, int nlayers, const int* lev, const double* er,
                                  const double* ei) {
  if (nlayers < 1 || nlayers > 16 || !lev || !er || !ei) {
    ctx->err = "need 1..16 layers with level counts and permittivities";
    return CAVITY_EINVAL;
  }
  long long sum = 0;
  for (int l = 0; l < nlayers; ++l) {
    if (lev[l] < 2) {
      ctx->err = "every layer must span at least two grid steps";
      return CAVITY_EINVAL;
    }
    if (!std::isfinite(er[l]) || !std::isfinite(ei[l])) {
      ctx->err = "non-finite permittivity";
      return CAVITY_EINVAL;
    }
    sum += lev[l];
  }
  if (sum != ctx->g.nz) {
    ctx->err = "layer level counts must sum to nz";
    return CAVITY_EINVAL;
  }
  return CAVITY_OK;
}

extern "C" cavity_status cavity_prepare(cavity_ctx* ctx, double kappa0, int nlayers,
                                        const int* layer_levels, const double* eps_re,
                                        const double* eps_im) {
  if (!ctx) return CAVITY_EINVAL;
  if (!(kappa0 > 0) || !std::isfinite(kappa0)) {
    ctx->err = "kappa0 must be positive";
    return CAVITY_EINVAL;
  }
  CKS(check_layers(ctx, nlayers, layer_levels, eps_re, eps_im));
  std::vector<LayerDev> L(nlayers);
  for (int l = 0; l < nlayers; ++l) L[l] = LayerDev{layer_levels[l], eps_re[l], eps_im[l]};
  bool same = ctx->prepared && ctx->kappa0 == kappa0 && ctx->layers.size() == L.size();
  if (same)
    for (int l = 0; l < nlayers; ++l)
      same = same && L[l].nlev == ctx->layers[l].nlev && L[l].eps_re == ctx->layers[l].eps_re &&
             L[l].eps_im == ctx->layers[l].eps_im;
  if (same) return CAVITY_OK;
  ctx->prepared = false;
  ctx->dn.ready = false;
  ctx->cs.ready = false;
  bool kappa_same = ctx->khat64 && ctx->kappa0 == kappa0;
  ctx->kappa0 = kappa0;
  ctx->layers = L;
  if (!kappa_same) CKS(launch_khat(ctx, kappa0));
  CKS(launch_zsweep(ctx, kappa0));
  if (ctx->g.fft_ok) {   // the Krylov path's preconditioner and operator tables
    CKS(launch_precond(ctx));
    CKS(launch_pair_tables(ctx));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  ctx->prepared = true;
  if (ctx->desc.aperture_solver == CAVITY_SOLVER_DENSE) {
    // Step 3 of Algorithm I/II as a direct solve: the kept block's factors
    // are part of the resident state of this (kappa0, eps)
    cavity_status s = launch_dense_factor(ctx);
    if (s == CAVITY_OK) {
      cudaError_t e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) {
        ctx->err = cudaGetErrorString(e);
        s = CAVITY_ECUDA;
      }
    }
    if (s != CAVITY_OK) {
      ctx->prepared = false;
      return s;
    }
  }
  return CAVITY_OK;
}

extern "C" cavity_status cavity_rhs(cavity_ctx* ctx, int ndir, const double* theta,
                                    const double* phi, const double* alpha, void* out) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared) {
    ctx->err = "call cavity_prepare (or cavity_solve) first";
    return CAVITY_EINVAL;
  }
  if (ndir < 1 || !theta || !phi || !alpha || !out) {
    ctx->err = "bad rhs arguments";
    return CAVITY_EINVAL;
  }
  CKS(launch_rhs(ctx, ndir, theta, phi, alpha, (double2*)out));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_apply(cavity_ctx* ctx, int ndir, int precision, const void* x,
                                      void* y) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared || ndir < 1 || !x || !y) {
    ctx->err = "cavity_apply: not prepared or bad arguments";
    return CAVITY_EINVAL;
  }
  if (precision == CAVITY_FP64) {
    CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, apply_work_bytes(ctx->g, ndir, sizeof(double2))));
    CKS(launch_apply<double>(ctx, ndir, (const double2*)x, (double2*)y, ctx->ws));
  } else if (precision == CAVITY_MIXED) {
    CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, apply_work_bytes(ctx->g, ndir, sizeof(float2))));
    CKS(launch_apply<float>(ctx, ndir, (const float2*)x, (float2*)y, ctx->ws));
  } else if (precision == CAVITY_PAIR32) {
    CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, apply_pair_work_bytes(ctx->g, ndir)));
    CKS(launch_apply_pair(ctx, ndir, (const double2*)x, (double2*)y, ctx->ws));
  } else {
    ctx->err = "unknown precision";
    return CAVITY_EINVAL;
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_field(cavity_ctx* ctx, int ndir, const void* aperture, void* field) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared || ndir < 1 || !aperture || !field) {
    ctx->err = "cavity_field: not prepared or bad arguments";
    return CAVITY_EINVAL;
  }
  if (ctx->desc.precision == CAVITY_FP64)
    CKS(launch_field<double>(ctx, ndir, (const double2*)aperture, (double2*)field));
  else
    CKS(launch_field<float>(ctx, ndir, (const double2*)aperture, (float2*)field));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_export_elimination(cavity_ctx* ctx, void* top, void* prof,
                                                   void* profq) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared) {
    ctx->err = "not prepared";
    return CAVITY_EINVAL;
  }
  const Geo& g = ctx->g;
  if (top)
    CK(cudaMemcpyAsync(top, ctx->top64, sizeof(double2) * (g.nap + g.n1 + g.n2),
                       cudaMemcpyDeviceToDevice, ctx->stream));
  if (prof)
    CK(cudaMemcpyAsync(prof, ctx->prof, sizeof(double2) * (size_t)(g.nz - 1) * g.nap,
                       cudaMemcpyDeviceToDevice, ctx->stream));
  if (profq) {
    size_t nq = sizeof(double2) * (size_t)(g.nz - 1) * (g.n1 + g.n2);
    if (ctx->layers.size() > 1)
      CK(cudaMemcpyAsync(profq, ctx->profq, nq, cudaMemcpyDeviceToDevice, ctx->stream));
    else
      CK(cudaMemsetAsync(profq, 0, nq, ctx->stream));
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_export_khat(cavity_ctx* ctx, void* khat) {
  if (!ctx || !khat) return CAVITY_EINVAL;
  if (!ctx->prepared) {
    ctx->err = "not prepared";
    return CAVITY_EINVAL;
  }
  const Geo& g = ctx->g;
  CK(cudaMemcpyAsync(khat, ctx->khat_raw, sizeof(double2) * (size_t)(g.Px / 2) * (g.Py / 2),
                     cudaMemcpyDeviceToDevice, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_solve(cavity_ctx* ctx, double kappa0, int nlayers,
                                      const int* layer_levels, const double* eps_re,
                                      const double* eps_im, int ndir, const double* theta,
                                      const double* phi, const double* alpha, int out_mode,
                                      int out_mem, void* aperture_out, void* field_out,
                                      int* iters_out, double* resid_out) {
  if (!ctx) return CAVITY_EINVAL;
  if (ndir < 1 || !theta || !phi || !alpha || !aperture_out ||
      (out_mode == CAVITY_OUT_FIELD && !field_out) ||
      (out_mode != CAVITY_OUT_FIELD && out_mode != CAVITY_OUT_APERTURE) ||
      (out_mem != CAVITY_MEM_DEVICE && out_mem != CAVITY_MEM_HOST)) {
    ctx->err = "cavity_solve: bad arguments";
    return CAVITY_EINVAL;
  }
  CKS(cavity_prepare(ctx, kappa0, nlayers, layer_levels, eps_re, eps_im));
  const Geo& g = ctx->g;
  const size_t nv = (size_t)ndir * g.nap;
  const bool host = out_mem == CAVITY_MEM_HOST;
  const size_t fbytes = (size_t)ndir * g.field_per_dir *
                        (ctx->desc.precision == CAVITY_FP64 ? sizeof(double2) : sizeof(float2));
  // b and (for host output) x and the field are staged on the device
  size_t need = sizeof(double2) * nv * (host ? 2 : 1) +
                ((host && out_mode == CAVITY_OUT_FIELD) ? fbytes : 0) + 512;
  CKS(ensure_ws(ctx, &ctx->stage, &ctx->stage_bytes, need));
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  char* p = (char*)ctx->stage;
  double2* b = (double2*)p;
  p += al(sizeof(double2) * nv);
  double2* x = host ? (double2*)p : (double2*)aperture_out;
  if (host) p += al(sizeof(double2) * nv);
  void* fld = host ? (void*)p : field_out;
  CKS(launch_rhs(ctx, ndir, theta, phi, alpha, b));
  CKS(launch_mode_mask(ctx, ndir, b));  // truncated expansion: the kept rows only
  cavity_status st;
  if (ctx->desc.aperture_solver == CAVITY_SOLVER_DENSE)
    st = run_dense_solve(ctx, ndir, b, x, iters_out, resid_out);
  else if (ctx->desc.precision == CAVITY_FP64)
    st = run_gmres64(ctx, ndir, b, x, iters_out, resid_out);
  else
    st = run_mixed_solve(ctx, ndir, b, x, iters_out, resid_out);
  if (st != CAVITY_OK && st != CAVITY_ENOCONV) return st;
  if (host) {
    // host outputs go out on the copy stream, overlapped with the field
    // synthesis: the aperture now, the field chunk by chunk (launch_field)
    CKS(ensure_copy_stream(ctx, 2));
    CK(cudaEventRecord(ctx->copy_evs[0], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->copy_stream, ctx->copy_evs[0], 0));
    CK(cudaMemcpyAsync(aperture_out, x, sizeof(double2) * nv, cudaMemcpyDeviceToHost,
                       ctx->copy_stream));
  }
  if (out_mode == CAVITY_OUT_FIELD) {
    void* hf = host ? field_out : nullptr;
    if (ctx->desc.precision == CAVITY_FP64)
      CKS(launch_field<double>(ctx, ndir, x, (double2*)fld, hf));
    else
      CKS(launch_field<float>(ctx, ndir, x, (float2*)fld, hf));
  }
  if (host) {
    CK(cudaEventRecord(ctx->copy_evs[1], ctx->copy_stream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->copy_evs[1], 0));
    for (int k = 0; k < 3; ++k) {
      CK(cudaEventRecord(ctx->copy_join[k], ctx->copy_more[k]));
      CK(cudaStreamWaitEvent(ctx->stream, ctx->copy_join[k], 0));
    }
  }
  CK(cudaStreamSynchronize(ctx->stream));
  return st;
}

extern "C" cavity_status cavity_rcs(cavity_ctx* ctx, int ndir, const void* aperture, int mem,
                                    const double* obs_theta, const double* obs_phi, int pol,
                                    double* sigma_out) {
  if (!ctx) return CAVITY_EINVAL;
  if (!ctx->prepared || ndir < 1 || !aperture || !obs_theta || !obs_phi || !sigma_out ||
      (pol != CAVITY_POL_THETA && pol != CAVITY_POL_PHI) ||
      (mem != CAVITY_MEM_DEVICE && mem != CAVITY_MEM_HOST)) {
    ctx->err = "cavity_rcs: bad arguments or not prepared";
    return CAVITY_EINVAL;
  }
  const double2* ap = (const double2*)aperture;
  void* tmp = nullptr;
  if (mem == CAVITY_MEM_HOST) {
    size_t nb = sizeof(double2) * (size_t)ndir * ctx->g.nap;
    CK(cudaMalloc(&tmp, nb));
    cudaError_t e = cudaMemcpyAsync(tmp, aperture, nb, cudaMemcpyHostToDevice, ctx->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      ctx->err = cudaGetErrorString(e);
      return CAVITY_ECUDA;
    }
    ap = (const double2*)tmp;
  }
  cavity_status s = launch_rcs(ctx, ndir, ap, obs_theta, obs_phi, pol, sigma_out);
  if (tmp) cudaFree(tmp);
  return s;
}

static const char* kclass_names[KC_N] = {
    "tbc_A_fp64", "tbc_B_fp64", "tbc_C_fp64", "tbc_D_fp64", "tbc_combine_fp64",
    "tbc_A_fp32", "tbc_B_fp32", "tbc_C_fp32", "tbc_D_fp32", "tbc_combine_fp32",
    "krylov", "precond", "field_y", "field_x", "rhs_rcs", "setup",
    "tbc_A_pair32", "tbc_B_pair32", "tbc_C_pair32", "tbc_D_pair32", "tbc_combine_pair32",
    "dense_assemble", "dense_lu", "dense_solve"};
static_assert(KC_N == CAVITY_NUM_KCLASS, "class count");

extern "C" const char* cavity_kernel_class(int k) {
  return (k >= 0 && k < KC_N) ? kclass_names[k] : "";
}

static void drain_events(cavity_ctx* ctx) {
  for (auto& e : ctx->evs) {
    float t = 0;
    if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ctx->ms[e.cls] += t;
    ctx->evpool.push_back(e.a);
    ctx->evpool.push_back(e.b);
  }
  ctx->evs.clear();
}

extern "C" cavity_status cavity_timing(cavity_ctx* ctx, int enable) {
  if (!ctx) return CAVITY_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  drain_events(ctx);
  for (int k = 0; k < KC_N; ++k) {
    ctx->nlaunch[k] = 0;
    ctx->ms[k] = 0;
  }
  ctx->timing = enable != 0;
  return CAVITY_OK;
}

extern "C" cavity_status cavity_timing_read(cavity_ctx* ctx, int nclass, double* ms,
                                            long long* launches) {
  if (!ctx || nclass < 0 || nclass > KC_N) return CAVITY_EINVAL;
  CK(cudaStreamSynchronize(ctx->stream));
  drain_events(ctx);
  for (int k = 0; k < nclass; ++k) {
    if (ms) ms[k] = ctx->ms[k];
    if (launches) launches[k] = ctx->nlaunch[k];
  }
  return CAVITY_OK;
}

extern "C" cavity_status cavity_dense_size(const cavity_ctx* ctx, int* n) {
  if (!ctx || !n) return CAVITY_EINVAL;
  *n = kept_set(ctx->desc, ctx->g).nk;
  return CAVITY_OK;
}

extern "C" cavity_status cavity_dense_assemble(cavity_ctx* ctx, void* a, int lda) {
  if (!ctx) return CAVITY_EINVAL;
  if (!a) {
    ctx->err = "cavity_dense_assemble: a is NULL";
    return CAVITY_EINVAL;
  }
  CKS(dense_assemble(ctx, kept_set(ctx->desc, ctx->g), (float2*)a, lda));
  CK(cudaStreamSynchronize(ctx->stream));
  return CAVITY_OK;
}

extern "C" cavity_status cavity_lu_factor(cavity_ctx* ctx, void* a, int n, int lda, int* ipiv,
                                          int* info) {
  if (!ctx) return CAVITY_EINVAL;
  int inf = -1;
  cavity_status s = dense_lu(ctx, (float2*)a, n, lda, ipiv, &inf);
  if (info) *info = inf;
  return s;
}

extern "C" cavity_status cavity_lu_solve(cavity_ctx* ctx, const void* lu, int n, int lda,
                                         const int* ipiv, int nrhs, void* b, int ldb) {
  if (!ctx) return CAVITY_EINVAL;
  return dense_lu_solve(ctx, (const float2*)lu, n, lda, ipiv, nullptr, nrhs, (float2*)b, ldb);
}

extern "C" cavity_status cavity_set_option(cavity_ctx* ctx, int option, int value) {
  if (!ctx) return CAVITY_EINVAL;
  bool ok = false;
  switch (option) {
    case CAVITY_OPT_PASS_B_2048:
    case CAVITY_OPT_PASS_C_2048: ok = value == 0 || value == 1; break;
    case CAVITY_OPT_GROUP_WIDTH: ok = value >= 1 && value <= 16; break;
    case CAVITY_OPT_FIELD_FUSED:
      ok = value >= 0 && value <= 2;
      // the FP32 profiles are laid out for one kernel or the other
      if (ok && value != ctx->opt[option]) ctx->prepared = false;
      break;
    case CAVITY_OPT_COARSE_MODES: {
      const KeptSet all = kept_set(ctx->desc, ctx->g);
      ok = value == 0 ||
           (value > 0 && kept_set_of(std::min(value, all.mm), std::min(value, all.nn)).nk <=
                             CAVITY_DENSE_MAX_N);
      if (ok && value != ctx->opt[option]) ctx->cs.ready = false;
      break;
    }
    default: break;
  }
  if (!ok) {
    ctx->err = "cavity_set_option: unknown option " + std::to_string(option) + " or value " +
               std::to_string(value) + " out of range";
    return CAVITY_EINVAL;
  }
  ctx->opt[option] = value;
  return CAVITY_OK;
}

extern "C" cavity_status cavity_get_option(const cavity_ctx* ctx, int option, int* value) {
  if (!ctx || !value || option < 0 || option >= CAVITY_NUM_OPT) return CAVITY_EINVAL;
  *value = ctx->opt[option];
  return CAVITY_OK;
}
