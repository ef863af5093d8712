// Aperture solve of (EJ1)/(uT1): restarted GMRES with right block-diagonal
// preconditioning, batched over the incident directions (one Krylov basis per
// right-hand side, all advanced together).
//
// The paper solves the aperture system directly and notes that large
// apertures need an iterative solver (Sec. 6); GMRES is that solver here.
// Orthogonalisation: classical Gram-Schmidt with a second pass where the first
// removed more than half of ||w||^2 ("twice is enough"): batched dot-product
// passes and basis updates, the second skipped per direction.  All reductions
// are fixed-order block trees, so a direction's result does not depend on the
// other directions in the batch.  The small Hessenberg least-squares problems
// (complex Givens rotations) are solved on the host from the coefficients
// copied back once per iteration.
//
// Mixed precision (CAVITY_MIXED): iterative refinement in FP64 around FP32
// block GMRES (bgmres.cu; all directions of a group share one Krylov basis):
// solve A d = r with FP32 block GMRES to ~1e-5;  x += d (FP64);  update r;
// repeat until ||r|| <= tol ||b||.  The residual is updated two ways:
//   while the correction is large (||r|| > RES32_MAX ||b||, always after the
//   first solve): r = b - A x with the operator in pair-of-FP32 arithmetic
//   (relative error ~1e-12: FP64-grade for a residual, at FP32 instruction
//   rates; see df64.cuh);
//   afterwards:    r = r - A d with the FP32 operator applied to the (scaled)
//   correction, subtracted in FP64.
// The second form is exact algebra (b - A(x + d) = r - A d); its only error is
// the FP32 operator's, eps32 ||A d|| <= eps32 (||r|| + ||r_new||), and the
// parity tests bound eps32 (relative error of the FP32 operator) far below
// 1e-5, so with ||r|| <= 1e-4 ||b|| the updated residual is within 2e-9 ||b||
// of the true one.  One FP64 operator application per solve instead of one per
// refinement step, and that one in pair-of-FP32 arithmetic.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"

// h[d*hstride + i] = sum_e conj(V[d*vs + i*nap + e]) w[d*ws + e]   (grid (cnt, ndir))
template <typename T>
__global__ void __launch_bounds__(256) k_dots(const C<T>* __restrict__ V, long long vs,
                                              const C<T>* __restrict__ w, long long ws,
                                              double2* __restrict__ h, int hstride, int nap) {
  const int i = blockIdx.x, d = blockIdx.y;
  const C<T>* v = V + (size_t)d * vs + (size_t)i * nap;
  const C<T>* x = w + (size_t)d * ws;
  double sr = 0, si = 0;
  for (int e = threadIdx.x; e < nap; e += blockDim.x) {
    C<T> a = v[e], b = x[e];
    sr += (double)a.x * b.x + (double)a.y * b.y;
    si += (double)a.x * b.y - (double)a.y * b.x;
  }
  for (int off = 16; off > 0; off >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, off);
    si += __shfl_xor_sync(0xffffffffu, si, off);
  }
  __shared__ double rr[8], ri[8];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { rr[wid] = sr; ri[wid] = si; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < 8; ++k) { a += rr[k]; b += ri[k]; }
    h[(size_t)d * hstride + i] = make_double2(a, b);
  }
}

// Multi-dot V^H w in two fixed-order stages: each block keeps one chunk of w
// in shared memory and forms the partial dots of that chunk with all cnt basis
// vectors; a second kernel adds the chunk partials in chunk order.
#define MDOT_CHUNK 2048
template <typename T>
__global__ void __launch_bounds__(256) k_mdot_partial(const C<T>* __restrict__ V, long long vs,
                                                      const C<T>* __restrict__ w, long long ws,
                                                      double2* __restrict__ part, int cnt, int nap,
                                                      int nchunk, const int* __restrict__ flag) {
  __shared__ C<T> sw[MDOT_CHUNK];
  __shared__ double rr[8], ri[8];
  const int c = blockIdx.x, d = blockIdx.y, tid = threadIdx.x;
  if (flag && !flag[d]) {
    // pass skipped for this direction: zero partials
    for (int i = tid; i < cnt; i += blockDim.x)
      part[((size_t)d * nchunk + c) * cnt + i] = make_double2(0.0, 0.0);
    return;
  }
  const int e0 = c * MDOT_CHUNK;
  const int ne = min(nap - e0, MDOT_CHUNK);
  const C<T>* wd = w + (size_t)d * ws + e0;
  for (int e = tid; e < ne; e += 256) sw[e] = wd[e];
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  const int nsub = cnt >= 8 ? 1 : 8 / cnt;  // warps per basis vector
  const int ng = 8 / nsub;                  // basis vectors per round
  for (int i0 = 0; i0 < cnt; i0 += ng) {
    const int i = i0 + warp / nsub, sub = warp - (warp / nsub) * nsub;
    double sr = 0, si = 0;
    if (i < cnt) {
      // per-lane partial sums (at most 64 terms) and the sum across the warp
      // in the vector precision; FP64 across warps and chunks.  (FP64
      // instructions are scarce on this GPU: an FP64 shuffle tree per warp
      // would cost more than the FP32 products themselves.)
      const C<T>* v = V + (size_t)d * vs + (size_t)i * nap + e0;
      T ar = 0, ai = 0;
      if (nsub == 1 && ne == MDOT_CHUNK) {
        // full chunk, one warp per vector: 8 loads in flight, 4 partial sums
        T pr[4] = {0, 0, 0, 0}, pi[4] = {0, 0, 0, 0};
#pragma unroll 8
        for (int k = 0; k < MDOT_CHUNK / 32; ++k) {
          const int e = lane + 32 * k;
          const C<T> a = v[e], b = sw[e];
          pr[k & 3] += a.x * b.x + a.y * b.y;
          pi[k & 3] += a.x * b.y - a.y * b.x;
        }
        ar = (pr[0] + pr[1]) + (pr[2] + pr[3]);
        ai = (pi[0] + pi[1]) + (pi[2] + pi[3]);
      } else {
        for (int e = sub * 32 + lane; e < ne; e += nsub * 32) {
          const C<T> a = v[e], b = sw[e];
          ar += a.x * b.x + a.y * b.y;
          ai += a.x * b.y - a.y * b.x;
        }
      }
      for (int off = 16; off > 0; off >>= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, off);
        ai += __shfl_xor_sync(0xffffffffu, ai, off);
      }
      sr = (double)ar;
      si = (double)ai;
    }
    if (lane == 0) { rr[warp] = sr; ri[warp] = si; }
    __syncthreads();
    if (tid < ng && i0 + tid < cnt) {
      double a = 0, b = 0;
      for (int q = 0; q < nsub; ++q) { a += rr[tid * nsub + q]; b += ri[tid * nsub + q]; }
      part[((size_t)d * nchunk + c) * cnt + i0 + tid] = make_double2(a, b);
    }
    __syncthreads();
  }
}

// h[d][i] = sum over chunks of the partials, in chunk order within each lane
// and a fixed shuffle tree across lanes: one warp per (i, d), grid (cnt, ndir)
__global__ void k_mdot_final(const double2* __restrict__ part, double2* __restrict__ h, int hstride,
                             int cnt, int nchunk) {
  const int i = blockIdx.x, d = blockIdx.y, lane = threadIdx.x;
  double a = 0, b = 0;
  for (int c = lane; c < nchunk; c += 32) {
    const double2 v = part[((size_t)d * nchunk + c) * cnt + i];
    a += v.x;
    b += v.y;
  }
  for (int off = 16; off > 0; off >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, off);
    b += __shfl_xor_sync(0xffffffffu, b, off);
  }
  if (lane == 0) h[(size_t)d * hstride + i] = make_double2(a, b);
}

// w[d][e] += sgn * sum_{i<cnt} V[d*vs + i*nap + e] c[d*cstride + i]
// grid (ceil(nap / 256), ndir); the coefficients are rounded to the vector
// precision once per block (cnt <= GMRES_MAXC)
#define GMRES_MAXC 128
template <typename T>
__global__ void __launch_bounds__(256) k_basis_axpy(const C<T>* __restrict__ V, long long vs,
                                                    const double2* __restrict__ c, int cstride,
                                                    int cnt, C<T>* __restrict__ w, int nap, T sgn,
                                                    const int* __restrict__ flag = nullptr,
                                                    long long wstride = -1) {
  __shared__ C<T> cf[GMRES_MAXC];
  const int d = blockIdx.y;
  if (flag && !flag[d]) return;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const double2 bd = c[(size_t)d * cstride + i];
    cf[i] = mk<T>((T)(sgn * bd.x), (T)(sgn * bd.y));
  }
  __syncthreads();
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const C<T>* v = V + (size_t)d * vs + e;
  T ar = 0, ai = 0;
  int i = 0;
  for (; i + 8 <= cnt; i += 8) {
    C<T> a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = v[(size_t)(i + k) * nap];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const C<T> b = cf[i + k];
      ar += a[k].x * b.x - a[k].y * b.y;
      ai += a[k].x * b.y + a[k].y * b.x;
    }
  }
  for (; i < cnt; ++i) {
    const C<T> a = v[(size_t)i * nap], b = cf[i];
    ar += a.x * b.x - a.y * b.y;
    ai += a.x * b.y + a.y * b.x;
  }
  const size_t o = (size_t)d * (wstride >= 0 ? wstride : nap) + e;
  const C<T> ov = w[o];
  w[o] = mk<T>(ov.x + ar, ov.y + ai);
}

// out[d*os + e] = s[d] * in[d*is + e]   (grid (ceil(nap / 256), ndir))
template <typename T>
__global__ void k_copy_scale(const C<T>* __restrict__ in, long long is, C<T>* __restrict__ out,
                             long long os, const double* __restrict__ s, int nap) {
  const int d = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const C<T> a = in[(size_t)d * is + e];
  const T f = (T)s[d];
  out[(size_t)d * os + e] = mk<T>(a.x * f, a.y * f);
}

// Second Gram-Schmidt pass needed?  ("twice is enough": reorthogonalise when
// the first pass removed more than half of ||w||^2.)  ||w - V h||^2 is
// estimated as ||w||^2 - sum |h_i|^2 (V orthonormal).
__global__ void k_reorth_flag(const double2* __restrict__ h, int hstride, int cnt,
                              const double2* __restrict__ wn2, int wstride, int* __restrict__ flag,
                              int ndir) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= ndir) return;
  double s = 0;
  for (int i = 0; i < cnt; ++i) {
    const double2 v = h[(size_t)d * hstride + i];
    s += v.x * v.x + v.y * v.y;
  }
  const double w0 = wn2[(size_t)d * wstride].x;
  flag[d] = (w0 - s < 0.5 * w0) ? 1 : 0;
}

// y += x  (contiguous [d][nap])
template <typename T>
__global__ void k_add(const C<T>* __restrict__ x, C<T>* __restrict__ y, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) y[k] = cadd<T>(y[k], x[k]);
}

// w = b - w
template <typename T>
__global__ void k_bminus(const C<T>* __restrict__ b, C<T>* __restrict__ w, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) w[k] = csub<T>(b[k], w[k]);
}

// x64 += d32 / s[d]   (grid (ceil(nap / 256), ndir))
__global__ void k_acc32(double2* __restrict__ x, const float2* __restrict__ dx,
                        const double* __restrict__ s, int nap) {
  const int d = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const size_t k = (size_t)d * nap + e;
  const double f = s[d] > 0 ? 1.0 / s[d] : 0.0;
  const float2 v = dx[k];
  x[k].x += f * (double)v.x;
  x[k].y += f * (double)v.y;
}

// r32 = s[d] * r64   (grid (ceil(nap / 256), ndir))
__global__ void k_to32(const double2* __restrict__ r, float2* __restrict__ o,
                       const double* __restrict__ s, int nap) {
  const int d = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const size_t k = (size_t)d * nap + e;
  const double f = s[d];
  o[k] = make_float2((float)(r[k].x * f), (float)(r[k].y * f));
}

static inline unsigned nblk(long long n, int b) { return (unsigned)((n + b - 1) / b); }

static inline double2 h_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
static inline double2 h_mul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
static inline double2 h_conj(double2 a) { return make_double2(a.x, -a.y); }
static inline double h_abs(double2 a) { return std::hypot(a.x, a.y); }

template <typename T> struct GW {
  C<T>* V;      // ndir x (m+1) x nap
  C<T>* w;      // ndir x nap
  C<T>* z;      // ndir x nap
  double2* h;   // ndir x (m+1)
  double2* h2;  // ndir x (m+1)
  double2* y;   // ndir x (m+1)
  double* s;    // ndir
  double2* part;  // ndir x nchunk x (m+1) multi-dot partials
  double2* wn;    // ndir: ||w||^2 before orthogonalisation
  int* flag;      // ndir: second Gram-Schmidt pass needed
  void* apw;    // operator workspace
};

static inline int mdot_chunks(int nap) { return (nap + MDOT_CHUNK - 1) / MDOT_CHUNK; }

template <typename T>
static size_t gw_bytes(const Geo& g, int ndir, int m) {
  size_t b = 0;
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  b += al(sizeof(C<T>) * (size_t)ndir * (m + 1) * g.nap);
  b += 2 * al(sizeof(C<T>) * (size_t)ndir * g.nap);
  b += 3 * al(sizeof(double2) * (size_t)ndir * (m + 1));
  b += al(sizeof(double) * ndir);
  b += al(sizeof(double2) * (size_t)ndir * mdot_chunks(g.nap) * (m + 1));
  b += al(sizeof(double2) * ndir) + al(sizeof(int) * ndir);
  b += al(apply_work_bytes(g, ndir, sizeof(C<T>)));
  return b;
}

template <typename T>
static GW<T> gw_carve(void* base, const Geo& g, int ndir, int m) {
  auto al = [](size_t x) { return (x + 255) / 256 * 256; };
  char* p = (char*)base;
  GW<T> W;
  W.V = (C<T>*)p; p += al(sizeof(C<T>) * (size_t)ndir * (m + 1) * g.nap);
  W.w = (C<T>*)p; p += al(sizeof(C<T>) * (size_t)ndir * g.nap);
  W.z = (C<T>*)p; p += al(sizeof(C<T>) * (size_t)ndir * g.nap);
  W.h = (double2*)p; p += al(sizeof(double2) * (size_t)ndir * (m + 1));
  W.h2 = (double2*)p; p += al(sizeof(double2) * (size_t)ndir * (m + 1));
  W.y = (double2*)p; p += al(sizeof(double2) * (size_t)ndir * (m + 1));
  W.s = (double*)p; p += al(sizeof(double) * ndir);
  W.part = (double2*)p; p += al(sizeof(double2) * (size_t)ndir * mdot_chunks(g.nap) * (m + 1));
  W.wn = (double2*)p; p += al(sizeof(double2) * ndir);
  W.flag = (int*)p; p += al(sizeof(int) * ndir);
  W.apw = p;
  return W;
}

// out[d*ostride + i] = <V_i, w> for i < cnt, all directions
template <typename T>
static void mdot(cavity_ctx* ctx, const C<T>* V, long long vs, const C<T>* w, long long ws, int cnt,
                 double2* out, int ostride, double2* part, int ndir, const int* flag = nullptr) {
  const int nap = ctx->g.nap, nchunk = mdot_chunks(nap);
  {
    KScope ks_(ctx, KC_KRYLOV);
    k_mdot_partial<T><<<dim3(nchunk, ndir), 256, 0, ctx->stream>>>(V, vs, w, ws, part, cnt, nap,
                                                                   nchunk, flag);
  }
  {
    KScope ks_(ctx, KC_KRYLOV);
    k_mdot_final<<<dim3(cnt, ndir), 32, 0, ctx->stream>>>(part, out, ostride, cnt, nchunk);
  }
}

// norms of ndir contiguous vectors (host result)
template <typename T>
static cavity_status norms(cavity_ctx* ctx, const C<T>* v, int ndir, double2* scratch, int sstride,
                           std::vector<double>& out, double2* part) {
  const int nap = ctx->g.nap;
  mdot<T>(ctx, v, nap, v, nap, 1, scratch, sstride, part, ndir);
  std::vector<double2> hh((size_t)ndir);
  CK(cudaMemcpy2DAsync(hh.data(), sizeof(double2), scratch, sizeof(double2) * sstride,
                       sizeof(double2), ndir, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  out.resize(ndir);
  for (int d = 0; d < ndir; ++d) out[d] = std::sqrt(std::max(hh[d].x, 0.0));
  return CAVITY_OK;
}

// Solve A x = b (x starts at zero).  tol[d]: relative target per direction.
// iters[d] accumulates Arnoldi steps; est[d] is the final GMRES residual
// estimate relative to ||b_d||.
template <typename T>
static cavity_status gmres_core(cavity_ctx* ctx, int ndir, const C<T>* b, C<T>* x,
                                const std::vector<double>& tol, int m, int maxit, GW<T> W,
                                std::vector<int>& iters, std::vector<double>& est) {
  const Geo& g = ctx->g;
  const int nap = g.nap;
  const long long nv = (long long)ndir * nap;
  const long long vs = (long long)(m + 1) * nap;
  cudaStream_t st = ctx->stream;
  std::vector<double> bnorm, rn;
  CKS(norms<T>(ctx, b, ndir, W.h, m + 1, bnorm, W.part));
  rn = bnorm;
  est.assign(ndir, 0.0);
  CK(cudaMemsetAsync(x, 0, sizeof(C<T>) * nv, st));
  CK(cudaMemcpyAsync(W.w, b, sizeof(C<T>) * nv, cudaMemcpyDeviceToDevice, st));   // r = b
  std::vector<char> done(ndir, 0);
  for (int d = 0; d < ndir; ++d) {
    if (!(bnorm[d] > 0)) done[d] = 1;
    else est[d] = 1.0;
  }
  std::vector<double> sc(ndir);
  std::vector<double2> h1((size_t)ndir * (m + 1)), h2v((size_t)ndir * (m + 1)), nw((size_t)ndir * (m + 1));
  std::vector<double2> hy((size_t)ndir * (m + 1));
  int total = 0;
  while (true) {
    bool alldone = true;
    for (int d = 0; d < ndir; ++d) alldone = alldone && done[d];
    if (alldone || total >= maxit) break;
    // V_0 = r / ||r||
    for (int d = 0; d < ndir; ++d) sc[d] = (!done[d] && rn[d] > 0) ? 1.0 / rn[d] : 0.0;
    CK(cudaMemcpyAsync(W.s, sc.data(), sizeof(double) * ndir, cudaMemcpyHostToDevice, st));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_copy_scale<T><<<dim3(nblk(nap, 256), ndir), 256, 0, st>>>(W.w, nap, W.V, vs, W.s, nap);
    }
    std::vector<std::vector<std::vector<double2>>> H(ndir);
    std::vector<std::vector<double>> cs(ndir, std::vector<double>(m, 0.0));
    std::vector<std::vector<double2>> sn(ndir, std::vector<double2>(m, make_double2(0, 0)));
    std::vector<std::vector<double2>> gv(ndir, std::vector<double2>(m + 1, make_double2(0, 0)));
    std::vector<int> kd(ndir, 0);
    std::vector<char> act(ndir, 0);
    for (int d = 0; d < ndir; ++d) {
      act[d] = !done[d];
      gv[d][0] = make_double2(rn[d], 0);
    }
    for (int k = 0; k < m && total < maxit; ++k, ++total) {
      // V_{k+1} <- A M^{-1} V_k, written straight into the next basis slot
      C<T>* Vn = W.V + (size_t)(k + 1) * nap;
      CKS(launch_precond_apply<T>(ctx, ndir, W.V + (size_t)k * nap, W.z, vs, nap));
      CKS(launch_apply<T>(ctx, ndir, W.z, Vn, W.apw, vs));
      // classical Gram-Schmidt: <V_i, w> for i <= k and ||w||^2 (i = k+1) in
      // one pass; a second pass only where the first cancelled
      mdot<T>(ctx, W.V, vs, Vn, vs, k + 2, W.h, m + 1, W.part, ndir);
      {
        KScope ks_(ctx, KC_KRYLOV);
        k_basis_axpy<T><<<dim3(nblk(nap, 256), ndir), 256, 0, st>>>(W.V, vs, W.h, m + 1, k + 1, Vn, nap,
                                                                    (T)-1, nullptr, vs);
      }
      {
        KScope ks_(ctx, KC_KRYLOV);
        k_reorth_flag<<<1, std::max(32, ndir), 0, st>>>(W.h, m + 1, k + 1, W.h + (k + 1), m + 1,
                                                        W.flag, ndir);
      }
      mdot<T>(ctx, W.V, vs, Vn, vs, k + 1, W.h2, m + 1, W.part, ndir, W.flag);
      {
        KScope ks_(ctx, KC_KRYLOV);
        k_basis_axpy<T><<<dim3(nblk(nap, 256), ndir), 256, 0, st>>>(W.V, vs, W.h2, m + 1, k + 1, Vn, nap,
                                                                    (T)-1, W.flag, vs);
      }
      mdot<T>(ctx, Vn, vs, Vn, vs, 1, W.y, m + 1, W.part, ndir);
      CK(cudaMemcpyAsync(h1.data(), W.h, sizeof(double2) * ndir * (m + 1), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(h2v.data(), W.h2, sizeof(double2) * ndir * (m + 1), cudaMemcpyDeviceToHost, st));
      CK(cudaMemcpyAsync(nw.data(), W.y, sizeof(double2) * ndir * (m + 1), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      bool any = false;
      for (int d = 0; d < ndir; ++d) {
        sc[d] = 0.0;
        if (!act[d]) continue;
        const double hn = std::sqrt(std::max(nw[(size_t)d * (m + 1)].x, 0.0));
        std::vector<double2> col(k + 2);
        for (int i = 0; i <= k; ++i)
          col[i] = h_add(h1[(size_t)d * (m + 1) + i], h2v[(size_t)d * (m + 1) + i]);
        col[k + 1] = make_double2(hn, 0);
        for (int i = 0; i < k; ++i) {
          double2 a = col[i], bb = col[i + 1];
          const double c = cs[d][i];
          const double2 s = sn[d][i];
          col[i] = h_add(make_double2(c * a.x, c * a.y), h_mul(s, bb));
          double2 t = h_mul(h_conj(s), a);
          col[i + 1] = make_double2(c * bb.x - t.x, c * bb.y - t.y);
        }
        double2 a = col[k], bb = col[k + 1];
        const double na = h_abs(a), nb = h_abs(bb), rho = std::hypot(na, nb);
        double c;
        double2 s, r;
        if (na == 0.0) {
          c = 0.0;
          s = nb > 0 ? make_double2(bb.x / nb, -bb.y / nb) : make_double2(1, 0);
          r = make_double2(nb, 0);
        } else {
          const double2 ph = make_double2(a.x / na, a.y / na);
          c = na / rho;
          // s = (a/|a|) conj(b) / rho
          s = make_double2((ph.x * bb.x + ph.y * bb.y) / rho, (ph.y * bb.x - ph.x * bb.y) / rho);
          r = make_double2(ph.x * rho, ph.y * rho);
        }
        cs[d][k] = c;
        sn[d][k] = s;
        col[k] = r;
        col[k + 1] = make_double2(0, 0);
        const double2 gk = gv[d][k];
        gv[d][k] = make_double2(c * gk.x, c * gk.y);
        const double2 t = h_mul(h_conj(s), gk);
        gv[d][k + 1] = make_double2(-t.x, -t.y);
        H[d].push_back(col);
        kd[d] = k + 1;
        iters[d] += 1;
        const double e = h_abs(gv[d][k + 1]);
        est[d] = e / bnorm[d];
        const bool breakdown = hn <= 1e-300 || hn < 1e-15 * rho;
        if (e <= tol[d] * bnorm[d] || breakdown) act[d] = 0;
        else sc[d] = 1.0 / hn;
        any = any || act[d];
      }
      CK(cudaMemcpyAsync(W.s, sc.data(), sizeof(double) * ndir, cudaMemcpyHostToDevice, st));
      {
        // normalise V_{k+1} in place (zero for directions that stopped)
        KScope ks_(ctx, KC_KRYLOV);
        k_copy_scale<T><<<dim3(nblk(nap, 256), ndir), 256, 0, st>>>(Vn, vs, Vn, vs, W.s, nap);
      }
      if (!any) { ++total; break; }
    }
    // y = H^{-1} g; x += M^{-1} (V y)
    std::fill(hy.begin(), hy.end(), make_double2(0, 0));
    int kmax = 0;
    for (int d = 0; d < ndir; ++d) {
      const int kk = kd[d];
      kmax = std::max(kmax, kk);
      for (int i = kk - 1; i >= 0; --i) {
        double2 s = gv[d][i];
        for (int j = i + 1; j < kk; ++j) {
          double2 t = h_mul(H[d][j][i], hy[(size_t)d * (m + 1) + j]);
          s = make_double2(s.x - t.x, s.y - t.y);
        }
        const double2 dg = H[d][i][i];
        const double den = dg.x * dg.x + dg.y * dg.y;
        hy[(size_t)d * (m + 1) + i] =
            den > 0 ? make_double2((s.x * dg.x + s.y * dg.y) / den, (s.y * dg.x - s.x * dg.y) / den)
                    : make_double2(0, 0);
      }
    }
    CK(cudaMemcpyAsync(W.y, hy.data(), sizeof(double2) * ndir * (m + 1), cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(W.w, 0, sizeof(C<T>) * nv, st));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_basis_axpy<T><<<dim3(nblk(nap, 256), ndir), 256, 0, st>>>(W.V, vs, W.y, m + 1, kmax, W.w, nap,
                                                                  (T)1);
    }
    CKS(launch_precond_apply<T>(ctx, ndir, W.w, W.z));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_add<T><<<nblk(nv, 256), 256, 0, st>>>(W.z, x, nv);
    }
    for (int d = 0; d < ndir; ++d)
      if (est[d] <= tol[d]) done[d] = 1;
    bool finished = true;
    for (int d = 0; d < ndir; ++d) finished = finished && done[d];
    if (finished || total >= maxit) break;
    // restart from the true residual r = b - A x
    CKS(launch_apply<T>(ctx, ndir, x, W.w, W.apw));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_bminus<T><<<nblk(nv, 256), 256, 0, st>>>(b, W.w, nv);
    }
    CKS(norms<T>(ctx, W.w, ndir, W.h, m + 1, rn, W.part));
    for (int d = 0; d < ndir; ++d) {
      if (bnorm[d] > 0) est[d] = rn[d] / bnorm[d];
      if (est[d] <= tol[d]) done[d] = 1;
    }
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

static void solver_params(const cavity_ctx* ctx, double& tol, int& m, int& maxit) {
  tol = ctx->desc.gmres_tol > 0 ? ctx->desc.gmres_tol : 1e-12;
  m = ctx->desc.gmres_restart > 0 ? ctx->desc.gmres_restart : 40;
  maxit = ctx->desc.gmres_max_iter > 0 ? ctx->desc.gmres_max_iter : 400;
}

// FP64 path: GMRES in FP64, then the true residual.
cavity_status run_gmres64(cavity_ctx* ctx, int ndir, const double2* b, double2* x, int* iters,
                          double* resid) {
  const Geo& g = ctx->g;
  double tol;
  int m, maxit;
  solver_params(ctx, tol, m, maxit);
  size_t need = gw_bytes<double>(g, ndir, m);
  CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, need));
  GW<double> W = gw_carve<double>(ctx->ws, g, ndir, m);
  std::vector<int> it(ndir, 0);
  std::vector<double> est;
  std::vector<double> tv(ndir, tol);
  CKS(gmres_core<double>(ctx, ndir, b, x, tv, m, maxit, W, it, est));
  // true residual
  const long long nv = (long long)ndir * g.nap;
  CKS(launch_apply<double>(ctx, ndir, x, W.w, W.apw));
  {
    KScope ks_(ctx, KC_KRYLOV);
    k_bminus<double><<<nblk(nv, 256), 256, 0, ctx->stream>>>(b, W.w, nv);
  }
  std::vector<double> rn, bn;
  CKS(norms<double>(ctx, W.w, ndir, W.h, m + 1, rn, W.part));
  CKS(norms<double>(ctx, b, ndir, W.h, m + 1, bn, W.part));
  bool ok = true;
  for (int d = 0; d < ndir; ++d) {
    double r = bn[d] > 0 ? rn[d] / bn[d] : 0.0;
    if (iters) iters[d] = it[d];
    if (resid) resid[d] = r;
    ok = ok && (r <= tol * 10);
  }
  if (!ok) {
    ctx->err = "aperture GMRES stopped above tolerance";
    return CAVITY_ENOCONV;
  }
  return CAVITY_OK;
}

// r64 -= y32 / s[d]   (grid (ceil(nap / 256), ndir))
__global__ void k_sub32(double2* __restrict__ r, const float2* __restrict__ y,
                        const double* __restrict__ s, int nap) {
  const int d = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const size_t k = (size_t)d * nap + e;
  const double f = s[d] > 0 ? 1.0 / s[d] : 0.0;
  const float2 v = y[k];
  r[k].x -= f * (double)v.x;
  r[k].y -= f * (double)v.y;
}

// residuals above this fraction of ||b|| are recomputed with the FP64 operator
#define RES32_MAX 1e-4

// MIXED path: FP64 iterative refinement around FP32 block GMRES (bgmres.cu).
cavity_status run_mixed_solve(cavity_ctx* ctx, int ndir, const double2* b, double2* x, int* iters,
                              double* resid) {
  const Geo& g = ctx->g;
  double tol;
  int m, maxit;
  solver_params(ctx, tol, m, maxit);
  // block steps per cycle: the block basis grows by one column per direction
  // and step, and the inner solves converge in about a dozen steps
  const int mb = std::max(2, std::min(m, 30));
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const long long nv = (long long)ndir * g.nap;
  const size_t nb = al(block_inner_work_bytes(g, ndir, mb, ctx->opt[CAVITY_OPT_GROUP_WIDTH]));
  size_t extra = 2 * al(sizeof(double2) * nv) + 2 * al(sizeof(float2) * nv) +
                 al(apply_pair_work_bytes(g, ndir)) + al(apply_work_bytes(g, ndir, sizeof(float2))) +
                 al(sizeof(double) * ndir) + al(sizeof(double2) * ndir) +
                 al(sizeof(double2) * (size_t)ndir * mdot_chunks(g.nap));
  CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, nb + extra));
  void* bw = ctx->ws;
  char* p = (char*)ctx->ws + nb;
  double2* r64 = (double2*)p; p += al(sizeof(double2) * nv);
  double2* tmp64 = (double2*)p; p += al(sizeof(double2) * nv);
  float2* r32 = (float2*)p; p += al(sizeof(float2) * nv);
  float2* d32 = (float2*)p; p += al(sizeof(float2) * nv);
  void* apw64 = p; p += al(apply_pair_work_bytes(g, ndir));
  void* apw32 = p; p += al(apply_work_bytes(g, ndir, sizeof(float2)));
  double* sdev = (double*)p; p += al(sizeof(double) * ndir);
  double2* sc2 = (double2*)p; p += al(sizeof(double2) * ndir);
  double2* part = (double2*)p;
  cudaStream_t st = ctx->stream;
  std::vector<double> bn, rn;
  CKS(coarse_prepare(ctx));
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * nv, st));
  CK(cudaMemcpyAsync(r64, b, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
  CKS(norms<double>(ctx, b, ndir, sc2, 1, bn, part));
  rn = bn;
  std::vector<int> it(ndir, 0);
  std::vector<double> est, s(ndir), tin(ndir);
  int used = 0;
  bool conv = false;
  for (int outer = 0; outer < 12 && used < maxit; ++outer) {
    bool all = true;
    for (int d = 0; d < ndir; ++d) all = all && (bn[d] == 0 || rn[d] <= tol * bn[d]);
    if (all) { conv = true; break; }
    for (int d = 0; d < ndir; ++d) {
      s[d] = rn[d] > 0 ? 1.0 / rn[d] : 0.0;
      // reduction still needed, with a margin of 0.8 (the inner estimate is
      // accurate well above the FP32 floor), and not below what the FP32
      // inner solve reaches reliably (about 1e-6): a floor of 3e-6 split the
      // work of the two refinement cycles best when measured (16 block steps
      // in total on the 16-direction 256^2 workload, against 17 with 1e-5 or
      // 1e-6)
      double need = bn[d] > 0 ? 0.8 * tol * bn[d] / std::max(rn[d], 1e-300) : 1.0;
      tin[d] = std::min(0.5, std::max(need, 3e-6));
      if (bn[d] == 0 || rn[d] <= tol * bn[d]) s[d] = 0.0;
    }
    CK(cudaMemcpyAsync(sdev, s.data(), sizeof(double) * ndir, cudaMemcpyHostToDevice, st));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_to32<<<dim3(nblk(g.nap, 256), ndir), 256, 0, st>>>(r64, r32, sdev, g.nap);
    }
    std::vector<int> it_in(ndir, 0);
    std::vector<char> act(ndir, 0);
    for (int d = 0; d < ndir; ++d) act[d] = s[d] > 0;
    CKS(run_block_inner(ctx, ndir, r32, d32, tin, act, mb, maxit - used, bw, it_in, est));
    int mx = 0;
    for (int d = 0; d < ndir; ++d) { it[d] += it_in[d]; mx = std::max(mx, it_in[d]); }
    used += std::max(mx, 1);
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_acc32<<<dim3(nblk(g.nap, 256), ndir), 256, 0, st>>>(x, d32, sdev, g.nap);
    }
    bool big = false;
    for (int d = 0; d < ndir; ++d) big = big || (bn[d] > 0 && rn[d] > RES32_MAX * bn[d]);
    if (big) {
      // r = b - A x with the pair-of-FP32 operator (~1e-12 relative)
      CKS(launch_apply_pair(ctx, ndir, x, tmp64, apw64));
      {
        KScope ks_(ctx, KC_KRYLOV);
        k_bminus<double><<<nblk(nv, 256), 256, 0, st>>>(b, tmp64, nv);
      }
      CK(cudaMemcpyAsync(r64, tmp64, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
    } else {
      // r = r - A d with the FP32 operator on the scaled correction
      CKS(launch_apply<float>(ctx, ndir, d32, r32, apw32));
      {
        KScope ks_(ctx, KC_KRYLOV);
        k_sub32<<<dim3(nblk(g.nap, 256), ndir), 256, 0, st>>>(r64, r32, sdev, g.nap);
      }
    }
    CKS(norms<double>(ctx, r64, ndir, sc2, 1, rn, part));
  }
  bool all = true;
  for (int d = 0; d < ndir; ++d) {
    double r = bn[d] > 0 ? rn[d] / bn[d] : 0.0;
    if (iters) iters[d] = it[d];
    if (resid) resid[d] = r;
    all = all && r <= tol;
  }
  conv = conv || all;
  if (!conv) {
    ctx->err = "mixed-precision aperture solve stopped above tolerance";
    return CAVITY_ENOCONV;
  }
  return CAVITY_OK;
}

// Dense path (aperture_solver == CAVITY_SOLVER_DENSE): FP64 iterative
// refinement around the FP32 LU factors of the kept block (dense.cu).  Each
// step solves with the factors for the scaled residual of the kept rows,
// adds the correction in FP64, and recomputes r = b - A x: with the FP64 kept
// block where it is resident (the Parseval rule; the FP64 path), else with
// the pair-of-FP32 FFT operator (rule D, CAVITY_MIXED), whose rows outside
// the kept set are zero.  iters counts refinement steps.
cavity_status run_dense_solve(cavity_ctx* ctx, int ndir, const double2* b, double2* x, int* iters,
                              double* resid) {
  const Geo& g = ctx->g;
  double tol;
  int m, maxit;
  solver_params(ctx, tol, m, maxit);
  auto al = [](size_t v) { return (v + 255) / 256 * 256; };
  const long long nv = (long long)ndir * g.nap;
  const bool fp64 = ctx->desc.precision == CAVITY_FP64;
  const size_t apw = fp64 ? apply_work_bytes(g, ndir, sizeof(double2)) : apply_pair_work_bytes(g, ndir);
  const size_t need = 2 * al(sizeof(double2) * nv) + al(apw) + al(dense_inner_work_bytes(ctx, ndir)) +
                      al(sizeof(double) * ndir) + al(sizeof(double2) * ndir) +
                      al(sizeof(double2) * (size_t)ndir * mdot_chunks(g.nap));
  CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, need));
  char* p = (char*)ctx->ws;
  double2* r64 = (double2*)p; p += al(sizeof(double2) * nv);
  double2* tmp = (double2*)p; p += al(sizeof(double2) * nv);
  void* apwk = p; p += al(apw);
  void* inner = p; p += al(dense_inner_work_bytes(ctx, ndir));
  double* sdev = (double*)p; p += al(sizeof(double) * ndir);
  double2* sc2 = (double2*)p; p += al(sizeof(double2) * ndir);
  double2* part = (double2*)p;
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(x, 0, sizeof(double2) * nv, st));
  CK(cudaMemcpyAsync(r64, b, sizeof(double2) * nv, cudaMemcpyDeviceToDevice, st));
  std::vector<double> bn, rn, prev;
  CKS(norms<double>(ctx, b, ndir, sc2, 1, bn, part));
  rn = bn;
  std::vector<double> s(ndir);
  int steps = 0;
  const int max_steps = std::max(1, std::min(maxit, 30));
  bool conv = false, stalled = false;
  for (; steps < max_steps; ++steps) {
    bool all = true;
    for (int d = 0; d < ndir; ++d) all = all && (bn[d] == 0 || rn[d] <= tol * bn[d]);
    if (all) { conv = true; break; }
    if (stalled) break;
    for (int d = 0; d < ndir; ++d)
      s[d] = (bn[d] == 0 || rn[d] <= tol * bn[d] || !(rn[d] > 0)) ? 0.0 : 1.0 / rn[d];
    CK(cudaMemcpyAsync(sdev, s.data(), sizeof(double) * ndir, cudaMemcpyHostToDevice, st));
    CKS(dense_inner_solve(ctx, ndir, r64, sdev, x, inner));
    if (ctx->dn.a64) {
      // r = b - A x with the FP64 kept block (rows outside the kept set stay 0)
      CKS(dense_residual(ctx, ndir, b, x, r64));
    } else {
      if (fp64) CKS(launch_apply<double>(ctx, ndir, x, tmp, apwk));
      else CKS(launch_apply_pair(ctx, ndir, x, tmp, apwk));
      {
        KScope ks_(ctx, KC_DENSE_TRS);
        k_bminus<double><<<nblk(nv, 256), 256, 0, st>>>(b, tmp, nv);
      }
      std::swap(r64, tmp);
    }
    prev = rn;
    CKS(norms<double>(ctx, r64, ndir, sc2, 1, rn, part));
    // a step that does not halve some unconverged residual: the factors of
    // the FP32 block are too inaccurate for this system; stop after it
    for (int d = 0; d < ndir; ++d)
      if (s[d] > 0 && rn[d] > 0.5 * prev[d]) stalled = true;
  }
  int terr = 0;
  CK(cudaMemcpyAsync(&terr, dense_inner_err(ctx, ndir, inner), sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (terr) {
    ctx->err = "dense aperture solve: a grid barrier of the substitution timed out";
    return CAVITY_ETIMEOUT;
  }
  bool all = true;
  for (int d = 0; d < ndir; ++d) {
    const double r = bn[d] > 0 ? rn[d] / bn[d] : 0.0;
    if (iters) iters[d] = steps;
    if (resid) resid[d] = r;
    all = all && r <= tol;
  }
  if (!(conv || all)) {
    ctx->err = "dense aperture solve: the refinement stopped above tolerance";
    return CAVITY_ENOCONV;
  }
  return CAVITY_OK;
}
