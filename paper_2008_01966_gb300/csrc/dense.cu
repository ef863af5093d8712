// Dense direct solve of the aperture system (EJ1)/(uT1) restricted to the kept
// modes m <= mm, n <= nn: Algorithm I/II Step 3 (the paper solves the reduced
// aperture system directly), with the paper's truncation of the aperture
// expansion to few modes per axis (Sec. 7, Table 2: M ~ 2a/lambda).
//
// Assembly.  Under the discrete rule of Sec. 5.2 every TBC integral is a
// product of per-axis factors (Sec. 5.1 (sig1)-(sig3) with the FFT route):
//   I^{mn}_{k1 k2} = sum_{j1, j2} Ax(m, k1, j1) F(G)(|j1|, |j2|) Ay(n, k2, j2),
//   Ax(m, k, j1) = X(m, j1) Phi(j1, k),
// X the trapezoid projection of the torus mode exp(2 pi i j1 x / Lx) on
// cos/sin(m pi x / a), Phi the exact transform of the truncated basis
// function.  F(G) is even in j1 and j2, so each axis folds onto j >= 0 and the
// kept block is two complex GEMMs per basis pair:
//   T[j1][(n, k2)] = sum_{j2} F(G)(j1, j2) Ayf[(n, k2)][j2],
//   I[(m, k1)][(n, k2)] = sum_{j1} Axf[(m, k1)][j1] T[j1][(n, k2)],
// followed by one pass that adds the cavity part (mode-diagonal: tau, varsigma
// and the h m pi/a, h n pi/b couplings) and combines I1, I2, I3 into the rows
// of (EJ1)/(uT1) exactly as the matrix-free operator does.
//
// Factorisation.  Right-looking blocked LU with partial pivoting in FP32
// complex: per panel of LU_NB columns one cooperative kernel keeps the panel
// rows in shared memory, picks each pivot by a reduction over all CTAs
// (candidate rows published in global memory, one grid barrier per column,
// every wait bounded), then the row exchanges on the other columns, the
// triangular solve for the block row of U and the rank-LU_NB update of the
// trailing matrix (complex GEMM).
//
// Solve.  FP64 iterative refinement (gmres.cu run_dense_solve) calls
// dense_inner_solve: gather the scaled kept residual in pivot order, forward
// and back substitution by blocks of TS_B rows, scatter-add into x.
#include <algorithm>
#include <atomic>
#include <climits>

#include "common.cuh"
#include "tc05.cuh"

// ------------------------------------------------------------ kept set
KeptSet kept_set(const cavity_desc& d, const Geo& g) {
  return kept_set_of(d.modes_m > 0 ? d.modes_m : g.M, d.modes_n > 0 ? d.modes_n : g.N);
}
KeptSet kept_set_of(int mm, int nn) {
  KeptSet k;
  k.mm = mm;
  k.nn = nn;
  k.n1 = (k.mm + 1) * k.nn;
  k.n2 = k.mm * (k.nn + 1);
  k.n3 = k.mm * k.nn;
  k.nk = k.n1 + k.n2 + k.n3;
  return k;
}

// compact kept index -> full unknown index (Appendix A order)
static std::vector<int> kept_map(const KeptSet& k, const Geo& g) {
  std::vector<int> map(k.nk);
  int i = 0;
  for (int m = 0; m <= k.mm; ++m)
    for (int n = 1; n <= k.nn; ++n) map[i++] = m * g.N + (n - 1);
  for (int m = 1; m <= k.mm; ++m)
    for (int n = 0; n <= k.nn; ++n) map[i++] = g.n1 + (m - 1) * (g.N + 1) + n;
  for (int m = 1; m <= k.mm; ++m)
    for (int n = 1; n <= k.nn; ++n) map[i++] = g.n1 + g.n2 + (m - 1) * g.N + (n - 1);
  return map;
}

static inline int nblk(long long n, int b) { return (int)((n + b - 1) / b); }

// ------------------------------------------------------------ per-axis factors
// X[kind][m][j] = sum_{p=0}^{nint} w_p trig(m pi p / nint) exp(2 pi i j1 p / Pn)
// for m = 0..mk-1, j in FFT order over the box (Nyquist slot zero); trig = cos
// (kind 0) or sin (kind 1); w_p the trapezoid weights of [0, side]
__global__ void k_dn_x(double2* __restrict__ X, int mk, int nint, int Pn, double side,
                       const double2* __restrict__ tw, int TW) {
  const int kind = blockIdx.z, m = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Pn; j += gridDim.x * blockDim.x) {
    double2 r = make_double2(0, 0);
    if (j != Pn / 2 && !(kind == 1 && m == 0)) {
      const long long j1 = j < Pn / 2 ? j : j - Pn;
      for (int p = 0; p <= nint; ++p) {
        double w = side / nint;
        if (p == 0 || p == nint) w *= 0.5;
        const double2 t = tw_at(tw, TW, (long long)m * p, 2 * nint);   // exp(-i pi m p / nint)
        const double tr = kind == 0 ? t.x : -t.y;
        const double2 e = cconj<double>(tw_at(tw, TW, j1 * p, Pn));     // exp(2 pi i j1 p / Pn)
        r = cadd<double>(r, cscale<double>(e, w * tr));
      }
    }
    X[((size_t)kind * mk + m) * Pn + j] = r;
  }
}

// Phi[kind][k][j]: exact transform at j1 / (pad side) of cos (kind 0) or sin
// (kind 1) (k pi y / side) on [0, side]; the basis frequency k / (2 side) is
// (pad / 2) k on the torus grid: [E(j1 - pad k / 2) +- E(j1 + pad k / 2)] / (2 or 2i)
__global__ void k_dn_phi(double2* __restrict__ Phi, int mk, int Pn, double side, int pad) {
  const int kind = blockIdx.z, k = blockIdx.y;
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < Pn; j += gridDim.x * blockDim.x) {
    double2 r = make_double2(0, 0);
    if (j != Pn / 2 && !(kind == 1 && k == 0)) {
      const long long j1 = j < Pn / 2 ? j : j - Pn;
      const long long sh = (long long)(pad / 2) * k;
      const double2 em = eps_d(j1 - sh, side, pad), ep = eps_d(j1 + sh, side, pad);
      if (kind == 0) r = make_double2(0.5 * (em.x + ep.x), 0.5 * (em.y + ep.y));
      else r = make_double2(0.5 * (em.y - ep.y), -0.5 * (em.x - ep.x));
    }
    Phi[((size_t)kind * mk + k) * Pn + j] = r;
  }
}

// Af[kind][m * mk + k][ja] = sum over j1 = +-ja of X(m, j1) Phi(j1, k), ja < Pn/2;
// with conj_x, X(m, j1) = conj(Phi(j1, m)) (the outer integral taken exactly by
// Parseval's identity: the test function transformed like the trial function);
// grid (mk * mk * ceil(Pn/2 / 256), 1, 2)
template <typename T>
__global__ void k_dn_fold(const double2* __restrict__ X, const double2* __restrict__ Phi,
                          C<T>* __restrict__ Af, int mk, int Pn, int conj_x) {
  const int H = Pn / 2, hb = (H + 255) / 256;
  const int kind = blockIdx.z, mkk = blockIdx.x / hb, m = mkk / mk, k = mkk % mk;
  const int ja = (blockIdx.x % hb) * blockDim.x + threadIdx.x;
  if (ja >= H) return;
  const double2* x = (conj_x ? Phi : X) + ((size_t)kind * mk + m) * Pn;
  const double2* f = Phi + ((size_t)kind * mk + k) * Pn;
  auto xv = [&](int j) { return conj_x ? cconj<double>(x[j]) : x[j]; };
  double2 r = cmul<double>(xv(ja), f[ja]);
  if (ja > 0) r = cadd<double>(r, cmul<double>(xv(Pn - ja), f[Pn - ja]));
  Af[((size_t)kind * mk * mk + mkk) * H + ja] = conv<T>(r);
}

// ------------------------------------------------------------ complex GEMMs
// C[i][j] = alpha sum_k A(i, k) B(k, j) (+ C[i][j] if beta), A(i, k) at
// A[i sar + k sak], B(k, j) at B[k sbk + j sbc], C row-major (ldc): FP32 on
// the tensor cores (k_cgemm_tc below), FP64 on the FMA pipes (k_zgemm).
template <typename T> struct GemmArgsT {
  const C<T>* A;
  long long sar, sak;
  const C<T>* B;
  long long sbk, sbc;
  C<T>* C;
  long long ldc;
  int M, N, K;
  T alpha;
  int beta;
};
typedef GemmArgsT<float> GemmArgs;

// FP64: 64 x 64 outputs per CTA of 256 threads (4 x 4 per thread, strided by
// 16 so that the shared-memory reads are broadcasts or consecutive); k-tiles of 16
#define GZ_BM 64
#define GZ_BN 64
#define GZ_BK 16
__global__ void __launch_bounds__(256, 2) k_zgemm(GemmArgsT<double> g) {
  __shared__ double2 As[GZ_BK][GZ_BM + 1];
  __shared__ double2 Bs[GZ_BK][GZ_BN + 1];
  const int t = threadIdx.x, tr = t >> 4, tc = t & 15;
  const int i0 = blockIdx.y * GZ_BM, j0 = blockIdx.x * GZ_BN;
  double2 acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_double2(0.0, 0.0);
  const bool ak = g.sak == 1, bc = g.sbc == 1;
  for (int kb = 0; kb < g.K; kb += GZ_BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * 256;
      const int r = ak ? e >> 4 : e & (GZ_BM - 1), k = ak ? e & 15 : e >> 6;
      const int gi = i0 + r, gk = kb + k;
      As[k][r] = (gi < g.M && gk < g.K) ? g.A[gi * g.sar + gk * g.sak] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * 256;
      const int c = bc ? e & (GZ_BN - 1) : e >> 4, k = bc ? e >> 6 : e & 15;
      const int gj = j0 + c, gk = kb + k;
      Bs[k][c] = (gj < g.N && gk < g.K) ? g.B[gk * g.sbk + gj * g.sbc] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < GZ_BK; ++k) {
      double2 a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][tr + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tc + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[i][j].x = fma(a[i].x, b[j].x, fma(-a[i].y, b[j].y, acc[i][j].x));
          acc[i][j].y = fma(a[i].x, b[j].y, fma(a[i].y, b[j].x, acc[i][j].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gi = i0 + tr + 16 * i;
    if (gi >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gj = j0 + tc + 16 * j;
      if (gj >= g.N) continue;
      double2* c = g.C + gi * g.ldc + gj;
      double2 v = make_double2(g.alpha * acc[i][j].x, g.alpha * acc[i][j].y);
      if (g.beta) {
        const double2 o = *c;
        v.x += o.x;
        v.y += o.y;
      }
      *c = v;
    }
  }
}

// The FP32 GEMM on the fifth-generation tensor cores: the complex product as
// a real one, [Re C, Im C] = [Re A, Im A] [[Re B, Im B], [-Im B, Re B]]
// (each complex entry of B a 2 x 2 real block), with tcgen05.mma kind::tf32
// and FP32 accuracy from the three-product split (tc05.cuh).  One warpgroup
// per CTA computes 128 rows x 32 complex columns (M = 128, N = 64 real) in 128
// columns of tensor memory: hi hi in columns 0..63, the two corrections in
// 64..127, drained into FP32 registers every TC_DRAIN chunks.  Chunks of 8
// complex inner terms (16 real, two MMA k-steps, three products each) pass
// through two shared-memory buffers: the threads stage chunk c + 1 while the
// tensor cores multiply chunk c.  Thread t stages row t of the A tile and two
// entries of the B tile.  A wait that runs out sets g_gt_err, skips the
// output, and waits (bounded) for the MMAs in flight before the tensor memory
// is freed.  In the LU of an 8,216-unknown block the 128 rank-64 trailing updates
// take about 48 ms in total on this kernel, the same as on an FMA-pipe kernel
// with 128 x 64 tiles: with 64 inner terms a tile is bound by its staging and
// by the round trip of its C tile, not by the products.
#define GT_BN 32          // complex columns per CTA
#define GT_CH 8           // complex inner terms per chunk
struct GtBuf {
  float a_hi[2][128 * 8], a_lo[2][128 * 8];   // [k-step][K-major tile]
  float b_hi[2][64 * 8], b_lo[2][64 * 8];
};

__device__ int g_gt_err;  // set when a tensor-core wait of k_cgemm_tc ran out

__global__ void __launch_bounds__(128) k_cgemm_tc(GemmArgs g) {
  extern __shared__ __align__(128) unsigned char gtraw[];
  GtBuf* bufs = (GtBuf*)gtraw;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int i0 = blockIdx.y * 128, j0 = blockIdx.x * GT_BN;
  const int nch = (g.K + GT_CH - 1) / GT_CH;
  if (tid == 0) {
    tc_mbar_init(&mbar[0]);
    tc_mbar_init(&mbar[1]);
  }
  if (warp == 0) tc_alloc(&tslot, 128);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc_idesc_tf32(128, 64);
  bool ok = true;
  int last = -1;   // the last chunk whose MMAs were committed
  float racc[64];
#pragma unroll
  for (int n = 0; n < 64; ++n) racc[n] = 0.f;
  const int gi = i0 + tid;
  float2 va[GT_CH], vb[2];
  // B entries of this thread: (k = q / GT_BN, column q mod GT_BN), q = tid, tid + 128
  auto load_chunk = [&](int cn) {
    const int kb = cn * GT_CH;
#pragma unroll
    for (int u = 0; u < GT_CH; ++u)
      va[u] = (gi < g.M && kb + u < g.K) ? g.A[gi * g.sar + (long long)(kb + u) * g.sak]
                                         : make_float2(0.f, 0.f);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = tid + 128 * h, u = q / GT_BN, j = q % GT_BN;
      vb[h] = (j0 + j < g.N && kb + u < g.K) ? g.B[(long long)(kb + u) * g.sbk + (long long)(j0 + j) * g.sbc]
                                              : make_float2(0.f, 0.f);
    }
  };
  load_chunk(0);
  for (int c = 0; c < nch && ok; ++c) {
    const int b = c & 1;
    GtBuf& Bf = bufs[b];
    if (c >= 2) ok = tc_mbar_wait(&mbar[b], ((c - 2) >> 1) & 1);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    // A: row tid, complex inner term u -> real inner terms 2u (Re), 2u + 1 (Im)
#pragma unroll
    for (int u = 0; u < GT_CH; ++u) {
      uint32_t hr, lr, hi, li;
      tc_split(va[u].x, hr, lr);
      tc_split(va[u].y, hi, li);
      const int ks = u >> 2, k8 = (2 * u) & 7, off = tc_koff(tid, k8);
      *(uint2*)((char*)Bf.a_hi[ks] + off) = make_uint2(hr, hi);
      *(uint2*)((char*)Bf.a_lo[ks] + off) = make_uint2(lr, li);
    }
    // B (N x K, K-major): real rows n = 2j (Re C), 2j + 1 (Im C) against inner
    // terms k = 2u (Re A), 2u + 1 (Im A): (Re B, -Im B) and (Im B, Re B)
    {
      float2 bb[2] = {vb[0], vb[1]};
      if (c + 1 < nch) load_chunk(c + 1);   // in flight during the barrier and the MMAs
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int q = tid + 128 * h, u = q / GT_BN, j = q % GT_BN;
        const int ks = u >> 2, k8 = (2 * u) & 7;
        uint32_t h0, l0, h1, l1, h2, l2;
        tc_split(bb[h].x, h0, l0);
        tc_split(bb[h].y, h1, l1);
        tc_split(-bb[h].y, h2, l2);
        *(uint2*)((char*)Bf.b_hi[ks] + tc_koff(2 * j, k8)) = make_uint2(h0, h2);
        *(uint2*)((char*)Bf.b_lo[ks] + tc_koff(2 * j, k8)) = make_uint2(l0, l2);
        *(uint2*)((char*)Bf.b_hi[ks] + tc_koff(2 * j + 1, k8)) = make_uint2(h1, h0);
        *(uint2*)((char*)Bf.b_lo[ks] + tc_koff(2 * j + 1, k8)) = make_uint2(l1, l0);
      }
    }
    tc_fence_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ah = tc_desc(Bf.a_hi[ks]), al = tc_desc(Bf.a_lo[ks]);
        const uint64_t bh = tc_desc(Bf.b_hi[ks]), bl = tc_desc(Bf.b_lo[ks]);
        const uint32_t acc = (c % TC_DRAIN != 0 || ks > 0) ? 1u : 0u;
        tc_mma(tmem, ah, bh, idesc, acc);          // hi hi
        tc_mma(tmem + 64, al, bh, idesc, acc);     // the corrections apart
        tc_mma(tmem + 64, ah, bl, idesc, 1u);
      }
      tc_commit(&mbar[b]);
    }
    last = c;
    if (c % TC_DRAIN == TC_DRAIN - 1 || c == nch - 1) {
      ok = __syncthreads_and(tc_mbar_wait(&mbar[b], (c >> 1) & 1));
      tc_after_sync();
      if (ok) {
        const uint32_t lane = (uint32_t)(32 * warp) << 16;
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
          float x[32], y[32];
          tc_ld32(tmem + lane + 32 * hh, x);
          tc_ld32(tmem + lane + 64 + 32 * hh, y);
#pragma unroll
          for (int q = 0; q < 32; ++q) racc[32 * hh + q] += x[q] + y[q];
        }
      }
      tc_before_sync();
      __syncthreads();
    }
  }
  if (ok) {
    if (gi < g.M) {
      float2* crow = g.C + gi * g.ldc + j0;
      const int nj = min(GT_BN, g.N - j0);
      // all loads of the row first (independent, in flight together), then the stores
      float2 o[GT_BN];
#pragma unroll
      for (int j = 0; j < GT_BN; ++j)
        o[j] = (g.beta && j < nj) ? crow[j] : make_float2(0.f, 0.f);
#pragma unroll
      for (int j = 0; j < GT_BN; ++j)
        if (j < nj)
          crow[j] = make_float2(g.alpha * racc[2 * j] + o[j].x, g.alpha * racc[2 * j + 1] + o[j].y);
    }
  } else if (tid == 0) {
    atomicExch(&g_gt_err, 1);
    tc_settle(mbar, last);   // MMAs in flight end before the tensor memory is freed
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 128);
}

static std::atomic<bool> g_gt_smem{false};

// the tensor-core GEMM's timeout flag: cleared before a dense step, read after it
static cavity_status gt_err_clear(cavity_ctx* ctx) {
  const int zero = 0;
  CK(cudaMemcpyToSymbolAsync(g_gt_err, &zero, sizeof(int), 0, cudaMemcpyHostToDevice, ctx->stream));
  return CAVITY_OK;
}
static cavity_status gt_err_check(cavity_ctx* ctx) {
  int terr = 0;
  CK(cudaMemcpyFromSymbolAsync(&terr, g_gt_err, sizeof(int), 0, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (terr) {
    ctx->err = "dense kept block: a tensor-core wait of the GEMM timed out";
    return CAVITY_ETIMEOUT;
  }
  return CAVITY_OK;
}

static cavity_status cgemm(cavity_ctx* ctx, const GemmArgs& a, int cls) {
  if (a.M <= 0 || a.N <= 0) return CAVITY_OK;
  if (!g_gt_smem) {
    CK(cudaFuncSetAttribute(k_cgemm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(2 * sizeof(GtBuf))));
    g_gt_smem = true;
  }
  KScope ks_(ctx, cls);
  k_cgemm_tc<<<dim3(nblk(a.N, GT_BN), nblk(a.M, 128)), 128, 2 * sizeof(GtBuf), ctx->stream>>>(a);
  CK(cudaGetLastError());
  return CAVITY_OK;
}
static cavity_status cgemm(cavity_ctx* ctx, const GemmArgsT<double>& a, int cls) {
  if (a.M <= 0 || a.N <= 0) return CAVITY_OK;
  KScope ks_(ctx, cls);
  k_zgemm<<<dim3(nblk(a.N, GZ_BN), nblk(a.M, GZ_BM)), 256, 0, ctx->stream>>>(a);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// ------------------------------------------------------------ kept block
__device__ __forceinline__ double2 to_d2(float2 a) { return to_d(a); }
__device__ __forceinline__ double2 to_d2(double2 a) { return a; }

struct AsmP {
  int nk, n1k, n2k, mk, nkk;   // kept sizes; mk = mm + 1, nkk = nn + 1
  int nn, N, gn1, gn2, nap;    // full-index layout
  double pa, pb, h, ab, k2;
};

// A[r][c] of the kept block: the TBC rows from the integrals Ics, Isc, Icc
// ([(m, k1)][(n, k2)], FP32) and the cavity part from top (tau of every
// unknown, then varsigma of the E1 and E2 unknowns); grid (ceil(nk/256), nk)
template <typename T>
__global__ void k_dn_assemble(const C<T>* __restrict__ Ics, const C<T>* __restrict__ Isc,
                              const C<T>* __restrict__ Icc, const double2* __restrict__ top,
                              C<T>* __restrict__ A, int lda, AsmP p) {
  const int r = blockIdx.y;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= p.nk) return;
  // decode row and column: component (0, 1, 2) and mode
  auto decode = [&](int i, int& comp, int& m, int& n) {
    if (i < p.n1k) { comp = 0; m = i / p.nn; n = i % p.nn + 1; }
    else if (i < p.n1k + p.n2k) { i -= p.n1k; comp = 1; m = i / (p.nn + 1) + 1; n = i % (p.nn + 1); }
    else { i -= p.n1k + p.n2k; comp = 2; m = i / p.nn + 1; n = i % p.nn + 1; }
  };
  int cr, m, n, cc, k1, k2;
  decode(r, cr, m, n);
  decode(c, cc, k1, k2);
  const bool same = m == k1 && n == k2;
  const size_t npy = (size_t)p.nkk * p.nkk;
  const size_t o = ((size_t)m * p.mk + k1) * npy + (size_t)n * p.nkk + k2;
  const double s1 = p.h / (m == 0 ? p.ab / 2 : p.ab / 4), s2 = p.h / (n == 0 ? p.ab / 2 : p.ab / 4);
  const double mpa = m * p.pa, npb = n * p.pb, k1pa = k1 * p.pa, k2pb = k2 * p.pb;
  double2 v = make_double2(0, 0);
  if (cr == 0) {
    const int i1 = m * p.N + (n - 1);
    if (cc == 0) {
      const double2 a = to_d2(Ics[o]), w = to_d2(Icc[o]);
      v.x = s1 * (p.k2 * a.x - 2 * npb * k2pb * w.x);
      v.y = s1 * (p.k2 * a.y - 2 * npb * k2pb * w.y);
      if (same) v = cadd<double>(v, cadd<double>(make_double2(-1, 0), top[i1]));
    } else if (cc == 1) {
      const double2 w = to_d2(Icc[o]);
      v = make_double2(s1 * 2 * npb * k1pa * w.x, s1 * 2 * npb * k1pa * w.y);
    } else if (same) {
      v = cadd<double>(make_double2(mpa * p.h, 0), top[p.nap + i1]);
    }
  } else if (cr == 1) {
    const int i2 = p.gn1 + (m - 1) * (p.N + 1) + n;
    if (cc == 0) {
      const double2 w = to_d2(Icc[o]);
      v = make_double2(s2 * 2 * mpa * k2pb * w.x, s2 * 2 * mpa * k2pb * w.y);
    } else if (cc == 1) {
      const double2 a = to_d2(Isc[o]), w = to_d2(Icc[o]);
      v.x = s2 * (p.k2 * a.x - 2 * mpa * k1pa * w.x);
      v.y = s2 * (p.k2 * a.y - 2 * mpa * k1pa * w.y);
      if (same) v = cadd<double>(v, cadd<double>(make_double2(-1, 0), top[i2]));
    } else if (same) {
      v = cadd<double>(make_double2(npb * p.h, 0), top[p.nap + i2]);
    }
  } else if (same) {
    const int i3 = p.gn1 + p.gn2 + (m - 1) * p.N + (n - 1);
    if (cc == 0) v = make_double2(mpa * p.h, 0);
    else if (cc == 1) v = make_double2(npb * p.h, 0);
    else v = cadd<double>(make_double2(-1, 0), top[i3]);
  }
  A[(size_t)r * lda + c] = conv<T>(v);
}

static size_t al256(size_t v) { return (v + 255) / 256 * 256; }

template <typename T> static const C<T>* khat_of(const cavity_ctx* ctx);
template <> const float2* khat_of<float>(const cavity_ctx* ctx) { return ctx->khat32; }
template <> const double2* khat_of<double>(const cavity_ctx* ctx) { return ctx->khat64; }

// the kept block ks in precision T under the context's outer rule
template <typename T>
static cavity_status dense_assemble_t(cavity_ctx* ctx, const KeptSet& ks, C<T>* a, int lda) {
  const Geo& g = ctx->g;
  if (!ctx->prepared) {
    ctx->err = "dense assembly: call cavity_prepare first";
    return CAVITY_EINVAL;
  }
  if (ks.nk > CAVITY_DENSE_MAX_N || lda < ks.nk) {
    ctx->err = "dense assembly: kept block of " + std::to_string(ks.nk) +
               " unknowns exceeds the limit, or lda too small";
    return CAVITY_EINVAL;
  }
  const bool parseval = ctx->desc.outer_rule == CAVITY_OUTER_PARSEVAL;
  const int mk = ks.mm + 1, nkk = ks.nn + 1;
  const int Hx = g.Px / 2, Hy = g.Py / 2;
  const size_t npx = (size_t)mk * mk, npy = (size_t)nkk * nkk;
  // scratch: X, Phi per axis (FP64), folded factors, T per y kind, three I
  const size_t bx = al256(sizeof(double2) * 2 * mk * (size_t)g.Px);
  const size_t by = al256(sizeof(double2) * 2 * nkk * (size_t)g.Py);
  const size_t bfx = al256(sizeof(C<T>) * 2 * npx * Hx), bfy = al256(sizeof(C<T>) * 2 * npy * Hy);
  const size_t bt = al256(sizeof(C<T>) * (size_t)Hx * npy);
  const size_t bi = al256(sizeof(C<T>) * npx * npy);
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, 2 * bx + 2 * by + bfx + bfy + 2 * bt + 3 * bi));
  char* q = (char*)ctx->ws2;
  double2* Xx = (double2*)q; q += bx;
  double2* Fx = (double2*)q; q += bx;
  double2* Xy = (double2*)q; q += by;
  double2* Fy = (double2*)q; q += by;
  C<T>* Axf = (C<T>*)q; q += bfx;
  C<T>* Ayf = (C<T>*)q; q += bfy;
  C<T>* Tm[2];
  Tm[0] = (C<T>*)q; q += bt;
  Tm[1] = (C<T>*)q; q += bt;
  C<T>* I[3];
  for (int f = 0; f < 3; ++f) { I[f] = (C<T>*)q; q += bi; }
  cudaStream_t st = ctx->stream;
  if (!parseval) {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_x<<<dim3(nblk(g.Px, 256), mk, 2), 256, 0, st>>>(Xx, mk, g.nx, g.Px, g.a, ctx->tw64, ctx->TW);
  }
  {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_phi<<<dim3(nblk(g.Px, 256), mk, 2), 256, 0, st>>>(Fx, mk, g.Px, g.a, g.padx);
  }
  if (!parseval) {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_x<<<dim3(nblk(g.Py, 256), nkk, 2), 256, 0, st>>>(Xy, nkk, g.ny, g.Py, g.b, ctx->tw64, ctx->TW);
  }
  {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_phi<<<dim3(nblk(g.Py, 256), nkk, 2), 256, 0, st>>>(Fy, nkk, g.Py, g.b, g.pady);
  }
  {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_fold<T><<<dim3((unsigned)(npx * nblk(Hx, 256)), 1, 2), 256, 0, st>>>(Xx, Fx, Axf, mk, g.Px,
                                                                              parseval);
  }
  {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_fold<T><<<dim3((unsigned)(npy * nblk(Hy, 256)), 1, 2), 256, 0, st>>>(Xy, Fy, Ayf, nkk, g.Py,
                                                                              parseval);
  }
  CK(cudaGetLastError());
  // T[yk][j1][(n, k2)] = sum_j2 Kq[j2][j1] Ayf[yk][(n, k2)][j2]   (Kq: the quarter box, [j2][j1])
  for (int yk = 0; yk < 2; ++yk) {
    GemmArgsT<T> ga;
    ga.A = khat_of<T>(ctx); ga.sar = 1; ga.sak = Hx;
    ga.B = Ayf + (size_t)yk * npy * Hy; ga.sbk = 1; ga.sbc = Hy;
    ga.C = Tm[yk]; ga.ldc = (long long)npy;
    ga.M = Hx; ga.N = (int)npy; ga.K = Hy;
    ga.alpha = 1; ga.beta = 0;
    CKS(cgemm(ctx, ga, KC_DENSE_ASM));
  }
  // I_f[(m, k1)][(n, k2)] = sum_j1 Axf[xk][(m, k1)][j1] T[yk][j1][(n, k2)]
  // f = cs (x cos, y sin), sc (x sin, y cos), cc
  const int xk_of[3] = {0, 1, 0}, yk_of[3] = {1, 0, 0};
  for (int f = 0; f < 3; ++f) {
    GemmArgsT<T> ga;
    ga.A = Axf + (size_t)xk_of[f] * npx * Hx; ga.sar = Hx; ga.sak = 1;
    ga.B = Tm[yk_of[f]]; ga.sbk = (long long)npy; ga.sbc = 1;
    ga.C = I[f]; ga.ldc = (long long)npy;
    ga.M = (int)npx; ga.N = (int)npy; ga.K = Hx;
    ga.alpha = 1; ga.beta = 0;
    CKS(cgemm(ctx, ga, KC_DENSE_ASM));
  }
  AsmP p;
  p.nk = ks.nk; p.n1k = ks.n1; p.n2k = ks.n2; p.mk = mk; p.nkk = nkk;
  p.nn = ks.nn; p.N = g.N; p.gn1 = g.n1; p.gn2 = g.n2; p.nap = g.nap;
  p.pa = M_PI / g.a; p.pb = M_PI / g.b; p.h = g.h; p.ab = g.a * g.b;
  p.k2 = 2.0 * ctx->kappa0 * ctx->kappa0;
  {
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_assemble<T><<<dim3(nblk(ks.nk, 256), ks.nk), 256, 0, st>>>(I[0], I[1], I[2], ctx->top64, a,
                                                                     lda, p);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

cavity_status dense_assemble(cavity_ctx* ctx, const KeptSet& ks, float2* a, int lda) {
  CKS(gt_err_clear(ctx));
  CKS(dense_assemble_t<float>(ctx, ks, a, lda));
  return gt_err_check(ctx);
}

// ------------------------------------------------------------ LU factorisation
#define LU_NB 64          // panel width
#define LU_RMAX 32        // panel rows per CTA at most
#define LU_VS (LU_NB + 1) // row stride of the panel rows in shared memory
#define LU_THREADS 256
#define LU_SPIN (1 << 21) // polls of a grid barrier before it gives up

struct LuScr {
  unsigned long long* best;  // [n] per step: max over CTAs of the key of (|pivot|^2, row)
  float2* cand;       // [2][G][LU_NB] each CTA's candidate panel row
  float2* drow;       // [2][LU_NB] the panel row at the diagonal position
  unsigned int* bar;  // one counter per panel
  int* err;           // [0] barrier timeout; [1] first zero pivot (INT_MAX: none)
  int gmax;
};

// grid-wide barrier number `target / G`: returns false (and records the
// timeout) when the other CTAs do not arrive within LU_SPIN polls
__device__ __forceinline__ bool lu_grid_bar(unsigned int* cnt, unsigned int target, int* err) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(cnt, 1u);
    int good = 0;
    for (int it = 0; it < LU_SPIN; ++it) {
      unsigned int v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(cnt) : "memory");
      if (v >= target) { good = 1; break; }
      if (it > 256) __nanosleep(32);
    }
    if (!good) atomicExch(err, 1);
    ok = good;
  }
  __syncthreads();
  return ok != 0;
}

// key of a pivot candidate: |x|^2 in the high word (non-negative floats order
// like their bit patterns), the complement of the row in the low word (the
// smaller row wins a tie); 0 = no candidate
__device__ __forceinline__ unsigned long long lu_key(float m, int row) {
  return ((unsigned long long)__float_as_uint(m) << 32) | (unsigned int)(~row);
}

// Panel k0 .. k0 + nb - 1 over rows k0 .. n - 1; CTA c holds rows
// k0 + c R .. k0 + (c + 1) R - 1 in shared memory for the whole panel.  Per
// column: each CTA publishes its best row (atomicMax of its key into best[kj],
// the row itself into its candidate slot), one grid barrier, then every CTA
// reads the winning key, the winner's row (from the slot of the CTA that owns
// it) and the row at the diagonal position, exchanges the two and eliminates
// below the pivot in its own rows.
__global__ void __launch_bounds__(LU_THREADS) k_lu_panel(float2* __restrict__ A, int lda, int n,
                                                         int k0, int nb, int R,
                                                         int* __restrict__ ipiv, LuScr s,
                                                         unsigned int* bar) {
  extern __shared__ float2 v[];   // [R][LU_VS]: rows padded by one entry (column reads)
  __shared__ float2 prow[LU_NB], drow[LU_NB], lmul[LU_RMAX];
  __shared__ unsigned long long wk[LU_THREADS / 32];
  __shared__ int s_br, s_p;
  __shared__ float2 s_pinv;
  const int G = gridDim.x, c = blockIdx.x, t = threadIdx.x;
  const int r0 = k0 + c * R, r1 = min(r0 + R, n), nr = max(r1 - r0, 0);
  for (int e = t; e < nr * nb; e += LU_THREADS) {
    const int i = e / nb, k = e % nb;
    v[i * LU_VS + k] = A[(size_t)(r0 + i) * lda + k0 + k];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    const int kj = k0 + j, par = j & 1;
    // this CTA's candidate: largest |v[i][j]| over its rows i >= kj
    unsigned long long key = 0;
    for (int i = t; i < nr; i += LU_THREADS) {
      if (r0 + i < kj) continue;
      const float2 x = v[i * LU_VS + j];
      const unsigned long long kk = lu_key(x.x * x.x + x.y * x.y, r0 + i);
      key = kk > key ? kk : key;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long ok2 = __shfl_xor_sync(0xffffffffu, key, o);
      key = ok2 > key ? ok2 : key;
    }
    if ((t & 31) == 0) wk[t >> 5] = key;
    __syncthreads();
    if (t == 0) {
      for (int w = 1; w < LU_THREADS / 32; ++w) key = wk[w] > key ? wk[w] : key;
      s_br = key ? (int)(~(unsigned int)(key & 0xffffffffu)) : -1;
      if (key) atomicMax(&s.best[kj], key);
    }
    __syncthreads();
    if (s_br >= 0)
      for (int k = t; k < nb; k += LU_THREADS)
        __stcg(&s.cand[((size_t)par * G + c) * LU_NB + k], v[(s_br - r0) * LU_VS + k]);
    if (kj >= r0 && kj < r1)
      for (int k = t; k < nb; k += LU_THREADS) __stcg(&s.drow[par * LU_NB + k], v[(kj - r0) * LU_VS + k]);
    if (!lu_grid_bar(bar, (unsigned int)(j + 1) * G, s.err)) return;
    // the pivot: the best key over all CTAs; its row sits in the slot of the
    // CTA that owns it
    if (t == 0) {
      const unsigned long long b = __ldcg(&s.best[kj]);
      s_p = (int)(~(unsigned int)(b & 0xffffffffu));
    }
    __syncthreads();
    const int p = s_p, w = (p - k0) / R;
    for (int k = t; k < nb; k += LU_THREADS) {
      prow[k] = __ldcg(&s.cand[((size_t)par * G + w) * LU_NB + k]);
      drow[k] = __ldcg(&s.drow[par * LU_NB + k]);
    }
    __syncthreads();
    if (t == 0) {
      const float2 pv = prow[j];
      if (pv.x == 0.f && pv.y == 0.f) {
        atomicMin(&s.err[1], kj);
        s_pinv = make_float2(0.f, 0.f);
      } else {
        s_pinv = cdiv<float>(make_float2(1.f, 0.f), pv);
      }
      if (c == 0) ipiv[kj] = p;
    }
    // row exchange inside the panel: row kj takes the pivot row, row p the old row kj
    if (kj >= r0 && kj < r1)
      for (int k = t; k < nb; k += LU_THREADS) v[(kj - r0) * LU_VS + k] = prow[k];
    if (p != kj && p >= r0 && p < r1)
      for (int k = t; k < nb; k += LU_THREADS) v[(p - r0) * LU_VS + k] = drow[k];
    __syncthreads();
    const float2 pinv = s_pinv;
    for (int i = t; i < nr; i += LU_THREADS)
      if (r0 + i > kj) lmul[i] = cmul<float>(v[i * LU_VS + j], pinv);
    __syncthreads();
    // elimination below the pivot: thread t owns column t mod LU_NB and
    // every (LU_THREADS / LU_NB)-th row
    {
      const int k = t & (LU_NB - 1);
      if (k >= j && k < nb) {
        const float2 pk = prow[k];
        for (int i = t / LU_NB; i < nr; i += LU_THREADS / LU_NB) {
          if (r0 + i <= kj) continue;
          if (k == j) v[i * LU_VS + k] = lmul[i];
          else v[i * LU_VS + k] = csub<float>(v[i * LU_VS + k], cmul<float>(lmul[i], pk));
        }
      }
    }
    __syncthreads();
  }
  for (int e = t; e < nr * nb; e += LU_THREADS) {
    const int i = e / nb, k = e % nb;
    A[(size_t)(r0 + i) * lda + k0 + k] = v[i * LU_VS + k];
  }
}

// the panel's row exchanges on every column outside it
__global__ void k_lu_swap(float2* __restrict__ A, int lda, int n, int k0, int nb,
                          const int* __restrict__ ipiv) {
  const int col = blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= n || (col >= k0 && col < k0 + nb)) return;
  for (int j = 0; j < nb; ++j) {
    const int p = ipiv[k0 + j];
    if (p == k0 + j) continue;
    float2* a = A + (size_t)(k0 + j) * lda + col;
    float2* b = A + (size_t)p * lda + col;
    const float2 x = *a;
    *a = *b;
    *b = x;
  }
}

// U12 = L11^{-1} A12 for the block row of the panel, 32 columns per CTA
__global__ void __launch_bounds__(256) k_lu_trsm(float2* __restrict__ A, int lda, int n, int k0, int nb) {
  __shared__ float2 L[LU_NB][LU_NB + 1];
  __shared__ float2 X[LU_NB][33];
  const int t = threadIdx.x, cb = k0 + nb + blockIdx.x * 32;
  for (int e = t; e < nb * nb; e += 256) L[e / nb][e % nb] = A[(size_t)(k0 + e / nb) * lda + k0 + e % nb];
  for (int e = t; e < nb * 32; e += 256) {
    const int i = e >> 5, cc = e & 31, col = cb + cc;
    X[i][cc] = col < n ? A[(size_t)(k0 + i) * lda + col] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  for (int k = 0; k < nb - 1; ++k) {
    for (int e = t; e < (nb - 1 - k) * 32; e += 256) {
      const int i = k + 1 + (e >> 5), cc = e & 31;
      X[i][cc] = csub<float>(X[i][cc], cmul<float>(L[i][k], X[k][cc]));
    }
    __syncthreads();
  }
  for (int e = t; e < nb * 32; e += 256) {
    const int i = e >> 5, cc = e & 31, col = cb + cc;
    if (col < n) A[(size_t)(k0 + i) * lda + col] = X[i][cc];
  }
}

// perm = the row exchanges ipiv applied in order to 0..n-1 (one CTA).  An
// entry outside 0..n-1 is skipped and, when bad is given, *bad = 1 (else 0).
__global__ void k_lu_perm(const int* __restrict__ ipiv, int* __restrict__ perm, int n,
                          int* __restrict__ bad) {
  extern __shared__ int pm[];
  for (int i = threadIdx.x; i < n; i += blockDim.x) pm[i] = i;
  __syncthreads();
  if (threadIdx.x == 0) {
    int out = 0;
    for (int i = 0; i < n; ++i) {
      const int p = ipiv[i];
      if (p < 0 || p >= n) {
        out = 1;
        continue;
      }
      const int x = pm[i];
      pm[i] = pm[p];
      pm[p] = x;
    }
    if (bad) *bad = out;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) perm[i] = pm[i];
}

static std::atomic<bool> g_lu_smem{false};

cavity_status dense_lu(cavity_ctx* ctx, float2* a, int n, int lda, int* ipiv, int* info) {
  if (n < 1 || n > CAVITY_DENSE_MAX_N || lda < n || !a || !ipiv) {
    ctx->err = "LU: bad size or pointer";
    return CAVITY_EINVAL;
  }
  cudaStream_t st = ctx->stream;
  const int npanel = nblk(n, LU_NB);
  const int gmax = nblk(n, LU_RMAX);
  const size_t bbest = al256(sizeof(unsigned long long) * n);
  const size_t bcand = al256(sizeof(float2) * 2 * (size_t)gmax * LU_NB);
  const size_t bdrow = al256(sizeof(float2) * 2 * LU_NB), bbar = al256(sizeof(unsigned) * npanel);
  const size_t berr = al256(sizeof(int) * 2);
  CKS(ensure_ws(ctx, &ctx->dn_scr, &ctx->dn_scr_bytes, bbest + bcand + bdrow + bbar + berr));
  char* q = (char*)ctx->dn_scr;
  LuScr s;
  s.best = (unsigned long long*)q; q += bbest;
  s.cand = (float2*)q; q += bcand;
  s.drow = (float2*)q; q += bdrow;
  s.bar = (unsigned int*)q; q += bbar;
  s.err = (int*)q;
  s.gmax = gmax;
  CK(cudaMemsetAsync(s.bar, 0, sizeof(unsigned) * npanel, st));
  CK(cudaMemsetAsync(s.best, 0, sizeof(unsigned long long) * n, st));
  CKS(gt_err_clear(ctx));
  const int err0[2] = {0, INT_MAX};
  CK(cudaMemcpyAsync(s.err, err0, sizeof(err0), cudaMemcpyHostToDevice, st));
  if (!g_lu_smem) {
    CK(cudaFuncSetAttribute(k_lu_panel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(float2) * LU_RMAX * LU_VS)));
    CK(cudaFuncSetAttribute(k_lu_perm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(int) * CAVITY_DENSE_MAX_N)));
    g_lu_smem = true;
  }
  for (int p = 0; p < npanel; ++p) {
    const int k0 = p * LU_NB, nb = std::min(LU_NB, n - k0), H = n - k0;
    const int G = nblk(H, LU_RMAX), R = nblk(H, G);
    unsigned int* bar = s.bar + p;
    {
      KScope ks_(ctx, KC_DENSE_LU);
      void* args[] = {&a, &lda, &n, (void*)&k0, (void*)&nb, (void*)&R, &ipiv, &s, &bar};
      CK(cudaLaunchCooperativeKernel((const void*)k_lu_panel, dim3(G), dim3(LU_THREADS), args,
                                     sizeof(float2) * R * LU_VS, st));
    }
    if (n > nb) {
      KScope ks_(ctx, KC_DENSE_LU);
      k_lu_swap<<<nblk(n, 256), 256, 0, st>>>(a, lda, n, k0, nb, ipiv);
    }
    const int rest = n - k0 - nb;
    if (rest > 0) {
      {
        KScope ks_(ctx, KC_DENSE_LU);
        k_lu_trsm<<<nblk(rest, 32), 256, 0, st>>>(a, lda, n, k0, nb);
      }
      GemmArgs ga;
      ga.A = a + (size_t)(k0 + nb) * lda + k0; ga.sar = lda; ga.sak = 1;
      ga.B = a + (size_t)k0 * lda + k0 + nb; ga.sbk = lda; ga.sbc = 1;
      ga.C = a + (size_t)(k0 + nb) * lda + k0 + nb; ga.ldc = lda;
      ga.M = rest; ga.N = rest; ga.K = nb;
      ga.alpha = -1.f; ga.beta = 1;
      CKS(cgemm(ctx, ga, KC_DENSE_LU));
    }
    CK(cudaGetLastError());
  }
  int err[2];
  CK(cudaMemcpyAsync(err, s.err, sizeof(err), cudaMemcpyDeviceToHost, st));
  CKS(gt_err_check(ctx));
  if (err[0]) {
    ctx->err = "LU: a grid barrier of the panel factorisation timed out";
    return CAVITY_ETIMEOUT;
  }
  if (info) *info = err[1] == INT_MAX ? -1 : err[1];
  if (err[1] != INT_MAX) {
    ctx->err = "LU: zero pivot at step " + std::to_string(err[1]);
    return CAVITY_ESINGULAR;
  }
  return CAVITY_OK;
}

// ------------------------------------------------------------ triangular solves
#define TS_B 64   // rows per block
#define TS_D 16   // right-hand sides per sweep
#define TS_T (TS_B * (TS_B + 1))

// Inverses of the diagonal blocks of the factors, one CTA per block b:
// Dinv[b][0] = L_bb^{-1} (unit lower), Dinv[b][1] = U_bb^{-1}, 64 x 64 each,
// zero outside the block's nb x nb corner.
__global__ void __launch_bounds__(256) k_lu_dinv(const float2* __restrict__ A, int lda, int n,
                                                 float2* __restrict__ Dinv) {
  extern __shared__ float2 sm[];
  float2* M = sm;          // [TS_B][TS_B + 1]
  float2* R = sm + TS_T;
  const int t = threadIdx.x, b = blockIdx.x, r0 = b * TS_B, nb = min(TS_B, n - r0);
  for (int e = t; e < TS_B * TS_B; e += 256) {
    const int i = e / TS_B, k = e % TS_B;
    M[i * (TS_B + 1) + k] = (i < nb && k < nb) ? A[(size_t)(r0 + i) * lda + r0 + k] : make_float2(0.f, 0.f);
  }
  for (int up = 0; up < 2; ++up) {
    for (int e = t; e < TS_B * TS_B; e += 256) {
      const int i = e / TS_B, j = e % TS_B;
      R[i * (TS_B + 1) + j] = make_float2(i == j && i < nb ? 1.f : 0.f, 0.f);
    }
    __syncthreads();
    if (!up) {
      for (int k = 0; k < nb - 1; ++k) {
        for (int e = t; e < (nb - 1 - k) * nb; e += 256) {
          const int i = k + 1 + e / nb, j = e % nb;
          R[i * (TS_B + 1) + j] = csub<float>(R[i * (TS_B + 1) + j],
                                              cmul<float>(M[i * (TS_B + 1) + k], R[k * (TS_B + 1) + j]));
        }
        __syncthreads();
      }
    } else {
      for (int k = nb - 1; k >= 0; --k) {
        const float2 dk = M[k * (TS_B + 1) + k];
        for (int j = t; j < nb; j += 256) R[k * (TS_B + 1) + j] = cdiv<float>(R[k * (TS_B + 1) + j], dk);
        __syncthreads();
        for (int e = t; e < k * nb; e += 256) {
          const int i = e / nb, j = e % nb;
          R[i * (TS_B + 1) + j] = csub<float>(R[i * (TS_B + 1) + j],
                                              cmul<float>(M[i * (TS_B + 1) + k], R[k * (TS_B + 1) + j]));
        }
        __syncthreads();
      }
    }
    float2* o = Dinv + ((size_t)b * 2 + up) * TS_B * TS_B;
    for (int e = t; e < TS_B * TS_B; e += 256) o[e] = R[(e / TS_B) * (TS_B + 1) + e % TS_B];
    __syncthreads();
  }
}

// tile rows [q0, q0 + qn) x columns [r0, r0 + nb) of A into T (row stride TS_B + 1),
// 16 independent loads per thread in flight
__device__ __forceinline__ void trs_tile(const float2* __restrict__ A, int lda, int q0, int qn, int r0,
                                         int nb, float2* T) {
  float2 v[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = threadIdx.x + u * 256, i = e >> 6, k = e & 63;
    v[u] = (i < qn && k < nb) ? A[(size_t)(q0 + i) * lda + r0 + k] : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = threadIdx.x + u * 256;
    T[(e >> 6) * (TS_B + 1) + (e & 63)] = v[u];
  }
}
__device__ __forceinline__ void trs_dinv(const float2* __restrict__ D, float2* T) {
  float2 v[16];
#pragma unroll
  for (int u = 0; u < 16; ++u) v[u] = D[threadIdx.x + u * 256];
#pragma unroll
  for (int u = 0; u < 16; ++u) {
    const int e = threadIdx.x + u * 256;
    T[(e >> 6) * (TS_B + 1) + (e & 63)] = v[u];
  }
}

// One whole forward (L, unit diagonal) or backward (U) substitution for up to
// TS_D right-hand sides in one cooperative launch.  The rows are cut into
// blocks of TS_B; block q belongs to CTA q mod G.  Step s takes block b in
// order (backward: from the last): its owner forms x_b = D_b^{-1} y_b with the
// inverted diagonal block and writes it into Y; after a grid barrier every
// CTA subtracts A_qb x_b from each block q it owns further on (below for L,
// above for U).  The tiles a step needs do not depend on the solution, so each
// CTA loads the next step's tiles (its inverse block, its first coupling
// tile) between arriving at the barrier and waiting on it.  Y holds
// right-hand side d at Y + d ldy.  Waits are bounded: on a timeout the kernel
// records err and returns.
template <bool UPPER>
__global__ void __launch_bounds__(256, 1) k_trs_sweep(const float2* __restrict__ A, int lda, int n,
                                                      const float2* __restrict__ Dinv,
                                                      float2* __restrict__ Y, int ldy, int nd,
                                                      unsigned int* bar, int* err) {
  extern __shared__ float2 sm[];
  float2* Tb[2] = {sm, sm + TS_T};
  float2* Db[2] = {sm + 2 * TS_T, sm + 3 * TS_T};
  float2* X = sm + 4 * TS_T;                    // [TS_D][TS_B + 1]
  float2* Yb = X + TS_D * (TS_B + 1);           // owner's y_b
  __shared__ int ok;
  const int t = threadIdx.x, G = gridDim.x, c = blockIdx.x;
  const int nbk = (n + TS_B - 1) / TS_B;
  auto blk = [&](int s) { return UPPER ? nbk - 1 - s : s; };
  // first block this CTA owns beyond b in its update order, or -1
  auto first_after = [&](int b) {
    if (!UPPER) {
      int q = b + 1 + ((c - (b + 1)) % G + G) % G;
      return q < nbk ? q : -1;
    }
    int q = b - 1 - (((b - 1) - c) % G + G) % G;
    return q >= 0 ? q : -1;
  };
  auto prefetch = [&](int s) {
    if (s >= nbk) return;
    const int b = blk(s), r0 = b * TS_B, nb = min(TS_B, n - r0);
    if (b % G == c) trs_dinv(Dinv + ((size_t)b * 2 + (UPPER ? 1 : 0)) * TS_B * TS_B, Db[s & 1]);
    const int q = first_after(b);
    if (q >= 0) trs_tile(A, lda, q * TS_B, min(TS_B, n - q * TS_B), r0, nb, Tb[s & 1]);
  };
  prefetch(0);
  __syncthreads();
  for (int s = 0; s < nbk; ++s) {
    const int b = blk(s), r0 = b * TS_B, nb = min(TS_B, n - r0);
    if (b % G == c) {
      for (int e = t; e < nd * TS_B; e += 256) {
        const int d = e / TS_B, k = e % TS_B;
        Yb[d * (TS_B + 1) + k] = k < nb ? Y[(size_t)d * ldy + r0 + k] : make_float2(0.f, 0.f);
      }
      __syncthreads();
      const float2* D = Db[s & 1];
      for (int e = t; e < nd * nb; e += 256) {
        const int d = e / nb, i = e % nb;
        float2 acc = make_float2(0.f, 0.f);
        for (int k = 0; k < TS_B; ++k) {
          const float2 l = D[i * (TS_B + 1) + k], y = Yb[d * (TS_B + 1) + k];
          acc.x = fmaf(l.x, y.x, fmaf(-l.y, y.y, acc.x));
          acc.y = fmaf(l.x, y.y, fmaf(l.y, y.x, acc.y));
        }
        X[d * (TS_B + 1) + i] = acc;
        __stcg(&Y[(size_t)d * ldy + r0 + i], acc);
      }
    }
    // grid barrier: arrive, load the next step's tiles, then wait
    __syncthreads();
    if (t == 0) {
      __threadfence();
      atomicAdd(bar, 1u);
    }
    prefetch(s + 1);
    if (t == 0) {
      int good = 0;
      const unsigned int target = (unsigned int)(s + 1) * G;
      for (int it = 0; it < LU_SPIN; ++it) {
        unsigned int v;
        asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
        if (v >= target) { good = 1; break; }
        __nanosleep(32);
      }
      if (!good) atomicExch(err, 1);
      ok = good;
    }
    __syncthreads();
    if (!ok) return;
    if (b % G != c)
      for (int e = t; e < nd * nb; e += 256) {
        const int d = e / nb, k = e % nb;
        X[d * (TS_B + 1) + k] = __ldcg(&Y[(size_t)d * ldy + r0 + k]);
      }
    __syncthreads();
    // y_q -= A_qb x_b for the owned blocks beyond b; the first from the
    // prefetched tile, any further ones (n > G TS_B) straight from memory
    const int q1 = first_after(b);
    for (int q = q1; q >= 0 && q < nbk; q += UPPER ? -G : G) {
      const int q0 = q * TS_B, qn = min(TS_B, n - q0);
      const float2* T = Tb[s & 1];
      for (int e = t; e < qn * nd; e += 256) {
        const int i = e / nd, d = e % nd;
        float2 acc = make_float2(0.f, 0.f);
        if (q == q1) {
          for (int k = 0; k < nb; ++k) {
            const float2 l = T[i * (TS_B + 1) + k], x = X[d * (TS_B + 1) + k];
            acc.x = fmaf(l.x, x.x, fmaf(-l.y, x.y, acc.x));
            acc.y = fmaf(l.x, x.y, fmaf(l.y, x.x, acc.y));
          }
        } else {
          const float2* ar = A + (size_t)(q0 + i) * lda + r0;
          for (int k = 0; k < nb; ++k) {
            const float2 l = ar[k], x = X[d * (TS_B + 1) + k];
            acc.x = fmaf(l.x, x.x, fmaf(-l.y, x.y, acc.x));
            acc.y = fmaf(l.x, x.y, fmaf(l.y, x.x, acc.y));
          }
        }
        float2* y = Y + (size_t)d * ldy + q0 + i;
        *y = csub<float>(*y, acc);
      }
    }
    __syncthreads();
  }
}

static const size_t TRS_SMEM = sizeof(float2) * (4 * TS_T + 2 * TS_D * (TS_B + 1));
static std::atomic<bool> g_trs_smem{false};

// scratch of the substitutions: one barrier counter per sweep and an error flag
static size_t subst_scratch_bytes(int nrhs) {
  return al256(sizeof(unsigned int) * 2 * ((nrhs + TS_D - 1) / TS_D) + sizeof(int));
}
static size_t dinv_bytes(int n) { return sizeof(float2) * 2 * (size_t)TS_B * TS_B * ((n + TS_B - 1) / TS_B); }

static std::atomic<bool> g_dinv_smem{false};
static cavity_status launch_dinv(cavity_ctx* ctx, const float2* lu, int n, int lda, float2* dinv) {
  if (!g_dinv_smem) {
    CK(cudaFuncSetAttribute(k_lu_dinv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(float2) * 2 * TS_T)));
    g_dinv_smem = true;
  }
  KScope ks_(ctx, KC_DENSE_LU);
  k_lu_dinv<<<(n + TS_B - 1) / TS_B, 256, sizeof(float2) * 2 * TS_T, ctx->stream>>>(lu, lda, n, dinv);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// solves with the factors and the inverted diagonal blocks; Y holds P b on
// entry (rows already in pivot order); the caller reads *err (nonzero: a
// barrier timed out) after the stream
static cavity_status lu_substitute(cavity_ctx* ctx, const float2* lu, int n, int lda,
                                   const float2* dinv, int nrhs, float2* Y, int ldy, void* scratch) {
  cudaStream_t st = ctx->stream;
  if (!g_trs_smem) {
    CK(cudaFuncSetAttribute(k_trs_sweep<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRS_SMEM));
    CK(cudaFuncSetAttribute(k_trs_sweep<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TRS_SMEM));
    g_trs_smem = true;
  }
  const int nch = (nrhs + TS_D - 1) / TS_D;
  unsigned int* bars = (unsigned int*)scratch;
  int* err = (int*)(bars + 2 * nch);
  CK(cudaMemsetAsync(scratch, 0, sizeof(unsigned int) * 2 * nch + sizeof(int), st));
  const int nbk = (n + TS_B - 1) / TS_B;
  const int G = std::min(nbk, 148);
  for (int ch = 0; ch < nch; ++ch) {
    float2* y = Y + (size_t)ch * TS_D * ldy;
    int nd = std::min(TS_D, nrhs - ch * TS_D);
    for (int up = 0; up < 2; ++up) {
      unsigned int* bar = bars + 2 * ch + up;
      void* args[] = {(void*)&lu, &lda, &n, (void*)&dinv, &y, &ldy, &nd, &bar, &err};
      KScope ks_(ctx, KC_DENSE_TRS);
      CK(cudaLaunchCooperativeKernel(up ? (const void*)k_trs_sweep<true> : (const void*)k_trs_sweep<false>,
                                     dim3(G), dim3(256), args, TRS_SMEM, st));
    }
  }
  return CAVITY_OK;
}

// Y[d][i] = B[d][perm[i]] (grid (ceil(n/256), nrhs))
__global__ void k_lu_gather(const float2* __restrict__ B, int ldb, const int* __restrict__ perm,
                            float2* __restrict__ Y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i < n) Y[(size_t)d * n + i] = B[(size_t)d * ldb + perm[i]];
}
__global__ void k_lu_put(const float2* __restrict__ Y, float2* __restrict__ B, int ldb, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i < n) B[(size_t)d * ldb + i] = Y[(size_t)d * n + i];
}

cavity_status dense_lu_solve(cavity_ctx* ctx, const float2* lu, int n, int lda, const int* ipiv,
                             const int* perm, int nrhs, float2* y, int ldy) {
  if (n < 1 || n > CAVITY_DENSE_MAX_N || lda < n || ldy < n || nrhs < 1 || !lu || !ipiv || !y) {
    ctx->err = "LU solve: bad size or pointer";
    return CAVITY_EINVAL;
  }
  cudaStream_t st = ctx->stream;
  // scratch: the permutation (unless given) with its range flag, and the
  // permuted right-hand sides
  const size_t bp = al256(sizeof(int) * (n + 1)), by = al256(sizeof(float2) * (size_t)n * nrhs);
  const size_t bd = al256(dinv_bytes(n));
  CKS(ensure_ws(ctx, &ctx->ws, &ctx->ws_bytes, bp + by + bd + subst_scratch_bytes(nrhs)));
  int* pm = (int*)ctx->ws;
  float2* Y = (float2*)((char*)ctx->ws + bp);
  float2* dinv = (float2*)((char*)ctx->ws + bp + by);
  void* scr = (char*)ctx->ws + bp + by + bd;
  if (!g_lu_smem) {
    CK(cudaFuncSetAttribute(k_lu_perm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)(sizeof(int) * CAVITY_DENSE_MAX_N)));
    g_lu_smem = true;
  }
  if (!perm) {
    {
      KScope ks_(ctx, KC_DENSE_TRS);
      k_lu_perm<<<1, 256, sizeof(int) * n, st>>>(ipiv, pm, n, pm + n);
    }
    CK(cudaGetLastError());
    // a caller's ipiv is checked before b is touched
    int bad = 0;
    CK(cudaMemcpyAsync(&bad, pm + n, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (bad) {
      ctx->err = "LU solve: an ipiv entry is outside 0..n-1";
      return CAVITY_EINVAL;
    }
    perm = pm;
  }
  CKS(launch_dinv(ctx, lu, n, lda, dinv));
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_lu_gather<<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(y, ldy, perm, Y, n);
  }
  CKS(lu_substitute(ctx, lu, n, lda, dinv, nrhs, Y, n, scr));
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_lu_put<<<dim3(nblk(n, 256), nrhs), 256, 0, st>>>(Y, y, ldy, n);
  }
  CK(cudaGetLastError());
  int err = 0;
  CK(cudaMemcpyAsync(&err, (char*)scr + sizeof(unsigned int) * 2 * ((nrhs + TS_D - 1) / TS_D),
                     sizeof(int), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (err) {
    ctx->err = "LU solve: a grid barrier of the substitution timed out";
    return CAVITY_ETIMEOUT;
  }
  return CAVITY_OK;
}

// ------------------------------------------------------------ the dense path
void dense_free(DenseLU& f) {
  void* ptrs[] = {f.a, f.a64, f.dinv, f.ipiv, f.perm, f.map, f.work};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  f = DenseLU();
}

__global__ void k_dn_narrow(const double2* __restrict__ a64, float2* __restrict__ a, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) a[i] = to_f(a64[i]);
}

cavity_status dense_factor(cavity_ctx* ctx, DenseLU& f, const KeptSet& ks, bool keep64) {
  const Geo& g = ctx->g;
  f.ready = false;
  if (ks.nk > CAVITY_DENSE_MAX_N) {
    ctx->err = "dense kept block of " + std::to_string(ks.nk) +
               " unknowns, more than CAVITY_DENSE_MAX_N";
    return CAVITY_EINVAL;
  }
  const int lda = (ks.nk + 3) / 4 * 4;
  if (f.n != ks.nk || f.ks.mm != ks.mm || f.ks.nn != ks.nn || !f.a || (keep64 && !f.a64)) {
    dense_free(f);
    cudaError_t e = cudaMalloc(&f.a, sizeof(float2) * (size_t)ks.nk * lda);
    if (e == cudaSuccess) e = cudaMalloc(&f.ipiv, sizeof(int) * ks.nk);
    if (e == cudaSuccess) e = cudaMalloc(&f.perm, sizeof(int) * ks.nk);
    if (e == cudaSuccess) e = cudaMalloc(&f.map, sizeof(int) * ks.nk);
    if (e == cudaSuccess) e = cudaMalloc(&f.dinv, dinv_bytes(ks.nk));
    if (e == cudaSuccess && keep64) e = cudaMalloc(&f.a64, sizeof(double2) * (size_t)ks.nk * lda);
    if (e != cudaSuccess) {
      dense_free(f);
      ctx->err = std::string("dense kept block: allocation failed: ") + cudaGetErrorString(e);
      return CAVITY_ENOMEM;
    }
    const std::vector<int> map = kept_map(ks, g);
    CK(cudaMemcpy(f.map, map.data(), sizeof(int) * ks.nk, cudaMemcpyHostToDevice));
    f.ks = ks;
    f.n = ks.nk;
    f.lda = lda;
  }
  CKS(gt_err_clear(ctx));
  if (keep64) {
    CKS(dense_assemble_t<double>(ctx, ks, f.a64, lda));
    const long long tot = (long long)ks.nk * lda;
    KScope ks_(ctx, KC_DENSE_ASM);
    k_dn_narrow<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(f.a64, f.a, tot);
  } else {
    CKS(dense_assemble(ctx, ks, f.a, lda));
  }
  int info = -1;
  CKS(dense_lu(ctx, f.a, ks.nk, lda, f.ipiv, &info));
  {
    KScope ks_(ctx, KC_DENSE_LU);
    k_lu_perm<<<1, 256, sizeof(int) * ks.nk, ctx->stream>>>(f.ipiv, f.perm, ks.nk, nullptr);
  }
  CK(cudaGetLastError());
  CKS(launch_dinv(ctx, f.a, ks.nk, lda, f.dinv));
  CKS(gt_err_check(ctx));
  f.ready = true;
  return CAVITY_OK;
}

// The solver keeps the block in FP64 as well where the refinement takes its
// residual from it: always under the Parseval rule (the FFT operator
// implements rule D only) and for periods other than 4 sides (the FFT
// operator's layout), and on the FP64 path (one dense FP64 product per step
// is cheaper than the FP64 FFT operator on the full grid)
cavity_status launch_dense_factor(cavity_ctx* ctx) {
  const bool keep64 = ctx->desc.outer_rule == CAVITY_OUTER_PARSEVAL ||
                      ctx->desc.precision == CAVITY_FP64 || !ctx->g.fft_ok;
  return dense_factor(ctx, ctx->dn, kept_set(ctx->desc, ctx->g), keep64);
}

// r[d][map[i]] = b[d][map[i]] - sum_k A64[i][k] x[d][map[k]]: 64 rows x 16
// right-hand sides per CTA, k in tiles of 32 through shared memory
#define RS_R 64
#define RS_K 32
__global__ void __launch_bounds__(256) k_dn_resid(const double2* __restrict__ A, int lda, int nk,
                                                  const int* __restrict__ map, const double2* __restrict__ b,
                                                  const double2* __restrict__ x, double2* __restrict__ r,
                                                  int nap, int ndir) {
  __shared__ double2 As[RS_R][RS_K + 1];
  __shared__ double2 Xs[TS_D][RS_K + 1];
  const int t = threadIdx.x, row = t >> 2, g = t & 3;
  const int i0 = blockIdx.x * RS_R, d0 = blockIdx.y * TS_D;
  double2 acc[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) acc[u] = make_double2(0.0, 0.0);
  for (int kb = 0; kb < nk; kb += RS_K) {
#pragma unroll
    for (int u = 0; u < RS_R * RS_K / 256; ++u) {
      const int e = t + u * 256, i = e / RS_K, k = e % RS_K;
      As[i][k] = (i0 + i < nk && kb + k < nk) ? A[(size_t)(i0 + i) * lda + kb + k] : make_double2(0.0, 0.0);
    }
#pragma unroll
    for (int u = 0; u < TS_D * RS_K / 256; ++u) {
      const int e = t + u * 256, d = e / RS_K, k = e % RS_K;
      Xs[d][k] = (d0 + d < ndir && kb + k < nk) ? x[(size_t)(d0 + d) * nap + map[kb + k]]
                                                 : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < RS_K; ++k) {
      const double2 a = As[row][k];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const double2 v = Xs[g + 4 * u][k];
        acc[u].x = fma(a.x, v.x, fma(-a.y, v.y, acc[u].x));
        acc[u].y = fma(a.x, v.y, fma(a.y, v.x, acc[u].y));
      }
    }
    __syncthreads();
  }
  const int i = i0 + row;
  if (i >= nk) return;
  const int mi = map[i];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int d = d0 + g + 4 * u;
    if (d >= ndir) continue;
    const double2 bv = b[(size_t)d * nap + mi];
    r[(size_t)d * nap + mi] = make_double2(bv.x - acc[u].x, bv.y - acc[u].y);
  }
}

cavity_status dense_residual(cavity_ctx* ctx, int ndir, const double2* b, const double2* x,
                             double2* r) {
  const DenseLU& f = ctx->dn;
  if (!f.ready || !f.a64) {
    ctx->err = "dense residual: no FP64 kept block";
    return CAVITY_EINVAL;
  }
  KScope ks_(ctx, KC_DENSE_TRS);
  k_dn_resid<<<dim3(nblk(f.n, RS_R), nblk(ndir, TS_D)), 256, 0, ctx->stream>>>(
      f.a64, f.lda, f.n, f.map, b, x, r, ctx->g.nap, ndir);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// Y[d][i] = (float) (s[d] r[d][map[perm[i]]])  (grid (ceil(nk/256), ndir))
__global__ void k_dn_gather(const double2* __restrict__ r, int nap, const int* __restrict__ map,
                            const int* __restrict__ perm, const double* __restrict__ s,
                            float2* __restrict__ Y, int nk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i >= nk) return;
  const double2 v = r[(size_t)d * nap + map[perm[i]]];
  Y[(size_t)d * nk + i] = make_float2((float)(s[d] * v.x), (float)(s[d] * v.y));
}
// x[d][map[i]] += Y[d][i] / s[d]   (s[d] = 0: direction left alone)
__global__ void k_dn_scatter(double2* __restrict__ x, int nap, const int* __restrict__ map,
                             const double* __restrict__ s, const float2* __restrict__ Y, int nk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i >= nk || !(s[d] > 0)) return;
  const double f = 1.0 / s[d];
  const float2 v = Y[(size_t)d * nk + i];
  double2* o = x + (size_t)d * nap + map[i];
  o->x += f * (double)v.x;
  o->y += f * (double)v.y;
}

// y[d][map[perm^-1 ...]]: the coarse correction overwrites the coarse
// unknowns of y with the solution for the coarse unknowns of x
__global__ void k_cs_gather(const float2* __restrict__ x, long long xs, const int* __restrict__ map,
                            const int* __restrict__ perm, float2* __restrict__ Y, int nk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i < nk) Y[(size_t)d * nk + i] = x[(size_t)d * xs + map[perm[i]]];
}
__global__ void k_cs_put(const float2* __restrict__ Y, const int* __restrict__ map,
                         float2* __restrict__ y, long long ys, int nk) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (i < nk) y[(size_t)d * ys + map[i]] = Y[(size_t)d * nk + i];
}

cavity_status coarse_prepare(cavity_ctx* ctx) {
  const int mc = ctx->opt[CAVITY_OPT_COARSE_MODES];
  if (mc <= 0 || ctx->cs.ready) return CAVITY_OK;
  const KeptSet all = kept_set(ctx->desc, ctx->g);
  return dense_factor(ctx, ctx->cs, kept_set_of(std::min(mc, all.mm), std::min(mc, all.nn)));
}

cavity_status coarse_correct(cavity_ctx* ctx, int ndir, const float2* x, long long xs, float2* y,
                             long long ys) {
  DenseLU& f = ctx->cs;
  if (!f.ready || ctx->opt[CAVITY_OPT_COARSE_MODES] <= 0) return CAVITY_OK;
  const size_t need = al256(sizeof(float2) * (size_t)f.n * ndir) + subst_scratch_bytes(ndir);
  CKS(ensure_ws(ctx, &f.work, &f.work_bytes, need));
  float2* Y = (float2*)f.work;
  cudaStream_t st = ctx->stream;
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_cs_gather<<<dim3(nblk(f.n, 256), ndir), 256, 0, st>>>(x, xs, f.map, f.perm, Y, f.n);
  }
  CKS(lu_substitute(ctx, f.a, f.n, f.lda, f.dinv, ndir, Y, f.n,
                    (char*)f.work + al256(sizeof(float2) * (size_t)f.n * ndir)));
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_cs_put<<<dim3(nblk(f.n, 256), ndir), 256, 0, st>>>(Y, f.map, y, ys, f.n);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

size_t dense_inner_work_bytes(const cavity_ctx* ctx, int ndir) {
  const KeptSet ks = kept_set(ctx->desc, ctx->g);
  return al256(sizeof(float2) * (size_t)ks.nk * ndir) + subst_scratch_bytes(ndir);
}

int* dense_inner_err(const cavity_ctx* ctx, int ndir, void* work) {
  const KeptSet ks = kept_set(ctx->desc, ctx->g);
  return (int*)((char*)work + al256(sizeof(float2) * (size_t)ks.nk * ndir) +
                sizeof(unsigned int) * 2 * ((ndir + TS_D - 1) / TS_D));
}

cavity_status dense_inner_solve(cavity_ctx* ctx, int ndir, const double2* r, const double* s,
                                double2* x, void* work) {
  if (!ctx->dn.ready) {
    ctx->err = "dense aperture solve: no factorisation (cavity_prepare with the dense solver)";
    return CAVITY_EINVAL;
  }
  const int nk = ctx->dn.n;
  float2* Y = (float2*)work;
  cudaStream_t st = ctx->stream;
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_dn_gather<<<dim3(nblk(nk, 256), ndir), 256, 0, st>>>(r, ctx->g.nap, ctx->dn.map, ctx->dn.perm, s,
                                                          Y, nk);
  }
  CKS(lu_substitute(ctx, ctx->dn.a, nk, ctx->dn.lda, ctx->dn.dinv, ndir, Y, nk,
                    (char*)work + al256(sizeof(float2) * (size_t)nk * ndir)));
  {
    KScope ks_(ctx, KC_DENSE_TRS);
    k_dn_scatter<<<dim3(nblk(nk, 256), ndir), 256, 0, st>>>(x, ctx->g.nap, ctx->dn.map, s, Y, nk);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}
