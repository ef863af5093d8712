// Block GMRES in FP32 for the inner solves of the mixed-precision refinement.
//
// All incident directions of a solve share the operator, so their Krylov
// spaces are built together (block Arnoldi): the directions are split into
// groups of at most BG_MAX, and step k of a group extends its basis by the
// block A M^{-1} V_k of all its directions at once.  A direction's correction
// is then sought in the whole block space, which contains its own
// single-direction Krylov space of the same step count; the block solve reaches
// the inner tolerance in fewer operator applications (measured with the oracle
// on the 16-direction 64^2 and 128^2 workloads: 10-11 block steps against
// 13-14 per-direction steps to 1e-5).
//
// Orthogonalisation of the new block W against the basis V: one classical
// Gram-Schmidt pass as two GEMM-shaped tensor-core kernels, TF32 operands
// split into three products for FP32 accuracy.  W -= V H (k_bnn_tc5) runs on
// the fifth-generation tensor cores (tcgen05.mma kind::tf32, accumulators in
// tensor memory; tc05.cuh).  V^H W is a split reduction over the rows
// (k_bproj_tc, then k_bproj_final in a fixed order) on warp-level mma.sync: a
// tcgen05 version measured 2x slower, its threads having to split and place
// every element in the core-matrix layout of the reduction dimension, where
// the mma.sync version splits fragments in registers from tiles staged by
// cp.async.  The Gram matrix of the projected block is then formed
// (k_bproj_tc with W against itself) and the block is
// orthonormalised by Cholesky QR, or by SVQB (Stathopoulos and Wu, 2002:
// W = V' S with V' = W U Lambda^{-1/2} from G = W^H W = U Lambda U^H,
// eigenvalues below a floor raised to it) when it is nearly dependent
// (repeated incident directions, converged columns), so W = V' S holds
// exactly and nothing divides by ~0; a vanished block is an exact breakdown.
//
// The least-squares problems min || E_1 S_0 - Hbar Y || (block upper Hessenberg,
// one right-hand side per direction of the group) are solved on the host in
// FP64 by Householder reflections, one new column at a time; the norm of the
// tail of each transformed right-hand side is that direction's residual.
//
// Reductions are fixed-order trees, so the result is deterministic for a given
// batch; unlike per-direction GMRES it depends (within the tolerance) on which
// directions share a group.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <vector>

#include "bgmres_host.h"
#include "common.cuh"
#include "tc05.cuh"

#define BG_GROUPS 32      // groups per call (BG_GROUPS * BG_MAX directions)
#define BG_PART_CTAS 608  // bound on groups x row chunks of one projection

struct BGrp {
  const float2* V;  // Kv basis columns, stride nap
  const float2* W;  // r block columns, stride nap
  float2* O;        // output columns, stride nap (k_bnn_tc5)
  int Kv;           // columns taken from V (k_bnn_tc5 multiplies these)
  int K;            // projected columns (k_bproj_tc): V_0..V_{Kv-1}, then W_0..W_{K-Kv-1}
  int r;
  int coff;         // offset of this group's coefficient matrix (BG_MAX wide)
};
struct BGSet {
  BGrp g[BG_GROUPS];
};

#define BP_ROWS 128  // rows per staged tile (slabs are whole tiles)

__device__ __forceinline__ void cp_async8(float2* dst, const float2* src, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const int n = valid ? 8 : 0;  // 0: the 8 bytes are zero-filled
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// h[z][i][j] = sum over the nct slabs of part[z][x][i][j] in a fixed order.
// grid (K, groups), 256 threads: thread t adds the slabs x = t >> 4 (mod 16)
// of column j = t & 15 (16 consecutive threads read one 256-byte row of
// partials), and the 16 slab classes are added in class order.
__global__ void __launch_bounds__(256) k_bproj_final(BGSet set, const double2* __restrict__ part,
                                                     double2* __restrict__ h, int nct, int kcap) {
  __shared__ double2 q16[16][16];
  const BGrp& gd = set.g[blockIdx.y];
  const int i = blockIdx.x;
  if (i >= gd.K) return;  // uniform over the block
  const int t = threadIdx.x, j = t & 15, xg = t >> 4;
  double sx = 0, sy = 0;
  if (j < gd.r) {
#pragma unroll 4
    for (int x = xg; x < nct; x += 16) {
      const double2 v = part[((size_t)(blockIdx.y * nct + x) * kcap + i) * BG_MAX + j];
      sx += v.x;
      sy += v.y;
    }
  }
  q16[xg][j] = make_double2(sx, sy);
  __syncthreads();
  if (t < 16 && t < gd.r) {
    double ax = 0, ay = 0;
#pragma unroll
    for (int q = 0; q < 16; ++q) { ax += q16[q][t].x; ay += q16[q][t].y; }
    h[((size_t)blockIdx.y * kcap + i) * BG_MAX + t] = make_double2(ax, ay);
  }
}

// Block update: O_j[e] = beta O_j[e] + sgn sum_{i<Kv} V_i[e] C[i][j] for j < r
// (C: the group's coefficient matrix at cmat + coff, FP64, BG_MAX wide).  The
// complex product is a real GEMM,
//   [Re O_j, Im O_j] = sum_i [Re V_i, Im V_i] [[Re C_ij, Im C_ij], [-Im C_ij, Re C_ij]],
// of n_ap rows, 2 Kv inner terms and 32 outputs.
// It runs on the fifth-generation tensor cores (tcgen05.mma
// kind::tf32, accumulator in tensor memory; layouts and the TF32 split in
// tc05.cuh): grid (ceil(nap / 128), 1, groups), 128 threads (one warpgroup),
// the block's 128 rows x 32 real outputs in 32 columns of tensor memory.
// Chunks of T5_CH = 8 complex basis columns (16 real inner terms, two MMA
// k-steps, three products each) pass through two shared-memory buffers: the
// threads stage chunk c + 1 while the tensor cores multiply chunk c.  The
// products hi hi and the two corrections go to separate accumulators (32
// columns each), drained into FP32 registers every TC_DRAIN chunks (see
// tc05.cuh).  Thread
// t stages row row0 + t of V (eight 8-byte loads, one per column, a warp's
// 32 rows contiguous) and one complex coefficient (u, j) = (t / 16, t % 16)
// as its 2 x 2 real block.  A wait that runs out sets *err and skips the
// output.
#define T5_CH 8
struct T5Buf {
  float a_hi[2][128 * 8], a_lo[2][128 * 8];  // [k-step][K-major tile]
  float b_hi[2][32 * 8], b_lo[2][32 * 8];
};
__device__ int g_tc_err;  // set when a tensor-core wait ran out

__global__ void __launch_bounds__(128) k_bnn_tc5(BGSet set, const double2* __restrict__ cmat,
                                                 int nap, float beta, float sgn) {
  extern __shared__ __align__(128) unsigned char t5raw[];
  T5Buf* bufs = (T5Buf*)t5raw;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tslot;
  const BGrp& gd = set.g[blockIdx.z];
  const double2* Cm = cmat + gd.coff;
  const int Kv = gd.Kv, r = gd.r;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row0 = blockIdx.x * 128, e = row0 + tid;
  const int nch = (Kv + T5_CH - 1) / T5_CH;
  if (nch == 0) {  // uniform over the block: O = beta O
    if (e < nap)
      for (int j = 0; j < r; ++j) {
        float2* o = gd.O + (size_t)j * nap + e;
        const float2 ov = beta != 0.f ? *o : make_float2(0.f, 0.f);
        *o = make_float2(beta * ov.x, beta * ov.y);
      }
    return;
  }
  if (tid == 0) {
    tc_mbar_init(&mbar[0]);
    tc_mbar_init(&mbar[1]);
  }
  if (warp == 0) tc_alloc(&tslot, 64);
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  const uint32_t tmem = tslot;
  constexpr uint32_t idesc = tc_idesc_tf32(128, 32);
  bool ok = true;
  int last = -1;   // the last chunk whose MMAs were committed
  float racc[32];
#pragma unroll
  for (int n = 0; n < 32; ++n) racc[n] = 0.f;
  float2 v[T5_CH];
  double2 cnext;
  auto load_chunk = [&](int cn) {
#pragma unroll
    for (int u = 0; u < T5_CH; ++u) {
      const int i = cn * T5_CH + u;
      v[u] = (i < Kv && e < nap) ? gd.V[(size_t)i * nap + e] : make_float2(0.f, 0.f);
    }
    const int iu = cn * T5_CH + (tid >> 4), j = tid & 15;
    cnext = (iu < Kv && j < r) ? Cm[(size_t)iu * BG_MAX + j] : make_double2(0.0, 0.0);
  };
  load_chunk(0);
  for (int c = 0; c < nch && ok; ++c) {
    const int b = c & 1;
    T5Buf& B = bufs[b];
    // the MMAs of chunk c - 2 read this buffer
    if (c >= 2) ok = tc_mbar_wait(&mbar[b], ((c - 2) >> 1) & 1);
    ok = __syncthreads_and(ok);
    if (!ok) break;
    // A: row tid, complex columns i = c T5_CH + u -> real inner terms 2u, 2u + 1
    // (values loaded one iteration ahead)
#pragma unroll
    for (int u = 0; u < T5_CH; ++u) {
      uint32_t hr, lr, hi, li;
      tc_split(v[u].x, hr, lr);
      tc_split(v[u].y, hi, li);
      const int ks = u >> 2, k8 = (2 * u) & 7, off = tc_koff(tid, k8);
      *(uint2*)((char*)B.a_hi[ks] + off) = make_uint2(hr, hi);
      *(uint2*)((char*)B.a_lo[ks] + off) = make_uint2(lr, li);
    }
    // B (N x K, K-major): real rows n = 2j + c' against inner terms k = 2u + c
    {
      const int u = tid >> 4, j = tid & 15;
      const double2 cc = cnext;
      if (c + 1 < nch) load_chunk(c + 1);   // in flight during the barrier and the MMAs
      const float cr = (float)(sgn * cc.x), ci = (float)(sgn * cc.y);
      const int ks = u >> 2, k8 = (2 * u) & 7;
      uint32_t h0, l0, h1, l1, h2, l2;
      tc_split(cr, h0, l0);
      tc_split(ci, h1, l1);
      tc_split(-ci, h2, l2);
      // (n = 2j: k = 2u -> cr, k = 2u + 1 -> -ci), (n = 2j + 1: ci, cr)
      *(uint2*)((char*)B.b_hi[ks] + tc_koff(2 * j, k8)) = make_uint2(h0, h2);
      *(uint2*)((char*)B.b_lo[ks] + tc_koff(2 * j, k8)) = make_uint2(l0, l2);
      *(uint2*)((char*)B.b_hi[ks] + tc_koff(2 * j + 1, k8)) = make_uint2(h1, h0);
      *(uint2*)((char*)B.b_lo[ks] + tc_koff(2 * j + 1, k8)) = make_uint2(l1, l0);
    }
    tc_fence_smem();
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < 2; ++ks) {
        const uint64_t ah = tc_desc(B.a_hi[ks]), al = tc_desc(B.a_lo[ks]);
        const uint64_t bh = tc_desc(B.b_hi[ks]), bl = tc_desc(B.b_lo[ks]);
        const uint32_t acc = (c % TC_DRAIN != 0 || ks > 0) ? 1u : 0u;
        tc_mma(tmem, ah, bh, idesc, acc);         // hi hi
        tc_mma(tmem + 32, al, bh, idesc, acc);    // the corrections apart
        tc_mma(tmem + 32, ah, bl, idesc, 1u);
      }
      tc_commit(&mbar[b]);
    }
    last = c;
    if (c % TC_DRAIN == TC_DRAIN - 1 || c == nch - 1) {
      ok = __syncthreads_and(tc_mbar_wait(&mbar[b], (c >> 1) & 1));
      tc_after_sync();
      if (ok) tc_drain(tmem + ((uint32_t)(32 * warp) << 16), racc);
      tc_before_sync();
      __syncthreads();
    }
  }
  // every MMA done: the last chunk was drained
  if (ok) {
    const float* d = racc;
    if (e < nap) {
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        if (j >= r) break;
        float2* o = gd.O + (size_t)j * nap + e;
        const float2 ov = beta != 0.f ? *o : make_float2(0.f, 0.f);
        *o = make_float2(beta * ov.x + d[2 * j], beta * ov.y + d[2 * j + 1]);
      }
    }
  } else if (tid == 0) {
    atomicExch(&g_tc_err, 1);
    tc_settle(mbar, last);   // MMAs in flight end before the tensor memory is freed
  }
  tc_before_sync();
  __syncthreads();
  if (warp == 0) tc_dealloc(tmem, 64);
}

__device__ __forceinline__ unsigned tf32_of(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tf32_split(float x, unsigned& hi, unsigned& lo) {
  hi = tf32_of(x);
  lo = tf32_of(x - __uint_as_float(hi));
}
// D += A B for one 16 x 8 x 8 tile; fragments as in the PTX ISA for .tf32:
// lane = 4 g + t; a0 (g, t), a1 (g + 8, t), a2 (g, t + 4), a3 (g + 8, t + 4);
// b0 (t, g), b1 (t + 4, g); d0 (g, 2t), d1 (g, 2t + 1), d2 (g + 8, 2t), d3 (g + 8, 2t + 1)
__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Partial projections: part[z][x][i][j] = sum over the rows e of slab x of
// conj(X_i[e]) W_j[e] for group z, i < K, j < r, where X_i is basis column i
// for i < Kv and block column i - Kv after that, on the tensor pipe.
// With real columns m = 2 i + c of V (component c of column i) and n = 2 j + c'
// of W, the real product P = Vr^T Wr over the rows of a slab gives
//   Re H_ij = P(2i, 2j) + P(2i+1, 2j+1),   Im H_ij = P(2i, 2j+1) - P(2i+1, 2j)
// (H = V^H W), with the three-product TF32 split.  grid (nslab,
// ceil(K / 16), groups), 128 threads: the block owns 16 complex V columns (32
// real rows of P, two m16 tiles) against all 16 W columns (32 real, four n8
// tiles) over its slab, walked in 64-row tiles staged by cp.async into two
// buffers (row pitch 40 words: the fragment loads of a warp hit distinct
// banks); warp w takes rows 16 w .. 16 w + 15 of each tile, and the four
// warps' sums are added in warp order at the end.
#define TP_ROWS 64
#define TP_LD 40
#define TP_SMEM (sizeof(float) * 2 * 2 * TP_ROWS * TP_LD)
__global__ void __launch_bounds__(128, 4) k_bproj_tc(BGSet set, double2* __restrict__ part, int nap,
                                                  int rs, int nct, int kcap) {
  extern __shared__ __align__(16) float tsm[];  // [buf][V | W][row][TP_LD]
  const BGrp& gd = set.g[blockIdx.z];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  const int ib = blockIdx.y * 16, K = gd.K, Kv = gd.Kv, r = gd.r;
  const int e0 = blockIdx.x * rs, e1 = min(nap, e0 + rs);
  // staging: element q = tid + 128 u (u < 8) of a 64 x 16 tile has row bits
  // 0-1 from q bits 0-1 and bits 2-5 from q bits 6-9, column q bits 2-5; a
  // half-warp writes 4 rows x 4 columns (distinct banks at the 40-word pitch)
  // and a warp reads 8 whole 32-byte sectors
  auto stage = [&](int buf, int eb) {
    float* vs = tsm + (size_t)buf * 2 * TP_ROWS * TP_LD;
    float* ws = vs + TP_ROWS * TP_LD;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int q = tid + 128 * u, c = (q >> 2) & 15, el = (q & 3) | ((q >> 6) << 2);
      const int e = eb + el, i = ib + c;
      const bool in = e < e1;
      const float2* src = i < Kv ? gd.V + (size_t)i * nap : gd.W + (size_t)(i - Kv) * nap;
      cp_async8((float2*)(vs + el * TP_LD + 2 * c), (in && i < K) ? src + e : gd.W, in && i < K);
      cp_async8((float2*)(ws + el * TP_LD + 2 * c), (in && c < r) ? gd.W + (size_t)c * nap + e : gd.W,
                in && c < r);
    }
    cp_async_commit();
  };
  float acc[2][4][4];
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[mt][nt][q] = 0.f;
  const int ntile = (e1 - e0 + TP_ROWS - 1) / TP_ROWS;
  if (ntile > 0) stage(0, e0);
  if (ntile > 1) stage(1, e0 + TP_ROWS);
  for (int it = 0; it < ntile; ++it) {
    if (it + 1 < ntile) cp_async_wait<1>();
    else cp_async_wait<0>();
    __syncthreads();
    const float* vs = tsm + (size_t)(it & 1) * 2 * TP_ROWS * TP_LD;
    const float* ws = vs + TP_ROWS * TP_LD;
#pragma unroll 1
    for (int ks = 0; ks < 2; ++ks) {
      const int ea = warp * 16 + ks * 8 + t, eb = ea + 4;  // rows of the k8 step
      unsigned ahi[2][4], alo[2][4];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        // real rows m = 16 mt + g (+ 8): word 16 mt + g (+ 8) of a staged row
        const int w0 = 16 * mt + g;
        tf32_split(vs[ea * TP_LD + w0], ahi[mt][0], alo[mt][0]);
        tf32_split(vs[ea * TP_LD + w0 + 8], ahi[mt][1], alo[mt][1]);
        tf32_split(vs[eb * TP_LD + w0], ahi[mt][2], alo[mt][2]);
        tf32_split(vs[eb * TP_LD + w0 + 8], ahi[mt][3], alo[mt][3]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        unsigned bh0, bl0, bh1, bl1;
        tf32_split(ws[ea * TP_LD + 8 * nt + g], bh0, bl0);
        tf32_split(ws[eb * TP_LD + 8 * nt + g], bh1, bl1);
#pragma unroll
        for (int mt = 0; mt < 2; ++mt) {
          mma_tf32(acc[mt][nt], alo[mt], bh0, bh1);
          mma_tf32(acc[mt][nt], ahi[mt], bl0, bl1);
          mma_tf32(acc[mt][nt], ahi[mt], bh0, bh1);
        }
      }
    }
    __syncthreads();
    if (it + 2 < ntile) stage(it & 1, e0 + (it + 2) * TP_ROWS);
  }
  // P tiles of the four warps into shared memory: warp w's P(m, n) at
  // red[w][m][n] (32 x 33 floats), d0 (m = 16 mt + g, n = 8 nt + 2t), d1 n + 1,
  // d2, d3 at m + 8
  float* red = tsm;
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int m = 16 * mt + g, n = 8 * nt + 2 * t;
      float* rw = red + warp * 32 * 33;
      rw[m * 33 + n] = acc[mt][nt][0];
      rw[m * 33 + n + 1] = acc[mt][nt][1];
      rw[(m + 8) * 33 + n] = acc[mt][nt][2];
      rw[(m + 8) * 33 + n + 1] = acc[mt][nt][3];
    }
  __syncthreads();
  // thread -> 2 of the 256 complex outputs (i, j) of the tile
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int o = tid + 128 * h, li = o >> 4, lj = o & 15;
    if (ib + li >= K || lj >= r) continue;
    double pr = 0, pi = 0;
#pragma unroll
    for (int w = 0; w < 4; ++w) {
      const float* rw = red + w * 32 * 33;
      pr += (double)rw[(2 * li) * 33 + 2 * lj] + (double)rw[(2 * li + 1) * 33 + 2 * lj + 1];
      pi += (double)rw[(2 * li) * 33 + 2 * lj + 1] - (double)rw[(2 * li + 1) * 33 + 2 * lj];
    }
    part[((size_t)(blockIdx.z * nct + blockIdx.x) * kcap + ib + li) * BG_MAX + lj] = make_double2(pr, pi);
  }
}

// dst[map[c]] += src[c]  (column c of a contiguous block; grid (ceil(nap/256), ncol))
__global__ void k_scatter_add(const float2* __restrict__ src, float2* __restrict__ dst,
                              const int* __restrict__ map, int nap) {
  const int c = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  const float2 a = src[(size_t)c * nap + e];
  float2* o = dst + (size_t)map[c] * nap + e;
  *o = make_float2(o->x + a.x, o->y + a.y);
}

// dst[c] = src[map[c]]  (gather into a contiguous block)
__global__ void k_gather_cols(const float2* __restrict__ src, float2* __restrict__ dst,
                              const int* __restrict__ map, int nap) {
  const int c = blockIdx.y, e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nap) return;
  dst[(size_t)c * nap + e] = src[(size_t)map[c] * nap + e];
}

// dst[c] -= src[c]  (contiguous blocks; grid (ceil(nap/256), ncol))
__global__ void k_sub_cols(const float2* __restrict__ src, float2* __restrict__ dst, int nap) {
  const size_t k = (size_t)blockIdx.y * nap + blockIdx.x * blockDim.x + threadIdx.x;
  if (blockIdx.x * blockDim.x + threadIdx.x >= (unsigned)nap) return;
  dst[k] = make_float2(dst[k].x - src[k].x, dst[k].y - src[k].y);
}

static inline unsigned bg_blocks(long long n, int b) { return (unsigned)((n + b - 1) / b); }

// ------------------------------------------------------------------ host side
// (herm_eig, cholqr, svqb, matmul_left, BlockLS: bgmres_host.h)

struct BWork {
  float2 *V, *Rc, *Z, *Wb, *Tt;
  double2 *part, *hb, *cb;
  int* map;
  void* apw;
  int kcap, gmax;
};

static size_t al256(size_t x) { return (x + 255) / 256 * 256; }

// gw: directions per group (1..BG_MAX); a call takes up to BG_GROUPS groups
size_t block_inner_work_bytes(const Geo& g, int ndir, int mb, int gw) {
  const int nd = std::min(ndir, BG_GROUPS * gw);
  const int gm = (nd + gw - 1) / gw;
  const size_t kcap = (size_t)(mb + 1) * BG_MAX;
  const size_t col = sizeof(float2) * (size_t)g.nap;
  size_t b = 0;
  b += al256(col * gm * kcap);                              // V
  b += 4 * al256(col * nd);                                 // Rc, Z, Wb, Tt
  b += al256(sizeof(double2) * BG_PART_CTAS * kcap * BG_MAX);  // part
  b += al256(sizeof(double2) * 3 * gm * kcap * BG_MAX);      // hb
  b += al256(sizeof(double2) * gm * kcap * BG_MAX);          // cb
  b += al256(sizeof(int) * nd);                              // map
  b += al256(apply_work_bytes(g, nd, sizeof(float2)));
  return b;
}

static BWork bwork_carve(void* base, const Geo& g, int ndir, int mb, int gw) {
  const int nd = std::min(ndir, BG_GROUPS * gw);
  const int gm = (nd + gw - 1) / gw;
  const size_t kcap = (size_t)(mb + 1) * BG_MAX;
  const size_t col = sizeof(float2) * (size_t)g.nap;
  char* p = (char*)base;
  BWork w;
  w.V = (float2*)p; p += al256(col * gm * kcap);
  w.Rc = (float2*)p; p += al256(col * nd);
  w.Z = (float2*)p; p += al256(col * nd);
  w.Wb = (float2*)p; p += al256(col * nd);
  w.Tt = (float2*)p; p += al256(col * nd);
  w.part = (double2*)p; p += al256(sizeof(double2) * BG_PART_CTAS * kcap * BG_MAX);
  w.hb = (double2*)p; p += al256(sizeof(double2) * 3 * gm * kcap * BG_MAX);
  w.cb = (double2*)p; p += al256(sizeof(double2) * gm * kcap * BG_MAX);
  w.map = (int*)p; p += al256(sizeof(int) * nd);
  w.apw = p;
  w.kcap = (int)kcap;
  w.gmax = gm;
  return w;
}

// V^H W for every group of `set` (ng groups, K and r per group) into
// hb + slot * gmax * kcap * BG_MAX, laid out [z][i][j].
static void bproj(cavity_ctx* ctx, const BGSet& set, int ng, int kmax, const BWork& w, int slot) {
  const int nap = ctx->g.nap;
  const int ytiles = (kmax + 15) / 16;
  // slabs of rows such that slabs x column tiles x groups fill one wave of
  // resident blocks (four per SM, BG_PART_CTAS in all): no tail wave, and a
  // short projection (the Gram matrix, K = 16) still spreads over every SM
  int nct = std::max(1, BG_PART_CTAS / (ytiles * ng));
  nct = std::min(nct, (nap + BP_ROWS - 1) / BP_ROWS);
  int rs = (nap + nct - 1) / nct;
  rs = (rs + BP_ROWS - 1) / BP_ROWS * BP_ROWS;
  nct = (nap + rs - 1) / rs;
  double2* h = w.hb + (size_t)slot * w.gmax * w.kcap * BG_MAX;
  static std::atomic<bool> done{false};  // set once; host threads may race
  if (!done) {
    cudaFuncSetAttribute(k_bproj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TP_SMEM);
    done = true;
  }
  {
    KScope ks_(ctx, KC_KRYLOV);
    k_bproj_tc<<<dim3(nct, ytiles, ng), 128, TP_SMEM, ctx->stream>>>(set, w.part, nap, rs, nct,
                                                                     w.kcap);
  }
  {
    KScope ks_(ctx, KC_KRYLOV);
    k_bproj_final<<<dim3(kmax, ng), 256, 0, ctx->stream>>>(set, w.part, h, nct, w.kcap);
  }
}

static cavity_status bnn(cavity_ctx* ctx, const BGSet& set, int ng, const double2* cmat, float beta,
                         float sgn) {
  const int nap = ctx->g.nap;
  KScope ks_(ctx, KC_KRYLOV);
  k_bnn_tc5<<<dim3(bg_blocks(nap, 128), 1, ng), 128, 2 * sizeof(T5Buf), ctx->stream>>>(
      set, cmat, nap, beta, sgn);
  return CAVITY_OK;
}

// Solves A M^{-1} y = r_d for the directions with active[d] (r: ndir scaled
// FP32 residual columns), accumulating d = M^{-1} y into the d columns (zeroed
// first).  tol[d] is the relative target (the columns have unit norm); iters[d]
// is increased by the block steps taken, est[d] is the final least-squares
// residual.  Groups still above tolerance after mb steps restart from their
// true inner residual.
cavity_status run_block_inner(cavity_ctx* ctx, int ndir, const float2* r, float2* d,
                              const std::vector<double>& tol, const std::vector<char>& active, int mb,
                              int maxit, void* work, std::vector<int>& iters,
                              std::vector<double>& est) {
  const Geo& g = ctx->g;
  const int nap = g.nap;
  cudaStream_t st = ctx->stream;
  CK(cudaMemsetAsync(d, 0, sizeof(float2) * (size_t)ndir * nap, st));
  std::vector<int> all;
  for (int q = 0; q < ndir; ++q)
    if (active[q]) all.push_back(q);
  est.assign(ndir, 0.0);
  // directions beyond one call's capacity are solved in further batches
  const int gw = std::max(1, std::min(BG_MAX, ctx->opt[CAVITY_OPT_GROUP_WIDTH]));
  for (size_t b0 = 0; b0 < all.size(); b0 += (size_t)BG_GROUPS * gw) {
    const int na = (int)std::min(all.size() - b0, (size_t)BG_GROUPS * gw);
    std::vector<int> dirs(all.begin() + b0, all.begin() + b0 + na);
    BWork w = bwork_carve(work, g, ndir, mb, gw);
    const int ng = (na + gw - 1) / gw;
    // balanced groups: group z holds directions [goff[z], goff[z] + gr[z])
    std::vector<int> gr(ng), goff(ng);
    for (int z = 0, o = 0; z < ng; ++z) {
      gr[z] = na / ng + (z < na % ng ? 1 : 0);
      goff[z] = o;
      o += gr[z];
    }
    CK(cudaMemcpyAsync(w.map, dirs.data(), sizeof(int) * na, cudaMemcpyHostToDevice, st));
    {
      KScope ks_(ctx, KC_KRYLOV);
      k_gather_cols<<<dim3(bg_blocks(nap, 256), na), 256, 0, st>>>(r, w.Rc, w.map, nap);
    }
    std::vector<char> gdone(ng, 0);
    int used = 0;
    auto Vg = [&](int z) { return w.V + (size_t)z * w.kcap * nap; };
    auto hptr = [&](int slot, int z) {
      return w.hb + ((size_t)slot * w.gmax + z) * w.kcap * BG_MAX;
    };
    const size_t hsz = (size_t)w.kcap * BG_MAX;
    // pinned staging: three fetched coefficient slots, then the upload slot;
    // an upload is rewritten only after a stream synchronisation that follows
    // the previous one
    CKS(ensure_pin(ctx, sizeof(double2) * 4 * w.gmax * hsz));
    double2* hh = (double2*)ctx->pin;
    double2* cup = hh + (size_t)3 * w.gmax * hsz;
    bool upl_pending = false;  // an upload may still be queued behind GPU work
    auto sync = [&]() -> cavity_status {
      CK(cudaStreamSynchronize(st));
      upl_pending = false;
      return CAVITY_OK;
    };
    auto fetch = [&](int slot) -> cavity_status {
      CK(cudaMemcpyAsync(hh + (size_t)slot * w.gmax * hsz, hptr(slot, 0),
                         sizeof(double2) * ng * hsz, cudaMemcpyDeviceToHost, st));
      return CAVITY_OK;
    };
    auto hval = [&](int slot, int z, int i, int j) {
      const double2 t = hh[(size_t)slot * w.gmax * hsz + (size_t)z * hsz + (size_t)i * BG_MAX + j];
      return cd(t.x, t.y);
    };
    auto upload = [&](const std::vector<std::vector<cd>>& mats, const std::vector<int>& zs) -> cavity_status {
      if (upl_pending) CKS(sync());
      for (size_t q = 0; q < zs.size(); ++q) {
        const auto& m = mats[q];
        for (size_t t = 0; t < m.size(); ++t)
          cup[(size_t)zs[q] * hsz + t] = make_double2(m[t].real(), m[t].imag());
      }
      CK(cudaMemcpyAsync(w.cb, cup, sizeof(double2) * ng * hsz, cudaMemcpyHostToDevice, st));
      upl_pending = true;
      return CAVITY_OK;
    };
    // Orthonormalise block columns [col0, col0 + r) of each listed group's
    // basis in place by repeated SVQB; S[z] receives the r x r factor with
    // old block = new block * S.  G0, when given, holds the Gram matrices of
    // the blocks as they are (first pass without a device Gram).
    auto orthonormalise = [&](const std::vector<int>& zs, const std::vector<int>& col0,
                              std::vector<std::vector<cd>>& S,
                              const std::vector<std::vector<cd>>* G0) -> cavity_status {
      const int nz = (int)zs.size();
      S.assign(nz, {});
      std::vector<char> ok(nz, 0);
      for (int pass = 0; pass < 4; ++pass) {
        std::vector<int> todo;
        for (int q = 0; q < nz; ++q)
          if (!ok[q]) todo.push_back(q);
        if (todo.empty()) break;
        if (pass > 0 || !G0) {
          BGSet set;
          for (size_t t = 0; t < todo.size(); ++t) {
            const int q = todo[t], z = zs[q];
            float2* blk = Vg(z) + (size_t)col0[q] * nap;
            set.g[t] = BGrp{blk, blk, blk, 0, gr[z], gr[z], 0};
          }
          bproj(ctx, set, (int)todo.size(), BG_MAX, w, 2);
          CKS(fetch(2));
          CKS(sync());
        }
        std::vector<std::vector<cd>> Ts(todo.size());
        std::vector<int> tz;
        BGSet set2;
        int n2 = 0;
        for (size_t t = 0; t < todo.size(); ++t) {
          const int q = todo[t], z = zs[q], n = gr[z];
          std::vector<cd> G((size_t)n * n);
          if (pass == 0 && G0) G = (*G0)[q];
          else
            for (int i = 0; i < n; ++i)
              for (int j = 0; j < n; ++j) G[(size_t)i * n + j] = hval(2, (int)t, i, j);
          double dev = 0;
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
              dev = std::max(dev, std::abs(G[(size_t)i * n + j] - (i == j ? 1.0 : 0.0)));
          if (pass > 0 && dev <= 2e-6) {
            ok[q] = 1;
            continue;
          }
          // Cholesky QR; its FP32 transform leaves an orthogonality error
          // within the block of ~ eps32 cond(G), accepted without a check for
          // cond(G) <= 1e3: it perturbs the least-squares residual norms by
          // that relative amount, far below the inner tolerance, while the
          // orthogonality to the earlier blocks comes from the two
          // Gram-Schmidt passes.  Nearly dependent blocks take the
          // eigendecomposition and further passes.
          std::vector<cd> T, Sk;
          double cond = 1e300, ratio;
          if (cholqr(G, n, T, Sk, cond)) {
            if (cond <= 1e3) ok[q] = 1;
          } else {
            svqb(G, n, T, Sk, ratio);
          }
          if (S[q].empty()) S[q] = Sk;
          else matmul_left(Sk, S[q], n);
          Ts[n2] = T;
          tz.push_back(n2);
          float2* blk = Vg(z) + (size_t)col0[q] * nap;
          set2.g[n2] = BGrp{blk, blk, blk, n, n, n, n2 * (int)hsz};
          ++n2;
        }
        if (n2 == 0) break;
        Ts.resize(n2);
        CKS(upload(Ts, tz));
        CKS(bnn(ctx, set2, n2, w.cb, 0.f, 1.f));
      }
      for (int q = 0; q < nz; ++q)
        if (S[q].empty()) {  // first pass always transforms, so this is unreachable
          const int n = gr[zs[q]];
          S[q].assign((size_t)n * n, cd(0, 0));
          for (int i = 0; i < n; ++i) S[q][(size_t)i * n + i] = 1.0;
        }
      return CAVITY_OK;
    };

    while (true) {
      std::vector<int> act;
      for (int z = 0; z < ng; ++z)
        if (!gdone[z]) act.push_back(z);
      if (act.empty() || used >= maxit) break;
      // cycle start: V_0 = orthonormalised residual block of each active group
      for (int z : act)
        CK(cudaMemcpyAsync(Vg(z), w.Rc + (size_t)goff[z] * nap, sizeof(float2) * gr[z] * nap,
                           cudaMemcpyDeviceToDevice, st));
      std::vector<std::vector<cd>> S0;
      CKS(orthonormalise(act, std::vector<int>(act.size(), 0), S0, nullptr));
      std::vector<BlockLS> ls(ng);
      for (size_t q = 0; q < act.size(); ++q) ls[act[q]].start(gr[act[q]], S0[q]);
      std::vector<int> cyc = act;  // groups of this cycle
      std::vector<char> cdone(ng, 0);
      // GPU work of block step k for the groups in `run`: W = A M^{-1} V_k,
      // one classical Gram-Schmidt pass, the Gram matrix of the result, W into
      // basis slot k + 1, and the coefficients on their way to the host
      std::vector<int> woff(ng, 0);
      auto launch_step = [&](int k, const std::vector<int>& run) -> cavity_status {
        int nc = 0;
        for (int z : run) {
          woff[z] = nc;
          CKS(launch_precond_apply<float>(ctx, gr[z], Vg(z) + (size_t)k * gr[z] * nap,
                                          w.Z + (size_t)nc * nap));
          nc += gr[z];
        }
        CKS(launch_apply<float>(ctx, nc, w.Z, w.Wb, w.apw));
        BGSet set;
        int kmax = 0;
        for (size_t t = 0; t < run.size(); ++t) {
          const int z = run[t], kv = (k + 1) * gr[z];
          float2* wz = w.Wb + (size_t)woff[z] * nap;
          set.g[t] = BGrp{Vg(z), wz, wz, kv, kv, gr[z], (int)(t * hsz)};
          kmax = std::max(kmax, kv);
        }
        const int nr = (int)run.size();
        bproj(ctx, set, nr, kmax, w, 0);
        CKS(bnn(ctx, set, nr, hptr(0, 0), 1.f, -1.f));
        // Gram matrix of the projected block, formed from it directly (the
        // difference G(W) - H^H H cancels when W lies almost in the basis)
        BGSet gs;
        for (size_t t = 0; t < run.size(); ++t) {
          float2* wz = w.Wb + (size_t)woff[run[t]] * nap;
          gs.g[t] = BGrp{wz, wz, wz, 0, gr[run[t]], gr[run[t]], 0};
        }
        bproj(ctx, gs, nr, BG_MAX, w, 1);
        for (int z : run)
          CK(cudaMemcpyAsync(Vg(z) + (size_t)(k + 1) * gr[z] * nap, w.Wb + (size_t)woff[z] * nap,
                             sizeof(float2) * gr[z] * nap, cudaMemcpyDeviceToDevice, st));
        CKS(fetch(0));
        CKS(fetch(1));
        return CAVITY_OK;
      };
      // residual estimates of the last two steps per direction (convergence
      // forecast for launching the next step before the least squares)
      std::vector<double> e1(ndir, 1.0), e2(ndir, 1.0);
      // run: the groups of the step being processed, in launch (slot) order;
      // a group that converged under a step launched ahead stays in it but
      // takes no further least-squares columns
      std::vector<int> run = cyc, lnext;
      bool launched = false;
      int k = 0;
      for (; k < mb && used < maxit; ++k) {
        if (run.empty()) break;
        if (!launched) CKS(launch_step(k, run));
        launched = false;
        CKS(sync());
        // Gram matrix of the projected block (slot 1)
        std::vector<std::vector<cd>> G0(run.size()), Hc(run.size());
        for (size_t t = 0; t < run.size(); ++t) {
          const int n = gr[run[t]], K = (k + 1) * n;
          auto& G = G0[t];
          G.assign((size_t)n * n, cd(0, 0));
          for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j) G[(size_t)i * n + j] = hval(1, (int)t, i, j);
          for (int i = 0; i < n; ++i)  // exactly Hermitian
            for (int j = 0; j < i; ++j) {
              const cd m = 0.5 * (G[(size_t)i * n + j] + std::conj(G[(size_t)j * n + i]));
              G[(size_t)i * n + j] = m;
              G[(size_t)j * n + i] = std::conj(m);
            }
          Hc[t].resize((size_t)K * n);  // H, kept before the slots are reused
          for (int i = 0; i < K; ++i)
            for (int j = 0; j < n; ++j) Hc[t][(size_t)i * n + j] = hval(0, (int)t, i, j);
        }
        std::vector<std::vector<cd>> S;
        std::vector<int> c0;
        for (int z : run) c0.push_back((k + 1) * gr[z]);
        CKS(orthonormalise(run, c0, S, &G0));
        ++used;
        // launch step k + 1 now unless some group is forecast to converge at
        // step k (geometric extrapolation of its estimates)
        std::vector<int> active;
        for (int z : run)
          if (!cdone[z]) active.push_back(z);
        bool soon = false;
        for (int z : active)
          for (int j = 0; j < gr[z]; ++j) {
            const int dd = dirs[goff[z] + j];
            const double f = e2[dd] > 0 ? e1[dd] * std::min(1.0, e1[dd] / e2[dd]) : e1[dd];
            soon = soon || f <= 2.0 * tol[dd];
          }
        if (!soon && k + 1 < mb && used < maxit) {
          CKS(launch_step(k + 1, active));
          launched = true;
          lnext = active;
        }
        // least squares of step k (overlaps the GPU work just launched)
        std::vector<int> next;
        for (size_t t = 0; t < run.size(); ++t) {
          const int z = run[t], n = gr[z], K = (k + 1) * n;
          if (cdone[z]) continue;
          std::vector<std::vector<cd>> cols(n, std::vector<cd>((size_t)K + n, cd(0, 0)));
          for (int j = 0; j < n; ++j) {
            for (int i = 0; i < K; ++i) cols[j][i] = Hc[t][(size_t)i * n + j];
            for (int i = 0; i < n; ++i) cols[j][K + i] = S[t][(size_t)i * n + j];
          }
          ls[z].add(cols, K + n);
          bool conv = true;
          for (int j = 0; j < n; ++j) {
            const int dd = dirs[goff[z] + j];
            iters[dd] += 1;
            est[dd] = ls[z].resid(j);
            e2[dd] = e1[dd];
            e1[dd] = est[dd];
            conv = conv && est[dd] <= tol[dd];
          }
          if (conv) cdone[z] = 1;
          else next.push_back(z);
        }
        if (next.empty()) break;
        run = launched ? lnext : next;
      }
      // corrections of this cycle: d += M^{-1} V Y per group
      std::vector<std::vector<cd>> Ys;
      std::vector<int> yz;
      BGSet set;
      int n = 0;
      for (int z : cyc) {
        std::vector<cd> Y;
        ls[z].solve(Y);
        if (ls[z].cols == 0) continue;
        Ys.push_back(Y);
        yz.push_back(n);
        set.g[n] = BGrp{Vg(z), nullptr, w.Tt + (size_t)goff[z] * nap, ls[z].cols, ls[z].cols, gr[z],
                        n * (int)hsz};
        ++n;
      }
      if (n > 0) {
        CKS(upload(Ys, yz));
        CKS(bnn(ctx, set, n, w.cb, 0.f, 1.f));
      }
      // T -> Z = M^{-1} T, scattered into the direction columns of d
      std::vector<int> done_now;
      for (int z : cyc) {
        if (ls[z].cols == 0) continue;
        CKS(launch_precond_apply<float>(ctx, gr[z], w.Tt + (size_t)goff[z] * nap,
                                        w.Z + (size_t)goff[z] * nap));
        KScope ks_(ctx, KC_KRYLOV);
        k_scatter_add<<<dim3(bg_blocks(nap, 256), gr[z]), 256, 0, st>>>(
            w.Z + (size_t)goff[z] * nap, d, w.map + goff[z], nap);
      }
      for (int z : cyc)
        if (cdone[z]) gdone[z] = 1;
      bool rest = false;
      for (int z : cyc) rest = rest || !gdone[z];
      if (!rest || used >= maxit) break;
      // restart: R_c <- R_c - A M^{-1} (V Y) for the groups still running
      for (int z : cyc) {
        if (gdone[z]) continue;
        CKS(launch_precond_apply<float>(ctx, gr[z], w.Tt + (size_t)goff[z] * nap,
                                        w.Z + (size_t)goff[z] * nap));
        CKS(launch_apply<float>(ctx, gr[z], w.Z + (size_t)goff[z] * nap,
                                w.Wb + (size_t)goff[z] * nap, w.apw));
        KScope ks_(ctx, KC_KRYLOV);
        k_sub_cols<<<dim3(bg_blocks(nap, 256), gr[z]), 256, 0, st>>>(
            w.Wb + (size_t)goff[z] * nap, w.Rc + (size_t)goff[z] * nap, nap);
      }
    }
  }
  CK(cudaGetLastError());
  {
    int terr = 0;
    CK(cudaMemcpyFromSymbolAsync(&terr, g_tc_err, sizeof(int), 0, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (terr) {
      ctx->err = "block Krylov update: a tensor-core completion wait ran out";
      return CAVITY_ETIMEOUT;
    }
  }
  return CAVITY_OK;
}
