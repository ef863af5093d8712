// Interior field of the mixed path (complex64 output) in one persistent
// kernel: back-substitution (EInter) and both inverse transforms of (E123F).
//
// The arithmetic is that of field.cu -- per level j and direction d the
// modal coefficients E_{l,j}^{mn} = P_{l,j}^{mn} E_l^{mn} (+ Q_{l,j}^{mn}
// E_3^{mn}), the paired cosine/sine syntheses along x2 into the intermediate
// T1, then along x1 into the output -- but scheduled so that T1 never leaves
// the L2 cache:
//
//  * A slab is one (level, direction).  Slabs are ordered in blocks of G = 4
//    levels: inside a block the directions, and for each direction its G
//    levels, so a block's profiles are read from HBM once and reused from L2
//    by every direction, and a direction's aperture vector is reused from L2
//    by the G levels.  Each slab has row items (R rows: R paired E2/E1 lines
//    and R E3 lines along x2, written to T1) and column items (C columns
//    along x1, read from T1, written to the field).
//  * Items are handed out in a fixed order by one atomic counter: the row
//    items of slab s, then the column items of slab s - LAG.  T1 lives in a
//    ring of RING = LAG + 2 slab buffers (25 MB at 512 x 512), so it stays in
//    L2 between its write and its read.  A column item waits until every row
//    item of its slab is done; a row item waits until the column items of the
//    slab that used its ring buffer before are done.  Both wait only on items
//    handed out earlier, which are held by running blocks that never wait on
//    later ones, so the schedule cannot deadlock; every wait is bounded and
//    reports a timeout through an error word instead of spinning forever.
//  * Inside a block, eight loader warps form the next item's input lines in
//    shared memory (profile times aperture value, or the T1 columns) while
//    eight transform warps run the current item's line FFTs and store their
//    results: two stages, handed over by named barriers.
//
// Output per direction and level j = 1..Nz: E1 on p = 0..Nx, q = 1..Ny-1,
// E2 on p = 1..Nx-1, q = 0..Ny, E3 on p = 1..Nx-1, q = 1..Ny-1, row-major.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "fft.cuh"

namespace {

// schedule parameters (compile-time; the defaults were chosen by timing)
#ifndef FIELD_FUSED_NL
#define FIELD_FUSED_NL 8
#endif
#ifndef FIELD_FUSED_LAG
#define FIELD_FUSED_LAG 2
#endif
#ifndef FIELD_FUSED_G
#define FIELD_FUSED_G 4
#endif
constexpr int FF_NF = 8;                    // transform warps
constexpr int FF_NL = FIELD_FUSED_NL;       // loader warps
constexpr int FF_THREADS = (FF_NF + FF_NL) * 32;
constexpr int FF_LAG = FIELD_FUSED_LAG;     // column items of slab s follow row items of s + LAG
constexpr int FF_RING = FF_LAG + 2;         // T1 slab buffers
constexpr int FF_G = FIELD_FUSED_G;         // levels per block of the slab order
// named barriers (0 is __syncthreads; the warp transforms use none)
constexpr int BAR_FULL = 1;                 // + stage: loaders arrive, transform warps wait
constexpr int BAR_EMPTY = 3;                // + stage: transform warps arrive, loaders wait
constexpr int BAR_XF = 5;                   // transform warps among themselves
constexpr int BAR_LD = 6;                   // loader warps among themselves
constexpr int KIND_ROW = 0, KIND_COL = 1, KIND_END = 2, KIND_ABORT = 3;
constexpr long long SPIN_LIMIT = 1ll << 24;  // ~ seconds with the backoff below

struct FFP {
  int nx, ny, nz, M, N, n1, n2, nap;
  int recw;                  // float4 per profile record: 2 (homogeneous), 3 (layered)
  int ndir, j0, nslab;       // slabs s = (j - j0) * ndir + d
  int nR, nC, R, Cq;         // items per slab, rows / columns per item
  int lag, twlog;
  bool layered;
  long long S, t1slab, total;
};

struct FFCtl {                // device control words, zeroed before each launch
  unsigned long long next;    // item counter
  int rows_done[FF_RING];
  int cols_done[FF_RING];
  int err;                    // 1: a wait ran out
  int pad[5];
};

__device__ __forceinline__ void bar_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// L2 policies: keep T1, stream the field out
__device__ __forceinline__ unsigned long long pol_last() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// T1 is rewritten by other blocks between uses of a ring buffer: read it
// from L2 (never from a possibly stale L1 line)
__device__ __forceinline__ float2 ld_t1(const float2* a, unsigned long long pol) {
  float2 v;
  asm volatile("ld.global.cg.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(v.x), "=f"(v.y) : "l"(a), "l"(pol) : "memory");
  return v;
}
__device__ __forceinline__ void st_t1(float2* a, float2 v, unsigned long long pol) {
  asm volatile("st.global.cg.L2::cache_hint.v2.f32 [%0], {%1, %2}, %3;"
               :: "l"(a), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}
__device__ __forceinline__ void st_out(float2* a, float2 v) {
  asm volatile("st.global.cs.v2.f32 [%0], {%1, %2};" :: "l"(a), "f"(v.x), "f"(v.y) : "memory");
}

// item t -> (kind, slab, index) of the fixed schedule
__device__ __forceinline__ void decode(const FFP& p, long long t, int& kind, int& slab, int& idx) {
  const long long a = (long long)p.lag * p.nR;
  if (t < a) {
    kind = KIND_ROW;
    slab = (int)(t / p.nR);
    idx = (int)(t % p.nR);
    return;
  }
  t -= a;
  const long long per = p.nR + p.nC;
  const long long b = (long long)(p.nslab - p.lag) * per;
  if (t < b) {
    const int ph = p.lag + (int)(t / per), r = (int)(t % per);
    if (r < p.nR) {
      kind = KIND_ROW;
      slab = ph;
      idx = r;
    } else {
      kind = KIND_COL;
      slab = ph - p.lag;
      idx = r - p.nR;
    }
    return;
  }
  t -= b;
  kind = KIND_COL;
  slab = p.nslab - p.lag + (int)(t / p.nC);
  idx = (int)(t % p.nC);
}

// bounded wait until *c >= target; false when it ran out (or another wait did)
__device__ bool wait_count(const int* c, int target, int* err) {
  int ns = 32;
  for (long long it = 0; it < SPIN_LIMIT; ++it) {
    if (ld_acquire(c) >= target) return true;
    if (ld_acquire(err) != 0) return false;
    __nanosleep(ns);
    if (ns < 256) ns *= 2;
  }
  atomicExch(err, 1);
  return false;
}

struct StageMeta {
  int kind, slab, idx, pad;
};

// Slab order: blocks of G levels; inside a block the directions, and for
// each direction its G levels.  A block's profiles (G levels) and one
// direction's aperture vector stay in L2 while they are reused.
__device__ __forceinline__ void slab_level_dir(const FFP& p, int s, int& jl, int& d) {
  const int per = FF_G * p.ndir;
  const int b = s / per, w = s - b * per;
  const int gb = min(FF_G, p.nslab / p.ndir - b * FF_G);
  d = w / gb;
  jl = b * FF_G + (w - d * gb);
}

template <int LNX, int LNY>
struct FFShape {
  static constexpr int nx = 1 << LNX, ny = 1 << LNY;
  static constexpr int LOGY = LNY + 1, LOGX = LNX + 1;         // line lengths 2 ny, 2 nx
  static constexpr int LWY = LineShape<float, LOGY>::LW, LWX = LineShape<float, LOGX>::LW;
  static constexpr int LPWY = 32 / LWY, LPWX = 32 / LWX;      // lines per warp
  static constexpr int R = FF_NF * LPWY / 2;                   // rows per row item
  static constexpr int Cq = FF_NF * LPWX / 2;                  // columns per column item
  static constexpr int LSY = padded_len(2 * ny) | 1, LSX = padded_len(2 * nx) | 1;
  static constexpr int STAGE = (2 * R * LSY > 2 * Cq * LSX) ? 2 * R * LSY : 2 * Cq * LSX;
  static constexpr size_t SMEM = sizeof(float2) * 2 * (size_t)STAGE + 64;
};

template <int LNX, int LNY>
__global__ void __launch_bounds__(FF_THREADS, 1)
    k_field_fused(const float4* __restrict__ apr, const float4* __restrict__ prec,
                  float2* __restrict__ T1, float2* __restrict__ out, FFCtl* ctl, FFP p,
                  const float2* __restrict__ tw) {
  using S = FFShape<LNX, LNY>;
  constexpr int nx = S::nx, ny = S::ny, R = S::R, Cq = S::Cq;
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float2* stage_buf = (float2*)sm_raw;
  StageMeta* meta = (StageMeta*)(stage_buf + 2 * (size_t)S::STAGE);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned long long keep = pol_last();

  if (warp >= FF_NF) {
    // ------------------------------------------------------------ loaders
    const int lt = threadIdx.x - FF_NF * 32;                 // 0 .. FF_NL * 32 - 1
    __shared__ StageMeta s_item[2];   // per stage: reused only after that stage's EMPTY wait
    // lt == 0 fetches each item one item ahead, so the atomic's round trip
    // overlaps the loads of the current item (a fetched item is always
    // loaded next, so holding it cannot stall the schedule)
    long long t_next = 0;
    if (lt == 0) t_next = (long long)atomicAdd(&ctl->next, 1ull);
    for (int it = 0;; ++it) {
      const int st = it & 1;
      if (it >= 2) bar_sync(BAR_EMPTY + st, FF_THREADS);
      if (lt == 0) {
        StageMeta m;
        const long long t = t_next;
        if (t >= p.total || ld_acquire(&ctl->err) != 0) {
          m.kind = t >= p.total ? KIND_END : KIND_ABORT;
          m.slab = m.idx = 0;
        } else {
          decode(p, t, m.kind, m.slab, m.idx);
          if (m.kind == KIND_COL) {
            const int slot = m.slab % FF_RING, use = m.slab / FF_RING;
            if (!wait_count(&ctl->rows_done[slot], (use + 1) * p.nR, &ctl->err))
              m.kind = KIND_ABORT;
          }
          if (m.kind != KIND_ABORT) t_next = (long long)atomicAdd(&ctl->next, 1ull);
        }
        s_item[st] = m;
      }
      bar_sync(BAR_LD, FF_NL * 32);
      const StageMeta m = s_item[st];
      if (m.kind == KIND_END || m.kind == KIND_ABORT) {
        if (lt == 0) meta[st] = m;
        bar_arrive(BAR_FULL + st, FF_THREADS);
        // the transform warps release the other stage once more
        if (it >= 1) bar_sync(BAR_EMPTY + (st ^ 1), FF_THREADS);
        break;
      }
      // every loader thread acquires the counter its column item waited on,
      // so its reads of T1 below are ordered after the writes that were counted
      if (m.kind == KIND_COL) (void)ld_acquire(&ctl->rows_done[m.slab % FF_RING]);
      float2* buf = stage_buf + (size_t)st * S::STAGE;
      int jl, d;
      slab_level_dir(p, m.slab, jl, d);
      const int j = p.j0 + jl;
      float2* t1 = T1 + (size_t)(m.slab % FF_RING) * p.t1slab;
      if (m.kind == KIND_ROW) {
        // lines 0..R-1: row m (E2 cos + E1 sin), lines R..2R-1: row m (E3 sin).
        // One record index per mode: the aperture record {E1, E2}, {E3, 0} and
        // the profile record of level j (entries outside an index set are 0,
        // so no masks); batches of U elements per thread, every load of a
        // batch issued before the first is used.
        constexpr int n2 = 2 * ny, ls = S::LSY;
        constexpr int PER = R * ny / (FF_NL * 32);
        constexpr int U = PER < 4 ? PER : 4;
        static_assert(PER % U == 0 && PER * FF_NL * 32 == R * ny, "row items tile the loaders");
        const float4* A = apr + (size_t)d * 2 * nx * ny;
        const bool top = (j == p.nz);
        const bool lay = p.recw == 3;
        const float4* Pj = prec + (size_t)(top ? 0 : j - 1) * p.recw * nx * ny;
        const int M = p.M;
        const float2 z = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int k0 = 0; k0 < PER; k0 += U) {
          float4 a01[U], a3[U], p01[U], p3q1[U], q2[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = lt + (k0 + u) * (FF_NL * 32);
            const int r = e >> LNY, n = e & (ny - 1);
            const int mm = min(m.idx * R + r, M);   // rows beyond M: any record, masked below
            const int rec = mm * ny + n;
            a01[u] = __ldg(A + 2 * rec);
            a3[u] = __ldg(A + 2 * rec + 1);
            if (!top) {
              p01[u] = __ldg(Pj + (size_t)p.recw * rec);
              p3q1[u] = __ldg(Pj + (size_t)p.recw * rec + 1);
              if (lay) q2[u] = __ldg(Pj + (size_t)p.recw * rec + 2);
            }
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = lt + (k0 + u) * (FF_NL * 32);
            const int r = e >> LNY, n = e & (ny - 1);
            const bool in = m.idx * R + r <= M;
            float2 e1 = make_float2(a01[u].x, a01[u].y), e2 = make_float2(a01[u].z, a01[u].w);
            float2 e3 = make_float2(a3[u].x, a3[u].y);
            if (!top) {
              const float2 E3 = e3;
              e1 = cmul<float>(make_float2(p01[u].x, p01[u].y), e1);
              e2 = cmul<float>(make_float2(p01[u].z, p01[u].w), e2);
              e3 = cmul<float>(make_float2(p3q1[u].x, p3q1[u].y), E3);
              if (lay) {
                e1 = cadd<float>(e1, cmul<float>(make_float2(p3q1[u].z, p3q1[u].w), E3));
                e2 = cadd<float>(e2, cmul<float>(make_float2(q2[u].x, q2[u].y), E3));
              }
            }
            if (!in) e1 = e2 = e3 = z;
            float2* lp = buf + (size_t)r * ls;
            float2* l3 = buf + (size_t)(R + r) * ls;
            if (n == 0) {
              lp[0] = cscale<float>(e2, 2.f);
              lp[pidx(ny)] = z;
              l3[0] = z;
              l3[pidx(ny)] = z;
            } else {
              lp[pidx(n)] = cadd<float>(e2, e1);
              lp[pidx(n2 - n)] = csub<float>(e2, e1);
              l3[pidx(n)] = e3;
              l3[pidx(n2 - n)] = make_float2(-e3.x, -e3.y);
            }
          }
        }
      } else {
        // lines 0..C-1: column q (E1 cos + E2 sin), lines C..2C-1: column q (E3 sin)
        constexpr int n2 = 2 * nx, ls = S::LSX;
        constexpr int lC = clog2(Cq);
        constexpr int PER = nx * Cq / (FF_NL * 32);
        constexpr int U = PER < 8 ? PER : 8;
        static_assert(PER % U == 0 && PER * FF_NL * 32 == nx * Cq, "column items tile the loaders");
        const float2* tE1 = t1;
        const float2* tE2 = t1 + (size_t)nx * (ny + 1);
        const float2* tE3 = t1 + (size_t)2 * nx * (ny + 1);
        const float2 z = make_float2(0.f, 0.f);
#pragma unroll 1
        for (int k0 = 0; k0 < PER; k0 += U) {
          float2 ce[U], so[U], s3[U];
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = lt + (k0 + u) * (FF_NL * 32);
            const int t = e >> lC, c = e & (Cq - 1);
            const int q = m.idx * Cq + c;
            const bool hc = q >= 1 && q < ny, hs = t >= 1 && q <= ny, h3 = t >= 1 && hc;
            const int qc = q <= ny ? q : ny, tm = t >= 1 ? t - 1 : 0;
            ce[u] = ld_t1(tE1 + (size_t)t * (ny + 1) + qc, keep);
            so[u] = ld_t1(tE2 + (size_t)tm * (ny + 1) + qc, keep);
            s3[u] = ld_t1(tE3 + (size_t)tm * (ny + 1) + qc, keep);
            if (!hc) ce[u] = z;
            if (!hs) so[u] = z;
            if (!h3) s3[u] = z;
          }
#pragma unroll
          for (int u = 0; u < U; ++u) {
            const int e = lt + (k0 + u) * (FF_NL * 32);
            const int t = e >> lC, c = e & (Cq - 1);
            float2* lp = buf + (size_t)c * ls;
            float2* l3 = buf + (size_t)(Cq + c) * ls;
            if (t == 0) {
              lp[0] = cscale<float>(ce[u], 2.f);
              lp[pidx(nx)] = z;
              l3[0] = z;
              l3[pidx(nx)] = z;
            } else {
              lp[pidx(t)] = cadd<float>(ce[u], so[u]);
              lp[pidx(n2 - t)] = csub<float>(ce[u], so[u]);
              l3[pidx(t)] = s3[u];
              l3[pidx(n2 - t)] = make_float2(-s3[u].x, -s3[u].y);
            }
          }
        }
      }
      if (lt == 0) {
        // a row item's results overwrite the T1 buffer of slab - RING: it is
        // free once that slab's column items are done.  Waited here, after
        // the loads, so the wait overlaps them; the transform warps write T1
        // only after this stage is handed over.  On a time-out err is set and
        // every later item aborts.
        if (m.kind == KIND_ROW && m.slab >= FF_RING)
          (void)wait_count(&ctl->cols_done[m.slab % FF_RING], (m.slab / FF_RING) * p.nC, &ctl->err);
        meta[st] = m;
      }
      bar_arrive(BAR_FULL + st, FF_THREADS);
    }
    return;
  }

  // -------------------------------------------------------------- transforms
  for (int it = 0;; ++it) {
    const int st = it & 1;
    bar_sync(BAR_FULL + st, FF_THREADS);
    const StageMeta m = meta[st];
    if (m.kind == KIND_END || m.kind == KIND_ABORT) break;
    float2* buf = stage_buf + (size_t)st * S::STAGE;
    int jl, d;
    slab_level_dir(p, m.slab, jl, d);
    const int j = p.j0 + jl;
    const int slot = m.slab % FF_RING;
    float2* t1 = T1 + (size_t)slot * p.t1slab;
    if (m.kind == KIND_ROW) {
      constexpr int n2 = 2 * ny, ls = S::LSY, LPW = S::LPWY;
      fft_warp_lines<float, true, S::LOGY>(buf, ls, warp * LPW, LPW, tw, p.twlog);
      __syncwarp();
      for (int k = 0; k < LPW; ++k) {
        const int l = warp * LPW + k;
        const bool e3line = l >= R;
        const int mm = m.idx * R + (e3line ? l - R : l);
        if (mm > p.M || (e3line && mm < 1)) continue;
        const float2* line = buf + (size_t)l * ls;
        for (int q = lane; q <= ny; q += 32) {
          const float2 zq = line[pidx(q)];
          if (!e3line) {
            const float2 zm = line[pidx((n2 - q) & (n2 - 1))];
            const float2 c = cscale<float>(cadd<float>(zq, zm), 0.25f);
            const float2 sn = cscale<float>(csub<float>(zq, zm), 0.25f);
            st_t1(t1 + (size_t)mm * (ny + 1) + q, make_float2(sn.y, -sn.x), keep);   // E1 row m
            if (mm >= 1) st_t1(t1 + ((size_t)nx + mm - 1) * (ny + 1) + q, c, keep);   // E2 row m-1
          } else {
            st_t1(t1 + ((size_t)2 * nx + mm - 1) * (ny + 1) + q,
                  make_float2(zq.y * 0.5f, -zq.x * 0.5f), keep);                       // E3 row m-1
          }
        }
      }
    } else {
      constexpr int n2 = 2 * nx, ls = S::LSX, LPW = S::LPWX, lC = clog2(Cq);
      fft_warp_lines<float, true, S::LOGX>(buf, ls, warp * LPW, LPW, tw, p.twlog);
      bar_sync(BAR_XF, FF_NF * 32);
      float2* o = out + ((size_t)d * p.nz + (j - 1)) * p.S;
      const long long offE2 = (long long)(nx + 1) * (ny - 1);
      const long long offE3 = offE2 + (long long)(nx - 1) * (ny + 1);
      const int q0 = m.idx * Cq;
      for (int e = threadIdx.x; e < (nx + 1) * Cq; e += FF_NF * 32) {
        const int pp = e >> lC, c = e & (Cq - 1);
        const int q = q0 + c;
        if (q > ny) continue;
        const float2* lp = buf + (size_t)c * ls;
        const float2 zq = lp[pidx(pp)];
        const float2 zm = lp[pidx((n2 - pp) & (n2 - 1))];
        if (q >= 1 && q < ny)                                      // E1 (cos in x1), p = 0..nx
          st_out(o + (size_t)pp * (ny - 1) + (q - 1), cscale<float>(cadd<float>(zq, zm), 0.25f));
        if (pp >= 1 && pp < nx) {                                  // E2 (sin in x1), p = 1..nx-1
          const float2 sn = cscale<float>(csub<float>(zq, zm), 0.25f);
          st_out(o + offE2 + (size_t)(pp - 1) * (ny + 1) + q, make_float2(sn.y, -sn.x));
          if (q >= 1 && q < ny) {                                  // E3 on p = 1..nx-1, q = 1..ny-1
            const float2 z3 = buf[(size_t)(Cq + c) * ls + pidx(pp)];
            st_out(o + offE3 + (size_t)(pp - 1) * (ny - 1) + (q - 1),
                   make_float2(z3.y * 0.5f, -z3.x * 0.5f));
          }
        }
      }
    }
    // the item's results are visible device-wide before it is counted: the
    // barrier orders every transform thread's stores before the counting
    // thread's fence and atomic
    bar_sync(BAR_XF, FF_NF * 32);
    if (threadIdx.x == 0) {
      __threadfence();
      if (m.kind == KIND_ROW) atomicAdd(&ctl->rows_done[slot], 1);
      else atomicAdd(&ctl->cols_done[slot], 1);
    }
    bar_arrive(BAR_EMPTY + st, FF_THREADS);
  }
}

template <int LN>
cavity_status run_fused(cavity_ctx* ctx, const float4* apr, const float4* prec, float2* T1,
                        FFCtl* ctl, float2* out, FFP p) {
  using S = FFShape<LN, LN>;
  auto kern = k_field_fused<LN, LN>;
  static std::atomic<bool> done{false};  // set once; host threads may race
  static int blocks_per_sm = 1;
  if (!done) {
    CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::SMEM));
    int b = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, FF_THREADS, S::SMEM));
    blocks_per_sm = std::max(1, b);
    done = true;
  }
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  p.R = S::R;
  p.Cq = S::Cq;
  p.nR = (p.nx + S::R - 1) / S::R;
  p.nC = (p.ny + 1 + S::Cq - 1) / S::Cq;
  p.lag = std::min(FF_LAG, p.nslab);
  p.total = (long long)p.nslab * (p.nR + p.nC);
  CK(cudaMemsetAsync(ctl, 0, sizeof(FFCtl), ctx->stream));
  const long long grid = std::min<long long>((long long)sms * blocks_per_sm, p.total);
  {
    KScope ks_(ctx, KC_FIELD_X);
    kern<<<(unsigned)grid, FF_THREADS, S::SMEM, ctx->stream>>>(apr, prec, T1, out, ctl, p,
                                                              ctx->tw32);
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

}  // namespace

// Grids the fused kernel covers: square, 32 <= nx = ny <= 512 (warp
// transforms of length 64 .. 1024).
bool field_fused_supported(const Geo& g) {
  return g.nx == g.ny && g.lnx >= 5 && g.lnx <= 9;
}

// measured at the 16-direction 256^2 x 128 workload: fused 10.1 ms against
// 5.5 ms for the two-pass kernels per step; at the 8-direction four-layer
// 512^2 x 256 workload the fused kernel is the faster (20.5 against 26.8 ms)
bool field_fused_use(const cavity_ctx* ctx) {
  const int o = ctx->opt[CAVITY_OPT_FIELD_FUSED];
  if (o == 2 || !field_fused_supported(ctx->g)) return false;
  return o == 1 || ctx->g.lnx == 9;
}

size_t field_fused_work_bytes(const Geo& g) {
  return sizeof(float2) * (size_t)FF_RING * 3 * g.nx * (g.ny + 1) + 256;
}

// Levels j0 .. j0 + nlev - 1 of ndir directions; apr: the aperture records
// (ap_records), work: field_fused_work_bytes (T1 ring, then the control words).
cavity_status launch_field_fused(cavity_ctx* ctx, int ndir, const float4* apr, float2* out,
                                 int j0, int nlev, void* work) {
  const Geo& g = ctx->g;
  if (!ctx->prof_rec) {
    ctx->err = "field: profile records missing (not a mixed-precision context)";
    return CAVITY_EINVAL;
  }
  FFP p;
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz; p.M = g.M; p.N = g.N; p.n1 = g.n1; p.n2 = g.n2;
  p.nap = g.nap; p.ndir = ndir; p.j0 = j0; p.nslab = nlev * ndir;
  p.recw = ctx->prof_rec_w;
  p.twlog = ilog2(ctx->TW);
  p.layered = ctx->layers.size() > 1;
  p.S = g.field_per_level;
  p.t1slab = 3ll * g.nx * (g.ny + 1);
  float2* T1 = (float2*)work;
  FFCtl* ctl = (FFCtl*)((char*)work + sizeof(float2) * (size_t)FF_RING * p.t1slab);
  return dispatch_log<5, 9>(g.lnx, [&](auto c) -> cavity_status {
    constexpr int LN = decltype(c)::value;
    return run_fused<LN>(ctx, apr, ctx->prof_rec, T1, ctl, out, p);
  });
}

// aperture records: {E1, E2}, {E3, 0} per direction and mode (m, n) of the
// nx x ny mode grid, FP32, zero outside each component's index set
__global__ void k_ap_records(const double2* __restrict__ ap, float4* __restrict__ rec, int nx,
                             int ny, int N, int n1, int n2, int nap) {
  const int mn = blockIdx.x * blockDim.x + threadIdx.x, d = blockIdx.y;
  if (mn >= nx * ny) return;
  const int m = mn / ny, n = mn - m * ny;
  const double2* E = ap + (size_t)d * nap;
  const double2 z = make_double2(0.0, 0.0);
  const double2 e1 = n >= 1 ? E[m * N + (n - 1)] : z;
  const double2 e2 = m >= 1 ? E[n1 + (m - 1) * (N + 1) + n] : z;
  const double2 e3 = (m >= 1 && n >= 1) ? E[n1 + n2 + (m - 1) * N + (n - 1)] : z;
  float4* o = rec + ((size_t)d * nx * ny + mn) * 2;
  o[0] = make_float4((float)e1.x, (float)e1.y, (float)e2.x, (float)e2.y);
  o[1] = make_float4((float)e3.x, (float)e3.y, 0.f, 0.f);
}

size_t ap_records_bytes(const Geo& g, int ndir) {
  return sizeof(float4) * 2 * (size_t)ndir * g.nx * g.ny;
}

cavity_status launch_ap_records(cavity_ctx* ctx, int ndir, const double2* ap, float4* rec) {
  const Geo& g = ctx->g;
  KScope ks_(ctx, KC_FIELD_Y);
  k_ap_records<<<dim3((g.nx * g.ny + 255) / 256, ndir), 256, 0, ctx->stream>>>(
      ap, rec, g.nx, g.ny, g.N, g.n1, g.n2, g.nap);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// profile records of levels 1..nz-1 (see cavity_ctx::prof_rec)
__global__ void k_prof_records(const double2* __restrict__ prof, const double2* __restrict__ profq,
                               float4* __restrict__ rec, int nx, int ny, int N, int n1, int n2,
                               int nap, int nlev, int w) {
  const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (t >= (long long)nlev * nx * ny) return;
  const int jl = (int)(t / (nx * ny)), mn = (int)(t - (long long)jl * nx * ny);
  const int m = mn / ny, n = mn - m * ny;
  const double2* P = prof + (size_t)jl * nap;
  const double2 z = make_double2(0.0, 0.0);
  const bool h1 = n >= 1, h2 = m >= 1, h3 = h1 && h2;
  const int i1 = m * N + (n - 1), i2 = n1 + (m - 1) * (N + 1) + n, i3 = n1 + n2 + (m - 1) * N + (n - 1);
  const double2 p1 = h1 ? P[i1] : z, p2 = h2 ? P[i2] : z, p3 = h3 ? P[i3] : z;
  float4* o = rec + (size_t)t * w;
  o[0] = make_float4((float)p1.x, (float)p1.y, (float)p2.x, (float)p2.y);
  if (w == 3) {
    const double2* Q = profq + (size_t)jl * (n1 + n2);
    const double2 q1 = h3 ? Q[i1] : z, q2 = h3 ? Q[i2] : z;
    o[1] = make_float4((float)p3.x, (float)p3.y, (float)q1.x, (float)q1.y);
    o[2] = make_float4((float)q2.x, (float)q2.y, 0.f, 0.f);
  } else {
    o[1] = make_float4((float)p3.x, (float)p3.y, 0.f, 0.f);
  }
}

cavity_status launch_prof_records(cavity_ctx* ctx) {
  const Geo& g = ctx->g;
  const bool layered = ctx->layers.size() > 1;
  const int w = layered ? 3 : 2;
  const long long n = (long long)(g.nz - 1) * g.nx * g.ny;
  if (!ctx->prof_rec || ctx->prof_rec_w < w) {
    if (ctx->prof_rec) cudaFree(ctx->prof_rec);
    ctx->prof_rec = nullptr;
    ctx->prof_rec_w = 0;
    // size for the layered layout, so a later layered prepare reuses it
    CK(cudaMalloc(&ctx->prof_rec, sizeof(float4) * 3 * (size_t)n));
  }
  ctx->prof_rec_w = w;
  KScope ks_(ctx, KC_SETUP);
  k_prof_records<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(
      ctx->prof, layered ? ctx->profq : nullptr, ctx->prof_rec, g.nx, g.ny, g.N, g.n1, g.n2,
      g.nap, g.nz - 1, w);
  CK(cudaGetLastError());
  return CAVITY_OK;
}

// the error word of the last fused launch (0: every wait ended in time)
cavity_status field_fused_check(cavity_ctx* ctx, void* work) {
  const Geo& g = ctx->g;
  FFCtl* ctl = (FFCtl*)((char*)work + sizeof(float2) * (size_t)FF_RING * 3 * g.nx * (g.ny + 1));
  int err = 0;
  CK(cudaMemcpyAsync(&err, &ctl->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (err) {
    ctx->err = "field synthesis: a wait between blocks ran out (item schedule stalled)";
    return CAVITY_ETIMEOUT;
  }
  return CAVITY_OK;
}
