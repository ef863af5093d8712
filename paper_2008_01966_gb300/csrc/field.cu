// Interior field: back-substitution (EInter) fused with the inverse cos/sin
// transforms of (E123F) per level.
//
// For direction d and level j the modal coefficients are
//   E_{l,j}^{mn} = P_{l,j}^{mn} E_l^{mn} (+ Q_{l,j}^{mn} E_3^{mn} for l = 1, 2 in
//   a layered fill),
// and the field on the grid is
//   E1(p, q) = sum_{m=0}^{M} sum_{n=1}^{N} E1^{mn} cos(m pi p/Nx) sin(n pi q/Ny),
//   E2 with sin/cos, E3 with sin/sin.
// Pass 1 forms the coefficients of one row m on the fly (profile times aperture
// value, never stored) and synthesises along x2 with an extended FFT of length
// 2Ny; pass 2 synthesises along x1 for a tile of columns q and writes output
// rows of the tile contiguously.  Levels are processed in chunks whose
// intermediate is at most 512 MB: grids of thousands of blocks (no tail
// waves), at the price of one write and one read of the intermediate, which
// at HBM speed is small next to the transforms (measured: 64 MB chunks that
// stay in L2 were 25 % slower overall than 512 MB chunks).
//
// Output per direction and level j = 1..Nz: E1 on p = 0..Nx, q = 1..Ny-1,
// E2 on p = 1..Nx-1, q = 0..Ny, E3 on p = 1..Nx-1, q = 1..Ny-1, row-major.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "fft.cuh"

struct FP {
  int nx, ny, nz, M, N, n1, n2, nap, lnx, lny, twlog;
  int j0, lc;           // first level (1-based) and levels in this chunk
  int ndir;
  bool layered;
  long long S;          // samples per level
};

#define FIELD_THREADS 256
template <typename T> __host__ __device__ constexpr int field_lines(int n) {
  return fft_tpl<T>(n) >= FIELD_THREADS ? 1 : FIELD_THREADS / fft_tpl<T>(n);
}

// Pairing.  The cosine synthesis of one coefficient row and the sine synthesis
// of another share one complex FFT: the extended line of the cosine row is
// even, that of the sine row odd, so the transform Z of their sum splits into
// the two syntheses as the even and odd parts,
//   C(q) = (Z(q) + Z(-q)) / 2,   S(q) = (Z(q) - Z(-q)) / 2.
// Along x2, E2 (cos) row m pairs with E1 (sin) row m; along x1, E1 (cos)
// column q pairs with E2 (sin) column q.  E3 (sin, sin) lines stay single.
// Group g = blockIdx.y: 0 the pairs, 1 the E3 lines.

// modal coefficient of component c (0, 1, 2) at (m, n) for level j, zero
// outside the component's index set: profile times aperture value, plus the
// E3-driven term for E1, E2 in a layered fill
template <typename T>
struct FieldCoef {
  const C<T>* E;                  // aperture coefficients of this direction
  const C<T>* Pj;                 // profiles of level j
  const C<T>* Qj;                 // E3-driven profiles of level j (layered) or null
  int M, N, n1, n2;
  bool top, layered;
  __device__ __forceinline__ C<T> operator()(int c, int m, int n) const {
    int i;
    if (c == 0) {
      if (m > M || n < 1 || n > N) return mk<T>(0, 0);
      i = m * N + (n - 1);
    } else if (c == 1) {
      if (m < 1 || m > M || n > N) return mk<T>(0, 0);
      i = n1 + (m - 1) * (N + 1) + n;
    } else {
      if (m < 1 || m > M || n < 1 || n > N) return mk<T>(0, 0);
      i = n1 + n2 + (m - 1) * N + (n - 1);
    }
    C<T> v = E[i];
    if (!top) {
      v = cmul<T>(Pj[i], v);
      if (layered && c < 2 && m >= 1 && n >= 1)
        v = cadd<T>(v, cmul<T>(Qj[i], E[n1 + n2 + (m - 1) * N + (n - 1)]));
    }
    return v;
  }
};

// pass 1: grid (ceil(nx / L), 2 groups, ndir * lc slabs); instantiated per
// LNY = log2 ny.  Line l of group 0 is row m = r0 + l (E2 even + E1 odd), of
// group 1 row m = r0 + l + 1 (E3 odd).  T1 rows: E1 at m, E2 and E3 at m - 1.
template <typename T, int LNY>
__global__ void __launch_bounds__(FIELD_THREADS, 2) k_field_y(const C<T>* __restrict__ ap,
                                                           const C<T>* __restrict__ prof,
                                                           const C<T>* __restrict__ profq,
                                                           C<T>* __restrict__ T1, FP p,
                                                           const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  // odd line pitch: accesses across the lines of a block hit distinct banks
  constexpr int ny = 1 << LNY, n2 = 2 * ny, ls = padded_len(n2) | 1;
  constexpr int L = field_lines<T>(n2);
  const int grp = blockIdx.y, s = blockIdx.z;
  const int jj = s / p.ndir, d = s - jj * p.ndir;  // directions fastest: a level's profile is reused from L2
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  FieldCoef<T> cf;
  cf.E = ap + (size_t)d * p.nap;
  cf.Pj = prof + (size_t)(j - 1) * p.nap;
  cf.Qj = profq ? profq + (size_t)(j - 1) * (p.n1 + p.n2) : nullptr;
  cf.M = p.M;
  cf.N = p.N;
  cf.n1 = p.n1;
  cf.n2 = p.n2;
  cf.top = (j == p.nz);
  cf.layered = p.layered;
  const int r0 = blockIdx.x * L;
  const int mo = grp == 0 ? 0 : 1;  // row m of line l is r0 + l + mo
  // cooperative gather: consecutive threads take consecutive n of a row; all
  // loads of a thread are issued before its first store into the lines
  constexpr int PER = L * ny / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * ny, "rows must tile the block");
  C<T> ce[PER], so[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int m = r0 + (idx >> LNY) + mo, n = idx & (ny - 1);
    if (grp == 0) {
      ce[k] = cf(1, m, n);
      so[k] = cf(0, m, n);
    } else {
      ce[k] = mk<T>(0, 0);
      so[k] = cf(2, m, n);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int l = idx >> LNY, n = idx & (ny - 1);
    C<T>* line = buf + (size_t)l * ls;
    if (n == 0) {
      line[0] = cscale<T>(ce[k], (T)2);
      line[pidx(ny)] = mk<T>(0, 0);
    } else {
      line[pidx(n)] = cadd<T>(ce[k], so[k]);
      line[pidx(n2 - n)] = csub<T>(ce[k], so[k]);
    }
  }
  __syncthreads();
  fft_lines<T, true, LNY + 1>(buf, ls, L, tw, p.twlog);
  // split and store: cos part scaled by 1/2, sine part by 1/(2i)
  C<T>* t1 = T1 + (size_t)s * 3 * p.nx * (ny + 1);
  for (int idx = threadIdx.x; idx < L * (ny + 1); idx += FIELD_THREADS) {
    const int l = idx / (ny + 1), q = idx - l * (ny + 1);
    const int m = r0 + l + mo;
    if (m > p.M) continue;
    const C<T>* line = buf + (size_t)l * ls;
    const C<T> zq = line[pidx(q)];
    const C<T> zm = line[pidx((n2 - q) & (n2 - 1))];
    if (grp == 0) {
      const C<T> c = cscale<T>(cadd<T>(zq, zm), (T)0.25);
      const C<T> sn = cscale<T>(csub<T>(zq, zm), (T)0.25);
      t1[(size_t)m * (ny + 1) + q] = mk<T>(sn.y, -sn.x);  // E1 row m
      if (m >= 1) t1[((size_t)p.nx + m - 1) * (ny + 1) + q] = c;  // E2 row m - 1
    } else {
      t1[((size_t)2 * p.nx + m - 1) * (ny + 1) + q] = mk<T>(zq.y * (T)0.5, -zq.x * (T)0.5);
    }
  }
}

// pass 2: grid (ceil((ny+1) / L) column groups, 2 groups, ndir * lc slabs);
// instantiated per LNX = log2 nx.  Line l of group 0 is column q = q0 + l
// (E1 even + E2 odd), of group 1 column q = q0 + l + 1 (E3 odd).  The split
// samples are written a row segment of L columns at a time.
template <typename T, int LNX>
__global__ void __launch_bounds__(FIELD_THREADS, 2) k_field_x(const C<T>* __restrict__ T1,
                                                           C<T>* __restrict__ out, FP p,
                                                           const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int nx = 1 << LNX, n2 = 2 * nx, ls = padded_len(n2) | 1;
  constexpr int L = field_lines<T>(n2);
  const int ny = p.ny;
  const int grp = blockIdx.y, s = blockIdx.z;
  const int jj = s / p.ndir, d = s - jj * p.ndir;  // directions fastest: a level's profile is reused from L2
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  const C<T>* t1 = T1 + (size_t)s * 3 * nx * (ny + 1);
  const int q0 = blockIdx.x * L + (grp == 0 ? 0 : 1);
  const int qhi = grp == 0 ? ny : ny - 1;  // last column of the group
  constexpr int lL = clog2(L);
  constexpr int PER = L * nx / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * nx, "columns must tile the block");
  // cooperative gather of the L columns: consecutive threads take consecutive
  // columns of a T1 row (row t of the cos part is E1 row t, of the sine part
  // E2 / E3 row t - 1)
  C<T> ce[PER], so[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int t = idx >> lL, q = q0 + (idx & (L - 1));
    const bool in = q <= qhi;
    if (grp == 0) {
      ce[k] = (in && q >= 1 && q < ny) ? t1[(size_t)t * (ny + 1) + q] : mk<T>(0, 0);
      so[k] = (in && t >= 1) ? t1[((size_t)nx + t - 1) * (ny + 1) + q] : mk<T>(0, 0);
    } else {
      ce[k] = mk<T>(0, 0);
      so[k] = (in && t >= 1) ? t1[((size_t)2 * nx + t - 1) * (ny + 1) + q] : mk<T>(0, 0);
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int t = idx >> lL, l = idx & (L - 1);
    C<T>* line = buf + (size_t)l * ls;
    if (t == 0) {
      line[0] = cscale<T>(ce[k], (T)2);
      line[pidx(nx)] = mk<T>(0, 0);
    } else {
      line[pidx(t)] = cadd<T>(ce[k], so[k]);
      line[pidx(n2 - t)] = csub<T>(ce[k], so[k]);
    }
  }
  __syncthreads();
  fft_lines<T, true, LNX + 1>(buf, ls, L, tw, p.twlog);
  // split and store, consecutive threads on consecutive columns of a row
  C<T>* o = out + ((size_t)d * p.nz + (j - 1)) * p.S;
  const long long offE2 = (long long)(nx + 1) * (ny - 1);
  const long long offE3 = offE2 + (long long)(nx - 1) * (ny + 1);
  for (int idx = threadIdx.x; idx < (nx + 1) * L; idx += FIELD_THREADS) {
    const int pp = idx >> lL, l = idx & (L - 1);
    const int q = q0 + l;
    if (q > qhi) continue;
    const C<T>* line = buf + (size_t)l * ls;
    const C<T> zq = line[pidx(pp)];
    if (grp == 0) {
      const C<T> zm = line[pidx((n2 - pp) & (n2 - 1))];
      if (q >= 1 && q < ny) {  // E1 (cos in x1) on p = 0..nx
        const C<T> c = cscale<T>(cadd<T>(zq, zm), (T)0.25);
        o[(size_t)pp * (ny - 1) + (q - 1)] = c;
      }
      if (pp >= 1 && pp < nx) {  // E2 (sin in x1) on p = 1..nx-1
        const C<T> sn = cscale<T>(csub<T>(zq, zm), (T)0.25);
        o[offE2 + (size_t)(pp - 1) * (ny + 1) + q] = mk<T>(sn.y, -sn.x);
      }
    } else if (pp >= 1 && pp < nx) {  // E3 on p = 1..nx-1, q = 1..ny-1
      o[offE3 + (size_t)(pp - 1) * (ny - 1) + (q - 1)] = mk<T>(zq.y * (T)0.5, -zq.x * (T)0.5);
    }
  }
}

__global__ void k_ap32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

// the persistent single-kernel synthesis of field_fused.cu (complex64 field)
bool field_fused_supported(const Geo& g);
size_t field_fused_work_bytes(const Geo& g);
cavity_status launch_field_fused(cavity_ctx* ctx, int ndir, const float4* apr, float2* out,
                                 int j0, int nlev, void* work);
size_t ap_records_bytes(const Geo& g, int ndir);
cavity_status launch_ap_records(cavity_ctx* ctx, int ndir, const double2* ap, float4* rec);
cavity_status field_fused_check(cavity_ctx* ctx, void* work);

static cavity_status launch_field_fused_all(cavity_ctx* ctx, int ndir, const double2* ap,
                                            float2* out, void* host_out) {
  const Geo& g = ctx->g;
  const size_t apb = ((ap_records_bytes(g, ndir) + 255) / 256) * 256;
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, apb + field_fused_work_bytes(g)));
  float4* apr = (float4*)ctx->ws2;
  void* work = (char*)ctx->ws2 + apb;
  CKS(launch_ap_records(ctx, ndir, ap, apr));
  // device output: one launch over all levels; host output: chunks of levels,
  // each copied out (one segment per direction, over four copy streams)
  // while the next is synthesised
  const int nchunk = host_out ? std::min(g.nz, 8) : 1;
  const int lc = (g.nz + nchunk - 1) / nchunk;
  if (host_out) CKS(ensure_copy_stream(ctx, (size_t)nchunk + 2));
  int chunk = 0;
  for (int j0 = 1; j0 <= g.nz; j0 += lc, ++chunk) {
    const int nl = std::min(lc, g.nz - j0 + 1);
    CKS(launch_field_fused(ctx, ndir, apr, out, j0, nl, work));
    if (host_out) {
      cudaEvent_t ev = ctx->copy_evs[2 + chunk];
      CK(cudaEventRecord(ev, ctx->stream));
      cudaStream_t cs[4] = {ctx->copy_stream, ctx->copy_more[0], ctx->copy_more[1],
                            ctx->copy_more[2]};
      for (int k = 0; k < 4; ++k) CK(cudaStreamWaitEvent(cs[k], ev, 0));
      for (int d = 0; d < ndir; ++d) {
        const size_t off = ((size_t)d * g.nz + (j0 - 1)) * (size_t)g.field_per_level;
        CK(cudaMemcpyAsync((float2*)host_out + off, out + off,
                           sizeof(float2) * (size_t)nl * g.field_per_level,
                           cudaMemcpyDeviceToHost, cs[d & 3]));
      }
    }
  }
  return field_fused_check(ctx, work);
}

template <typename T>
cavity_status launch_field(cavity_ctx* ctx, int ndir, const double2* ap, C<T>* out,
                           void* host_out) {
  const Geo& g = ctx->g;
  if constexpr (sizeof(T) == 4) {
    if (field_fused_use(ctx)) return launch_field_fused_all(ctx, ndir, ap, out, host_out);
  }
  const bool layered = ctx->layers.size() > 1;
  const size_t slab = (size_t)3 * g.nx * (g.ny + 1) * sizeof(C<T>);
  int lc = (int)std::max<size_t>(1, ((size_t)512 << 20) / (slab * ndir));
  lc = std::min(lc, g.nz);
  const size_t t1 = slab * ndir * lc;
  const size_t apb = sizeof(C<T>) == 8 ? ((sizeof(float2) * (size_t)ndir * g.nap + 255) / 256) * 256 : 0;
  CKS(ensure_ws(ctx, &ctx->ws2, &ctx->ws2_bytes, t1 + apb));
  C<T>* T1 = (C<T>*)((char*)ctx->ws2 + apb);
  const C<T>* apT;
  const C<T>* prof;
  const C<T>* profq;
  if (sizeof(T) == 8) {
    apT = (const C<T>*)ap;
    prof = (const C<T>*)ctx->prof;
    profq = layered ? (const C<T>*)ctx->profq : nullptr;
  } else {
    float2* a32 = (float2*)ctx->ws2;
    long long n = (long long)ndir * g.nap;
    {
      KScope ks_(ctx, KC_FIELD_Y);
      k_ap32<<<(unsigned)((n + 255) / 256), 256, 0, ctx->stream>>>(ap, a32, n);
    }
    apT = (const C<T>*)a32;
    prof = (const C<T>*)ctx->prof32;
    profq = layered ? (const C<T>*)ctx->profq32 : nullptr;
  }
  const C<T>* tw = sizeof(T) == 8 ? (const C<T>*)ctx->tw64 : (const C<T>*)ctx->tw32;
  FP p;
  p.nx = g.nx; p.ny = g.ny; p.nz = g.nz; p.M = g.M; p.N = g.N; p.n1 = g.n1; p.n2 = g.n2;
  p.nap = g.nap; p.lnx = g.lnx; p.lny = g.lny; p.twlog = ilog2(ctx->TW);
  p.lc = lc; p.ndir = ndir; p.layered = layered; p.S = g.field_per_level;
  const int nchunk = (g.nz + lc - 1) / lc;
  if (host_out) CKS(ensure_copy_stream(ctx, (size_t)nchunk + 2));
  int chunk = 0;
  for (int j0 = 1; j0 <= g.nz; j0 += lc, ++chunk) {
    p.j0 = j0;
    CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lny, [&](auto c) -> cavity_status {
      constexpr int LN = decltype(c)::value, L = field_lines<T>(2 << LN);
      static std::atomic<bool> done{false};  // set once; host threads may race
      if (!done) {
        CK(allow_max_smem(k_field_y<T, LN>));
        done = true;
      }
      KScope ks_(ctx, KC_FIELD_Y);
      k_field_y<T, LN><<<dim3((g.nx + L - 1) / L, 2, ndir * lc), FIELD_THREADS,
                         sizeof(C<T>) * (size_t)L * (padded_len(2 << LN) | 1), ctx->stream>>>(
          apT, prof, profq, T1, p, tw);
      return CAVITY_OK;
    }));
    CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lnx, [&](auto c) -> cavity_status {
      constexpr int LN = decltype(c)::value, L = field_lines<T>(2 << LN);
      static std::atomic<bool> done{false};  // set once; host threads may race
      if (!done) {
        CK(allow_max_smem(k_field_x<T, LN>));
        done = true;
      }
      KScope ks_(ctx, KC_FIELD_X);
      k_field_x<T, LN><<<dim3((g.ny + 1 + L - 1) / L, 2, ndir * lc), FIELD_THREADS,
                         sizeof(C<T>) * (size_t)L * (padded_len(2 << LN) | 1), ctx->stream>>>(
          T1, out, p, tw);
      return CAVITY_OK;
    }));
    if (host_out) {
      // this chunk's levels of every direction to the host while the next
      // chunk is synthesised (one contiguous segment per direction)
      // segments round-robin over four copy streams (several copy engines)
      cudaEvent_t ev = ctx->copy_evs[2 + chunk];
      CK(cudaEventRecord(ev, ctx->stream));
      cudaStream_t cs[4] = {ctx->copy_stream, ctx->copy_more[0], ctx->copy_more[1],
                            ctx->copy_more[2]};
      for (int k = 0; k < 4; ++k) CK(cudaStreamWaitEvent(cs[k], ev, 0));
      const int nl = std::min(lc, g.nz - j0 + 1);
      for (int d = 0; d < ndir; ++d) {
        const size_t off = ((size_t)d * g.nz + (j0 - 1)) * (size_t)g.field_per_level;
        CK(cudaMemcpyAsync((C<T>*)host_out + off, out + off,
                           sizeof(C<T>) * (size_t)nl * g.field_per_level, cudaMemcpyDeviceToHost,
                           cs[d & 3]));
      }
    }
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

template cavity_status launch_field<double>(cavity_ctx*, int, const double2*, double2*, void*);
template cavity_status launch_field<float>(cavity_ctx*, int, const double2*, float2*, void*);
