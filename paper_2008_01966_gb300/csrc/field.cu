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

// pass 1: grid (ceil(nx / L) row groups, 3 components, ndir * lc slabs);
// instantiated per LNY = log2 ny.  A cooperative gather forms the
// coefficients (profile times aperture value) and mirrors them into the lines;
// the scaled store of T1 (q <= ny) is the transform's last write.
template <typename T, int LNY>
struct FieldY {
  const C<T>* E;                  // aperture coefficients of this direction
  const C<T>* Pj;                 // profiles of level j
  const C<T>* Qj;                 // E3-driven profiles of level j (layered) or null
  C<T>* dst;                      // T1 rows of this (slab, component)
  int r0, nx, M, N, n1, n2, comp;
  bool top, layered;
  __device__ __forceinline__ C<T> coef(int r, int n) const {
    const int m = comp == 0 ? r : r + 1;
    if (r >= nx || m > M) return mk<T>(0, 0);
    int i;
    if (comp == 0) {
      if (n < 1) return mk<T>(0, 0);
      i = m * N + (n - 1);
    } else if (comp == 1) {
      i = n1 + (m - 1) * (N + 1) + n;
    } else {
      if (n < 1) return mk<T>(0, 0);
      i = n1 + n2 + (m - 1) * N + (n - 1);
    }
    C<T> c = E[i];
    if (!top) {
      c = cmul<T>(Pj[i], c);
      if (layered && comp < 2 && m >= 1 && n >= 1)
        c = cadd<T>(c, cmul<T>(Qj[i], E[n1 + n2 + (m - 1) * N + (n - 1)]));
    }
    return c;
  }
  __device__ __forceinline__ C<T> ld(int l, const C<T>*, int k) const {
    constexpr int ny = 1 << LNY, n2x = 2 * ny;
    const bool ycos = comp == 1;
    const int r = r0 + l;
    if (k < ny) {
      if (k == 0) return ycos ? cscale<T>(coef(r, 0), (T)2) : mk<T>(0, 0);
      return coef(r, k);
    }
    if (k == ny) return mk<T>(0, 0);
    const C<T> c = coef(r, n2x - k);
    return ycos ? c : mk<T>(-c.x, -c.y);
  }
  __device__ __forceinline__ void st(int l, C<T>*, int q, C<T> v) const {
    constexpr int ny = 1 << LNY;
    const int r = r0 + l;
    if (q > ny || r >= nx) return;
    // cos: Z/2 ; sin: Z/(2i)
    dst[(size_t)r * (ny + 1) + q] =
        comp == 1 ? mk<T>(v.x * (T)0.5, v.y * (T)0.5) : mk<T>(v.y * (T)0.5, -v.x * (T)0.5);
  }
};

// the gathered line as the first read, FieldY's store as the last write
template <typename T, int LNY>
struct FieldYStore : FieldY<T, LNY> {
  __device__ __forceinline__ C<T> ld(int, const C<T>* line, int t) const { return line[pidx(t)]; }
};

template <typename T, int LNY>
__global__ void __launch_bounds__(FIELD_THREADS, 2) k_field_y(const C<T>* __restrict__ ap,
                                                           const C<T>* __restrict__ prof,
                                                           const C<T>* __restrict__ profq,
                                                           C<T>* __restrict__ T1, FP p,
                                                           const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int ny = 1 << LNY, n2 = 2 * ny, ls = padded_len(n2);
  constexpr int L = field_lines<T>(n2);
  const int comp = blockIdx.y, s = blockIdx.z;
  const int d = s / p.lc, jj = s - d * p.lc;
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  FieldY<T, LNY> op;
  op.E = ap + (size_t)d * p.nap;
  op.Pj = prof + (size_t)(j - 1) * p.nap;
  op.Qj = profq ? profq + (size_t)(j - 1) * (p.n1 + p.n2) : nullptr;
  op.dst = T1 + ((size_t)s * 3 + comp) * p.nx * (ny + 1);
  op.r0 = blockIdx.x * L;
  op.nx = p.nx;
  op.M = p.M;
  op.N = p.N;
  op.n1 = p.n1;
  op.n2 = p.n2;
  op.comp = comp;
  op.top = (j == p.nz);
  op.layered = p.layered;
  // cooperative gather: consecutive threads take consecutive n of a row, all
  // of a thread's loads are issued before its first store, and the mirrored
  // coefficients go straight into the lines (every slot is written)
  constexpr int PER = L * ny / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * ny, "rows must tile the block");
  C<T> cv[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    cv[k] = op.coef(op.r0 + (idx >> LNY), idx & (ny - 1));
  }
  const bool ycos = comp == 1;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int l = idx >> LNY, n = idx & (ny - 1);
    C<T>* line = buf + (size_t)l * ls;
    const C<T> c = cv[k];
    if (n == 0) {
      line[0] = ycos ? cscale<T>(c, (T)2) : mk<T>(0, 0);
      line[pidx(ny)] = mk<T>(0, 0);
    } else {
      line[pidx(n)] = c;
      line[pidx(n2 - n)] = ycos ? c : mk<T>(-c.x, -c.y);
    }
  }
  __syncthreads();
  FieldYStore<T, LNY> st;
  static_cast<FieldY<T, LNY>&>(st) = op;
  fft_lines<T, true, LNY + 1>(buf, ls, L, tw, p.twlog, st);
}

// pass 2: grid (ceil((ny+1) / L) column groups, 3 components, ndir * lc
// slabs); instantiated per LNX = log2 nx.  The column gather of T1 and the
// mirroring are the transform's first read, the scaled store of the output
// rows its last write.
template <typename T, int LNX>
struct FieldX {
  const C<T>* src;                // T1 rows of this (slab, component)
  C<T>* dst;                      // this component's output block of level j
  int q0, ny, comp, ncol, qlo, qhi, plo, phi;
  __device__ __forceinline__ C<T> ld(int l, const C<T>*, int t) const {
    constexpr int nx = 1 << LNX, n2 = 2 * nx;
    const int q = q0 + l;
    if (q > ny || t == nx) return mk<T>(0, 0);
    const bool xcos = comp == 0;
    // E1: rows r = m (m = 0..nx-1); E2, E3: rows r = m - 1 (m = 1..nx-1)
    if (t < nx) {
      if (t == 0) return xcos ? cscale<T>(src[q], (T)2) : mk<T>(0, 0);
      return src[(size_t)(xcos ? t : t - 1) * (ny + 1) + q];
    }
    const int m = n2 - t;
    const C<T> c = src[(size_t)(xcos ? m : m - 1) * (ny + 1) + q];
    return xcos ? c : mk<T>(-c.x, -c.y);
  }
  __device__ __forceinline__ void st(int l, C<T>*, int pp, C<T> v) const {
    const int q = q0 + l;
    if (pp < plo || pp > phi || q < qlo || q > qhi) return;
    dst[(size_t)(pp - plo) * ncol + (q - qlo)] =
        comp == 0 ? mk<T>(v.x * (T)0.5, v.y * (T)0.5) : mk<T>(v.y * (T)0.5, -v.x * (T)0.5);
  }
};

// the gathered line as the first read, FieldX's store as the last write
template <typename T, int LNX>
struct FieldXStore : FieldX<T, LNX> {
  __device__ __forceinline__ C<T> ld(int, const C<T>* line, int t) const { return line[pidx(t)]; }
};

template <typename T, int LNX>
__global__ void __launch_bounds__(FIELD_THREADS, 2) k_field_x(const C<T>* __restrict__ T1,
                                                           C<T>* __restrict__ out, FP p,
                                                           const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int nx = 1 << LNX, n2 = 2 * nx, ls = padded_len(n2);
  constexpr int L = field_lines<T>(n2);
  const int ny = p.ny;
  const int comp = blockIdx.y, s = blockIdx.z;
  const int d = s / p.lc, jj = s - d * p.lc;
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  FieldX<T, LNX> op;
  op.src = T1 + ((size_t)s * 3 + comp) * nx * (ny + 1);
  op.q0 = blockIdx.x * L;
  op.ny = ny;
  op.comp = comp;
  long long off;
  if (comp == 0) {
    off = 0; op.ncol = ny - 1; op.qlo = 1; op.qhi = ny - 1; op.plo = 0; op.phi = nx;
  } else if (comp == 1) {
    off = (long long)(nx + 1) * (ny - 1);
    op.ncol = ny + 1; op.qlo = 0; op.qhi = ny; op.plo = 1; op.phi = nx - 1;
  } else {
    off = (long long)(nx + 1) * (ny - 1) + (long long)(nx - 1) * (ny + 1);
    op.ncol = ny - 1; op.qlo = 1; op.qhi = ny - 1; op.plo = 1; op.phi = nx - 1;
  }
  op.dst = out + ((size_t)d * p.nz + (j - 1)) * p.S + off;
  // cooperative gather of the L columns of T1: consecutive threads take
  // consecutive columns of a row, all loads of a thread in flight before its
  // first store; mirrored into the lines (slots m = nx, and m = 0 for the sine
  // extension, cleared)
  constexpr int lL = clog2(L);
  constexpr int PER = L * nx / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * nx, "columns must tile the block");
  const bool xcos = comp == 0;
  const int nrows = xcos ? nx : nx - 1;    // E1: m = 0..M; E2/E3: m = 1..M
  C<T> cv[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int r = idx >> lL, q = op.q0 + (idx & (L - 1));
    cv[k] = (q <= ny && r < nrows) ? op.src[(size_t)r * (ny + 1) + q] : mk<T>(0, 0);
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = threadIdx.x + k * FIELD_THREADS;
    const int r = idx >> lL, l = idx & (L - 1);
    C<T>* line = buf + (size_t)l * ls;
    const C<T> c = cv[k];
    if (xcos) {
      if (r == 0) {
        line[0] = cscale<T>(c, (T)2);
        line[pidx(nx)] = mk<T>(0, 0);
      } else {
        line[pidx(r)] = c;
        line[pidx(n2 - r)] = c;
      }
    } else if (r < nx - 1) {
      line[pidx(r + 1)] = c;
      line[pidx(n2 - r - 1)] = mk<T>(-c.x, -c.y);
    } else {
      line[0] = mk<T>(0, 0);
      line[pidx(nx)] = mk<T>(0, 0);
    }
  }
  __syncthreads();
  FieldXStore<T, LNX> st;
  static_cast<FieldX<T, LNX>&>(st) = op;
  fft_lines<T, true, LNX + 1>(buf, ls, L, tw, p.twlog, st);
}

__global__ void k_ap32(const double2* __restrict__ a, float2* __restrict__ b, long long n) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k < n) b[k] = make_float2((float)a[k].x, (float)a[k].y);
}

template <typename T>
cavity_status launch_field(cavity_ctx* ctx, int ndir, const double2* ap, C<T>* out) {
  const Geo& g = ctx->g;
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
  for (int j0 = 1; j0 <= g.nz; j0 += lc) {
    p.j0 = j0;
    CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lny, [&](auto c) -> cavity_status {
      constexpr int LN = decltype(c)::value, L = field_lines<T>(2 << LN);
      static bool done = false;
      if (!done) {
        CK(allow_max_smem(k_field_y<T, LN>));
        done = true;
      }
      KScope ks_(ctx, KC_FIELD_Y);
      k_field_y<T, LN><<<dim3((g.nx + L - 1) / L, 3, ndir * lc), FIELD_THREADS,
                         sizeof(C<T>) * (size_t)L * padded_len(2 << LN), ctx->stream>>>(
          apT, prof, profq, T1, p, tw);
      return CAVITY_OK;
    }));
    CKS(dispatch_log<CAV_LOG_MIN, CAV_LOG_MAX>(g.lnx, [&](auto c) -> cavity_status {
      constexpr int LN = decltype(c)::value, L = field_lines<T>(2 << LN);
      static bool done = false;
      if (!done) {
        CK(allow_max_smem(k_field_x<T, LN>));
        done = true;
      }
      KScope ks_(ctx, KC_FIELD_X);
      k_field_x<T, LN><<<dim3((g.ny + 1 + L - 1) / L, 3, ndir * lc), FIELD_THREADS,
                         sizeof(C<T>) * (size_t)L * padded_len(2 << LN), ctx->stream>>>(
          T1, out, p, tw);
      return CAVITY_OK;
    }));
  }
  CK(cudaGetLastError());
  return CAVITY_OK;
}

template cavity_status launch_field<double>(cavity_ctx*, int, const double2*, double2*);
template cavity_status launch_field<float>(cavity_ctx*, int, const double2*, float2*);
