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
// intermediate fits in L2, so HBM traffic is essentially the field write plus
// the profile read (amortised over the directions of a batch).
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
// instantiated per LNY = log2 ny
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
  const int r0 = blockIdx.x * L;
  const int d = s / p.lc, jj = s - d * p.lc;
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const C<T>* E = ap + (size_t)d * p.nap;
  const bool top = (j == p.nz);
  const C<T>* Pj = prof + (size_t)(j - 1) * p.nap;
  const C<T>* Qj = profq ? profq + (size_t)(j - 1) * (p.n1 + p.n2) : nullptr;
  const bool ycos = (comp == 1);
  // coefficients of the L rows, loaded first (all loads in flight), then
  // mirrored into the lines: every slot except n = ny (and n = 0 for the sine
  // extension) is written, so only those are cleared
  constexpr int PER = L * ny / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * ny, "rows must tile the block");
  C<T> cv[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * FIELD_THREADS;
    const int l = idx >> LNY, n = idx & (ny - 1);
    const int r = r0 + l;
    const int m = comp == 0 ? r : r + 1;
    int i = -1;
    if (r < p.nx && m <= p.M) {
      if (comp == 0) { if (n >= 1) i = m * p.N + (n - 1); }
      else if (comp == 1) i = p.n1 + (m - 1) * (p.N + 1) + n;
      else if (n >= 1) i = p.n1 + p.n2 + (m - 1) * p.N + (n - 1);
    }
    C<T> c = mk<T>(0, 0);
    if (i >= 0) {
      c = E[i];
      if (!top) {
        c = cmul<T>(Pj[i], c);
        if (p.layered && comp < 2 && m >= 1 && n >= 1)
          c = cadd<T>(c, cmul<T>(Qj[i], E[p.n1 + p.n2 + (m - 1) * p.N + (n - 1)]));
      }
    }
    cv[k] = c;
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * FIELD_THREADS;
    const int l = idx >> LNY, n = idx & (ny - 1);
    C<T>* line = buf + (size_t)l * ls;
    const C<T> c = cv[k];
    if (n == 0) {
      line[0] = ycos ? cscale<T>(c, (T)2) : mk<T>(0, 0);
      line[pidx(ny)] = mk<T>(0, 0);
    } else if (ycos) {
      line[pidx(n)] = c;
      line[pidx(n2 - n)] = c;
    } else {
      line[pidx(n)] = c;
      line[pidx(n2 - n)] = mk<T>(-c.x, -c.y);
    }
  }
  __syncthreads();
  fft_lines<T, true, LNY + 1>(buf, ls, L, tw, p.twlog);
  C<T>* dst = T1 + (((size_t)s * 3 + comp) * p.nx + r0) * (ny + 1);
  const int nr = min(L, p.nx - r0);
  for (int idx = tid; idx < nr * (ny + 1); idx += nthr) {
    const int l = idx / (ny + 1), q = idx - l * (ny + 1);
    const C<T> v = buf[(size_t)l * ls + pidx(q)];
    // cos: Z/2 ; sin: Z/(2i)
    dst[idx] = ycos ? mk<T>(v.x * (T)0.5, v.y * (T)0.5) : mk<T>(v.y * (T)0.5, -v.x * (T)0.5);
  }
}

// pass 2: grid (ceil((ny+1) / L) column groups, 3 components, ndir * lc
// slabs); instantiated per LNX = log2 nx
template <typename T, int LNX>
__global__ void __launch_bounds__(FIELD_THREADS, 2) k_field_x(const C<T>* __restrict__ T1,
                                                           C<T>* __restrict__ out, FP p,
                                                           const C<T>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  C<T>* buf = (C<T>*)sm_raw;
  constexpr int nx = 1 << LNX, n2 = 2 * nx, ls = padded_len(n2);
  constexpr int L = field_lines<T>(n2), lL = clog2(L);
  const int ny = p.ny;
  const int comp = blockIdx.y, s = blockIdx.z;
  const int q0 = blockIdx.x * L;
  const int d = s / p.lc, jj = s - d * p.lc;
  const int j = p.j0 + jj;
  if (j > p.nz) return;
  const int tid = threadIdx.x, nthr = blockDim.x;
  const bool xcos = (comp == 0);
  const C<T>* src = T1 + ((size_t)s * 3 + comp) * nx * (ny + 1);
  // rows r of the L columns, loaded first, then mirrored; unwritten slots
  // (m = nx, and m = 0 for the sine extension) are cleared
  constexpr int PER = L * nx / FIELD_THREADS;
  static_assert(PER * FIELD_THREADS == L * nx, "columns must tile the block");
  const int nrows = xcos ? nx : nx - 1;    // E1: m = 0..M; E2/E3: m = 1..M
  C<T> cv[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * FIELD_THREADS;
    const int r = idx >> lL, l = idx & (L - 1);
    const int q = q0 + l;
    cv[k] = (q <= ny && r < nrows) ? src[(size_t)r * (ny + 1) + q] : mk<T>(0, 0);
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int idx = tid + k * FIELD_THREADS;
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
      const int m = r + 1;
      line[pidx(m)] = c;
      line[pidx(n2 - m)] = mk<T>(-c.x, -c.y);
    } else {
      line[0] = mk<T>(0, 0);
      line[pidx(nx)] = mk<T>(0, 0);
    }
  }
  __syncthreads();
  fft_lines<T, true, LNX + 1>(buf, ls, L, tw, p.twlog);
  long long off;
  int ncol, qlo, qhi, plo, phi;
  if (comp == 0) { off = 0; ncol = ny - 1; qlo = 1; qhi = ny - 1; plo = 0; phi = nx; }
  else if (comp == 1) { off = (long long)(nx + 1) * (ny - 1); ncol = ny + 1; qlo = 0; qhi = ny; plo = 1; phi = nx - 1; }
  else { off = (long long)(nx + 1) * (ny - 1) + (long long)(nx - 1) * (ny + 1); ncol = ny - 1; qlo = 1; qhi = ny - 1; plo = 1; phi = nx - 1; }
  C<T>* dst = out + ((size_t)d * p.nz + (j - 1)) * p.S + off;
  const int np = phi - plo + 1;
  for (int idx = tid; idx < L * np; idx += nthr) {
    const int pr = idx >> lL, l = idx & (L - 1);
    const int q = q0 + l;
    if (q < qlo || q > qhi) continue;
    const C<T> v = buf[(size_t)l * ls + pidx(plo + pr)];
    dst[(size_t)pr * ncol + (q - qlo)] =
        xcos ? mk<T>(v.x * (T)0.5, v.y * (T)0.5) : mk<T>(v.y * (T)0.5, -v.x * (T)0.5);
  }
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
  int lc = (int)std::max<size_t>(1, ((size_t)64 << 20) / (slab * ndir));
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
