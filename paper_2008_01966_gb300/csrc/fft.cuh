// Shared-memory FFTs of power-of-two length for the cavity solver.
//
// All transforms of the hot path -- the Fourier-series synthesis (E123F), the
// trapezoid projections and the torus convolution of Sec. 5.2 -- are batches
// of 1-D transforms of lines held in shared memory.  A CTA transforms
// `nlines` consecutive lines of length n (line stride n) at once; every thread
// loops over the butterflies of all lines, so the same routine serves one long
// line per CTA and many short lines per CTA.
//
// Algorithm: Stockham auto-sort, radix 4 with one leading radix-2 stage when
// log2(n) is odd, ping-ponging between two shared buffers (out-of-place per
// stage, natural-order output).  Twiddles come from a table
// tw[k] = exp(-2 pi i k / TW) (TW a power of two >= n) computed once in FP64
// and rounded for the FP32 table, so no transcendental is evaluated here.
// Forward = exp(-...), inverse = exp(+...) without normalisation.
#pragma once
#include "common.cuh"

template <typename T, bool INV>
__device__ __forceinline__ void bfly4(C<T>& v0, C<T>& v1, C<T>& v2, C<T>& v3) {
  C<T> s0 = cadd<T>(v0, v2), d0 = csub<T>(v0, v2);
  C<T> s1 = cadd<T>(v1, v3), d1 = csub<T>(v1, v3);
  C<T> id1 = cmul_i<T>(d1);
  v0 = cadd<T>(s0, s1);
  v2 = csub<T>(s0, s1);
  if (!INV) {
    v1 = csub<T>(d0, id1);
    v3 = cadd<T>(d0, id1);
  } else {
    v1 = cadd<T>(d0, id1);
    v3 = csub<T>(d0, id1);
  }
}

template <typename T, bool INV>
__device__ __forceinline__ C<T> twid(const C<T>* __restrict__ tw, int idx) {
  C<T> w = tw[idx];
  if (INV) w.y = -w.y;
  return w;
}

// Transform `nlines` lines of length n = 2^logn stored consecutively in `a`.
// `b` is scratch of the same size.  Returns the buffer holding the result.
// Must be called by all threads of the CTA (contains __syncthreads()).
template <typename T, bool INV>
__device__ C<T>* fft_lines(C<T>* a, C<T>* b, int n, int logn, int nlines,
                           const C<T>* __restrict__ tw, int twlog) {
  const int tid = threadIdx.x + threadIdx.y * blockDim.x;
  const int nthr = blockDim.x * blockDim.y;
  C<T>* in = a;
  C<T>* out = b;
  int s = 0;  // log2(Ns)
  if (logn & 1) {
    // radix-2 stage with Ns = 1 (no twiddles)
    const int nb = n >> 1;
    const int total = nb * nlines;
    for (int t = tid; t < total; t += nthr) {
      const int l = t / nb, j = t - l * nb;
      const C<T>* li = in + l * n;
      C<T>* lo = out + l * n;
      C<T> v0 = li[j], v1 = li[j + nb];
      lo[2 * j] = cadd<T>(v0, v1);
      lo[2 * j + 1] = csub<T>(v0, v1);
    }
    __syncthreads();
    C<T>* t_ = in; in = out; out = t_;
    s = 1;
  }
  while (s < logn) {
    const int Ns = 1 << s;
    const int nb = n >> 2;
    const int total = nb * nlines;
    const int shift = twlog - (s + 2);  // tw index step for exp(-2 pi i/(4 Ns))
    for (int t = tid; t < total; t += nthr) {
      const int l = t / nb, j = t - l * nb;
      const C<T>* li = in + l * n;
      C<T>* lo = out + l * n;
      const int k = j & (Ns - 1);
      C<T> v0 = li[j], v1 = li[j + nb], v2 = li[j + 2 * nb], v3 = li[j + 3 * nb];
      if (s > 0) {
        v1 = cmul<T>(v1, twid<T, INV>(tw, (k) << shift));
        v2 = cmul<T>(v2, twid<T, INV>(tw, (2 * k) << shift));
        v3 = cmul<T>(v3, twid<T, INV>(tw, (3 * k) << shift));
      }
      bfly4<T, INV>(v0, v1, v2, v3);
      const int base = ((j - k) << 2) + k;
      lo[base] = v0;
      lo[base + Ns] = v1;
      lo[base + 2 * Ns] = v2;
      lo[base + 3 * Ns] = v3;
    }
    __syncthreads();
    C<T>* t_ = in; in = out; out = t_;
    s += 2;
  }
  return in;
}
