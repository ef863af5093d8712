// Fifth-generation tensor cores (tcgen05) for FP32-accurate real GEMM tiles:
// D[M x N] (FP32, in tensor memory) += A[M x K] B[K x N] with TF32 operands
// staged in shared memory, one MMA issued by one thread, completion tracked
// by an mbarrier.
//
// Operand layout in shared memory: K-major, no swizzle.  A tile of R rows and
// 8 K elements (one MMA k-step of kind::tf32) is made of 8-row x 16-byte core
// matrices: element (row, k) at byte (row / 8) * 256 + (k / 4) * 128 +
// (row % 8) * 16 + (k % 4) * 4, so the leading-dimension byte offset (between
// the two core matrices along K) is 128 and the stride-dimension byte offset
// (between 8-row groups) is 256; a tile takes 32 R bytes.
//
// FP32 accuracy from TF32 products: each operand is split into TF32 parts,
// x = hi + lo, and the product is hi_A hi_B + (lo_A hi_B + hi_A lo_B) (the
// dropped lo lo term is below 2^-22 |x y|).  The tensor-core accumulator does
// not keep FP32 accuracy over long sums: measured on a GB300 for 4096 inner
// terms, one accumulator for all three products gave a relative error of
// 2.7e-5 (the same as hi hi alone, 2.6e-5: the corrections are lost); with
// the corrections in a second accumulator, 9.8e-6; with both drained into
// FP32 registers every 1, 4 or 16 MMA k-steps (8, 32 or 128 terms), 3.5e-7,
// 1.9e-7, 3.0e-7.  So the kernels keep hi hi and the corrections in two
// accumulators and drain them every TC_DRAIN chunks.
//
// Every wait on an mbarrier is bounded; a wait that runs out returns false and
// the caller records an error instead of spinning forever.
#pragma once
#include <stdint.h>

#include <cuda_runtime.h>

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// byte offset of element (row, k), k < 8, in a K-major tile of one k-step
__device__ __forceinline__ int tc_koff(int row, int k) {
  return (row >> 3) * 256 + (k >> 2) * 128 + (row & 7) * 16 + (k & 3) * 4;
}
// shared-memory matrix descriptor: start address, LBO 128, SBO 256, version 1
// (tcgen05 descriptors), no swizzle
__device__ __forceinline__ uint64_t tc_desc(const void* tile) {
  const uint32_t a = tc_smem_u32(tile);
  uint64_t d = (uint64_t)((a >> 4) & 0x3FFF);
  d |= (uint64_t)(128 >> 4) << 16;
  d |= (uint64_t)(256 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// instruction descriptor of kind::tf32: FP32 accumulator, TF32 A and B, both
// K-major, M x N
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ uint32_t tc_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ void tc_split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tc_tf32(x);
  lo = tc_tf32(x - __uint_as_float(hi));
}

// tensor memory: allocated by one whole warp; the base address is written to
// shared memory
__device__ __forceinline__ void tc_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
               ::"r"(tc_smem_u32(slot)), "r"(ncols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tc_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                       uint32_t idesc, uint32_t accumulate) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
               ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
// the mbarrier receives one arrival when every MMA issued so far by this
// thread has completed
__device__ __forceinline__ void tc_commit(uint64_t* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               ::"r"(tc_smem_u32(mbar)));
}
__device__ __forceinline__ void tc_mbar_init(uint64_t* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc_smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;");
}
// bounded wait for phase `parity` of the mbarrier
__device__ __forceinline__ bool tc_mbar_wait(uint64_t* mbar, uint32_t parity) {
  uint32_t done = 0;
  for (long long it = 0; it < (1ll << 22) && !done; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}\n"
                 : "=r"(done) : "r"(tc_smem_u32(mbar)), "r"(parity) : "memory");
  }
  return done != 0;
}
// After a wait ran out: the issuing thread waits, again bounded, for the MMAs
// it still has in flight before the tensor memory is freed.  A commit
// arrives once every MMA issued before it has completed, so the last one
// covers all: `last` is the last chunk whose MMAs were committed (to
// mbar[last & 1], phase last >> 1), -1 if none.
__device__ __forceinline__ void tc_settle(uint64_t* mbar, int last) {
  if (last >= 0) (void)tc_mbar_wait(&mbar[last & 1], (last >> 1) & 1);
}
// operand tiles written by threads become visible to the tensor cores
__device__ __forceinline__ void tc_fence_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
// chunks (of two k-steps) between drains of the accumulators: 128 inner terms
#define TC_DRAIN 8

// 32 lanes x 32 columns of FP32 from tensor memory (warp w of a warpgroup
// reads lanes 32 w .. 32 w + 31): thread t gets lane 32 w + t, columns c0..c0+31
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
               "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
               "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                 "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]),
                 "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                 "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]),
                 "=r"(r[30]), "=r"(r[31])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// add the two accumulators (hi hi at taddr, corrections at taddr + 32) of this
// thread's lane into acc
__device__ __forceinline__ void tc_drain(uint32_t taddr, float (&acc)[32]) {
  float a[32], b[32];
  tc_ld32(taddr, a);
  tc_ld32(taddr + 32, b);
#pragma unroll
  for (int j = 0; j < 32; ++j) acc[j] += a[j] + b[j];
}
