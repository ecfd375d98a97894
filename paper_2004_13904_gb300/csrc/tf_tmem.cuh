// Tensor memory (TMEM, sm_100 family) as per-thread private storage for the column kernels.
//
// Each SM has 128 lanes x 512 columns of 32-bit TMEM.  A CTA allocates a power-of-two
// number of columns (32 .. 512) across all 128 lanes; warp w of the CTA reaches lanes
// 32 (w mod 4) .. 32 (w mod 4) + 31, and with the 32x32b access shape every thread of the
// warp reads or writes its own lane.  Warps w and w + 4 share lanes, so they use disjoint
// column ranges.  TMEM traffic does not use the shared-memory banks that the FFT passes
// work through, so values a thread keeps across the layer loop (the layer accumulator of
// G x) can live there instead of in shared memory.
//
// Rules kept by the callers: every tcgen05 instruction here is warp-collective
// (.sync.aligned), so it is executed by all 32 threads of a warp with the same address;
// the CTA deallocates exactly what it allocated before it exits; the resident CTAs of an
// SM never hold more than its 512 columns (the caller caps residency through its shared
// memory request), so an allocation never waits.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace tfk {
namespace tmem {

// Allocate ncols columns (warp-collective; one warp of the CTA); the TMEM address is
// written to the shared word *slot.
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t ncols) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(slot);
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(s), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Release (warp-collective; the warp that allocated).
__device__ __forceinline__ void dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// Ordering of TMEM operations around a CTA barrier.
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// The address of this thread's lane at column col of the allocation based at taddr.
__device__ __forceinline__ uint32_t lane_addr(uint32_t taddr, int col) {
  return taddr + ((uint32_t)(((threadIdx.x >> 5) & 3) * 32) << 16) + (uint32_t)col;
}

// Four consecutive 32-bit columns of this thread's lane.  The load and its wait are one
// asm statement, so no use of the registers can be scheduled before the data arrive.
// TMEM is not memory the compiler tracks: loads, stores and waits keep their order as
// volatile asm statements, and need no memory clobber (which would also pin the
// surrounding global and shared accesses).
__device__ __forceinline__ void ld4(uint32_t a, float* v) {
  uint32_t r0, r1, r2, r3;
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
      : "r"(a));
  v[0] = __uint_as_float(r0);
  v[1] = __uint_as_float(r1);
  v[2] = __uint_as_float(r2);
  v[3] = __uint_as_float(r3);
}
// 16 consecutive columns (load and wait in one statement, as ld4).
__device__ __forceinline__ void ld16(uint32_t a, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(a));
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void st4(uint32_t a, const float* v) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(a),
               "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
               "r"(__float_as_uint(v[3])));
}
// Wait for this thread's earlier stores (before the same columns are loaded again).
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace tmem
}  // namespace tfk
