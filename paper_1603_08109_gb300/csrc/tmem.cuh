// Tensor memory (TMEM) as per-thread private storage for non-MMA kernels.
//
// Each SM has 128 lanes x 512 columns of 32-bit tensor memory.  A CTA of 128
// threads that allocates kCols columns gives every thread one lane: warp w
// reads and writes lanes 32w .. 32w + 31 (its lane quadrant), thread t the
// kCols words of lane t.  tcgen05.ld / tcgen05.st move consecutive columns
// of the thread's lane to and from registers at several times the bandwidth
// of shared memory and without its bank structure, which makes TMEM a
// register-file extension for values a thread re-reads many times.
//
// Allocation discipline: one warp allocates and frees; a kernel that uses
// these helpers must be limited (by its shared memory) to 512 / kCols
// resident CTAs per SM so that an allocation never has to wait, and must
// free on every path.  tcgen05.ld / tcgen05.st are warp-collective
// (.sync.aligned): every lane of the warp executes them, outside divergent
// code.
#pragma once
#include <cstdint>

namespace bft {

constexpr int kCols = 128;

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Warp-collective: allocate kCols columns, write the base address to *dst
// (shared memory), give up the right to allocate again.
__device__ __forceinline__ void alloc(uint32_t *dst) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(dst)),
               "n"(kCols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

// Warp-collective: free the columns at taddr.
__device__ __forceinline__ void dealloc(uint32_t taddr) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "n"(kCols)
               : "memory");
}

// Order tensor-memory operations across a block barrier.
__device__ __forceinline__ void fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Wait until this thread's tcgen05.st operations have completed.
__device__ __forceinline__ void wait_st() {
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// Columns [taddr, taddr + 12) / [taddr, taddr + 6) of this thread's lane.
// The loads wait for their data inside the same asm statement, so no use of
// the results can be scheduled before it has arrived.  As volatile asm these
// keep their order among themselves and with wait_st (a load after a store
// to the same columns follows a wait_st); they touch no memory the compiler
// sees, so shared-memory accesses may be scheduled around them.
__device__ __forceinline__ void st12(uint32_t taddr, const float (&v)[12]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%1], {%10, %11, %12, %13};" ::"r"(taddr),
      "r"(taddr + 8), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]),
      "f"(v[7]), "f"(v[8]), "f"(v[9]), "f"(v[10]), "f"(v[11]));
}

__device__ __forceinline__ void st6(uint32_t taddr, const float (&v)[6]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%2, %3, %4, %5};\n\t"
      "tcgen05.st.sync.aligned.32x32b.x2.b32 [%1], {%6, %7};" ::"r"(taddr),
      "r"(taddr + 4), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]));
}

__device__ __forceinline__ void ld12(uint32_t taddr, float (&v)[12]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%12];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%8, %9, %10, %11}, [%13];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]),
        "=f"(v[7]), "=f"(v[8]), "=f"(v[9]), "=f"(v[10]), "=f"(v[11])
      : "r"(taddr), "r"(taddr + 8));
}

__device__ __forceinline__ void ld6(uint32_t taddr, float (&v)[6]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%6];\n\t"
      "tcgen05.ld.sync.aligned.32x32b.x2.b32 {%4, %5}, [%7];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5])
      : "r"(taddr), "r"(taddr + 4));
}

}  // namespace bft
