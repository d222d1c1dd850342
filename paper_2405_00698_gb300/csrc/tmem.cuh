// Tensor memory (TMEM) as per-thread storage next to the register file.
//
// An SM's 256 KB of tensor memory is 128 lanes x 512 columns of 32-bit cells.  A warp reaches
// only the 32 lanes of its quarter (warp % 4), so with the 24 warps of a 768-thread block six
// warps share each quarter and each can own 80 columns: 80 private 32-bit cells per thread.  The
// adjoint's reverse sweep, which leaves the tensor cores idle, keeps there the per-thread arrays
// that do not fit in its registers (instead of spilling them to local memory, which with the
// sweep's shared-memory footprint misses L1).
//
// tcgen05.ld / tcgen05.st are warp-collective (.sync.aligned): every thread of the warp issues
// them together with the same address.  Loads are asynchronous: the registers they fill are read
// only after tcgen05.wait::ld, which here takes those registers as operands so that the compiler
// cannot move a use of them above the wait.  A store must have completed (tcgen05.wait::st)
// before a later load of the same cells.
#pragma once

#include <cstdint>

namespace vx {

constexpr int kTmemAllocCols = 512;
constexpr int kTmemColsPerWarp = 80;

// Allocation by one whole warp; the base address is written to shared memory at *dst.
__device__ __forceinline__ void tmem_alloc_warp(uint32_t* dst)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     (uint32_t)__cvta_generic_to_shared(dst)),
                 "r"(kTmemAllocCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_dealloc_warp(uint32_t base)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(base), "r"(kTmemAllocCols));
}

__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// This warp's first cell: lane quarter warp % 4, columns 80 * (warp / 4) onwards.
__device__ __forceinline__ uint32_t tmem_warp_base(uint32_t base, int warp)
{
    return base + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemColsPerWarp * (warp >> 2));
}

// Two consecutive columns of this thread's lane (the first even).
__device__ __forceinline__ void tmem_ld2(uint32_t ta, uint32_t& x, uint32_t& y)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x2.b32 {%0, %1}, [%2];" : "=r"(x), "=r"(y) : "r"(ta));
}

__device__ __forceinline__ void tmem_st2(uint32_t ta, uint32_t x, uint32_t y)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x2.b32 [%0], {%1, %2};" ::"r"(ta), "r"(x), "r"(y) : "memory");
}

// Four consecutive columns (the first a multiple of 4).
__device__ __forceinline__ void tmem_ld4(uint32_t ta, uint32_t& x, uint32_t& y, uint32_t& z, uint32_t& w)
{
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(x), "=r"(y), "=r"(z), "=r"(w)
                 : "r"(ta));
}

__device__ __forceinline__ void tmem_st4(uint32_t ta, uint32_t x, uint32_t y, uint32_t z, uint32_t w)
{
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(ta), "r"(x), "r"(y), "r"(z),
                 "r"(w)
                 : "memory");
}

// Wait for this thread's outstanding loads; the six registers they fill become readable.
__device__ __forceinline__ void tmem_wait_ld6(uint32_t (&r)[6])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5])
                 :
                 : "memory");
}

__device__ __forceinline__ void tmem_wait_ld4(uint32_t (&r)[4])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;" : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]) : : "memory");
}

__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

}  // namespace vx
