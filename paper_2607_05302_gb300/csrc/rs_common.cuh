// Shared device helpers of the Radsort CUDA library (sm_103a).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "rs_kernels.cuh"

namespace rs {

// ---------------------------------------------------------------- status
// Sticky device status word (bit set = error class seen); read and cleared by
// radsort_device_status().  Kernels never trap: they record and return.
// One word per translation unit (no relocatable device code needed); each
// unit exports a host function that reads and clears its word.
static __device__ unsigned g_status = 0;

static inline unsigned take_status_word()
{
    unsigned v = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&v, g_status, sizeof(v)) != cudaSuccess)
        return ST_INTERNAL;
    cudaMemcpyToSymbol(g_status, &zero, sizeof(zero));
    return v;
}

__device__ __forceinline__ void set_status(unsigned bits) { atomicOr(&g_status, bits); }

// Iteration limit of every spin-wait (each iteration sleeps >= 64 ns, so the
// limit is several seconds of wall time on a healthy GPU).
constexpr unsigned SPIN_LIMIT = 1u << 26;

// True once any wait of this translation unit has run out: the other waits
// give up at their next check instead of running out one after another.
__device__ __forceinline__ bool wait_failed()
{
    return (*reinterpret_cast<volatile unsigned *>(&g_status) & ST_TIMEOUT) != 0;
}

// ---------------------------------------------------------------- smem / mbarrier / bulk copy
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase with the given parity to complete.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity)
{
    for (unsigned it = 0; it < SPIN_LIMIT; ++it) {
        if (mbar_try_wait(bar, parity))
            return true;
        if ((it & 1023u) == 1023u && wait_failed())
            return false;
        __nanosleep(64);
    }
    set_status(ST_TIMEOUT);
    return false;
}

// Orders this thread's earlier generic-proxy accesses to shared memory before
// later async-proxy (bulk copy) accesses to the same bytes.  Every thread that
// read or wrote a buffer with plain loads and stores executes it before the
// barrier / mbarrier arrive that hands the buffer back to a bulk-copy issuer.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared through the TMA engine; completion is
// signalled on `bar` as transaction bytes.  dst, src and bytes must be
// multiples of 16.
__device__ __forceinline__ void bulk_g2s(void *dst_smem, const void *src_gmem, uint32_t bytes,
                                         uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// ---------------------------------------------------------------- warp / block scans
__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T> __device__ __forceinline__ T warp_incl_scan(T v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o)
            v += t;
    }
    return v;
}

template <typename T> __device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Named barrier over the first `nthreads` threads of the block (id != 0).
__device__ __forceinline__ void named_bar(int id, int nthreads)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
}

// Mask of the lanes whose digit equals this lane's, among lanes with
// `valid` set: one ballot per digit bit (warp-level multisplit).  All 32
// lanes must call it.
template <int DB> __device__ __forceinline__ unsigned peer_mask(uint32_t d, bool valid)
{
    unsigned m = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int bit = 0; bit < DB; ++bit) {
        const bool on = (d >> bit) & 1u;
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        m &= on ? bal : ~bal;
    }
    return m;
}

// ---------------------------------------------------------------- keys
template <typename KT> __device__ __forceinline__ uint32_t digit_of(KT k, uint32_t shift,
                                                                     uint32_t mask)
{
    return static_cast<uint32_t>(k >> shift) & mask;
}

} // namespace rs
