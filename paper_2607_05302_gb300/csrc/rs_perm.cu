// Kernels of the permuted representation kept between calls (Sec. 4.1,
// "Avoiding Finalisation"), grid layout: the digit histograms of the current
// logical sequence read through the block map, the list of its blocks in
// logical order, and the partial-block state after a truncation (Alg. 8).
//
// In the grid layout every logical data block but the last is full (a round
// writes its output on the block grid, and setup and truncation leave only
// the final block partial), so the sequence is described by the block map
// pi and the element count n alone: logical block H + q holds elements
// [q*b, (q+1)*b) of the sequence.
#include "radsort.h"
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_perm() { return take_status_word(); }

namespace {

// Counts of every digit position over the sequence's elements, read block by
// block through pi (a histogram of the multiset, so any order will do).
// Consecutive threads read consecutive elements of one block.
template <typename KT, int DB>
__global__ void __launch_bounds__(512) k_block_hist(const KT *Ak, const KT *Tk, const uint32_t *pi,
                                                    uint32_t H, uint32_t nT, uint32_t npi, uint32_t lb,
                                                    uint32_t n, uint32_t *hist)
{
    constexpr int SIGMA = 1 << DB;
    constexpr int NTD = (8 * int(sizeof(KT)) + DB - 1) / DB;
    extern __shared__ uint32_t sh[];
    for (int i = threadIdx.x; i < NTD * SIGMA; i += blockDim.x)
        sh[i] = 0;
    __syncthreads();
    const uint32_t mask = (1u << lb) - 1;
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        const uint32_t phys = pi[H + (e >> lb)];
        if (phys >= npi) {
            set_status(ST_INTERNAL);
            continue;
        }
        const KT *blk = phys < nT ? Tk + (size_t(phys) << lb) : Ak + (size_t(phys - nT) << lb);
        const KT k = blk[e & mask];
#pragma unroll
        for (int r = 0; r < NTD; ++r)
            atomicAdd(&sh[r * SIGMA + digit_of(k, uint32_t(r * DB), SIGMA - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < NTD * SIGMA; i += blockDim.x)
        if (sh[i])
            atomicAdd(&hist[i], sh[i]);
}

// Entry q of the list: logical block H + q as (key address, value address,
// used elements); the final block (logical H + floor(n/b)) holds n mod b.
template <typename KT>
__global__ void k_block_list(const KT *Ak, const uint32_t *Av, const KT *Tk, const uint32_t *Tv,
                             const uint32_t *pi, uint32_t H, uint32_t nT, uint32_t npi, uint32_t lb,
                             uint32_t n, radsort_block *out)
{
    const uint32_t nfull = n >> lb, nl = nfull + 1;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < nl; q += gridDim.x * blockDim.x) {
        const uint32_t phys = pi[H + q];
        radsort_block r{};
        if (phys < npi) {
            const size_t off = size_t(phys < nT ? phys : phys - nT) << lb;
            r.keys = reinterpret_cast<uint64_t>((phys < nT ? Tk : Ak) + off);
            r.values = Av ? reinterpret_cast<uint64_t>((phys < nT ? Tv : Av) + off) : 0ull;
            r.len = q < nfull ? (1u << lb) : n - (nfull << lb);
        } else {
            set_status(ST_INTERNAL);
        }
        out[q] = r;
    }
}

// The state after keeping the first n elements: the final block is logical
// H + floor(n/b) with n mod b elements (an empty partial block when b
// divides n, reading G15 of Alg. 8), f = that block + 1, one partial block.
__global__ void k_set_tail(uint2 *P, uint32_t *state, uint32_t H, uint32_t lb, uint32_t n)
{
    const uint32_t q = n >> lb;
    P[0] = make_uint2(H + q, n - (q << lb));
    state[ST_F] = H + q + 1;
    state[ST_NP] = 1;
}

} // namespace

cudaError_t launch_block_hist(const Geom &g, const Bufs &w, const uint32_t *pi, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(w.hist, 0, size_t(g.nt) * g.sigma * 4, st);
    if (e != cudaSuccess || g.n == 0)
        return e;
    const uint32_t n = static_cast<uint32_t>(g.n);
    int grid = num_sms() * 2;
    const int need = static_cast<int>((g.n + 511) / 512);
    if (grid > need)
        grid = need;
    const size_t smem = size_t(g.nt) * g.sigma * 4;
    using u64 = unsigned long long;
    if (g.kb == 4 && g.db == 8)
        k_block_hist<uint32_t, 8><<<grid, 512, smem, st>>>(static_cast<const uint32_t *>(w.Ak),
                                                            static_cast<const uint32_t *>(w.Tk), pi, g.H,
                                                            g.nT, g.npi, g.lb, n, w.hist);
    else if (g.kb == 4)
        k_block_hist<uint32_t, 11><<<grid, 512, smem, st>>>(static_cast<const uint32_t *>(w.Ak),
                                                             static_cast<const uint32_t *>(w.Tk), pi, g.H,
                                                             g.nT, g.npi, g.lb, n, w.hist);
    else if (g.db == 8)
        k_block_hist<u64, 8><<<grid, 512, smem, st>>>(static_cast<const u64 *>(w.Ak),
                                                       static_cast<const u64 *>(w.Tk), pi, g.H, g.nT, g.npi,
                                                       g.lb, n, w.hist);
    else
        k_block_hist<u64, 11><<<grid, 512, smem, st>>>(static_cast<const u64 *>(w.Ak),
                                                        static_cast<const u64 *>(w.Tk), pi, g.H, g.nT,
                                                        g.npi, g.lb, n, w.hist);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_block_list(const Geom &g, const Bufs &w, const uint32_t *pi, radsort_block *out,
                              cudaStream_t st)
{
    const uint32_t n = static_cast<uint32_t>(g.n);
    const uint32_t nl = (n >> g.lb) + 1;
    int grid = static_cast<int>((nl + 255) / 256);
    if (grid > num_sms() * 8)
        grid = num_sms() * 8;
    using u64 = unsigned long long;
    if (g.kb == 4)
        k_block_list<uint32_t><<<grid, 256, 0, st>>>(static_cast<const uint32_t *>(w.Ak), g.hasv ? w.Av : nullptr,
                                                     static_cast<const uint32_t *>(w.Tk), w.Tv, pi, g.H, g.nT,
                                                     g.npi, g.lb, n, out);
    else
        k_block_list<u64><<<grid, 256, 0, st>>>(static_cast<const u64 *>(w.Ak), g.hasv ? w.Av : nullptr,
                                                static_cast<const u64 *>(w.Tk), w.Tv, pi, g.H, g.nT, g.npi,
                                                g.lb, n, out);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_set_tail(const Geom &g, const Bufs &w, cudaStream_t st)
{
    k_set_tail<<<1, 1, 0, st>>>(w.P, w.state, g.H, g.lb, static_cast<uint32_t>(g.n));
    g_launches += 1;
    return cudaGetLastError();
}

} // namespace rs
