// Radsort rounds with one block chain per bucket for the whole array, and the
// out-of-place comparison sort (Alg. 1), on one pipelined round kernel for
// sm_103a.
//
// Grid layout of the block chains.  The paper's parallel variant (Sec. 4.3)
// gives every chunk its own head start and its own open block per bucket, so
// the scratch array grows with the chunk count (2*sigma*p blocks).  Here all
// CTAs share one free list and one chain per bucket, like the sequential
// algorithm (Alg. 5 with a head start of sigma blocks, Sec. 2.1), and the
// chains are laid on the block grid of the round's output: logical data block
// j holds output positions [j*b, (j+1)*b) of the stably sorted sequence.  A
// block that contains the start of a bucket (strictly inside) is shared by
// two or more buckets; every other block belongs to one bucket.
//   * The bucket sizes of every digit come from one upfront histogram pass
//     (the paper's "generic" variant, Sec. 5), so bucket c's output range
//     [O_c, O_c + n_c) and the shared blocks are known before a round.
//   * Before the round, the shared blocks (fewer than sigma) and the first
//     L = GRID_AHEAD non-shared blocks of every bucket take the first
//     nP < (L+1)*sigma free-list entries.
//   * A tile learns where its elements of bucket c go, O_c + E_c(t), from a
//     decoupled look-back over the per-bucket counts of earlier tiles.
//     Every other block j of bucket c is taken eagerly, as newBucketBlock
//     does in Alg. 5 but L blocks ahead: by the tile that writes the first
//     position of block j - L, at a free-list index in  nP + (blocks taken
//     by earlier tiles) + [0, blocks this tile takes); the count for earlier
//     tiles follows from E(t) alone, the order within the tile is free.  A tile that continues
//     a block therefore finds it taken long before (a bounded wait covers
//     the rest), and tiles in flight together do not wait on each other.
//   * The free list is the current logical order: (L+2)*sigma head-start
//     blocks, then the input blocks in order.  Tiles are dispatched in input
//     order, a tile reads its blocks before it publishes its counts, and
//     after the tiles up to t at most  nP + (elements)/b + sigma <
//     (L+2)*sigma + (blocks read)  blocks have been taken (Lemma 1 with a
//     head start of (L+2)*sigma).
//   * The tile that takes a block records it in the next block map pi',
//     where later tiles find it.
// The next round's head start is the (L+2)*sigma entries after the last
// taken one, so the scratch array holds (L+2)*sigma + 1 blocks whatever the
// number of CTAs, and after the last round every block but the array's tail
// is full: Finalize is a block permutation plus one tail copy.
//
// Round kernel (both layouts): a producer warp takes tiles in ticket order
// and streams them into a ring of shared-memory stages with bulk copies
// (TMA) that complete on mbarriers; the consumer warps rank each tile's
// digits stably, publish the tile's per-digit counts, reorder the tile by
// digit in shared memory, resolve the global per-digit offsets by look-back,
// and store each digit run into its output blocks (Radsort) or contiguously
// (out of place).  Look-back words live in a ring of R tiles x sigma 64-bit
// words: (tag << 32) | value, the tag naming the round and the tile, the
// value the tile's count or 0x80000000 | inclusive prefix (n < 2^31).  Tile t
// reuses the slot of tile t - R only after every tile up to t - R + 1 has
// finished its look-back (per-slot done tags that the producer checks).  A
// reader that finds a slot already reused starts its look-back over: tile
// t - R + 1 is inclusive by then, so the new walk stops above the reused slot.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_oop() { return take_status_word(); }

namespace {

constexpr uint32_t LB_INCL = 0x80000000u;
constexpr uint32_t PI_NONE = 0xFFFFFFFFu;
constexpr uint32_t SH_NONE = 0xFFFFu;
constexpr uint32_t TILE_END = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p)
{
    return *reinterpret_cast<const volatile uint32_t *>(p);
}
__device__ __forceinline__ void st_volatile(uint32_t *p, uint32_t v)
{
    *reinterpret_cast<volatile uint32_t *>(p) = v;
}
__device__ __forceinline__ unsigned long long ld_volatile64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ void st_volatile64(unsigned long long *p, unsigned long long v)
{
    *reinterpret_cast<volatile unsigned long long *>(p) = v;
}
__device__ __forceinline__ unsigned long long lbw(uint32_t tag, uint32_t v)
{
    return (static_cast<unsigned long long>(tag) << 32) | v;
}

// ---------------------------------------------------------------- digit histograms
// Counts of every digit position in one read of the keys.  Each thread
// keeps, per digit position, the digit of its last key and the run length,
// and adds a run to the shared histogram when the digit changes (one atomic
// per key on random keys, one per run on sorted or constant ones).  Four
// 16-byte loads per thread are in flight per step.
template <typename KT, int DB>
__global__ void __launch_bounds__(512) k_digit_hist(const KT *keys, uint32_t n, uint32_t *hist)
{
    constexpr int SIGMA = 1 << DB;
    constexpr int NTD = (8 * int(sizeof(KT)) + DB - 1) / DB;
    constexpr int V = 16 / sizeof(KT), U = 4;
    extern __shared__ uint32_t sh[];
    for (int i = threadIdx.x; i < NTD * SIGMA; i += blockDim.x)
        sh[i] = 0;
    __syncthreads();
    uint32_t last[NTD], run[NTD];
#pragma unroll
    for (int r = 0; r < NTD; ++r) {
        last[r] = 0;
        run[r] = 0;
    }
    auto put = [&](KT k) {
#pragma unroll
        for (int r = 0; r < NTD; ++r) {
            const uint32_t d = digit_of(k, uint32_t(r * DB), SIGMA - 1);
            if (d == last[r]) {
                ++run[r];
            } else {
                if (run[r])
                    atomicAdd(&sh[r * SIGMA + last[r]], run[r]);
                last[r] = d;
                run[r] = 1;
            }
        }
    };
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    const size_t first = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    const size_t nv = vec ? n / V : 0;
    const uint4 *kv = reinterpret_cast<const uint4 *>(keys);
    for (size_t i = first; i < nv; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < nv)
                v[u] = kv[i + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < nv) {
                KT k[V];
                memcpy(k, &v[u], 16);
#pragma unroll
                for (int q = 0; q < V; ++q)
                    put(k[q]);
            }
    }
    for (size_t i = nv * V + first; i < n; i += stride)
        put(keys[i]);
#pragma unroll
    for (int r = 0; r < NTD; ++r)
        if (run[r])
            atomicAdd(&sh[r * SIGMA + last[r]], run[r]);
    __syncthreads();
    for (int i = threadIdx.x; i < NTD * SIGMA; i += blockDim.x)
        if (sh[i])
            atomicAdd(&hist[i], sh[i]);
}

// 8-bit digits: counts of four digit positions r0 .. r0+3 with one counter
// column per lane (counter (r, d) of lane l at word (r*256 + d)*32 + l), so
// the 32 atomics of a warp instruction fall in 32 different banks whatever
// the digits.  One CTA of 1024 threads per SM, 128 KB of counters.
template <typename KT>
__global__ void __launch_bounds__(1024) k_digit_hist_lanes(const KT *keys, uint32_t n, int r0, uint32_t *hist)
{
    constexpr int NTD = 8 * int(sizeof(KT)) / 8;
    constexpr int G = 4; // digit positions per pass
    constexpr int V = 16 / sizeof(KT);
    extern __shared__ uint32_t sh[]; // G * 256 * 32
    const int lane = threadIdx.x & 31;
    for (int i = threadIdx.x; i < G * 256 * 32; i += blockDim.x)
        sh[i] = 0;
    __syncthreads();
    const int npos = min(G, NTD - r0);
    auto put = [&](KT k) {
#pragma unroll
        for (int r = 0; r < G; ++r)
            if (r < npos)
                atomicAdd(&sh[(r * 256 + digit_of(k, uint32_t((r0 + r) * 8), 255u)) * 32 + lane], 1u);
    };
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    const size_t first = size_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
    const size_t nv = vec ? n / V : 0;
    const uint4 *kv = reinterpret_cast<const uint4 *>(keys);
    constexpr int U = 4;
    for (size_t i = first; i < nv; i += U * stride) {
        uint4 v[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < nv)
                v[u] = kv[i + u * stride];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i + u * stride < nv) {
                KT k[V];
                memcpy(k, &v[u], 16);
#pragma unroll
                for (int q = 0; q < V; ++q)
                    put(k[q]);
            }
    }
    for (size_t i = nv * V + first; i < n; i += stride)
        put(keys[i]);
    __syncthreads();
    // per (position, digit): the sum of the 32 lane columns
    for (int i = threadIdx.x; i < npos * 256; i += blockDim.x) {
        const uint32_t *row = sh + size_t(i) * 32;
        uint32_t sum = 0;
#pragma unroll
        for (int l = 0; l < 32; ++l)
            sum += row[(l + i) & 31]; // rotated start: consecutive threads, different banks
        if (sum)
            atomicAdd(&hist[(r0 + i / 256) * 256 + (i % 256)], sum);
    }
}

// Launches the digit histograms for the key and digit widths.
static cudaError_t launch_digit_hist(const void *keys, uint32_t n, int kb, int db, uint32_t *hist,
                                     cudaStream_t st)
{
    using u64 = unsigned long long;
    if (db == 8) {
        constexpr int LSM = 4 * 256 * 32 * 4;
        static DeviceOnce attr;
        const cudaError_t ea = attr.run([] {
            cudaError_t e = cudaFuncSetAttribute(k_digit_hist_lanes<uint32_t>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, LSM);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_digit_hist_lanes<u64>, cudaFuncAttributeMaxDynamicSharedMemorySize, LSM);
            return e;
        });
        if (ea != cudaSuccess)
            return ea;
        const int grid = num_sms();
        if (kb == 4) {
            k_digit_hist_lanes<uint32_t><<<grid, 1024, LSM, st>>>(static_cast<const uint32_t *>(keys), n, 0, hist);
            g_launches += 1;
        } else {
            for (int r0 = 0; r0 < 8; r0 += 4)
                k_digit_hist_lanes<u64><<<grid, 1024, LSM, st>>>(static_cast<const u64 *>(keys), n, r0, hist);
            g_launches += 2;
        }
        return cudaGetLastError();
    }
    const int grid = num_sms() * 2;
    if (kb == 4)
        k_digit_hist<uint32_t, 11><<<grid, 512, 3 * 2048 * 4, st>>>(static_cast<const uint32_t *>(keys), n, hist);
    else
        k_digit_hist<u64, 11><<<grid, 512, 6 * 2048 * 4, st>>>(static_cast<const u64 *>(keys), n, hist);
    g_launches += 1;
    return cudaGetLastError();
}

// Exclusive scan over an N-element array by NT threads (each thread a run of
// IPT consecutive elements); returns the total.  t: the caller's index among
// the NT threads (whole warps: thread t is lane t % 32 of the group's warp
// t / 32), bar: a barrier over exactly those threads.  tmp: NT/32+1 words.
// Ends with a barrier.
template <int N, int NT, typename F>
__device__ __forceinline__ uint32_t block_scan(uint32_t *a, uint32_t *tmp, F &&bar, int t)
{
    constexpr int NWARP = NT / 32;
    constexpr int IPT = (N + NT - 1) / NT;
    const int lane = t & 31, w = t >> 5;
    uint32_t v[IPT], s = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = t * IPT + i;
        v[i] = idx < N ? a[idx] : 0;
        s += v[i];
    }
    const uint32_t inc = warp_incl_scan(s);
    if (lane == 31)
        tmp[w] = inc;
    bar();
    if (w == 0) {
        const uint32_t x = lane < NWARP ? tmp[lane] : 0;
        const uint32_t sx = warp_incl_scan(x);
        if (lane < NWARP)
            tmp[lane] = sx - x;
        if (lane == 31)
            tmp[NWARP] = sx;
    }
    bar();
    uint32_t e = inc - s + tmp[w];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = t * IPT + i;
        if (idx < N)
            a[idx] = e;
        e += v[i];
    }
    const uint32_t tot = tmp[NWARP];
    bar();
    return tot;
}

// Per-round bucket offsets of the out-of-place sort: O[r][c] exclusive over
// digits, O[r][sigma] = n (one block per digit position).
template <int DB> __global__ void __launch_bounds__(1024) k_offsets(const uint32_t *hist, uint32_t *off, uint32_t n)
{
    constexpr int SIGMA = 1 << DB;
    __shared__ uint32_t s_a[SIGMA], s_tmp[40];
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        s_a[c] = hist[r * SIGMA + c];
    __syncthreads();
    block_scan<SIGMA, 1024>(s_a, s_tmp, [] { __syncthreads(); }, threadIdx.x);
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        off[r * (SIGMA + 1) + c] = s_a[c];
    if (threadIdx.x == 0)
        off[r * (SIGMA + 1) + SIGMA] = n;
}

// ---------------------------------------------------------------- grid layout: setup, tables
// pi = [scratch 0 .. H) ++ [A's blocks] ++ [scratch block H: the input
// tail]; the tail is copied there; P holds the one partial block.
template <typename KT>
__global__ void k_grid_setup(const KT *Ak, const uint32_t *Av, KT *Tk, uint32_t *Tv, uint32_t n,
                             uint32_t b, uint32_t H, uint32_t nA, uint32_t npi, uint32_t *pi,
                             uint2 *P, uint32_t *state)
{
    const uint32_t nT = H + 1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npi; i += gridDim.x * blockDim.x)
        pi[i] = i < H ? i : (i < H + nA ? nT + (i - H) : H);
    const uint32_t tail = n - nA * b;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < tail; j += gridDim.x * blockDim.x) {
        Tk[size_t(H) * b + j] = Ak[size_t(nA) * b + j];
        if (Av)
            Tv[size_t(H) * b + j] = Av[size_t(nA) * b + j];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        P[0] = make_uint2(H + nA, tail);
        state[ST_F] = H + nA + 1;
        state[ST_NP] = 1;
        state[ST_FPREV] = H + nA + 1;
        state[ST_LOFFTOT] = 0;
    }
}

// Tables of one round (one CTA of 1024 threads): bucket starts O, the shared
// blocks (those with a bucket start strictly inside), per bucket the ranks
// of its first / last block among the shared ones and its range of
// non-shared blocks [ns0, ns1); pi' prefilled with the blocks taken before
// the round (shared blocks, then the first non-shared block of each bucket),
// the next head start and (n % b == 0) the empty tail block.  A digit with
// one non-empty bucket leaves the sequence unchanged: pi' = pi and the round
// is skipped.
template <int DB>
__global__ void __launch_bounds__(1024) k_grid_prep(const uint32_t *hist_r, uint32_t n, uint32_t lb,
                                                     uint32_t H, uint32_t nA, uint32_t npi,
                                                     const uint32_t *pi, uint32_t *pin,
                                                     uint32_t *tab, uint32_t *state, uint32_t clear)
{
    constexpr int SIGMA = 1 << DB;
    // s_a: scan buffer; s_list: bucket of the k-th bucket start strictly
    // inside a block, later the k-th shared block
    __shared__ uint32_t s_O[SIGMA + 1], s_cnt[SIGMA], s_a[SIGMA], s_list[SIGMA], s_tmp[40];
    __shared__ int s_skip;
    const uint32_t b = 1u << lb;
    auto bar = [] { __syncthreads(); };
    // a small map is cleared here rather than by a memset launch
    for (uint32_t i = threadIdx.x; i < clear; i += blockDim.x)
        pin[H + i] = 0xFFFFFFFFu;
    if (threadIdx.x == 0)
        s_skip = 0;
    __syncthreads();
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x) {
        const uint32_t v = hist_r[c];
        s_cnt[c] = v;
        s_O[c] = v;
        if (v == n)
            s_skip = 1;
    }
    __syncthreads();
    block_scan<SIGMA, 1024>(s_O, s_tmp, bar, threadIdx.x);
    if (s_skip) {
        for (uint32_t i = threadIdx.x; i < npi; i += blockDim.x)
            pin[i] = pi[i];
        if (threadIdx.x == 0)
            state[ST_SKIP] = 1;
        return;
    }
    if (threadIdx.x == 0)
        s_O[SIGMA] = n;
    // bucket starts strictly inside a block, in order
    auto inner = [&](int c) { return s_cnt[c] > 0 && (s_O[c] & (b - 1)) != 0; };
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        s_a[c] = inner(c) ? 1u : 0u;
    __syncthreads();
    block_scan<SIGMA, 1024>(s_a, s_tmp, bar, threadIdx.x);
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        if (inner(c))
            s_list[s_a[c]] = static_cast<uint32_t>(c);
    __syncthreads();
    // the first start inside each block makes it a shared block
    uint32_t fl[(SIGMA + 1023) / 1024];
    int q = 0;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x, ++q) {
        bool first = false;
        if (inner(c)) {
            const uint32_t r = s_a[c];
            first = r == 0 || (s_O[s_list[r - 1]] >> lb) != (s_O[c] >> lb);
        }
        fl[q] = first ? 1u : 0u;
    }
    __syncthreads();
    q = 0;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x, ++q)
        s_a[c] = fl[q];
    __syncthreads();
    const uint32_t nS = block_scan<SIGMA, 1024>(s_a, s_tmp, bar, threadIdx.x);
    q = 0;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x, ++q)
        if (fl[q])
            s_list[s_a[c]] = s_O[c] >> lb;
    __syncthreads();
    auto find = [&](uint32_t j) -> uint32_t { // rank of shared block j, or SH_NONE
        uint32_t lo = 0, hi = nS;
        while (lo < hi) {
            const uint32_t m = (lo + hi) >> 1;
            if (s_list[m] < j)
                lo = m + 1;
            else
                hi = m;
        }
        return (lo < nS && s_list[lo] == j) ? lo : SH_NONE;
    };
    uint32_t *tO = tab, *tns0 = tab + SIGMA + 1, *tns1 = tns0 + SIGMA, *tsh = tns1 + SIGMA;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x) {
        const uint32_t O = s_O[c], cn = s_cnt[c];
        uint32_t ns0, ns1, fsh = SH_NONE, lsh = SH_NONE;
        if (cn > 0) {
            const uint32_t jf = O >> lb, jl = (O + cn - 1) >> lb;
            fsh = find(jf);
            lsh = find(jl);
            ns0 = jf + (fsh != SH_NONE ? 1u : 0u);
            ns1 = jl + 1 - (lsh != SH_NONE ? 1u : 0u);
            if (ns1 < ns0)
                ns1 = ns0;
        } else {
            ns0 = ns1 = (O + b - 1) >> lb;
        }
        tO[c] = O;
        tns0[c] = ns0;
        tns1[c] = ns1;
        tsh[c] = fsh | (lsh << 16);
    }
    __syncthreads();
    // the first GRID_AHEAD non-shared blocks of each bucket: entries nS .. nP-1
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        s_a[c] = min(GRID_AHEAD, tns1[c] - tns0[c]);
    __syncthreads();
    const uint32_t nF = block_scan<SIGMA, 1024>(s_a, s_tmp, bar, threadIdx.x);
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x) {
        const uint32_t k = min(GRID_AHEAD, tns1[c] - tns0[c]);
        for (uint32_t i = 0; i < k; ++i)
            pin[H + tns0[c] + i] = pi[nS + s_a[c] + i];
    }
    if (threadIdx.x == 0) {
        tO[SIGMA] = n;
        state[ST_SKIP] = 0;
        state[ST_NS] = nS + nF;
    }
    // pi': shared blocks take free-list entries 0 .. nS-1; the entries after
    // the last data block taken form the next head start
    const uint32_t NB = (n + b - 1) >> lb;
    for (uint32_t k = threadIdx.x; k < nS; k += blockDim.x)
        pin[H + s_list[k]] = pi[k];
    for (uint32_t i = threadIdx.x; i < H; i += blockDim.x)
        pin[i] = pi[NB + i];
    if (threadIdx.x == 0 && NB == nA)
        pin[H + nA] = pi[NB + H]; // the empty tail block
    // the round reads free-list entries 0 .. H + nA only; blocks past them
    // (free blocks left behind when the sequence was cut short, Alg. 8) keep
    // their map entries
    for (uint32_t i = H + nA + 1 + threadIdx.x; i < npi; i += blockDim.x)
        pin[i] = pi[i];
}

// ---------------------------------------------------------------- round kernel
template <typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES, bool OOP> struct LbCfg {
    static constexpr int SIGMA = 1 << DB;
    // NG consumer groups of NW warps each; a group takes every NG-th tile and
    // works through it on its own (its own named barrier, tables and lists),
    // so the latency-bound phases of one group (look-back, block lists,
    // stores) overlap the shared-memory-bound phases of another
    static constexpr int NT = NW * 32;            // consumer threads per group
    static constexpr int THREADS = NG * NT + 32;  // + one producer warp
    static constexpr int MAXM = TILE / 64;   // blocks per tile (b >= 64)
    static constexpr int R = TILE / NW;      // tile elements ranked per warp
    static constexpr int ITEMS = R / 32;     // elements per consumer thread
    static_assert(R % 32 == 0, "warp range must be a multiple of 32");
    static_assert(THREADS <= 1024, "one CTA holds at most 1024 threads");
    // stage s serves group s % NG only: a group waits on the phases of its
    // own stages, in order (a stage shared by two groups could let one group
    // see an earlier phase of the other's fill as its own)
    static_assert(STAGES % NG == 0, "stages split evenly between the groups");
    // threads per bucket in the column passes (each sums NW / TPB warp rows):
    // measured with 16 warps, one thread per bucket is fastest for sigma =
    // 256 (round 1.86 -> 1.83 ms at 2^28); for sigma = 2048 two were 5%
    // faster at 2^26 but at 2^30 u64 left some rounds 3x slower, four do not
    static constexpr int TPB = NW >= 16 ? (DB <= 8 ? 1 : 4) : (NT >= (1 << DB) ? 1 : 2);
    static_assert(NW % TPB == 0, "rows split evenly");
    // more than 16 elements per thread: digits are recomputed from the keys
    // and warp ranks kept as 16-bit halves, to stay within the registers
    static constexpr bool LEAN = ITEMS > 16;
    // CTAs per SM the configuration is built for (registers are capped to fit)
    static constexpr int MINB = (NG * NW <= 8 && DB <= 8) ? 2 : 1;
    // sigma <= 256: a per-warp table of 32-bit lane masks by digit, built
    // with shared-memory atomicOr; sigma = 2048: one ballot per digit bit.
    // Either way a per-warp 16-bit row keeps the running count of each
    // digit, later the warp's start per digit in the reordered tile.
    static constexpr bool PTAB = DB <= 8;
    static constexpr bool PAIR = HASV && sizeof(KT) == 4;
    static constexpr int HROW = SIGMA + 2;
    // sigma <= 256: bucket tables and block lists (key / value pointers) in
    // shared memory; sigma = 2048: tables read from global memory, block
    // lists of block indices
    static constexpr bool SMALL = DB <= 8;
    static constexpr size_t al(size_t x) { return (x + 127) & ~size_t(127); }
    // 16 bytes of slack per array: the lead of a misaligned source (out of place)
    static constexpr size_t KBYTES = al(size_t(TILE) * sizeof(KT) + 16);
    static constexpr size_t STAGE = al(KBYTES + (HASV ? size_t(TILE) * 4 + 16 : 0));
    static constexpr size_t o_stage = 0;
    // per group: warp rows, mask tables, per-bucket words (tcnt, bstart,
    // gpos), run offsets, block list, counters and scan scratch
    static constexpr size_t HIST_BYTES = al(size_t(NW) * HROW * 2);
    static constexpr size_t TAB_BYTES = PTAB ? al(size_t(NW) * 2 * SIGMA * 4) : 0;
    static constexpr size_t BK_BYTES = al(size_t(3) * SIGMA * 4);
    // touched blocks per tile: at most TILE/b + 2 per bucket with elements
    static constexpr int LIST = MAXM + 2 * (SIGMA < TILE ? SIGMA : TILE) + 2;
    // Radsort with sigma <= 256: per bucket a 16-byte run descriptor (offset,
    // end of the run's first block, that block's base address) and the list
    // slot of its first block; otherwise 8 bytes (offset, list slot)
    static constexpr bool QB16 = !OOP && SMALL;
    static constexpr size_t QLO_OFF = al(size_t(SIGMA) * (QB16 ? 16 : 8));
    static constexpr size_t QB_BYTES = QLO_OFF + (QB16 ? al(size_t(SIGMA) * 4) : 0);
    static constexpr size_t LK_BYTES = OOP ? 0 : al(size_t(LIST) * (SMALL ? 8 : 4));
    // sigma = 2048: the per-bucket run offsets and the block list live in
    // the warp-row region, which the tile no longer needs once reordered
    static constexpr bool ALIAS = !SMALL && QB_BYTES + LK_BYTES <= HIST_BYTES;
    static constexpr size_t MISC_BYTES = 512;
    static constexpr size_t g_hist = 0;
    static constexpr size_t g_tab = g_hist + HIST_BYTES;
    static constexpr size_t g_bk = g_tab + TAB_BYTES;
    static constexpr size_t g_qb = ALIAS ? g_hist : g_bk + BK_BYTES;
    static constexpr size_t g_lk = g_qb + QB_BYTES;
    static constexpr size_t g_misc = ALIAS ? g_bk + BK_BYTES : g_lk + LK_BYTES;
    static constexpr size_t GROUP = al(g_misc + MISC_BYTES);
    static constexpr size_t o_group = o_stage + STAGES * STAGE;
    // shared by the groups (read only after the start): O (sigma + 1) and,
    // with SMALL, Radsort's tables ns0, ns1, sh
    static constexpr int NTAB = (!OOP && SMALL) ? 4 : 1;
    static constexpr size_t o_tabs = o_group + NG * GROUP;
    static constexpr size_t o_meta = o_tabs + al((size_t(NTAB) * SIGMA + 4) * 4);
    static constexpr size_t o_bar = o_meta + al(STAGES * 16);
    static constexpr size_t SMEM = o_bar + al(2 * STAGES * 8);
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

template <typename KT> struct LbArgs {
    const KT *ik;           // out of place: source
    const uint32_t *iv;
    KT *ok;                 // out of place: destination
    uint32_t *ov;
    KT *Ak;                 // Radsort: block storage (A's blocks after nT scratch blocks)
    uint32_t *Av;
    KT *Tk;
    uint32_t *Tv;
    const uint32_t *pi;     // Radsort: current block map (= the free list)
    uint32_t *pin;          // Radsort: next block map
    const uint32_t *tab;    // O[sigma+1] (+ Radsort: ns0, ns1, sh)
    unsigned long long *ring; // R x sigma look-back words (tags below tagbase)
    uint32_t *done;         // R done tags
    uint32_t *ticket;       // zeroed
    uint32_t rmask;         // R - 1 (R a power of two)
    uint32_t tagbase;       // tag of tile t: tagbase + t (grows with the round)
    const uint32_t *state;  // Radsort: ST_NS, ST_SKIP
    uint32_t n, ntiles, H, nT, npi, lb, shift;
};

// Exclusive prefix of bucket c before tile t: sum of the counts of the tiles
// back to the nearest inclusive prefix, LBW words in flight per step.
template <int SIGMA>
__device__ __forceinline__ uint32_t look_back(const unsigned long long *ring, uint32_t rmask,
                                              uint32_t tagbase, uint32_t t, int c)
{
    constexpr int LBW = 8;
    uint32_t excl = 0;
    int x = static_cast<int>(t) - 1;
    unsigned spins = 0;
    while (x >= 0) {
        unsigned long long v[LBW];
#pragma unroll
        for (int k = 0; k < LBW; ++k)
            v[k] = x - k >= 0 ? ld_volatile64(ring + size_t((x - k) & rmask) * SIGMA + c)
                              : lbw(0xFFFFFFFFu, LB_INCL);
        int k = 0;
        for (; k < LBW; ++k) {
            const int y = x - k;
            const uint32_t want = y >= 0 ? tagbase + uint32_t(y) : 0xFFFFFFFFu;
            const uint32_t tag = static_cast<uint32_t>(v[k] >> 32), s = static_cast<uint32_t>(v[k]);
            if (tag != want) {
                if (tag > want) {
                    // the slot was reused, so tile y + 1 has finished and is
                    // inclusive by now: start over from tile t - 1
                    excl = 0;
                    x = static_cast<int>(t) - 1 + k; // x - k below = t - 1
                }
                break; // tile y has not published yet (or restart)
            }
            if (s & LB_INCL)
                return excl + (s & ~LB_INCL);
            excl += s;
        }
        x -= k;
        if (k < LBW) {
            if (++spins > SPIN_LIMIT || ((spins & 1023u) == 0 && wait_failed())) {
                set_status(ST_TIMEOUT);
                return excl;
            }
            __nanosleep(32);
        }
    }
    return excl;
}

__device__ __forceinline__ uint32_t wait_pi(const uint32_t *p)
{
    for (unsigned it = 0; it < SPIN_LIMIT; ++it) {
        const uint32_t v = ld_volatile(p);
        if (v != PI_NONE)
            return v;
        if ((it & 1023u) == 1023u && wait_failed())
            return PI_NONE;
        __nanosleep(64);
    }
    set_status(ST_TIMEOUT);
    return PI_NONE;
}

template <typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES, bool OOP>
__global__ void __launch_bounds__(LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>::THREADS,
                                   LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>::MINB)
    k_lb_round(LbArgs<KT> a)
{
    using C = LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>;
    constexpr int SIGMA = C::SIGMA, NT = C::NT;
    extern __shared__ __align__(128) unsigned char sm[];
    if (!OOP && a.state[ST_SKIP])
        return; // the digit is constant: the round is the identity
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // this warp's consumer group (the producer warp maps past the last one)
    const int grp = warp / NW < NG ? warp / NW : 0;
    unsigned char *gb = sm + C::o_group + size_t(grp) * C::GROUP;
    uint16_t *hist = reinterpret_cast<uint16_t *>(gb + C::g_hist);
    unsigned *ptab = reinterpret_cast<unsigned *>(gb + C::g_tab);
    uint32_t *bk = reinterpret_cast<uint32_t *>(gb + C::g_bk);
    uint32_t *tcnt = bk, *bstart = bk + SIGMA, *gpos = bk + 2 * SIGMA;
    uint32_t *sO = reinterpret_cast<uint32_t *>(sm + C::o_tabs); // sigma + 1 entries
    uint32_t *stab = sO + SIGMA + 1;
    // bucket tables: shared memory (SMALL) or global
    const uint32_t *ns0 = C::SMALL ? stab : a.tab + SIGMA + 1;
    const uint32_t *ns1 = ns0 + SIGMA, *shr = ns1 + SIGMA;
    uint2 *qb = reinterpret_cast<uint2 *>(gb + C::g_qb);
    uint4 *qb16 = reinterpret_cast<uint4 *>(gb + C::g_qb);
    uint32_t *qlo = reinterpret_cast<uint32_t *>(gb + C::g_qb + C::QLO_OFF);
    // list entries: the key block pointer tagged with its array (SMALL), or
    // the block index
    unsigned long long *listk = reinterpret_cast<unsigned long long *>(gb + C::g_lk);
    uint32_t *listb = reinterpret_cast<uint32_t *>(gb + C::g_lk);
    // byte distance from a key block to its value block, in T and in A
    const long long dvT = reinterpret_cast<const char *>(a.Tv) - reinterpret_cast<const char *>(a.Tk);
    const long long dvA = reinterpret_cast<const char *>(a.Av) - reinterpret_cast<const char *>(a.Ak);
    uint32_t *meta = reinterpret_cast<uint32_t *>(sm + C::o_meta);
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + C::o_bar);
    uint64_t *empty = full + STAGES;
    // the group's [1..3] a tile's list slots, blocks taken and blocks taken
    // by earlier tiles, [8..] scan scratch
    uint32_t *misc = reinterpret_cast<uint32_t *>(gb + C::g_misc);

    const uint32_t b = 1u << a.lb;
    const uint32_t mask = SIGMA - 1;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        fence_mbar_init();
    }
    for (int c = tid; c <= SIGMA; c += C::THREADS)
        sO[c] = a.tab[c];
    if constexpr (!OOP && C::SMALL) {
        for (int c = tid; c < 3 * SIGMA; c += C::THREADS)
            stab[c] = a.tab[SIGMA + 1 + c];
    }
    if constexpr (C::PTAB)
        for (int g = 0; g < NG; ++g) {
            unsigned *pt = reinterpret_cast<unsigned *>(sm + C::o_group + size_t(g) * C::GROUP + C::g_tab);
            for (int i = tid; i < 2 * NW * SIGMA; i += C::THREADS)
                pt[i] = 0u;
        }
    __syncthreads();

    auto kaddr = [&](uint32_t blk) -> KT * {
        return blk < a.nT ? a.Tk + (size_t(blk) << a.lb) : a.Ak + (size_t(blk - a.nT) << a.lb);
    };
    auto vaddr = [&](uint32_t blk) -> uint32_t * {
        return blk < a.nT ? a.Tv + (size_t(blk) << a.lb) : a.Av + (size_t(blk - a.nT) << a.lb);
    };

    if (warp == NG * NW) {
        // ================================================================ producer
        uint32_t k = 0;
        uint32_t wm = 0; // tiles below wm have finished their look-back
        for (;; ++k) {
            const int s = k % STAGES;
            const uint32_t par = ((k / STAGES) & 1u) ^ 1u;
            if (!mbar_wait(&empty[s], par))
                break;
            uint32_t t = 0;
            if (lane == 0)
                t = atomicAdd(a.ticket, 1u);
            t = __shfl_sync(0xffffffffu, t, 0);
            uint32_t *mt = meta + s * 4;
            // the ring slot of tile t held tile t - R: wait until every tile
            // up to t - R + 1 has finished its look-back
            if (t < a.ntiles && t > a.rmask) {
                const uint32_t need = t - a.rmask + 1; // tiles below `need` must be done
                unsigned spins = 0;
                while (wm < need) {
                    const uint32_t z = wm + lane;
                    const bool ok = z >= need || ld_volatile(a.done + (z & a.rmask)) >= a.tagbase + z;
                    const unsigned bal = __ballot_sync(0xffffffffu, ok);
                    const uint32_t adv = bal == 0xffffffffu ? 32u : uint32_t(__ffs(~bal) - 1);
                    wm = min(need, wm + adv);
                    if (wm < need) {
                        if (++spins > SPIN_LIMIT || ((spins & 1023u) == 0 && wait_failed())) {
                            set_status(ST_TIMEOUT);
                            break;
                        }
                        __nanosleep(64);
                    }
                }
            }
            if (t >= a.ntiles) {
                // every group stops at its next tile: NG end marks, each in
                // the next stage in fill order
                if (lane == 0) {
                    mt[0] = TILE_END;
                    mbar_arrive(&full[s]);
                }
                ++k;
                bool ok = true;
                for (int g = 1; g < NG && ok; ++g, ++k) {
                    const int s2 = k % STAGES;
                    ok = mbar_wait(&empty[s2], ((k / STAGES) & 1u) ^ 1u);
                    if (ok && lane == 0) {
                        meta[s2 * 4] = TILE_END;
                        mbar_arrive(&full[s2]);
                    }
                }
                break;
            }
            unsigned char *st = sm + C::o_stage + size_t(s) * C::STAGE;
            KT *stk = reinterpret_cast<KT *>(st);
            uint32_t *stv = reinterpret_cast<uint32_t *>(st + C::KBYTES);
            const uint32_t e0 = t * uint32_t(TILE);
            const uint32_t cnt = min(uint32_t(TILE), a.n - e0);
            uint32_t leadk = 0, leadv = 0;
            if constexpr (OOP) {
                // the 16-byte-aligned middle by bulk copies, the ragged ends
                // (under 16 bytes each) by plain loads
                const uintptr_t ka = reinterpret_cast<uintptr_t>(a.ik + e0);
                const uintptr_t kz = ka + uintptr_t(cnt) * sizeof(KT);
                const uintptr_t ka16 = (ka + 15) & ~uintptr_t(15), kz16 = kz & ~uintptr_t(15);
                leadk = static_cast<uint32_t>((ka & 15) / sizeof(KT));
                const bool kmid = ka16 < kz16;
                const uint32_t khead = kmid ? static_cast<uint32_t>((ka16 - ka) / sizeof(KT)) : cnt;
                const uint32_t ktail = kmid ? static_cast<uint32_t>((kz16 - ka) / sizeof(KT)) : cnt;
                uint32_t bytes = kmid ? static_cast<uint32_t>(kz16 - ka16) : 0u;
                uintptr_t va = 0, va16 = 0, vz16 = 0;
                uint32_t vhead = 0, vtail = 0;
                bool vmid = false;
                if (HASV) {
                    va = reinterpret_cast<uintptr_t>(a.iv + e0);
                    const uintptr_t vz = va + uintptr_t(cnt) * 4;
                    va16 = (va + 15) & ~uintptr_t(15);
                    vz16 = vz & ~uintptr_t(15);
                    leadv = static_cast<uint32_t>((va & 15) / 4);
                    vmid = va16 < vz16;
                    vhead = vmid ? static_cast<uint32_t>((va16 - va) / 4) : cnt;
                    vtail = vmid ? static_cast<uint32_t>((vz16 - va) / 4) : cnt;
                    bytes += vmid ? static_cast<uint32_t>(vz16 - va16) : 0u;
                }
                if (lane == 0 && bytes)
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])),
                                 "r"(bytes)
                                 : "memory");
                __syncwarp();
                if (lane == 0 && kmid)
                    bulk_g2s(stk + leadk + khead, reinterpret_cast<const void *>(ka16),
                             static_cast<uint32_t>(kz16 - ka16), &full[s]);
                if (HASV && lane == 1 && vmid)
                    bulk_g2s(stv + leadv + vhead, reinterpret_cast<const void *>(va16),
                             static_cast<uint32_t>(vz16 - va16), &full[s]);
                for (uint32_t e = lane; e < khead; e += 32)
                    stk[leadk + e] = a.ik[e0 + e];
                for (uint32_t e = ktail + lane; e < cnt; e += 32)
                    stk[leadk + e] = a.ik[e0 + e];
                if (HASV) {
                    for (uint32_t e = lane; e < vhead; e += 32)
                        stv[leadv + e] = a.iv[e0 + e];
                    for (uint32_t e = vtail + lane; e < cnt; e += 32)
                        stv[leadv + e] = a.iv[e0 + e];
                }
            } else {
                // blocks t*M .. of the logical data: block i at stage offset i*b
                const uint32_t nb = (cnt + b - 1) >> a.lb;
                const uint32_t i0 = a.H + t * (uint32_t(TILE) >> a.lb);
                uint32_t tot = 0;
                // (a block index outside the block store is reported and skipped)
                for (uint32_t base = 0; base < nb; base += 32) {
                    const uint32_t i = base + lane;
                    uint32_t bytes = 0;
                    if (i < nb && a.pi[i0 + i] < a.npi) {
                        const uint32_t len = min(b, cnt - i * b);
                        bytes = ((len * uint32_t(sizeof(KT)) + 15u) & ~15u) + (HASV ? ((len * 4u + 15u) & ~15u) : 0u);
                    }
                    tot += warp_sum(bytes);
                }
                if (lane == 0 && tot)
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])),
                                 "r"(tot)
                                 : "memory");
                __syncwarp();
                for (uint32_t i = lane; i < nb; i += 32) {
                    const uint32_t len = min(b, cnt - i * b);
                    const uint32_t phys = a.pi[i0 + i];
                    if (phys >= a.npi) {
                        set_status(ST_INTERNAL);
                        continue;
                    }
                    bulk_g2s(stk + size_t(i) * b, kaddr(phys), (len * uint32_t(sizeof(KT)) + 15u) & ~15u, &full[s]);
                    if (HASV)
                        bulk_g2s(stv + size_t(i) * b, vaddr(phys), (len * 4u + 15u) & ~15u, &full[s]);
                }
            }
            __syncwarp();
            if (lane == 0) {
                mt[0] = t;
                mt[1] = cnt;
                mt[2] = leadk;
                mt[3] = leadv;
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&full[s]); // release: the plain stores above are visible
        }
        // drain: every issued copy lands before this CTA exits (only the last
        // STAGES fills can still be in flight, and no fill follows them, so
        // the phase each of them completes stays readable)
        if (lane == 0) {
            const uint32_t t0 = k > STAGES ? k - STAGES : 0;
            for (uint32_t t = t0; t < k; ++t)
                mbar_wait(&full[t % STAGES], (t / STAGES) & 1u);
        }
        return;
    }

    // ==================================================================== consumers
    // thread and warp index within the group
    const int ctid = tid - grp * NT, cw = warp - grp * NW;
    uint32_t *tmp = misc + 8;
    auto bar = [grp] { named_bar(1 + grp, NT); };
    const uint32_t nP = OOP ? 0u : a.state[ST_NS]; // free-list entries taken before the round
    const uint32_t M = uint32_t(TILE) >> a.lb;

    for (uint32_t k = grp;; k += NG) { // fills grp, grp + NG, ...
        const int s = k % STAGES;
        if (!mbar_wait(&full[s], (k / STAGES) & 1u))
            break;
        const uint32_t *mt = meta + s * 4;
        const uint32_t t = mt[0];
        if (t == TILE_END)
            break;
        const uint32_t cnt = mt[1], leadk = mt[2], leadv = mt[3];
        unsigned char *st = sm + C::o_stage + size_t(s) * C::STAGE;
        KT *tk = reinterpret_cast<KT *>(st);
        uint32_t *tv = reinterpret_cast<uint32_t *>(st + C::KBYTES);
        uint2 *tp = reinterpret_cast<uint2 *>(st); // (key, value) pairs after the reorder

        // ---- 1. this thread's elements into registers; stable rank within the warp
        KT key[C::ITEMS];
        uint32_t val[C::ITEMS];
        uint32_t digs[C::LEAN ? 1 : C::ITEMS];
        uint32_t rks[C::LEAN ? (C::ITEMS + 1) / 2 : C::ITEMS];
        // digit of item it (SIGMA past the tile's end) and its rank in the warp
        auto dig = [&](int it) -> uint32_t {
            if constexpr (C::LEAN)
                return cw * C::R + it * 32 + lane < cnt ? digit_of(key[it], a.shift, mask)
                                                          : uint32_t(SIGMA);
            else
                return digs[it];
        };
        auto set_rk = [&](int it, uint32_t v) {
            if constexpr (C::LEAN)
                rks[it >> 1] = (it & 1) ? ((rks[it >> 1] & 0xFFFFu) | (v << 16)) : ((rks[it >> 1] & 0xFFFF0000u) | v);
            else
                rks[it] = v;
        };
        auto get_rk = [&](int it) -> uint32_t {
            if constexpr (C::LEAN)
                return (it & 1) ? (rks[it >> 1] >> 16) : (rks[it >> 1] & 0xFFFFu);
            else
                return rks[it];
        };
#pragma unroll
        for (int it = 0; it < C::ITEMS; ++it) {
            const uint32_t e = cw * C::R + it * 32 + lane;
            key[it] = tk[leadk + e];
            if (HASV)
                val[it] = tv[leadv + e];
            if constexpr (!C::LEAN)
                digs[it] = e < cnt ? digit_of(key[it], a.shift, mask) : uint32_t(SIGMA);
        }
        const unsigned lt = lanemask_lt();
        uint16_t *hw = hist + cw * C::HROW;
        for (int c = lane; c < SIGMA; c += 32)
            hw[c] = 0;
        if constexpr (C::PTAB) {
            // row by row: lanes with the same digit OR their bit into the
            // digit's mask word, read back the mask and the warp's running
            // count; the lowest of those lanes advances the count and clears
            // the word.  Rows alternate between two mask tables, so the
            // clearing of one row and the ORs of the next never meet (a
            // table is all zero again two rows later)
            unsigned *pt0 = ptab + cw * 2 * SIGMA;
            __syncwarp();
#pragma unroll
            for (int it = 0; it < C::ITEMS; ++it) {
                unsigned *pt = pt0 + (it & 1) * SIGMA;
                const uint32_t d = dig(it);
                const bool v = d < SIGMA;
                if (v)
                    atomicOr(&pt[d], 1u << lane);
                __syncwarp();
                const unsigned pm = v ? pt[d] : 0u;
                const uint32_t base = v ? hw[d] : 0u;
                set_rk(it, base + __popc(pm & lt));
                __syncwarp();
                if (v && (__ffs(pm) - 1) == lane) {
                    hw[d] = static_cast<uint16_t>(base + __popc(pm));
                    pt[d] = 0u;
                }
            }
            __syncwarp();
        } else {
            // a few rows at a time: their peer masks (independent ballots),
            // then row by row the lowest lane of each digit group reads and
            // advances the running count and passes the old count to its
            // group with a shuffle
            constexpr int CH = C::ITEMS % 4 == 0 ? 4 : (C::ITEMS % 2 == 0 ? 2 : 1);
            __syncwarp();
#pragma unroll
            for (int i0 = 0; i0 < C::ITEMS; i0 += CH) {
                unsigned peers[CH];
#pragma unroll
                for (int q = 0; q < CH; ++q)
                    peers[q] = peer_mask<DB>(dig(i0 + q), dig(i0 + q) < SIGMA);
#pragma unroll
                for (int q = 0; q < CH; ++q) {
                    const uint32_t d = dig(i0 + q);
                    const unsigned pm = peers[q];
                    const int ld = pm ? __ffs(pm) - 1 : lane;
                    uint32_t base = 0;
                    if (d < SIGMA && ld == lane) {
                        base = hw[d];
                        hw[d] = static_cast<uint16_t>(base + __popc(pm));
                    }
                    base = __shfl_sync(0xffffffffu, base, ld);
                    set_rk(i0 + q, base + __popc(pm & lt));
                    __syncwarp();
                }
            }
        }
        bar();

        if (ctid == 0) // this tile's slot counters (step 4)
            misc[1] = misc[2] = misc[3] = 0u;

        // ---- 2. tile counts per bucket, published for the look-back, and
        // their exclusive scan (bucket starts in the reordered tile)
        auto cnt_at = [&](int w, int c) -> uint32_t { return hist[w * C::HROW + c]; };
        constexpr int RPT = NW / C::TPB;
        for (int i = ctid; i < SIGMA * C::TPB; i += NT) {
            const int c = i / C::TPB, part = i % C::TPB;
            uint32_t sum = 0;
#pragma unroll
            for (int r = 0; r < RPT; ++r)
                sum += cnt_at(part * RPT + r, c);
#pragma unroll
            for (int o = C::TPB / 2; o > 0; o >>= 1)
                sum += __shfl_xor_sync(0xffffffffu, sum, o, C::TPB);
            if (part == C::TPB - 1) {
                tcnt[c] = sum;
                bstart[c] = sum;
                st_volatile64(a.ring + size_t(t & a.rmask) * SIGMA + c,
                              lbw(a.tagbase + t, t == 0 ? (LB_INCL | sum) : sum));
            }
        }
        bar();
        block_scan<SIGMA, NT>(bstart, tmp, bar, ctid);
        // each warp's start per bucket in the reordered tile: bucket start +
        // the counts of the warps before it (the ranks are warp-relative)
        for (int i = ctid; i < SIGMA * C::TPB; i += NT) {
            const int c = i / C::TPB, part = i % C::TPB;
            uint32_t h[RPT], sum = 0;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                h[r] = cnt_at(part * RPT + r, c);
                sum += h[r];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < C::TPB; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o, C::TPB);
                if (part >= o)
                    incl += x;
            }
            uint32_t run = bstart[c] + incl - sum;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                hist[(part * RPT + r) * C::HROW + c] = static_cast<uint16_t>(run);
                run += h[r];
            }
        }
        bar();

        // ---- 3. reorder the tile by digit, in place in its stage buffer
        // (every element is in registers since the barriers above)
#pragma unroll
        for (int it = 0; it < C::ITEMS; ++it) {
            const uint32_t d = dig(it);
            if (d < SIGMA) {
                const uint32_t pos = cnt_at(cw, d) + get_rk(it);
                if (pos >= uint32_t(TILE)) { // only a broken scan gets here
                    set_status(ST_INTERNAL);
                    continue;
                }
                if constexpr (C::PAIR) {
                    tp[pos] = make_uint2(static_cast<uint32_t>(key[it]), val[it]);
                } else {
                    tk[pos] = key[it];
                    if (HASV)
                        tv[pos] = val[it];
                }
            }
        }

        if constexpr (C::ALIAS)
            bar(); // every warp has read its row before qb and the list overwrite it

        // ---- 4. global offset of each bucket's run (look-back); Radsort:
        // blocks touched, blocks taken here and by earlier tiles, list slots
        // and free-list offsets (shared counters: the order of the blocks a
        // tile takes does not matter, only that each index is used once), and
        // a prefetch of the map entry of the first block touched
        constexpr int PFN = (SIGMA + NT - 1) / NT;
        uint32_t pf[PFN], l0s[PFN], kos[PFN];
#pragma unroll
        for (int q = 0; q < PFN; ++q) {
            const int c = ctid + q * NT;
            pf[q] = PI_NONE;
            l0s[q] = kos[q] = 0;
            if (c >= SIGMA) // whole warps: SIGMA and NT are multiples of 32
                continue;
            const uint32_t cn = tcnt[c];
            uint32_t excl = 0;
            if (t > 0) {
                excl = look_back<SIGMA>(a.ring, a.rmask, a.tagbase, t, c);
                st_volatile64(a.ring + size_t(t & a.rmask) * SIGMA + c,
                              lbw(a.tagbase + t, LB_INCL | (excl + cn)));
            }
            const uint32_t g = sO[c] + excl;
            if constexpr (OOP) {
                qb[c] = make_uint2(g - bstart[c], 0u);
            } else {
                gpos[c] = g;
                // the run lies inside the bucket's output range unless the
                // look-back words were corrupted: then it is reported and
                // its blocks are left alone
                const bool bad = g + cn > sO[c + 1] || g + cn < g;
                if (bad)
                    set_status(ST_INTERNAL);
                const uint32_t cn = bad ? 0u : tcnt[c];
                const uint32_t e = g + cn;
                const uint32_t touched = cn ? ((e - 1) >> a.lb) - (g >> a.lb) + 1 : 0u;
                const uint32_t cs = (g + b - 1) >> a.lb, ce = (e + b - 1) >> a.lb;
                const uint32_t n0 = ns0[c], n1 = ns1[c];
                // block j in [n0 + L, n1) is taken by the writer of the first
                // position of block j - L: by earlier tiles for j - L < cs,
                // here for cs <= j - L < ce
                const uint32_t mb = min(cs + GRID_AHEAD, n1), e0 = n0 + GRID_AHEAD;
                const uint32_t before = mb > e0 ? mb - e0 : 0u;
                const uint32_t f0 = max(cs, n0) + GRID_AHEAD, f1 = min(ce + GRID_AHEAD, n1);
                const uint32_t kk = f1 > f0 ? f1 - f0 : 0u;
                // warp-aggregated slots: list entries, blocks taken, and the
                // count of blocks taken by earlier tiles
                const uint32_t it_ = warp_incl_scan(touched), ik = warp_incl_scan(kk);
                const uint32_t sb = warp_sum(before);
                uint32_t bt = 0, bk2 = 0;
                if (lane == 31) {
                    bt = atomicAdd(&misc[1], it_);
                    bk2 = atomicAdd(&misc[2], ik);
                    atomicAdd(&misc[3], sb);
                }
                l0s[q] = __shfl_sync(0xffffffffu, bt, 31) + it_ - touched;
                kos[q] = __shfl_sync(0xffffffffu, bk2, 31) + ik - kk;
                // the first block touched was taken before this tile unless
                // this tile takes it (then its map entry is not read)
                if (cn && (g >> a.lb) < f0)
                    pf[q] = ld_volatile(a.pin + a.H + (g >> a.lb));
            }
        }
        bar();
        if (ctid == 0) // this tile reads no more look-back words
            st_volatile(a.done + (t & a.rmask), a.tagbase + t);

        uint32_t TT = 0; // list entries of this tile
        if constexpr (!OOP) {
            // ---- 5. the physical block of every block this tile touches, and
            // the blocks it takes beyond those
            TT = misc[1];
            const uint32_t fbase = nP + misc[3]; // free-list index of this tile's first new block
            // free-list entries consumed so far (Lemma 1), within the list
            const uint32_t fcap = min(a.H + (t + 1) * M, a.npi);
#pragma unroll
            for (int q = 0; q < PFN; ++q) {
                const int c = ctid + q * NT;
                if (c >= SIGMA)
                    continue;
                const uint32_t g = gpos[c], cn = tcnt[c];
                const uint32_t l0 = l0s[q], j0 = g >> a.lb;
                if constexpr (C::QB16) {
                    // the run's first block is filled in below; an element
                    // past it reads its block from the list
                    qb16[c] = make_uint4(g - bstart[c], 0u, 0u, 0u);
                    qlo[c] = l0 - j0;
                } else {
                    qb[c] = make_uint2(g - bstart[c], l0 - j0);
                }
                if (!cn || g + cn > sO[c + 1] || g + cn < g)
                    continue; // (a corrupted run was reported in step 4)
                const uint32_t touched = ((g + cn - 1) >> a.lb) - j0 + 1;
                const uint32_t n0 = ns0[c], n1 = ns1[c];
                const uint32_t cs = (g + b - 1) >> a.lb, ce = (g + cn + b - 1) >> a.lb;
                const uint32_t first = max(cs, n0) + GRID_AHEAD;
                const uint32_t last = min(ce + GRID_AHEAD, n1); // blocks first .. last-1 taken here
                const uint32_t sh = shr[c], fsh = sh & 0xFFFFu, lsh = sh >> 16;
                const uint32_t jf = sO[c] >> a.lb, jl = (sO[c + 1] - 1) >> a.lb;
                auto take = [&](uint32_t j) -> uint32_t {
                    const uint32_t idx = fbase + kos[q] + (j - first);
                    if (idx >= fcap) {
                        set_status(ST_INTERNAL); // Lemma 1 would be violated
                        return PI_NONE;
                    }
                    const uint32_t ph = __ldg(a.pi + idx);
                    a.pin[a.H + j] = ph;
                    return ph;
                };
                for (uint32_t i = 0; i < touched; ++i) {
                    const uint32_t j = j0 + i;
                    uint32_t phys;
                    if (j >= first && j < last && !(fsh != SH_NONE && j == jf) &&
                        !(lsh != SH_NONE && j == jl)) {
                        phys = take(j); // this tile writes the first position of block j - L
                    } else { // taken before the round or by an earlier tile
                        phys = i == 0 ? pf[q] : PI_NONE;
                        if (phys == PI_NONE)
                            phys = wait_pi(a.pin + a.H + j);
                    }
                    if (phys != PI_NONE && phys >= a.npi) {
                        set_status(ST_INTERNAL);
                        phys = PI_NONE;
                    }
                    if constexpr (C::SMALL) {
                        // one word per entry: the key block pointer, bit 0 set
                        // for a block of A (the value pointer follows from it)
                        const unsigned long long w =
                            phys == PI_NONE ? 0ull
                                            : (reinterpret_cast<unsigned long long>(kaddr(phys)) |
                                               (phys >= a.nT ? 1ull : 0ull));
                        listk[l0 + i] = w;
                        if (i == 0 && w) {
                            // the first block as a base for the run's
                            // positions: key address of position p in it is
                            // base + p elements (bit 1 marks it valid)
                            const unsigned long long base =
                                ((w & ~1ull) - (static_cast<unsigned long long>(j0) << a.lb) * sizeof(KT)) |
                                (w & 1ull) | 2ull;
                            qb16[c] = make_uint4(g - bstart[c], (j0 + 1) << a.lb, static_cast<uint32_t>(base),
                                                 static_cast<uint32_t>(base >> 32));
                        }
                    } else {
                        listb[l0 + i] = phys;
                    }
                }
                for (uint32_t j = max(first, j0 + touched); j < last; ++j) // taken, not touched
                    (void)take(j);
            }
            bar();
        }

        // ---- 7. store every bucket run
        constexpr int SI = (TILE + NT - 1) / NT;
#pragma unroll 4
        for (int kk = 0; kk < SI; ++kk) {
            const uint32_t i = ctid + kk * NT;
            if (i < cnt) {
                KT kv;
                uint32_t vv = 0;
                if constexpr (C::PAIR) {
                    const uint2 pr = tp[i];
                    kv = pr.x;
                    vv = pr.y;
                } else {
                    kv = tk[i];
                    if (HASV)
                        vv = tv[i];
                }
                const uint32_t dg = digit_of(kv, a.shift, mask);
                if constexpr (C::QB16) {
                    // Radsort, sigma <= 256: most runs lie in one block, whose
                    // base address the run descriptor holds; the rest read
                    // their block from the list
                    const uint4 qd = qb16[dg];
                    const uint32_t pos = i + qd.x;
                    unsigned long long w;
                    uint32_t idx;
                    if (pos < qd.y) {
                        w = (static_cast<unsigned long long>(qd.w) << 32) | qd.z;
                        idx = pos;
                    } else {
                        const uint32_t l = (pos >> a.lb) + qlo[dg];
                        w = l < TT ? listk[l] : 0ull;
                        idx = pos & (b - 1);
                    }
                    if (w) {
                        KT *pk = reinterpret_cast<KT *>(w & ~3ull) + idx;
                        *pk = kv;
                        if (HASV) {
                            uint32_t *pv;
                            if constexpr (sizeof(KT) == 4)
                                pv = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(pk) + ((w & 1ull) ? dvA : dvT));
                            else
                                pv = ((w & 1ull) ? a.Av + (pk - a.Ak) : a.Tv + (pk - a.Tk));
                            *pv = vv;
                        }
                    }
                    continue;
                }
                const uint2 qd = qb[dg];
                const uint32_t pos = i + qd.x;
                if constexpr (OOP) {
                    if (pos < a.n) {
                        a.ok[pos] = kv;
                        if (HASV)
                            a.ov[pos] = vv;
                    }
                } else {
                    const uint32_t l = (pos >> a.lb) + qd.y, off = pos & (b - 1);
                    if constexpr (C::SMALL) {
                        const unsigned long long w = l < TT ? listk[l] : 0ull;
                        if (w) {
                            KT *pk = reinterpret_cast<KT *>(w & ~1ull);
                            pk[off] = kv;
                            if (HASV) {
                                uint32_t *pv;
                                if constexpr (sizeof(KT) == 4)
                                    pv = reinterpret_cast<uint32_t *>(reinterpret_cast<char *>(pk) + ((w & 1ull) ? dvA : dvT));
                                else
                                    pv = ((w & 1ull) ? a.Av + (pk - a.Ak) : a.Tv + (pk - a.Tk));
                                pv[off] = vv;
                            }
                        }
                    } else {
                        const uint32_t blk = l < TT ? listb[l] : PI_NONE;
                        if (blk != PI_NONE) {
                            kaddr(blk)[off] = kv;
                            if (HASV)
                                vaddr(blk)[off] = vv;
                        }
                    }
                }
            }
        }
        // the stage was read and rewritten with generic accesses; the
        // producer refills it with bulk copies (async proxy)
        fence_proxy_async_smem();
        bar();
        if (ctid == 0)
            mbar_arrive(&empty[s]); // stage consumed: the producer may refill it
    }
}

// ---------------------------------------------------------------- launch helpers
template <typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES, bool OOP>
static int lb_ctas(size_t ntiles)
{
    using C = LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>;
    static DeviceOnce attr; // per template instance
    if (attr.run([] {
            return cudaFuncSetAttribute(k_lb_round<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
        }) != cudaSuccess)
        return -1;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_lb_round<KT, HASV, DB, TILE, NW, NG, STAGES, OOP>,
                                                  C::THREADS, C::SMEM);
    if (per_sm < 1)
        per_sm = 1;
    size_t grid = size_t(num_sms()) * per_sm;
    if (grid > ntiles)
        grid = ntiles;
    return grid < 1 ? 1 : static_cast<int>(grid);
}

// Calls f.template operator()<KT, HASV, DB, TILE, NW, NG, STAGES>() for the configuration.
template <typename F> static cudaError_t lb_dispatch(int kb, int db, bool hasv, F &&f)
{
    using u64 = unsigned long long;
    // The largest tiles that two stages and the tables leave room for
    // (per-tile costs scale with sigma, not with the tile), each a multiple
    // of 2048 so that blocks of up to 2048 elements fit whole; 11-bit digits
    // keep their run offsets and block list in the warp rows (ALIAS).
    // One group of 16 consumer warps and two stages throughout.  Measured at
    // 2^30 u32 keys + values, 8-bit digits (round kernel): tiles of 10240,
    // 7.29 ms; tiles of 4096, 10.7 ms; two groups of 8 warps on tiles of
    // 4096 with two stages each, 8.21 ms; two groups on 8192 / 6144 with one
    // stage each, 9.34 / 9.93 ms.  Per-tile work over the sigma buckets
    // (column sums, scan, look-back, block lists) costs about 6800 cycles a
    // tile whatever its size, so the largest tile wins even though a second
    // group overlaps some of it.
    if (kb == 4) {
        if (db == 8)
            return hasv ? f.template operator()<uint32_t, true, 8, 10240, 16, 1, 2>()
                        : f.template operator()<uint32_t, false, 8, 16384, 16, 1, 2>();
        return hasv ? f.template operator()<uint32_t, true, 11, 8192, 16, 1, 2>()
                    : f.template operator()<uint32_t, false, 11, 16384, 16, 1, 2>();
    }
    if (db == 8)
        return hasv ? f.template operator()<u64, true, 8, 6144, 16, 1, 2>()
                    : f.template operator()<u64, false, 8, 10240, 16, 1, 2>();
    return hasv ? f.template operator()<u64, true, 11, 4096, 16, 1, 2>()
                : f.template operator()<u64, false, 11, 8192, 16, 1, 2>();
}

// Radsort rounds with a tile shape: 0 or 1, the configuration above; 2 (8-bit
// digits), two groups of 8 warps on smaller tiles with two stages each, which
// the autotuner may pick where the arrays hold few tiles per SM
template <typename F> static cudaError_t lb_dispatch_shape(int kb, int db, bool hasv, int shape, F &&f)
{
    using u64 = unsigned long long;
    if (shape == 2 && db == 8) {
        if (kb == 4)
            return hasv ? f.template operator()<uint32_t, true, 8, 4096, 8, 2, 4>()
                        : f.template operator()<uint32_t, false, 8, 8192, 8, 2, 4>();
        return hasv ? f.template operator()<u64, true, 8, 4096, 8, 2, 2>()
                    : f.template operator()<u64, false, 8, 4096, 8, 2, 4>();
    }
    return lb_dispatch(kb, db, hasv, f);
}

} // namespace

bool lb_shape_differs(int db, int shape) { return shape == 2 && db == 8; }

uint32_t lb_tile(int kb, int db, bool hasv, int shape)
{
    uint32_t r = 0;
    lb_dispatch_shape(kb, db, hasv, shape,
                      [&]<typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES>() {
                          r = TILE;
                          return cudaSuccess;
                      });
    return r;
}

// ---------------------------------------------------------------- look-back ring
// Rows of the look-back ring: a power of two, no more than the tiles' power
// of two up to 512 rows, a quarter of it beyond (the tiles in flight at once,
// at most STAGES per SM, mostly fit; a tile whose slot is still in use waits
// for it), at most 2048 rows (sigma = 256) or 1024 (sigma = 2048): a few MB
// whatever n.
static uint32_t ring_rows(size_t ntiles, uint32_t sigma)
{
    const uint32_t cap = sigma <= 256 ? 2048u : 1024u;
    uint32_t r = 1;
    while (r < ntiles && r < 4 * cap)
        r <<= 1;
    if (r > 512)
        r = r / 4 > 512 ? r / 4 : 512u;
    return r < cap ? r : cap;
}

static size_t ring_bytes(size_t ntiles, uint32_t sigma)
{
    const size_t r = ring_rows(ntiles, sigma);
    return r * sigma * 8 + r * 4;
}

size_t grid_ring_bytes(const Geom &g)
{
    const uint32_t tile = lb_tile(g.kb, g.db, g.hasv, g.shape);
    return ring_bytes((g.n + tile - 1) / tile, g.sigma);
}

// ---------------------------------------------------------------- grid-layout Radsort
cudaError_t launch_grid_setup(const Geom &g, const Bufs &w, uint32_t *pi, cudaStream_t st)
{
    // all digit histograms from the input keys, before any block moves; the
    // look-back ring starts with no tags
    cudaError_t e = cudaMemsetAsync(w.hist, 0, size_t(g.nt) * g.sigma * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(w.status, 0, grid_ring_bytes(g), st);
    if (e != cudaSuccess)
        return e;
    e = launch_digit_hist(w.Ak, static_cast<uint32_t>(g.n), g.kb, g.db, w.hist, st);
    if (e != cudaSuccess)
        return e;
    const uint32_t n = static_cast<uint32_t>(g.n);
    int blocks = static_cast<int>((g.npi + 255) / 256);
    if (blocks > 4096)
        blocks = 4096;
    if (g.kb == 4)
        k_grid_setup<uint32_t><<<blocks, 256, 0, st>>>(static_cast<const uint32_t *>(w.Ak), w.Av,
                                                       static_cast<uint32_t *>(w.Tk), w.Tv, n, g.b,
                                                       g.H, g.nA, g.npi, pi, w.P, w.state);
    else
        k_grid_setup<unsigned long long><<<blocks, 256, 0, st>>>(
            static_cast<const unsigned long long *>(w.Ak), w.Av, static_cast<unsigned long long *>(w.Tk),
            w.Tv, n, g.b, g.H, g.nA, g.npi, pi, w.P, w.state);
    g_launches += 2;
    return cudaGetLastError();
}

cudaError_t launch_grid_prep(const Geom &g, const Bufs &w, const uint32_t *pi, uint32_t *pin,
                             int round, cudaStream_t st)
{
    const uint32_t NB = static_cast<uint32_t>((g.n + g.b - 1) / g.b);
    // the new map's data entries start unset: cleared by the prep kernel
    // itself when there are few of them, else by a memset
    const uint32_t clear = NB <= 65536 ? NB : 0u;
    if (!clear) {
        cudaError_t e = cudaMemsetAsync(pin + g.H, 0xFF, size_t(NB) * 4, st);
        if (e != cudaSuccess)
            return e;
    }
    const uint32_t n = static_cast<uint32_t>(g.n);
    if (g.db == 8)
        k_grid_prep<8><<<1, 1024, 0, st>>>(w.hist + size_t(round) * g.sigma, n, g.lb, g.H, g.nA, g.npi,
                                           pi, pin, w.tab, w.state, clear);
    else
        k_grid_prep<11><<<1, 1024, 0, st>>>(w.hist + size_t(round) * g.sigma, n, g.lb, g.H, g.nA,
                                            g.npi, pi, pin, w.tab, w.state, clear);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_grid_round(const Geom &g, const Bufs &w, const uint32_t *pi, uint32_t *pin,
                              int round, cudaStream_t st)
{
    const uint32_t n = static_cast<uint32_t>(g.n);
    return lb_dispatch_shape(g.kb, g.db, g.hasv, g.shape,
                             [&]<typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES>() {
        using C = LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, false>;
        const size_t ntiles = (g.n + TILE - 1) / TILE;
        const int grid = lb_ctas<KT, HASV, DB, TILE, NW, NG, STAGES, false>(ntiles);
        if (grid < 0)
            return cudaErrorInvalidValue;
        LbArgs<KT> a{};
        a.Ak = static_cast<KT *>(w.Ak);
        a.Av = w.Av;
        a.Tk = static_cast<KT *>(w.Tk);
        a.Tv = w.Tv;
        a.pi = pi;
        a.pin = pin;
        a.tab = w.tab;
        const uint32_t R = ring_rows(ntiles, g.sigma);
        a.ring = reinterpret_cast<unsigned long long *>(w.status);
        a.done = reinterpret_cast<uint32_t *>(a.ring + size_t(R) * g.sigma);
        a.rmask = R - 1;
        a.tagbase = uint32_t(round + 1) << 24;
        a.ticket = w.ctr + round;
        a.state = w.state;
        a.n = n;
        a.ntiles = static_cast<uint32_t>(ntiles);
        a.H = g.H;
        a.nT = g.nT;
        a.npi = g.npi;
        a.lb = g.lb;
        a.shift = static_cast<uint32_t>(round * g.db);
        k_lb_round<KT, HASV, DB, TILE, NW, NG, STAGES, false><<<grid, C::THREADS, C::SMEM, st>>>(a);
        g_launches += 1;
        return cudaGetLastError();
    });
}

// ---------------------------------------------------------------- out-of-place comparator
size_t lsd_oop_scratch_bytes(size_t n, int kb, int db, bool hasv)
{
    const size_t sigma = size_t(1) << db;
    const int nt = (8 * kb + db - 1) / db;
    const uint32_t tile = lb_tile(kb, db, hasv, 0);
    const size_t ntiles = (n + tile - 1) / tile;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    return al(nt * sigma * 4) + al(nt * (sigma + 1) * 4) + al(ring_bytes(ntiles, uint32_t(sigma))) + al(64 * 4);
}

cudaError_t launch_lsd_oop_ws(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                              size_t n, int kb, int db, void *scratch, cudaStream_t st)
{
    if (n >= (size_t(1) << 31))
        return cudaErrorInvalidValue;
    const uint32_t sigma = 1u << db;
    const int nt = (8 * kb + db - 1) / db;
    const size_t total = lsd_oop_scratch_bytes(n, kb, db, vals != nullptr);
    char *scr = static_cast<char *>(scratch);
    const bool own = scr == nullptr;
    cudaError_t e = cudaSuccess;
    if (own)
        e = cudaMallocAsync(reinterpret_cast<void **>(&scr), total, st);
    if (e != cudaSuccess)
        return e;
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    const uint32_t tile = lb_tile(kb, db, vals != nullptr, 0);
    const size_t ntiles = (n + tile - 1) / tile;
    uint32_t *hist = reinterpret_cast<uint32_t *>(scr);
    uint32_t *off = reinterpret_cast<uint32_t *>(scr + al(nt * sigma * 4));
    char *ringp = scr + al(nt * sigma * 4) + al(nt * (sigma + 1) * 4);
    uint32_t *ctr = reinterpret_cast<uint32_t *>(ringp + al(ring_bytes(ntiles, sigma)));
    const uint32_t R = ring_rows(ntiles, sigma);
    e = cudaMemsetAsync(hist, 0, size_t(nt) * sigma * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ctr, 0, 64 * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(ringp, 0, ring_bytes(ntiles, sigma), st);
    const uint32_t nn = static_cast<uint32_t>(n);
    if (e == cudaSuccess)
        e = launch_digit_hist(keys, nn, kb, db, hist, st);
    if (e == cudaSuccess) {
        if (db == 8)
            k_offsets<8><<<nt, 1024, 0, st>>>(hist, off, nn);
        else
            k_offsets<11><<<nt, 1024, 0, st>>>(hist, off, nn);
        g_launches += 1;
    }
    if (e == cudaSuccess)
        e = lb_dispatch(kb, db, vals != nullptr, [&]<typename KT, bool HASV, int DB, int TILE, int NW, int NG, int STAGES>() {
        using C = LbCfg<KT, HASV, DB, TILE, NW, NG, STAGES, true>;
        const int grid = lb_ctas<KT, HASV, DB, TILE, NW, NG, STAGES, true>(ntiles);
        if (grid < 0)
            return cudaErrorInvalidValue;
        KT *src = static_cast<KT *>(keys), *dst = static_cast<KT *>(keys_alt);
        uint32_t *vs = vals, *vd = vals_alt;
        for (int r = 0; r < nt; ++r) {
            LbArgs<KT> a{};
            a.ik = src;
            a.iv = vs;
            a.ok = dst;
            a.ov = vd;
            a.tab = off + size_t(r) * (sigma + 1);
            a.ring = reinterpret_cast<unsigned long long *>(ringp);
            a.done = reinterpret_cast<uint32_t *>(a.ring + size_t(R) * sigma);
            a.rmask = R - 1;
            a.tagbase = uint32_t(r + 1) << 24;
            a.ticket = ctr + r;
            a.n = nn;
            a.ntiles = static_cast<uint32_t>(ntiles);
            a.shift = static_cast<uint32_t>(r * DB);
            k_lb_round<KT, HASV, DB, TILE, NW, NG, STAGES, true><<<grid, C::THREADS, C::SMEM, st>>>(a);
            g_launches += 1;
            std::swap(src, dst);
            std::swap(vs, vd);
        }
        cudaError_t ec = cudaGetLastError();
        if (ec == cudaSuccess && (nt & 1)) { // the result is in the alternate buffers: copy back
            ec = cudaMemcpyAsync(keys, src, n * sizeof(KT), cudaMemcpyDeviceToDevice, st);
            if (ec == cudaSuccess && HASV)
                ec = cudaMemcpyAsync(vals, vs, n * 4, cudaMemcpyDeviceToDevice, st);
        }
        return ec;
    });
    cudaError_t e2 = own ? cudaFreeAsync(scr, st) : cudaSuccess;
    return e != cudaSuccess ? e : e2;
}

cudaError_t launch_lsd_oop(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                           size_t n, int kb, int db, cudaStream_t st)
{
    return launch_lsd_oop_ws(keys, vals, keys_alt, vals_alt, n, kb, db, nullptr, st);
}

} // namespace rs
