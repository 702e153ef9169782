// Batched segmented sort for sm_103a: many independent arrays in one call.
//
// Each segment [off[s], off[s+1]) is sorted stably on its own.  Segments fall
// into three classes by length:
//   * small (<= SEG_SMALL): one CTA holds the whole segment in shared memory
//     and runs n_t stable counting-sort passes there (ping-pong buffers);
//   * medium (<= SEG_MED): one CTA runs an out-of-place LSD sort between the
//     segment and its own scratch region.  This is the paper's suggestion of
//     using the scratch array T as A' of Alg. 1 for arrays smaller than T
//     (Sec. 5, results).  With 8-bit digits and a workspace too small for
//     those regions, one CTA runs Radsort itself on the segment's own blocks
//     of 32 elements plus 2 sigma + 2 scratch blocks of its own (Alg. 4-7 on
//     one processor), a scratch that does not grow with the segments;
//   * large: the full Radsort path (Alg. 2) on the segment alone.
// The small and medium classes are listed on the device, and each is
// processed by one persistent launch that takes segments from an atomic
// work counter.  Nothing reads device memory on the host, so the whole call
// is stream-ordered and can be captured in a CUDA graph.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_seg() { return take_status_word(); }

namespace {

constexpr int SEG_T = 256; // threads per CTA (8 warps)
constexpr int SEG_NW = SEG_T / 32;

// One stable counting-sort pass of a tile in shared memory:
// src[0..cnt) -> dst[0..cnt) by digit (key >> shift) & (SIGMA-1).  On return
// (after a barrier) tcnt[c] holds the tile's count of digit c and bstart[c]
// its exclusive prefix.  Elements beyond cnt are ignored.  ITEMS * 32 * SEG_NW
// >= cnt.  All SEG_T threads call it.
template <typename KT, bool HASV, int DB, int ITEMS> struct TilePass {
    static constexpr int SIGMA = 1 << DB;
    static constexpr int R = ITEMS * 32; // elements per warp
    static constexpr int HROW = SIGMA + 2;
    static constexpr bool PTAB = DB <= 8;
    static constexpr size_t SCRATCH =
        size_t(SEG_NW) * HROW * 2 + (PTAB ? size_t(SEG_NW) * SIGMA * 4 : 0) + size_t(SIGMA) * 8 + 128;

    __device__ static void run(const KT *srck, const uint32_t *srcv, KT *dstk, uint32_t *dstv,
                               uint32_t cnt, uint32_t shift, unsigned char *scratch, uint32_t *tcnt,
                               uint32_t *bstart)
    {
        uint16_t *hist = reinterpret_cast<uint16_t *>(scratch);
        unsigned *ptab = reinterpret_cast<unsigned *>(scratch + size_t(SEG_NW) * HROW * 2);
        const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
        const uint32_t mask = SIGMA - 1;
        uint16_t *hw = hist + warp * HROW;
        for (int c = lane; c < SIGMA; c += 32)
            hw[c] = 0;
        if constexpr (PTAB)
            for (int c = lane; c < SIGMA; c += 32)
                ptab[warp * SIGMA + c] = 0u;
        KT key[ITEMS];
        uint32_t val[ITEMS], dig[ITEMS], rk[ITEMS];
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t e = warp * R + it * 32 + lane;
            const bool v = e < cnt;
            key[it] = v ? srck[e] : KT(0);
            if (HASV)
                val[it] = v ? srcv[e] : 0u;
            dig[it] = v ? digit_of(key[it], shift, mask) : uint32_t(SIGMA);
        }
        const unsigned lt = lanemask_lt();
        __syncwarp();
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t d = dig[it];
            const bool v = d < SIGMA;
            unsigned pm;
            if constexpr (PTAB) {
                unsigned *pt = ptab + warp * SIGMA;
                if (v)
                    atomicOr(&pt[d], 1u << lane);
                __syncwarp();
                pm = v ? pt[d] : 0u;
            } else {
                pm = peer_mask<DB>(d, v);
            }
            const uint32_t base = v ? hw[d] : 0u;
            rk[it] = base + __popc(pm & lt);
            __syncwarp();
            if (v && (__ffs(pm) - 1) == lane) {
                hw[d] = static_cast<uint16_t>(base + __popc(pm));
                if constexpr (PTAB)
                    ptab[warp * SIGMA + d] = 0u;
            }
            __syncwarp();
        }
        __syncthreads();
        for (int c = tid; c < SIGMA; c += SEG_T) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < SEG_NW; ++w) {
                const uint32_t h = hist[w * HROW + c];
                hist[w * HROW + c] = static_cast<uint16_t>(run);
                run += h;
            }
            tcnt[c] = run;
        }
        __syncthreads();
        // exclusive scan of tcnt into bstart (one warp, SIGMA/32 steps)
        if (warp == 0) {
            uint32_t carry = 0;
            for (int c0 = 0; c0 < SIGMA; c0 += 32) {
                const uint32_t v = tcnt[c0 + lane];
                const uint32_t inc = warp_incl_scan(v);
                bstart[c0 + lane] = carry + inc - v;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < ITEMS; ++it) {
            const uint32_t d = dig[it];
            if (d < SIGMA) {
                const uint32_t pos = bstart[d] + hist[warp * HROW + d] + rk[it];
                dstk[pos] = key[it];
                if (HASV)
                    dstv[pos] = val[it];
            }
        }
        __syncthreads();
    }
};

struct SegArgs {
    void *keys;
    uint32_t *vals;
    const unsigned long long *off; // num_segments + 1 (device)
    uint32_t nseg;
    uint32_t *ctr;                 // [0] small count, [1] medium count, [2] small ticket, [3] medium ticket
    uint32_t *small_list, *med_list;
    void *scr_k;                   // medium scratch, med_stride elements per CTA
    uint32_t *scr_v;
    uint32_t med_stride;           // the longest medium segment of the call
    uint32_t med_ip;               // medium segments sorted in place (Radsort per CTA)
    int nt, db;
};

__global__ void k_seg_classify(SegArgs a, uint32_t small_max, uint32_t med_max)
{
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < a.nseg; s += gridDim.x * blockDim.x) {
        const unsigned long long len = a.off[s + 1] - a.off[s];
        if (len <= 1)
            continue;
        if (len <= small_max)
            a.small_list[atomicAdd(&a.ctr[0], 1u)] = s;
        else if (len <= med_max)
            a.med_list[atomicAdd(&a.ctr[1], 1u)] = s;
    }
}

// small segments: whole segment in shared memory
template <typename KT, bool HASV, int DB, int SMALL>
__global__ void __launch_bounds__(SEG_T) k_seg_small(SegArgs a)
{
    using TP = TilePass<KT, HASV, DB, SMALL / (32 * SEG_NW)>;
    constexpr int SIGMA = 1 << DB;
    extern __shared__ __align__(16) unsigned char sm[];
    KT *k0 = reinterpret_cast<KT *>(sm);
    KT *k1 = k0 + SMALL;
    uint32_t *v0 = reinterpret_cast<uint32_t *>(k1 + SMALL);
    uint32_t *v1 = v0 + (HASV ? SMALL : 0);
    uint32_t *tcnt = v1 + (HASV ? SMALL : 0);
    uint32_t *bstart = tcnt + SIGMA;
    unsigned char *scratch = reinterpret_cast<unsigned char *>(bstart + SIGMA);
    __shared__ uint32_t s_t;
    KT *keys = static_cast<KT *>(a.keys);
    const uint32_t count = a.ctr[0];
    for (;;) {
        if (threadIdx.x == 0)
            s_t = atomicAdd(&a.ctr[2], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= count)
            break;
        const uint32_t sgi = a.small_list[t];
        const unsigned long long o = a.off[sgi];
        const uint32_t len = static_cast<uint32_t>(a.off[sgi + 1] - o);
        for (uint32_t i = threadIdx.x; i < len; i += SEG_T) {
            k0[i] = keys[o + i];
            if (HASV)
                v0[i] = a.vals[o + i];
        }
        __syncthreads();
        KT *sk = k0, *dk = k1;
        uint32_t *svp = v0, *dvp = v1;
        for (int r = 0; r < a.nt; ++r) {
            TP::run(sk, svp, dk, dvp, len, uint32_t(r * DB), scratch, tcnt, bstart);
            KT *tk = sk;
            sk = dk;
            dk = tk;
            uint32_t *tv = svp;
            svp = dvp;
            dvp = tv;
        }
        for (uint32_t i = threadIdx.x; i < len; i += SEG_T) {
            keys[o + i] = sk[i];
            if (HASV)
                a.vals[o + i] = svp[i];
        }
        __syncthreads();
    }
}

// element copies global -> shared memory that complete asynchronously (4 or 8
// bytes: the segments start at any element)
template <int BYTES> __device__ __forceinline__ void cp_async_elem(void *smem, const void *gmem)
{
    const uint32_t sa = static_cast<uint32_t>(__cvta_generic_to_shared(smem));
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// medium segments: out-of-place LSD between the segment and this CTA's
// scratch region (Alg. 1 per digit), tile by tile.  Every digit's counts come
// from one read of the segment; the next tile is copied into the second
// buffer while the current one is ranked and stored.
template <typename KT, bool HASV, int DB, int TILE>
__global__ void __launch_bounds__(SEG_T, 2) k_seg_medium(SegArgs a)
{
    using TP = TilePass<KT, HASV, DB, TILE / (32 * SEG_NW)>;
    constexpr int SIGMA = 1 << DB, NTD = (8 * int(sizeof(KT)) + DB - 1) / DB, LIT = TILE / SEG_T;
    extern __shared__ __align__(16) unsigned char sm[];
    KT *tkb = reinterpret_cast<KT *>(sm); // two tile buffers
    uint32_t *tvb = reinterpret_cast<uint32_t *>(tkb + 2 * TILE);
    uint32_t *tcnt = tvb + (HASV ? 2 * TILE : 0);
    uint32_t *bstart = tcnt + SIGMA;
    uint32_t *run = bstart + SIGMA;
    uint32_t *gh = run + SIGMA; // NTD x SIGMA
    unsigned char *scratch = reinterpret_cast<unsigned char *>(gh + NTD * SIGMA);
    __shared__ uint32_t s_t;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    KT *keys = static_cast<KT *>(a.keys);
    KT *sck = static_cast<KT *>(a.scr_k) + size_t(blockIdx.x) * a.med_stride;
    uint32_t *scv = HASV ? a.scr_v + size_t(blockIdx.x) * a.med_stride : nullptr;
    const uint32_t count = a.ctr[1];
    const uint32_t mask = SIGMA - 1;
    for (;;) {
        __syncthreads(); // every thread has read s_t and finished the last segment
        if (tid == 0)
            s_t = atomicAdd(&a.ctr[3], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= count)
            break;
        const uint32_t sgi = a.med_list[t];
        const unsigned long long o = a.off[sgi];
        const unsigned long long len64 = a.off[sgi + 1] - o;
        if (len64 > a.med_stride) { // the host sized the scratch from its offsets
            if (tid == 0)
                set_status(ST_INTERNAL);
            continue;
        }
        const uint32_t len = static_cast<uint32_t>(len64);
        // every digit's counts in one pass: the multiset is the same in every round
        for (int i = tid; i < NTD * SIGMA; i += SEG_T)
            gh[i] = 0;
        __syncthreads();
        for (uint32_t i = tid; i < len; i += SEG_T) {
            const KT k = keys[o + i];
#pragma unroll
            for (int r = 0; r < NTD; ++r)
                if (r < a.nt)
                    atomicAdd(&gh[r * SIGMA + digit_of(k, uint32_t(r * DB), mask)], 1u);
        }
        __syncthreads();
        KT *sk = keys + o, *dk = sck;
        uint32_t *svp = HASV ? a.vals + o : nullptr, *dvp = scv;
        const uint32_t ntile = (len + TILE - 1) / TILE;
        for (int r = 0; r < a.nt; ++r) {
            const uint32_t shift = uint32_t(r * DB);
            if (warp == 0) { // bucket starts: exclusive prefix of the round's counts
                uint32_t carry = 0;
                for (int c0 = 0; c0 < SIGMA; c0 += 32) {
                    const uint32_t v = gh[r * SIGMA + c0 + lane];
                    const uint32_t inc = warp_incl_scan(v);
                    run[c0 + lane] = carry + inc - v;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
            auto issue = [&](uint32_t ti) { // tile ti into buffer ti & 1
                const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), len - t0);
                KT *bk = tkb + (ti & 1) * TILE;
                uint32_t *bv = tvb + (ti & 1) * TILE;
#pragma unroll
                for (int it = 0; it < LIT; ++it) {
                    const uint32_t i = it * SEG_T + tid;
                    if (i < cnt) {
                        cp_async_elem<sizeof(KT)>(bk + i, sk + t0 + i);
                        if (HASV)
                            cp_async_elem<4>(bv + i, svp + t0 + i);
                    }
                }
                cp_async_commit();
            };
            issue(0);
            for (uint32_t ti = 0; ti < ntile; ++ti) {
                const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), len - t0);
                KT *tk = tkb + (ti & 1) * TILE;
                uint32_t *tv = tvb + (ti & 1) * TILE;
                cp_async_wait_all();
                __syncthreads(); // the tile is in place; the other buffer is free
                if (ti + 1 < ntile)
                    issue(ti + 1);
                TP::run(tk, tv, tk, tv, cnt, shift, scratch, tcnt, bstart);
#pragma unroll
                for (int it = 0; it < LIT; ++it) {
                    const uint32_t i = it * SEG_T + tid;
                    if (i >= cnt)
                        continue;
                    const KT kk = tk[i];
                    const uint32_t d = digit_of(kk, shift, mask);
                    const uint32_t dst = run[d] + (i - bstart[d]);
                    if (dst >= len) { // only inconsistent counts get here
                        set_status(ST_INTERNAL);
                        continue;
                    }
                    dk[dst] = kk;
                    if (HASV)
                        dvp[dst] = tv[i];
                }
                __syncthreads();
                for (int c = tid; c < SIGMA; c += SEG_T)
                    run[c] += tcnt[c];
            }
            __syncthreads(); // the round's stores precede the next round's copies
            KT *tkp = sk;
            sk = dk;
            dk = tkp;
            uint32_t *tvp = svp;
            svp = dvp;
            dvp = tvp;
        }
        if (sk != keys + o) { // odd number of passes: the result is in the scratch
            for (uint32_t i = tid; i < len; i += SEG_T) {
                keys[o + i] = sk[i];
                if (HASV)
                    a.vals[o + i] = svp[i];
            }
        }
    }
}

// ---- medium segments sorted in place: Radsort on one CTA ----------------
//
// The segment is a sequence of logical blocks of IP_B elements; pi[q] names
// the physical block that holds logical block q: one of the segment's own
// full blocks (id < nfull) or one of this CTA's scratch blocks (nfull ..
// nfull + IP_S - 1).  Before the first round the map is the identity and the
// segment's partial last block lies in place (IP_TAIL).  A round (Alg. 5 on
// one processor, with the output on the block grid of the grid layout) reads
// the sequence tile by tile (the next tile copied while the current one is
// ranked); a tile's blocks go to the free list once it is in shared memory;
// the tile is ranked stably by the round's digit; every
// output block that the tile is the first to touch takes the next free block;
// then the tile is stored.  After the last round, Finalize (Alg. 7) moves
// logical block j to place j along chains, which start at a place that holds
// no block (a free one, or the segment's tail), and along cycles, which are
// first cut into chains through free scratch blocks.
//
// Free blocks suffice: after a tile the output touches at most (elements
// stored) / IP_B + 2 sigma blocks (each bucket's run adds at most a partial
// block at each end), the unread input holds at most the rest of the
// segment's blocks, and the CTA owns nfull + IP_S blocks, IP_S = 2 sigma + 2.
// A segment no longer than the scratch is sorted out of place between the
// two instead (the paper's switch for arrays up to the size of T, Sec. 5).
constexpr uint32_t IP_LB = 5;
constexpr uint32_t IP_B = 1u << IP_LB;
constexpr uint32_t IP_NB = SEG_MED >> IP_LB; // blocks of the longest medium segment
constexpr uint32_t IP_S = 2 * 256 + 2;       // scratch blocks per CTA (8-bit digits)
constexpr uint32_t IP_FCAP = IP_NB + IP_S;   // free list: every block at most once
constexpr uint16_t IP_NONE = 0xFFFF, IP_CLAIM = 0xFFFE, IP_TAIL = 0xFFFD;
constexpr int IP_K = 16;                     // block moves per warp step in Finalize
constexpr uint32_t IP_CUT = 16;              // a cycle is cut into chains of at most this many moves

template <typename KT, bool HASV, int TILE> struct IpCfg {
    static constexpr int SIGMA = 256;
    static constexpr int NTD = int(sizeof(KT)) * 8 / 8;
    using TP = TilePass<KT, HASV, 8, TILE / (32 * SEG_NW)>;
    // two tile buffers of keys, then two of values: the next tile is copied
    // while the current one is ranked
    static constexpr size_t O_TV = size_t(2) * TILE * sizeof(KT);
    static constexpr size_t O_CNT = O_TV + (HASV ? size_t(2) * TILE * 4 : 0);
    static constexpr size_t O_GH = O_CNT + size_t(3) * SIGMA * 4; // tcnt, bstart, run
    static constexpr size_t O_MAP = O_GH + size_t(NTD) * SIGMA * 4;
    static constexpr size_t O_RING = O_MAP + size_t(2) * IP_NB * 2;
    static constexpr size_t O_SCR = (O_RING + size_t(IP_FCAP) * 2 + 15) / 16 * 16;
    static constexpr size_t SMEM = O_SCR + TP::SCRATCH;
    // Finalize reuses the tile buffer: the free scratch blocks and the cut list
    static_assert(size_t(2) * TILE * sizeof(KT) >= 1600 + IP_NB, "tile buffers hold the Finalize lists");
    static_assert(TP::SCRATCH >= size_t(SEG_NW) * 2 * IP_K * 4, "scratch holds the move lists");
};

template <typename KT, bool HASV, int TILE>
__global__ void __launch_bounds__(SEG_T, 2) k_seg_medium_ip(SegArgs a)
{
    using C = IpCfg<KT, HASV, TILE>;
    constexpr int SIGMA = C::SIGMA, DB = 8, LIT = TILE / SEG_T;
    constexpr uint32_t IP_HELD = 0xFFFFFFFFu, IP_TAILDST = 0xFFFFFFFEu;
    extern __shared__ __align__(16) unsigned char sm[];
    KT *tkb = reinterpret_cast<KT *>(sm);
    uint32_t *tvb = reinterpret_cast<uint32_t *>(sm + C::O_TV);
    uint32_t *tcnt = reinterpret_cast<uint32_t *>(sm + C::O_CNT);
    uint32_t *bstart = tcnt + SIGMA;
    uint32_t *run = bstart + SIGMA;
    uint32_t *gh = reinterpret_cast<uint32_t *>(sm + C::O_GH);
    uint16_t *mapA = reinterpret_cast<uint16_t *>(sm + C::O_MAP);
    uint16_t *mapB = mapA + IP_NB;
    uint16_t *ring = reinterpret_cast<uint16_t *>(sm + C::O_RING);
    unsigned char *scratch = sm + C::O_SCR;
    __shared__ uint32_t s_t, s_fh, s_ft, s_next, s_next2, s_nfree, s_fuse, s_nfl, s_fl2;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    KT *keys = static_cast<KT *>(a.keys);
    KT *Tk = static_cast<KT *>(a.scr_k) + size_t(blockIdx.x) * (IP_S * IP_B);
    uint32_t *Tv = HASV ? a.scr_v + size_t(blockIdx.x) * (IP_S * IP_B) : nullptr;
    const uint32_t count = a.ctr[1];
    for (;;) {
        __syncthreads(); // every thread has read s_t and finished the last segment
        if (tid == 0)
            s_t = atomicAdd(&a.ctr[3], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= count)
            break;
        const uint32_t sgi = a.med_list[t];
        const unsigned long long o = a.off[sgi];
        const unsigned long long len = a.off[sgi + 1] - o;
        if (len > SEG_MED) { // the classifier lists no such segment
            if (tid == 0)
                set_status(ST_INTERNAL);
            continue;
        }
        const uint32_t m = static_cast<uint32_t>(len);
        KT *Ak = keys + o;
        uint32_t *Av = HASV ? a.vals + o : nullptr;
        const uint32_t nfull = m >> IP_LB, part = m & (IP_B - 1), nb = nfull + (part ? 1u : 0u);
        const uint32_t nphys = nfull + IP_S;
        // the block of physical id ph < nphys (the partial block in place is
        // only ever read, in the first round, straight from the segment)
        auto koff = [&](uint32_t ph) -> KT * {
            return ph < nfull ? Ak + (size_t(ph) << IP_LB) : Tk + (size_t(ph - nfull) << IP_LB);
        };
        auto voff = [&](uint32_t ph) -> uint32_t * {
            return ph < nfull ? Av + (size_t(ph) << IP_LB) : Tv + (size_t(ph - nfull) << IP_LB);
        };
        uint16_t *pi = mapA, *pin = mapB;
        // setup (Alg. 4): the segment's blocks in order, the partial one in
        // place; the free list holds the scratch blocks
        for (uint32_t q = tid; q < nb; q += SEG_T)
            pi[q] = q < nfull ? static_cast<uint16_t>(q) : IP_TAIL;
        for (uint32_t k = tid; k < IP_S; k += SEG_T)
            ring[k] = static_cast<uint16_t>(nfull + k);
        for (int i = tid; i < C::NTD * SIGMA; i += SEG_T)
            gh[i] = 0;
        if (tid == 0) {
            s_fh = 0;
            s_ft = IP_S;
        }
        __syncthreads();
        // every digit's counts in one pass: the multiset is the same in every round
        for (uint32_t i = tid; i < m; i += SEG_T) {
            const KT k = Ak[i];
#pragma unroll
            for (int r = 0; r < C::NTD; ++r)
                atomicAdd(&gh[r * SIGMA + digit_of(k, uint32_t(r * DB), SIGMA - 1)], 1u);
        }
        __syncthreads();
        auto starts = [&](int r) { // bucket starts: exclusive prefix of round r's counts (warp 0)
            if (warp == 0) {
                uint32_t carry = 0;
                for (int c0 = 0; c0 < SIGMA; c0 += 32) {
                    const uint32_t v = gh[r * SIGMA + c0 + lane];
                    const uint32_t inc = warp_incl_scan(v);
                    run[c0 + lane] = carry + inc - v;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
        };
        if (m <= IP_S * IP_B) {
            // no longer than the scratch: out of place between the segment
            // and the scratch, which serves as A' of Alg. 1
            KT *sk = Ak, *dk = Tk;
            uint32_t *sv = Av, *dv = Tv;
            const uint32_t ntile = (m + TILE - 1) / TILE;
            for (int r = 0; r < C::NTD; ++r) {
                const uint32_t shift = uint32_t(r * DB);
                starts(r);
                auto issue = [&](uint32_t ti) { // tile ti into buffer ti & 1
                    const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), m - t0);
                    KT *bk = tkb + (ti & 1) * TILE;
                    uint32_t *bv = tvb + (ti & 1) * TILE;
#pragma unroll
                    for (int it = 0; it < LIT; ++it) {
                        const uint32_t i = it * SEG_T + tid;
                        if (i < cnt) {
                            cp_async_elem<sizeof(KT)>(bk + i, sk + t0 + i);
                            if (HASV)
                                cp_async_elem<4>(bv + i, sv + t0 + i);
                        }
                    }
                    cp_async_commit();
                };
                issue(0);
                for (uint32_t ti = 0; ti < ntile; ++ti) {
                    const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), m - t0);
                    KT *tk = tkb + (ti & 1) * TILE;
                    uint32_t *tv = tvb + (ti & 1) * TILE;
                    cp_async_wait_all();
                    __syncthreads(); // the tile is in place; the other buffer is free
                    if (ti + 1 < ntile)
                        issue(ti + 1);
                    C::TP::run(tk, tv, tk, tv, cnt, shift, scratch, tcnt, bstart);
#pragma unroll
                    for (int it = 0; it < LIT; ++it) {
                        const uint32_t i = it * SEG_T + tid;
                        if (i >= cnt)
                            continue;
                        const KT k = tk[i];
                        const uint32_t d = digit_of(k, shift, SIGMA - 1);
                        const uint32_t pos = run[d] + (i - bstart[d]);
                        if (pos >= m) { // only inconsistent counts get here
                            set_status(ST_INTERNAL);
                            continue;
                        }
                        dk[pos] = k;
                        if (HASV)
                            dv[pos] = tv[i];
                    }
                    __syncthreads();
                    for (int c = tid; c < SIGMA; c += SEG_T)
                        run[c] += tcnt[c];
                }
                __syncthreads(); // the round's stores precede the next round's copies
                KT *xk = sk;
                sk = dk;
                dk = xk;
                uint32_t *xv = sv;
                sv = dv;
                dv = xv;
            }
            if (sk != Ak) // an odd number of rounds: the result is in the scratch
                for (uint32_t i = tid; i < m; i += SEG_T) {
                    Ak[i] = sk[i];
                    if (HASV)
                        Av[i] = sv[i];
                }
            continue;
        }
        for (int r = 0; r < C::NTD; ++r) {
            const uint32_t shift = uint32_t(r * DB);
            starts(r);
            for (uint32_t j = tid; j < nb; j += SEG_T)
                pin[j] = IP_NONE;
            // tile ti into buffer ti & 1, read through the block map (the
            // first round's map is the identity: the segment in place); the
            // next tile's blocks are not on the free list yet, so nothing
            // stores into them while they are copied
            auto issue = [&](uint32_t ti) {
                const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), m - t0);
                KT *bk = tkb + (ti & 1) * TILE;
                uint32_t *bv = tvb + (ti & 1) * TILE;
#pragma unroll
                for (int it = 0; it < LIT; ++it) {
                    const uint32_t i = it * SEG_T + tid;
                    if (i < cnt) {
                        const uint32_t e = t0 + i;
                        const KT *srck;
                        const uint32_t *srcv;
                        if (r == 0) {
                            srck = Ak + e;
                            srcv = HASV ? Av + e : nullptr;
                        } else {
                            const uint32_t ph = pi[e >> IP_LB], w = e & (IP_B - 1);
                            if (ph >= nphys) { // a broken map, reported
                                set_status(ST_INTERNAL);
                                bk[i] = KT(0);
                                if (HASV)
                                    bv[i] = 0u;
                                continue;
                            }
                            srck = koff(ph) + w;
                            srcv = HASV ? voff(ph) + w : nullptr;
                        }
                        cp_async_elem<sizeof(KT)>(bk + i, srck);
                        if (HASV)
                            cp_async_elem<4>(bv + i, srcv);
                    }
                }
                cp_async_commit();
            };
            __syncthreads(); // pin cleared, starts written, the last round's stores done
            const uint32_t ntile = (m + TILE - 1) / TILE;
            issue(0);
            for (uint32_t ti = 0; ti < ntile; ++ti) {
                const uint32_t t0 = ti * TILE, cnt = min(uint32_t(TILE), m - t0);
                KT *tk = tkb + (ti & 1) * TILE;
                uint32_t *tv = tvb + (ti & 1) * TILE;
                const uint32_t ft = s_ft;
                cp_async_wait_all();
                __syncthreads(); // the tile is in place; the other buffer is free
                if (ti + 1 < ntile)
                    issue(ti + 1);
                // its blocks are free now (the partial block in place is never
                // reused: it is shorter than a block)
                const uint32_t q0 = t0 >> IP_LB, nq = ((t0 + cnt - 1) >> IP_LB) - q0 + 1;
                const uint32_t npush = nq - (pi[q0 + nq - 1] == IP_TAIL ? 1u : 0u);
                for (uint32_t k = tid; k < npush; k += SEG_T)
                    ring[(ft + k) % IP_FCAP] = pi[q0 + k];
                const uint32_t fend = ft + npush;
                __syncthreads();
                if (tid == 0)
                    s_ft = fend;
                C::TP::run(tk, tv, tk, tv, cnt, shift, scratch, tcnt, bstart);
                // each output block this tile touches first takes a free block
                auto take = [&](uint32_t k) -> uint16_t {
                    if (k >= fend) { // more blocks than the bound allows
                        set_status(ST_INTERNAL);
                        return IP_NONE;
                    }
                    return ring[k % IP_FCAP];
                };
                auto claim = [&](uint32_t j) {
                    return pin[j] == IP_NONE && atomicCAS(&pin[j], IP_NONE, IP_CLAIM) == IP_NONE;
                };
                for (int c = tid; c < SIGMA; c += SEG_T) { // whole warps: SIGMA % SEG_T == 0
                    const uint32_t cn = tcnt[c];
                    uint32_t j0 = 0, j1 = 0, need = 0;
                    bool w0 = false, w1 = false;
                    if (cn) {
                        const uint32_t g = run[c];
                        j0 = g >> IP_LB;
                        j1 = (g + cn - 1) >> IP_LB;
                        if (j1 >= nb) {
                            set_status(ST_INTERNAL);
                        } else {
                            // the run's end blocks may be shared with the
                            // neighbouring buckets; blocks inside it are its own
                            w0 = claim(j0);
                            w1 = j1 != j0 && claim(j1);
                            need = (w0 ? 1u : 0u) + (w1 ? 1u : 0u) + (j1 > j0 + 1 ? j1 - j0 - 1 : 0u);
                        }
                    }
                    // one free-list reservation per warp
                    const uint32_t incl = warp_incl_scan(need), tot = __shfl_sync(0xffffffffu, incl, 31);
                    uint32_t k = 0;
                    if (lane == 31 && tot)
                        k = atomicAdd(&s_fh, tot);
                    k = __shfl_sync(0xffffffffu, k, 31) + incl - need;
                    if (need) {
                        if (w0)
                            pin[j0] = take(k++);
                        for (uint32_t j = j0 + 1; j < j1; ++j)
                            pin[j] = take(k++);
                        if (w1)
                            pin[j1] = take(k++);
                    }
                }
                __syncthreads();
                // stores: a bucket's elements are consecutive in the tile and in the output
#pragma unroll
                for (int it = 0; it < LIT; ++it) {
                    const uint32_t i = it * SEG_T + tid;
                    if (i >= cnt)
                        continue;
                    const KT k = tk[i];
                    const uint32_t d = digit_of(k, shift, SIGMA - 1);
                    const uint32_t pos = run[d] + (i - bstart[d]);
                    const uint32_t ph = (pos >> IP_LB) < nb ? pin[pos >> IP_LB] : IP_NONE;
                    if (ph >= nphys) {
                        set_status(ST_INTERNAL);
                        continue;
                    }
                    koff(ph)[pos & (IP_B - 1)] = k;
                    if (HASV)
                        voff(ph)[pos & (IP_B - 1)] = tv[i];
                }
                __syncthreads();
                for (int c = tid; c < SIGMA; c += SEG_T)
                    run[c] += tcnt[c];
            }
            __syncthreads(); // the round's stores precede the next round's copies
            uint16_t *x = pi;
            pi = pin;
            pin = x;
        }
        // Finalize (Alg. 7): logical block j to place j, the partial one to
        // the segment's tail.  occ[p]: the logical block in place p's block.
        // The tile buffer holds the free scratch blocks, their use flags and
        // the cycles left uncut.
        uint16_t *occ = pin;
        uint16_t *freeT = reinterpret_cast<uint16_t *>(sm); // the tile buffers are free now
        unsigned char *usedT = sm + 1040;
        uint16_t *flist = reinterpret_cast<uint16_t *>(sm + 1600);
        for (uint32_t p = tid; p < nb; p += SEG_T)
            occ[p] = IP_NONE;
        for (uint32_t k = tid; k < IP_S; k += SEG_T)
            usedT[k] = 0;
        if (tid == 0)
            s_next = s_next2 = s_nfree = s_fuse = s_nfl = s_fl2 = 0;
        __syncthreads();
        for (uint32_t j = tid; j < nb; j += SEG_T) {
            const uint32_t ph = pi[j];
            if (ph < nfull)
                occ[ph] = static_cast<uint16_t>(j);
            else if (ph < nphys)
                usedT[ph - nfull] = 1;
        }
        __syncthreads();
        for (uint32_t k = tid; k < IP_S; k += SEG_T)
            if (!usedT[k])
                freeT[atomicAdd(&s_nfree, 1u)] = static_cast<uint16_t>(nfull + k);
        __syncthreads();
        const uint32_t nfree = s_nfree;
        // a warp moves blocks IP_K at a time: every source into registers,
        // then every destination.  mv: this warp's list of (destination,
        // source block); IP_HELD names a cycle's first block, held in hk/hv
        uint32_t *mv = reinterpret_cast<uint32_t *>(scratch) + warp * (2 * IP_K);
        auto step = [&](int n, KT hk, uint32_t hv) {
            __syncwarp();
            KT rk[IP_K];
            uint32_t rv[IP_K];
#pragma unroll
            for (int i = 0; i < IP_K; ++i) {
                rk[i] = hk;
                rv[i] = hv;
                const uint32_t src = i < n ? mv[2 * i + 1] : IP_HELD;
                if (src < nphys) {
                    rk[i] = koff(src)[lane];
                    if (HASV)
                        rv[i] = voff(src)[lane];
                }
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < IP_K; ++i) {
                if (i >= n)
                    continue;
                const uint32_t dst = mv[2 * i], src = mv[2 * i + 1];
                if ((src >= nphys && src != IP_HELD) || (dst >= nphys && dst != IP_TAILDST)) {
                    if (lane == 0)
                        set_status(ST_INTERNAL); // a broken map
                    continue;
                }
                const bool tail = dst == IP_TAILDST;
                const uint32_t lim = tail ? part : IP_B;
                if (uint32_t(lane) < lim) {
                    (tail ? Ak + (size_t(nfull) << IP_LB) : koff(dst))[lane] = rk[i];
                    if (HASV)
                        (tail ? Av + (size_t(nfull) << IP_LB) : voff(dst))[lane] = rv[i];
                }
            }
            __syncwarp();
        };
        // cycles: the least place of each cycle leads it; the leader's warp
        // copies every IP_CUT-th block of the cycle to a free scratch block,
        // which leaves that place empty, so the cycle falls into chains of at
        // most IP_CUT moves.  Without free scratch blocks left, a cycle is
        // moved whole after the chains.
        for (;;) {
            uint32_t b0 = 0;
            if (lane == 0)
                b0 = atomicAdd(&s_next, 32u);
            const uint32_t base = __shfl_sync(0xffffffffu, b0, 0);
            if (base >= nfull)
                break;
            const uint32_t p = base + lane;
            bool lead = false;
            if (p < nfull) {
                uint32_t x = pi[p];
                if (x < nfull && x != p) {
                    for (uint32_t g = 0; g <= nb; ++g) {
                        if (x >= nfull || x < p) // a chain, or not the least place of its cycle
                            break;
                        if (x == p) {
                            lead = true;
                            break;
                        }
                        x = pi[x];
                    }
                }
            }
            unsigned lm = __ballot_sync(0xffffffffu, lead);
            while (lm) {
                const int l = __ffs(lm) - 1;
                lm &= lm - 1;
                const uint32_t d0 = base + l;
                uint32_t L = 1;
                for (uint32_t x = pi[d0]; x != d0 && x < nfull && L <= nb; x = pi[x])
                    ++L;
                const uint32_t ncut = (L + IP_CUT - 1) / IP_CUT;
                uint32_t k = 0;
                if (lane == 0)
                    k = atomicAdd(&s_fuse, ncut);
                k = __shfl_sync(0xffffffffu, k, 0);
                if (k + ncut > nfree) {
                    if (lane == 0)
                        flist[atomicAdd(&s_nfl, 1u)] = static_cast<uint16_t>(d0);
                    continue;
                }
                uint32_t x = d0;
                int n = 0;
                for (uint32_t i = 0; i < L; ++i) {
                    if (i % IP_CUT == 0) {
                        if (lane == 0) {
                            mv[2 * n] = freeT[k];
                            mv[2 * n + 1] = x;
                        }
                        ++k;
                        ++n;
                    }
                    const bool last = i + 1 == L;
                    if (n == IP_K || (last && n)) {
                        step(n, KT(0), 0u);
                        // the cut places hold nothing now; their blocks'
                        // logical owners point at the copies
                        if (lane == 0)
                            for (int q = 0; q < n; ++q) {
                                const uint32_t cx = mv[2 * q + 1];
                                pi[occ[cx]] = static_cast<uint16_t>(mv[2 * q]);
                                occ[cx] = IP_NONE;
                            }
                        __syncwarp();
                        n = 0;
                    }
                    if (!last)
                        x = pi[x];
                }
            }
        }
        __syncthreads();
        // chains: every place that holds no block starts one (a free place,
        // or the tail); each step takes up to IP_K moves, the next chain
        // where one ends.  A move reads a place that the chain's previous
        // move writes only in a later step, or later in the same step.
        {
            uint32_t base = 0, cur = 0, moves = 0;
            unsigned smask = 0;
            auto next_start = [&]() -> bool { // warp-uniform
                while (!smask) {
                    uint32_t b0 = 0;
                    if (lane == 0)
                        b0 = atomicAdd(&s_next2, 32u);
                    base = __shfl_sync(0xffffffffu, b0, 0);
                    if (base >= nb)
                        return false;
                    const uint32_t p = base + lane;
                    smask = __ballot_sync(0xffffffffu, p < nb && (p == nfull || occ[p] == IP_NONE));
                }
                const int l = __ffs(smask) - 1;
                smask &= smask - 1;
                cur = base + l;
                return true;
            };
            bool have = next_start();
            while (have) {
                int n = 0;
                while (have && n < IP_K) {
                    const uint32_t src = pi[cur];
                    if (lane == 0) {
                        mv[2 * n] = cur == nfull ? IP_TAILDST : cur;
                        mv[2 * n + 1] = src;
                    }
                    ++n;
                    if (++moves > nb) { // only a broken map walks this far
                        if (lane == 0)
                            set_status(ST_INTERNAL);
                        have = false;
                    } else if (src >= nfull) { // a scratch block: the chain ends
                        have = next_start();
                    } else {
                        cur = src;
                    }
                }
                step(n, KT(0), 0u);
            }
        }
        __syncthreads();
        // cycles left whole: the first place's block waits in registers
        // until the cycle closes
        const uint32_t nfl = s_nfl;
        for (;;) {
            uint32_t f = 0;
            if (lane == 0)
                f = atomicAdd(&s_fl2, 1u);
            f = __shfl_sync(0xffffffffu, f, 0);
            if (f >= nfl)
                break;
            const uint32_t d0 = flist[f];
            const KT hk = Ak[(size_t(d0) << IP_LB) + lane];
            const uint32_t hv = HASV ? Av[(size_t(d0) << IP_LB) + lane] : 0u;
            uint32_t cur = d0, moves = 0;
            bool end = false;
            while (!end) {
                int n = 0;
                while (!end && n < IP_K) {
                    uint32_t src = pi[cur];
                    if (src == d0 || ++moves > nb || src >= nfull) {
                        if (src != d0 && lane == 0)
                            set_status(ST_INTERNAL); // a cycle runs through no scratch block
                        src = IP_HELD;
                        end = true;
                    }
                    if (lane == 0) {
                        mv[2 * n] = cur;
                        mv[2 * n + 1] = src;
                    }
                    ++n;
                    cur = src;
                }
                step(n, hk, hv);
            }
        }
    }
}

// ---- a long segment whose start is not 16-byte aligned (low-memory plan) --
//
// Its first h < 4 elements (the head) are set aside and sorted, the rest
// (the body, which starts aligned) is sorted by Radsort, and the head is
// merged back.  A head element goes before the body's equal keys (it came
// first), so body element i moves to i + (head keys <= its key) and head
// element k to k + (body keys < its key).  Every body element moves left by
// h at most: a chunk of the body is read whole before it is written, and the
// h elements at its end, whose places the next chunk writes, are read from
// copies taken before the merge.  A head element is written by the chunk
// that reads the element it replaces.
constexpr uint32_t HM_CH = 4096; // body elements per chunk
constexpr size_t HM_HDR = 128;   // head keys at 0, values at 32, places at 64

template <typename KT> __global__ void k_head_save(const KT *k, const uint32_t *v, uint32_t h, unsigned char *buf)
{
    if (threadIdx.x != 0 || blockIdx.x != 0)
        return;
    KT *hk = reinterpret_cast<KT *>(buf);
    uint32_t *hv = reinterpret_cast<uint32_t *>(buf + 32);
    for (uint32_t i = 0; i < h; ++i) { // stable insertion sort of at most 3 elements
        const KT key = k[i];
        const uint32_t val = v ? v[i] : 0u;
        uint32_t j = i;
        for (; j > 0 && hk[j - 1] > key; --j) {
            hk[j] = hk[j - 1];
            hv[j] = hv[j - 1];
        }
        hk[j] = key;
        hv[j] = val;
    }
}

// the head's places (binary search in the sorted body) and the copies of the
// last h elements of every chunk but the last
template <typename KT>
__global__ void k_head_prep(const KT *k, const uint32_t *v, uint32_t h, unsigned long long nbody, unsigned char *buf)
{
    const KT *hk = reinterpret_cast<const KT *>(buf);
    unsigned long long *hpos = reinterpret_cast<unsigned long long *>(buf + 64);
    const unsigned long long nch = (nbody + HM_CH - 1) / HM_CH;
    KT *bk = reinterpret_cast<KT *>(buf + HM_HDR);
    uint32_t *bv = reinterpret_cast<uint32_t *>(buf + HM_HDR + (nch * 3 * sizeof(KT) + 15) / 16 * 16);
    const unsigned long long gid = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
    if (gid < h) {
        const KT key = hk[gid];
        unsigned long long lo = 0, hi = nbody; // body keys below key: [0, lo)
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) / 2;
            if (k[h + mid] < key)
                lo = mid + 1;
            else
                hi = mid;
        }
        hpos[gid] = gid + lo;
    }
    for (unsigned long long x = gid; x < (nch - 1) * h; x += stride) {
        const unsigned long long c = x / h, j = x % h, e = (c + 1) * HM_CH;
        bk[c * 3 + j] = k[e + j]; // body element e - h + j
        if (v)
            bv[c * 3 + j] = v[e + j];
    }
}

template <typename KT>
__global__ void __launch_bounds__(SEG_T) k_head_merge(KT *k, uint32_t *v, uint32_t h, unsigned long long nbody,
                                                     const unsigned char *buf)
{
    constexpr int IT = HM_CH / SEG_T;
    const KT *hkp = reinterpret_cast<const KT *>(buf);
    const uint32_t *hvp = reinterpret_cast<const uint32_t *>(buf + 32);
    const unsigned long long *hpos = reinterpret_cast<const unsigned long long *>(buf + 64);
    const unsigned long long nch = (nbody + HM_CH - 1) / HM_CH;
    const KT *bk = reinterpret_cast<const KT *>(buf + HM_HDR);
    const uint32_t *bv = reinterpret_cast<const uint32_t *>(buf + HM_HDR + (nch * 3 * sizeof(KT) + 15) / 16 * 16);
    KT hk[3];
#pragma unroll
    for (int q = 0; q < 3; ++q)
        hk[q] = uint32_t(q) < h ? hkp[q] : KT(0);
    for (unsigned long long c = blockIdx.x; c < nch; c += gridDim.x) {
        const unsigned long long s0 = c * HM_CH, e = min(s0 + HM_CH, nbody);
        const unsigned long long tail = c + 1 < nch ? e - h : e; // from here on: the copies
        KT key[IT];
        uint32_t val[IT];
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const unsigned long long i = s0 + uint32_t(it * SEG_T + threadIdx.x);
            key[it] = KT(0);
            val[it] = 0u;
            if (i < e) {
                key[it] = i >= tail ? bk[c * 3 + (i - tail)] : k[h + i];
                if (v)
                    val[it] = i >= tail ? bv[c * 3 + (i - tail)] : v[h + i];
            }
        }
        __syncthreads();
#pragma unroll
        for (int it = 0; it < IT; ++it) {
            const unsigned long long i = s0 + uint32_t(it * SEG_T + threadIdx.x);
            if (i < e) {
                uint32_t le = 0;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    le += (uint32_t(q) < h && hk[q] <= key[it]) ? 1u : 0u;
                k[i + le] = key[it];
                if (v)
                    v[i + le] = val[it];
            }
        }
        if (threadIdx.x < h) {
            const unsigned long long p = hpos[threadIdx.x];
            const unsigned long long owner = p < h ? 0ull : (p - h) / HM_CH;
            if (owner == c) {
                k[p] = hkp[threadIdx.x];
                if (v)
                    v[p] = hvp[threadIdx.x];
            }
        }
        __syncthreads();
    }
}

} // namespace

// ---------------------------------------------------------------- host side
template <typename KT, bool HASV, int DB> struct SegImpl {
    static constexpr int SIGMA = 1 << DB;
    static constexpr int SMALL = DB <= 8 ? 4096 : 2048;
    static constexpr int TILE = DB <= 8 ? 4096 : 2048;
    using TPs = TilePass<KT, HASV, DB, SMALL / (32 * SEG_NW)>;
    using TPm = TilePass<KT, HASV, DB, TILE / (32 * SEG_NW)>;
    static size_t small_smem()
    {
        return 2 * SMALL * sizeof(KT) + (HASV ? 2 * SMALL * 4 : 0) + 2 * SIGMA * 4 + TPs::SCRATCH;
    }
    static size_t med_smem()
    {
        constexpr int NTD = (8 * int(sizeof(KT)) + DB - 1) / DB;
        return 2 * TILE * sizeof(KT) + (HASV ? 2 * TILE * 4 : 0) + 3 * SIGMA * 4 + size_t(NTD) * SIGMA * 4 +
               TPm::SCRATCH;
    }
    // the in-place medium pass (8-bit digits): two buffers of 2048-element
    // tiles for 4-byte keys, 1024 for 8-byte ones, so that two CTAs fit on an SM
    static constexpr int IP_TILE = sizeof(KT) == 4 ? 2048 : 1024;
    using IC = IpCfg<KT, HASV, IP_TILE>;
    static cudaError_t launch(const SegArgs &a, cudaStream_t st, int med_ctas)
    {
        static DeviceOnce attr;
        const cudaError_t ea = attr.run([] {
            cudaError_t e = cudaFuncSetAttribute(k_seg_small<KT, HASV, DB, SMALL>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(small_smem()));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_seg_medium<KT, HASV, DB, TILE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(med_smem()));
            if constexpr (DB == 8)
                if (e == cudaSuccess)
                    e = cudaFuncSetAttribute(k_seg_medium_ip<KT, HASV, IP_TILE>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(IC::SMEM));
            return e;
        });
        if (ea != cudaSuccess)
            return ea;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_seg_small<KT, HASV, DB, SMALL>, SEG_T,
                                                      small_smem());
        const int sms = num_sms();
        k_seg_small<KT, HASV, DB, SMALL><<<sms * (per > 0 ? per : 1), SEG_T, small_smem(), st>>>(a);
        if (a.med_ip) {
            if constexpr (DB == 8)
                k_seg_medium_ip<KT, HASV, IP_TILE><<<med_ctas, SEG_T, IC::SMEM, st>>>(a);
            else
                return cudaErrorInvalidValue; // the planner picks it for 8-bit digits only
        } else if (a.med_stride) {
            k_seg_medium<KT, HASV, DB, TILE><<<med_ctas, SEG_T, med_smem(), st>>>(a);
        }
        g_launches += 2;
        return cudaGetLastError();
    }
};

uint32_t seg_small_max(int db) { return db <= 8 ? 4096u : 2048u; }

// CTAs of the medium pass: two per SM, fewer when their scratch (med_max
// elements each) would pass `budget` bytes, at least 16
uint32_t seg_med_ctas(uint32_t med_max, int kb, bool hasv, size_t budget)
{
    const uint32_t most = static_cast<uint32_t>(num_sms()) * 2;
    if (!med_max)
        return 0;
    const size_t per = size_t(med_max) * (kb + (hasv ? 4 : 0));
    size_t c = budget / per;
    if (c < 16)
        c = 16;
    return c < most ? static_cast<uint32_t>(c) : most;
}

// CTAs of the in-place medium pass: two per SM
uint32_t seg_ip_ctas() { return static_cast<uint32_t>(num_sms()) * 2; }

// elements of scratch per CTA of the medium pass: its scratch blocks in
// place (ip), else an out-of-place buffer as long as the longest medium
// segment (med_max, 0: none)
static size_t seg_med_stride(bool ip, uint32_t med_max) { return !med_max ? 0 : ip ? size_t(IP_S) * IP_B : med_max; }

size_t seg_scratch_bytes(int kb, bool hasv, size_t nseg, uint32_t med_max, uint32_t med_ctas, bool ip)
{
    const size_t al = 256;
    auto up = [&](size_t x) { return (x + al - 1) / al * al; };
    const size_t per = seg_med_stride(ip, med_max);
    return up(64) + 2 * up(nseg * 4) + up(size_t(med_ctas) * per * kb) +
           (hasv ? up(size_t(med_ctas) * per * 4) : 0);
}

cudaError_t launch_segmented(void *keys, uint32_t *vals, const unsigned long long *off_dev,
                             size_t nseg, int kb, int db, uint32_t med_max, uint32_t med_ctas, bool ip,
                             void *scratch, cudaStream_t st)
{
    if (ip && db != 8)
        return cudaErrorInvalidValue;
    const size_t al = 256;
    auto up = [&](size_t x) { return (x + al - 1) / al * al; };
    char *p = static_cast<char *>(scratch);
    SegArgs a{};
    a.keys = keys;
    a.vals = vals;
    a.off = off_dev;
    a.nseg = static_cast<uint32_t>(nseg);
    a.ctr = reinterpret_cast<uint32_t *>(p);
    p += up(64);
    a.small_list = reinterpret_cast<uint32_t *>(p);
    p += up(nseg * 4);
    a.med_list = reinterpret_cast<uint32_t *>(p);
    p += up(nseg * 4);
    const size_t per = seg_med_stride(ip, med_max);
    a.scr_k = p;
    p += up(size_t(med_ctas) * per * kb);
    a.scr_v = vals ? reinterpret_cast<uint32_t *>(p) : nullptr;
    a.med_stride = med_max;
    a.med_ip = ip && med_max ? 1u : 0u;
    a.nt = (8 * kb + db - 1) / db;
    a.db = db;
    cudaError_t e = cudaMemsetAsync(a.ctr, 0, 64, st);
    if (e != cudaSuccess)
        return e;
    k_seg_classify<<<(nseg + 255) / 256 > 0 ? (nseg + 255) / 256 : 1, 256, 0, st>>>(
        a, seg_small_max(db), SEG_MED);
    g_launches += 1;
    const int mc = static_cast<int>(med_ctas);
    using u64 = unsigned long long;
    if (kb == 4) {
        if (db == 8)
            return vals ? SegImpl<uint32_t, true, 8>::launch(a, st, mc) : SegImpl<uint32_t, false, 8>::launch(a, st, mc);
        return vals ? SegImpl<uint32_t, true, 11>::launch(a, st, mc) : SegImpl<uint32_t, false, 11>::launch(a, st, mc);
    }
    if (db == 8)
        return vals ? SegImpl<u64, true, 8>::launch(a, st, mc) : SegImpl<u64, false, 8>::launch(a, st, mc);
    return vals ? SegImpl<u64, true, 11>::launch(a, st, mc) : SegImpl<u64, false, 11>::launch(a, st, mc);
}

size_t head_merge_bytes(size_t nbody, int kb, bool hasv)
{
    const size_t nch = (nbody + HM_CH - 1) / HM_CH;
    const size_t b = HM_HDR + (nch * 3 * kb + 15) / 16 * 16 + (hasv ? nch * 3 * 4 : 0);
    return (b + 255) / 256 * 256;
}

cudaError_t launch_head_save(const void *keys, const uint32_t *vals, uint32_t h, int kb, void *buf, cudaStream_t st)
{
    unsigned char *b = static_cast<unsigned char *>(buf);
    if (kb == 4)
        k_head_save<uint32_t><<<1, 32, 0, st>>>(static_cast<const uint32_t *>(keys), vals, h, b);
    else
        k_head_save<unsigned long long><<<1, 32, 0, st>>>(static_cast<const unsigned long long *>(keys), vals, h, b);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_head_merge(void *keys, uint32_t *vals, uint32_t h, size_t nbody, int kb, void *buf, cudaStream_t st)
{
    unsigned char *b = static_cast<unsigned char *>(buf);
    const size_t nch = (nbody + HM_CH - 1) / HM_CH;
    int grid = num_sms() * 2;
    if (size_t(grid) > nch)
        grid = static_cast<int>(nch);
    const int pgrid = static_cast<int>(((nch - 1) * h + 255) / 256) + 1;
    if (kb == 4) {
        k_head_prep<uint32_t><<<pgrid, 256, 0, st>>>(static_cast<const uint32_t *>(keys), vals, h, nbody, b);
        k_head_merge<uint32_t><<<grid, SEG_T, 0, st>>>(static_cast<uint32_t *>(keys), vals, h, nbody, b);
    } else {
        using u64 = unsigned long long;
        k_head_prep<u64><<<pgrid, 256, 0, st>>>(static_cast<const u64 *>(keys), vals, h, nbody, b);
        k_head_merge<u64><<<grid, SEG_T, 0, st>>>(static_cast<u64 *>(keys), vals, h, nbody, b);
    }
    g_launches += 2;
    return cudaGetLastError();
}

} // namespace rs
