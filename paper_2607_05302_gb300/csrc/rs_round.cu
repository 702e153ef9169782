// Radsort setup (Alg. 4), sortPhase (Alg. 5) and fixupPhase (Alg. 6) for
// GB300 (sm_103a).
//
// Parallel form (Sec. 4.3): the logical blocks sigma*p .. f-1 of the current
// sequence are split into p chunks of about n/p elements each.  One CTA sorts
// one chunk.  Each chunk has its own head start of sigma blocks (T holds
// 2*sigma*p blocks).  Its free list is that head start followed by its own
// input blocks in logical order, which is Lemma 1 applied per chunk.  So no
// CTA ever waits for another inside a round.
//
// Per CTA: a producer warp streams the chunk's input blocks into a ring of
// shared-memory stages with 1-D bulk copies (TMA) completing on mbarriers.
// The consumer warps then, for each tile of M = TILE/b blocks:
//   1. rank the tile's digits stably: a per-warp shared-memory table of lane
//      masks (atomicOr by digit) gives each lane the set of lanes with its
//      digit, hence its rank among a warp's equal digits; per-warp
//      histograms give each warp's offset;
//   2. scan the tile histogram for bucket starts inside the tile;
//   3. count the blocks each bucket fills and take that many new blocks
//      from the free list (newBucketBlock, eagerly, as in Alg. 5), recording
//      U (bucket) and the block's sequence number within its bucket chain;
//   4. reorder the tile by digit in shared memory, then store each bucket's
//      run into its open block and the new ones: consecutive threads write
//      consecutive addresses.
// Every element of a tile is read into shared memory before any element of
// that tile is written.  A new block's free-list index is below sigma + the
// number of blocks loaded so far (Lemma 1).  So a block is overwritten only
// after it has been consumed.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_round() { return take_status_word(); }

// ====================================================================== setup
__global__ void k_setup_pi(uint32_t *pi, uint32_t npi, uint32_t H, uint32_t nA)
{
    const uint32_t f = H + nA + 1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npi; i += gridDim.x * blockDim.x) {
        uint32_t v;
        if (i < H)
            v = i;                      // head start
        else if (i + 1 < f)
            v = 2 * H + (i - H);        // the blocks overlaying A
        else
            v = H + (i - (f - 1));      // remaining scratch blocks, the first holds the tail
        pi[i] = v;
    }
}

template <typename KT>
__global__ void k_setup_tail(const KT *Ak, const uint32_t *Av, KT *Tk, uint32_t *Tv, size_t n,
                             uint32_t b, uint32_t H, uint32_t nA, uint32_t p, uint2 *P,
                             uint32_t *state, uint32_t *lo)
{
    const uint32_t tail = static_cast<uint32_t>(n - static_cast<size_t>(nA) * b);
    const size_t src0 = static_cast<size_t>(nA) * b, dst0 = static_cast<size_t>(H) * b;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < tail; j += gridDim.x * blockDim.x) {
        Tk[dst0 + j] = Ak[src0 + j];
        if (Av)
            Tv[dst0 + j] = Av[src0 + j];
    }
    if (blockIdx.x == 0) {
        const uint32_t f = H + nA + 1;
        if (threadIdx.x == 0) {
            P[0] = make_uint2(f - 1, tail); // the input tail is a partial block
            state[ST_F] = f;
            state[ST_NP] = 1;
            state[ST_FPREV] = f;
            state[ST_LOFFTOT] = 0;
        }
        // chunk q starts at the first logical block whose first element is at
        // position >= floor(q*n/p); block H+k starts at position k*b.
        for (uint32_t q = threadIdx.x; q <= p; q += blockDim.x) {
            uint32_t v;
            if (q == p) {
                v = f;
            } else {
                unsigned long long e = (unsigned long long)(((unsigned __int128)q * n) / p);
                unsigned long long k = (e + b - 1) / b;
                v = static_cast<uint32_t>(k + H < f ? k + H : f);
            }
            lo[q] = v;
        }
    }
}

cudaError_t launch_setup(const Geom &g, const Bufs &w, uint32_t *pi, cudaStream_t st)
{
    const int T = 256;
    int blocks = static_cast<int>((g.npi + T - 1) / T);
    if (blocks > 4096)
        blocks = 4096;
    k_setup_pi<<<blocks, T, 0, st>>>(pi, g.npi, g.H, g.nA);
    const uint32_t tail = static_cast<uint32_t>(g.n - static_cast<size_t>(g.nA) * g.b);
    int tb = static_cast<int>((tail + T - 1) / T);
    if (tb < 1)
        tb = 1;
    if (g.kb == 4)
        k_setup_tail<uint32_t><<<tb, T, 0, st>>>(
            static_cast<const uint32_t *>(w.Ak), w.Av, static_cast<uint32_t *>(w.Tk), w.Tv, g.n,
            g.b, g.H, g.nA, g.p, w.P, w.state, w.lo0);
    else
        k_setup_tail<unsigned long long><<<tb, T, 0, st>>>(
            static_cast<const unsigned long long *>(w.Ak), w.Av,
            static_cast<unsigned long long *>(w.Tk), w.Tv, g.n, g.b, g.H, g.nA, g.p, w.P,
            w.state, w.lo0);
    g_launches += 2;
    return cudaGetLastError();
}

// ====================================================================== sortPhase
template <typename KT, bool HASV, int DB, int TILE, int NW, int STAGES> struct RoundCfg {
    static constexpr int SIGMA = 1 << DB;
    static constexpr int NT = NW * 32;       // consumer threads
    static constexpr int THREADS = NT + 32;  // + one producer warp
    static constexpr int MAXM = TILE / 64;   // blocks per tile (b >= 64)
    static constexpr int PF = 2 * MAXM + 64; // free-list entries prefetched per tile
    static constexpr int R = TILE / NW;      // tile elements ranked per warp
    static constexpr int ITEMS = R / 32;     // elements per consumer thread
    static_assert(R % 32 == 0, "warp range must be a multiple of 32");
    static_assert(THREADS <= 1024, "one CTA holds at most 1024 threads");
    // CTAs per SM the configuration is built for (registers are capped accordingly)
    static constexpr int MINB = (NW <= 8 && DB <= 8) ? 2 : 1;
    // column scan over the warps' counts: TPB adjacent lanes per bucket
    static constexpr int TPB = NW >= 16 ? 4 : (NW >= 4 ? 2 : 1);
    static_assert(NW % TPB == 0, "rows split evenly");
    // sigma <= 256: a per-warp table of 32-bit lane masks by digit, built
    // with shared-memory atomicOr (far cheaper here than __match_any_sync or
    // a ballot per digit bit); sigma = 2048: ballot-per-bit masks.  Either
    // way a per-warp 16-bit table keeps the running count of each digit.
    static constexpr bool PTAB = DB <= 8;
    // 32-bit key + 32-bit value: the in-place reorder writes (key, value)
    // pairs as one 8-byte word
    static constexpr bool PAIR = HASV && sizeof(KT) == 4;
    static constexpr int HROW = SIGMA + 2; // padded u16 histogram row
    static constexpr size_t al(size_t x) { return (x + 127) & ~size_t(127); }
    static constexpr size_t KBYTES = size_t(TILE) * sizeof(KT);
    static constexpr size_t STAGE = al(KBYTES + (HASV ? size_t(TILE) * 4 : 0));
    static constexpr size_t o_stage = 0;
    static constexpr size_t o_hist = o_stage + STAGES * STAGE;
    static constexpr size_t o_tab = o_hist + al(size_t(NW) * HROW * 2);
    static constexpr size_t o_bk = o_tab + (PTAB ? al(size_t(NW) * SIGMA * 4) : 0);
    static constexpr int NBK = 8; // tcnt, bstart, fill, cur, ccnt, nb, nbase, ncur
    static constexpr size_t o_psum = o_bk + al(size_t(NBK) * SIGMA * 4);
    static constexpr size_t o_qb = o_psum;
    static constexpr int LIST = 2 * SIGMA + MAXM + 1;
    // sigma <= 256: the block lists hold key/value pointers; sigma = 2048
    // (shared memory is tight): block indices
    static constexpr bool LPTR = DB <= 8;
    static constexpr size_t o_lk = o_qb + al(size_t(SIGMA) * 8);
    static constexpr size_t o_lv = o_lk + al(size_t(LIST) * (LPTR ? 8 : 4));
    static constexpr size_t o_fl = o_lv + (HASV && LPTR ? al(size_t(LIST) * 8) : 0);
    static constexpr size_t o_meta = o_fl + al(size_t(PF) * 4);
    static constexpr size_t META = 16 + MAXM * 4; // nblk, m0, lens[MAXM]
    static constexpr size_t o_bar = o_meta + al(STAGES * META);
    static constexpr size_t o_misc = o_bar + al(2 * STAGES * 8);
    static constexpr size_t SMEM = o_misc + 512;
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

template <typename KT> struct RoundArgs {
    KT *Ak;
    uint32_t *Av;
    KT *Tk;
    uint32_t *Tv;
    const uint32_t *pi;
    const uint2 *P;
    const uint32_t *state;
    const uint32_t *lo;
    uint32_t *UC;
    uint32_t *Cout;
    uint32_t *Fout;
    uint32_t *Aout;
    uint32_t p, nT, lb, shift;
};

constexpr uint32_t META_END = 0xFFFFFFFFu;
constexpr uint32_t NO_BLOCK = 0xFFFFFFFFu;

// Block-wide exclusive scan of two SIGMA-long arrays (in place allowed) by
// the NT consumer threads.  tmp: 2*NW+2 words.  Returns the totals.
template <int N, int NT> __device__ __forceinline__ void
scan2(uint32_t *a, uint32_t *bb, uint32_t *tmp, uint32_t &tot_a, uint32_t &tot_b)
{
    constexpr int NW = NT / 32;
    constexpr int IPT = (N + NT - 1) / NT;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    uint32_t va[IPT], vb[IPT], sa = 0, sb = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = t * IPT + i;
        va[i] = idx < N ? a[idx] : 0;
        vb[i] = idx < N ? bb[idx] : 0;
        sa += va[i];
        sb += vb[i];
    }
    const uint32_t ia = warp_incl_scan(sa), ib = warp_incl_scan(sb);
    if (lane == 31) {
        tmp[w] = ia;
        tmp[NW + w] = ib;
    }
    named_bar(1, NT);
    if (w == 0) {
        uint32_t x = lane < NW ? tmp[lane] : 0, y = lane < NW ? tmp[NW + lane] : 0;
        const uint32_t sx = warp_incl_scan(x), sy = warp_incl_scan(y);
        if (lane < NW) {
            tmp[lane] = sx - x;
            tmp[NW + lane] = sy - y;
        }
        if (lane == 31) {
            tmp[2 * NW] = sx;
            tmp[2 * NW + 1] = sy;
        }
    }
    named_bar(1, NT);
    uint32_t ea = ia - sa + tmp[w], eb = ib - sb + tmp[NW + w];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const int idx = t * IPT + i;
        if (idx < N) {
            a[idx] = ea;
            bb[idx] = eb;
        }
        ea += va[i];
        eb += vb[i];
    }
    tot_a = tmp[2 * NW];
    tot_b = tmp[2 * NW + 1];
}

template <typename KT, bool HASV, int DB, int TILE, int NW, int STAGES>
__global__ void __launch_bounds__(RoundCfg<KT, HASV, DB, TILE, NW, STAGES>::THREADS,
                                   RoundCfg<KT, HASV, DB, TILE, NW, STAGES>::MINB)
    k_round(RoundArgs<KT> a)
{
    using C = RoundCfg<KT, HASV, DB, TILE, NW, STAGES>;
    constexpr int SIGMA = C::SIGMA, NT = C::NT;
    constexpr uint32_t SB = 32 - DB; // UC: bucket in the top DB bits, sequence below
    extern __shared__ __align__(128) unsigned char sm[];
    uint16_t *hist = reinterpret_cast<uint16_t *>(sm + C::o_hist);
    unsigned *ptab = reinterpret_cast<unsigned *>(sm + C::o_tab);
    uint32_t *bk = reinterpret_cast<uint32_t *>(sm + C::o_bk);
    uint32_t *tcnt = bk, *bstart = bk + SIGMA, *fill = bk + 2 * SIGMA, *cur = bk + 3 * SIGMA;
    uint32_t *ccnt = bk + 4 * SIGMA, *nb = bk + 5 * SIGMA, *nbase = bk + 6 * SIGMA;
    uint32_t *ncur = bk + 7 * SIGMA;
    // per bucket: (chain offset of the tile's first element minus its start
    // in the reordered tile, index of the bucket's open block in the lists)
    uint2 *qb = reinterpret_cast<uint2 *>(sm + C::o_qb);
    // per bucket, contiguous: the open block, then the blocks opened in this
    // tile, as key and value pointers
    KT **listk = reinterpret_cast<KT **>(sm + C::o_lk);
    uint32_t **listv = reinterpret_cast<uint32_t **>(sm + C::o_lv);
    uint32_t *listb = reinterpret_cast<uint32_t *>(sm + C::o_lk); // !LPTR: block indices
    uint32_t *flbuf = reinterpret_cast<uint32_t *>(sm + C::o_fl);
    unsigned char *meta = sm + C::o_meta;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + C::o_bar);
    uint64_t *empty = full + STAGES;
    uint32_t *misc = reinterpret_cast<uint32_t *>(sm + C::o_misc);
    // misc: [0] consumed tiles, [8..] scan scratch

    const uint32_t q = blockIdx.x;
    const uint32_t b = 1u << a.lb, M = static_cast<uint32_t>(TILE) >> a.lb;
    const uint32_t lo = a.lo[q], hi = a.lo[q + 1], nblocks = hi - lo;
    const uint32_t fl_len = SIGMA + nblocks; // free-list length of this chunk
    const uint32_t mask = SIGMA - 1;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        misc[0] = 0;
        fence_mbar_init();
    }
    __syncthreads();

    // old-pi index of free-list entry k
    auto fl_index = [&](uint32_t k) -> uint32_t { return k < SIGMA ? q * SIGMA + k : lo + (k - SIGMA); };
    auto kaddr = [&](uint32_t blk) -> KT * {
        return blk < a.nT ? a.Tk + size_t(blk) * b : a.Ak + size_t(blk - a.nT) * b;
    };
    auto vaddr = [&](uint32_t blk) -> uint32_t * {
        return blk < a.nT ? a.Tv + size_t(blk) * b : a.Av + size_t(blk - a.nT) * b;
    };

    if (warp == NW) {
        // ================================================================ producer
        const uint32_t nP = a.state[ST_NP];
        // first partial with logical index >= lo
        uint32_t ip = 0;
        {
            uint32_t l = 0, r = nP;
            while (l < r) {
                uint32_t mid = (l + r) >> 1;
                if (a.P[mid].x < lo)
                    l = mid + 1;
                else
                    r = mid;
            }
            ip = l;
        }
        uint32_t m = 0, tile = 0;
        for (;; ++tile) {
            const int s = tile % STAGES;
            const uint32_t par = ((tile / STAGES) & 1u) ^ 1u;
            if (!mbar_wait(&empty[s], par))
                break;
            uint32_t *mt = reinterpret_cast<uint32_t *>(meta + s * C::META);
            if (m >= nblocks) {
                if (lane == 0) {
                    mt[0] = META_END;
                    mbar_arrive(&full[s]);
                }
                ++tile;
                break;
            }
            unsigned char *st = sm + C::o_stage + size_t(s) * C::STAGE;
            KT *stk = reinterpret_cast<KT *>(st);
            uint32_t *stv = reinterpret_cast<uint32_t *>(st + C::KBYTES);
            const uint32_t Mt = min(M, nblocks - m);
            uint32_t *lens = mt + 4;
            for (uint32_t base = 0; base < Mt; base += 32) {
                const uint32_t j = base + lane;
                const uint32_t cnt = min(32u, Mt - base);
                const uint32_t i0 = lo + m + base;
                uint32_t phys = 0;
                if (j < Mt) {
                    phys = a.pi[lo + m + j];
                    lens[j] = b;
                }
                uint2 pe = make_uint2(0xFFFFFFFFu, 0);
                if (ip + lane < nP)
                    pe = a.P[ip + lane];
                const bool inb = (ip + lane < nP) && pe.x < i0 + cnt;
                __syncwarp();
                if (inb)
                    lens[pe.x - lo - m] = pe.y;
                ip += __popc(__ballot_sync(0xffffffffu, inb));
                __syncwarp();
                uint32_t bytes = 0, len = 0;
                if (j < Mt) {
                    len = lens[j];
                    if (len) {
                        bytes = (len * sizeof(KT) + 15u) & ~15u;
                        if (HASV)
                            bytes += (len * 4u + 15u) & ~15u;
                    }
                }
                const uint32_t tot = warp_sum(bytes);
                if (lane == 0 && tot)
                    asm volatile("mbarrier.expect_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&full[s])),
                                 "r"(tot)
                                 : "memory");
                __syncwarp();
                if (j < Mt && len) {
                    bulk_g2s(stk + size_t(j) * b, kaddr(phys), (len * sizeof(KT) + 15u) & ~15u, &full[s]);
                    if (HASV)
                        bulk_g2s(stv + size_t(j) * b, vaddr(phys), (len * 4u + 15u) & ~15u, &full[s]);
                }
            }
            if (lane == 0) {
                mt[0] = Mt;
                mt[1] = m;
            }
            __syncwarp();
            if (lane == 0)
                mbar_arrive(&full[s]);
            m += Mt;
        }
        // drain: every issued copy must land before this CTA exits (only the
        // last STAGES issued tiles can still be in flight)
        if (lane == 0) {
            const uint32_t done = *(volatile uint32_t *)&misc[0];
            uint32_t t0 = tile > STAGES ? tile - STAGES : 0;
            if (done > t0)
                t0 = done;
            for (uint32_t t = t0; t < tile; ++t)
                mbar_wait(&full[t % STAGES], (t / STAGES) & 1u);
        }
        return;
    }

    // ==================================================================== consumers
    for (int c = tid; c < SIGMA; c += NT) {
        // initial output block of every bucket: head-start entry c (Alg. 5)
        cur[c] = a.pi[q * SIGMA + c];
        fill[c] = 0;
        ccnt[c] = 1;
        a.UC[q * SIGMA + c] = (uint32_t(c) << SB);
    }
    if constexpr (C::PTAB)
        for (int i = tid; i < NW * SIGMA; i += NT)
            ptab[i] = 0u;
    uint32_t alloc = SIGMA; // i_out as a free-list index
    uint32_t fl0 = SIGMA;   // free-list index of flbuf[0]
    uint32_t pfv = 0;
    if (tid < C::PF && SIGMA + tid < fl_len)
        flbuf[tid] = a.pi[fl_index(SIGMA + tid)];
    uint32_t *tmp = misc + 8;
    named_bar(1, NT);

    for (uint32_t tile = 0;; ++tile) {
        const int s = tile % STAGES;
        if (!mbar_wait(&full[s], (tile / STAGES) & 1u))
            break;
        const uint32_t *mt = reinterpret_cast<const uint32_t *>(meta + s * C::META);
        const uint32_t nblk = mt[0];
        if (nblk == META_END) {
            if (tid == 0)
                misc[0] = tile + 1;
            break;
        }
        const uint32_t m0 = mt[1];
        const uint32_t *lens = mt + 4;
        unsigned char *st = sm + C::o_stage + size_t(s) * C::STAGE;
        KT *tk = reinterpret_cast<KT *>(st);
        uint32_t *tv = reinterpret_cast<uint32_t *>(st + C::KBYTES);
        uint2 *tp = reinterpret_cast<uint2 *>(st); // (key, value) pairs after the reorder

        // ---- 1. this thread's elements into registers; stable rank within the warp
        KT key[C::ITEMS];
        uint32_t val[C::ITEMS], dig[C::ITEMS], rk[C::ITEMS];
#pragma unroll
        for (int it = 0; it < C::ITEMS; ++it) {
            const uint32_t e = warp * C::R + it * 32 + lane;
            const uint32_t slot = e >> a.lb, j = e & (b - 1);
            const bool valid = slot < nblk && j < lens[slot];
            key[it] = tk[e];
            if (HASV)
                val[it] = tv[e];
            dig[it] = valid ? digit_of(key[it], a.shift, mask) : uint32_t(SIGMA);
        }
        const unsigned lt = lanemask_lt();
        uint16_t *hw = hist + warp * C::HROW;
        for (int c = lane; c < SIGMA; c += 32)
            hw[c] = 0;
        if constexpr (C::PTAB) {
            // row by row: lanes with the same digit OR their bit into the
            // digit's mask word, read back the mask and the warp's running
            // count; the lowest of those lanes advances the count and clears
            // the word (the mask table is all zero between rows)
            unsigned *pt = ptab + warp * SIGMA;
            __syncwarp();
#pragma unroll
            for (int it = 0; it < C::ITEMS; ++it) {
                const uint32_t d = dig[it];
                const bool v = d < SIGMA;
                if (v)
                    atomicOr(&pt[d], 1u << lane);
                __syncwarp();
                const unsigned pm = v ? pt[d] : 0u;
                const uint32_t base = v ? hw[d] : 0u;
                rk[it] = base + __popc(pm & lt);
                __syncwarp();
                if (v && (__ffs(pm) - 1) == lane) {
                    hw[d] = static_cast<uint16_t>(base + __popc(pm));
                    pt[d] = 0u;
                }
                __syncwarp();
            }
        } else {
            unsigned peers[C::ITEMS];
#pragma unroll
            for (int it = 0; it < C::ITEMS; ++it)
                peers[it] = peer_mask<DB>(dig[it], dig[it] < SIGMA);
            __syncwarp();
#pragma unroll
            for (int it = 0; it < C::ITEMS; ++it) {
                const uint32_t d = dig[it];
                uint32_t base = 0;
                if (d < SIGMA)
                    base = hw[d];
                rk[it] = base + __popc(peers[it] & lt);
                __syncwarp();
                if (d < SIGMA && (__ffs(peers[it]) - 1) == lane)
                    hw[d] = static_cast<uint16_t>(base + __popc(peers[it]));
                __syncwarp();
            }
        }
        named_bar(1, NT);

        // ---- 2. per-bucket warp offsets (exclusive over warps) and tile counts:
        // TPB adjacent lanes share a bucket, each scanning NW/TPB warp rows
        // (rows are padded so that these accesses are free of bank conflicts)
        for (int t = tid; t < SIGMA * C::TPB; t += NT) {
            const int c = t / C::TPB, part = t % C::TPB;
            constexpr int RPT = NW / C::TPB;
            uint32_t h[RPT], sum = 0;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                h[r] = hist[(part * RPT + r) * C::HROW + c];
                sum += h[r];
            }
            uint32_t incl = sum;
#pragma unroll
            for (int o = 1; o < C::TPB; o <<= 1) {
                const uint32_t x = __shfl_up_sync(0xffffffffu, incl, o, C::TPB);
                if (part >= o)
                    incl += x;
            }
            uint32_t run = incl - sum;
#pragma unroll
            for (int r = 0; r < RPT; ++r) {
                hist[(part * RPT + r) * C::HROW + c] = static_cast<uint16_t>(run);
                run += h[r];
            }
            if (part == C::TPB - 1) {
                tcnt[c] = incl;
                bstart[c] = incl;
                const uint32_t fnew = fill[c] + incl;
                nb[c] = fnew >> a.lb; // blocks filled -> new blocks (eager, Alg. 5)
                nbase[c] = fnew >> a.lb;
            }
        }
        named_bar(1, NT);
        uint32_t nvalid, NB;
        scan2<SIGMA, NT>(bstart, nbase, tmp, nvalid, NB);
        named_bar(1, NT);

        // ---- 3. newBucketBlock for every block filled in this tile
        if (tid == 0 && alloc + NB > SIGMA + m0 + nblk)
            set_status(ST_INTERNAL); // Lemma 1 would be violated
        for (int c = tid; c < SIGMA; c += NT) {
            const uint32_t k0 = nbase[c], cnt = nb[c], l0 = k0 + c;
            qb[c] = make_uint2(fill[c] - bstart[c], l0);
            if constexpr (C::LPTR) {
                listk[l0] = kaddr(cur[c]);
                if (HASV)
                    listv[l0] = vaddr(cur[c]);
            } else {
                listb[l0] = cur[c];
            }
            uint32_t last = cur[c];
            for (uint32_t i = 0; i < cnt; ++i) {
                const uint32_t k = alloc + k0 + i; // free-list index
                uint32_t blk = NO_BLOCK;
                if (k < fl_len) { // always (Lemma 1); never take past the list
                    const uint32_t r = k - fl0;
                    blk = last = r < C::PF ? flbuf[r] : a.pi[fl_index(k)];
                    a.UC[fl_index(k)] = (uint32_t(c) << SB) | (ccnt[c] + i);
                }
                if constexpr (C::LPTR) {
                    listk[l0 + 1 + i] = blk == NO_BLOCK ? nullptr : kaddr(blk);
                    if (HASV)
                        listv[l0 + 1 + i] = blk == NO_BLOCK ? nullptr : vaddr(blk);
                } else {
                    listb[l0 + 1 + i] = blk;
                }
            }
            ncur[c] = last;
        }
        {   // prefetch the free-list entries the next tile may take
            const uint32_t k = alloc + NB + tid;
            if (tid < C::PF && k < fl_len)
                pfv = a.pi[fl_index(k)];
        }

        // ---- 4a. reorder the tile by digit, in place in its stage buffer
        // (every element is in registers since the barriers above)
#pragma unroll
        for (int it = 0; it < C::ITEMS; ++it) {
            const uint32_t d = dig[it];
            if (d < SIGMA) {
                const uint32_t pos = bstart[d] + hist[warp * C::HROW + d] + rk[it];
                if constexpr (C::PAIR) {
                    tp[pos] = make_uint2(static_cast<uint32_t>(key[it]), val[it]);
                } else {
                    tk[pos] = key[it];
                    if (HASV)
                        tv[pos] = val[it];
                }
            }
        }
        named_bar(1, NT);

        // ---- 4b. store every bucket run into its block chain
        constexpr int SI = (TILE + NT - 1) / NT;
#pragma unroll
        for (int k = 0; k < SI; ++k) {
            const uint32_t i = tid + k * NT;
            if (i < nvalid) {
                KT kk;
                uint32_t vv = 0;
                if constexpr (C::PAIR) {
                    const uint2 pr = tp[i];
                    kk = pr.x;
                    vv = pr.y;
                } else {
                    kk = tk[i];
                    if (HASV)
                        vv = tv[i];
                }
                const uint2 qd = qb[digit_of(kk, a.shift, mask)];
                const uint32_t qpos = i + qd.x;
                const uint32_t l = qd.y + (qpos >> a.lb), off = qpos & (b - 1);
                if constexpr (C::LPTR) {
                    KT *pk = listk[l];
                    if (pk) {
                        pk[off] = kk;
                        if (HASV)
                            listv[l][off] = vv;
                    }
                } else {
                    const uint32_t blk = listb[l];
                    if (blk != NO_BLOCK) {
                        kaddr(blk)[off] = kk;
                        if (HASV)
                            vaddr(blk)[off] = vv;
                    }
                }
            }
        }
        // the stage was read and rewritten with generic accesses; the
        // producer refills it with bulk copies (async proxy)
        fence_proxy_async_smem();
        named_bar(1, NT);
        if (tid == 0)
            mbar_arrive(&empty[s]); // stage consumed: the producer may refill it

        // ---- 5. bucket state after the tile
        for (int c = tid; c < SIGMA; c += NT) {
            const uint32_t cnt = nb[c];
            fill[c] = (fill[c] + tcnt[c]) & (b - 1);
            cur[c] = ncur[c];
            ccnt[c] += cnt;
        }
        alloc += NB;
        fl0 = alloc;
        if (tid < C::PF)
            flbuf[tid] = pfv;
        named_bar(1, NT);
    }

    for (int c = tid; c < SIGMA; c += NT) {
        a.Cout[c * a.p + q] = ccnt[c];
        a.Fout[c * a.p + q] = fill[c];
    }
    if (tid == 0)
        a.Aout[q] = alloc;
}

template <typename KT, bool HASV, int DB, int TILE, int NW, int STAGES>
static cudaError_t round_impl(const Geom &g, const Bufs &w, const uint32_t *pi, const uint32_t *lo,
                              uint32_t *UC, int round, cudaStream_t st)
{
    using C = RoundCfg<KT, HASV, DB, TILE, NW, STAGES>;
    static DeviceOnce attr; // per template instance
    cudaError_t e0 = attr.run([] {
        return cudaFuncSetAttribute(k_round<KT, HASV, DB, TILE, NW, STAGES>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    static_cast<int>(C::SMEM));
    });
    if (e0 != cudaSuccess)
        return e0;
    RoundArgs<KT> a;
    a.Ak = static_cast<KT *>(w.Ak);
    a.Av = w.Av;
    a.Tk = static_cast<KT *>(w.Tk);
    a.Tv = w.Tv;
    a.pi = pi;
    a.P = w.P;
    a.state = w.state;
    a.lo = lo;
    a.UC = UC;
    a.Cout = w.C;
    a.Fout = w.FILL;
    a.Aout = w.Aal;
    a.p = g.p;
    a.nT = g.nT;
    a.lb = g.lb;
    a.shift = static_cast<uint32_t>(round * g.db);
    k_round<KT, HASV, DB, TILE, NW, STAGES><<<g.p, C::THREADS, C::SMEM, st>>>(a);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_round(const Geom &g, const Bufs &w, const uint32_t *pi, const uint32_t *lo,
                         uint32_t *UC, int round, cudaStream_t st)
{
    using u64 = unsigned long long;
    //                       key  vals  d   TILE  NW  STAGES
    if (g.kb == 4) {
        if (g.db == 8) {
            // more chunks than SMs: two smaller CTAs per SM hide each other's barriers
            if (g.p > static_cast<uint32_t>(num_sms()))
                return g.hasv ? round_impl<uint32_t, true, 8, 4096, 8, 2>(g, w, pi, lo, UC, round, st)
                              : round_impl<uint32_t, false, 8, 4096, 8, 3>(g, w, pi, lo, UC, round, st);
            return g.hasv ? round_impl<uint32_t, true, 8, 8192, 16, 2>(g, w, pi, lo, UC, round, st)
                          : round_impl<uint32_t, false, 8, 8192, 16, 3>(g, w, pi, lo, UC, round, st);
        }
        return g.hasv ? round_impl<uint32_t, true, 11, 4096, 8, 2>(g, w, pi, lo, UC, round, st)
                      : round_impl<uint32_t, false, 11, 4096, 8, 3>(g, w, pi, lo, UC, round, st);
    }
    if (g.db == 8)
        return g.hasv ? round_impl<u64, true, 8, 4096, 16, 3>(g, w, pi, lo, UC, round, st)
                      : round_impl<u64, false, 8, 8192, 16, 2>(g, w, pi, lo, UC, round, st);
    return g.hasv ? round_impl<u64, true, 11, 2048, 8, 3>(g, w, pi, lo, UC, round, st)
                  : round_impl<u64, false, 11, 4096, 8, 2>(g, w, pi, lo, UC, round, st);
}

// ====================================================================== fixupPhase
// One CTA: scans over the sigma*p groups, the new P, f, the leftover offsets
// and the chunk bounds of the next round.  Group (bucket c, chunk q) is
// C[c*p + q].  Modes (FixMode):
//   EVEN: bucket-major, chunk-minor order (equal digits of earlier chunks
//     first: stability across chunks, Sec. 4.3); the next round's chunks
//     split the elements evenly;
//   SPLIT: the same order, and the next round's chunk q is bucket q (an MSD
//     split, Sec. 4.3: p = sigma);
//   PER_CHUNK: chunk-major, bucket-minor order: each chunk's output stays a
//     run of its own (the chunk is sorted independently), and the next
//     round's chunks are the same runs.
constexpr int FX_T = 1024;

// exclusive scan over a 1024-thread block; s_w holds 33 entries
template <typename T> __device__ __forceinline__ T block_excl_scan(T v, T *s_w, T &total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const T inc = warp_incl_scan(v);
    if (lane == 31)
        s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        const T x = s_w[lane];
        const T sx = warp_incl_scan(x);
        s_w[lane] = sx - x;
        if (lane == 31)
            s_w[32] = sx;
    }
    __syncthreads();
    const T r = inc - v + s_w[w];
    total = s_w[32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(FX_T) k_fixup_scan(const uint32_t *C, const uint32_t *FILL,
                                                      uint32_t *S, unsigned long long *E, uint2 *P,
                                                      const uint32_t *Aal, const uint32_t *lo_old,
                                                      uint32_t *lo_new, uint32_t *LOff,
                                                      uint32_t *state, uint32_t G, uint32_t p,
                                                      uint32_t sigma, uint32_t H, uint32_t npi,
                                                      uint32_t b, unsigned long long n, int mode)
{
    __shared__ unsigned long long s_e[33];
    __shared__ uint32_t s_c[33];
    const int t = threadIdx.x;
    // group of position i in the order of the output
    auto grp = [&](uint32_t i) -> uint32_t {
        return mode == FIX_PER_CHUNK ? (i % sigma) * p + i / sigma : i;
    };
    // groups: block counts and element counts
    const uint32_t per = (G + FX_T - 1) / FX_T;
    const uint32_t g0 = min(G, t * per), g1 = min(G, g0 + per);
    uint32_t sc = 0;
    unsigned long long se = 0;
    for (uint32_t i = g0; i < g1; ++i) {
        const uint32_t g = grp(i);
        sc += C[g];
        se += (unsigned long long)(C[g] - 1) * b + FILL[g];
    }
    uint32_t totC;
    unsigned long long totE;
    uint32_t ec = block_excl_scan<uint32_t>(sc, s_c, totC);
    unsigned long long ee = block_excl_scan<unsigned long long>(se, s_e, totE);
    for (uint32_t i = g0; i < g1; ++i) {
        const uint32_t g = grp(i);
        const uint32_t c = C[g];
        S[g] = H + ec;
        E[g] = ee;
        P[i] = make_uint2(H + ec + c - 1, FILL[g]); // each group's open block, in logical order
        ec += c;
        ee += (unsigned long long)(c - 1) * b + FILL[g];
    }
    const uint32_t f_new = H + totC;
    // leftover free-list entries per chunk
    const uint32_t perq = (p + FX_T - 1) / FX_T;
    const uint32_t q0 = min(p, t * perq), q1 = min(p, q0 + perq);
    uint32_t sl = 0, sa = 0;
    for (uint32_t qq = q0; qq < q1; ++qq) {
        sl += sigma + (lo_old[qq + 1] - lo_old[qq]) - Aal[qq];
        sa += Aal[qq];
    }
    uint32_t totL, totA;
    uint32_t el = block_excl_scan<uint32_t>(sl, s_c, totL);
    (void)block_excl_scan<uint32_t>(sa, s_c, totA);
    for (uint32_t qq = q0; qq < q1; ++qq) {
        LOff[qq] = el;
        el += sigma + (lo_old[qq + 1] - lo_old[qq]) - Aal[qq];
    }
    if (t == 0) {
        LOff[p] = totL;
        if (totE != n || totA != totC)
            set_status(ST_INTERNAL); // element / block counts of the groups
        if (npi - totC < H)
            set_status(ST_INTERNAL); // Lemma 2
        if (totL + (npi - state[ST_F]) != npi - totC)
            set_status(ST_INTERNAL); // unallocated-block count
    }
    __syncthreads(); // S, E visible to the whole block
    // next round's chunk bounds: EVEN, the first logical block whose first
    // element is at position >= floor(q*n/p); SPLIT, the first block of
    // bucket q (group (q, 0)); PER_CHUNK, the first block of chunk q (group
    // (0, q))
    for (uint32_t qq = t; qq <= p; qq += FX_T) {
        uint32_t v;
        if (qq == 0) {
            v = H;
        } else if (qq == p) {
            v = f_new;
        } else if (mode == FIX_SPLIT) {
            v = S[qq * p];
        } else if (mode == FIX_PER_CHUNK) {
            v = S[qq];
        } else {
            const unsigned long long e = (unsigned long long)(((unsigned __int128)qq * n) / p);
            uint32_t l = 0, r = G;
            while (l < r) { // first group whose last block starts at >= e
                const uint32_t mid = (l + r) >> 1;
                const unsigned long long last = E[mid] + (unsigned long long)(C[mid] - 1) * b;
                if (last < e)
                    l = mid + 1;
                else
                    r = mid;
            }
            if (l == G) {
                v = f_new;
            } else {
                const unsigned long long k = e > E[l] ? (e - E[l] + b - 1) / b : 0;
                v = S[l] + static_cast<uint32_t>(k);
            }
        }
        lo_new[qq] = v;
    }
    __syncthreads();
    if (t == 0) {
        state[ST_LOFFTOT] = totL;
        state[ST_FPREV] = state[ST_F];
        state[ST_F] = f_new;
        state[ST_NP] = G;
    }
}

// pi'[dst] = pi[i] for every old logical index i (Alg. 6's shuffle plus the
// head start and the remaining unallocated blocks).
__global__ void k_fixup_place(const uint32_t *pi_old, uint32_t *pi_new, const uint32_t *UC,
                              const uint32_t *S, const uint32_t *Aal, const uint32_t *lo_old,
                              const uint32_t *LOff, const uint32_t *state, uint32_t npi,
                              uint32_t sigma, uint32_t p, uint32_t H, uint32_t db)
{
    extern __shared__ uint32_t s_lo[];
    for (uint32_t i = threadIdx.x; i <= p; i += blockDim.x)
        s_lo[i] = lo_old[i];
    __syncthreads();
    const uint32_t f_old = state[ST_FPREV], f_new = state[ST_F], lofftot = state[ST_LOFFTOT];
    const uint32_t SB = 32 - db, smask = (1u << SB) - 1;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npi; i += gridDim.x * blockDim.x) {
        uint32_t fidx; // index into the list of unallocated blocks
        uint32_t dst;
        bool allocated = false;
        if (i < f_old) {
            uint32_t qq, k;
            if (i < H) {
                qq = i / sigma;
                k = i - qq * sigma;
            } else {
                uint32_t l = 0, r = p; // last chunk with lo <= i
                while (l < r) {
                    const uint32_t mid = (l + r + 1) >> 1;
                    if (s_lo[mid] <= i)
                        l = mid;
                    else
                        r = mid - 1;
                }
                qq = l;
                k = sigma + (i - s_lo[qq]);
            }
            if (k < Aal[qq]) {
                const uint32_t uc = UC[i];
                dst = S[(uc >> SB) * p + qq] + (uc & smask);
                allocated = true;
            } else {
                fidx = LOff[qq] + (k - Aal[qq]);
            }
        } else {
            fidx = lofftot + (i - f_old);
        }
        if (!allocated)
            dst = fidx < H ? fidx : f_new + (fidx - H);
        pi_new[dst] = pi_old[i];
    }
}

cudaError_t launch_fixup(const Geom &g, const Bufs &w, const uint32_t *pi_old, uint32_t *pi_new,
                         const uint32_t *UC, const uint32_t *lo_old, uint32_t *lo_new, int mode,
                         cudaStream_t st)
{
    if ((mode == FIX_SPLIT && g.p != g.sigma) || mode < FIX_EVEN || mode > FIX_PER_CHUNK)
        return cudaErrorInvalidValue;
    k_fixup_scan<<<1, FX_T, 0, st>>>(w.C, w.FILL, w.S, w.E, w.P, w.Aal, lo_old, lo_new, w.LOff,
                                     w.state, g.G, g.p, g.sigma, g.H, g.npi, g.b,
                                     (unsigned long long)g.n, mode);
    int blocks = static_cast<int>((g.npi + 255) / 256);
    if (blocks > 8192)
        blocks = 8192;
    k_fixup_place<<<blocks, 256, (g.p + 1) * 4, st>>>(pi_old, pi_new, UC, w.S, w.Aal, lo_old,
                                                      w.LOff, w.state, g.npi, g.sigma, g.p, g.H,
                                                      g.db);
    g_launches += 2;
    return cudaGetLastError();
}

// ====================================================================== gather
// Deficit prefix over P: D[j] = sum over partials j' < j of (b - len).
__global__ void k_deficit(const uint2 *P, const uint32_t *state, unsigned long long *D, uint32_t b)
{
    __shared__ unsigned long long s_w[32];
    const uint32_t nP = state[ST_NP];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint32_t per = (nP + blockDim.x - 1) / blockDim.x;
    const uint32_t j0 = min(nP, t * per), j1 = min(nP, j0 + per);
    unsigned long long s = 0;
    for (uint32_t j = j0; j < j1; ++j)
        s += b - P[j].y;
    unsigned long long inc = warp_incl_scan(s);
    if (lane == 31)
        s_w[w] = inc;
    __syncthreads();
    if (w == 0) {
        unsigned long long x = lane < (int)(blockDim.x / 32) ? s_w[lane] : 0;
        unsigned long long sx = warp_incl_scan(x);
        s_w[lane] = sx - x;
    }
    __syncthreads();
    unsigned long long e = inc - s + s_w[w];
    for (uint32_t j = j0; j < j1; ++j) {
        D[j] = e;
        e += b - P[j].y;
    }
    if (j1 == nP && j0 < j1)
        D[nP] = e;
    if (nP == 0 && t == 0)
        D[0] = 0;
}

// One warp per logical block: its first element is at (i-H)*b - D[#partials
// before i]; its length comes from P (sizeOfNextBlock, Alg. 3).
template <typename KT>
__global__ void k_gather(const KT *Ak, const uint32_t *Av, const KT *Tk, const uint32_t *Tv,
                         const uint32_t *pi, const uint2 *P, const unsigned long long *D,
                         const uint32_t *state, KT *ok, uint32_t *ov, uint32_t H, uint32_t nT,
                         uint32_t b)
{
    const uint32_t f = state[ST_F], nP = state[ST_NP];
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t i = H + wid; i < f; i += nwarps) {
        uint32_t l = 0, r = nP;
        while (l < r) {
            const uint32_t mid = (l + r) >> 1;
            if (P[mid].x < i)
                l = mid + 1;
            else
                r = mid;
        }
        const unsigned long long pos = (unsigned long long)(i - H) * b - D[l];
        const uint32_t len = (l < nP && P[l].x == i) ? P[l].y : b;
        const uint32_t phys = pi[i];
        const size_t off = (phys < nT ? size_t(phys) : size_t(phys - nT)) * b;
        const KT *sk = (phys < nT ? Tk : Ak) + off;
        const uint32_t *svp = Av ? (phys < nT ? Tv : Av) + off : nullptr;
        for (uint32_t j = lane; j < len; j += 32) {
            ok[pos + j] = sk[j];
            if (ov)
                ov[pos + j] = svp[j];
        }
    }
}

cudaError_t launch_deficit(const Geom &g, const Bufs &w, cudaStream_t st)
{
    k_deficit<<<1, 1024, 0, st>>>(w.P, w.state, w.E, g.b);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_gather(const Geom &g, const Bufs &w, const uint32_t *pi, void *out_k,
                          uint32_t *out_v, cudaStream_t st)
{
    launch_deficit(g, w, st);
    int blocks = static_cast<int>((size_t(g.npi) * 32 + 255) / 256);
    if (blocks > 16384)
        blocks = 16384;
    if (blocks < 1)
        blocks = 1;
    if (g.kb == 4)
        k_gather<uint32_t><<<blocks, 256, 0, st>>>(
            static_cast<const uint32_t *>(w.Ak), g.hasv ? w.Av : nullptr,
            static_cast<const uint32_t *>(w.Tk), w.Tv, pi, w.P, w.E, w.state,
            static_cast<uint32_t *>(out_k), g.hasv ? out_v : nullptr, g.H, g.nT, g.b);
    else
        k_gather<unsigned long long><<<blocks, 256, 0, st>>>(
            static_cast<const unsigned long long *>(w.Ak), g.hasv ? w.Av : nullptr,
            static_cast<const unsigned long long *>(w.Tk), w.Tv, pi, w.P, w.E, w.state,
            static_cast<unsigned long long *>(out_k), g.hasv ? out_v : nullptr, g.H, g.nT, g.b);
    g_launches += 1;
    return cudaGetLastError();
}

} // namespace rs
