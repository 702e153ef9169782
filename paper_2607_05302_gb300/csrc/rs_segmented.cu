// Batched segmented sort for sm_103a: many independent arrays in one call.
//
// Each segment [off[s], off[s+1]) is sorted stably on its own.  Segments fall
// into three classes by length:
//   * small (<= SEG_SMALL): one CTA holds the whole segment in shared memory
//     and runs n_t stable counting-sort passes there (ping-pong buffers);
//   * medium (<= SEG_MED): one CTA runs an out-of-place LSD sort between the
//     segment and its own scratch region.  This is the paper's suggestion of
//     using the scratch array T as A' of Alg. 1 for arrays smaller than T
//     (Sec. 5, results);
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

// medium segments: out-of-place LSD between the segment and this CTA's
// scratch region (Alg. 1 per digit), tile by tile
template <typename KT, bool HASV, int DB, int TILE>
__global__ void __launch_bounds__(SEG_T) k_seg_medium(SegArgs a)
{
    using TP = TilePass<KT, HASV, DB, TILE / (32 * SEG_NW)>;
    constexpr int SIGMA = 1 << DB;
    extern __shared__ __align__(16) unsigned char sm[];
    KT *tk0 = reinterpret_cast<KT *>(sm);
    KT *tk1 = tk0 + TILE;
    uint32_t *tv0 = reinterpret_cast<uint32_t *>(tk1 + TILE);
    uint32_t *tv1 = tv0 + (HASV ? TILE : 0);
    uint32_t *tcnt = tv1 + (HASV ? TILE : 0);
    uint32_t *bstart = tcnt + SIGMA;
    unsigned long long *run = reinterpret_cast<unsigned long long *>(bstart + SIGMA);
    uint32_t *gh = reinterpret_cast<uint32_t *>(run + SIGMA);
    unsigned char *scratch = reinterpret_cast<unsigned char *>(gh + SIGMA);
    __shared__ uint32_t s_t;
    KT *keys = static_cast<KT *>(a.keys);
    KT *sck = static_cast<KT *>(a.scr_k) + size_t(blockIdx.x) * a.med_stride;
    uint32_t *scv = HASV ? a.scr_v + size_t(blockIdx.x) * a.med_stride : nullptr;
    const uint32_t count = a.ctr[1];
    const uint32_t mask = SIGMA - 1;
    for (;;) {
        if (threadIdx.x == 0)
            s_t = atomicAdd(&a.ctr[3], 1u);
        __syncthreads();
        const uint32_t t = s_t;
        if (t >= count)
            break;
        const uint32_t sgi = a.med_list[t];
        const unsigned long long o = a.off[sgi];
        const uint32_t len = static_cast<uint32_t>(a.off[sgi + 1] - o);
        if (len > a.med_stride) { // the host sized the scratch from its offsets
            set_status(ST_INTERNAL);
            continue;
        }
        KT *sk = keys + o, *dk = sck;
        uint32_t *svp = HASV ? a.vals + o : nullptr, *dvp = scv;
        for (int r = 0; r < a.nt; ++r) {
            const uint32_t shift = uint32_t(r * DB);
            // histogram of digit r over the segment (Alg. 1), then its prefix
            for (int c = threadIdx.x; c < SIGMA; c += SEG_T)
                gh[c] = 0;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < len; i += SEG_T)
                atomicAdd(&gh[digit_of(sk[i], shift, mask)], 1u);
            __syncthreads();
            if (threadIdx.x < 32) {
                unsigned long long carry = 0;
                for (int c0 = 0; c0 < SIGMA; c0 += 32) {
                    const unsigned long long v = gh[c0 + threadIdx.x];
                    const unsigned long long inc = warp_incl_scan(v);
                    run[c0 + threadIdx.x] = carry + inc - v;
                    carry += __shfl_sync(0xffffffffu, inc, 31);
                }
            }
            __syncthreads();
            // stable scatter tile by tile
            for (uint32_t t0 = 0; t0 < len; t0 += TILE) {
                const uint32_t cnt = min(uint32_t(TILE), len - t0);
                for (uint32_t i = threadIdx.x; i < cnt; i += SEG_T) {
                    tk0[i] = sk[t0 + i];
                    if (HASV)
                        tv0[i] = svp[t0 + i];
                }
                __syncthreads();
                TP::run(tk0, tv0, tk1, tv1, cnt, shift, scratch, tcnt, bstart);
                for (uint32_t i = threadIdx.x; i < cnt; i += SEG_T) {
                    const KT kk = tk1[i];
                    const uint32_t d = digit_of(kk, shift, mask);
                    const unsigned long long dst = run[d] + (i - bstart[d]);
                    dk[dst] = kk;
                    if (HASV)
                        dvp[dst] = tv1[i];
                }
                __syncthreads();
                for (int c = threadIdx.x; c < SIGMA; c += SEG_T)
                    run[c] += tcnt[c];
                __syncthreads();
            }
            KT *tkp = sk;
            sk = dk;
            dk = tkp;
            uint32_t *tvp = svp;
            svp = dvp;
            dvp = tvp;
        }
        if (sk != keys + o) { // odd number of passes: the result is in the scratch
            for (uint32_t i = threadIdx.x; i < len; i += SEG_T) {
                keys[o + i] = sk[i];
                if (HASV)
                    a.vals[o + i] = svp[i];
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
        return 2 * TILE * sizeof(KT) + (HASV ? 2 * TILE * 4 : 0) + 2 * SIGMA * 4 + SIGMA * 8 +
               SIGMA * 4 + TPm::SCRATCH;
    }
    static cudaError_t launch(const SegArgs &a, cudaStream_t st, int med_ctas)
    {
        static DeviceOnce attr;
        const cudaError_t ea = attr.run([] {
            cudaError_t e = cudaFuncSetAttribute(k_seg_small<KT, HASV, DB, SMALL>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, int(small_smem()));
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(k_seg_medium<KT, HASV, DB, TILE>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, int(med_smem()));
            return e;
        });
        if (ea != cudaSuccess)
            return ea;
        int per = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_seg_small<KT, HASV, DB, SMALL>, SEG_T,
                                                      small_smem());
        const int sms = num_sms();
        k_seg_small<KT, HASV, DB, SMALL><<<sms * (per > 0 ? per : 1), SEG_T, small_smem(), st>>>(a);
        if (a.med_stride)
            k_seg_medium<KT, HASV, DB, TILE><<<med_ctas, SEG_T, med_smem(), st>>>(a);
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

// med_max: the longest medium segment (0: none), the per-CTA scratch stride
size_t seg_scratch_bytes(int kb, bool hasv, size_t nseg, uint32_t med_max, uint32_t med_ctas)
{
    const size_t al = 256;
    auto up = [&](size_t x) { return (x + al - 1) / al * al; };
    return up(64) + 2 * up(nseg * 4) + up(size_t(med_ctas) * med_max * kb) +
           (hasv ? up(size_t(med_ctas) * med_max * 4) : 0);
}

cudaError_t launch_segmented(void *keys, uint32_t *vals, const unsigned long long *off_dev,
                             size_t nseg, int kb, int db, uint32_t med_max, uint32_t med_ctas, void *scratch,
                             cudaStream_t st)
{
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
    a.scr_k = p;
    p += up(size_t(med_ctas) * med_max * kb);
    a.scr_v = vals ? reinterpret_cast<uint32_t *>(p) : nullptr;
    a.med_stride = med_max;
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

} // namespace rs
