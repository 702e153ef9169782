// Comparison baseline: out-of-place LSD radix sort (Alg. 1 per digit,
// t = n_t-1 .. 0) for sm_103a.
//
// One upfront pass histograms every digit position in a single read of the
// keys (the paper's "generic" variant, Sec. 5).  Each round then makes one
// pass A -> A'.  A tile takes a ticket (dispatch order), ranks its digits
// stably (lane masks by digit from a shared-memory atomicOr table, or a
// ballot per digit bit for 11-bit digits, plus per-warp histograms) and publishes its per-digit
// counts.  It gets its exclusive per-digit prefix by a decoupled look-back
// over earlier tiles, with bounded spins, and stores each digit run
// contiguously from a digit-sorted copy in shared memory.  The look-back
// status word is 0 (not ready), count+1 (tile aggregate) or
// 0x80000000|inclusive prefix.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_oop() { return take_status_word(); }

constexpr uint32_t LB_INCL = 0x80000000u;

template <typename KT, int DB>
__global__ void k_oop_hist(const KT *keys, size_t n, int nt, unsigned long long *hist)
{
    constexpr int SIGMA = 1 << DB;
    extern __shared__ uint32_t sh[]; // nt * SIGMA
    for (int i = threadIdx.x; i < nt * SIGMA; i += blockDim.x)
        sh[i] = 0;
    __syncthreads();
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const KT k = keys[i];
        for (int r = 0; r < nt; ++r)
            atomicAdd(&sh[r * SIGMA + digit_of(k, uint32_t(r * DB), SIGMA - 1)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nt * SIGMA; i += blockDim.x)
        if (sh[i])
            atomicAdd(&hist[i], (unsigned long long)sh[i]);
}

// exclusive scan of each digit position's histogram (one block per position)
template <int DB> __global__ void k_oop_offsets(const unsigned long long *hist, unsigned long long *off)
{
    constexpr int SIGMA = 1 << DB;
    __shared__ unsigned long long s[SIGMA];
    const int r = blockIdx.x;
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        s[c] = hist[r * SIGMA + c];
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long run = 0;
        for (int c = 0; c < SIGMA; ++c) {
            const unsigned long long v = s[c];
            s[c] = run;
            run += v;
        }
    }
    __syncthreads();
    for (int c = threadIdx.x; c < SIGMA; c += blockDim.x)
        off[r * SIGMA + c] = s[c];
}

template <typename KT, bool HASV, int DB, int TILE, int NW> struct OopCfg {
    static constexpr int SIGMA = 1 << DB;
    static constexpr int NT = NW * 32;
    static constexpr int R = TILE / NW;
    static constexpr size_t al(size_t x) { return (x + 127) & ~size_t(127); }
    static constexpr size_t o_k = 0;
    static constexpr size_t o_v = o_k + al(size_t(TILE) * sizeof(KT));
    static constexpr size_t o_sk = o_v + (HASV ? al(size_t(TILE) * 4) : 0);
    static constexpr size_t o_sv = o_sk + al(size_t(TILE) * sizeof(KT));
    static constexpr size_t o_rank = o_sv + (HASV ? al(size_t(TILE) * 4) : 0);
    static constexpr size_t o_hist = o_rank + al(size_t(TILE) * 2);
    static constexpr size_t o_bk = o_hist + al(size_t(NW) * SIGMA * 2);
    static constexpr bool PTAB = DB <= 8; // lane masks by digit via shared atomicOr
    static constexpr size_t o_ptab = o_bk + al(size_t(SIGMA) * 16); // after tcnt, bstart, gbase(u64)
    static constexpr size_t o_misc = o_ptab + (PTAB ? al(size_t(NW) * SIGMA * 4) : 0);
    static constexpr size_t SMEM = o_misc + 256;
    static_assert(SMEM <= 227 * 1024, "shared memory budget");
};

template <typename KT, bool HASV, int DB, int TILE, int NW>
__global__ void __launch_bounds__(NW * 32, 1)
    k_oop_round(const KT *ik, const uint32_t *iv, KT *ok, uint32_t *ov, size_t n, uint32_t shift,
                const unsigned long long *goff, uint32_t *status, uint32_t *ticket)
{
    using C = OopCfg<KT, HASV, DB, TILE, NW>;
    constexpr int SIGMA = C::SIGMA, NT = C::NT;
    extern __shared__ __align__(128) unsigned char sm[];
    KT *tk = reinterpret_cast<KT *>(sm + C::o_k);
    uint32_t *tv = reinterpret_cast<uint32_t *>(sm + C::o_v);
    KT *sk = reinterpret_cast<KT *>(sm + C::o_sk);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sm + C::o_sv);
    uint16_t *rank16 = reinterpret_cast<uint16_t *>(sm + C::o_rank);
    uint16_t *hist = reinterpret_cast<uint16_t *>(sm + C::o_hist);
    uint32_t *tcnt = reinterpret_cast<uint32_t *>(sm + C::o_bk);
    uint32_t *bstart = tcnt + SIGMA;
    unsigned long long *gbase = reinterpret_cast<unsigned long long *>(bstart + SIGMA);
    uint32_t *misc = reinterpret_cast<uint32_t *>(sm + C::o_misc);
    unsigned *ptab = reinterpret_cast<unsigned *>(sm + C::o_ptab);
    if constexpr (C::PTAB)
        for (int i = threadIdx.x; i < NW * SIGMA; i += blockDim.x)
            ptab[i] = 0u;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t mask = SIGMA - 1;
    const size_t ntiles = (n + TILE - 1) / TILE;

    for (;;) {
        if (tid == 0)
            misc[0] = atomicAdd(ticket, 1u);
        __syncthreads();
        const size_t tile = misc[0];
        if (tile >= ntiles)
            break;
        const size_t e0 = tile * TILE;
        const uint32_t cnt = static_cast<uint32_t>(min(size_t(TILE), n - e0));
        for (uint32_t i = tid; i < cnt; i += NT) {
            tk[i] = ik[e0 + i];
            if (HASV)
                tv[i] = iv[e0 + i];
        }
        uint16_t *hw = hist + warp * SIGMA;
        for (int c = lane; c < SIGMA; c += 32)
            hw[c] = 0;
        __syncthreads();
        const unsigned lt = lanemask_lt();
        for (int it = 0; it < C::R / 32; ++it) {
            const uint32_t e = warp * C::R + it * 32 + lane;
            const bool valid = e < cnt;
            const uint32_t d = valid ? digit_of(tk[e], shift, mask) : SIGMA;
            unsigned peers;
            if constexpr (C::PTAB) {
                unsigned *pt = ptab + warp * SIGMA;
                if (valid)
                    atomicOr(&pt[d], 1u << lane);
                __syncwarp();
                peers = valid ? pt[d] : 0u;
                __syncwarp();
                if (valid && (__ffs(peers) - 1) == lane)
                    pt[d] = 0u;
            } else {
                peers = peer_mask<DB>(d, valid);
            }
            uint32_t base = 0;
            if (valid) {
                base = hw[d];
                rank16[e] = static_cast<uint16_t>(base + __popc(peers & lt));
            }
            __syncwarp();
            if (valid && (__ffs(peers) - 1) == lane)
                hw[d] = static_cast<uint16_t>(base + __popc(peers));
            __syncwarp();
        }
        __syncthreads();
        for (int c = tid; c < SIGMA; c += NT) {
            uint32_t run = 0;
            for (int w = 0; w < NW; ++w) {
                const uint32_t h = hist[w * SIGMA + c];
                hist[w * SIGMA + c] = static_cast<uint16_t>(run);
                run += h;
            }
            tcnt[c] = run;
            // publish this tile's aggregate (or inclusive prefix for tile 0)
            volatile uint32_t *st = status + tile * SIGMA + c;
            *st = tile == 0 ? (LB_INCL | run) : (run + 1);
        }
        __syncthreads();
        // in-tile exclusive scan of the counts (single warp, SIGMA small)
        if (warp == 0) {
            uint32_t carry = 0;
            for (int c0 = 0; c0 < SIGMA; c0 += 32) {
                const uint32_t v = tcnt[c0 + lane];
                const uint32_t inc = warp_incl_scan(v);
                bstart[c0 + lane] = carry + inc - v;
                carry += __shfl_sync(0xffffffffu, inc, 31);
            }
        }
        // decoupled look-back for the global prefix of each digit
        for (int c = tid; c < SIGMA; c += NT) {
            unsigned long long excl = 0;
            if (tile > 0) {
                long long t = static_cast<long long>(tile) - 1;
                unsigned spins = 0;
                while (t >= 0) {
                    const uint32_t s = *(volatile uint32_t *)(status + size_t(t) * SIGMA + c);
                    if (s == 0) {
                        if (++spins > SPIN_LIMIT) {
                            set_status(ST_TIMEOUT);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    if (s & LB_INCL) {
                        excl += s & ~LB_INCL;
                        break;
                    }
                    excl += s - 1;
                    --t;
                }
                *(volatile uint32_t *)(status + tile * SIGMA + c) =
                    LB_INCL | static_cast<uint32_t>(excl + tcnt[c]);
            }
            gbase[c] = goff[c] + excl;
        }
        __syncthreads();
        for (int it = 0; it < C::R / 32; ++it) {
            const uint32_t e = warp * C::R + it * 32 + lane;
            if (e < cnt) {
                const KT key = tk[e];
                const uint32_t d = digit_of(key, shift, mask);
                const uint32_t pos = bstart[d] + hist[warp * SIGMA + d] + rank16[e];
                sk[pos] = key;
                if (HASV)
                    sv[pos] = tv[e];
            }
        }
        __syncthreads();
        for (uint32_t i = tid; i < cnt; i += NT) {
            const KT key = sk[i];
            const uint32_t d = digit_of(key, shift, mask);
            const unsigned long long dst = gbase[d] + (i - bstart[d]);
            ok[dst] = key;
            if (HASV)
                ov[dst] = sv[i];
        }
        __syncthreads();
    }
}

template <typename KT, bool HASV, int DB, int TILE, int NW>
static size_t oop_scratch(size_t n)
{
    constexpr int SIGMA = 1 << DB;
    const int nt = (8 * int(sizeof(KT)) + DB - 1) / DB;
    const size_t ntiles = (n + TILE - 1) / TILE;
    return 2 * size_t(nt) * SIGMA * 8 + ntiles * SIGMA * 4 + 256;
}

template <typename KT, bool HASV, int DB, int TILE, int NW>
static cudaError_t oop_impl(KT *keys, uint32_t *vals, KT *keys_alt, uint32_t *vals_alt, size_t n,
                            void *scratch, cudaStream_t st)
{
    using C = OopCfg<KT, HASV, DB, TILE, NW>;
    constexpr int SIGMA = 1 << DB;
    const int nt = (8 * int(sizeof(KT)) + DB - 1) / DB;
    const size_t ntiles = (n + TILE - 1) / TILE;
    if (n >= (size_t(1) << 31))
        return cudaErrorInvalidValue;
    // scratch: histograms, offsets, look-back status, tickets
    const size_t hbytes = size_t(nt) * SIGMA * 8;
    const size_t sbytes = ntiles * SIGMA * 4;
    char *scr = static_cast<char *>(scratch);
    const bool own = scr == nullptr;
    cudaError_t e = cudaSuccess;
    if (own)
        e = cudaMallocAsync(reinterpret_cast<void **>(&scr), oop_scratch<KT, HASV, DB, TILE, NW>(n), st);
    if (e != cudaSuccess)
        return e;
    unsigned long long *hist = reinterpret_cast<unsigned long long *>(scr);
    unsigned long long *off = reinterpret_cast<unsigned long long *>(scr + hbytes);
    uint32_t *status = reinterpret_cast<uint32_t *>(scr + 2 * hbytes);
    uint32_t *ticket = reinterpret_cast<uint32_t *>(scr + 2 * hbytes + sbytes);
    cudaMemsetAsync(hist, 0, hbytes, st);
    const int sms = num_sms();
    k_oop_hist<KT, DB><<<sms * 4, 512, nt * SIGMA * 4, st>>>(keys, n, nt, hist);
    k_oop_offsets<DB><<<nt, 256, 0, st>>>(hist, off);
    g_launches += 2 + nt;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_oop_round<KT, HASV, DB, TILE, NW>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, int(C::SMEM));
        attr = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_oop_round<KT, HASV, DB, TILE, NW>,
                                                  C::NT, C::SMEM);
    if (per_sm < 1)
        per_sm = 1;
    size_t grid = size_t(sms) * per_sm;
    if (grid > ntiles)
        grid = ntiles;
    KT *src = keys, *dst = keys_alt;
    uint32_t *vs = vals, *vd = vals_alt;
    for (int r = 0; r < nt; ++r) {
        cudaMemsetAsync(status, 0, sbytes + 256, st);
        k_oop_round<KT, HASV, DB, TILE, NW><<<unsigned(grid), C::NT, C::SMEM, st>>>(
            src, vs, dst, vd, n, uint32_t(r * DB), off + size_t(r) * SIGMA, status, ticket);
        KT *t = src;
        src = dst;
        dst = t;
        uint32_t *u = vs;
        vs = vd;
        vd = u;
    }
    if (nt & 1) { // result is in the alt buffers: copy back
        cudaMemcpyAsync(keys, src, n * sizeof(KT), cudaMemcpyDeviceToDevice, st);
        if (HASV)
            cudaMemcpyAsync(vals, vs, n * 4, cudaMemcpyDeviceToDevice, st);
    }
    e = cudaGetLastError();
    cudaError_t e2 = own ? cudaFreeAsync(scr, st) : cudaSuccess;
    return e != cudaSuccess ? e : e2;
}

// Calls f.template operator()<KT, HASV, DB, TILE, NW>() for the configuration.
template <typename F> static cudaError_t oop_dispatch(int kb, int db, bool hasv, F &&f)
{
    using u64 = unsigned long long;
    if (kb == 4) {
        if (db == 8)
            return hasv ? f.template operator()<uint32_t, true, 8, 4096, 16>()
                        : f.template operator()<uint32_t, false, 8, 4096, 16>();
        return hasv ? f.template operator()<uint32_t, true, 11, 4096, 8>()
                    : f.template operator()<uint32_t, false, 11, 4096, 8>();
    }
    if (db == 8)
        return hasv ? f.template operator()<u64, true, 8, 4096, 16>()
                    : f.template operator()<u64, false, 8, 4096, 16>();
    return hasv ? f.template operator()<u64, true, 11, 4096, 8>()
                : f.template operator()<u64, false, 11, 4096, 8>();
}

size_t lsd_oop_scratch_bytes(size_t n, int kb, int db, bool hasv)
{
    size_t r = 0;
    oop_dispatch(kb, db, hasv, [&]<typename KT, bool HASV, int DB, int TILE, int NW>() {
        r = oop_scratch<KT, HASV, DB, TILE, NW>(n);
        return cudaSuccess;
    });
    return r;
}

cudaError_t launch_lsd_oop_ws(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                              size_t n, int kb, int db, void *scratch, cudaStream_t st)
{
    return oop_dispatch(kb, db, vals != nullptr, [&]<typename KT, bool HASV, int DB, int TILE, int NW>() {
        return oop_impl<KT, HASV, DB, TILE, NW>(static_cast<KT *>(keys), vals, static_cast<KT *>(keys_alt),
                                                vals_alt, n, scratch, st);
    });
}

cudaError_t launch_lsd_oop(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                           size_t n, int kb, int db, cudaStream_t st)
{
    return launch_lsd_oop_ws(keys, vals, keys_alt, vals_alt, n, kb, db, nullptr, st);
}

} // namespace rs
