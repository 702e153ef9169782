// Radsort Finalize for sm_103a, and the float32 key transform.
//
// Finalize applies pi to the data blocks in place (Alg. 7, Sec. 2.4): after
// the last round the used elements of logical blocks H .. f-1 (H = sigma*p)
// hold the sorted sequence, and they must end up contiguous in A.  Alg. 7
// does this one block at a time.  Here it is split into two parallel passes;
// the paper suggests such a split for its parallel variant (Sec. 4.3: a
// parallel permutation, then moving elements to remove the gaps of partial
// blocks).
//
// F1, block permutation.  Logical block q = i - H goes to its target
// position: A block q for q < floor(n/b), scratch block q - floor(n/b) for the
// rest (at most sigma*p of them, all in T).  The moving blocks form paths
// (ending at a free target) and cycles.
//   * Pointer jumping over "block at x moves to t" finds each cycle's minimum
//     (min-jumping).  The cycles are cut there.  A second jumping pass ranks
//     every position by its distance to the head of its chain (the path's free
//     end, or the cycle's minimum).
//   * Each chain gets a contiguous range of an order array from an atomic
//     counter.
//   * The order array is cut into strides of K positions that CTAs take in
//     ticket order.  A stride reads every block it must move into shared
//     memory and publishes a flag.  It waits (bounded) for the previous
//     stride's flag only if its first chain continues from there, then
//     writes.  A cycle that spans strides saves its head block to a slot
//     first.  The few beyond the slot capacity are moved by one CTA each.
// F2, gap removal.  With block q at its target, A[off_q + e] = block_q[e]
// moves every element left by the unused tails of the partial blocks before
// it.  Windows of W destination elements are taken in ticket order.  A window
// loads its sources, publishes, and waits only for the earlier windows whose
// sources overlap its destinations.
//
// Every wait has an iteration limit.  When it runs out, the kernel sets the
// status word and returns; it never hangs.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_finalize() { return take_status_word(); }

namespace {

constexpr uint32_t ABS = 0xFFFFFFFFu;      // absorbing jump entry
constexpr uint32_t POS_MASK = 0x0FFFFFFFu; // positions < 2^28
constexpr uint32_t F_MOVE = 1u << 31, F_CYC = 1u << 30, F_MIN = 1u << 29; // pi flags
constexpr uint32_t O_FIRST = 1u << 31, O_LAST = 1u << 30, O_CYC = 1u << 29, O_DEFER = 1u << 28;
constexpr uint32_t H_CYC = 1u << 31, H_HEAD = 1u << 30, H_DEFER = 1u << 29;
constexpr uint32_t H_LEN = (1u << 29) - 1;
constexpr uint32_t SLOT_NONE = 0xFFFFFFFFu;
constexpr int FIN_T = 256;
constexpr uint32_t MAXK = 64;

// counters (words of the finalize scratch)
enum { C_ORDER = 0, C_REC = 1, C_STRIDE = 2, C_WIN = 3, C_WORDS = 8 };

struct FinArgs {
    void *Ak;
    uint32_t *Av;
    void *Tk;
    uint32_t *Tv;
    uint32_t nT, nA, H, b, npi;
    unsigned long long n;
    uint32_t *pi;                // logical -> physical, later the order array
    unsigned long long *jump;    // npi entries
    const uint2 *P;              // partial blocks of the last round
    const unsigned long long *D; // deficit prefix over P (nP + 1 entries)
    const uint32_t *state;
    uint32_t *ctr;               // counters
    uint32_t *sflag;             // per stride: reads done
    uint32_t *wflag;             // per window: reads done
    uint4 *rec;                  // straddling cycles: (base, len, slot, 0)
    uint32_t nrec_cap;
    void *slot_k;                // nslots saved head blocks
    uint32_t *slot_v;
    uint32_t *slot_flag;         // per slot: head saved
    uint32_t nslots;
    uint32_t K;                  // stride length (blocks)
    uint32_t W;                  // window length (elements)
};

__device__ __forceinline__ unsigned long long pk(uint32_t a, uint32_t b)
{
    return (unsigned long long)a | ((unsigned long long)b << 32);
}
__device__ __forceinline__ uint32_t lo32(unsigned long long v) { return uint32_t(v); }
__device__ __forceinline__ uint32_t hi32(unsigned long long v) { return uint32_t(v >> 32); }

__device__ __forceinline__ unsigned long long ld64(const unsigned long long *p)
{
    return *(const volatile unsigned long long *)p;
}
__device__ __forceinline__ void st64(unsigned long long *p, unsigned long long v)
{
    *(volatile unsigned long long *)p = v;
}

__device__ __forceinline__ uint32_t target_of(uint32_t q, uint32_t nA, uint32_t nT)
{
    return q < nA ? nT + q : q - nA;
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t *p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(uint32_t *p, uint32_t v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// TMA bulk store shared -> global (bulk-group completion)
__device__ __forceinline__ void bulk_s2g(void *dst_gmem, const void *src_smem, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst_gmem),
                 "r"(smem_u32(src_smem)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the shared-memory sources of this thread's bulk stores have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// this thread's bulk stores are complete
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// bounded wait until *p != 0
__device__ __forceinline__ bool wait_flag(const uint32_t *p, unsigned limit = SPIN_LIMIT)
{
    for (unsigned it = 0; it < limit; ++it) {
        if (ld_acquire(p))
            return true;
        if ((it & 1023u) == 1023u && wait_failed())
            return false;
        __nanosleep(64);
    }
    set_status(ST_TIMEOUT);
    return false;
}

template <typename KT> __device__ __forceinline__ KT *kblk(const FinArgs &a, uint32_t j)
{
    return j < a.nT ? static_cast<KT *>(a.Tk) + size_t(j) * a.b
                    : static_cast<KT *>(a.Ak) + size_t(j - a.nT) * a.b;
}
__device__ __forceinline__ uint32_t *vblk(const FinArgs &a, uint32_t j)
{
    return j < a.nT ? a.Tv + size_t(j) * a.b : a.Av + size_t(j - a.nT) * a.b;
}

// ---------------------------------------------------------------- pointer jumping
__global__ void k_fz_reset(unsigned long long *jump, uint32_t npi)
{
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < npi; x += gridDim.x * blockDim.x)
        jump[x] = pk(x, ABS);
}

// successor edges of the moving blocks: (target, own position) for min-jumping
__global__ void k_fz_edges(FinArgs a)
{
    const uint32_t NL = a.state[ST_F] - a.H;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < NL; q += gridDim.x * blockDim.x) {
        const uint32_t x = a.pi[a.H + q], t = target_of(q, a.nA, a.nT);
        if (x != t)
            a.jump[x] = pk(t, x);
    }
}

// In-place pointer jumping.  Entry (nxt, val); val == ABS is absorbing.
// mode 0: val = minimum position of the window; mode 1: val = window length.
// Each thread only rewrites its own entry, and any neighbour value it reads
// is a valid window, so asynchronous updates only speed convergence.
constexpr int JUMP_STEPS = 3;

__global__ void k_fz_jump(unsigned long long *jump, uint32_t npi, int mode, uint32_t *changes,
                          int round)
{
    // once a round changed nothing the entries are final: later rounds exit
    if (round > 0 && *(volatile uint32_t *)&changes[round - 1] == 0)
        return;
    // JUMP_STEPS steps per launch: every entry always describes a valid
    // window (its end and the min / sum over it), so an entry read while its
    // owner updates it is a valid window too, and each step adds at least the
    // window every entry had when the launch began: windows grow at least
    // (JUMP_STEPS + 1)-fold per launch
    bool changed = false;
    for (int step = 0; step < JUMP_STEPS; ++step)
        for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < npi; x += gridDim.x * blockDim.x) {
            const unsigned long long e = ld64(&jump[x]);
            const uint32_t v = hi32(e);
            if (v == ABS)
                continue;
            const unsigned long long f = ld64(&jump[lo32(e)]);
            const uint32_t fv = hi32(f);
            if (fv == ABS)
                continue; // x's window already ends at an absorbing entry
            const unsigned long long ne = pk(lo32(f), mode == 0 ? min(v, fv) : v + fv);
            if (ne != e) {
                st64(&jump[x], ne);
                changed = true;
            }
        }
    if (__syncthreads_or(changed) && threadIdx.x == 0)
        atomicAdd(&changes[round], 1u);
}

// The same pointer jumping for a small permutation (n_pi <= FZ_SMALL_NPI):
// one CTA with the entries in shared memory, steps until one changes
// nothing (windows at least double each step, so 33 steps bound it), in one
// launch instead of one per (JUMP_STEPS + 1)-fold growth.
constexpr uint32_t FZ_SMALL_NPI = 12288;

__global__ void __launch_bounds__(1024) k_fz_jump_small(unsigned long long *jump, uint32_t npi, int mode)
{
    extern __shared__ unsigned long long sj[];
    for (uint32_t x = threadIdx.x; x < npi; x += blockDim.x)
        sj[x] = jump[x];
    __syncthreads();
    for (int step = 0; step < 34; ++step) {
        bool changed = false;
        for (uint32_t x = threadIdx.x; x < npi; x += blockDim.x) {
            const unsigned long long e = sj[x];
            const uint32_t v = hi32(e);
            if (v == ABS)
                continue;
            const uint32_t nx = lo32(e);
            if (nx >= npi)
                continue; // only a broken entry points out of the permutation
            const unsigned long long f = sj[nx];
            const uint32_t fv = hi32(f);
            if (fv == ABS)
                continue;
            const unsigned long long ne = pk(lo32(f), mode == 0 ? min(v, fv) : v + fv);
            if (ne != e) {
                sj[x] = ne;
                changed = true;
            }
        }
        if (!__syncthreads_or(changed))
            break;
    }
    for (uint32_t x = threadIdx.x; x < npi; x += blockDim.x)
        jump[x] = sj[x];
}

// classify each moving block in pi's top bits: moving / on a cycle / the
// cycle's minimum position
__global__ void k_fz_classify(FinArgs a)
{
    const uint32_t NL = a.state[ST_F] - a.H;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < NL; q += gridDim.x * blockDim.x) {
        const uint32_t x = a.pi[a.H + q], t = target_of(q, a.nA, a.nT);
        if (x == t)
            continue;
        const unsigned long long e = a.jump[x];
        const bool cyc = hi32(a.jump[lo32(e)]) != ABS;
        const bool mn = cyc && hi32(e) == x;
        a.pi[a.H + q] = x | F_MOVE | (cyc ? F_CYC : 0u) | (mn ? F_MIN : 0u);
    }
}

// rank-pass edges: every moving block except a cycle minimum points to its
// target with length 1; minima stay absorbing (the cycles are cut there)
__global__ void k_fz_rank_edges(FinArgs a)
{
    const uint32_t NL = a.state[ST_F] - a.H;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < NL; q += gridDim.x * blockDim.x) {
        const uint32_t v = a.pi[a.H + q];
        if (!(v & F_MOVE) || (v & F_MIN))
            continue;
        a.jump[v & POS_MASK] = pk(target_of(q, a.nA, a.nT), 1u);
    }
}

// each chain reserves its range of the order array (paths from their start,
// cycles from their minimum) and writes it into the head's entry:
// (base, length | HEAD | CYC | DEFER)
__global__ void k_fz_chains(FinArgs a)
{
    const uint32_t NL = a.state[ST_F] - a.H;
    const uint32_t R = NL - a.nA;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < NL; q += gridDim.x * blockDim.x) {
        const uint32_t v = a.pi[a.H + q];
        if (!(v & F_MOVE))
            continue;
        const uint32_t x = v & POS_MASK;
        const bool cyc = (v & F_CYC) != 0;
        uint32_t h, r;
        if (cyc) {
            // a cycle is cut at its minimum m (rank 0); m's successor is the
            // farthest from m, so its rank + 1 is the cycle length
            if (!(v & F_MIN))
                continue;
            h = x;
            r = hi32(a.jump[target_of(q, a.nA, a.nT)]);
        } else {
            // a path starts at a position no block moves into: a scratch
            // block past the R targets in T or, after a truncation (Alg. 8),
            // an A block at or past the first one that no block targets
            if (!((x < a.nT && x >= R) || x >= a.nT + a.nA))
                continue; // not a path start: some block moves into x
            const unsigned long long e = a.jump[x];
            h = lo32(e);
            r = hi32(e);
        }
        const uint32_t len = r + 1;
        const uint32_t base = atomicAdd(&a.ctr[C_ORDER], len);
        uint32_t defer = 0;
        if (cyc && base / a.K != (base + len - 1) / a.K) {
            const uint32_t ri = atomicAdd(&a.ctr[C_REC], 1u);
            if (ri < a.nrec_cap) {
                const uint32_t slot = ri < a.nslots ? ri : SLOT_NONE;
                a.rec[ri] = make_uint4(base, len, slot, 0);
                defer = slot == SLOT_NONE ? H_DEFER : 0u;
            } else {
                set_status(ST_INTERNAL);
            }
        }
        a.jump[h] = pk(base, len | H_HEAD | (cyc ? H_CYC : 0u) | defer);
    }
}

__global__ void k_fz_order(FinArgs a)
{
    for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < a.npi; x += gridDim.x * blockDim.x) {
        const unsigned long long e = a.jump[x];
        const uint32_t v = hi32(e);
        if (v == ABS)
            continue;
        uint32_t base, info, r;
        if (v & H_HEAD) {
            base = lo32(e);
            info = v;
            r = 0;
        } else {
            const unsigned long long hd = a.jump[lo32(e)];
            base = lo32(hd);
            info = hi32(hd);
            r = v;
        }
        const uint32_t len = info & H_LEN;
        a.pi[base + r] = x | (r == 0 ? O_FIRST : 0u) | (r + 1 == len ? O_LAST : 0u) |
                         ((info & H_CYC) ? O_CYC : 0u) | ((info & H_DEFER) ? O_DEFER : 0u);
    }
}

// record of the straddling cycle that contains order index g (linear search;
// straddling cycles are few: random-like permutations have O(log n) cycles)
__device__ uint4 find_rec(const FinArgs &a, uint32_t g)
{
    const uint32_t nr = min(a.ctr[C_REC], a.nrec_cap);
    for (uint32_t i = 0; i < nr; ++i) {
        const uint4 r = a.rec[i];
        if (g >= r.x && g < r.x + r.y)
            return r;
    }
    return make_uint4(0, 0, SLOT_NONE, 0);
}

// copy `cnt` blocks between block addresses (flat over all 16-byte vectors)
template <typename KT> struct BlockIO {
    const FinArgs &a;
    uint32_t kvec, vvec, nvec;
    __device__ BlockIO(const FinArgs &aa) : a(aa)
    {
        kvec = a.b * sizeof(KT) / 16;
        vvec = a.Av ? a.b * 4 / 16 : 0;
        nvec = kvec + vvec;
    }
    // smem buffer i <-> block j
    __device__ uint4 *sbuf(unsigned char *base, uint32_t i) const
    {
        return reinterpret_cast<uint4 *>(base) + size_t(i) * nvec;
    }
    __device__ uint4 *gvec(uint32_t j, uint32_t v) const
    {
        return v < kvec ? reinterpret_cast<uint4 *>(kblk<KT>(a, j)) + v
                        : reinterpret_cast<uint4 *>(vblk(a, j)) + (v - kvec);
    }
    __device__ uint4 *slotvec(uint32_t s, uint32_t v) const
    {
        return v < kvec ? reinterpret_cast<uint4 *>(static_cast<KT *>(a.slot_k) + size_t(s) * a.b) + v
                        : reinterpret_cast<uint4 *>(a.slot_v + size_t(s) * a.b) + (v - kvec);
    }
};

// ---------------------------------------------------------------- F1 moves
// kinds: 0 nothing, 1 block src -> dst, 2 closing write of a cycle from its slot
template <typename KT>
__global__ void __launch_bounds__(FIN_T) k_fz_move(FinArgs a)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    __shared__ uint32_t s_ticket, s_src[MAXK], s_dst[MAXK], s_kind[MAXK], s_slot[MAXK], s_save[MAXK];
    __shared__ uint32_t s_wait, s_bytes;
    __shared__ __align__(8) uint64_t s_bar;
    const BlockIO<KT> io(a);
    const uint32_t total = a.ctr[C_ORDER];
    const uint32_t nstr = (total + a.K - 1) / a.K;
    const uint32_t kbytes = a.b * sizeof(KT), vbytes = a.Av ? a.b * 4 : 0;
    const uint32_t bbytes = kbytes + vbytes;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    for (;;) {
        if (threadIdx.x == 0)
            s_ticket = atomicAdd(&a.ctr[C_STRIDE], 1u);
        __syncthreads();
        const uint32_t t = s_ticket;
        if (t >= nstr)
            break;
        const uint32_t g0 = t * a.K, g1 = min(total, g0 + a.K), cnt = g1 - g0;
        if (threadIdx.x < cnt) {
            const uint32_t i = threadIdx.x, g = g0 + i;
            const uint32_t o = a.pi[g];
            uint32_t kind = 0, src = 0, slot = SLOT_NONE, save = SLOT_NONE;
            if (o & O_DEFER) {
                kind = 0; // the whole cycle is moved by k_fz_move_deferred
            } else if (o & O_LAST) {
                if (o & O_CYC) {
                    const uint4 r = find_rec(a, g);
                    if (r.y) { // head in an earlier stride: its block waits in a slot
                        kind = 2;
                        slot = r.z;
                    } else {   // head in this stride
                        uint32_t gh = g;
                        while (gh > g0 && !(a.pi[gh] & O_FIRST))
                            --gh;
                        kind = 1;
                        src = a.pi[gh] & POS_MASK;
                    }
                } // a path's start receives nothing
            } else {
                kind = 1;
                src = a.pi[g + 1] & POS_MASK;
                if ((o & O_FIRST) && (o & O_CYC)) {
                    const uint4 r = find_rec(a, g);
                    if (r.y)
                        save = r.z; // save the head block before it is overwritten
                }
            }
            s_kind[i] = kind;
            s_src[i] = src;
            s_dst[i] = o & POS_MASK;
            s_slot[i] = slot;
            s_save[i] = save;
        }
        if (threadIdx.x == 0) {
            const uint32_t o = a.pi[g0];
            s_wait = (t > 0 && !(o & O_FIRST) && !(o & O_DEFER)) ? 1u : 0u;
        }
        __syncthreads();
        // read phase: every source block into shared memory by TMA bulk
        // copies (warp 0, one entry per lane); heads of straddling cycles to
        // their slots with plain copies
        if (threadIdx.x < 32) {
            const uint32_t i = threadIdx.x;
            const bool mv = i < cnt && s_kind[i] == 1;
            const uint32_t tot = warp_sum(mv ? bbytes : 0u);
            if (i == 0)
                s_bytes = tot;
            if (i == 0 && tot)
                mbar_arrive_expect_tx(&s_bar, tot);
            __syncwarp();
            if (mv) {
                unsigned char *buf = fsm + size_t(i) * bbytes;
                bulk_g2s(buf, kblk<KT>(a, s_src[i]), kbytes, &s_bar);
                if (vbytes)
                    bulk_g2s(buf + kbytes, vblk(a, s_src[i]), vbytes, &s_bar);
            }
        }
        for (uint32_t i = 0; i < cnt; ++i)
            if (s_save[i] != SLOT_NONE)
                for (uint32_t v = threadIdx.x; v < io.nvec; v += blockDim.x)
                    *io.slotvec(s_save[i], v) = *io.gvec(s_dst[i], v);
        __syncthreads();
        if (s_bytes) {
            mbar_wait(&s_bar, phase);
            phase ^= 1u;
        }
        if (threadIdx.x == 0) {
            __threadfence();
            for (uint32_t i = 0; i < cnt; ++i)
                if (s_save[i] != SLOT_NONE)
                    st_release(&a.slot_flag[s_save[i]], 1u);
            st_release(&a.sflag[t], 1u);
            if (s_wait)
                wait_flag(&a.sflag[t - 1]);
            for (uint32_t i = 0; i < cnt; ++i)
                if (s_kind[i] == 2)
                    wait_flag(&a.slot_flag[s_slot[i]]);
        }
        __syncthreads();
        // write phase: bulk stores from shared memory; closing writes from slots
        if (threadIdx.x < 32) {
            const uint32_t i = threadIdx.x;
            if (i < cnt && s_kind[i] == 1) {
                const unsigned char *buf = fsm + size_t(i) * bbytes;
                bulk_s2g(kblk<KT>(a, s_dst[i]), buf, kbytes);
                if (vbytes)
                    bulk_s2g(vblk(a, s_dst[i]), buf + kbytes, vbytes);
            }
            bulk_commit();
        }
        for (uint32_t i = 0; i < cnt; ++i)
            if (s_kind[i] == 2)
                for (uint32_t v = threadIdx.x; v < io.nvec; v += blockDim.x)
                    *io.gvec(s_dst[i], v) = *io.slotvec(s_slot[i], v);
        if (threadIdx.x < 32)
            bulk_wait_read(); // shared buffers free for the next stride
        __syncthreads();
    }
    if (threadIdx.x < 32)
        bulk_wait_all();
}

// straddling cycles beyond the slot capacity: one CTA moves a whole cycle,
// K-1 blocks at a time, holding the head block in shared memory
template <typename KT>
__global__ void __launch_bounds__(FIN_T) k_fz_move_deferred(FinArgs a)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    const BlockIO<KT> io(a);
    const uint32_t nr = min(a.ctr[C_REC], a.nrec_cap);
    const uint32_t KB = a.K - 1;
    for (uint32_t ri = blockIdx.x; ri < nr; ri += gridDim.x) {
        const uint4 r = a.rec[ri];
        if (r.z != SLOT_NONE)
            continue;
        const uint32_t g0 = r.x, len = r.y;
        const uint32_t yh = a.pi[g0] & POS_MASK;
        for (uint32_t v = threadIdx.x; v < io.nvec; v += blockDim.x)
            io.sbuf(fsm, 0)[v] = *io.gvec(yh, v);
        __syncthreads();
        // y_g <- content(y_{g+1}) for g = g0 .. g0+len-2, then y_last <- head
        for (uint32_t g = g0; g + 1 < g0 + len; g += KB) {
            const uint32_t c = min(KB, g0 + len - 1 - g);
            for (uint32_t idx = threadIdx.x; idx < c * io.nvec; idx += blockDim.x) {
                const uint32_t i = idx / io.nvec, v = idx - i * io.nvec;
                io.sbuf(fsm, 1 + i)[v] = *io.gvec(a.pi[g + 1 + i] & POS_MASK, v);
            }
            __syncthreads();
            for (uint32_t idx = threadIdx.x; idx < c * io.nvec; idx += blockDim.x) {
                const uint32_t i = idx / io.nvec, v = idx - i * io.nvec;
                *io.gvec(a.pi[g + i] & POS_MASK, v) = io.sbuf(fsm, 1 + i)[v];
            }
            __syncthreads();
        }
        const uint32_t yl = a.pi[g0 + len - 1] & POS_MASK;
        for (uint32_t v = threadIdx.x; v < io.nvec; v += blockDim.x)
            *io.gvec(yl, v) = io.sbuf(fsm, 0)[v];
        __syncthreads();
    }
}

// ---------------------------------------------------------------- F2 gap removal
// first element position and length of logical block q (0-based), and the
// number of partial blocks before it
__device__ __forceinline__ void block_span(const FinArgs &a, uint32_t nP, uint32_t q,
                                           unsigned long long &off, uint32_t &len, uint32_t &jP)
{
    uint32_t l = 0, r = nP;
    while (l < r) {
        const uint32_t m = (l + r) >> 1;
        if (a.P[m].x < a.H + q)
            l = m + 1;
        else
            r = m;
    }
    jP = l;
    off = (unsigned long long)q * a.b - a.D[l];
    len = (l < nP && a.P[l].x == a.H + q) ? a.P[l].y : a.b;
}

// logical block holding element x (a non-empty one) and the number of
// partial blocks before it.  Partial j (logical q_j) spans [off_j, end_j)
// with off_j = q_j*b - D[j]; the blocks between partials are full.
__device__ __forceinline__ void block_of(const FinArgs &a, uint32_t nP, unsigned long long x,
                                         uint32_t &q, uint32_t &jp)
{
    uint32_t l = 0, r = nP; // J = first partial with end_J > x
    while (l < r) {
        const uint32_t m = (l + r) >> 1;
        const uint2 pm = a.P[m];
        const unsigned long long end = (unsigned long long)(pm.x - a.H) * a.b - a.D[m] + pm.y;
        if (end <= x)
            l = m + 1;
        else
            r = m;
    }
    jp = l;
    if (l < nP) {
        const uint2 pl = a.P[l];
        const unsigned long long off = (unsigned long long)(pl.x - a.H) * a.b - a.D[l];
        if (off <= x) {
            q = pl.x - a.H;
            return;
        }
    }
    if (l == 0) {
        q = static_cast<uint32_t>(x / a.b);
        return;
    }
    const uint2 pp = a.P[l - 1];
    const unsigned long long endp = (unsigned long long)(pp.x - a.H) * a.b - a.D[l - 1] + pp.y;
    q = pp.x - a.H + 1 + static_cast<uint32_t>((x - endp) / a.b);
}

// number of partial blocks with logical index < H + q
__device__ __forceinline__ uint32_t partials_before(const FinArgs &a, uint32_t nP, uint32_t q)
{
    uint32_t l = 0, r = nP;
    while (l < r) {
        const uint32_t m = (l + r) >> 1;
        if (a.P[m].x < a.H + q)
            l = m + 1;
        else
            r = m;
    }
    return l;
}

// Per window: first source block and the partials before it, the earliest
// window that reads from this window's destinations, whether it is in place,
// and up to MAXSEG runs of constant shift (between partial blocks the source
// of destination x is x + D, in A, or x + D - nA*b in T).
constexpr int MAXSEG = 4;
enum { WP_INPLACE = 1u, WP_SEGS = 2u };

__global__ void k_fz_winplan(FinArgs a, uint4 *plan, uint4 *segs)
{
    const uint32_t nP = a.state[ST_NP];
    const unsigned long long n = a.n;
    const uint32_t nwin = static_cast<uint32_t>((n + a.W - 1) / a.W);
    for (uint32_t w = blockIdx.x * blockDim.x + threadIdx.x; w < nwin; w += gridDim.x * blockDim.x) {
        const unsigned long long x0 = (unsigned long long)w * a.W;
        const uint32_t cnt = static_cast<uint32_t>(min((unsigned long long)a.W, n - x0));
        uint32_t q0, jp0, qe, jpe;
        block_of(a, nP, x0, q0, jp0);
        block_of(a, nP, x0 + cnt - 1, qe, jpe);
        // in place iff no partial block precedes the last block and it is in
        // A: every source is then its own destination
        uint32_t flags = (qe < a.nA && a.D[jpe] == 0) ? WP_INPLACE : 0u;
        // the destination of the element at virtual position x0 is the
        // smallest destination among sources inside [x0, x0 + W)
        const uint32_t qv = static_cast<uint32_t>(x0 / a.b);
        uint32_t wlo = w; // destinations beyond A's blocks: nobody reads them
        if (qv < a.nA) {
            const uint32_t j = partials_before(a, nP, qv);
            const unsigned long long offv = (unsigned long long)qv * a.b - a.D[j];
            wlo = static_cast<uint32_t>(offv / a.W);
        }
        // constant-shift runs
        const unsigned long long end = x0 + cnt, nAb = (unsigned long long)a.nA * a.b;
        unsigned long long x = x0;
        uint32_t k = 0;
        while (x < end && k < MAXSEG) {
            uint32_t q, jp;
            block_of(a, nP, x, q, jp);
            const unsigned long long g = a.D[jp];
            unsigned long long se = end;
            bool part_after_A = true;
            if (jp < nP) {
                const uint2 pj = a.P[jp];
                const unsigned long long endp = (unsigned long long)(pj.x - a.H) * a.b - g + pj.y;
                se = min(se, endp);
                part_after_A = pj.x - a.H >= a.nA;
            }
            const bool inT = q >= a.nA;
            if (!inT && part_after_A)
                se = min(se, nAb - g); // the run of A blocks ends at block nA
            const unsigned long long src = x + g - (inT ? nAb : 0ull);
            segs[size_t(w) * MAXSEG + k] =
                make_uint4(static_cast<uint32_t>(x - x0), static_cast<uint32_t>(se - x),
                           static_cast<uint32_t>(src), static_cast<uint32_t>(src >> 32) | (inT ? 0x80000000u : 0u));
            x = se;
            ++k;
        }
        if (x >= end)
            flags |= WP_SEGS | (k << 8);
        plan[w] = make_uint4(q0, jp0, wlo, flags);
    }
}

template <typename KT>
__global__ void __launch_bounds__(FIN_T) k_fz_compact(FinArgs a, const uint4 *plan, const uint4 *segs)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    // keys: W elements plus 16 bytes of slack per run; values likewise
    constexpr uint32_t KA = 16 / sizeof(KT); // elements per 16 bytes
    // each run's 16-byte-aligned superset adds at most 2*KA-2 elements
    const uint32_t kcap = a.W + 2 * KA * (MAXSEG + 1), vcap = a.W + 8 * (MAXSEG + 1);
    KT *wk = reinterpret_cast<KT *>(fsm);
    uint32_t *wv = reinterpret_cast<uint32_t *>(fsm + ((size_t(kcap) * sizeof(KT) + 15) & ~size_t(15)));
    __shared__ uint32_t s_ticket;
    __shared__ uint4 s_plan;
    __shared__ uint32_t s_kb[MAXSEG], s_vb[MAXSEG]; // smem start of each run (incl. lead)
    __shared__ __align__(8) uint64_t s_bar;
    if (threadIdx.x == 0) {
        mbar_init(&s_bar, 1);
        fence_mbar_init();
    }
    __syncthreads();
    uint32_t phase = 0;
    const uint32_t nP = a.state[ST_NP];
    const uint32_t NL = a.state[ST_F] - a.H;
    const unsigned long long n = a.n;
    const uint32_t nwin = static_cast<uint32_t>((n + a.W - 1) / a.W);
    const bool hv = a.Av != nullptr;
    KT *Ak = static_cast<KT *>(a.Ak);
    for (;;) {
        if (threadIdx.x == 0) {
            const uint32_t t = atomicAdd(&a.ctr[C_WIN], 1u);
            s_ticket = t;
            if (t < nwin)
                s_plan = plan[t];
        }
        __syncthreads();
        const uint32_t w = s_ticket;
        if (w >= nwin)
            break;
        const uint4 pl = s_plan;
        __syncthreads(); // everyone has read s_ticket before it is reused below
        const unsigned long long x0 = (unsigned long long)w * a.W;
        const uint32_t cnt = static_cast<uint32_t>(min((unsigned long long)a.W, n - x0));
        const bool inplace = (pl.w & WP_INPLACE) != 0;
        const bool segmode = !inplace && (pl.w & WP_SEGS);
        const uint32_t nseg = segmode ? (pl.w >> 8) & 0xFF : 0u;
        if (segmode) {
            // constant-shift runs: one TMA bulk load per run (keys, values) of
            // the 16-byte-aligned superset of its source; the lead is skipped
            // when writing.  The superset stays inside its region of A or T,
            // whose ends are multiples of the block size.
            if (threadIdx.x == 0) {
                uint32_t kpos = 0, vpos = 0, bytes = 0;
                uint32_t kb[MAXSEG], vb[MAXSEG];
                unsigned long long ks0[MAXSEG], vs0[MAXSEG];
                uint32_t kn[MAXSEG], vn[MAXSEG];
                bool kt[MAXSEG];
                for (uint32_t k = 0; k < nseg; ++k) {
                    const uint4 sg = segs[size_t(w) * MAXSEG + k];
                    const unsigned long long src = sg.z | ((unsigned long long)(sg.w & 0x7FFFFFFFu) << 32);
                    kt[k] = (sg.w & 0x80000000u) != 0;
                    ks0[k] = src & ~(unsigned long long)(KA - 1);
                    const uint32_t klead = static_cast<uint32_t>(src - ks0[k]);
                    kn[k] = (klead + sg.y + KA - 1) & ~(KA - 1);
                    kb[k] = kpos;
                    s_kb[k] = kpos + klead;
                    kpos += kn[k];
                    bytes += kn[k] * sizeof(KT);
                    if (hv) {
                        vs0[k] = src & ~3ull;
                        const uint32_t vlead = static_cast<uint32_t>(src - vs0[k]);
                        vn[k] = (vlead + sg.y + 3) & ~3u;
                        vb[k] = vpos;
                        s_vb[k] = vpos + vlead;
                        vpos += vn[k];
                        bytes += vn[k] * 4;
                    }
                }
                if (bytes) {
                    mbar_arrive_expect_tx(&s_bar, bytes);
                    for (uint32_t k = 0; k < nseg; ++k) {
                        const KT *sk = (kt[k] ? static_cast<const KT *>(a.Tk) : static_cast<const KT *>(a.Ak)) + ks0[k];
                        if (kn[k])
                            bulk_g2s(wk + kb[k], sk, kn[k] * sizeof(KT), &s_bar);
                        if (hv && vn[k])
                            bulk_g2s(wv + vb[k], (kt[k] ? a.Tv : a.Av) + vs0[k], vn[k] * 4, &s_bar);
                    }
                }
                s_ticket = bytes; // reuse: nonzero when a phase was armed
            }
            __syncthreads();
            if (s_ticket) {
                mbar_wait(&s_bar, phase);
                phase ^= 1u;
            }
        } else if (!inplace) {
            // read phase: the blocks covering destinations [x0, x0+cnt)
            uint32_t q = pl.x, jp = pl.y;
            unsigned long long off = (unsigned long long)q * a.b - a.D[jp];
            uint32_t len = (jp < nP && a.P[jp].x == a.H + q) ? a.P[jp].y : a.b;
            uint32_t done = 0;
            while (done < cnt && q < NL) {
                const uint32_t e0 = static_cast<uint32_t>(x0 + done - off);
                const uint32_t take = min(cnt - done, len > e0 ? len - e0 : 0u);
                if (take) {
                    const uint32_t phys = target_of(q, a.nA, a.nT);
                    const KT *sk = kblk<KT>(a, phys) + e0;
                    for (uint32_t i = threadIdx.x; i < take; i += blockDim.x)
                        wk[done + i] = sk[i];
                    if (hv) {
                        const uint32_t *sv = vblk(a, phys) + e0;
                        for (uint32_t i = threadIdx.x; i < take; i += blockDim.x)
                            wv[done + i] = sv[i];
                    }
                    done += take;
                }
                off += len;
                ++q;
                while (jp < nP && a.P[jp].x < a.H + q)
                    ++jp;
                len = (jp < nP && a.P[jp].x == a.H + q) ? a.P[jp].y : a.b;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            st_release(&a.wflag[w], 1u);
        }
        if (!inplace) {
            // wait for every earlier window that reads from our destinations
            for (uint32_t v = pl.z + threadIdx.x; v < w; v += blockDim.x)
                wait_flag(&a.wflag[v]);
            __syncthreads();
            if (segmode) {
                for (uint32_t k = 0; k < nseg; ++k) {
                    const uint4 sg = segs[size_t(w) * MAXSEG + k];
                    const KT *sk = wk + s_kb[k];
                    KT *dk = Ak + x0 + sg.x;
#pragma unroll 4
                    for (uint32_t i = threadIdx.x; i < sg.y; i += blockDim.x)
                        dk[i] = sk[i];
                    if (hv) {
                        const uint32_t *sv = wv + s_vb[k];
                        uint32_t *dv = a.Av + x0 + sg.x;
#pragma unroll 4
                        for (uint32_t i = threadIdx.x; i < sg.y; i += blockDim.x)
                            dv[i] = sv[i];
                    }
                }
            } else {
                for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) {
                    Ak[x0 + i] = wk[i];
                    if (hv)
                        a.Av[x0 + i] = wv[i];
                }
            }
        }
        // wk / wv were accessed with generic loads and stores; the next
        // window may refill them with bulk copies (async proxy)
        fence_proxy_async_smem();
        __syncthreads();
    }
}

// grid layout: the tail block (logical nA) was moved to scratch block 0
template <typename KT> __global__ void k_fz_tail(FinArgs a, uint32_t tail)
{
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= tail)
        return;
    const size_t dst = size_t(a.nA) * a.b + j;
    static_cast<KT *>(a.Ak)[dst] = kblk<KT>(a, 0)[j];
    if (a.Av)
        a.Av[dst] = vblk(a, 0)[j];
}

struct FinLayout {
    size_t ctr, sflag, wflag, slotflag, rec, wplan, wsegs, slotk, slotv, total;
    uint32_t K, W, nstr, nwin, nrec, nslots;
};

FinLayout fin_layout(const Geom &g)
{
    FinLayout L{};
    const size_t bbytes = size_t(g.b) * (g.kb + (g.hasv ? 4 : 0));
    // strides of 64 KB: three CTAs per SM keep enough bytes in flight, and
    // each stride's ticket, classification and flag waits are paid per 64 KB
    // (measured at 2^28, b = 2048: Finalize 1.02 ms with 32 KB, 0.98 ms with
    // 64 or 96 KB)
    uint32_t K = static_cast<uint32_t>((64u << 10) / bbytes);
    if (K > 32)
        K = 32; // one warp issues the bulk copies, one entry per lane
    if (K < 2)
        K = 2;
    L.K = K;
    L.W = g.kb == 4 ? 8192 : 4096;
    L.nstr = g.npi / K + 2;
    L.nwin = g.grid ? 0u : static_cast<uint32_t>(g.n / L.W + 2); // windows of F2 (chunk layout only)
    L.nrec = L.nstr + 1;
    // slots for cycles that span strides: a handful in practice; the rest are
    // moved by one CTA each, so small sorts keep a small workspace
    L.nslots = g.npi / 64 < 16 ? 16 : (g.npi / 64 > 1024 ? 1024 : g.npi / 64);
    auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
    size_t off = 0;
    L.ctr = off;
    off += al((C_WORDS + 128) * 4); // counters, then the jump rounds' change counts
    L.sflag = off;
    off += al(size_t(L.nstr) * 4);
    L.wflag = off;
    off += al(size_t(L.nwin) * 4);
    L.slotflag = off;
    off += al(size_t(L.nslots) * 4);
    L.rec = off; // everything before here is cleared per sort
    off += al(size_t(L.nrec) * 16);
    L.wplan = off;
    off += al(size_t(L.nwin) * 16);
    L.wsegs = off;
    off += al(size_t(L.nwin) * 16 * MAXSEG);
    L.slotk = off;
    off += al(size_t(L.nslots) * g.b * g.kb);
    L.slotv = off;
    off += g.hasv ? al(size_t(L.nslots) * g.b * 4) : 0;
    L.total = off;
    return L;
}

template <typename KT>
cudaError_t fin_impl(const Geom &g, const Bufs &w, uint32_t *pi, unsigned long long *jump,
                     cudaStream_t st)
{
    const FinLayout L = fin_layout(g);
    char *base = static_cast<char *>(w.fin);
    FinArgs a{};
    a.Ak = w.Ak;
    a.Av = g.hasv ? w.Av : nullptr;
    a.Tk = w.Tk;
    a.Tv = w.Tv;
    a.nT = g.nT;
    a.nA = g.nA;
    a.H = g.H;
    a.b = g.b;
    a.npi = g.npi;
    a.n = g.n;
    a.pi = pi;
    a.jump = jump;
    a.P = w.P;
    a.D = w.E;
    a.state = w.state;
    a.ctr = reinterpret_cast<uint32_t *>(base + L.ctr);
    a.sflag = reinterpret_cast<uint32_t *>(base + L.sflag);
    a.wflag = reinterpret_cast<uint32_t *>(base + L.wflag);
    a.slot_flag = reinterpret_cast<uint32_t *>(base + L.slotflag);
    a.rec = reinterpret_cast<uint4 *>(base + L.rec);
    a.nrec_cap = L.nrec;
    a.slot_k = base + L.slotk;
    a.slot_v = g.hasv ? reinterpret_cast<uint32_t *>(base + L.slotv) : nullptr;
    a.nslots = L.nslots;
    a.K = L.K;
    a.W = L.W;

    cudaError_t e = cudaMemsetAsync(base, 0, L.rec, st);
    if (e != cudaSuccess)
        return e;
    if (!g.grid) {
        e = launch_deficit(g, w, st); // D over the last round's P, used by F2
        if (e != cudaSuccess)
            return e;
    }
    const int sms = num_sms();
    int grid = static_cast<int>((g.npi + FIN_T - 1) / FIN_T);
    if (grid > sms * 8)
        grid = sms * 8;
    if (grid < 1)
        grid = 1;
    // launches until every window reaches n_pi (growth (JUMP_STEPS+1)-fold
    // each), plus one that sees no change
    int rounds = 1;
    for (unsigned long long w = JUMP_STEPS + 1; w < g.npi; w *= JUMP_STEPS + 1)
        ++rounds;
    rounds += 1;
    static DeviceOnce jattr;
    const cudaError_t ej = jattr.run([] {
        return cudaFuncSetAttribute(k_fz_jump_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    int(FZ_SMALL_NPI * 8));
    });
    if (ej != cudaSuccess)
        return ej;
    const bool small = g.npi <= FZ_SMALL_NPI;
    k_fz_reset<<<grid, FIN_T, 0, st>>>(a.jump, g.npi);
    k_fz_edges<<<grid, FIN_T, 0, st>>>(a);
    uint32_t *chg = a.ctr + C_WORDS; // per-round change counters (cleared with the flags)
    if (small)
        k_fz_jump_small<<<1, 1024, size_t(g.npi) * 8, st>>>(a.jump, g.npi, 0);
    else
        for (int r = 0; r < rounds; ++r)
            k_fz_jump<<<grid, FIN_T, 0, st>>>(a.jump, g.npi, 0, chg, r);
    k_fz_classify<<<grid, FIN_T, 0, st>>>(a);
    k_fz_reset<<<grid, FIN_T, 0, st>>>(a.jump, g.npi);
    k_fz_rank_edges<<<grid, FIN_T, 0, st>>>(a);
    if (small)
        k_fz_jump_small<<<1, 1024, size_t(g.npi) * 8, st>>>(a.jump, g.npi, 1);
    else
        for (int r = 0; r < rounds; ++r)
            k_fz_jump<<<grid, FIN_T, 0, st>>>(a.jump, g.npi, 1, chg + 64, r);
    k_fz_chains<<<grid, FIN_T, 0, st>>>(a);
    k_fz_order<<<grid, FIN_T, 0, st>>>(a);
    const size_t bbytes = size_t(g.b) * (g.kb + (g.hasv ? 4 : 0));
    const size_t msm = bbytes * L.K;
    const size_t kcap = L.W + 2 * (16 / g.kb) * (MAXSEG + 1), vcap = L.W + 8 * (MAXSEG + 1);
    const size_t csm = ((kcap * g.kb + 15) & ~size_t(15)) + (g.hasv ? vcap * 4 : 0);
    static DeviceOnce attr;
    const cudaError_t ea = attr.run([] {
        cudaError_t e = cudaFuncSetAttribute(k_fz_move<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 160 << 10);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fz_move_deferred<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     160 << 10);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(k_fz_compact<KT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     160 << 10);
        return e;
    });
    if (ea != cudaSuccess)
        return ea;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fz_move<KT>, FIN_T, msm);
    k_fz_move<KT><<<sms * (per_sm > 0 ? per_sm : 1), FIN_T, msm, st>>>(a);
    k_fz_move_deferred<KT><<<sms, FIN_T, msm, st>>>(a);
    if (g.grid) {
        // every block but the last is full: only the tail (now in scratch
        // block 0) remains to be copied behind A's last block
        const uint32_t tail = static_cast<uint32_t>(g.n - size_t(g.nA) * g.b);
        if (tail)
            k_fz_tail<KT><<<(tail + FIN_T - 1) / FIN_T, FIN_T, 0, st>>>(a, tail);
        g_launches += 10 + 2 * (small ? 1 : rounds);
        return cudaGetLastError();
    }
    uint4 *wplan = reinterpret_cast<uint4 *>(base + L.wplan);
    uint4 *wsegs = reinterpret_cast<uint4 *>(base + L.wsegs);
    k_fz_winplan<<<(L.nwin + FIN_T - 1) / FIN_T, FIN_T, 0, st>>>(a, wplan, wsegs);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fz_compact<KT>, FIN_T, csm);
    k_fz_compact<KT><<<sms * (per_sm > 0 ? per_sm : 1), FIN_T, csm, st>>>(a, wplan, wsegs);
    g_launches += 11 + 2 * (small ? 1 : rounds);
    return cudaGetLastError();
}

} // namespace

size_t finalize_extra_bytes(const Geom &g) { return fin_layout(g).total; }

cudaError_t launch_finalize(const Geom &g, const Bufs &w, uint32_t *pi, unsigned long long *jump,
                            cudaStream_t st)
{
    if (g.kb == 4)
        return fin_impl<uint32_t>(g, w, pi, jump, st);
    return fin_impl<unsigned long long>(g, w, pi, jump, st);
}

// ---------------------------------------------------------------- float keys
// IEEE float32 bits -> unsigned-orderable bits: flip the sign bit of
// non-negative values and every bit of negative ones (and back).
__global__ void k_float_keys(uint32_t *u, size_t n, int inverse)
{
    const size_t stride = size_t(gridDim.x) * blockDim.x;
    for (size_t i = size_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t x = u[i];
        const bool top = (x & 0x80000000u) != 0;
        u[i] = inverse ? (x ^ (top ? 0x80000000u : 0xFFFFFFFFu))
                       : (x ^ (top ? 0xFFFFFFFFu : 0x80000000u));
    }
}

// One thread waits for *flag like the stride and slot waits above, with at
// most `limit` polls; a flag that stays 0 makes the wait run out and records
// ST_TIMEOUT (the failure path, exercised without a fault or a hang)
__global__ void k_wait_probe(const uint32_t *flag, unsigned limit)
{
    if (threadIdx.x == 0)
        (void)wait_flag(flag, limit);
}

unsigned wait_spin_limit() { return SPIN_LIMIT; }

cudaError_t launch_wait_probe(const uint32_t *flag, unsigned limit, cudaStream_t st)
{
    k_wait_probe<<<1, 32, 0, st>>>(flag, limit);
    g_launches += 1;
    return cudaGetLastError();
}

cudaError_t launch_float_keys(uint32_t *keys, size_t n, int inverse, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    int blocks = static_cast<int>((n + 1023) / 1024);
    const int cap = num_sms() * 8;
    if (blocks > cap)
        blocks = cap;
    k_float_keys<<<blocks, 256, 0, st>>>(keys, n, inverse);
    g_launches += 1;
    return cudaGetLastError();
}

} // namespace rs
