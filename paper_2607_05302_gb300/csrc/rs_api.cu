// C ABI of the Radsort library (include/radsort.h): argument checks, the
// planner (block size b and chunk count p), the workspace layout, and the
// stream-ordered sequence setup -> n_t x (sortPhase, fixupPhase) -> Finalize
// (Alg. 2).  Nothing here touches element data; every step runs in the
// kernels of rs_round.cu and rs_finalize.cu.
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <vector>

#include "radsort.h"
#include "rs_kernels.cuh"

namespace rs {
// the failure-path probe (csrc/rs_finalize.cu)
cudaError_t launch_wait_probe(const uint32_t *flag, unsigned limit, cudaStream_t st);
unsigned wait_spin_limit();
} // namespace rs

namespace rs {

std::atomic<unsigned long long> g_launches{0};

// ---------------------------------------------------------------- tracing
namespace {
struct TraceRec {
    cudaEvent_t a, b;
    int phase, round;
};
std::mutex g_tmu;
std::vector<TraceRec> g_trace;
std::vector<cudaEvent_t> g_pool;
bool g_trace_on = false;

cudaEvent_t take_event()
{
    if (!g_pool.empty()) {
        cudaEvent_t e = g_pool.back();
        g_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Records an event pair around a scope on `st` while tracing is enabled.
struct Scope {
    TraceRec r{};
    cudaStream_t st;
    bool on;
    Scope(int phase, int round, cudaStream_t s) : st(s)
    {
        std::lock_guard<std::mutex> lk(g_tmu);
        on = g_trace_on;
        if (on) {
            r.a = take_event();
            r.b = take_event();
            r.phase = phase;
            r.round = round;
            cudaEventRecord(r.a, st);
        }
    }
    ~Scope()
    {
        if (!on)
            return;
        cudaEventRecord(r.b, st);
        std::lock_guard<std::mutex> lk(g_tmu);
        g_trace.push_back(r);
    }
};
} // namespace

// SM count of the current device (cached per device ordinal)
int num_sms()
{
    static std::atomic<int> cache[MAX_DEVICES] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES)
        dev = -1;
    if (dev >= 0) {
        const int c = cache[dev].load(std::memory_order_relaxed);
        if (c > 0)
            return c;
    }
    int sms = 0;
    if (dev < 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        sms <= 0)
        return 152;
    cache[dev].store(sms, std::memory_order_relaxed);
    return sms;
}

int current_device()
{
    int dev = 0;
    return cudaGetDevice(&dev) == cudaSuccess ? dev : -1;
}

static size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

static bool pow2(uint32_t x) { return x && !(x & (x - 1)); }

static uint32_t ilog2(uint32_t x)
{
    uint32_t r = 0;
    while ((1u << r) < x)
        ++r;
    return r;
}

static size_t layout(const Geom &g, void *base, Bufs *w);

// Geometry of a sort with block size b and p chunks (no planning).
static radsort_status fill_geom(size_t n, int kb, bool hasv, int db, uint32_t b, uint32_t p,
                                Geom *g)
{
    if (!pow2(b) || b < 64 || b > 4096 || p < 1 || p > 65536)
        return RADSORT_EINVAL;
    g->n = n;
    g->kb = kb;
    g->hasv = hasv;
    g->db = db;
    g->sigma = 1u << db;
    g->nt = (8 * kb + db - 1) / db;
    g->b = b;
    g->lb = ilog2(b);
    g->p = p;
    const unsigned long long nA = n / b;
    const unsigned long long H = (unsigned long long)g->sigma * p;
    const unsigned long long npi = nA + 2 * H;
    if (npi >= (1ull << 28))
        return RADSORT_EINVAL; // 32-bit block indices with four flag bits to spare
    // sequence number of a block in its chunk's bucket chain: < 2^(32-db)
    if ((unsigned long long)g->sigma + npi >= (1ull << (32 - db)))
        return RADSORT_EINVAL;
    g->nA = static_cast<uint32_t>(nA);
    g->H = static_cast<uint32_t>(H);
    g->nT = static_cast<uint32_t>(2 * H);
    g->npi = static_cast<uint32_t>(npi);
    g->G = static_cast<uint32_t>(H);
    g->grid = false;
    g->msd = false;
    g->shape = 0;
    return RADSORT_OK;
}

// Geometry of the grid layout (one chain per bucket on the output block
// grid): head start (GRID_AHEAD + 2)*sigma, scratch H + 1 blocks (the last
// holds the input tail), the data in logical blocks H .. H + nA.
static radsort_status fill_geom_grid(size_t n, int kb, bool hasv, int db, uint32_t b, int shape, Geom *g)
{
    if (shape < 0 || shape > 2)
        return RADSORT_EINVAL;
    if (!pow2(b) || b < 64 || b > 4096 || lb_tile(kb, db, hasv, shape) % b != 0)
        return RADSORT_EINVAL; // a tile holds whole blocks
    if (n >= (size_t(1) << 31))
        return RADSORT_EINVAL; // look-back words hold 31-bit prefixes
    g->n = n;
    g->kb = kb;
    g->hasv = hasv;
    g->db = db;
    g->sigma = 1u << db;
    g->nt = (8 * kb + db - 1) / db;
    g->b = b;
    g->lb = ilog2(b);
    g->p = 1;
    g->grid = true;
    g->msd = false;
    g->shape = shape;
    const unsigned long long nA = n / b;
    const unsigned long long H = (GRID_AHEAD + 2ull) * g->sigma;
    const unsigned long long npi = nA + H + 1;
    if (npi >= (1ull << 28))
        return RADSORT_EINVAL;
    g->nA = static_cast<uint32_t>(nA);
    g->H = static_cast<uint32_t>(H);
    g->nT = static_cast<uint32_t>(H + 1);
    g->npi = static_cast<uint32_t>(npi);
    g->G = 1;
    return RADSORT_OK;
}

// Automatic plan.  The scratch array costs 2*sigma*p*b*E bytes, so the plan
// trades chunk parallelism p against block size b.  It keeps the whole
// workspace within 2% of the array's bytes (with a floor for small arrays),
// uses at most one chunk per SM and at least ~64K elements per chunk.
static void auto_plan_chunks(size_t n, int kb, int vb, int db, radsort_plan *pl);

// Automatic plan: the grid layout (its extra memory does not grow with the
// number of CTAs); the chunk layout (Sec. 4.3) when n >= 2^31 or when the
// plan asks for it.  Larger blocks are faster (fewer list entries and bulk
// copies per tile, fewer blocks to permute in Finalize) but the scratch array
// grows with b, so the plan takes the largest block size whose workspace is
// within 2% of the array's bytes, 1.25x the least workspace of any block
// size, or 4 MiB above that least as long as that stays within a quarter of
// the array's bytes (below about 2^26 elements no block size meets 2%: the
// look-back ring and tables alone take ~2 MB; a quarter keeps the footprint
// well below an out-of-place sort's).
// Measured (u32 keys + values, us a sort): 2^20 b = 256 309, 512 259;
// 2^22 506, 390; 2^24 1231, 820; 2^25 2233, 1398 -- blocks of 256 leave many
// list entries per tile.
static void auto_plan(size_t n, int kb, int vb, int db, radsort_plan *pl)
{
    if (pl->layout != RADSORT_LAYOUT_CHUNKS && n < (size_t(1) << 31)) {
        const uint32_t cands[] = {256, 512, 1024, 2048, 4096};
        size_t ws[5] = {};
        size_t least = 0;
        for (int i = 0; i < 5; ++i) {
            Geom g;
            if (fill_geom_grid(n, kb, vb != 0, db, cands[i], 0, &g) != RADSORT_OK)
                continue;
            ws[i] = layout(g, nullptr, nullptr);
            if (!least || ws[i] < least)
                least = ws[i];
        }
        const double two = 0.02 * double(n) * double(kb + vb);
        const double some = std::min(double(least) + double(4u << 20), 0.25 * double(n) * double(kb + vb));
        const double budget = std::max({two, 1.25 * double(least), some});
        uint32_t best_b = 0;
        for (int i = 0; i < 5; ++i)
            if (ws[i] && double(ws[i]) <= budget)
                best_b = cands[i];
        if (best_b) {
            pl->layout = RADSORT_LAYOUT_GRID;
            pl->block_size = best_b;
            pl->num_chunks = 1;
            return;
        }
    }
    pl->layout = RADSORT_LAYOUT_CHUNKS;
    auto_plan_chunks(n, kb, vb, db, pl);
}

static void auto_plan_chunks(size_t n, int kb, int vb, int db, radsort_plan *pl)
{
    const size_t E = kb + vb;
    const double budget = 0.02 * double(n) * double(E);
    uint32_t pcap = static_cast<uint32_t>(n / 65536);
    const uint32_t pmax = static_cast<uint32_t>(num_sms());
    if (pcap > pmax)
        pcap = pmax;
    if (pcap < 1)
        pcap = 1;
    uint32_t best_b = 256, best_p = 0;
    const uint32_t cands[] = {256, 512, 1024, 2048};
    for (uint32_t b : cands) {
        Geom g;
        if (fill_geom(n, kb, vb != 0, db, b, 1, &g) != RADSORT_OK)
            continue;
        uint32_t lo = 1, hi = pcap; // largest p within the budget
        if (double(layout(g, nullptr, nullptr)) > budget) {
            hi = 0;
        } else {
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) / 2;
                if (fill_geom(n, kb, vb != 0, db, b, mid, &g) == RADSORT_OK &&
                    double(layout(g, nullptr, nullptr)) <= budget)
                    lo = mid;
                else
                    hi = mid - 1;
            }
        }
        if (hi > best_p) {
            best_p = hi;
            best_b = b;
        }
    }
    if (best_p == 0) { // array too small for 2%: smallest sound plan
        best_p = 1;
        best_b = 256;
        Geom g;
        if (fill_geom(n, kb, vb != 0, db, best_b, 1, &g) != RADSORT_OK)
            best_b = 2048;
    }
    pl->block_size = best_b;
    pl->num_chunks = best_p;
}

// MSD split, then every bucket on its own (Sec. 4.3, last paragraph): the
// chunk layout with one chunk per bucket of the top digit, p = sigma (8-bit
// digits: T holds 2*sigma^2 blocks).  Block size: the plan's, else the
// largest in 64 .. 1024 whose workspace is within 2% of the array's bytes,
// else the smallest the block indices allow.
static radsort_status make_geom_msd(size_t n, int kb, bool hasv, int db, uint32_t b, Geom *g)
{
    if (db != 8)
        return RADSORT_EINVAL;
    const uint32_t sigma = 1u << db;
    if (!b) {
        uint32_t within = 0, valid = 0;
        for (uint32_t cb = 64; cb <= 1024; cb *= 2) {
            Geom t;
            if (fill_geom(n, kb, hasv, db, cb, sigma, &t) != RADSORT_OK)
                continue;
            if (!valid)
                valid = cb;
            if (double(layout(t, nullptr, nullptr)) <= 0.02 * double(n) * double(kb + (hasv ? 4 : 0)))
                within = cb;
        }
        b = within ? within : valid;
        if (!b)
            return RADSORT_EINVAL;
    }
    const radsort_status s = fill_geom(n, kb, hasv, db, b, sigma, g);
    if (s == RADSORT_OK)
        g->msd = true;
    return s;
}

static radsort_status make_geom(size_t n, int kb, bool hasv, int db, const radsort_plan *plan,
                                Geom *g)
{
    if ((kb != 4 && kb != 8) || (db != 8 && db != 11))
        return RADSORT_EINVAL;
    if (plan && plan->layout > RADSORT_LAYOUT_MSD)
        return RADSORT_EINVAL;
    if (plan && plan->layout == RADSORT_LAYOUT_MSD)
        return plan->num_chunks ? RADSORT_EINVAL : make_geom_msd(n, kb, hasv, db, plan->block_size, g);
    radsort_plan pl{};
    if (plan && plan->layout != RADSORT_LAYOUT_SCRATCH)
        pl.layout = plan->layout;
    // a chunk count without a layout means the chunk layout
    if (plan && plan->num_chunks && !plan->layout)
        pl.layout = RADSORT_LAYOUT_CHUNKS;
    if (!plan || !plan->block_size || (pl.layout != RADSORT_LAYOUT_GRID && !plan->num_chunks))
        auto_plan(n, kb, hasv ? 4 : 0, db, &pl);
    if (plan && plan->block_size)
        pl.block_size = plan->block_size;
    if (pl.layout == RADSORT_LAYOUT_GRID)
        return fill_geom_grid(n, kb, hasv, db, pl.block_size, plan ? static_cast<int>(plan->shape) : 0, g);
    if (plan && plan->num_chunks)
        pl.num_chunks = plan->num_chunks;
    return fill_geom(n, kb, hasv, db, pl.block_size, pl.num_chunks, g);
}

// Carves the workspace; with base == nullptr only computes the size.
static size_t layout(const Geom &g, void *base, Bufs *w)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> void * {
        off = align_up(off, 256);
        void *p = base ? static_cast<char *>(base) + off : nullptr;
        off += bytes;
        return p;
    };
    const size_t tel = size_t(g.nT) * g.b;
    const size_t npi2 = g.npi + (g.npi & 1);
    Bufs b{};
    if (g.grid) {
        // [T keys | T values | piX | piY | tables | state | Z], Z = the
        // look-back words during the rounds, then Finalize's jump array and
        // scratch
        b.Tk = take(tel * g.kb);
        b.Tv = static_cast<uint32_t *>(g.hasv ? take(tel * 4) : nullptr);
        b.aux = static_cast<uint32_t *>(take(2 * npi2 * 4));
        b.P = static_cast<uint2 *>(take(8));
        b.E = static_cast<unsigned long long *>(take(2 * 8));
        b.state = static_cast<uint32_t *>(take(ST_WORDS * 4));
        b.ctr = static_cast<uint32_t *>(take(64 * 4));
        b.hist = static_cast<uint32_t *>(take(size_t(g.nt) * g.sigma * 4));
        b.tab = static_cast<uint32_t *>(take((4 * size_t(g.sigma) + 4) * 4));
        const size_t jump = align_up(npi2 * 8, 256), fin = finalize_extra_bytes(g);
        const size_t lbw = grid_ring_bytes(g);
        char *z = static_cast<char *>(take(lbw > jump + fin ? lbw : jump + fin));
        b.status = reinterpret_cast<uint32_t *>(z);
        b.fin = base ? z + jump : nullptr;
        off = align_up(off, 256);
        if (w)
            *w = b;
        return off;
    }
    b.Tk = take(tel * g.kb);
    b.Tv = static_cast<uint32_t *>(g.hasv ? take(tel * 4) : nullptr);
    b.aux = static_cast<uint32_t *>(take(3 * npi2 * 4));
    b.C = static_cast<uint32_t *>(take(size_t(g.G) * 4));
    b.FILL = static_cast<uint32_t *>(take(size_t(g.G) * 4));
    b.S = static_cast<uint32_t *>(take(size_t(g.G) * 4));
    b.P = static_cast<uint2 *>(take(size_t(g.G) * 8));
    b.E = static_cast<unsigned long long *>(take(size_t(g.G + 1) * 8));
    b.lo0 = static_cast<uint32_t *>(take(size_t(g.p + 1) * 4));
    b.lo1 = static_cast<uint32_t *>(take(size_t(g.p + 1) * 4));
    b.Aal = static_cast<uint32_t *>(take(size_t(g.p) * 4));
    b.LOff = static_cast<uint32_t *>(take(size_t(g.p + 1) * 4));
    b.state = static_cast<uint32_t *>(take(ST_WORDS * 4));
    b.fin = take(finalize_extra_bytes(g));
    off = align_up(off, 256);
    if (w)
        *w = b;
    return off;
}

static cudaStream_t as_stream(void *s) { return static_cast<cudaStream_t>(s); }

// The scratch layout: a full sort of a short array (or an explicit request)
// runs Alg. 1 with the alternate arrays inside the workspace.
static bool use_scratch(size_t n, const radsort_plan *plan, bool full_sort)
{
    if (!full_sort)
        return false;
    if (plan && plan->layout == RADSORT_LAYOUT_SCRATCH)
        return true;
    const bool automatic = !plan || (plan->layout == RADSORT_LAYOUT_AUTO && !plan->block_size &&
                                     !plan->num_chunks);
    return automatic && n <= RADSORT_SCRATCH_MAX_N;
}

// [alternate keys | alternate values | Alg. 1 scratch]
static size_t scratch_bytes(size_t n, int kb, bool hasv, int db)
{
    return align_up(n * kb, 256) + (hasv ? align_up(n * 4, 256) : 0) +
           align_up(lsd_oop_scratch_bytes(n, kb, db, hasv), 256);
}

static radsort_status cuda_status(cudaError_t e)
{
    if (e == cudaSuccess)
        return RADSORT_OK;
    if (e == cudaErrorMemoryAllocation)
        return RADSORT_ENOMEM;
    return RADSORT_ECUDA;
}

static bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Runs setup and `rounds` rounds; returns the current pi buffer through *pi_cur.
static cudaError_t run_rounds(const Geom &g, Bufs &w, int rounds, cudaStream_t st,
                              uint32_t **pi_cur, uint32_t **pi_oth)
{
    const size_t npi2 = g.npi + (g.npi & 1);
    cudaError_t e;
    if (g.grid) {
        uint32_t *pc = w.aux, *pn = w.aux + npi2;
        e = cudaMemsetAsync(w.state, 0, ST_WORDS * 4, st);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(w.ctr, 0, 64 * 4, st);
        if (e == cudaSuccess) {
            Scope sc(0, -1, st);
            e = launch_grid_setup(g, w, pc, st);
        }
        for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
            {   // the tables of this digit and the parts of the next map
                // known before the round (head start, shared blocks)
                Scope sc(2, r, st);
                e = launch_grid_prep(g, w, pc, pn, r, st);
            }
            if (e == cudaSuccess) {
                Scope sc(1, r, st);
                e = launch_grid_round(g, w, pc, pn, r, st);
            }
            uint32_t *t = pc;
            pc = pn;
            pn = t;
        }
        *pi_cur = pc;
        *pi_oth = pn;
        return e;
    }
    uint32_t *piX = w.aux, *UC = w.aux + npi2, *piY = w.aux + 2 * npi2;
    uint32_t *pc = piX, *pn = piY, *lc = w.lo0, *ln = w.lo1;
    {
        Scope sc(0, -1, st);
        e = launch_setup(g, w, pc, st);
    }
    for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
        // digit of round r and the order of its output: least significant
        // first across all chunks; with the MSD split, the top digit first
        // (its buckets become the chunks), then each chunk on its own from
        // its least significant digit
        int pos = r, mode = FIX_EVEN;
        if (g.msd) {
            pos = r == 0 ? g.nt - 1 : r - 1;
            mode = r == 0 ? FIX_SPLIT : FIX_PER_CHUNK;
        }
        {
            Scope sc(1, pos, st);
            e = launch_round(g, w, pc, lc, UC, pos, st);
        }
        if (e == cudaSuccess) {
            Scope sc(2, pos, st);
            e = launch_fixup(g, w, pc, pn, UC, lc, ln, mode, st);
        }
        uint32_t *t = pc;
        pc = pn;
        pn = t;
        t = lc;
        lc = ln;
        ln = t;
    }
    *pi_cur = pc;
    *pi_oth = pn;
    return e;
}

} // namespace rs

using namespace rs;

// Workspace bytes of a plan (0 if the plan is not valid for these sizes).
static size_t workspace_of(size_t n, int kb, int vb, int db, const radsort_plan &p)
{
    size_t bytes = 0;
    return radsort_workspace_size(n, kb, vb, db, &p, &bytes) == RADSORT_OK ? bytes : 0;
}

namespace {
// autotuner cache: (device, ceil log2 n, key bytes, value bytes, digit bits)
// -> plan (a plan's timing and chunk count depend on the device)
struct TuneEntry {
    int dev, lg, kb, vb, db;
    radsort_plan plan;
    float ms; // its timed sort (-1: chosen without timing)
};
constexpr int TUNE_CAP = 256;
std::mutex g_tune_mu;
TuneEntry g_tune[TUNE_CAP];
int g_tune_n = 0;

constexpr int MAX_CANDS = 16;
struct Cands {
    radsort_plan p[MAX_CANDS];
    int n = 0;
    void push_back(const radsort_plan &x)
    {
        if (n < MAX_CANDS)
            p[n++] = x;
    }
    bool empty() const { return n == 0; }
};

// The candidate plans of the automatic plan's layout within its budget.
Cands tune_candidates(size_t n, int kb, int vb, int db, const radsort_plan &base)
{
    Cands out;
    const double two = 0.02 * double(n) * double(kb + vb);
    if (base.layout == RADSORT_LAYOUT_GRID) {
        // block sizes x tile shapes (the second shape where it differs)
        const uint32_t cands[] = {256, 512, 1024, 2048, 4096};
        const int shapes[] = {0, 2};
        for (int sh : shapes) {
            if (sh && !lb_shape_differs(db, sh))
                continue;
            size_t ws[5] = {}, least = 0;
            for (int i = 0; i < 5; ++i) {
                Geom g;
                if (fill_geom_grid(n, kb, vb != 0, db, cands[i], sh, &g) != RADSORT_OK)
                    continue;
                ws[i] = layout(g, nullptr, nullptr);
                if (!least || ws[i] < least)
                    least = ws[i];
            }
            const double budget = two > 1.25 * double(least) ? two : 1.25 * double(least);
            for (int i = 0; i < 5; ++i)
                if (ws[i] && double(ws[i]) <= budget) {
                    radsort_plan p{};
                    p.layout = RADSORT_LAYOUT_GRID;
                    p.block_size = cands[i];
                    p.num_chunks = 1;
                    p.shape = static_cast<uint32_t>(sh);
                    out.push_back(p);
                }
        }
    } else {
        const double budget = two > double(workspace_of(n, kb, vb, db, base)) ? two
                                                                           : double(workspace_of(n, kb, vb, db, base));
        const uint32_t cands[] = {256, 512, 1024, 2048};
        for (uint32_t b : cands) {
            radsort_plan p = base;
            p.block_size = b;
            const size_t ws = workspace_of(n, kb, vb, db, p);
            if (ws && double(ws) <= budget)
                out.push_back(p);
        }
    }
    if (out.empty())
        out.push_back(base);
    return out;
}
} // namespace

extern "C" {

const char *radsort_status_str(radsort_status s)
{
    switch (s) {
    case RADSORT_OK: return "ok";
    case RADSORT_EINVAL: return "invalid argument";
    case RADSORT_ENOMEM: return "out of device memory / workspace too small";
    case RADSORT_ECUDA: return "CUDA runtime error";
    case RADSORT_ETIMEOUT: return "bounded device wait ran out";
    case RADSORT_EINTERNAL: return "device invariant check failed";
    }
    return "unknown status";
}

radsort_status radsort_plan_default(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                    radsort_plan *plan)
{
    if (!plan || (key_bytes != 4 && key_bytes != 8) || (value_bytes != 0 && value_bytes != 4) ||
        (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    std::memset(plan, 0, sizeof(*plan));
    if (n <= RADSORT_SCRATCH_MAX_N) {
        plan->layout = RADSORT_LAYOUT_SCRATCH;
        return RADSORT_OK;
    }
    auto_plan(n, key_bytes, value_bytes, digit_bits, plan);
    return RADSORT_OK;
}

radsort_status radsort_workspace_size(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                      const radsort_plan *plan, size_t *bytes)
{
    if (!bytes || (value_bytes != 0 && value_bytes != 4))
        return RADSORT_EINVAL;
    *bytes = 0;
    if (n <= 1)
        return RADSORT_OK;
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (use_scratch(n, plan, true)) {
        *bytes = scratch_bytes(n, key_bytes, value_bytes == 4, digit_bits);
        return RADSORT_OK;
    }
    Geom g;
    radsort_status s = make_geom(n, key_bytes, value_bytes == 4, digit_bits, plan, &g);
    if (s != RADSORT_OK)
        return s;
    *bytes = layout(g, nullptr, nullptr);
    return RADSORT_OK;
}

static radsort_status sort_common(void *keys, uint32_t *values, size_t n, int key_bytes,
                                  int digit_bits, uint32_t flags, const radsort_plan *plan,
                                  void *workspace, size_t workspace_bytes, void *stream,
                                  int rounds, void *out_keys, uint32_t *out_values)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if ((flags & RADSORT_KEY_FLOAT32) && key_bytes != 4)
        return RADSORT_EINVAL;
    if (flags & ~RADSORT_KEY_FLOAT32)
        return RADSORT_EINVAL;
    if (n <= 1 && rounds < 0)
        return RADSORT_OK;
    if (!keys || !aligned16(keys) || (values && !aligned16(values)))
        return RADSORT_EINVAL;
    if (plan && plan->layout == RADSORT_LAYOUT_SCRATCH && rounds >= 0)
        return RADSORT_EINVAL; // no permuted representation to read
    if (use_scratch(n, plan, rounds < 0)) {
        cudaStream_t st = as_stream(stream);
        const bool hasv = values != nullptr;
        const size_t need = scratch_bytes(n, key_bytes, hasv, digit_bits);
        void *ws = workspace;
        bool own = false;
        if (ws) {
            if (workspace_bytes < need || !aligned16(ws))
                return workspace_bytes < need ? RADSORT_ENOMEM : RADSORT_EINVAL;
        } else {
            cudaError_t e = cudaMallocAsync(&ws, need, st);
            if (e != cudaSuccess)
                return cuda_status(e);
            own = true;
        }
        char *ak = static_cast<char *>(ws);
        char *av = ak + align_up(n * key_bytes, 256);
        char *sc = av + (hasv ? align_up(n * 4, 256) : 0);
        cudaError_t e = cudaSuccess;
        if (flags & RADSORT_KEY_FLOAT32) {
            Scope sc0(4, -1, st);
            e = launch_float_keys(static_cast<uint32_t *>(keys), n, 0, st);
        }
        if (e == cudaSuccess) {
            Scope sc1(1, -1, st);
            e = launch_lsd_oop_ws(keys, values, ak, hasv ? reinterpret_cast<uint32_t *>(av) : nullptr, n,
                                  key_bytes, digit_bits, sc, st);
        }
        if (e == cudaSuccess && (flags & RADSORT_KEY_FLOAT32)) {
            Scope sc2(4, -1, st);
            e = launch_float_keys(static_cast<uint32_t *>(keys), n, 1, st);
        }
        if (own) {
            cudaError_t e2 = cudaFreeAsync(ws, st);
            if (e == cudaSuccess)
                e = e2;
        }
        return cuda_status(e);
    }
    Geom g;
    radsort_status s = make_geom(n < 2 ? 2 : n, key_bytes, values != nullptr, digit_bits, plan, &g);
    if (s != RADSORT_OK)
        return s;
    g.n = n;
    g.nA = static_cast<uint32_t>(n / g.b);
    g.npi = g.nA + g.nT;
    if (rounds > g.nt)
        return RADSORT_EINVAL;
    cudaStream_t st = as_stream(stream);
    const size_t need = layout(g, nullptr, nullptr);
    void *ws = workspace;
    bool own = false;
    if (ws) {
        if (workspace_bytes < need || !aligned16(ws))
            return workspace_bytes < need ? RADSORT_ENOMEM : RADSORT_EINVAL;
    } else {
        cudaError_t e = cudaMallocAsync(&ws, need, st);
        if (e != cudaSuccess)
            return cuda_status(e);
        own = true;
    }
    Bufs w;
    layout(g, ws, &w);
    w.Ak = keys;
    w.Av = values;
    cudaError_t e = cudaSuccess;
    if (flags & RADSORT_KEY_FLOAT32) {
        Scope sc(4, -1, st);
        e = launch_float_keys(static_cast<uint32_t *>(keys), n, 0, st);
    }
    uint32_t *pc = nullptr, *po = nullptr;
    if (e == cudaSuccess)
        e = run_rounds(g, w, rounds < 0 ? g.nt : rounds, st, &pc, &po);
    if (e == cudaSuccess) {
        if (rounds < 0) {
            Scope sc(3, -1, st);
            // 2*npi words of scratch: U and the idle pi buffer, adjacent
            // (grid layout: the look-back words, no longer needed)
            const size_t npi2 = g.npi + (g.npi & 1);
            uint32_t *jw = g.grid ? w.status : (pc == w.aux ? w.aux + npi2 : w.aux);
            e = launch_finalize(g, w, pc, reinterpret_cast<unsigned long long *>(jw), st);
            (void)po;
        } else
            e = launch_gather(g, w, pc, out_keys, out_values, st);
    }
    if (e == cudaSuccess && (flags & RADSORT_KEY_FLOAT32) && rounds < 0) {
        Scope sc(4, -1, st);
        e = launch_float_keys(static_cast<uint32_t *>(keys), n, 1, st);
    }
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, st);
        if (e == cudaSuccess)
            e = e2;
    }
    return cuda_status(e);
}

radsort_status radsort_sort_ex(void *keys, uint32_t *values, size_t n, int key_bytes,
                               int digit_bits, uint32_t flags, const radsort_plan *plan,
                               void *workspace, size_t workspace_bytes, void *stream)
{
    return sort_common(keys, values, n, key_bytes, digit_bits, flags, plan, workspace,
                       workspace_bytes, stream, -1, nullptr, nullptr);
}


} // extern "C"

// The fastest plan for one digit width, and its time (-1 if not timed).
static radsort_status tune_one(const void *keys, const uint32_t *values, size_t n, int key_bytes, int digit_bits,
                               void *stream, radsort_plan *plan, float *out_ms)
{
    *out_ms = -1.f;
    const int vb = values ? 4 : 0;
    radsort_plan base{};
    radsort_status s = radsort_plan_default(n < 2 ? 2 : n, key_bytes, vb, digit_bits, &base);
    if (s != RADSORT_OK)
        return s;
    if (n <= 1 || base.layout == RADSORT_LAYOUT_SCRATCH) {
        *plan = base; // one out-of-place pass in the workspace: nothing to choose
        return RADSORT_OK;
    }
    int lg = 0;
    while ((size_t(1) << lg) < n)
        ++lg;
    const int dev = current_device();
    {
        // a cached plan is reused when it is valid for this n as well (the
        // limits of a layout can fall inside a size class)
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (int i = 0; i < g_tune_n; ++i)
            if (g_tune[i].dev == dev && g_tune[i].lg == lg && g_tune[i].kb == key_bytes && g_tune[i].vb == vb &&
                g_tune[i].db == digit_bits && g_tune[i].plan.layout == base.layout &&
                workspace_of(n, key_bytes, vb, digit_bits, g_tune[i].plan)) {
                *plan = g_tune[i].plan;
                *out_ms = g_tune[i].ms;
                return RADSORT_OK;
            }
    }
    const Cands cands = tune_candidates(n, key_bytes, vb, digit_bits, base);
    size_t wsmax = 0;
    for (int ci = 0; ci < cands.n; ++ci) {
        const size_t ws = workspace_of(n, key_bytes, vb, digit_bits, cands.p[ci]);
        wsmax = ws > wsmax ? ws : wsmax;
    }
    cudaStream_t st = as_stream(stream);
    const size_t kbytes = align_up(n * key_bytes, 256), vbytes = values ? align_up(n * 4, 256) : 0;
    char *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), kbytes + vbytes + wsmax, st);
    if (e != cudaSuccess)
        return cuda_status(e);
    void *ck = buf;
    uint32_t *cv = values ? reinterpret_cast<uint32_t *>(buf + kbytes) : nullptr;
    void *ws = buf + kbytes + vbytes;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    radsort_plan best = base;
    float best_ms = -1.f;
    s = RADSORT_OK;
    for (int ci = 0; ci < cands.n; ++ci) {
        const radsort_plan &p = cands.p[ci];
        float pm = -1.f;
        for (int rep = 0; rep < 2 && s == RADSORT_OK; ++rep) {
            e = cudaMemcpyAsync(ck, keys, n * key_bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && values)
                e = cudaMemcpyAsync(cv, values, n * 4, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaEventRecord(e0, st);
            if (e != cudaSuccess) {
                s = cuda_status(e);
                break;
            }
            s = radsort_sort_ex(ck, cv, n, key_bytes, digit_bits, 0, &p, ws, wsmax, stream);
            if (s != RADSORT_OK)
                break;
            e = cudaEventRecord(e1, st);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) {
                s = cuda_status(e);
                break;
            }
            pm = pm < 0.f || ms < pm ? ms : pm;
        }
        if (s != RADSORT_OK)
            break;
        if (best_ms < 0.f || pm < best_ms) {
            best_ms = pm;
            best = p;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const cudaError_t ef = cudaFreeAsync(buf, st);
    if (s == RADSORT_OK)
        s = radsort_device_status(stream); // a timed sort whose bounded wait ran out
    if (s == RADSORT_OK && ef != cudaSuccess)
        s = cuda_status(ef);
    if (s != RADSORT_OK)
        return s;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        int slot = -1;
        for (int i = 0; i < g_tune_n && slot < 0; ++i)
            if (g_tune[i].dev == dev && g_tune[i].lg == lg && g_tune[i].kb == key_bytes &&
                g_tune[i].vb == vb && g_tune[i].db == digit_bits)
                slot = i; // replaces an entry that did not fit this n
        if (slot < 0 && g_tune_n < TUNE_CAP)
            slot = g_tune_n++;
        if (slot >= 0)
            g_tune[slot] = TuneEntry{dev, lg, key_bytes, vb, digit_bits, best, best_ms};
    }
    *plan = best;
    *out_ms = best_ms;
    return RADSORT_OK;
}

extern "C" {

radsort_status radsort_autotune(const void *keys, const uint32_t *values, size_t n, int key_bytes,
                                int digit_bits, void *stream, radsort_plan *plan)
{
    if (!plan || (key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (n > 1 && (!keys || !aligned16(keys) || (values && !aligned16(values))))
        return RADSORT_EINVAL;
    float ms;
    return tune_one(keys, values, n, key_bytes, digit_bits, stream, plan, &ms);
}

radsort_status radsort_autotune_digits(const void *keys, const uint32_t *values, size_t n, int key_bytes,
                                       void *stream, int *digit_bits, radsort_plan *plan)
{
    if (!plan || !digit_bits || (key_bytes != 4 && key_bytes != 8))
        return RADSORT_EINVAL;
    if (n > 1 && (!keys || !aligned16(keys) || (values && !aligned16(values))))
        return RADSORT_EINVAL;
    radsort_plan p8{}, p11{};
    float m8, m11;
    radsort_status s = tune_one(keys, values, n, key_bytes, 8, stream, &p8, &m8);
    if (s == RADSORT_OK)
        s = tune_one(keys, values, n, key_bytes, 11, stream, &p11, &m11);
    if (s != RADSORT_OK)
        return s;
    const bool eleven = m8 >= 0.f && m11 >= 0.f && m11 < m8;
    *digit_bits = eleven ? 11 : 8;
    *plan = eleven ? p11 : p8;
    return RADSORT_OK;
}

radsort_status radsort_sort(void *keys, uint32_t *values, size_t n, int key_bytes, int digit_bits,
                            void *stream)
{
    return sort_common(keys, values, n, key_bytes, digit_bits, 0, nullptr, nullptr, 0, stream, -1,
                       nullptr, nullptr);
}

} // extern "C"

// ---------------------------------------------------------------- segmented
namespace {
// plan of one large segment: the grid layout with the block size of least
// workspace (all SMs work on the segment whatever its length)
radsort_plan large_plan(size_t len)
{
    radsort_plan pl{};
    pl.layout = RADSORT_LAYOUT_GRID;
    (void)len;
    return pl;
}

bool seg_aligned(size_t off, int kb, bool hasv)
{
    // keys and values start 16-byte aligned (the arrays themselves are)
    return (off * kb) % 16 == 0 && (!hasv || (off * 4) % 16 == 0);
}

// elements from a segment's start to the next element whose key and value
// start 16-byte aligned
size_t seg_head(size_t off) { return (4 - off % 4) % 4; }

// Long segments run on up to SEG_STREAMS internal streams forked from the
// caller's stream, so that several of them share the SMs (a segment of 2^19
// elements fills a third of them); each stream has its own workspace slice.
constexpr int SEG_STREAMS = 8;
// streams used by the plans whose long-segment slices hold alternate arrays
constexpr int SEG_STREAMS_ALT = 4;
// the medium pass's scratch (one out-of-place buffer per CTA) is held to
// this share of the arrays' bytes by running fewer CTAs (at least 16).
// Measured on 20,000 lognormal arrays (2^29 keys + values, the longest
// medium one near 2^18, long segments beside it on the library's streams):
// 1.5% -> 7.1 Gkeys/s, 3% -> 13.5, 6% -> 24.0, no limit (2 CTAs per SM,
// 14%) -> 20.7.  The low-memory plan (8-bit digits) sorts the medium
// segments in place instead, in a fixed 514 blocks of 32 elements per CTA.
constexpr double SEG_MED_SHARE = 0.06;

struct SegPlan {
    size_t base = 0;    // classify lists + medium scratch
    size_t large = 0;   // workspace of one long-segment stream
    size_t total = 0;   // base + nstr * large
    uint32_t med_max = 0, med_ctas = 0;
    bool ip = false;    // medium segments in place (level >= 1)
    int level = 0;      // see seg_plan
    int nstr = 0;       // internal streams used (0: no long segment)
};

// oop: long segments sorted out of place (Alg. 1) into the caller's
// alternate arrays, so a stream's slice holds only the comparator's scratch;
// level (8-bit digits, not oop): 0 the fastest plan; 1 medium segments
// sorted in place (Radsort per CTA); 2 as 1, and long segments with an
// unaligned start sorted in place too (their first elements merged back)
// instead of out of place
radsort_status seg_plan(const uint64_t *offh, size_t nseg, int kb, bool hasv, int db, bool oop, int level,
                        SegPlan *sp)
{
    size_t large = 0, nlong = 0, nmed = 0;
    uint32_t med_max = 0;
    const uint32_t small_max = seg_small_max(db);
    const size_t n = nseg ? offh[nseg] - offh[0] : 0;
    for (size_t s = 0; s < nseg; ++s) {
        if (offh[s + 1] < offh[s])
            return RADSORT_EINVAL;
        const size_t len = offh[s + 1] - offh[s];
        if (len <= SEG_MED) {
            if (len > small_max) {
                ++nmed;
                if (len > med_max)
                    med_max = static_cast<uint32_t>(len);
            }
            continue;
        }
        ++nlong;
        size_t need;
        if (oop) {
            need = lsd_oop_scratch_bytes(len, kb, db, hasv) + 256;
        } else if (seg_aligned(offh[s], kb, hasv)) {
            const radsort_plan pl = large_plan(len);
            Geom g;
            if (make_geom(len, kb, hasv, db, &pl, &g) != RADSORT_OK)
                return RADSORT_EINVAL;
            need = layout(g, nullptr, nullptr);
        } else if (level >= 2 && db == 8) { // Radsort on the aligned body, the head merged back
            const size_t h = seg_head(offh[s]), nbody = len - h;
            const radsort_plan pl = large_plan(nbody);
            Geom g;
            if (make_geom(nbody, kb, hasv, db, &pl, &g) != RADSORT_OK)
                return RADSORT_EINVAL;
            need = (layout(g, nullptr, nullptr) + 255) / 256 * 256 + head_merge_bytes(nbody, kb, hasv);
        } else { // out of place, Alg. 1, with alternate buffers in the workspace
            need = (len * kb + 255) / 256 * 256 + (hasv ? (len * 4 + 255) / 256 * 256 : 0) +
                   lsd_oop_scratch_bytes(len, kb, db, hasv) + 256;
        }
        if (need > large)
            large = (need + 255) / 256 * 256;
    }
    sp->med_max = med_max;
    sp->ip = level >= 1 && !oop && db == 8;
    // the in-place medium pass: two CTAs per SM, but one per SM on 7/8 of
    // the SMs when long segments run beside it, so that their sorts find SMs
    // of their own (measured on 20,000 lognormal arrays, medium-in-place
    // plan: 304 CTAs 17.0 Gkeys/s, 136 19.2, 120 17.3, 100 14.7; smallest
    // plan: 304 13.7, 136 15.0, 120 15.6, 100 14.6; medium arrays alone: 304
    // the fastest)
    const size_t ip_ctas = nlong ? size_t(num_sms()) * 7 / 8 : size_t(seg_ip_ctas());
    sp->level = sp->ip ? level : 0;
    sp->med_ctas = !med_max ? 0
                   : sp->ip ? static_cast<uint32_t>(nmed < ip_ctas ? nmed : ip_ctas)
                            : seg_med_ctas(med_max, kb, hasv,
                                           static_cast<size_t>(SEG_MED_SHARE * double(n) * (kb + (hasv ? 4 : 0))));
    sp->base = (seg_scratch_bytes(kb, hasv, nseg, med_max, sp->med_ctas, sp->ip) + 255) / 256 * 256;
    sp->large = large;
    const size_t smax = sp->level >= 2 ? size_t(SEG_STREAMS) : size_t(SEG_STREAMS_ALT);
    sp->nstr = static_cast<int>(nlong < smax ? nlong : smax);
    sp->total = sp->base + size_t(sp->nstr) * large;
    return RADSORT_OK;
}

struct SegStreams {
    cudaStream_t s[SEG_STREAMS];
    cudaEvent_t fork;
    cudaEvent_t join[SEG_STREAMS];
};
SegStreams g_seg_streams[MAX_DEVICES];
std::mutex g_seg_mu; // one call at a time forks onto the internal streams

// the current device's internal streams and events (created on first use)
radsort_status seg_streams(SegStreams **out)
{
    static DeviceOnce once;
    const int dev = current_device();
    if (dev < 0 || dev >= MAX_DEVICES)
        return RADSORT_ECUDA;
    const cudaError_t e = once.run([dev] {
        SegStreams &x = g_seg_streams[dev];
        cudaError_t r = cudaEventCreateWithFlags(&x.fork, cudaEventDisableTiming);
        for (int i = 0; i < SEG_STREAMS && r == cudaSuccess; ++i) {
            r = cudaStreamCreateWithFlags(&x.s[i], cudaStreamNonBlocking);
            if (r == cudaSuccess)
                r = cudaEventCreateWithFlags(&x.join[i], cudaEventDisableTiming);
        }
        return r;
    });
    if (e != cudaSuccess)
        return cuda_status(e);
    *out = &g_seg_streams[dev];
    return RADSORT_OK;
}

// Enqueues main() on st (the short and medium segments) and sorts the long
// segments beside it: each goes, longest first, to the internal stream with
// the fewest elements so far; sort_one(offset, length, slice, stream).  The
// internal streams start after the work already on st (so the workspace is
// free), and st waits for them at the end.
template <typename M, typename F>
radsort_status seg_run(const uint64_t *offh, size_t nseg, const SegPlan &sp, char *lw, cudaStream_t st,
                       M &&main, F &&sort_one)
{
    if (sp.nstr == 0)
        return main();
    std::vector<uint32_t> idx;
    for (size_t s = 0; s < nseg; ++s)
        if (offh[s + 1] - offh[s] > SEG_MED)
            idx.push_back(static_cast<uint32_t>(s));
    std::stable_sort(idx.begin(), idx.end(), [&](uint32_t x, uint32_t y) {
        return offh[x + 1] - offh[x] > offh[y + 1] - offh[y];
    });
    SegStreams *ss = nullptr;
    radsort_status rs = seg_streams(&ss);
    if (rs != RADSORT_OK)
        return rs;
    std::lock_guard<std::mutex> lk(g_seg_mu);
    cudaError_t e = cudaEventRecord(ss->fork, st);
    for (int i = 0; i < sp.nstr && e == cudaSuccess; ++i)
        e = cudaStreamWaitEvent(ss->s[i], ss->fork, 0);
    if (e != cudaSuccess)
        return cuda_status(e);
    rs = main();
    unsigned long long load[SEG_STREAMS] = {};
    for (uint32_t sg : idx) {
        if (rs != RADSORT_OK)
            break;
        int best = 0;
        for (int i = 1; i < sp.nstr; ++i)
            if (load[i] < load[best])
                best = i;
        const size_t off = offh[sg], len = offh[sg + 1] - off;
        load[best] += len;
        rs = sort_one(off, len, lw + size_t(best) * sp.large, ss->s[best]);
    }
    // the join is recorded even after a failure, so st never runs ahead
    for (int i = 0; i < sp.nstr; ++i) {
        cudaError_t ej = cudaEventRecord(ss->join[i], ss->s[i]);
        if (ej == cudaSuccess)
            ej = cudaStreamWaitEvent(st, ss->join[i], 0);
        if (ej != cudaSuccess && rs == RADSORT_OK)
            rs = cuda_status(ej);
    }
    return rs;
}

// the caller's workspace, or one allocated stream-ordered
radsort_status seg_workspace(void *workspace, size_t workspace_bytes, size_t need, cudaStream_t st,
                             void **ws, bool *own)
{
    *own = false;
    *ws = workspace;
    if (workspace) {
        if (workspace_bytes < need)
            return RADSORT_ENOMEM;
        return aligned16(workspace) ? RADSORT_OK : RADSORT_EINVAL;
    }
    const cudaError_t e = cudaMallocAsync(ws, need ? need : 256, st);
    if (e != cudaSuccess)
        return cuda_status(e);
    *own = true;
    return RADSORT_OK;
}
} // namespace

extern "C" {

radsort_status radsort_segmented_workspace_size(const uint64_t *offsets_host, size_t num_segments,
                                                int key_bytes, int value_bytes, int digit_bits,
                                                size_t *bytes)
{
    if (!bytes || (key_bytes != 4 && key_bytes != 8) || (value_bytes != 0 && value_bytes != 4) ||
        (digit_bits != 8 && digit_bits != 11) || (num_segments && !offsets_host))
        return RADSORT_EINVAL;
    SegPlan sp;
    radsort_status s = seg_plan(offsets_host, num_segments, key_bytes, value_bytes == 4, digit_bits, false, 0, &sp);
    *bytes = s == RADSORT_OK ? sp.total : 0;
    return s;
}

radsort_status radsort_segmented_workspace_size_min(const uint64_t *offsets_host, size_t num_segments,
                                                    int key_bytes, int value_bytes, int digit_bits,
                                                    size_t *bytes)
{
    if (!bytes || (key_bytes != 4 && key_bytes != 8) || (value_bytes != 0 && value_bytes != 4) ||
        (digit_bits != 8 && digit_bits != 11) || (num_segments && !offsets_host))
        return RADSORT_EINVAL;
    size_t best = 0;
    radsort_status s = RADSORT_OK;
    for (int level = 0; level <= 2 && s == RADSORT_OK; ++level) {
        SegPlan sp;
        s = seg_plan(offsets_host, num_segments, key_bytes, value_bytes == 4, digit_bits, false, level, &sp);
        if (s == RADSORT_OK && (level == 0 || sp.total < best))
            best = sp.total;
    }
    *bytes = s == RADSORT_OK ? best : 0;
    return s;
}

radsort_status radsort_sort_segmented(void *keys, uint32_t *values, const uint64_t *offsets_dev,
                                      const uint64_t *offsets_host, size_t num_segments,
                                      int key_bytes, int digit_bits, void *workspace,
                                      size_t workspace_bytes, void *stream)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (num_segments == 0)
        return RADSORT_OK;
    if (!keys || !offsets_dev || !offsets_host || !aligned16(keys) || (values && !aligned16(values)))
        return RADSORT_EINVAL;
    if (num_segments >= (size_t(1) << 31))
        return RADSORT_EINVAL;
    const bool hasv = values != nullptr;
    SegPlan sp;
    radsort_status s = seg_plan(offsets_host, num_segments, key_bytes, hasv, digit_bits, false, 0, &sp);
    // a caller workspace below the fastest plan: the fastest one that fits
    for (int level = 1; s == RADSORT_OK && workspace && workspace_bytes < sp.total && digit_bits == 8 && level <= 2;
         ++level) {
        SegPlan lo;
        s = seg_plan(offsets_host, num_segments, key_bytes, hasv, digit_bits, false, level, &lo);
        if (s == RADSORT_OK && workspace_bytes >= lo.total)
            sp = lo;
    }
    if (s != RADSORT_OK)
        return s;
    cudaStream_t st = as_stream(stream);
    void *ws = nullptr;
    bool own = false;
    s = seg_workspace(workspace, workspace_bytes, sp.total, st, &ws, &own);
    if (s != RADSORT_OK)
        return s;
    auto main = [&]() -> radsort_status {
        return cuda_status(launch_segmented(keys, values, reinterpret_cast<const unsigned long long *>(offsets_dev),
                                            num_segments, key_bytes, digit_bits, sp.med_max, sp.med_ctas, sp.ip, ws,
                                            st));
    };
    radsort_status rs = seg_run(offsets_host, num_segments, sp, static_cast<char *>(ws) + sp.base, st, main,
                      [&](size_t off, size_t len, char *lw, cudaStream_t ls) -> radsort_status {
                          char *sk = static_cast<char *>(keys) + off * key_bytes;
                          uint32_t *sv = hasv ? values + off : nullptr;
                          if (seg_aligned(off, key_bytes, hasv)) {
                              const radsort_plan pl = large_plan(len);
                              return sort_common(sk, sv, len, key_bytes, digit_bits, 0, &pl, lw, sp.large, ls,
                                                 -1, nullptr, nullptr);
                          }
                          if (sp.level >= 2) { // low memory: the head set aside, the aligned body by Radsort
                              const size_t h = seg_head(off), nbody = len - h;
                              const size_t hmb = head_merge_bytes(nbody, key_bytes, hasv);
                              char *mb = lw + sp.large - hmb;
                              radsort_status r = cuda_status(launch_head_save(sk, sv, static_cast<uint32_t>(h),
                                                                              key_bytes, mb, ls));
                              const radsort_plan pl = large_plan(nbody);
                              if (r == RADSORT_OK)
                                  r = sort_common(sk + h * key_bytes, hasv ? sv + h : nullptr, nbody, key_bytes,
                                                  digit_bits, 0, &pl, lw, sp.large - hmb, ls, -1, nullptr, nullptr);
                              if (r == RADSORT_OK)
                                  r = cuda_status(launch_head_merge(sk, sv, static_cast<uint32_t>(h), nbody,
                                                                    key_bytes, mb, ls));
                              return r;
                          }
                          char *ak = lw;
                          char *av = ak + (len * key_bytes + 255) / 256 * 256;
                          char *sc = av + (hasv ? (len * 4 + 255) / 256 * 256 : 0);
                          return cuda_status(launch_lsd_oop_ws(sk, sv, ak,
                                                               hasv ? reinterpret_cast<uint32_t *>(av) : nullptr,
                                                               len, key_bytes, digit_bits, sc, ls));
                      });
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, st);
        if (rs == RADSORT_OK)
            rs = cuda_status(e2);
    }
    return rs;
}

radsort_status radsort_lsd_oop_segmented_workspace_size(const uint64_t *offsets_host, size_t num_segments,
                                                        int key_bytes, int value_bytes, int digit_bits,
                                                        size_t *bytes)
{
    if (!bytes || (key_bytes != 4 && key_bytes != 8) || (value_bytes != 0 && value_bytes != 4) ||
        (digit_bits != 8 && digit_bits != 11) || (num_segments && !offsets_host))
        return RADSORT_EINVAL;
    SegPlan sp;
    radsort_status s = seg_plan(offsets_host, num_segments, key_bytes, value_bytes == 4, digit_bits, true, 0, &sp);
    *bytes = s == RADSORT_OK ? sp.total : 0;
    return s;
}

radsort_status radsort_segmented_autotune(const void *keys, const uint32_t *values, const uint64_t *offsets_dev,
                                         const uint64_t *offsets_host, size_t num_segments, int key_bytes,
                                         void *stream, int *digit_bits)
{
    if (!digit_bits || (key_bytes != 4 && key_bytes != 8) || (num_segments && (!offsets_host || !offsets_dev)))
        return RADSORT_EINVAL;
    *digit_bits = 8;
    if (num_segments == 0)
        return RADSORT_OK;
    if (!keys || !aligned16(keys) || (values && !aligned16(values)))
        return RADSORT_EINVAL;
    const bool hasv = values != nullptr;
    const size_t n = offsets_host[num_segments] - offsets_host[0];
    SegPlan s8, s11;
    radsort_status s = seg_plan(offsets_host, num_segments, key_bytes, hasv, 8, false, 0, &s8);
    if (s == RADSORT_OK)
        s = seg_plan(offsets_host, num_segments, key_bytes, hasv, 11, false, 0, &s11);
    if (s != RADSORT_OK)
        return s;
    const size_t end = offsets_host[num_segments];
    const size_t kbytes = align_up(end * key_bytes, 256), vbytes = hasv ? align_up(end * 4, 256) : 0;
    const size_t wsb = s8.total > s11.total ? s8.total : s11.total;
    cudaStream_t st = as_stream(stream);
    char *buf = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void **>(&buf), kbytes + vbytes + wsb + 256, st);
    if (e != cudaSuccess)
        return cuda_status(e);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    e = cudaEventCreate(&e0);
    if (e == cudaSuccess)
        e = cudaEventCreate(&e1);
    float best[2] = {-1.f, -1.f};
    for (int w = 0; w < 2 && e == cudaSuccess && s == RADSORT_OK && n > 1; ++w) {
        const int db = w ? 11 : 8;
        for (int rep = 0; rep < 2 && e == cudaSuccess && s == RADSORT_OK; ++rep) {
            e = cudaMemcpyAsync(buf, keys, end * key_bytes, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess && hasv)
                e = cudaMemcpyAsync(buf + kbytes, values, end * 4, cudaMemcpyDeviceToDevice, st);
            if (e == cudaSuccess)
                e = cudaEventRecord(e0, st);
            if (e != cudaSuccess)
                break;
            s = radsort_sort_segmented(buf, hasv ? reinterpret_cast<uint32_t *>(buf + kbytes) : nullptr, offsets_dev,
                                       offsets_host, num_segments, key_bytes, db, buf + kbytes + vbytes, wsb,
                                       stream);
            if (s != RADSORT_OK)
                break;
            e = cudaEventRecord(e1, st);
            if (e == cudaSuccess)
                e = cudaEventSynchronize(e1);
            float ms = 0.f;
            if (e == cudaSuccess)
                e = cudaEventElapsedTime(&ms, e0, e1);
            if (e == cudaSuccess && (best[w] < 0.f || ms < best[w]))
                best[w] = ms;
        }
    }
    if (e0)
        cudaEventDestroy(e0);
    if (e1)
        cudaEventDestroy(e1);
    const cudaError_t ef = cudaFreeAsync(buf, st);
    if (s == RADSORT_OK && e != cudaSuccess)
        s = cuda_status(e);
    if (s == RADSORT_OK)
        s = radsort_device_status(stream);
    if (s == RADSORT_OK && ef != cudaSuccess)
        s = cuda_status(ef);
    if (s == RADSORT_OK && best[0] >= 0.f && best[1] >= 0.f && best[1] < best[0])
        *digit_bits = 11;
    return s;
}

radsort_status radsort_lsd_oop_sort_segmented(void *keys, uint32_t *values, void *keys_alt,
                                              uint32_t *values_alt, const uint64_t *offsets_dev,
                                              const uint64_t *offsets_host, size_t num_segments,
                                              int key_bytes, int digit_bits, void *workspace,
                                              size_t workspace_bytes, void *stream)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (num_segments == 0)
        return RADSORT_OK;
    if (!keys || !keys_alt || !offsets_dev || !offsets_host || !aligned16(keys) ||
        (values && (!aligned16(values) || !values_alt)))
        return RADSORT_EINVAL;
    if (num_segments >= (size_t(1) << 31))
        return RADSORT_EINVAL;
    const bool hasv = values != nullptr;
    SegPlan sp;
    radsort_status s = seg_plan(offsets_host, num_segments, key_bytes, hasv, digit_bits, true, 0, &sp);
    if (s != RADSORT_OK)
        return s;
    cudaStream_t st = as_stream(stream);
    void *ws = nullptr;
    bool own = false;
    s = seg_workspace(workspace, workspace_bytes, sp.total, st, &ws, &own);
    if (s != RADSORT_OK)
        return s;
    auto main = [&]() -> radsort_status {
        return cuda_status(launch_segmented(keys, values, reinterpret_cast<const unsigned long long *>(offsets_dev),
                                            num_segments, key_bytes, digit_bits, sp.med_max, sp.med_ctas, sp.ip, ws,
                                            st));
    };
    radsort_status rs = seg_run(offsets_host, num_segments, sp, static_cast<char *>(ws) + sp.base, st, main,
                      [&](size_t off, size_t len, char *lw, cudaStream_t ls) -> radsort_status {
                          char *sk = static_cast<char *>(keys) + off * key_bytes;
                          char *ak = static_cast<char *>(keys_alt) + off * key_bytes;
                          return cuda_status(launch_lsd_oop_ws(sk, hasv ? values + off : nullptr, ak,
                                                               hasv ? values_alt + off : nullptr, len, key_bytes,
                                                               digit_bits, lw, ls));
                      });
    if (own) {
        cudaError_t e2 = cudaFreeAsync(ws, st);
        if (rs == RADSORT_OK)
            rs = cuda_status(e2);
    }
    return rs;
}

} // extern "C"

// ---------------------------------------------------------------- no allocation
// Scratch of radsort_sort_noalloc: one array in this library's device image.
// Every GPU that loads the library holds these bytes until the process
// exits.  Host code must never pass the symbol itself to a kernel: on the
// host it names a stand-in, not device memory.  Its device address is looked
// up with cudaGetSymbolAddress on the current device at every call: the
// lookup allocates nothing, and a context that was reset and created again
// (cudaDeviceReset) may place the array elsewhere, so a cached address could
// go stale.
namespace {
static __device__ __align__(256) unsigned char g_noalloc_scratch[RADSORT_NOALLOC_SCRATCH_BYTES];

// device address of the scratch on the current device
radsort_status noalloc_scratch(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return e != cudaSuccess ? cuda_status(e) : RADSORT_ECUDA;
    *out = p;
    return RADSORT_OK;
}

// the automatic plan (grid layout) when its workspace fits in the scratch;
// otherwise the chunk layout with block size 256 and as many chunks (up to
// one per SM) as fit
radsort_status noalloc_plan(size_t n, int kb, bool hasv, int db, radsort_plan *pl)
{
    std::memset(pl, 0, sizeof(*pl));
    Geom g;
    if (make_geom(n, kb, hasv, db, nullptr, &g) == RADSORT_OK && g.grid &&
        layout(g, nullptr, nullptr) <= RADSORT_NOALLOC_SCRATCH_BYTES) {
        pl->layout = RADSORT_LAYOUT_GRID;
        pl->block_size = g.b;
        return RADSORT_OK;
    }
    pl->layout = RADSORT_LAYOUT_CHUNKS;
    pl->block_size = 256;
    uint32_t lo = 1, hi = static_cast<uint32_t>(num_sms());
    if (fill_geom(n, kb, hasv, db, 256, 1, &g) != RADSORT_OK ||
        layout(g, nullptr, nullptr) > RADSORT_NOALLOC_SCRATCH_BYTES)
        return RADSORT_ENOMEM; // n too large for the fixed scratch
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) / 2;
        if (fill_geom(n, kb, hasv, db, 256, mid, &g) == RADSORT_OK &&
            layout(g, nullptr, nullptr) <= RADSORT_NOALLOC_SCRATCH_BYTES)
            lo = mid;
        else
            hi = mid - 1;
    }
    pl->num_chunks = lo;
    return RADSORT_OK;
}
} // namespace

extern "C" {

radsort_status radsort_sort_noalloc(void *keys, uint32_t *values, size_t n, int key_bytes,
                                    int digit_bits, void *stream)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (n <= 1)
        return RADSORT_OK;
    radsort_plan pl;
    radsort_status s = noalloc_plan(n, key_bytes, values != nullptr, digit_bits, &pl);
    if (s != RADSORT_OK)
        return s;
    void *ws = nullptr;
    s = noalloc_scratch(&ws);
    if (s != RADSORT_OK)
        return s;
    return sort_common(keys, values, n, key_bytes, digit_bits, 0, &pl, ws,
                       RADSORT_NOALLOC_SCRATCH_BYTES, stream, -1, nullptr, nullptr);
}

radsort_status radsort_sort_rounds(void *keys, uint32_t *values, size_t n, int key_bytes,
                                   int digit_bits, int rounds, const radsort_plan *plan,
                                   void *out_keys, uint32_t *out_values, void *stream)
{
    if (rounds < 0 || !out_keys || !aligned16(out_keys) || (out_values && !values))
        return RADSORT_EINVAL;
    if (n == 0)
        return RADSORT_OK;
    return sort_common(keys, values, n, key_bytes, digit_bits, 0, plan, nullptr, 0, stream, rounds,
                       out_keys, out_values);
}

} // extern "C"

// ---------------------------------------------------------------- permuted representation
// Host handle of a Radsort state kept between calls (grid layout).  g0 is
// the geometry of the array as opened (its block count npi never changes);
// the current geometry has the current element count.
struct radsort_perm {
    Geom g0;
    size_t n;          // current element count
    Bufs w;
    uint32_t *pc, *pn; // current and next block map
    bool hist_ok;      // w.hist holds the current sequence's digit counts
    bool finalized;
};

namespace {
Geom perm_geom(const radsort_perm *h)
{
    Geom g = h->g0;
    g.n = h->n;
    g.nA = static_cast<uint32_t>(h->n / g.b);
    return g; // npi, nT, H as opened
}

radsort_status perm_plan(size_t n, int kb, bool hasv, int db, uint32_t block_size, Geom *g)
{
    radsort_plan pl{};
    pl.layout = RADSORT_LAYOUT_GRID;
    pl.block_size = block_size;
    return make_geom(n < 2 ? 2 : n, kb, hasv, db, &pl, g);
}
} // namespace

extern "C" {

radsort_status radsort_perm_workspace_size(size_t n, int key_bytes, int value_bytes, int digit_bits,
                                           uint32_t block_size, size_t *bytes)
{
    if (!bytes || (value_bytes != 0 && value_bytes != 4))
        return RADSORT_EINVAL;
    *bytes = 0;
    Geom g;
    const radsort_status s = perm_plan(n, key_bytes, value_bytes == 4, digit_bits, block_size, &g);
    if (s != RADSORT_OK)
        return s;
    g.n = n;
    g.nA = static_cast<uint32_t>(n / g.b);
    g.npi = g.nA + g.nT;
    *bytes = layout(g, nullptr, nullptr);
    return RADSORT_OK;
}

radsort_status radsort_perm_open(void *keys, uint32_t *values, size_t n, int key_bytes, int digit_bits,
                                 uint32_t block_size, void *workspace, size_t workspace_bytes,
                                 void *stream, radsort_perm **out)
{
    if (!out || !keys || !workspace || !aligned16(keys) || (values && !aligned16(values)) ||
        !aligned16(workspace))
        return RADSORT_EINVAL;
    *out = nullptr;
    Geom g;
    radsort_status s = perm_plan(n, key_bytes, values != nullptr, digit_bits, block_size, &g);
    if (s != RADSORT_OK)
        return s;
    g.n = n;
    g.nA = static_cast<uint32_t>(n / g.b);
    g.npi = g.nA + g.nT;
    if (workspace_bytes < layout(g, nullptr, nullptr))
        return RADSORT_ENOMEM;
    radsort_perm *h = static_cast<radsort_perm *>(std::malloc(sizeof(radsort_perm)));
    if (!h)
        return RADSORT_ENOMEM;
    h->g0 = g;
    h->n = n;
    layout(g, workspace, &h->w);
    h->w.Ak = keys;
    h->w.Av = values;
    const size_t npi2 = g.npi + (g.npi & 1);
    h->pc = h->w.aux;
    h->pn = h->w.aux + npi2;
    h->hist_ok = true; // setup takes the histograms of the input
    h->finalized = false;
    cudaStream_t st = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(h->w.state, 0, ST_WORDS * 4, st);
    if (e == cudaSuccess) {
        Scope sc(0, -1, st);
        e = launch_grid_setup(g, h->w, h->pc, st);
    }
    if (e != cudaSuccess) {
        std::free(h);
        return cuda_status(e);
    }
    *out = h;
    return RADSORT_OK;
}

radsort_status radsort_perm_rounds(radsort_perm *h, int first, int count, void *stream)
{
    if (!h || h->finalized || first < 0 || count < 0 || first + count > h->g0.nt)
        return RADSORT_EINVAL;
    if (count == 0 || h->n <= 1)
        return RADSORT_OK; // a sequence of at most one element is sorted
    const Geom g = perm_geom(h);
    cudaStream_t st = as_stream(stream);
    // fresh tickets and an untagged look-back ring for this call's rounds
    cudaError_t e = cudaMemsetAsync(h->w.ctr, 0, 64 * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(h->w.status, 0, grid_ring_bytes(h->g0), st);
    if (e == cudaSuccess && !h->hist_ok) {
        Scope sc(0, -1, st);
        e = launch_block_hist(g, h->w, h->pc, st);
        if (e == cudaSuccess)
            h->hist_ok = true;
    }
    for (int r = first; r < first + count && e == cudaSuccess; ++r) {
        {
            Scope sc(2, r, st);
            e = launch_grid_prep(g, h->w, h->pc, h->pn, r, st);
        }
        if (e == cudaSuccess) {
            Scope sc(1, r, st);
            e = launch_grid_round(g, h->w, h->pc, h->pn, r, st);
        }
        std::swap(h->pc, h->pn);
    }
    return cuda_status(e);
}

radsort_status radsort_perm_keys_changed(radsort_perm *h)
{
    if (!h || h->finalized)
        return RADSORT_EINVAL;
    h->hist_ok = false;
    return RADSORT_OK;
}

radsort_status radsort_perm_size(const radsort_perm *h, size_t *n, size_t *entries)
{
    if (!h)
        return RADSORT_EINVAL;
    if (n)
        *n = h->n;
    if (entries)
        *entries = h->n / h->g0.b + 1;
    return RADSORT_OK;
}

radsort_status radsort_perm_blocks(radsort_perm *h, radsort_block *out_dev, size_t cap, void *stream)
{
    if (!h || h->finalized || !out_dev || cap < h->n / h->g0.b + 1)
        return RADSORT_EINVAL;
    return cuda_status(launch_block_list(perm_geom(h), h->w, h->pc, out_dev, as_stream(stream)));
}

radsort_status radsort_perm_gather(radsort_perm *h, void *out_keys, uint32_t *out_values, void *stream)
{
    if (!h || h->finalized || (h->n && (!out_keys || !aligned16(out_keys))) ||
        (out_values && !h->w.Av))
        return RADSORT_EINVAL;
    if (h->n == 0)
        return RADSORT_OK;
    const Geom g = perm_geom(h);
    return cuda_status(launch_gather(g, h->w, h->pc, out_keys, out_values, as_stream(stream)));
}

radsort_status radsort_perm_truncate(radsort_perm *h, size_t m, void *stream)
{
    if (!h || h->finalized || m > h->n)
        return RADSORT_EINVAL;
    if (m == h->n)
        return RADSORT_OK;
    h->n = m;
    h->hist_ok = false;
    return cuda_status(launch_set_tail(perm_geom(h), h->w, as_stream(stream)));
}

radsort_status radsort_perm_finalize(radsort_perm *h, void *stream)
{
    if (!h || h->finalized)
        return RADSORT_EINVAL;
    h->finalized = true;
    cudaStream_t st = as_stream(stream);
    Scope sc(3, -1, st);
    return cuda_status(launch_finalize(perm_geom(h), h->w, h->pc,
                                       reinterpret_cast<unsigned long long *>(h->w.status), st));
}

radsort_status radsort_perm_close(radsort_perm *h)
{
    std::free(h);
    return RADSORT_OK;
}

radsort_status radsort_float_keys(uint32_t *keys, size_t n, int inverse, void *stream)
{
    if (n && !keys)
        return RADSORT_EINVAL;
    return cuda_status(launch_float_keys(keys, n, inverse, as_stream(stream)));
}

radsort_status radsort_lsd_oop_sort(void *keys, uint32_t *values, void *keys_alt,
                                    uint32_t *values_alt, size_t n, int key_bytes, int digit_bits,
                                    void *stream)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11))
        return RADSORT_EINVAL;
    if (n <= 1)
        return RADSORT_OK;
    if (!keys || !keys_alt || (values && !values_alt))
        return RADSORT_EINVAL;
    return cuda_status(
        launch_lsd_oop(keys, values, keys_alt, values_alt, n, key_bytes, digit_bits, as_stream(stream)));
}

radsort_status radsort_lsd_oop_scratch_size(size_t n, int key_bytes, int value_bytes,
                                            int digit_bits, size_t *bytes)
{
    if ((key_bytes != 4 && key_bytes != 8) || (digit_bits != 8 && digit_bits != 11) ||
        (value_bytes != 0 && value_bytes != 4) || !bytes)
        return RADSORT_EINVAL;
    *bytes = n <= 1 ? 0 : lsd_oop_scratch_bytes(n, key_bytes, digit_bits, value_bytes == 4);
    return RADSORT_OK;
}

radsort_status radsort_debug_wait_probe(const uint32_t *flag, unsigned iterations, void *stream)
{
    if (!flag || iterations == 0 || iterations > wait_spin_limit())
        return RADSORT_EINVAL;
    return cuda_status(launch_wait_probe(flag, iterations, as_stream(stream)));
}

radsort_status radsort_device_status(void *stream)
{
    cudaError_t e = cudaStreamSynchronize(as_stream(stream));
    if (e != cudaSuccess)
        return cuda_status(e);
    const unsigned v = take_status_round() | take_status_finalize() | take_status_oop() | take_status_seg() |
                       take_status_perm();
    if (v & ST_TIMEOUT)
        return RADSORT_ETIMEOUT;
    if (v & ST_INTERNAL)
        return RADSORT_EINTERNAL;
    return RADSORT_OK;
}

radsort_status radsort_trace_enable(int on)
{
    std::lock_guard<std::mutex> lk(rs::g_tmu);
    rs::g_trace_on = on != 0;
    return RADSORT_OK;
}

radsort_status radsort_trace_read(radsort_trace_rec *out, int cap, int *count)
{
    if (!count || (cap > 0 && !out))
        return RADSORT_EINVAL;
    std::vector<rs::TraceRec> recs;
    {
        std::lock_guard<std::mutex> lk(rs::g_tmu);
        recs.swap(rs::g_trace);
    }
    radsort_status st = RADSORT_OK;
    int k = 0;
    for (auto &r : recs) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e == cudaSuccess)
            e = cudaEventElapsedTime(&ms, r.a, r.b);
        if (e != cudaSuccess)
            st = cuda_status(e);
        if (k < cap) {
            out[k].phase = r.phase;
            out[k].round = r.round;
            out[k].ms = ms;
        }
        ++k;
        std::lock_guard<std::mutex> lk(rs::g_tmu);
        rs::g_pool.push_back(r.a);
        rs::g_pool.push_back(r.b);
    }
    *count = k;
    return st;
}

radsort_status radsort_launch_count(uint64_t *launches)
{
    if (!launches)
        return RADSORT_EINVAL;
    *launches = rs::g_launches.load();
    return RADSORT_OK;
}

} // extern "C"
