// Kernel launchers of the Radsort library (host side declarations).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <atomic>
#include <mutex>

#include "radsort.h"

namespace rs {

// bits of the device status words
enum : unsigned { ST_TIMEOUT = 1u, ST_INTERNAL = 2u };

// Sizes of one sort (host view).  Block indices are 32-bit.
struct Geom {
    size_t n;          // elements
    int kb;            // key bytes 4 | 8
    bool hasv;         // 32-bit values present
    int db;            // digit bits 8 | 11
    uint32_t sigma;    // 2^db
    int nt;            // digits per key
    uint32_t b, lb;    // block size and log2
    uint32_t p;        // chunks
    uint32_t nA;       // floor(n/b): blocks overlaying A
    uint32_t H;        // head start sigma*p
    uint32_t nT;       // scratch blocks 2H
    uint32_t npi;      // nA + nT
    uint32_t G;        // groups (bucket, chunk) = sigma*p
    bool grid;         // one chain per bucket on the output block grid (H = (GRID_AHEAD + 2) sigma, nT = H + 1)
    bool msd;          // chunk layout with p = sigma: a split on the top digit, then each bucket on its own
    int shape;         // grid layout: tile shape of the round kernel (radsort_plan.shape)
};

// Device buffers of one sort, carved from one workspace allocation.
struct Bufs {
    void *Ak;          // caller's keys
    uint32_t *Av;      // caller's values (nullable)
    void *Tk;          // scratch keys, nT*b
    uint32_t *Tv;      // scratch values, nT*b (nullable)
    uint32_t *aux;     // [piX | UC | piY]: 3*npi words (pi ping-pong around UC)
    uint32_t *C;       // G  block counts, bucket-major (c*p + q)
    uint32_t *FILL;    // G  open-block fill
    uint32_t *S;       // G  group start (logical index)
    uint2 *P;          // G  partial blocks (logical index, length)
    unsigned long long *E; // G group first element position
    uint32_t *lo0, *lo1;   // p+1 chunk bounds (ping-pong)
    uint32_t *Aal;     // p   allocations per chunk
    uint32_t *LOff;    // p+1 leftover offsets
    uint32_t *state;   // scalars, see ST_*
    void *fin;         // Finalize scratch (finalize_extra_bytes)
    // grid layout only
    uint32_t *hist;    // nt*sigma digit counts of the input
    uint32_t *tab;     // per-round bucket tables (4*sigma + 1 words)
    uint32_t *status;  // look-back ring (after the rounds: Finalize's jump array and scratch)
    uint32_t *ctr;     // per-round tile tickets
};

// grid layout: blocks a bucket's chain takes ahead of its writes (the head
// start is (GRID_AHEAD + 2) * sigma blocks)
constexpr uint32_t GRID_AHEAD = 2;

// indices into Bufs::state
enum { ST_F = 0, ST_NP = 1, ST_FPREV = 2, ST_LOFFTOT = 3, ST_NS = 4, ST_SKIP = 5, ST_WORDS = 8 };

// setup (Alg. 4) + chunk bounds of round 0
cudaError_t launch_setup(const Geom &g, const Bufs &w, uint32_t *pi, cudaStream_t st);
// one sortPhase (Alg. 5) over p chunks on the digit at bits [pos*d, (pos+1)*d)
cudaError_t launch_round(const Geom &g, const Bufs &w, const uint32_t *pi, const uint32_t *lo,
                         uint32_t *UC, int pos, cudaStream_t st);
// fixupPhase (Alg. 6): scan + placement into pi_new; the group order and the
// next chunk bounds by mode
enum FixMode { FIX_EVEN = 0, FIX_SPLIT = 1, FIX_PER_CHUNK = 2 };
cudaError_t launch_fixup(const Geom &g, const Bufs &w, const uint32_t *pi_old, uint32_t *pi_new,
                         const uint32_t *UC, const uint32_t *lo_old, uint32_t *lo_new, int mode,
                         cudaStream_t st);
// grid layout: digit histograms + setup; per round the tables and the
// prefilled next map (prep), then sortPhase
cudaError_t launch_grid_setup(const Geom &g, const Bufs &w, uint32_t *pi, cudaStream_t st);
cudaError_t launch_grid_prep(const Geom &g, const Bufs &w, const uint32_t *pi, uint32_t *pin,
                             int round, cudaStream_t st);
cudaError_t launch_grid_round(const Geom &g, const Bufs &w, const uint32_t *pi, uint32_t *pin,
                              int round, cudaStream_t st);
size_t grid_ring_bytes(const Geom &g); // look-back ring of the grid layout
// elements per tile of the look-back round kernel with a tile shape (0: the
// default), and whether a shape differs from the default for the digit width
uint32_t lb_tile(int kb, int db, bool hasv, int shape);
bool lb_shape_differs(int db, int shape);
// gather of the logical sequence (Sec. 4.1 iterator)
cudaError_t launch_gather(const Geom &g, const Bufs &w, const uint32_t *pi, void *out_k,
                          uint32_t *out_v, cudaStream_t st);
// Finalize (Alg. 7 semantics): pi applied to the data in place
// deficit prefix over the current P into Bufs::E (nP + 1 entries)
cudaError_t launch_deficit(const Geom &g, const Bufs &w, cudaStream_t st);
// jump: 2*npi words of scratch, 8-byte aligned (U plus the idle pi buffer)
cudaError_t launch_finalize(const Geom &g, const Bufs &w, uint32_t *pi, unsigned long long *jump,
                            cudaStream_t st);
size_t finalize_extra_bytes(const Geom &g);
// float32 key transform
cudaError_t launch_float_keys(uint32_t *keys, size_t n, int inverse, cudaStream_t st);
// out-of-place LSD comparator
cudaError_t launch_lsd_oop(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                           size_t n, int kb, int db, cudaStream_t st);

// out-of-place LSD with caller scratch (nullptr: allocate stream-ordered)
cudaError_t launch_lsd_oop_ws(void *keys, uint32_t *vals, void *keys_alt, uint32_t *vals_alt,
                              size_t n, int kb, int db, void *scratch, cudaStream_t st);
size_t lsd_oop_scratch_bytes(size_t n, int kb, int db, bool hasv);
// batched segmented sort of the small and medium segments
constexpr uint32_t SEG_MED = 1u << 18;
uint32_t seg_small_max(int db);
uint32_t seg_med_ctas(uint32_t med_max, int kb, bool hasv, size_t budget);
uint32_t seg_ip_ctas();
// a long segment with an unaligned start, in the low-memory plan: its first
// h < 4 elements set aside (save), the rest sorted, then merged back
size_t head_merge_bytes(size_t nbody, int kb, bool hasv);
cudaError_t launch_head_save(const void *keys, const uint32_t *vals, uint32_t h, int kb, void *buf, cudaStream_t st);
cudaError_t launch_head_merge(void *keys, uint32_t *vals, uint32_t h, size_t nbody, int kb, void *buf, cudaStream_t st);
size_t seg_scratch_bytes(int kb, bool hasv, size_t nseg, uint32_t med_max, uint32_t med_ctas, bool ip);
cudaError_t launch_segmented(void *keys, uint32_t *vals, const unsigned long long *off_dev,
                             size_t nseg, int kb, int db, uint32_t med_max, uint32_t med_ctas, bool ip,
                             void *scratch, cudaStream_t st);
unsigned take_status_seg();

// devices a process may use (per-device caches are sized for this many)
constexpr int MAX_DEVICES = 64;
int num_sms();     // SM count of the current device
int current_device(); // current device ordinal, -1 on error

// Runs a set-up step once per device (the device current at the call), for
// example a cudaFuncSetAttribute opt-in: thread-safe, and repeated on a
// device where it failed.  One object per call site (a function-local
// static).
class DeviceOnce {
  public:
    template <typename F> cudaError_t run(F &&f)
    {
        const int dev = current_device();
        if (dev < 0 || dev >= MAX_DEVICES)
            return cudaErrorInvalidDevice;
        if (done_[dev].load(std::memory_order_acquire))
            return cudaSuccess;
        std::lock_guard<std::mutex> lk(mu_);
        if (done_[dev].load(std::memory_order_relaxed))
            return cudaSuccess;
        const cudaError_t e = f();
        if (e == cudaSuccess)
            done_[dev].store(true, std::memory_order_release);
        return e;
    }

  private:
    std::mutex mu_;
    std::atomic<bool> done_[MAX_DEVICES] = {};
};
// kernels launched by this library (host counter)
extern std::atomic<unsigned long long> g_launches;
// read and clear the device status words of each translation unit
unsigned take_status_round();
unsigned take_status_finalize();
unsigned take_status_oop();
unsigned take_status_perm();

// permuted representation kept between calls (grid layout; g.n is the
// current element count, g.npi the block count of the original array)
// digit histograms of the current sequence, read through pi
cudaError_t launch_block_hist(const Geom &g, const Bufs &w, const uint32_t *pi, cudaStream_t st);
// (key address, value address, length) of every logical block in order
cudaError_t launch_block_list(const Geom &g, const Bufs &w, const uint32_t *pi, radsort_block *out,
                              cudaStream_t st);
// P and f after the sequence was cut to g.n elements (Alg. 8)
cudaError_t launch_set_tail(const Geom &g, const Bufs &w, cudaStream_t st);

} // namespace rs
