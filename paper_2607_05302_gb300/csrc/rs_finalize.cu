// Radsort Finalize (Alg. 7) and the float32 key transform, sm_103a.
//
// This first Finalize is the paper's sequential procedure run by a single
// CTA.  Thread 0 keeps the logical/physical bookkeeping (pi, pi^-1, the free
// spot, sizeOfNextBlock).  All threads move each block through shared memory.
// The pull reads the whole source block before writing, so an overlapping
// pull toward lower addresses (source and target the same block) is a
// memmove.
#include "rs_common.cuh"
#include "rs_kernels.cuh"

namespace rs {

unsigned take_status_finalize() { return take_status_word(); }

__global__ void k_inverse(const uint32_t *pi, uint32_t *pinv, uint32_t npi)
{
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < npi; i += gridDim.x * blockDim.x)
        pinv[pi[i]] = i;
}

template <typename KT>
__global__ void __launch_bounds__(1024) k_finalize_seq(KT *Ak, uint32_t *Av, KT *Tk, uint32_t *Tv,
                                                       uint32_t *pi, uint32_t *pinv, const uint2 *P,
                                                       const uint32_t *state, uint32_t H,
                                                       uint32_t nT, uint32_t nA, uint32_t b,
                                                       unsigned long long n)
{
    extern __shared__ __align__(16) unsigned char fsm[];
    KT *bk = reinterpret_cast<KT *>(fsm);
    uint32_t *bv = reinterpret_cast<uint32_t *>(fsm + size_t(b) * sizeof(KT));
    __shared__ uint32_t s_jin, s_jout, s_jfree, s_l, s_push;
    __shared__ unsigned long long s_k;
    const uint32_t f = state[ST_F], nP = state[ST_NP];
    const int t = threadIdx.x, T = blockDim.x;
    // thread-0 state
    uint32_t iP = 0, i_free = 0, j_free = 0;
    unsigned long long k = 0;
    if (t == 0)
        j_free = pi[0]; // logical 0 is in the head start: unallocated
    auto keys_of = [&](uint32_t j) -> KT * { return j < nT ? Tk + size_t(j) * b : Ak + size_t(j - nT) * b; };
    auto vals_of = [&](uint32_t j) -> uint32_t * { return j < nT ? Tv + size_t(j) * b : Av + size_t(j - nT) * b; };
    const bool hv = Av != nullptr;

    for (uint32_t i_in = H; i_in < f; ++i_in) {
        uint32_t i_out = 0;
        if (t == 0) {
            const uint32_t j_in = pi[i_in];
            uint32_t push = 0, j_out = 0;
            if (i_in < H + nA) {
                j_out = i_in + H; // A block i_in - H
                i_out = pinv[j_out];
                push = (i_in < i_out && i_out < f) ? 1u : 0u;
            }
            uint32_t l = b;
            if (iP < nP && P[iP].x == i_in) // sizeOfNextBlock (Alg. 3)
                l = P[iP++].y;
            s_jin = j_in;
            s_jout = j_out;
            s_jfree = j_free;
            s_l = l;
            s_push = push;
            s_k = k;
        }
        __syncthreads();
        const uint32_t j_in = s_jin, j_out = s_jout, l = s_l;
        if (s_push) { // push the block at j_out to the free spot
            KT *dk = keys_of(s_jfree);
            const KT *sk = keys_of(j_out);
            for (uint32_t e = t; e < b; e += T)
                dk[e] = sk[e];
            if (hv) {
                uint32_t *dv = vals_of(s_jfree);
                const uint32_t *sv = vals_of(j_out);
                for (uint32_t e = t; e < b; e += T)
                    dv[e] = sv[e];
            }
        }
        __syncthreads();
        { // pull l elements of block j_in to A[k..k+l)
            const KT *sk = keys_of(j_in);
            for (uint32_t e = t; e < l; e += T)
                bk[e] = sk[e];
            if (hv) {
                const uint32_t *sv = vals_of(j_in);
                for (uint32_t e = t; e < l; e += T)
                    bv[e] = sv[e];
            }
            __syncthreads();
            const unsigned long long kk = s_k;
            for (uint32_t e = t; e < l; e += T) {
                Ak[kk + e] = bk[e];
                if (hv)
                    Av[kk + e] = bv[e];
            }
        }
        if (t == 0) {
            k += l;
            if (i_in < H + nA) {
                if (s_push) { // swap(i_out, j_out, i_free, j_free)
                    pi[i_out] = j_free;
                    pi[i_free] = j_out;
                    pinv[j_out] = i_free;
                    pinv[j_free] = i_out;
                    i_out = i_free;
                }
                // swap(i_out, j_out, i_in, j_in)
                pi[i_out] = j_in;
                pi[i_in] = j_out;
                pinv[j_out] = i_in;
                pinv[j_in] = i_out;
                if (i_in != i_out) {
                    i_free = i_out;
                    j_free = j_in;
                }
            }
        }
        __syncthreads();
    }
    if (t == 0 && k != n)
        set_status(ST_INTERNAL);
}

size_t finalize_extra_bytes(const Geom &) { return 0; }

cudaError_t launch_finalize(const Geom &g, const Bufs &w, uint32_t *pi, uint32_t *pi_other,
                            cudaStream_t st)
{
    int blocks = static_cast<int>((g.npi + 255) / 256);
    if (blocks > 8192)
        blocks = 8192;
    k_inverse<<<blocks, 256, 0, st>>>(pi, pi_other, g.npi);
    const size_t smem = size_t(g.b) * (g.kb + (g.hasv ? 4 : 0));
    if (g.kb == 4) {
        cudaFuncSetAttribute(k_finalize_seq<uint32_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(smem));
        k_finalize_seq<uint32_t><<<1, 1024, smem, st>>>(
            static_cast<uint32_t *>(w.Ak), g.hasv ? w.Av : nullptr, static_cast<uint32_t *>(w.Tk),
            w.Tv, pi, pi_other, w.P, w.state, g.H, g.nT, g.nA, g.b, (unsigned long long)g.n);
    } else {
        cudaFuncSetAttribute(k_finalize_seq<unsigned long long>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
        k_finalize_seq<unsigned long long><<<1, 1024, smem, st>>>(
            static_cast<unsigned long long *>(w.Ak), g.hasv ? w.Av : nullptr,
            static_cast<unsigned long long *>(w.Tk), w.Tv, pi, pi_other, w.P, w.state, g.H, g.nT,
            g.nA, g.b, (unsigned long long)g.n);
    }
    return cudaGetLastError();
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

cudaError_t launch_float_keys(uint32_t *keys, size_t n, int inverse, cudaStream_t st)
{
    if (n == 0)
        return cudaSuccess;
    int blocks = static_cast<int>((n + 1023) / 1024);
    const int cap = num_sms() * 8;
    if (blocks > cap)
        blocks = cap;
    k_float_keys<<<blocks, 256, 0, st>>>(keys, n, inverse);
    return cudaGetLastError();
}

} // namespace rs
