/*
 * Radsort oracle -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded CPU restatement of the algorithms of
 * "Parallel O(sqrt n) Overhead LSD Radix Sort" (Clausecker & Schintke):
 *
 *   ora_lsd_oop   -- Alg. 1 (out-of-place LSD round), applied for
 *                    t = n_t-1 ... 0 with a ping-pong buffer.
 *   ora_radsort   -- Alg. 2 (driver): Alg. 4 (setup), Alg. 5 (sortPhase,
 *                    newBucketBlock), Alg. 3 (sizeOfNextBlock), Alg. 6
 *                    (fixupPhase), Alg. 7 (swap/finalize), with the data
 *                    invariant of Sec. 2.2 and Lemmas 1 and 2 asserted.
 *                    p > 1 is the parallel variant of Sec. 4.3: the
 *                    logical blocks are split into p chunks, each with its
 *                    own head start of sigma blocks (T = 2*sigma*p blocks),
 *                    its own bucket array B, and one P entry per
 *                    (bucket, chunk) after the fixup.  p = 1 is exactly the
 *                    sequential algorithm of Sec. 2.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline leg
 * may load this library.  It shares no code with the CUDA path.
 *
 * Readings of passages that are garbled or ambiguous in the paper:
 *   G1 Alg. 3 compares pi[i] with P's entry, but P holds logical indices
 *      (Sec. 2.1): we compare i itself, and return the length read before
 *      i_P is advanced.
 *   G2 Alg. 7 sets j_out from i_in - sigma, which would address T; the text
 *      puts the data at physical blocks 2*sigma.. : j_out = i_in + H where H
 *      is the head-start size (sigma for p = 1), i.e. A block i_in - H.
 *   G3 Alg. 7's swap also exchanges the caller's variables; we keep the loop
 *      counter apart and track (i_free, j_free) as the text describes.
 *   G4 "up to b partial blocks described by B" (Sec. 2.3.2) means one per
 *      bucket: sigma (sigma*p with chunks).
 *   G5 setup uses floor(n/b)+1 data blocks with the tail always a partial
 *      block (possibly of length 0), as Alg. 4 does.
 *   G6 a pull whose source and target overlap is a memmove.
 *   G8 digit t (t = 0 most significant) of an unsigned key with d-bit digits
 *      covers bits [(n_t-1-t)d, (n_t-t)d); sigma = 2^d for every digit.
 *   G7 Lemma 1's i_in is the "next input block" of the variable table: once
 *      the last element of the current block has been copied, that block
 *      counts as consumed (read as the loop variable of Alg. 5, the bound
 *      fails by one at block ends, e.g. b = 1).
 *   G9 T and unallocated blocks are poisoned (0xA5 bytes) so that a read of
 *      unallocated data shows up in the output.
 *   G15 Alg. 8 (truncate) drops the P entries after the one it rewrites, and
 *      a cut at a block's last element makes the next logical block the
 *      final, empty partial block (see truncate_at).
 *   G16 Finalize after a truncation pushes a remaining block out of A block
 *      floor(n/b) before the gap-closing copies (see finalize).
 *
 *   ora_perm_*    -- the permuted representation kept between calls
 *                    (Sec. 4.1): rounds on it, truncate (Alg. 8), the
 *                    logical sequence, and a later Finalize.
 *
 * Function pins (tests/test_oracle_pins.py): every function here is pinned
 * to numpy's stable argsort, to brute-force stable sorting of exhaustive
 * tiny inputs, and to the invariants and lemmas of the paper.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORACLE_MUTANT
#define ORACLE_MUTANT 0 /* >0 plants a known mistake (used by the pin tests) */
#endif
/* Mutants 1-6 plant mistakes in the data path (caught by the output pins).
 * Mutants 7-13 corrupt only the algorithm state, to show that each check of
 * the data invariant (Sec. 2.2), of Lemmas 1-2 (Sec. 2.3) and of the copy
 * bound (Sec. 3) fires on its own:
 *   7  two P entries exchanged after fixupPhase   -> ORA_INV_PORDER
 *   8  fill level f one past the last used block  -> ORA_INV_LASTPARTIAL
 *   9  a block of pi' entered twice               -> ORA_INV_PERM
 *   10 a head start of sigma-1 blocks per chunk   -> ORA_LEMMA1
 *   11 one scratch block fewer (2H-1 blocks in T) -> ORA_LEMMA2
 *   12 an open block's fill recorded one short    -> ORA_INV_COUNT
 *   13 Finalize pulls through a bounce block      -> ORA_FIN_COPIES
 * Mutants 14-15 concern truncation (Alg. 8) and Finalize after it:
 *   14 truncate keeps a P entry past the new end  -> ORA_INV_PORDER
 *   15 Finalize without the push of reading G16   -> wrong output */

/* error codes (negative) */
#define ORA_OK 0
#define ORA_EARG -1
#define ORA_ENOMEM -2
#define ORA_LEMMA1 -10
#define ORA_LEMMA2 -11
#define ORA_INV_PERM -12
#define ORA_INV_PORDER -13
#define ORA_INV_LASTPARTIAL -14
#define ORA_INV_COUNT -15
#define ORA_FIN_COUNT -16
#define ORA_FIN_COPIES -17

typedef struct {
    uint64_t key;
    uint32_t val;
} elem_t;

typedef struct {
    uint64_t n_pi;          /* block count floor(n/b) + 2H */
    uint64_t head;          /* H = sigma * p */
    uint64_t t_blocks;      /* scratch blocks 2H */
    uint64_t lemma1_checks; /* newBucketBlock calls beyond the initial sigma */
    uint64_t min_unallocated; /* smallest unallocated count seen at fixup (Lemma 2) */
    uint64_t fin_copies_main; /* block copies in Finalize's first loop */
    uint64_t fin_copies_rest; /* block copies in Finalize's second loop */
    uint64_t fin_pushes;
    uint64_t extra_bytes;   /* T + bookkeeping, Sec. 3 "Space" / Sec. 4 */
    uint64_t fin_copies_trunc; /* Finalize's push out of A block floor(n/b) (reading G16) */
} ora_stats;

/* ---- key positions (Sec. 1; reading G8) -------------------------------- */
typedef struct {
    int n_t;
    uint32_t sigma;
    int bits;        /* >0: d-bit digit fields; 0: key is a base-sigma numeral */
} keyspec;

static uint32_t key_at(const keyspec *ks, uint64_t k, int t)
{
#if ORACLE_MUTANT == 3
    t = ks->n_t - 1 - t; /* planted mistake: digits numbered from the LSB */
#endif
    int pos = ks->n_t - 1 - t; /* number of digits below digit t */
    if (ks->bits > 0) {
        unsigned sh = (unsigned)(pos * ks->bits);
        if (sh >= 64)
            return 0;
        return (uint32_t)((k >> sh) & (uint64_t)(ks->sigma - 1));
    }
    for (int i = 0; i < pos; i++)
        k /= ks->sigma;
    return (uint32_t)(k % ks->sigma);
}

static int check_spec(const keyspec *ks)
{
    if (ks->n_t < 1 || ks->n_t > 64 || ks->sigma < 1)
        return ORA_EARG;
    if (ks->bits > 0) {
        if (ks->bits > 16 || ks->sigma != (1u << ks->bits))
            return ORA_EARG;
    } else if (ks->sigma < 2) {
        return ORA_EARG;
    }
    return ORA_OK;
}

/* ======================================================================
 * Alg. 1 -- out-of-place LSD radix sort round radixSortStep(A', A, t)
 * ====================================================================== */
static void radix_sort_step(elem_t *Ap, const elem_t *A, size_t n, const keyspec *ks, int t,
                            size_t *H, size_t *S)
{
    for (uint32_t c = 0; c < ks->sigma; c++)
        H[c] = 0;
    for (size_t i = 0; i < n; i++) /* histogram of key(A[i], t) */
        H[key_at(ks, A[i].key, t)]++;
    S[0] = 0;
    for (uint32_t c = 1; c < ks->sigma; c++) /* prefix sum over H */
        S[c] = S[c - 1] + H[c - 1];
#if ORACLE_MUTANT == 5
    /* planted mistake: scatter walking the input backwards (unstable) */
    for (size_t i = n; i-- > 0;) {
        uint32_t c = key_at(ks, A[i].key, t);
        Ap[S[c]++] = A[i];
    }
#else
    for (size_t i = 0; i < n; i++) {
        uint32_t c = key_at(ks, A[i].key, t); /* determine bucket */
        Ap[S[c]] = A[i];                      /* sort A[i] into A' */
        S[c]++;                               /* advance bucket c */
    }
#endif
}

/* keys/vals in place; `rounds` rounds for t = n_t-1, n_t-2, ... */
int ora_lsd_oop(uint64_t *keys, uint32_t *vals, size_t n, int n_t, uint32_t sigma, int bits,
                int rounds)
{
    keyspec ks = {n_t, sigma, bits};
    if (check_spec(&ks) != ORA_OK || rounds < 0 || rounds > n_t)
        return ORA_EARG;
    if (n == 0)
        return ORA_OK;
    elem_t *A = malloc(n * sizeof(elem_t));
    elem_t *Ap = malloc(n * sizeof(elem_t));
    size_t *H = malloc(sigma * sizeof(size_t));
    size_t *S = malloc(sigma * sizeof(size_t));
    if (!A || !Ap || !H || !S) {
        free(A), free(Ap), free(H), free(S);
        return ORA_ENOMEM;
    }
    for (size_t i = 0; i < n; i++) {
        A[i].key = keys[i];
        A[i].val = vals ? vals[i] : 0;
    }
    for (int r = 0; r < rounds; r++) {
        int t = n_t - 1 - r;
        radix_sort_step(Ap, A, n, &ks, t, H, S);
        elem_t *tmp = A;
        A = Ap;
        Ap = tmp;
    }
    for (size_t i = 0; i < n; i++) {
        keys[i] = A[i].key;
        if (vals)
            vals[i] = A[i].val;
    }
    free(A), free(Ap), free(H), free(S);
    return ORA_OK;
}

/* ======================================================================
 * Radsort state (Sec. 2.1)
 * ====================================================================== */
typedef struct {
    uint64_t idx; /* logical index */
    uint64_t len; /* used elements, 0 <= len < b */
} partial_t;

typedef struct {
    elem_t *next; /* p_next */
    elem_t *end;  /* p_end */
} bucket_t;

typedef struct {
    keyspec ks;
    size_t n, b;
    uint64_t p;     /* chunks (Sec. 4.3); 1 = sequential algorithm */
    uint64_t H;     /* head start = sigma * p */
    uint64_t tb;    /* scratch blocks in T: 2H */
    uint64_t n_pi;  /* floor(n/b) + 2H */
    elem_t *A;      /* input / output array */
    elem_t *T;      /* 2H scratch blocks */
    uint64_t *pi;   /* logical index -> physical block */
    uint64_t *pi2;  /* pi' (also reused for pi^-1 by Finalize) */
    partial_t *P;   /* partial blocks, ascending logical index */
    uint64_t nP;
    uint64_t f;     /* fill level */
    /* per-round, per-chunk scratch */
    uint64_t *lo;   /* chunk bounds in logical block indices, p+1 entries */
    uint64_t *C;    /* block counts, C[c*p + q] */
    uint64_t *S;    /* bucket starts, S[c*p + q] */
    bucket_t *B;    /* bucket allocation, B[q*sigma + c] */
    uint32_t *U;    /* usage per free-list entry, U[q*U_stride + k] */
    uint64_t U_stride;
    uint64_t *iout; /* i_out per chunk */
    elem_t *bounce; /* one block (mutant 13 only) */
    ora_stats *st;
} rs_t;

static elem_t *blockat(rs_t *s, uint64_t i)
{
    if (i < s->tb)
        return &s->T[i * s->b];
    return &s->A[(i - s->tb) * s->b];
}

/* Alg. 3 with reading G1 */
static uint64_t size_of_next_block(rs_t *s, uint64_t i, uint64_t *iP)
{
    if (*iP < s->nP && s->P[*iP].idx == i) {
        uint64_t l = s->P[*iP].len;
#if ORACLE_MUTANT == 6
        /* planted mistake: the literal listing, length of the entry after */
        if (*iP + 1 < s->nP)
            l = s->P[*iP + 1].len;
#endif
        (*iP)++;
        return l;
    }
    return s->b;
}

/* data invariant of Sec. 2.2 (clauses 1-3 and the element count of 5) */
static int check_invariant(rs_t *s)
{
    uint8_t *seen = calloc(s->n_pi, 1);
    if (!seen)
        return ORA_ENOMEM;
    for (uint64_t i = 0; i < s->n_pi; i++) {
        if (s->pi[i] >= s->n_pi || seen[s->pi[i]]) {
            free(seen);
            return ORA_INV_PERM;
        }
        seen[s->pi[i]] = 1;
    }
    free(seen);
    for (uint64_t j = 0; j < s->nP; j++) {
        if (s->P[j].idx < s->H || s->P[j].idx >= s->f || s->P[j].len >= s->b)
            return ORA_INV_PORDER;
        if (j > 0 && s->P[j].idx <= s->P[j - 1].idx)
            return ORA_INV_PORDER;
    }
    if (s->nP == 0 || s->P[s->nP - 1].idx != s->f - 1)
        return ORA_INV_LASTPARTIAL;
    uint64_t iP = 0, total = 0;
    for (uint64_t i = s->H; i < s->f; i++)
        total += size_of_next_block(s, i, &iP);
    if (total != s->n)
        return ORA_INV_COUNT;
    return ORA_OK;
}

/* Alg. 4 (setup), head start H = sigma*p */
static int setup(rs_t *s)
{
    uint64_t H = s->H, nb = s->n / s->b;
    s->f = H + nb + 1;
    for (uint64_t i = 0; i < H; i++) /* head start */
        s->pi[i] = i;
    for (uint64_t i = H; i + 1 < s->f; i++) /* contents of A */
        s->pi[i] = s->tb + (i - H);
    for (uint64_t i = s->f - 1; i < s->n_pi; i++) /* remaining T blocks */
        s->pi[i] = H + (i - (s->f - 1));
    memset(s->T, 0xA5, s->tb * s->b * sizeof(elem_t)); /* reading G9 */
    memcpy(blockat(s, H), &s->A[nb * s->b], (s->n % s->b) * sizeof(elem_t)); /* tail */
    s->P[0].idx = s->f - 1;
    s->P[0].len = s->n % s->b;
    s->nP = 1;
    return check_invariant(s);
}

/* chunk bounds (Sec. 4.3): chunk q starts at the first logical block whose
 * first element has position >= floor(q*n/p) in the current sequence. */
static void make_chunks(rs_t *s)
{
    uint64_t q = 1, iP = 0, pos = 0;
    s->lo[0] = s->H;
    for (uint64_t i = s->H; i < s->f && q < s->p; i++) {
        while (q < s->p && pos >= (uint64_t)(((unsigned __int128)q * s->n) / s->p))
            s->lo[q++] = i;
        pos += size_of_next_block(s, i, &iP);
    }
    while (q < s->p)
        s->lo[q++] = s->f;
    s->lo[s->p] = s->f;
}

static uint64_t free_list_entry(rs_t *s, uint64_t q, uint64_t k)
{
    uint32_t sigma = s->ks.sigma;
    if (k < sigma)
        return s->pi[q * sigma + k];
    return s->pi[s->lo[q] + (k - sigma)];
}

/* newBucketBlock of Alg. 5, for chunk q.  i_in_fl is the free-list index of
 * the next input block not yet fully read (reading G7 of Lemma 1: i_in as
 * "next input block", which is the current block's index plus one once its
 * last element has been copied). */
static int new_bucket_block(rs_t *s, uint64_t q, uint32_t c, uint64_t i_in_fl)
{
    uint32_t sigma = s->ks.sigma;
    uint64_t i_out = s->iout[q];
    if (i_out >= sigma) { /* Lemma 1: i_out < i_in (free-list indices) */
        s->st->lemma1_checks++;
        if (!(i_out < i_in_fl))
            return ORA_LEMMA1;
    }
    elem_t *pn = blockat(s, free_list_entry(s, q, i_out));
    s->B[q * sigma + c].next = pn;
    s->B[q * sigma + c].end = pn + s->b;
    s->C[(uint64_t)c * s->p + q]++;
    s->U[q * s->U_stride + i_out] = c;
    s->iout[q] = i_out + 1;
    return ORA_OK;
}

/* Alg. 5 (sortPhase) on every chunk in turn */
static int sort_phase(rs_t *s, int t)
{
    uint32_t sigma = s->ks.sigma;
    make_chunks(s);
    memset(s->C, 0, (uint64_t)sigma * s->p * sizeof(uint64_t));
    uint64_t iP = 0;
    for (uint64_t q = 0; q < s->p; q++) {
        s->iout[q] = 0;
#if ORACLE_MUTANT == 10
        s->iout[q] = 1; /* planted state mistake: head start of sigma-1 blocks */
#endif
        for (uint32_t c = 0; c < sigma; c++) { /* initial output blocks */
            int e = new_bucket_block(s, q, c, 0);
            if (e)
                return e;
        }
        for (uint64_t i_in = s->lo[q]; i_in < s->lo[q + 1]; i_in++) {
            uint64_t fl_in = sigma + (i_in - s->lo[q]); /* i_in as free-list index */
            elem_t *p_in = blockat(s, s->pi[i_in]);
            uint64_t l = size_of_next_block(s, i_in, &iP);
#if ORACLE_MUTANT == 1
            l = s->b; /* planted mistake: partial blocks read as full */
#endif
            for (uint64_t j = 0; j < l; j++) {
                uint32_t c = key_at(&s->ks, p_in[j].key, t);
                bucket_t *bk = &s->B[q * sigma + c];
                *bk->next = p_in[j]; /* copy p_in[j] to memory at p_next */
                if (bk->next + 1 == bk->end) {
                    int e = new_bucket_block(s, q, c, fl_in + (j + 1 == l ? 1 : 0));
                    if (e)
                        return e;
                } else {
                    bk->next++;
                }
            }
        }
    }
    return ORA_OK;
}

/* Alg. 6 (fixupPhase), generalised to p chunks */
static int fixup_phase(rs_t *s)
{
    uint32_t sigma = s->ks.sigma;
    uint64_t G = (uint64_t)sigma * s->p;
    uint64_t allocated = 0;
    for (uint64_t q = 0; q < s->p; q++)
        allocated += s->iout[q];
    /* Lemma 2: at least H unallocated blocks */
    uint64_t unalloc = s->n_pi - allocated;
    if (unalloc < s->st->min_unallocated)
        s->st->min_unallocated = unalloc;
    if (unalloc < s->H)
        return ORA_LEMMA2;
    /* S: prefix sum over C plus the head start, bucket-major, chunk-minor */
#if ORACLE_MUTANT == 2
    /* planted mistake: chunk-major order of the groups */
    {
        uint64_t acc = s->H;
        for (uint64_t q = 0; q < s->p; q++)
            for (uint32_t c = 0; c < sigma; c++) {
                s->S[(uint64_t)c * s->p + q] = acc;
                acc += s->C[(uint64_t)c * s->p + q];
            }
    }
#else
    s->S[0] = s->H;
    for (uint64_t g = 1; g < G; g++)
        s->S[g] = s->S[g - 1] + s->C[g - 1];
#endif
    /* unallocated blocks: each chunk's unused free-list tail, then pi[f..) */
    uint64_t nfree = 0, f_new = s->H + allocated;
    for (uint64_t q = 0; q < s->p; q++) {
        uint64_t fl_len = sigma + (s->lo[q + 1] - s->lo[q]);
        for (uint64_t k = s->iout[q]; k < fl_len; k++, nfree++) {
            uint64_t dst = nfree < s->H ? nfree : f_new + (nfree - s->H);
            s->pi2[dst] = free_list_entry(s, q, k);
        }
    }
    for (uint64_t i = s->f; i < s->n_pi; i++, nfree++) {
        uint64_t dst = nfree < s->H ? nfree : f_new + (nfree - s->H);
        s->pi2[dst] = s->pi[i];
    }
    if (nfree != unalloc)
        return ORA_INV_COUNT;
    /* shuffle used blocks into order of buckets; find the partial blocks */
    for (uint64_t q = 0; q < s->p; q++) {
        for (uint64_t k = 0; k < s->iout[q]; k++) {
            uint32_t c = s->U[q * s->U_stride + k];
            uint64_t g = (uint64_t)c * s->p + q;
            uint64_t phys = free_list_entry(s, q, k);
            s->pi2[s->S[g]] = phys;
            bucket_t *bk = &s->B[q * sigma + c];
            if (bk->end == blockat(s, phys) + s->b) { /* the open block? */
                s->P[g].idx = s->S[g];
                s->P[g].len = (uint64_t)(bk->next - blockat(s, phys));
#if ORACLE_MUTANT == 12
                if (s->P[g].len > 0) /* planted state mistake: fill one short */
                    s->P[g].len--;
#endif
            }
            s->S[g]++;
        }
    }
    s->nP = G;
    s->f = f_new;
#if ORACLE_MUTANT == 7
    if (G >= 2) { /* planted state mistake: two P entries exchanged */
        partial_t x = s->P[0];
        s->P[0] = s->P[G - 1];
        s->P[G - 1] = x;
    }
#elif ORACLE_MUTANT == 8
    s->f = f_new + 1; /* planted state mistake: f one past the last used block */
#elif ORACLE_MUTANT == 9
    s->pi2[0] = s->pi2[1]; /* planted state mistake: a block entered twice */
#endif
    uint64_t *tmp = s->pi;
    s->pi = s->pi2;
    s->pi2 = tmp;
    return check_invariant(s);
}

/* Alg. 7 (swap and finalize), readings G2, G3, G6 */
static void swap_blocks(rs_t *s, uint64_t *pinv, uint64_t i1, uint64_t j1, uint64_t i2, uint64_t j2)
{
    s->pi[i1] = j2;
    s->pi[i2] = j1;
    pinv[j1] = i2;
    pinv[j2] = i1;
}

static int finalize(rs_t *s)
{
    uint64_t H = s->H, nb = s->n / s->b, b = s->b;
    uint64_t *pinv = s->pi2; /* pi' reused for pi^-1 (Sec. 4) */
    uint64_t k = 0, iP = 0;
    uint64_t i_free = 0, j_free = s->pi[0]; /* unallocated as per invariant */
    for (uint64_t i = 0; i < s->n_pi; i++)
        pinv[s->pi[i]] = i;
    for (uint64_t i_in = H; i_in < H + nb; i_in++) {
        uint64_t j_in = s->pi[i_in];
        uint64_t j_out = s->tb + (i_in - H); /* A block i_in - H (reading G2) */
        uint64_t i_out = pinv[j_out];
        if (i_in < i_out && i_out < s->f) { /* occupied by a block still needed */
#if ORACLE_MUTANT != 4
            memcpy(blockat(s, j_free), blockat(s, j_out), b * sizeof(elem_t)); /* push */
#endif
            s->st->fin_copies_main++;
            s->st->fin_pushes++;
            swap_blocks(s, pinv, i_out, j_out, i_free, j_free);
            i_out = i_free; /* logical index now mapped to j_out (reading G3) */
        }
        uint64_t l = size_of_next_block(s, i_in, &iP);
#if ORACLE_MUTANT == 13
        /* planted mistake: the pull goes through a bounce block (the same
         * data lands in A, at one more block copy each) */
        memmove(s->bounce, blockat(s, j_in), l * sizeof(elem_t));
        s->st->fin_copies_main++;
        memmove(&s->A[k], s->bounce, l * sizeof(elem_t));
#else
        memmove(&s->A[k], blockat(s, j_in), l * sizeof(elem_t)); /* pull (G6) */
#endif
        s->st->fin_copies_main++;
        k += l;
        swap_blocks(s, pinv, i_out, j_out, i_in, j_in);
        if (i_in != i_out) { /* pulled from elsewhere: j_in is now free */
            i_free = i_out;
            j_free = j_in;
        }
    }
    /* reading G16: after a truncation (Alg. 8) physical A blocks nb .. hold
     * no data of the sequence's prefix, and a remaining block may sit in A
     * block nb, which the copies below overwrite (the untruncated sequence
     * has no A block nb).  Such a block is first pushed, as Alg. 7 pushes
     * occupants, to an unallocated block outside A[0 .. (nb+1)b). */
    uint64_t j_cut = s->tb + nb;
#if ORACLE_MUTANT == 15
    j_cut = s->n_pi; /* planted mistake: reading G16 left out */
#endif
    if (j_cut < s->n_pi && pinv[j_cut] >= H + nb && pinv[j_cut] < s->f) {
        uint64_t i_cut = pinv[j_cut], i_to = s->n_pi;
        for (uint64_t i = 0; i < s->n_pi && i_to == s->n_pi; i++)
            if ((i < H || i >= s->f) && (s->pi[i] < s->tb || s->pi[i] > j_cut))
                i_to = i;
        if (i_to == s->n_pi)
            return ORA_FIN_COUNT;
        uint64_t j_to = s->pi[i_to];
        memcpy(blockat(s, j_to), blockat(s, j_cut), b * sizeof(elem_t));
        s->st->fin_pushes++;
        s->st->fin_copies_trunc++;
        swap_blocks(s, pinv, i_cut, j_cut, i_to, j_to);
    }
    /* remaining blocks: in T, or (after a truncation) in A blocks past nb */
    for (uint64_t i_in = H + nb; i_in < s->f; i_in++) {
        uint64_t j_in = s->pi[i_in];
        uint64_t l = size_of_next_block(s, i_in, &iP);
        memmove(&s->A[k], blockat(s, j_in), l * sizeof(elem_t));
        s->st->fin_copies_rest++;
        k += l;
    }
    if (k != s->n)
        return ORA_FIN_COUNT;
    /* Sec. 3: at most two copies per A block, one per remaining block */
    if (s->st->fin_copies_main > 2 * nb || s->st->fin_copies_rest > s->f - H - nb)
        return ORA_FIN_COPIES;
    return ORA_OK;
}

/* the permuted representation read in logical order (Sec. 4.1 iterator) */
static void gather_sequence(rs_t *s, uint64_t *seq_keys, uint32_t *seq_vals)
{
    uint64_t iP = 0, k = 0;
    for (uint64_t i = s->H; i < s->f; i++) {
        elem_t *blk = blockat(s, s->pi[i]);
        uint64_t l = size_of_next_block(s, i, &iP);
        for (uint64_t j = 0; j < l; j++, k++) {
            if (seq_keys)
                seq_keys[k] = blk[j].key;
            if (seq_vals)
                seq_vals[k] = blk[j].val;
        }
    }
}

/* allocation of the state and setup (Alg. 4) on a copy of keys/vals */
static int rs_open(rs_t *s, ora_stats *st, const uint64_t *keys, const uint32_t *vals, size_t n,
                   int n_t, uint32_t sigma, int bits, size_t b, uint64_t p, uint64_t elem_bytes)
{
    keyspec ks = {n_t, sigma, bits};
    memset(st, 0, sizeof(*st));
    memset(s, 0, sizeof(*s));
    if (check_spec(&ks) != ORA_OK || b < 1 || p < 1)
        return ORA_EARG;
    s->ks = ks;
    s->n = n;
    s->b = b;
    s->p = p;
    s->H = (uint64_t)sigma * p;
    s->tb = 2 * s->H;
#if ORACLE_MUTANT == 11
    s->tb = 2 * s->H - 1; /* planted state mistake: one scratch block fewer */
#endif
    s->n_pi = n / b + s->tb;
    s->st = st;
    st->n_pi = s->n_pi;
    st->head = s->H;
    st->t_blocks = s->tb;
    st->min_unallocated = UINT64_MAX;
    uint64_t G = (uint64_t)sigma * p;
    s->U_stride = sigma + n / b + G + 2; /* >= sigma + longest chunk */
    s->A = malloc((n ? n : 1) * sizeof(elem_t));
    s->T = malloc(s->tb * b * sizeof(elem_t));
    s->bounce = malloc(b * sizeof(elem_t));
    s->pi = malloc(s->n_pi * sizeof(uint64_t));
    s->pi2 = malloc(s->n_pi * sizeof(uint64_t));
    s->P = malloc(G * sizeof(partial_t));
    s->lo = malloc((p + 1) * sizeof(uint64_t));
    s->C = malloc(G * sizeof(uint64_t));
    s->S = malloc(G * sizeof(uint64_t));
    s->B = malloc(G * sizeof(bucket_t));
    s->U = malloc(p * s->U_stride * sizeof(uint32_t));
    s->iout = malloc(p * sizeof(uint64_t));
    if (!s->A || !s->T || !s->pi || !s->pi2 || !s->P || !s->lo || !s->C || !s->S || !s->B ||
        !s->U || !s->iout || !s->bounce)
        return ORA_ENOMEM;
    /* Sec. 3/4 space: T, pi, pi' (reused as pi^-1), U, P, B, C, S */
    st->extra_bytes = s->tb * b * elem_bytes + s->n_pi * (4 + 4 + (sigma <= 256 ? 1 : 2)) +
                      G * (8 /*P*/ + 16 /*B*/ + 4 /*C*/ + 4 /*S*/);
    for (size_t i = 0; i < n; i++) {
        s->A[i].key = keys[i];
        s->A[i].val = vals ? vals[i] : 0;
    }
    return setup(s);
}

static void rs_close(rs_t *s)
{
    free(s->A), free(s->T), free(s->pi), free(s->pi2), free(s->P), free(s->lo);
    free(s->C), free(s->S), free(s->B), free(s->U), free(s->iout), free(s->bounce);
    memset(s, 0, sizeof(*s));
}

/* rounds first .. first+count-1 of Alg. 2's loop: sortPhase (Alg. 5) on
 * digit t = n_t-1-r, then fixupPhase (Alg. 6) */
static int run_rounds(rs_t *s, int first, int count)
{
    if (first < 0 || count < 0 || first + count > s->ks.n_t)
        return ORA_EARG;
    int err = ORA_OK;
    for (int r = first; r < first + count && !err; r++) {
        err = sort_phase(s, s->ks.n_t - 1 - r);
        if (!err)
            err = fixup_phase(s);
    }
    return err;
}

/*
 * Alg. 2 (radSort).  Runs setup and `rounds` rounds (t = n_t-1 downwards).
 * finalize != 0: Finalize, result in keys/vals (needs rounds == n_t for a
 * full sort, but any rounds value is accepted).
 * finalize == 0: the logical sequence after `rounds` rounds is written to
 * seq_keys/seq_vals (n entries each, nullable) and keys/vals are untouched.
 * elem_bytes only scales stats->extra_bytes.
 */
int ora_radsort(uint64_t *keys, uint32_t *vals, size_t n, int n_t, uint32_t sigma, int bits,
                size_t b, uint64_t p, int rounds, int do_finalize, uint64_t *seq_keys,
                uint32_t *seq_vals, uint64_t elem_bytes, ora_stats *st)
{
    ora_stats dummy;
    if (!st)
        st = &dummy;
    if (rounds < 0 || rounds > n_t) {
        memset(st, 0, sizeof(*st));
        return ORA_EARG;
    }
    rs_t s;
    int err = rs_open(&s, st, keys, vals, n, n_t, sigma, bits, b, p, elem_bytes);
    if (!err)
        err = run_rounds(&s, 0, rounds);
    if (!err) {
        if (do_finalize) {
            err = finalize(&s);
            for (size_t i = 0; !err && i < n; i++) {
                keys[i] = s.A[i].key;
                if (vals)
                    vals[i] = s.A[i].val;
            }
        } else {
            gather_sequence(&s, seq_keys, seq_vals);
        }
    }
    rs_close(&s);
    return err;
}

/* ======================================================================
 * The permuted representation kept between calls (Sec. 4.1): rounds on it,
 * truncation (Alg. 8), reading it in logical order, and a later Finalize.
 * ====================================================================== */
typedef struct {
    rs_t s;
    ora_stats st;
} perm_t;

/* setup (Alg. 4) on a copy of keys/vals; NULL on a bad argument or no memory */
void *ora_perm_new(const uint64_t *keys, const uint32_t *vals, size_t n, int n_t, uint32_t sigma,
                   int bits, size_t b, uint64_t p, uint64_t elem_bytes, int *err)
{
    perm_t *h = malloc(sizeof(perm_t));
    int e = h ? rs_open(&h->s, &h->st, keys, vals, n, n_t, sigma, bits, b, p, elem_bytes) : ORA_ENOMEM;
    if (e && h) {
        rs_close(&h->s);
        free(h);
        h = NULL;
    }
    if (err)
        *err = e;
    return h;
}

void ora_perm_free(void *hp)
{
    perm_t *h = hp;
    if (h) {
        rs_close(&h->s);
        free(h);
    }
}

int ora_perm_rounds(void *hp, int first, int count)
{
    perm_t *h = hp;
    return run_rounds(&h->s, first, count);
}

uint64_t ora_perm_count(void *hp)
{
    return ((perm_t *)hp)->s.n;
}

/* the logical sequence, n entries (Alg. 3 walk) */
void ora_perm_gather(void *hp, uint64_t *seq_keys, uint32_t *seq_vals)
{
    gather_sequence(&((perm_t *)hp)->s, seq_keys, seq_vals);
}

/*
 * Alg. 8: truncate the dataset so that logical block i, element j is the
 * final datum.  f becomes i+1 and the first partial block at or after i
 * becomes (i, j+1).  Readings:
 *   G15 the P entries after that one describe blocks past the new end and
 *       are dropped (nP = its index + 1); a cut at a block's last element
 *       (j+1 = b) leaves block i full, so logical block i+1 becomes the final
 *       block, partial with length 0 (clause 3 of the invariant, Sec. 2.2,
 *       wants block f-1 partial); the element count n is the count up to the
 *       cut.
 * ora_perm_truncate(h, m) keeps the first m <= n elements: (i, j) is the
 * position of element m-1 in the walk of Alg. 3; m = 0 leaves one empty
 * partial block at logical index H.
 */
static int truncate_at(rs_t *s, uint64_t i, uint64_t j, uint64_t m)
{
    s->f = i + 1; /* mark logical block i as the final block */
    for (uint64_t iP = 0; iP < s->nP; iP++) { /* skip partial blocks before i */
        if (i <= s->P[iP].idx) {
            s->P[iP].idx = i; /* logical block i ends at element j */
            s->P[iP].len = j + 1;
            s->nP = iP + 1;
#if ORACLE_MUTANT == 14
            s->nP = iP + 2 <= s->ks.sigma * s->p ? iP + 2 : iP + 1; /* planted: a stale entry kept */
#endif
            if (j + 1 == s->b) { /* reading G15: block i is full */
                s->P[iP].idx = i + 1;
                s->P[iP].len = 0;
                s->f = i + 2;
            }
            s->n = m;
            return check_invariant(s);
        }
    }
    return ORA_INV_PORDER; /* no partial block at or after i: not a valid state */
}

int ora_perm_truncate(void *hp, uint64_t m)
{
    rs_t *s = &((perm_t *)hp)->s;
    if (m > s->n)
        return ORA_EARG;
    if (m == 0) {
        s->f = s->H + 1;
        s->P[0].idx = s->H;
        s->P[0].len = 0;
        s->nP = 1;
        s->n = 0;
        return check_invariant(s);
    }
    uint64_t iP = 0, pos = 0;
    for (uint64_t i = s->H; i < s->f; i++) {
        uint64_t l = size_of_next_block(s, i, &iP);
        if (m - 1 < pos + l)
            return truncate_at(s, i, m - 1 - pos, m);
        pos += l;
    }
    return ORA_INV_COUNT;
}

/* Alg. 7 on the current state; keys/vals receive A[0..n) */
int ora_perm_finalize(void *hp, uint64_t *keys, uint32_t *vals)
{
    rs_t *s = &((perm_t *)hp)->s;
    int err = finalize(s);
    for (size_t i = 0; !err && i < s->n; i++) {
        keys[i] = s->A[i].key;
        if (vals)
            vals[i] = s->A[i].val;
    }
    return err;
}

void ora_perm_stats(void *hp, ora_stats *out)
{
    *out = ((perm_t *)hp)->st;
}

/* order-preserving bit transform of float32 keys (not in the paper): the
 * sign bit is flipped for non-negative values and every bit for negative
 * ones, so that unsigned order of the result is the IEEE total order. */
void ora_f32_to_ordered(uint32_t *u, size_t n)
{
    for (size_t i = 0; i < n; i++)
        u[i] ^= (u[i] & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u;
}

void ora_ordered_to_f32(uint32_t *u, size_t n)
{
    for (size_t i = 0; i < n; i++)
        u[i] ^= (u[i] & 0x80000000u) ? 0x80000000u : 0xFFFFFFFFu;
}

int ora_mutant_id(void) { return ORACLE_MUTANT; }
