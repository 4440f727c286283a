/*
 * sws_oracle.c -- plain CPU oracle for the sliding-window-sum hot path of
 * R. Snytsar and Y. Turakhia, "Parallel approach to sliding window sums" (arXiv 1811.10074).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Each function states, as directly as the
 * paper allows, what the GPU library computes, so that tests can compare the two element by
 * element.  It is deliberately slow and shares no code, header, table or constant with the
 * CUDA library.  Only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * load it.
 *
 * Conventions (the paper is silent on them; the readings are the project's):
 *   - DNA is 2-bit packed, A=0 C=1 G=2 T=3, base i in byte i>>2 at bits 2*(i&3).
 *     Complement of code b is 3-b.
 *   - The hash is T. Wang's 64-bit integer mix ("Integer Hash Function", 1997, rev. 2007),
 *     truncated to 2k bits after every step so that it is a bijection on [0, 4^k).
 *   - Minimizer keys are ordered by (value, position): ties go to the leftmost k-mer.
 *   - N-blocks are half-open base intervals; a window whose bases touch one is dropped and
 *     each maximal N-free run is handled as a sequence of its own.
 *
 * Every function carries the passage it follows.  Nothing here is blocked, fused or reordered.
 */
#include <stdint.h>
#include <stddef.h>
#include <stdlib.h>
#include <string.h>

/* Operator codes of this oracle (its own numbering; the Python wrapper maps names). */
enum {
    ORC_ADD_I32 = 0,    /* + mod 2^32 on int32 bit patterns   */
    ORC_MIN_I32 = 1,    /* signed minimum                      */
    ORC_MAX_I32 = 2,    /* signed maximum                      */
    ORC_XOR_I32 = 3,    /* bitwise exclusive or                */
    ORC_AFFINE_U32 = 4, /* composition of x -> a*x+b mod 2^32  */
    ORC_ADD_F32 = 5     /* real addition of fp32 inputs, in fp64 */
};

/* ------------------------------------------------------------------------------------------
 * Eq. 2 (Sec. 2.2): y_p = x_p (+) x_{p+1} (+) ... (+) x_{p+w-1}, each sum exactly w addends,
 * evaluated naively, left to right -- the O(wN) sum the paper calls naive.  Outputs are
 * y_0 .. y_{n-w}.
 * ---------------------------------------------------------------------------------------- */

/* One window of Eq. 2 for operator op; x is the raw element array (4 or 8 bytes per element). */
static void window_sum(int op, const void *x, uint64_t p, int w, void *y)
{
    int j;
    if (op == ORC_ADD_I32) {
        const uint32_t *v = (const uint32_t *)x;
        uint32_t acc = v[p];
        for (j = 1; j < w; ++j) acc = acc + v[p + j];
        *(uint32_t *)y = acc;
    } else if (op == ORC_MIN_I32) {
        const int32_t *v = (const int32_t *)x;
        int32_t acc = v[p];
        for (j = 1; j < w; ++j) acc = v[p + j] < acc ? v[p + j] : acc;
        *(int32_t *)y = acc;
    } else if (op == ORC_MAX_I32) {
        const int32_t *v = (const int32_t *)x;
        int32_t acc = v[p];
        for (j = 1; j < w; ++j) acc = v[p + j] > acc ? v[p + j] : acc;
        *(int32_t *)y = acc;
    } else if (op == ORC_XOR_I32) {
        const uint32_t *v = (const uint32_t *)x;
        uint32_t acc = v[p];
        for (j = 1; j < w; ++j) acc = acc ^ v[p + j];
        *(uint32_t *)y = acc;
    } else if (op == ORC_AFFINE_U32) {
        /* Element = map f(x) = a*x + b (mod 2^32).  acc (+) f means "apply acc, then f":
         * f(acc(x)) = a*(A*x + B) + b = (a*A)*x + (a*B + b).  The window sum is the map
         * f_{p+w-1} o ... o f_p, so the leftmost addend is applied first. */
        const uint32_t *v = (const uint32_t *)x;
        uint32_t A = v[2 * p], B = v[2 * p + 1];
        for (j = 1; j < w; ++j) {
            uint32_t a = v[2 * (p + j)], b = v[2 * (p + j) + 1];
            uint32_t nA = a * A;
            uint32_t nB = a * B + b;
            A = nA;
            B = nB;
        }
        ((uint32_t *)y)[0] = A;
        ((uint32_t *)y)[1] = B;
    } else { /* ORC_ADD_F32: exact-as-possible reference, accumulated in fp64 */
        const float *v = (const float *)x;
        double acc = (double)v[p];
        for (j = 1; j < w; ++j) acc = acc + (double)v[p + j];
        *(double *)y = acc;
    }
}

static size_t out_size(int op) { return (op == ORC_AFFINE_U32 || op == ORC_ADD_F32) ? 8 : 4; }

/* All n-w+1 outputs of Eq. 2.  Returns the number written (0 when n < w or w < 1). */
uint64_t oracle_sliding_sum(int op, int w, const void *x, uint64_t n, void *y)
{
    uint64_t p, m;
    if (w < 1 || n < (uint64_t)w) return 0;
    m = n - (uint64_t)w + 1;
    for (p = 0; p < m; ++p) window_sum(op, x, p, w, (char *)y + p * out_size(op));
    return m;
}

/* Eq. 2 at chosen output indices only (for spot checks of very long inputs). */
void oracle_sliding_sum_at(int op, int w, const void *x, uint64_t n, const uint64_t *idx, uint64_t m, void *y)
{
    uint64_t i;
    (void)n;
    for (i = 0; i < m; ++i) window_sum(op, x, idx[i], w, (char *)y + i * out_size(op));
}

/* ------------------------------------------------------------------------------------------
 * k-mers (Sec. 2.4): the k-mer at position i is the sliding sum over k bases with string
 * concatenation, r_i r_{i+1} ... r_{i+k-1}.  As a number in base 4 the first base is the most
 * significant digit, so numeric order equals lexicographic order of the strings.
 * ---------------------------------------------------------------------------------------- */

static int base_at(const uint8_t *s, uint64_t i) { return (s[i >> 2] >> (2 * (i & 3))) & 3; }

/* Forward k-mer: the string r_i .. r_{i+k-1} read as a base-4 number. */
static uint64_t kmer_forward(const uint8_t *s, uint64_t i, int k)
{
    uint64_t v = 0;
    int j;
    for (j = 0; j < k; ++j) v = v * 4 + (uint64_t)base_at(s, i + j);
    return v;
}

/* Reverse complement: the string comp(r_{i+k-1}) .. comp(r_i) read as a base-4 number. */
static uint64_t kmer_revcomp(const uint8_t *s, uint64_t i, int k)
{
    uint64_t v = 0;
    int j;
    for (j = k - 1; j >= 0; --j) v = v * 4 + (uint64_t)(3 - base_at(s, i + j));
    return v;
}

static uint64_t low_mask(int bits) { return bits >= 64 ? ~(uint64_t)0 : (((uint64_t)1 << bits) - 1); }

/* Wang's 64-bit mix with every step truncated to `bits` bits (a bijection on [0, 2^bits)). */
uint64_t oracle_hash(uint64_t key, int bits)
{
    uint64_t m = low_mask(bits);
    key &= m;
    key = (~key + (key << 21)) & m;
    key = key ^ (key >> 24);
    key = (key + (key << 3) + (key << 8)) & m;
    key = key ^ (key >> 14);
    key = (key + (key << 2) + (key << 4)) & m;
    key = key ^ (key >> 28);
    key = (key + (key << 31)) & m;
    return key;
}

/* Multiplicative inverse of an odd number modulo 2^64 (Newton's iteration). */
static uint64_t inv_odd(uint64_t a)
{
    uint64_t x = a; /* correct to 3 bits */
    int i;
    for (i = 0; i < 6; ++i) x = x * (2 - a * x);
    return x;
}

/* Inverse of y = x ^ (x >> s) restricted to `bits` bits. */
static uint64_t unxorshift(uint64_t y, int s, int bits)
{
    uint64_t x = y;
    int i;
    for (i = 0; i * s < bits + s; ++i) x = y ^ (x >> s);
    return x;
}

/* Inverse of oracle_hash on [0, 2^bits); used to pin that the hash is a bijection. */
uint64_t oracle_hash_inv(uint64_t h, int bits)
{
    uint64_t m = low_mask(bits);
    uint64_t x = h & m;
    x = (x * inv_odd(((uint64_t)1 << 31) + 1)) & m;
    x = unxorshift(x, 28, bits) & m;
    x = (x * inv_odd(21)) & m;
    x = unxorshift(x, 14, bits) & m;
    x = (x * inv_odd(265)) & m;
    x = unxorshift(x, 24, bits) & m;
    x = ((x + 1) * inv_odd(((uint64_t)1 << 21) - 1)) & m;
    return x;
}

/* 1 if oracle_hash is a bijection on [0, 2^bits) (exhaustive, bits <= 32). */
int oracle_hash_is_bijection(int bits)
{
    uint64_t size = (uint64_t)1 << bits, x;
    uint8_t *seen = (uint8_t *)calloc((size_t)((size + 7) / 8), 1);
    int ok = 1;
    if (!seen) return -1;
    for (x = 0; x < size; ++x) {
        uint64_t h = oracle_hash(x, bits);
        if (h >= size || (seen[h >> 3] >> (h & 7)) & 1) { ok = 0; break; }
        seen[h >> 3] |= (uint8_t)(1u << (h & 7));
    }
    free(seen);
    return ok;
}

/* k-mer value kinds for oracle_kmers. */
enum { ORC_KMER_FWD = 0, ORC_KMER_RC = 1, ORC_KMER_CANON = 2, ORC_KMER_HASH = 3 };

static uint64_t kmer_value(const uint8_t *s, uint64_t i, int k, int kind)
{
    uint64_t f, r, c;
    f = kmer_forward(s, i, k);
    if (kind == ORC_KMER_FWD) return f;
    r = kmer_revcomp(s, i, k);
    if (kind == ORC_KMER_RC) return r;
    c = f < r ? f : r;
    if (kind == ORC_KMER_CANON) return c;
    return oracle_hash(c, 2 * k);
}

/* Values of all n-k+1 k-mers of one kind (uint64 each).  Returns the count written. */
uint64_t oracle_kmers(const uint8_t *s, uint64_t n, int k, int kind, uint64_t *out)
{
    uint64_t i, m;
    if (k < 1 || k > 32 || n < (uint64_t)k) return 0;
    m = n - (uint64_t)k + 1;
    for (i = 0; i < m; ++i) out[i] = kmer_value(s, i, k, kind);
    return m;
}

/* ------------------------------------------------------------------------------------------
 * Minimizers (Sec. 2.4): for each window position p, the w consecutive k-mers starting at p
 * are compared and the minimum seed s with its position p' is recorded; adjacent windows that
 * share the same (s, p') store it once.  Keys here: ORC_MINI_HASH = hash of the canonical
 * k-mer (the measured workload uses hashed 15-mers), ORC_MINI_CANON = canonical k-mer,
 * ORC_MINI_FWD = forward k-mer (the lexicographic seeds of the paper's example).
 * ---------------------------------------------------------------------------------------- */
enum { ORC_MINI_HASH = 0, ORC_MINI_CANON = 1, ORC_MINI_FWD = 2 };

static uint64_t mini_key(const uint8_t *s, uint64_t i, int k, int mode)
{
    if (mode == ORC_MINI_FWD) return kmer_value(s, i, k, ORC_KMER_FWD);
    if (mode == ORC_MINI_CANON) return kmer_value(s, i, k, ORC_KMER_CANON);
    return kmer_value(s, i, k, ORC_KMER_HASH);
}

typedef struct {
    uint64_t *hash_out;
    uint32_t *pos_out;
    uint64_t cap;
    uint64_t count;
} sink_t;

static void sink_put(sink_t *o, uint64_t key, uint64_t pos)
{
    if (o->count < o->cap) {
        o->hash_out[o->count] = key;
        o->pos_out[o->count] = (uint32_t)pos;
    }
    o->count++;
}

/* Minimizers of one N-free stretch [a, b): naive O(w) scan per window.  Positions are
 * reported as (k-mer start - pos_base). */
static void run_minimizers_naive(const uint8_t *s, uint64_t a, uint64_t b, int k, int w, int mode,
                                 uint64_t pos_base, sink_t *o)
{
    uint64_t nk, p, j, best, last = 0;
    uint64_t *key;
    int have_last = 0;
    if (b - a < (uint64_t)(k + w - 1)) return;
    nk = b - a - (uint64_t)k + 1;
    key = (uint64_t *)malloc((size_t)nk * sizeof(uint64_t));
    for (j = 0; j < nk; ++j) key[j] = mini_key(s, a + j, k, mode);
    for (p = 0; p + (uint64_t)w <= nk; ++p) {
        best = p;
        for (j = p + 1; j < p + (uint64_t)w; ++j)
            if (key[j] < key[best]) best = j; /* strict: the leftmost minimum wins */
        if (!have_last || best != last) sink_put(o, key[best], a + best - pos_base);
        last = best;
        have_last = 1;
    }
    free(key);
}

/* The same stretch with the queue-based O(N) sliding minimum the paper cites (Sec. 2.4):
 * a deque of k-mer indices whose keys never decrease from front to back. */
static void run_minimizers_deque(const uint8_t *s, uint64_t a, uint64_t b, int k, int w, int mode,
                                 uint64_t pos_base, sink_t *o)
{
    uint64_t nk, j, head = 0, tail = 0, last = 0;
    uint64_t *key, *dq;
    int have_last = 0;
    if (b - a < (uint64_t)(k + w - 1)) return;
    nk = b - a - (uint64_t)k + 1;
    key = (uint64_t *)malloc((size_t)nk * sizeof(uint64_t));
    dq = (uint64_t *)malloc((size_t)nk * sizeof(uint64_t));
    for (j = 0; j < nk; ++j) key[j] = mini_key(s, a + j, k, mode);
    for (j = 0; j < nk; ++j) {
        while (tail > head && key[dq[tail - 1]] > key[j]) tail--; /* equal keys stay: leftmost wins */
        dq[tail++] = j;
        if (j + 1 >= (uint64_t)w) {
            uint64_t p = j + 1 - (uint64_t)w;
            while (dq[head] < p) head++;
            if (!have_last || dq[head] != last) sink_put(o, key[dq[head]], a + dq[head] - pos_base);
            last = dq[head];
            have_last = 1;
        }
    }
    free(dq);
    free(key);
}

/* Whole-sequence minimizers with N-blocks: every maximal stretch of bases outside the
 * intervals nb[2i]..nb[2i+1] (half-open) is processed on its own.  Returns the total count;
 * at most cap picks are stored.  use_deque selects the queue-based scan. */
uint64_t oracle_minimizers(const uint8_t *s, uint64_t n, int k, int w, int mode, const int64_t *nb,
                           uint64_t n_nb, uint64_t *hash_out, uint32_t *pos_out, uint64_t cap, int use_deque)
{
    sink_t o;
    uint8_t *isn;
    uint64_t i, a;
    o.hash_out = hash_out;
    o.pos_out = pos_out;
    o.cap = cap;
    o.count = 0;
    if (k < 1 || k > 32 || w < 1 || n == 0) return 0;
    isn = (uint8_t *)calloc((size_t)n, 1);
    for (i = 0; i < n_nb; ++i) {
        int64_t lo = nb[2 * i], hi = nb[2 * i + 1], t;
        if (lo < 0) lo = 0;
        if (hi > (int64_t)n) hi = (int64_t)n;
        for (t = lo; t < hi; ++t) isn[t] = 1;
    }
    a = 0;
    while (a < n) {
        uint64_t b;
        if (isn[a]) { a++; continue; }
        b = a;
        while (b < n && !isn[b]) b++;
        if (use_deque) run_minimizers_deque(s, a, b, k, w, mode, 0, &o);
        else run_minimizers_naive(s, a, b, k, w, mode, 0, &o);
        a = b;
    }
    free(isn);
    return o.count;
}

/* A batch of reads stored back to back in one packed stream: read r is bases
 * [offs[r], offs[r+1]).  Each read is an independent sequence; positions are read-local.
 * pick_offs[r] receives the index of read r's first pick (pick_offs[nreads] = total). */
uint64_t oracle_minimizers_batch(const uint8_t *s, const int64_t *offs, uint64_t nreads, int k, int w, int mode,
                                 uint64_t *hash_out, uint32_t *pos_out, uint64_t cap, uint64_t *pick_offs)
{
    sink_t o;
    uint64_t r;
    o.hash_out = hash_out;
    o.pos_out = pos_out;
    o.cap = cap;
    o.count = 0;
    for (r = 0; r < nreads; ++r) {
        pick_offs[r] = o.count;
        run_minimizers_naive(s, (uint64_t)offs[r], (uint64_t)offs[r + 1], k, w, mode, (uint64_t)offs[r], &o);
    }
    pick_offs[nreads] = o.count;
    return o.count;
}

/* Paper-equivalent task (Sec. 4): sliding minimum over a precomputed array of hashed k-mers,
 * with (value, position) keys and consecutive duplicates stored once. */
uint64_t oracle_minimizers_from_keys(const uint64_t *key, uint64_t m, int w, uint64_t *hash_out, uint32_t *pos_out,
                                     uint64_t cap)
{
    sink_t o;
    uint64_t p, j, best, last = 0;
    int have_last = 0;
    o.hash_out = hash_out;
    o.pos_out = pos_out;
    o.cap = cap;
    o.count = 0;
    if (w < 1 || m < (uint64_t)w) return 0;
    for (p = 0; p + (uint64_t)w <= m; ++p) {
        best = p;
        for (j = p + 1; j < p + (uint64_t)w; ++j)
            if (key[j] < key[best]) best = j;
        if (!have_last || best != last) sink_put(&o, key[best], best);
        last = best;
        have_last = 1;
    }
    return o.count;
}

/* The same task with the queue-based O(N) sliding minimum the paper times as "Dequeue" (Sec. 4,
 * after the method it cites in Sec. 2.4): a deque of key indices whose keys never decrease from
 * front to back; the front is the window's leftmost least key. */
uint64_t oracle_minimizers_from_keys_deque(const uint64_t *key, uint64_t m, int w, uint64_t *hash_out,
                                           uint32_t *pos_out, uint64_t cap)
{
    sink_t o;
    uint64_t i, front = 0, back = 0, prev = 0;
    uint64_t *q;
    int have_prev = 0;
    o.hash_out = hash_out;
    o.pos_out = pos_out;
    o.cap = cap;
    o.count = 0;
    if (w < 1 || m < (uint64_t)w) return 0;
    q = (uint64_t *)malloc((size_t)m * sizeof(uint64_t));
    for (i = 0; i < m; ++i) {
        /* drop queued candidates that the new key beats; an equal key keeps the older one */
        while (back > front && key[q[back - 1]] > key[i]) back--;
        q[back++] = i;
        if (i + 1 >= (uint64_t)w) {
            const uint64_t start = i + 1 - (uint64_t)w; /* window [start, i] */
            while (q[front] < start) front++;           /* candidates that left the window */
            if (!have_prev || q[front] != prev) sink_put(&o, key[q[front]], q[front]);
            prev = q[front];
            have_prev = 1;
        }
    }
    free(q);
    return o.count;
}

/* ------------------------------------------------------------------------------------------
 * Seed table (Sec. 2.4): a position table of (seed, position) hits sorted by seed, and a
 * pointer table giving, for every bucket of seed values, where its hits begin.  Bucket of a
 * hash h with hash_bits bits: h >> (hash_bits - bucket_bits) (h itself when equal).
 * ---------------------------------------------------------------------------------------- */
typedef struct {
    uint64_t h;
    uint32_t p;
} pair_t;

static int pair_cmp(const void *x, const void *y)
{
    const pair_t *a = (const pair_t *)x, *b = (const pair_t *)y;
    if (a->h != b->h) return a->h < b->h ? -1 : 1;
    if (a->p != b->p) return a->p < b->p ? -1 : 1;
    return 0;
}

int oracle_kmer_table(const uint64_t *hash, const uint32_t *pos, uint64_t m, int hash_bits, int bucket_bits,
                      uint64_t *sorted_hash, uint32_t *sorted_pos, uint64_t *offsets)
{
    pair_t *t;
    uint64_t i, nb, b;
    int shift;
    if (bucket_bits < 0 || bucket_bits > hash_bits || bucket_bits > 34) return -1;
    t = (pair_t *)malloc((size_t)(m ? m : 1) * sizeof(pair_t));
    for (i = 0; i < m; ++i) {
        t[i].h = hash[i];
        t[i].p = pos[i];
    }
    qsort(t, (size_t)m, sizeof(pair_t), pair_cmp);
    for (i = 0; i < m; ++i) {
        sorted_hash[i] = t[i].h;
        sorted_pos[i] = t[i].p;
    }
    nb = (uint64_t)1 << bucket_bits;
    shift = hash_bits - bucket_bits;
    memset(offsets, 0, (size_t)(nb + 1) * sizeof(uint64_t));
    for (i = 0; i < m; ++i) offsets[(t[i].h >> shift) + 1]++; /* counts, shifted by one */
    for (b = 0; b < nb; ++b) offsets[b + 1] += offsets[b];      /* running total = start of next */
    free(t);
    return 0;
}

/* Seed hits of the seeding stage (Sec. 2.3), through the seed table of Sec. 2.4 (Fig. 1): the
 * hits of query seed i (hash qh[i]) are the reference positions j whose seed hash equals qh[i].
 * A seed with more than max_occ hits is skipped (max_occ = 0: no limit), the usual filter for
 * repeats.  count[i] receives the number of hits of query i before the filter.  The kept hits are
 * written as (i, position) pairs in increasing i and, per query, increasing position; at most
 * cap are written.  Returns the number of kept hits.  Steps: sort the reference's (hash, pos)
 * pairs (the position table), then a binary search for each query's equal run. */
uint64_t oracle_seed_hits(const uint64_t *ref_hash, const uint32_t *ref_pos, uint64_t m, const uint64_t *qh,
                          uint64_t nq, uint32_t max_occ, uint32_t *count, uint32_t *hit_query, uint32_t *hit_pos,
                          uint64_t cap)
{
    pair_t *t;
    uint64_t i, j, lo, hi, mid, a, out = 0;
    t = (pair_t *)malloc((size_t)(m ? m : 1) * sizeof(pair_t));
    for (i = 0; i < m; ++i) {
        t[i].h = ref_hash[i];
        t[i].p = ref_pos[i];
    }
    qsort(t, (size_t)m, sizeof(pair_t), pair_cmp);
    for (i = 0; i < nq; ++i) {
        lo = 0; /* first index with hash >= qh[i] */
        hi = m;
        while (lo < hi) {
            mid = lo + (hi - lo) / 2;
            if (t[mid].h < qh[i]) lo = mid + 1;
            else hi = mid;
        }
        a = lo;
        while (a < m && t[a].h == qh[i]) ++a;
        count[i] = (uint32_t)(a - lo);
        if (max_occ != 0 && a - lo > max_occ) continue;
        for (j = lo; j < a; ++j, ++out) {
            if (out < cap) {
                hit_query[out] = (uint32_t)i;
                hit_pos[out] = t[j].p;
            }
        }
    }
    free(t);
    return out;
}

/* Strand of a minimizer pick (Sec. 2.4; minimizers over canonical k-mers pick min(forward,
 * reverse complement)): 0 when the forward k-mer at the pick is the smaller or they are equal (a
 * palindrome), 1 when its reverse complement is the smaller.  Picks of one sequence (offs = NULL:
 * base = pos[i]) or of a read batch (read r holds picks pick_offs[r] .. pick_offs[r+1]-1 and
 * starts at base offs[r]; pos is read-local).  A pick whose k-mer does not lie inside the
 * sequence gets 255. */
void oracle_strands(const uint8_t *s, uint64_t n, int k, const int64_t *offs, const uint64_t *pick_offs, uint64_t nreads,
                    const uint32_t *pos, uint64_t m, uint8_t *strand)
{
    uint64_t i, r = 0, base, f, rc;
    int j, b;
    for (i = 0; i < m; ++i) {
        base = pos[i];
        if (offs) {
            while (r + 1 < nreads && pick_offs[r + 1] <= i) ++r;
            base += (uint64_t)offs[r];
        }
        if (base + (uint64_t)k > n) {
            strand[i] = 255;
            continue;
        }
        f = 0;
        rc = 0;
        for (j = 0; j < k; ++j) {
            b = base_at(s, base + (uint64_t)j);
            f = f * 4 + (uint64_t)b;                    /* first base most significant */
            rc = rc + ((uint64_t)(3 - b) << (2 * j));  /* complement, read backwards */
        }
        strand[i] = rc < f ? 1 : 0;
    }
}
