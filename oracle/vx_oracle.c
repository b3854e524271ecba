/*
 * vx_oracle.c -- plain, slow, CPU reference of the VaultxGPU plotting path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file: only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header or constant table with the CUDA
 * path under paper_2606_14007_gb300/csrc.
 *
 * What it computes (paper: Sec. II-B, four-stage VaultX pipeline; Sec. III-A
 * and III-B, GPU semantics), with every unstated detail fixed by a numbered
 * reading (R1..R11) that the design notes list:
 *
 *   Table 1  For every nonce n in [0, 2^K): h = BLAKE3-keyed(key, LE32(n)),
 *            record = {LE32 nonce, h[0..7]} (12 bytes; R1, R3, R4).
 *            Records are sorted by (key64, nonce), key64 = big-endian u64 of
 *            h[0..7]; logical bucket = key64 >> 40, 2^24 buckets (R5, R6).
 *   Table 2  Inside each logical bucket, every pair i < j (Table-1 order)
 *            with key64_j - key64_i < D, D = 2^(64-K) by default (R8, R9),
 *            emits {LE32 a, LE32 b, hash2[0..7]} where
 *            hash2 = BLAKE3-keyed(key, LE32(a) || LE32(b)) (R10), in bucket,
 *            then i, then j order (R11).  A cross-bucket variant
 *            (orc_match_global) takes every pair of the whole Table-1 order
 *            under the same threshold.
 *
 * BLAKE3 here is the single-block, single-chunk case of the BLAKE3
 * specification (messages of at most 64 bytes), which is all the plotter
 * needs.  Pinning status: the G function, the round's column/diagonal
 * pattern and the IV are pinned against hashlib's BLAKE2s, which shares
 * them; the whole compression (message permutation, counter, block-length
 * and flag words, output fold) reproduces the published BLAKE3 digests of
 * the empty input and of "abc"; the keyed mode is that compression with the
 * key as chaining value and the KEYED_HASH flag (tests/test_oracle_pins.py).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* BLAKE3 compression (BLAKE3 specification, Sec. 2.2)                 */
/* ------------------------------------------------------------------ */

/* The eight IV words are the SHA-256 initial hash values, as in BLAKE2s. */
static const uint32_t ORC_IV[8] = {
    0x6A09E667u, 0xBB67AE85u, 0x3C6EF372u, 0xA54FF53Au,
    0x510E527Fu, 0x9B05688Cu, 0x1F83D9ABu, 0x5BE0CD19u};

/* Message word permutation applied between rounds. */
static const int ORC_PERM[16] = {2, 6, 3, 10, 7, 0, 4, 13, 1, 11, 12, 5, 9, 14, 15, 8};

/* Domain-separation flags. */
enum {
    ORC_CHUNK_START = 1u << 0,
    ORC_CHUNK_END = 1u << 1,
    ORC_PARENT = 1u << 2,
    ORC_ROOT = 1u << 3,
    ORC_KEYED_HASH = 1u << 4,
};

static uint32_t rotr32(uint32_t x, int n) { return (x >> n) | (x << (32 - n)); }

/* The quarter-round G: two message words mixed into four state words. */
static void orc_g(uint32_t v[16], int a, int b, int c, int d, uint32_t mx, uint32_t my)
{
    v[a] = v[a] + v[b] + mx;
    v[d] = rotr32(v[d] ^ v[a], 16);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 12);
    v[a] = v[a] + v[b] + my;
    v[d] = rotr32(v[d] ^ v[a], 8);
    v[c] = v[c] + v[d];
    v[b] = rotr32(v[b] ^ v[c], 7);
}

/* One round: G on the four columns, then on the four diagonals, consuming
 * the sixteen message words in slot order. */
void orc_round(uint32_t v[16], const uint32_t m[16])
{
    orc_g(v, 0, 4, 8, 12, m[0], m[1]);
    orc_g(v, 1, 5, 9, 13, m[2], m[3]);
    orc_g(v, 2, 6, 10, 14, m[4], m[5]);
    orc_g(v, 3, 7, 11, 15, m[6], m[7]);
    orc_g(v, 0, 5, 10, 15, m[8], m[9]);
    orc_g(v, 1, 6, 11, 12, m[10], m[11]);
    orc_g(v, 2, 7, 8, 13, m[12], m[13]);
    orc_g(v, 3, 4, 9, 14, m[14], m[15]);
}

void orc_iv(uint32_t out[8])
{
    for (int i = 0; i < 8; i++) out[i] = ORC_IV[i];
}

/* Full compression: 7 rounds, the message permuted after each of the first
 * six; output word i = v[i] ^ v[i+8] and word i+8 = v[i+8] ^ cv[i]. */
void orc_compress(const uint32_t cv[8], const uint32_t block[16], uint64_t counter,
                  uint32_t block_len, uint32_t flags, uint32_t out[16])
{
    uint32_t v[16], m[16], t[16];
    for (int i = 0; i < 8; i++) v[i] = cv[i];
    for (int i = 0; i < 4; i++) v[8 + i] = ORC_IV[i];
    v[12] = (uint32_t)counter;
    v[13] = (uint32_t)(counter >> 32);
    v[14] = block_len;
    v[15] = flags;
    memcpy(m, block, sizeof m);
    for (int r = 0; r < 7; r++) {
        orc_round(v, m);
        if (r < 6) {
            for (int i = 0; i < 16; i++) t[i] = m[ORC_PERM[i]];
            memcpy(m, t, sizeof m);
        }
    }
    for (int i = 0; i < 8; i++) {
        out[i] = v[i] ^ v[i + 8];
        out[i + 8] = v[i + 8] ^ cv[i];
    }
}

static uint32_t load_le32(const uint8_t *p)
{
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}

static void store_le32(uint8_t *p, uint32_t x)
{
    p[0] = (uint8_t)x;
    p[1] = (uint8_t)(x >> 8);
    p[2] = (uint8_t)(x >> 16);
    p[3] = (uint8_t)(x >> 24);
}

/* BLAKE3 keyed_hash of a message of at most 64 bytes: one chunk holding one
 * block, so the chaining value is the key itself, the counter is 0 and the
 * block carries CHUNK_START | CHUNK_END | ROOT | KEYED_HASH.  Writes up to 32
 * output bytes.  Returns 0, or -1 for an unsupported length. */
int orc_keyed_hash(const uint8_t key[32], const uint8_t *msg, size_t len,
                   uint8_t *out, size_t out_len)
{
    if (len > 64 || out_len > 32) return -1;
    uint8_t buf[64];
    memset(buf, 0, sizeof buf);
    if (len) memcpy(buf, msg, len);
    uint32_t cv[8], block[16], o[16];
    for (int i = 0; i < 8; i++) cv[i] = load_le32(key + 4 * i);
    for (int i = 0; i < 16; i++) block[i] = load_le32(buf + 4 * i);
    orc_compress(cv, block, 0, (uint32_t)len,
                 ORC_CHUNK_START | ORC_CHUNK_END | ORC_ROOT | ORC_KEYED_HASH, o);
    uint8_t full[32];
    for (int i = 0; i < 8; i++) store_le32(full + 4 * i, o[i]);
    memcpy(out, full, out_len);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Table 1 (paper Sec. II-B hash stage, Sec. III-A/III-B)              */
/* ------------------------------------------------------------------ */

/* key64 of a 12-byte record: the 8 hash bytes read as a big-endian u64 (R5). */
static uint64_t rec_key64(const uint8_t *rec)
{
    uint64_t k = 0;
    for (int i = 0; i < 8; i++) k = (k << 8) | rec[4 + i];
    return k;
}

static uint32_t rec_nonce(const uint8_t *rec) { return load_le32(rec); }

/* One record: LE32 nonce followed by the first 8 bytes of its keyed hash
 * (R1, R3, R4). */
static void make_record(const uint8_t key[32], uint32_t nonce, uint8_t *rec)
{
    uint8_t msg[4];
    store_le32(msg, nonce);
    store_le32(rec, nonce);
    orc_keyed_hash(key, msg, 4, rec + 4, 8);
}

/* Hash stage: records in nonce order (no bucketing yet). */
int orc_table1_unsorted(int K, const uint8_t key[32], uint8_t *recs)
{
    if (K < 1 || K > 32) return -1;
    uint64_t n = 1ull << K;
    for (uint64_t i = 0; i < n; i++) make_record(key, (uint32_t)i, recs + 12 * i);
    return 0;
}

struct hash_job {
    const uint8_t *key;
    uint8_t *recs; /* record of nonce i goes to recs + 12 * (i - base) */
    uint64_t base, lo, hi;
};

static void *hash_job_run(void *arg)
{
    struct hash_job *j = (struct hash_job *)arg;
    for (uint64_t i = j->lo; i < j->hi; i++)
        make_record(j->key, (uint32_t)i, j->recs + 12 * (i - j->base));
    return NULL;
}

/* Same as orc_table1_unsorted over a nonce range [lo, hi), split across
 * nthreads POSIX threads (the VaultX CPU plotter's threading, Sec. II-B).
 * recs receives hi - lo records, the one of nonce lo first. */
int orc_hash_range_mt(const uint8_t key[32], uint64_t lo, uint64_t hi, uint8_t *recs, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t tid[512];
    int started[512];
    struct hash_job jobs[512];
    uint64_t span = hi - lo;
    for (int t = 0; t < nthreads; t++) {
        jobs[t].key = key;
        jobs[t].recs = recs;
        jobs[t].base = lo;
        jobs[t].lo = lo + span * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = lo + span * (uint64_t)(t + 1) / (uint64_t)nthreads;
        started[t] = pthread_create(&tid[t], NULL, hash_job_run, &jobs[t]) == 0;
        if (!started[t]) hash_job_run(&jobs[t]);
    }
    for (int t = 0; t < nthreads; t++)
        if (started[t]) pthread_join(tid[t], NULL);
    return 0;
}

/* Sort order of Table 1: key64 ascending, ties by nonce ascending (R6). */
static int rec_cmp(const void *pa, const void *pb)
{
    const uint8_t *a = (const uint8_t *)pa, *b = (const uint8_t *)pb;
    uint64_t ka = rec_key64(a), kb = rec_key64(b);
    if (ka != kb) return ka < kb ? -1 : 1;
    uint32_t na = rec_nonce(a), nb = rec_nonce(b);
    if (na != nb) return na < nb ? -1 : 1;
    return 0;
}

/* Sort stage: with the records in (key64, nonce) order, logical buckets
 * 0 .. 2^24-1 come out concatenated, each sorted (R6). */
int orc_sort_table1(uint8_t *recs, uint64_t n)
{
    qsort(recs, (size_t)n, 12, rec_cmp);
    return 0;
}

/* Hash + sort: the finished Table 1. */
int orc_table1(int K, const uint8_t key[32], uint8_t *t1)
{
    int rc = orc_table1_unsorted(K, key, t1);
    if (rc) return rc;
    return orc_sort_table1(t1, 1ull << K);
}

/* offsets[b] = number of records whose logical bucket is below b, for
 * b = 0 .. 2^24 (R6).  Computed by counting, then a running sum. */
int orc_bucket_offsets(const uint8_t *t1, uint64_t n, uint64_t *offsets)
{
    const uint64_t nb = 1ull << 24;
    memset(offsets, 0, (nb + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < n; i++) offsets[(rec_key64(t1 + 12 * i) >> 40) + 1]++;
    for (uint64_t b = 0; b < nb; b++) offsets[b + 1] += offsets[b];
    return 0;
}

/* ------------------------------------------------------------------ */
/* Match stage and Table 2 (paper Sec. II-B match stage, Sec. III-A)   */
/* ------------------------------------------------------------------ */

/* Expected gap between consecutive sorted key64 values of 2^K uniform
 * keys, used as the default distance threshold (R8). */
uint64_t orc_default_distance(int K)
{
    if (K < 1 || K > 63) return 0;
    return 1ull << (64 - K);
}

/* Walks Table 1 bucket by bucket; inside a bucket, for each record i scans
 * j = i+1, i+2, ... while j is in the same bucket and key64_j - key64_i < D
 * (R8, R9), emitting {a, b, hash2} in that order (R10, R11).  Returns the
 * number of pairs; only the first `cap` are written (t2 may be NULL). */
int64_t orc_match(const uint8_t key[32], const uint8_t *t1, uint64_t n, uint64_t D,
                  uint8_t *t2, uint64_t cap)
{
    uint64_t count = 0;
    uint64_t i = 0;
    while (i < n) {
        uint64_t bucket = rec_key64(t1 + 12 * i) >> 40;
        uint64_t end = i;
        while (end < n && (rec_key64(t1 + 12 * end) >> 40) == bucket) end++;
        for (uint64_t x = i; x < end; x++) {
            uint64_t kx = rec_key64(t1 + 12 * x);
            for (uint64_t y = x + 1; y < end; y++) {
                uint64_t ky = rec_key64(t1 + 12 * y);
                if (!(ky - kx < D)) break;
                if (t2 && count < cap) {
                    uint8_t msg[8];
                    uint8_t *out = t2 + 16 * count;
                    memcpy(msg, t1 + 12 * x, 4);
                    memcpy(msg + 4, t1 + 12 * y, 4);
                    memcpy(out, msg, 8);
                    orc_keyed_hash(key, msg, 8, out + 8, 8);
                }
                count++;
            }
        }
        i = end;
    }
    return (int64_t)count;
}

/* Brute force for small K: every ordered pair (x, y) of the UNSORTED records
 * is tested with the match predicate written directly -- same logical bucket,
 * x before y in (key64, nonce) order, key64_y - key64_x < D.  Writes nonce
 * pairs (a, b) as 2 u32 each (first `cap` pairs) and returns the count. */
int64_t orc_match_bruteforce(const uint8_t *recs, uint64_t n, uint64_t D,
                             uint32_t *pairs, uint64_t cap)
{
    uint64_t count = 0;
    for (uint64_t x = 0; x < n; x++) {
        const uint8_t *rx = recs + 12 * x;
        uint64_t kx = rec_key64(rx);
        uint32_t nx = rec_nonce(rx);
        for (uint64_t y = 0; y < n; y++) {
            if (y == x) continue;
            const uint8_t *ry = recs + 12 * y;
            uint64_t ky = rec_key64(ry);
            uint32_t ny = rec_nonce(ry);
            if ((kx >> 40) != (ky >> 40)) continue;
            int before = (kx < ky) || (kx == ky && nx < ny);
            if (!before) continue;
            if (!(ky - kx < D)) continue;
            if (pairs && count < cap) {
                pairs[2 * count] = nx;
                pairs[2 * count + 1] = ny;
            }
            count++;
        }
    }
    return (int64_t)count;
}

/* Cross-bucket variant of the match (the "global" scope): every pair i < j
 * of the whole Table-1 order with key64_j - key64_i < D, whatever the
 * logical buckets, emitted in i, then j order.  The paper's match compares
 * pairs against the threshold (Sec. II-B) inside one bucket (the fused
 * Sort+Match kernel, Sec. III-A); this variant drops the bucket edge. */
int64_t orc_match_global(const uint8_t key[32], const uint8_t *t1, uint64_t n, uint64_t D,
                         uint8_t *t2, uint64_t cap)
{
    uint64_t count = 0;
    for (uint64_t x = 0; x < n; x++) {
        uint64_t kx = rec_key64(t1 + 12 * x);
        for (uint64_t y = x + 1; y < n; y++) {
            uint64_t ky = rec_key64(t1 + 12 * y);
            if (!(ky - kx < D)) break;
            if (t2 && count < cap) {
                uint8_t msg[8];
                uint8_t *out = t2 + 16 * count;
                memcpy(msg, t1 + 12 * x, 4);
                memcpy(msg + 4, t1 + 12 * y, 4);
                memcpy(out, msg, 8);
                orc_keyed_hash(key, msg, 8, out + 8, 8);
            }
            count++;
        }
    }
    return (int64_t)count;
}

/* Brute force of the cross-bucket variant: every ordered pair of the
 * UNSORTED records, x before y in (key64, nonce) order, key64 gap < D. */
int64_t orc_match_global_bruteforce(const uint8_t *recs, uint64_t n, uint64_t D,
                                    uint32_t *pairs, uint64_t cap)
{
    uint64_t count = 0;
    for (uint64_t x = 0; x < n; x++) {
        const uint8_t *rx = recs + 12 * x;
        uint64_t kx = rec_key64(rx);
        uint32_t nx = rec_nonce(rx);
        for (uint64_t y = 0; y < n; y++) {
            if (y == x) continue;
            const uint8_t *ry = recs + 12 * y;
            uint64_t ky = rec_key64(ry);
            uint32_t ny = rec_nonce(ry);
            int before = (kx < ky) || (kx == ky && nx < ny);
            if (!before || !(ky - kx < D)) continue;
            if (pairs && count < cap) {
                pairs[2 * count] = nx;
                pairs[2 * count + 1] = ny;
            }
            count++;
        }
    }
    return (int64_t)count;
}

/* ------------------------------------------------------------------ */
/* All-core variants (the VaultX CPU plotter's threading, Sec. II-B):   */
/* the same tables, the work split over POSIX threads.                  */
/* ------------------------------------------------------------------ */

struct sort_job {
    uint8_t *recs;
    const uint64_t *start; /* group g holds records start[g] .. start[g+1]-1 */
    int g0, step, ngroups;
};

static void *sort_job_run(void *arg)
{
    struct sort_job *j = (struct sort_job *)arg;
    for (int g = j->g0; g < j->ngroups; g += j->step) {
        uint64_t lo = j->start[g], hi = j->start[g + 1];
        if (hi - lo > 1) qsort(j->recs + 12 * lo, (size_t)(hi - lo), 12, rec_cmp);
    }
    return NULL;
}

/* Table 1 on nthreads threads: the records hashed in nonce order into
 * `scratch` (orc_hash_range_mt), moved into t1 grouped by the top 8 bits of
 * key64 (a counting pass; key64 order between groups is group order), then
 * each group sorted by (key64, nonce) with qsort, groups spread over the
 * threads.  Both buffers hold 2^K records. */
int orc_table1_mt(int K, const uint8_t key[32], uint8_t *t1, uint8_t *scratch, int nthreads)
{
    if (K < 1 || K > 32) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    const uint64_t n = 1ull << K;
    orc_hash_range_mt(key, 0, n, scratch, nthreads);
    uint64_t start[257], fill[256];
    memset(start, 0, sizeof start);
    for (uint64_t i = 0; i < n; i++) start[(rec_key64(scratch + 12 * i) >> 56) + 1]++;
    for (int g = 0; g < 256; g++) start[g + 1] += start[g];
    for (int g = 0; g < 256; g++) fill[g] = start[g];
    for (uint64_t i = 0; i < n; i++) {
        const uint8_t *r = scratch + 12 * i;
        memcpy(t1 + 12 * fill[rec_key64(r) >> 56]++, r, 12);
    }
    pthread_t tid[512];
    int started[512];
    struct sort_job jobs[512];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].recs = t1;
        jobs[t].start = start;
        jobs[t].g0 = t;
        jobs[t].step = nthreads;
        jobs[t].ngroups = 256;
        started[t] = pthread_create(&tid[t], NULL, sort_job_run, &jobs[t]) == 0;
        if (!started[t]) sort_job_run(&jobs[t]);
    }
    for (int t = 0; t < nthreads; t++)
        if (started[t]) pthread_join(tid[t], NULL);
    return 0;
}

struct match_job {
    const uint8_t *key, *t1;
    uint64_t lo, hi, D, off, count;
    uint8_t *t2;
};

static void *match_job_run(void *arg)
{
    struct match_job *j = (struct match_job *)arg;
    j->count = (uint64_t)orc_match(j->key, j->t1 + 12 * j->lo, j->hi - j->lo, j->D,
                                   j->t2 ? j->t2 + 16 * j->off : NULL, j->t2 ? j->count : 0);
    return NULL;
}

/* orc_match on nthreads threads.  Table 1 is cut into nthreads runs of whole
 * logical buckets (a cut moves forward to the next bucket start), so the
 * pairs of run t are orc_match of that run alone; a counting pass gives each
 * run its place in Table 2, a second pass writes the pairs there.  Returns
 * the number of pairs; t2 (NULL: count only) must hold all of them. */
int64_t orc_match_mt(const uint8_t key[32], const uint8_t *t1, uint64_t n, uint64_t D, uint8_t *t2,
                     int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    uint64_t cut[513];
    cut[0] = 0;
    for (int t = 1; t < nthreads; t++) {
        uint64_t c = n * (uint64_t)t / (uint64_t)nthreads;
        if (c < cut[t - 1]) c = cut[t - 1];
        while (c > 0 && c < n && (rec_key64(t1 + 12 * c) >> 40) == (rec_key64(t1 + 12 * (c - 1)) >> 40))
            c++;
        cut[t] = c;
    }
    cut[nthreads] = n;
    pthread_t tid[512];
    int started[512];
    struct match_job jobs[512];
    for (int pass = 0; pass < (t2 ? 2 : 1); pass++) {
        uint64_t off = 0;
        for (int t = 0; t < nthreads; t++) {
            if (pass == 1) {
                jobs[t].off = off;
                off += jobs[t].count;
            }
            jobs[t].key = key;
            jobs[t].t1 = t1;
            jobs[t].lo = cut[t];
            jobs[t].hi = cut[t + 1];
            jobs[t].D = D;
            jobs[t].t2 = pass == 1 ? t2 : NULL;
            started[t] = pthread_create(&tid[t], NULL, match_job_run, &jobs[t]) == 0;
            if (!started[t]) match_job_run(&jobs[t]);
        }
        for (int t = 0; t < nthreads; t++)
            if (started[t]) pthread_join(tid[t], NULL);
    }
    uint64_t total = 0;
    for (int t = 0; t < nthreads; t++) total += jobs[t].count;
    return (int64_t)total;
}

/* hash2 of a list of pairs (R10): for record i of `recs` (stride bytes
 * apart, LE32 a at byte 0 and LE32 b at byte 4), out[8 i .. 8 i + 7] = the
 * first 8 bytes of BLAKE3-keyed(key, LE32(a) || LE32(b)).  The list is cut
 * into nthreads contiguous ranges, one POSIX thread each. */
struct pair_job {
    const uint8_t *key, *recs;
    size_t stride;
    uint8_t *out;
    uint64_t lo, hi;
};

static void *pair_job_run(void *arg)
{
    struct pair_job *j = (struct pair_job *)arg;
    for (uint64_t i = j->lo; i < j->hi; i++)
        orc_keyed_hash(j->key, j->recs + j->stride * i, 8, j->out + 8 * i, 8);
    return NULL;
}

int orc_pair_hash_mt(const uint8_t key[32], const uint8_t *recs, uint64_t n, size_t stride,
                     uint8_t *out, int nthreads)
{
    if (stride < 8) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    pthread_t tid[512];
    int started[512];
    struct pair_job jobs[512];
    for (int t = 0; t < nthreads; t++) {
        jobs[t].key = key;
        jobs[t].recs = recs;
        jobs[t].stride = stride;
        jobs[t].out = out;
        jobs[t].lo = n * (uint64_t)t / (uint64_t)nthreads;
        jobs[t].hi = n * (uint64_t)(t + 1) / (uint64_t)nthreads;
        started[t] = pthread_create(&tid[t], NULL, pair_job_run, &jobs[t]) == 0;
        if (!started[t]) pair_job_run(&jobs[t]);
    }
    for (int t = 0; t < nthreads; t++)
        if (started[t]) pthread_join(tid[t], NULL);
    return 0;
}

int orc_abi_version(void) { return 1; }
