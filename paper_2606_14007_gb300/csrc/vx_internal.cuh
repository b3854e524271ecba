// vx_internal.cuh -- shared definitions of the sm_103a plotting kernels.
//
// The plot descriptor (one per plot, in device memory), the keyed BLAKE3
// device core, and the launch helpers the host engine and every kernel
// translation unit agree on.  Nothing here is shared with the CPU oracle.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vx {

// ---------------------------------------------------------------- limits
constexpr int kBucketBits = 24;          // 2^24 logical buckets (Sec. I-A, III-B)
constexpr int kMaxK = 32;                // u32 nonces
constexpr int kMaxCoarseBits = 10;       // first scatter level, <= 1024 bins
constexpr int kMaxFineBits = 10;         // second scatter level, <= 1024 bins
constexpr int kMaxFineBitsWide = 11;     // ... up to 2048 (2^21 partitions, K = 32)
constexpr int kScatterTile = 4096;       // records per CTA in the second scatter level
constexpr int kScatterThreads = 512;
constexpr int kSortThreads = 256;
constexpr int kMatchThreads = 256;
constexpr int kMaxSortDigitBits = 13;    // counting-sort digit of the partition sort
constexpr uint32_t kMaxPartition = 16384;  // records one partition may hold (smem)
constexpr size_t kMaxSmemPerCta = 227 * 1024;  // opt-in dynamic shared memory per CTA

// Status-word bits (device side; the host maps them to VX_E* codes).
constexpr uint32_t kStSlot1Overflow = 1u << 0;
constexpr uint32_t kStSlot2Overflow = 1u << 1;
constexpr uint32_t kStCountMismatch = 1u << 2;
constexpr uint32_t kStT2Capacity = 1u << 3;
constexpr uint32_t kStPartitionTooBig = 1u << 4;
constexpr uint32_t kStTimeout = 1u << 5;
constexpr uint32_t kStBadTicket = 1u << 6;
constexpr uint32_t kStPairSlot = 1u << 7;     // a partition's pairs exceed its pair slot
constexpr uint32_t kStHaloOverflow = 1u << 8; // a partition's halo exceeds its capacity
constexpr uint32_t kStSort2 = 1u << 9;        // sorted Table 2: slot overflow or lost records
constexpr uint32_t kStWinList = 1u << 10;     // a window's nonce list exceeds its capacity

// ------------------------------------------------------ plot descriptor
// One plot's plan and buffers.  The host fills everything but pre1/pre2,
// which the key-setup kernel derives from the key on the device.
struct Desc {
    uint64_t N;          // 2^K nonces
    uint64_t D;          // match distance
    uint64_t t2cap;      // Table-2 capacity (records)
    int32_t K;
    int32_t p;           // partition bits (physical partitions = 2^p)
    int32_t p1;          // first scatter level bits (hash kernel)
    int32_t p2;          // second scatter level bits (p = p1 + p2)
    int32_t dbits;       // counting-sort digit bits inside a partition
    uint32_t cap1;       // records per level-1 slot (p2 > 0 only)
    uint32_t cap2;       // records per level-2 slot (final partitions)
    uint32_t chunks1;    // scatter-2 CTAs per level-1 slot = ceil(cap1 / tile)
                         // level-1 slots: [hchunks][2^p1] of cap1 records each
    uint32_t spin_limit; // polls before a device-side wait gives up
    uint32_t test_flags; // vx_opts.test_flags (fault injection)
    int32_t hchunks;     // nonce chunks (hash / second-scatter pipeline); level-1 slots per chunk
    int32_t pchunks;     // partition chunks (sort / pair-hash pipeline)
    uint32_t scope;      // match: 0 = inside a logical bucket, 1 = cross-bucket
    uint32_t hcap;       // halo records per partition (scope 1 with p > 0), else 0
    int32_t pk;          // partition bits in key space (p + wbits): every key shift
    uint32_t wbits;      // window: the plot keeps the records whose top wbits
    uint32_t win;        //   key bits equal win (wbits 0: every record)
    uint32_t listcap;    // window nonce list capacity (entries), if wids
    const uint8_t *wids; // window id of every nonce (top wbits of key64), or null:
                         //   the hash kernels then hash every nonce and filter
    uint32_t *wlist;     // [listcap] the window's nonces, listed from wids
    uint32_t *wcount;    // entries in wlist (zeroed by the key setup)
    uint32_t *halo_cnt;  // [2^p] halo fill counters
    uint64_t *halo_keys; // [2^p * hcap] records of partition f within D of its
    uint32_t *halo_nonces; //            lower edge (unsorted): f - 1's halo
    uint64_t *a_keys;    // level-1 slots, SoA: key64 [hchunks * 2^p1 * cap1]
    uint32_t *a_nonces;  //                      nonce [hchunks * 2^p1 * cap1]
    uint64_t *b_keys;    // level-2 slots, SoA: key64 [2^p * cap2]
    uint32_t *b_nonces;  //                      nonce [2^p * cap2]
    uint32_t *cnt1;      // [hchunks * 2^p1] level-1 fill counters
    uint32_t *cnt2;      // [2^p]  level-2 fill counters
    uint64_t *t1off;     // [2^p + 1] Table-1 record offset of each partition
    uint64_t *pairs;     // [2^p] Table-2 pairs of each partition
    uint64_t *t2off;     // [2^p + 1] Table-2 record offset of each partition
    uint64_t *lb;        // [2^p] look-back words of the fused sort+match
    uint32_t *ticket;    // partition ticket of the fused sort+match
    uint64_t *lbs;       // [chunks] look-back words of the Table-1 offset scan
    uint32_t *ticket_s;  // chunk ticket of the Table-1 offset scan
    uint32_t *status;    // status word
    uint8_t *t1;         // Table 1, 12-byte records
    uint8_t *t2;         // Table 2, 16-byte records
    uint32_t key[8];     // plot key, LE words
    uint32_t pre1[16];   // Table-1 hash state after round-1 columns 1..3
    uint32_t pre2[16];   // pair-hash state after round-1 columns 1..3
};

// Table 2 sorted by hash2 (vx_sort_table2): one plot's second sorting pass
// over 16-byte records, with its own slots in a caller-provided work buffer.
struct Sort2Desc {
    const uint64_t *count; // device word with the Table-2 record count
    int32_t p;             // partition bits (2^p partitions of ~2^11 records)
    int32_t p1, p2;        // first / second scatter level bits (p = p1 + p2)
    int32_t dbits;         // counting-sort digit bits inside a partition
    uint32_t cap1, cap2;   // slot capacities (records) of the two levels
    uint32_t chunks1;      // second-level CTAs per first-level slot
    uint32_t spin_limit;   // polls before a bounded wait gives up
    uint4 *t2;             // Table 2: read by the first level, rewritten sorted
    uint64_t *a_keys, *a_vals; // first-level slots [2^p1][cap1]: key2, a << 32 | b
    uint64_t *b_keys, *b_vals; // partitions [2^p][cap2]
    uint32_t *cnt1, *cnt2; // fill counters
    uint64_t *off;         // [2^p + 1] partition offsets in the sorted table
    uint64_t *lbs;         // look-back words of the offset scan
    uint32_t *ticket;      // chunk ticket of the offset scan
    uint32_t *status;      // the plot's status word
};


// Nonces [lo, hi) of chunk `chunk` of a plot (chunks split 2^K evenly).
__device__ __forceinline__ void nonce_chunk(const Desc &d, int chunk, uint64_t &lo, uint64_t &hi)
{
    lo = d.N / (uint64_t)d.hchunks * (uint64_t)chunk;
    hi = d.N / (uint64_t)d.hchunks * (uint64_t)(chunk + 1);
}

// Maps a CTA's global tile index to (plot, local tile) through an exclusive
// prefix of per-plot tile counts (batch launches group many plots).
__device__ __forceinline__ int find_plot(const uint32_t *__restrict__ tile_start, int nplots,
                                         uint32_t tile)
{
    int lo = 0, hi = nplots;  // invariant: tile_start[lo] <= tile < tile_start[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (__ldg(tile_start + mid) <= tile) lo = mid; else hi = mid;
    }
    return lo;
}

// ------------------------------------------------------ keyed BLAKE3 core
// BLAKE3 constants: IV (the SHA-256 initial words) and domain flags.
constexpr uint32_t kIV0 = 0x6A09E667u, kIV1 = 0xBB67AE85u, kIV2 = 0x3C6EF372u,
                   kIV3 = 0xA54FF53Au;
constexpr uint32_t kFlagsKeyedRootChunk = 1u /*CHUNK_START*/ | 2u /*CHUNK_END*/ |
                                          8u /*ROOT*/ | 16u /*KEYED_HASH*/;

// Rotations by 16 and 8 are byte moves (PRMT); by 12 and 7 funnel shifts.
__device__ __forceinline__ uint32_t ror16(uint32_t x) { return __byte_perm(x, 0, 0x1032); }
__device__ __forceinline__ uint32_t ror8(uint32_t x) { return __byte_perm(x, 0, 0x0321); }
__device__ __forceinline__ uint32_t ror12(uint32_t x) { return __funnelshift_r(x, x, 12); }
__device__ __forceinline__ uint32_t ror7(uint32_t x) { return __funnelshift_r(x, x, 7); }
__device__ __forceinline__ uint32_t bswap32(uint32_t x) { return __byte_perm(x, 0, 0x0123); }

#define VX_G(a, b, c, d, mx, my)       \
    do {                               \
        a = a + b + (mx);              \
        d = ::vx::ror16(d ^ a);        \
        c = c + d;                     \
        b = ::vx::ror12(b ^ c);        \
        a = a + b + (my);              \
        d = ::vx::ror8(d ^ a);         \
        c = c + d;                     \
        b = ::vx::ror7(b ^ c);         \
    } while (0)

// Message schedule step between rounds: new m[i] = old m[perm[i]] with
// perm = {2,6,3,10,7,0,4,13,1,11,12,5,9,14,15,8}.  Pure register renaming.
#define VX_PERMUTE(m)                                                              \
    do {                                                                           \
        uint32_t t0 = m[2], t1 = m[6], t2 = m[3], t3 = m[10], t4 = m[7], t5 = m[0], \
                 t6 = m[4], t7 = m[13], t8 = m[1], t9 = m[11], t10 = m[12],         \
                 t11 = m[5], t12 = m[9], t13 = m[14], t14 = m[15], t15 = m[8];      \
        m[0] = t0; m[1] = t1; m[2] = t2; m[3] = t3; m[4] = t4; m[5] = t5;         \
        m[6] = t6; m[7] = t7; m[8] = t8; m[9] = t9; m[10] = t10; m[11] = t11;     \
        m[12] = t12; m[13] = t13; m[14] = t14; m[15] = t15;                       \
    } while (0)

// Per-key state of a one-block keyed hash whose message occupies words 0..1
// only: v = {key, IV0..3, counter 0, 0, block_len, flags}, with the three
// round-1 column G's that see only zero message words already applied.
__device__ __forceinline__ void b3_key_setup(const uint32_t key[8], uint32_t block_len,
                                             uint32_t pre[16])
{
    uint32_t v0 = key[0], v1 = key[1], v2 = key[2], v3 = key[3];
    uint32_t v4 = key[4], v5 = key[5], v6 = key[6], v7 = key[7];
    uint32_t v8 = kIV0, v9 = kIV1, v10 = kIV2, v11 = kIV3;
    uint32_t v12 = 0, v13 = 0, v14 = block_len, v15 = kFlagsKeyedRootChunk;
    VX_G(v1, v5, v9, v13, 0u, 0u);
    VX_G(v2, v6, v10, v14, 0u, 0u);
    VX_G(v3, v7, v11, v15, 0u, 0u);
    pre[0] = v0; pre[1] = v1; pre[2] = v2; pre[3] = v3;
    pre[4] = v4; pre[5] = v5; pre[6] = v6; pre[7] = v7;
    pre[8] = v8; pre[9] = v9; pre[10] = v10; pre[11] = v11;
    pre[12] = v12; pre[13] = v13; pre[14] = v14; pre[15] = v15;
}

// The rest of the compression for message words (m0, m1, 0, ..., 0):
// round-1 column 0 and diagonals, rounds 2..7, and output words 0 and 1
// (hash bytes 0..7).  TWO_WORDS = false fixes m1 = 0 (4-byte messages).
template <bool TWO_WORDS>
__device__ __forceinline__ void b3_finish(const uint32_t pre[16], uint32_t m0, uint32_t m1,
                                          uint32_t &h0, uint32_t &h1)
{
    uint32_t v0 = pre[0], v1 = pre[1], v2 = pre[2], v3 = pre[3];
    uint32_t v4 = pre[4], v5 = pre[5], v6 = pre[6], v7 = pre[7];
    uint32_t v8 = pre[8], v9 = pre[9], v10 = pre[10], v11 = pre[11];
    uint32_t v12 = pre[12], v13 = pre[13], v14 = pre[14], v15 = pre[15];
    uint32_t m[16];
    m[0] = m0;
    m[1] = TWO_WORDS ? m1 : 0u;
#pragma unroll
    for (int i = 2; i < 16; ++i) m[i] = 0u;
    // Round 1 (columns 1..3 are in pre).
    VX_G(v0, v4, v8, v12, m[0], m[1]);
    VX_G(v0, v5, v10, v15, m[8], m[9]);
    VX_G(v1, v6, v11, v12, m[10], m[11]);
    VX_G(v2, v7, v8, v13, m[12], m[13]);
    VX_G(v3, v4, v9, v14, m[14], m[15]);
#pragma unroll
    for (int r = 1; r < 7; ++r) {
        VX_PERMUTE(m);
        VX_G(v0, v4, v8, v12, m[0], m[1]);
        VX_G(v1, v5, v9, v13, m[2], m[3]);
        VX_G(v2, v6, v10, v14, m[4], m[5]);
        VX_G(v3, v7, v11, v15, m[6], m[7]);
        VX_G(v0, v5, v10, v15, m[8], m[9]);
        VX_G(v1, v6, v11, v12, m[10], m[11]);
        VX_G(v2, v7, v8, v13, m[12], m[13]);
        VX_G(v3, v4, v9, v14, m[14], m[15]);
    }
    h0 = v0 ^ v8;
    h1 = v1 ^ v9;
}

// key64 = big-endian u64 of hash bytes 0..7 (h0 holds bytes 0..3 LE).
__device__ __forceinline__ uint64_t key64_of(uint32_t h0, uint32_t h1)
{
    return ((uint64_t)bswap32(h0) << 32) | (uint64_t)bswap32(h1);
}

// --------------------------------------------------------- block helpers
// Exclusive scan of one u32 per thread over a CTA of NT threads; returns the
// thread's exclusive prefix, writes the CTA total to *total.  `ws` holds
// NT/32 + 1 words of shared memory.
template <int NT>
__device__ __forceinline__ uint32_t block_exclusive_scan_u32(uint32_t x, uint32_t *ws,
                                                             uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < NT / 32 ? ws[lane] : 0u;
        uint32_t wi = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, wi, o);
            if (lane >= o) wi += y;
        }
        if (lane < NT / 32) ws[lane] = wi - w;
        if (lane == NT / 32 - 1) ws[NT / 32] = wi;
    }
    __syncthreads();
    uint32_t r = ws[warp] + incl - x;
    *total = ws[NT / 32];
    __syncthreads();
    return r;
}

// In-place exclusive scan of A[0..M) by a CTA of NT threads; returns the
// total.  Warp w takes a contiguous run of A and walks it 32 entries at a
// time (lane i on entry i: no bank conflicts); `ws` holds NT/32 words.
// Ends with a __syncthreads.
template <int NT>
__device__ __forceinline__ uint32_t block_scan_inplace_u32(uint32_t *A, uint32_t M, uint32_t *ws)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t chunk = (M + NW - 1) / NW;
    const uint32_t lo = min(M, (uint32_t)warp * chunk), hi = min(M, lo + chunk);
    uint32_t sum = 0;
    for (uint32_t i = lo + lane; i < hi; i += 32) sum += A[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) ws[warp] = sum;
    __syncthreads();
    uint32_t carry = 0, total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t t = ws[w];
        carry += w < warp ? t : 0u;
        total += t;
    }
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t v = i < hi ? A[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (i < hi) A[i] = carry + incl - v;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncthreads();
    return total;
}

template <int NT>
__device__ __forceinline__ uint64_t block_sum_u64(uint64_t x, uint64_t *ws)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
    if (lane == 0) ws[warp] = x;
    __syncthreads();
    uint64_t s = 0;
    if (threadIdx.x == 0) {
        for (int w = 0; w < NT / 32; ++w) s += ws[w];
        ws[NT / 32] = s;
    }
    __syncthreads();
    s = ws[NT / 32];
    __syncthreads();
    return s;
}

// ------------------------------------------------ decoupled look-back
// Per-item words: 2 flag bits (aggregate / inclusive prefix / poisoned) and
// a 62-bit value.  Items are taken in ticket order, so every item an item
// waits on is already running; waits are bounded (spin limit) and a
// timeout poisons the item so that later items stop at once.
constexpr uint64_t kLbAgg = 1ull << 62;       // look-back: aggregate published
constexpr uint64_t kLbIncl = 2ull << 62;      // look-back: inclusive prefix published
constexpr uint64_t kLbPoison = 3ull << 62;    // look-back: chain broken (timeout)
constexpr uint64_t kLbMask = (1ull << 62) - 1;

__device__ __forceinline__ void st_release_u64(uint64_t *p, uint64_t v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t ld_acquire_u64(const uint64_t *p)
{
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Publishes item f's own value (lane 0): its inclusive prefix when f == 0,
// else its aggregate.  `withhold` (test hook) keeps item 0 silent.
__device__ __forceinline__ void lb_publish(uint64_t *lb, uint32_t f, uint64_t agg, bool withhold)
{
    if (f == 0) {
        if (!withhold) st_release_u64(lb, kLbIncl | agg);
    } else {
        st_release_u64(lb + f, kLbAgg | agg);
    }
}

// Exclusive prefix of item f (value agg, already published by lb_publish)
// by decoupled look-back, run by all 32 lanes of one warp: each step reads
// 32 predecessors at once, adds the aggregates back to the nearest
// published inclusive prefix, and retries (bounded) while one of them has
// published nothing yet.  Lane 0 publishes f's inclusive prefix.  Returns
// false (every lane) if the chain is poisoned or a wait ran out (status
// gets kStTimeout), or for item 0 when it was withheld.
__device__ __forceinline__ bool lb_resolve(uint64_t *lb, uint32_t f, uint64_t agg, uint32_t *status,
                                           uint32_t limit, bool withhold, uint64_t *excl_out)
{
    const int lane = threadIdx.x & 31;
    if (f == 0) {
        *excl_out = 0;
        return !withhold;
    }
    uint64_t excl = 0;
    int64_t hi = (int64_t)f - 1;   // newest predecessor not yet added
    uint32_t spins = 0;
    for (;;) {
        const int64_t j = hi - lane;
        // Items before 0 read as an inclusive prefix of 0.
        const uint64_t v = j >= 0 ? ld_acquire_u64(lb + j) : kLbIncl;
        const uint64_t fl = v & ~kLbMask;
        const uint32_t incl = __ballot_sync(0xffffffffu, fl == kLbIncl);
        const uint32_t stop = incl ? (uint32_t)(__ffs(incl) - 1) : 31u;
        const uint32_t upto = stop == 31u ? 0xffffffffu : ((2u << stop) - 1u);
        const uint32_t poison = __ballot_sync(0xffffffffu, fl == kLbPoison) & upto;
        const uint32_t waiting = __ballot_sync(0xffffffffu, fl == 0) & upto;
        if (poison) {
            if (lane == 0) st_release_u64(lb + f, kLbPoison);
            return false;
        }
        if (waiting) {
            if (++spins > limit) {
                if (lane == 0) {
                    atomicOr(status, kStTimeout);
                    st_release_u64(lb + f, kLbPoison);
                }
                return false;
            }
            __nanosleep(64);
            continue;
        }
        uint64_t x = ((uint32_t)lane <= stop) ? (v & kLbMask) : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        excl += x;
        if (incl) break;
        hi -= 32;
    }
    if (lane == 0) st_release_u64(lb + f, kLbIncl | (excl + agg));
    *excl_out = excl;
    return true;
}

// Both steps at once (publish, then resolve).
__device__ __forceinline__ bool lookback_warp(uint64_t *lb, uint32_t f, uint64_t agg,
                                              uint32_t *status, uint32_t limit, bool withhold,
                                              uint64_t *excl_out)
{
    if ((threadIdx.x & 31) == 0) lb_publish(lb, f, agg, withhold);
    __syncwarp();
    return lb_resolve(lb, f, agg, status, limit, withhold, excl_out);
}

// Cross-bucket match (scope 1): a record within D of its partition's lower
// edge also belongs to the halo of the partition before (partition 0 has
// no predecessor).  Called by every kernel that fills the final partitions.
__device__ __forceinline__ void halo_add(const Desc &d, uint64_t part, uint64_t key, uint32_t nonce,
                                         bool &overflow)
{
    if (d.hcap == 0 || part == 0) return;
    if ((key & (~0ull >> d.pk)) >= d.D) return;  // offset inside the partition (p >= 1)
    const uint32_t h = atomicAdd(&d.halo_cnt[part], 1u);
    if (h < d.hcap) {
        d.halo_keys[part * d.hcap + h] = key;
        d.halo_nonces[part * d.hcap + h] = nonce;
    } else {
        overflow = true;
    }
}

// -------------------------------------------------- TMA bulk copy helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("{ .reg .b64 st; mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1; }" ::"r"(
                     smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

// Bulk global -> shared copy (addresses 16-byte aligned, bytes % 16 == 0)
// completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk shared -> global copy (addresses 16-byte aligned, bytes % 16 == 0)
// in the issuing thread's bulk group; the thread first makes the CTA's
// ordinary shared-memory writes visible to the copy engine.
__device__ __forceinline__ void bulk_s2g(void *dst, const void *src, uint32_t bytes)
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst),
                 "r"(smem_u32(src)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// Waits until the issuing thread's bulk copies have read their shared
// memory (READ) or are complete.
template <bool READ>
__device__ __forceinline__ void bulk_wait_all()
{
    if (READ)
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    else
        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Waits for phase `parity` of the mbarrier; gives up after `limit` polls.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

}  // namespace vx

// ----------------------------------------------- launch entry points (host)
// Each returns the launch's cudaGetLastError().  `descs` and the tile_start
// arrays (exclusive prefixes of per-plot CTA counts, nplots + 1 entries)
// live in device memory; nplots >= 1.
namespace vx {
struct HashCfg {
    bool agg;     // warp-aggregated histogram (few first-level bins)
    bool halo;    // some plot of the launch matches across buckets (halo code)
    bool win;     // some plot of the launch is a window (window filter)
    bool list;    // the launch's one plot hashes its window's nonce list
    int npt;      // nonces per thread of the staged Table-1 hash (4, 8, 16; 8 with a window)
};
cudaError_t launch_key_setup(Desc *descs, int nplots, cudaStream_t s);
// Hash kernels and the second scatter level take one nonce chunk (of
// Desc::hchunks); the pair hash takes one partition chunk (of Desc::pchunks).
cudaError_t launch_hash_scatter(const Desc *descs, int nplots, const uint32_t *tile_start,
                                uint32_t total_tiles, HashCfg cfg, int chunk, cudaStream_t s);
cudaError_t launch_hash_direct(const Desc *descs, int nplots, const uint32_t *tile_start,
                               uint32_t total_tiles, int chunk, cudaStream_t s, HashCfg cfg);
// Sort + match variants: Table-2 records at final offsets found by a
// look-back ({a, b, 0, 0}, hashed later by launch_t2_hash; or hashed in the
// kernel), or pairs {a, b} written into each partition's own slot.
enum SortMatchOut { kOutLookback = 0, kOutLookbackHashed = 1, kOutSlots = 2 };
cudaError_t launch_sortmatch(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                             SortMatchOut out, bool halo);
cudaError_t launch_t2_hash(const Desc *descs, int nplots, const uint32_t *tile_start,
                           uint32_t total_tiles, int chunk, cudaStream_t s);
// Pair hash of the slot placement: kT2SlotGroup partitions per CTA, pairs
// read from the partition slots, records written at the scanned offsets.
constexpr uint32_t kT2SlotGroup = 8;
cudaError_t launch_t2_hash_slots(const Desc *descs, int nplots, const uint32_t *tile_start,
                                 uint32_t total_tiles, cudaStream_t s);
constexpr uint64_t kT2HashTile = 256 * 8;  // Table-2 records per pair-hash CTA
size_t sortmatch_smem_bytes(uint32_t cap, int dbits);
uint32_t sortmatch_max_cap();  // largest slot the sort keeps in registers
cudaError_t launch_scatter2(const Desc *descs, int nplots, const uint32_t *tile_start,
                            uint32_t total_tiles, int chunk, cudaStream_t s, bool halo,
                            int fine_bits);  // the launch's widest second level
cudaError_t launch_scan_counts(const Desc *descs, int nplots, const uint32_t *tile_start,
                               uint32_t total_tiles, cudaStream_t s);
// Same chunked look-back scan over the per-partition pair counts (slot
// placement) -> Table-2 offsets, with the Table-2 capacity check.
cudaError_t launch_scan_pair_counts(const Desc *descs, int nplots, const uint32_t *tile_start,
                                    uint32_t total_tiles, cudaStream_t s);
constexpr uint32_t kScanChunk = 4096;      // counters per CTA of the Table-1 offset scan
cudaError_t launch_sort(const Desc *descs, int nplots, const uint32_t *tile_start,
                        uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                        bool halo);
cudaError_t launch_scan_pairs(const Desc *descs, int nplots, cudaStream_t s);
cudaError_t launch_match(const Desc *descs, int nplots, const uint32_t *tile_start,
                         uint32_t total_tiles, cudaStream_t s, uint32_t max_cap);
cudaError_t launch_bucket_offsets(const Desc *desc, uint64_t *out, cudaStream_t s);
// Table 2 sorted by hash2: grids of the five kernels of one sort.
struct Sort2Launch {
    uint32_t tiles1, tiles2, tiles_scan, parts, cap2;
    int dbits;
};
cudaError_t launch_sort2(const Sort2Desc *d_desc, const Sort2Launch &g, cudaStream_t s);
size_t sort2_smem_bytes(uint32_t cap, int dbits);
// Window id (top c <= 8 bits of key64) of every nonce 0 .. N-1, one byte
// each at ids (16-byte aligned, N rounded up to 16 bytes).
cudaError_t launch_window_ids(const uint32_t key[8], uint64_t N, int c, uint8_t *ids, cudaStream_t s);
// Lists the nonces of one plot's window from its Desc::wids into Desc::wlist
// (single plot; N nonces).
cudaError_t launch_window_list(const Desc *desc, uint64_t N, cudaStream_t s);
cudaError_t launch_hash_records(const uint32_t key[8], uint64_t nonce0, uint64_t count,
                                uint32_t *out, cudaStream_t s);
cudaError_t launch_pair_hash(const uint32_t key[8], const uint32_t *pairs, uint64_t count,
                             uint4 *out, cudaStream_t s);
// Hash-only ceiling: `blocks` CTAs of kHashThreads fold their hashes into
// fold[blocks * kHashThreads].
cudaError_t launch_hash_peak(const uint32_t key[8], uint64_t nonce0, uint64_t count, uint32_t *fold,
                             uint32_t blocks, cudaStream_t s);
size_t sort_smem_bytes(uint32_t cap, int dbits);
size_t match_smem_bytes(uint32_t cap);
constexpr int kHashThreads = 256;
constexpr int kHashNoncesPerThread = 8;
constexpr int kHashTile = kHashThreads * kHashNoncesPerThread;
}  // namespace vx
