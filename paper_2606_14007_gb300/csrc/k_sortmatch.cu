// k_sortmatch.cu -- partition sort fused with the match stage.
//
// Paper: Sec. I-B / III-A / III-B fuse sort and Table-2 generation into one
// kernel that keeps each bucket in shared memory, one block per bucket,
// with a single-thread insertion sort; Sec. V names that O(n^2) sort as the
// K=31 bottleneck and proposes a parallel radix sort.  Kept here: the
// fusion (a partition never leaves shared memory between sort and match).
// Changed: a physical partition (a run of whole logical buckets, ~2048
// records) per work item, a counting sort on the key bits below the
// partition prefix (about one record per digit, half a record with the
// 16-bit counters of the persistent front end) whose digit runs are then
// ordered by (key64, nonce).  A partition's pairs either go to its own slot
// (kSortSlots, the default wherever the plan shows the pair slot safe: no
// partition waits on another, a scan and the slot pair hash place them) or
// straight to Table 2 at a base found by a decoupled look-back over the
// partitions before it (partition order comes from a ticket counter, so
// every partition an item waits on is held by a running CTA; every wait is
// bounded and a timeout poisons the chain instead of hanging).  With the
// cross-bucket match (HALO instances) the next partition's halo is sorted
// in behind the partition's records.
//
// After the sort every step walks the sorted records in chunks of 32, one
// record per lane, each warp over its own run of chunks: the pair counts
// (lanes probe the records after theirs), their warp scans, the Table-1
// words (coalesced 4-byte stores) and the pair emission.  So no thread
// walks a data-dependent list alone while its warp waits.
//
// Two front ends feed the same steps:
//  * k_sortmatch_pipe (the default): persistent CTAs, three per SM at the
//    default slot.  A CTA's next partition slot (keys and nonces, two
//    contiguous runs) comes into shared memory by cp.async.bulk while the
//    CTA matches and writes the current one; the sort runs between two
//    shared buffers, so a digit run is ordered by ranking its records, not
//    by one thread's insertion sort.
//  * k_sortmatch_gl: one CTA per partition reading its slot from global
//    memory, for slots too large to hold twice in shared memory.
//
// MODE kSortCount: the sort alone (Table 1 + per-partition pair counts),
// used by the split vx_table1 / vx_match path.
// MODE kSortHash: everything in one kernel, pairs hashed here.
// MODE kSortEmit: Table 1, then each pair written as a Table-2 record
// {a, b, 0, 0} at its final offset; the streaming pair-hash kernel fills in
// the hashes (no barriers, full occupancy: the ALU-bound part runs apart
// from the latency-bound sort).
// MODE kSortSlots: Table 1, then the partition's pairs {a, b} in (i, j)
// order into the partition's own level-2 slot, which the kernel has already
// read into shared memory: cap2 pairs in the key array, cap2 / 2 in the
// nonce array.  No partition waits on another; a scan of the pair counts
// and the slot pair hash place the records.
#include "vx_internal.cuh"

namespace vx {

enum { kSortCount = 0, kSortHash = 1, kSortEmit = 2, kSortSlots = 3 };
#define SLOTS_MODE(m) ((m) == kSortSlots)
constexpr uint32_t kSMList = 2048;  // pair-list window (entries), kSortHash only
constexpr int kPipeThreads = 256;   // persistent front end
constexpr int kGlThreads = 256;     // one-CTA-per-partition front end
// Tickets between a CTA of the global-memory front end and the partition
// whose slot it prefetches into L2: about half of the CTAs resident at once.
constexpr uint32_t kSlotPrefetchAhead = 384;

// Shared layout (bytes from the base), for slots of at most `cap` records
// (a multiple of 4) and digits of at most `dbits` bits:
//   buffer X: key64 [cap] | nonce [cap]
//   buffer Y: key64 [cap] | nonce [cap]     (pipelined front end only)
//   digit counters [2^dbits], dead once the digit runs are ordered, then
//   overlaid by the per-record pair count -> pair offset [cap]
//   pair list [kSMList] (kSortHash) | scan workspace | mbarrier
// The pipelined front end alternates the two buffers: an item's slot lands
// in one, is placed by digit into the other, and comes back sorted into the
// first, so the second is free for the next item's slot while the first
// holds the sorted partition.
struct SMLayout {
    size_t xk, xn, yk, yn, dc, list, ws, bar, bytes;
    __host__ __device__ SMLayout(uint32_t cap, int dbits, bool with_list, bool two)
    {
        cap = (cap + 3u) & ~3u;
        xk = 0;
        xn = xk + (size_t)cap * 8;
        yk = xn + (size_t)cap * 4;
        yn = yk + (two ? (size_t)cap * 8 : 0);
        dc = yn + (two ? (size_t)cap * 4 : 0);
        const size_t dcb = ((size_t)1 << dbits) * 4, stb = (size_t)cap * 4;
        list = dc + (dcb > stb ? dcb : stb);
        ws = list + (with_list ? (size_t)kSMList * 4 : 0);
        bar = (ws + 40 * 4 + 7) & ~(size_t)7;
        bytes = bar + 8;
    }
};

struct Part {
    uint64_t *SK;
    uint32_t *SN, *DC, *ST, *LS, *WS;
};

__device__ __forceinline__ bool rec_less(uint64_t ka, uint32_t na, uint64_t kb, uint32_t nb)
{
    return ka < kb || (ka == kb && na < nb);
}

// ---------------------------------------------------------------- sorts
// Both leave the partition's n records sorted by (key64, nonce) in a
// shared buffer.  DC (2^dbits zeroed counters) is the digit table; both
// start after a barrier and end with one.

// Inclusive scan of one u32 per lane.
__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t x)
{
    const uint32_t lane = threadIdx.x & 31u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    return x;
}

// Exclusive scan of the M digit counters in place.  When M is 32 * NW * R'
// with R' <= R (whole rows of 32 counters, the same number per warp), warp w scans its
// R' rows of 32 counters as R' independent warp scans and adds the row and
// warp prefixes; otherwise the general block scan.  Ends with a barrier.
template <int NT, int R>
__device__ __forceinline__ void counts_to_starts(uint32_t *DC, uint32_t M, uint32_t *WS)
{
    constexpr uint32_t NW = NT / 32;
    if (M < 32u * NW || M > 32u * NW * R || M % (32u * NW) != 0) {
        block_scan_inplace_u32<NT>(DC, M, WS);
        return;
    }
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t rows = M / (32u * NW);
    uint32_t *row0 = DC + warp * rows * 32u + lane;
    uint32_t v[R], incl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = (uint32_t)j < rows ? row0[32 * j] : 0u;
#pragma unroll
    for (int j = 0; j < R; ++j) incl[j] = warp_incl_scan(v[j]);
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t t = __shfl_sync(0xffffffffu, incl[j], 31);
        incl[j] += run - v[j];  // exclusive inside the warp's rows
        run += t;
    }
    if (lane == 0) WS[warp] = run;
    __syncthreads();
    uint32_t carry = 0;
#pragma unroll
    for (uint32_t w = 0; w < NW; ++w) carry += w < warp ? WS[w] : 0u;
#pragma unroll
    for (int j = 0; j < R; ++j)
        if ((uint32_t)j < rows) row0[32 * j] = carry + incl[j];
    __syncthreads();
}

// True when the M counter words fill whole rows of 32 per warp, at most R
// rows each: the shape in which counts_to_starts needs no general block
// scan, and the one counts_to_starts_packed requires.
template <int NT, int R>
__host__ __device__ __forceinline__ bool rows_shape(uint32_t M)
{
    constexpr uint32_t NW = NT / 32;
    return M >= 32u * NW && M <= 32u * NW * R && M % (32u * NW) == 0;
}

// counts_to_starts for 2M digit counters of 16 bits, two to a word (digit
// 2w in the low half of word w, 2w + 1 in the high half; every count and
// start below 2^16).  The words must have rows_shape<NT, R>.  Each word's
// two counts become their run starts: the exclusive prefix P of the
// word sums, and P plus the low count.  Ends with a barrier.
template <int NT, int R>
__device__ __forceinline__ void counts_to_starts_packed(uint32_t *DC, uint32_t M, uint32_t *WS)
{
    constexpr uint32_t NW = NT / 32;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t rows = M / (32u * NW);
    uint32_t *row0 = DC + warp * rows * 32u + lane;
    uint32_t lo[R], v[R], incl[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t w = (uint32_t)j < rows ? row0[32 * j] : 0u;
        lo[j] = w & 0xFFFFu;
        v[j] = lo[j] + (w >> 16);
    }
#pragma unroll
    for (int j = 0; j < R; ++j) incl[j] = warp_incl_scan(v[j]);
    uint32_t run = 0;
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t t = __shfl_sync(0xffffffffu, incl[j], 31);
        incl[j] += run - v[j];
        run += t;
    }
    if (lane == 0) WS[warp] = run;
    __syncthreads();
    uint32_t carry = 0;
#pragma unroll
    for (uint32_t w = 0; w < NW; ++w) carry += w < warp ? WS[w] : 0u;
#pragma unroll
    for (int j = 0; j < R; ++j)
        if ((uint32_t)j < rows) {
            const uint32_t P = carry + incl[j];
            row0[32 * j] = P | ((P + lo[j]) << 16);
        }
    __syncthreads();
}

// Ping-pong sort of the n records in buffer X (keys XK, nonces XN):
// digit histogram, scan, then each record placed by digit into buffer Y (a
// digit's run in arrival order); then every position of Y, 32 per warp
// step, finds its record's rank inside its run (runs hold about one
// record; a run of L compares L records) and writes the record to that
// place of X.  X ends sorted, Y is free.
//
// PACK: 16-bit digit counters, two to a word, so that the same counter
// words hold twice the digits (ndig digits in ndig / 2 words, which must
// have rows_shape; n < 2^16).  Runs then hold about half a record, and
// fewer of them need ranking.
//
// DRAIN: buffer Y may still be the source of thread 0's bulk stores (the
// previous item's staged pairs); their reads must end before the records
// are placed into it, so thread 0 waits for them after the histogram and
// the scan, which overlap the stores.
template <int NT, bool PACK, bool DRAIN>
__device__ __forceinline__ void sort_pingpong(const Part &A, uint64_t *XK, uint32_t *XN, uint64_t *YK,
                                              uint32_t *YN, uint32_t n, int shift, uint32_t ndig)
{
    constexpr uint32_t NW = NT / 32;
    const uint32_t dmask = ndig - 1u;
    // digit g's counter: word g (PACK: word g / 2, the half g & 1)
    auto bump = [&](uint32_t g) -> uint32_t {
        if (PACK) {
            const uint32_t h = (g & 1u) << 4;
            return (atomicAdd(&A.DC[g >> 1], 1u << h) >> h) & 0xFFFFu;
        }
        return atomicAdd(&A.DC[g], 1u);
    };
    const uint16_t *DC16 = reinterpret_cast<const uint16_t *>(A.DC);
    // end of run g once the records are placed (little-endian halves)
    auto run_end = [&](uint32_t g) -> uint32_t { return PACK ? (uint32_t)DC16[g] : A.DC[g]; };
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < n; i += NT) bump((uint32_t)(XK[i] >> shift) & dmask);
    __syncthreads();
    if (PACK)
        counts_to_starts_packed<NT, 8>(A.DC, ndig >> 1, A.WS);
    else
        counts_to_starts<NT, 8>(A.DC, ndig, A.WS);
    if (DRAIN) {
        if (threadIdx.x == 0) bulk_wait_all<true>();
        __syncthreads();
    }
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint64_t k = XK[i];
        const uint32_t pos = bump((uint32_t)(k >> shift) & dmask);
        YK[pos] = k;
        YN[pos] = XN[i];
    }
    __syncthreads();
    // DC[g] is now the end of run g: run g is [DC[g-1], DC[g]).  A record's
    // place is its run's start plus the run's records before it.  A run's
    // records sit in neighbouring lanes of a chunk of 32 positions, so each
    // lane compares with the lanes up to the longest run's length away
    // (shuffles, every lane in step), on a 32-bit compare key: the key bits
    // below the digit, or their top 32 -- records of a run agree above
    // them.  A lane whose run leaves its chunk, or that meets an equal
    // compare key, ranks itself again from shared memory on full keys and
    // nonces.  Two chunks per step so that their work overlaps.
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    const uint32_t nch = (n + 31u) >> 5;
    const int cs = shift > 32 ? shift - 32 : 0;
    for (uint32_t c = warp; c < nch; c += 2 * NW) {
        const uint32_t pa = 32u * c + lane, pb = pa + 32u * NW;
        const bool va = pa < n, vb = pb < n;
        const uint32_t xa = va ? pa : 0u, xb = vb ? pb : 0u;
        const uint64_t ka = YK[xa], kb = YK[xb];
        const uint32_t na = YN[xa], nb = YN[xb];
        const uint32_t ga = (uint32_t)(ka >> shift) & dmask, gb = (uint32_t)(kb >> shift) & dmask;
        const uint32_t sa = ga ? run_end(ga - 1) : 0u, sb = gb ? run_end(gb - 1) : 0u;
        const uint32_t ea = va ? run_end(ga) : 0u, eb = vb ? run_end(gb) : 0u;
        const uint32_t lmax = __reduce_max_sync(0xffffffffu, max(va ? ea - sa : 0u, vb ? eb - sb : 0u));
        uint32_t da = sa, db = sb;
        if (lmax > 1) {
            const uint32_t qa = (uint32_t)(ka >> cs), qb = (uint32_t)(kb >> cs);
            // the chunk's positions are [32 c, 32 c + 32): a run inside it
            // is seen whole by the shuffles
            bool slow_a = va && (sa < 32u * c || ea > 32u * c + 32u);
            bool slow_b = vb && (sb < 32u * (c + NW) || eb > 32u * (c + NW) + 32u);
            for (uint32_t t = 1; t < lmax; ++t) {
                const uint32_t da_ = __shfl_down_sync(0xffffffffu, qa, t), ua = __shfl_up_sync(0xffffffffu, qa, t);
                const uint32_t db_ = __shfl_down_sync(0xffffffffu, qb, t), ub = __shfl_up_sync(0xffffffffu, qb, t);
                const bool ina_d = pa + t < ea, ina_u = lane >= t && pa - t >= sa;
                const bool inb_d = pb + t < eb, inb_u = lane >= t && pb - t >= sb;
                da += (ina_d && da_ < qa ? 1u : 0u) + (ina_u && ua < qa ? 1u : 0u);
                db += (inb_d && db_ < qb ? 1u : 0u) + (inb_u && ub < qb ? 1u : 0u);
                slow_a = slow_a || (ina_d && da_ == qa) || (ina_u && ua == qa);
                slow_b = slow_b || (inb_d && db_ == qb) || (inb_u && ub == qb);
            }
            if (va && slow_a) {
                da = sa;
                for (uint32_t q = sa; q < ea; ++q) da += rec_less(YK[q], YN[q], ka, na) ? 1u : 0u;
            }
            if (vb && slow_b) {
                db = sb;
                for (uint32_t q = sb; q < eb; ++q) db += rec_less(YK[q], YN[q], kb, nb) ? 1u : 0u;
            }
        }
        if (va) {
            XK[da] = ka;
            XN[da] = na;
        }
        if (vb) {
            XK[db] = kb;
            XN[db] = nb;
        }
    }
    __syncthreads();
}

// Generic sort (any n): records from `src` (global memory) go into SK / SN
// grouped by digit, a digit's run in arrival order, then one thread per
// digit finishes its run (about one record) by insertion sort.
template <int NT, class Src>
__device__ __forceinline__ void sort_generic(const Part &A, uint32_t n, int shift, uint32_t ndig,
                                             const Src &src)
{
    const uint32_t dmask = ndig - 1u;
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t dg = (uint32_t)(src.key(i) >> shift) & dmask;
        atomicAdd(&A.DC[dg], 1u);
    }
    __syncthreads();
    block_scan_inplace_u32<NT>(A.DC, ndig, A.WS);  // counts -> run starts
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint64_t k = src.key(i);
        const uint32_t pos = atomicAdd(&A.DC[(uint32_t)(k >> shift) & dmask], 1u);
        A.SK[pos] = k;
        A.SN[pos] = src.nonce(i);
    }
    __syncthreads();
    // DC[g] is now the end of run g, i.e. run g is [DC[g-1], DC[g])
    uint64_t *SK = A.SK;
    uint32_t *SN = A.SN;
    for (uint32_t dg = threadIdx.x; dg < ndig; dg += NT) {
        const uint32_t s0 = dg ? A.DC[dg - 1] : 0u;
        const uint32_t s1 = A.DC[dg];
        for (uint32_t a = s0 + 1; a < s1; ++a) {
            const uint64_t kx = SK[a];
            const uint32_t nx = SN[a];
            uint32_t b = a;
            while (b > s0 && !rec_less(SK[b - 1], SN[b - 1], kx, nx)) {
                SK[b] = SK[b - 1];
                SN[b] = SN[b - 1];
                --b;
            }
            SK[b] = kx;
            SN[b] = nx;
        }
    }
    __syncthreads();
}

// ------------------------------------------------ match and the tables

// Everything after the sort, for partition f (n sorted records, Table-1
// offset `off`) of plot d: the next partition's halo (HALO), the pair
// counts and their scan, Table 1, then the mode's Table-2 output.  Starts
// and ends at a barrier; on failure (the status word says why) it skips
// the output, so a persistent caller goes on to its next item.
template <int MODE, bool HALO, int NT>
__device__ __forceinline__ void match_and_write(const Desc &d, uint32_t f, uint32_t n, uint64_t off,
                                                const Part &A, uint64_t *s_base, int *s_ok)
{
    constexpr bool EMIT = MODE == kSortHash || MODE == kSortEmit;  // look-back placement
    constexpr bool SLOTS = MODE == kSortSlots;
    constexpr uint32_t NW = NT / 32;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint64_t *SK = A.SK;
    uint32_t *SN = A.SN;
    uint32_t *ST = A.ST;  // overlays the dead digit counters
    // 1. cross-bucket match: the next partition's halo (its records within
    //    D of its lower edge, collected while the slots were filled) goes
    //    sorted right after this partition's records, so the pair scan
    //    below runs on into it; records n .. nt - 1 start no pairs here.
    uint32_t nt = n;
    if (HALO && d.hcap) {
        const uint32_t hcap = d.hcap;
        const uint64_t fn = (uint64_t)f + 1;
        const uint32_t hc = fn < (1ull << d.p) ? min(d.halo_cnt[fn], hcap) : 0u;
        for (uint32_t h = threadIdx.x; h < hc; h += NT) {
            SK[n + h] = d.halo_keys[fn * hcap + h];
            SN[n + h] = d.halo_nonces[fn * hcap + h];
        }
        __syncthreads();
        if (threadIdx.x == 0) {  // a few records (Poisson, mean 2^11 D / 2^(64-p))
            for (uint32_t a = n + 1; a < n + hc; ++a) {
                const uint64_t kx = SK[a];
                const uint32_t nx = SN[a];
                uint32_t b = a;
                for (; b > n && !rec_less(SK[b - 1], SN[b - 1], kx, nx); --b) {
                    SK[b] = SK[b - 1];
                    SN[b] = SN[b - 1];
                }
                SK[b] = kx;
                SN[b] = nx;
            }
        }
        __syncthreads();
        nt = n + hc;
    }
    // 2. per chunk of 32 sorted records (one per lane; warp w takes chunks
    //    [c0, c1), two at a time so that their loads overlap): the pairs
    //    starting at each record r, i.e. the later records up to
    //    lim = min(last key of r's logical bucket, key_r + D - 1), or
    //    key_r + D - 1 for the cross-bucket match (four probes, then one by
    //    one while all four match); the pair offsets inside the warp's
    //    chunks (warp scans); and the lane's Table-1 record {nonce, BE
    //    key64}, three 4-byte stores (a warp's stores cover its chunk's 384
    //    bytes).  Probes may read up to three entries past the records; they
    //    lie inside the shared allocation and are masked.
    const uint32_t nch = (n + 31u) >> 5;
    const uint32_t c0 = warp * nch / NW, c1 = (warp + 1) * nch / NW;
    const uint32_t rend = min(32u * c1, n);  // the warp's records end here
    const uint64_t D = d.D;
    const bool global = HALO && d.scope != 0;
    uint32_t *__restrict__ t1w = reinterpret_cast<uint32_t *>(d.t1) + 3 * off;
    auto limit_of = [&](uint64_t k) -> uint64_t {
        const uint64_t last_in_bucket = global ? ~0ull : (k | ((1ull << 40) - 1));
        uint64_t reach = k + (D - 1);
        if (reach < k) reach = ~0ull;  // saturate
        return reach < last_in_bucket ? reach : last_in_bucket;
    };
    auto count_from = [&](uint32_t r, uint64_t lim, uint64_t k1, uint64_t k2, uint64_t k3,
                          uint64_t k4) -> uint32_t {
        const bool m1 = r + 1 < nt && k1 <= lim;
        const bool m2 = m1 && r + 2 < nt && k2 <= lim;
        const bool m3 = m2 && r + 3 < nt && k3 <= lim;
        const bool m4 = m3 && r + 4 < nt && k4 <= lim;
        uint32_t cnt = (uint32_t)m1 + (uint32_t)m2 + (uint32_t)m3 + (uint32_t)m4;
        if (m4)
            for (uint32_t q = r + 5; q < nt && SK[q] <= lim; ++q) ++cnt;
        return cnt;
    };
    uint32_t carry = 0;  // pairs of the warp's chunks before the current one
    for (uint32_t c = c0; c < c1; c += 2) {
        const uint32_t ra = 32u * c + lane, rb = ra + 32u;
        const bool va = ra < n, vb = c + 1 < c1 && rb < n;
        const uint32_t xa = va ? ra : 0u, xb = vb ? rb : 0u;
        const uint64_t ka = SK[xa], kb = SK[xb];
        const uint64_t a1 = SK[xa + 1], a2 = SK[xa + 2], a3 = SK[xa + 3], a4 = SK[xa + 4];
        const uint64_t b1 = SK[xb + 1], b2 = SK[xb + 2], b3 = SK[xb + 3], b4 = SK[xb + 4];
        const uint32_t na = SN[xa], nb = SN[xb];
        if (va) {
            t1w[3u * ra] = na;
            t1w[3u * ra + 1] = bswap32((uint32_t)(ka >> 32));
            t1w[3u * ra + 2] = bswap32((uint32_t)ka);
        }
        if (vb) {
            t1w[3u * rb] = nb;
            t1w[3u * rb + 1] = bswap32((uint32_t)(kb >> 32));
            t1w[3u * rb + 2] = bswap32((uint32_t)kb);
        }
        const uint32_t cA = va ? count_from(ra, limit_of(ka), a1, a2, a3, a4) : 0u;
        const uint32_t cB = vb ? count_from(rb, limit_of(kb), b1, b2, b3, b4) : 0u;
        const uint32_t iA = warp_incl_scan(cA), iB = warp_incl_scan(cB);
        const uint32_t tA = __shfl_sync(0xffffffffu, iA, 31);
        if (va) ST[ra] = carry + iA - cA;
        if (vb) ST[rb] = carry + tA + iB - cB;
        carry += tA + __shfl_sync(0xffffffffu, iB, 31);
    }
    if (lane == 0) A.WS[warp] = carry;
    __syncthreads();
    uint32_t P = 0, wbase = 0;  // the partition's pairs; those before this warp's chunks
#pragma unroll
    for (uint32_t w = 0; w < NW; ++w) {
        const uint32_t t = A.WS[w];
        wbase += w < warp ? t : 0u;
        P += t;
    }
    const bool withhold = (d.test_flags & 1u) != 0;
    if (threadIdx.x == 0) {
        d.pairs[f] = P;  // lets vx_match re-run the match alone
        if (EMIT) lb_publish(d.lb, f, P, withhold);
    }
    if (MODE == kSortCount) {
        __syncthreads();
        return;
    }
    // 3. the Table-2 base: the look-back (warp 0), or the partition's slot
    bool ok = true;
    uint64_t base = 0;
    if (EMIT) {
        if (threadIdx.x < 32) {
            uint64_t excl = 0;
            int got = lb_resolve(d.lb, f, P, d.status, d.spin_limit, withhold, &excl) ? 1 : 0;
            if (threadIdx.x == 0) {
                if (got) {
                    const uint64_t np = 1ull << d.p;
                    d.t2off[f] = excl;
                    if (f + 1 == np) d.t2off[np] = excl + P;
                    if (excl + P > d.t2cap) {
                        atomicOr(d.status, kStT2Capacity);
                        got = 0;
                    }
                }
                *s_base = excl;
                *s_ok = got;
            }
        }
        __syncthreads();
        ok = *s_ok != 0;
        base = *s_base;
    } else if (P > d.cap2 + d.cap2 / 2u) {
        if (threadIdx.x == 0) atomicOr(d.status, kStPairSlot);
        ok = false;
    }
    // 4. the pairs, in (i, j) order: chunk by chunk (two at a time), a
    //    lane's record r starts its pairs (r, r + 1 + j) at its offset.
    //    Slot placement: when the pairs fit the key array of shared memory
    //    (dead since step 2) they are listed there and leave in one bulk
    //    copy (thread 0's bulk group; the caller waits for its read before
    //    the buffer is written again), else they go straight to the slot.
    uint4 *__restrict__ out = reinterpret_cast<uint4 *>(d.t2) + base;
    uint2 *__restrict__ pa = reinterpret_cast<uint2 *>(d.b_keys + (uint64_t)f * d.cap2);
    uint2 *__restrict__ pb = reinterpret_cast<uint2 *>(d.b_nonces + (uint64_t)f * d.cap2);
    const uint32_t capA = d.cap2;
    const bool staged = SLOTS && P < capA;
    uint2 *SP = reinterpret_cast<uint2 *>(SK);
    auto emit = [&](uint32_t x, uint32_t a, uint32_t b) {
        if (SLOTS)
            *(staged ? SP + x : x < capA ? pa + x : pb + (x - capA)) = make_uint2(a, b);
        else
            out[x] = make_uint4(a, b, 0u, 0u);
    };
    if (ok) {
        for (uint32_t c = c0; c < c1; c += 2) {
            const uint32_t ra = 32u * c + lane, rb = ra + 32u;
            const bool va = ra < n, vb = c + 1 < c1 && rb < n;
            // offsets inside the warp's pairs; a record's count is the gap
            // to the next record's offset (the warp's total after its last)
            const uint32_t sa = va ? ST[ra] : 0u, sb = vb ? ST[rb] : 0u;
            const uint32_t ea = va ? (ra + 1 < rend ? ST[ra + 1] : carry) : 0u;
            const uint32_t eb = vb ? (rb + 1 < rend ? ST[rb + 1] : carry) : 0u;
            const uint32_t aa = va ? SN[ra] : 0u, ab = vb ? SN[rb] : 0u;
            const uint32_t cA = ea - sa, cB = eb - sb;
            // the first four partners of each record, read together (the
            // reads past the records stay inside the shared allocation)
            const uint32_t xa = va ? ra : 0u, xb = vb ? rb : 0u;
            const uint32_t a1 = SN[xa + 1], a2 = SN[xa + 2], a3 = SN[xa + 3], a4 = SN[xa + 4];
            const uint32_t b1 = SN[xb + 1], b2 = SN[xb + 2], b3 = SN[xb + 3], b4 = SN[xb + 4];
            if (MODE == kSortHash) {
                __syncwarp();  // every lane has read its neighbour's offset
                if (va) ST[ra] = wbase + sa;  // offsets for the listing below
                if (vb) ST[rb] = wbase + sb;
                continue;
            }
            const uint32_t oa = wbase + sa, ob = wbase + sb;
            if (cA > 0) emit(oa, aa, a1);
            if (cA > 1) emit(oa + 1, aa, a2);
            if (cA > 2) emit(oa + 2, aa, a3);
            if (cA > 3) emit(oa + 3, aa, a4);
            if (cB > 0) emit(ob, ab, b1);
            if (cB > 1) emit(ob + 1, ab, b2);
            if (cB > 2) emit(ob + 2, ab, b3);
            if (cB > 3) emit(ob + 3, ab, b4);
            for (uint32_t j = 4; __any_sync(0xffffffffu, j < cA || j < cB); ++j) {
                if (j < cA) emit(oa + j, aa, SN[ra + 1 + j]);
                if (j < cB) emit(ob + j, ab, SN[rb + 1 + j]);
            }
        }
        if (staged) {
            __syncthreads();
            if (threadIdx.x == 0 && P) bulk_s2g(pa, SP, ((P + 1u) & ~1u) * 8u);
        }
    }
    if (MODE == kSortHash && ok) {
        // hash here: list the pairs window by window, every lane hashes
        __syncthreads();
        uint32_t g[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
        uint32_t *LS = A.LS;
        for (uint32_t w0 = 0; w0 < P; w0 += kSMList) {
            const uint32_t w1 = min(P, w0 + kSMList);
            for (uint32_t r = threadIdx.x; r < n; r += NT) {
                const uint32_t s = ST[r];
                const uint32_t e = r + 1 < n ? ST[r + 1] : P;
                const uint32_t lo = max(s, w0), hi = min(e, w1);
                for (uint32_t k = lo; k < hi; ++k) LS[k - w0] = r | ((r + 1 + (k - s)) << 16);
            }
            __syncthreads();
            for (uint32_t q = threadIdx.x; q < w1 - w0; q += NT) {
                const uint32_t e = LS[q];
                const uint32_t a = SN[e & 0xffffu], b = SN[e >> 16];
                uint32_t h0, h1;
                b3_finish<true>(g, a, b, h0, h1);
                out[w0 + q] = make_uint4(a, b, h0, h1);
            }
            __syncthreads();
        }
    }
    __syncthreads();
}

__device__ __forceinline__ Part part_arrays(unsigned char *base, const SMLayout &L)
{
    Part A;
    A.SK = reinterpret_cast<uint64_t *>(base + L.xk);
    A.SN = reinterpret_cast<uint32_t *>(base + L.xn);
    A.DC = reinterpret_cast<uint32_t *>(base + L.dc);
    A.ST = A.DC;  // overlays the digit counters (dead once the runs are sorted)
    A.LS = reinterpret_cast<uint32_t *>(base + L.list);
    A.WS = reinterpret_cast<uint32_t *>(base + L.ws);
    return A;
}

// A slot in global memory, read through the read-only path unless this
// kernel later overwrites it with the partition's pairs (RO false).
template <bool RO>
struct GlobalSrc {
    const uint64_t *k;
    const uint32_t *n;
    __device__ __forceinline__ uint64_t key(uint32_t i) const { return RO ? __ldg(k + i) : k[i]; }
    __device__ __forceinline__ uint32_t nonce(uint32_t i) const { return RO ? __ldg(n + i) : n[i]; }
};

// ------------------------------------------------- persistent front end
// Work item t of the launch (CTA b takes b, b + G, b + 2G, ...) belongs to
// plot find_plot(t); its partition is the plot's next ticket (look-back
// modes) or t - tile_start[plot].  A CTA takes the ticket of item k + 2
// and reads the fill count of item k + 1 at the start of item k, and
// starts item k + 1's slot copy once item k's slot has been sorted into
// registers, so the global round trips and the copy overlap item k's work.
// A CTA takes tickets in its processing order and only while running, so
// the lowest unpublished partition is always being worked on: the
// look-back chain cannot stall on a CTA that is not resident.
struct Item {
    int plot;
    uint32_t f;
    bool ok;
};

// Starts an L2 prefetch of the filled part of partition f's slot (f below
// 2^p), so that the reads that come for it later hit L2.  (Two items ahead
// in the persistent front end it measured 1% slower: its bulk copies do not
// wait on DRAM latency.)
__device__ __forceinline__ void prefetch_slot_l2(const Desc &d, uint32_t f)
{
    const uint32_t nf = min(d.cnt2[f], d.cap2);
    if (!nf) return;
    const uint32_t nk = (nf + 1u) & ~1u, nn = (nf + 3u) & ~3u;  // 16-byte multiples
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_keys + (uint64_t)f * d.cap2),
                 "r"(nk * 8u)
                 : "memory");
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_nonces + (uint64_t)f * d.cap2),
                 "r"(nn * 4u)
                 : "memory");
}

template <bool EMIT>
__device__ __forceinline__ Item take_item(const Desc *__restrict__ descs, int nplots,
                                          const uint32_t *__restrict__ tile_start, uint32_t t)
{
    Item it;
    it.plot = find_plot(tile_start, nplots, t);
    const Desc &d = descs[it.plot];
    it.f = EMIT ? atomicAdd(d.ticket, 1u) : t - __ldg(tile_start + it.plot);
    it.ok = true;
    return it;
}

template <int MODE, bool HALO>
__global__ void __launch_bounds__(kPipeThreads, MODE == kSortHash ? 2 : 3)
    k_sortmatch_pipe(const Desc *__restrict__ descs, int nplots, const uint32_t *__restrict__ tile_start,
                     uint32_t items, uint32_t max_cap, int max_dbits)
{
    constexpr bool EMIT = MODE == kSortHash || MODE == kSortEmit;
    constexpr int NT = kPipeThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_plot;
    __shared__ uint32_t s_f, s_n;
    __shared__ int s_valid;
    __shared__ uint64_t s_base;
    __shared__ int s_ok;
    const SMLayout L(max_cap, max_dbits, MODE == kSortHash, true);
    Part A = part_arrays(smem_raw, L);
    uint64_t *const XK = reinterpret_cast<uint64_t *>(smem_raw + L.xk);
    uint32_t *const XN = reinterpret_cast<uint32_t *>(smem_raw + L.xn);
    uint64_t *const YK = reinterpret_cast<uint64_t *>(smem_raw + L.yk);
    uint32_t *const YN = reinterpret_cast<uint32_t *>(smem_raw + L.yn);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + L.bar);
    const uint32_t G = gridDim.x;

    // Thread 0's pipeline: the item after the current one (its ticket and,
    // from the start of the current item on, its fill count) and the one
    // after that (its ticket).
    Item nx{0, 0, false}, nn{0, 0, false};
    uint32_t nx_n = 0;
    // Starts the copy of item `it` (n records) into buffer b and publishes
    // it as the next item; an invalid or empty item completes the barrier
    // phase with no copy.
    auto launch_copy = [&](const Item &it, uint32_t n, int b) {
        // Only if the ticket was not reset: report, never index with it.
        const bool valid = it.ok && it.f < (1u << descs[it.plot].p);
        if (it.ok && !valid) atomicOr(descs[it.plot].status, kStBadTicket);
        const uint32_t cnt = valid ? n : 0u;
        const uint32_t nk = (cnt + 1u) & ~1u, nnz = (cnt + 3u) & ~3u;  // 16-byte multiples
        // The buffer was last accessed by ordinary loads and stores: order
        // those before the copy engine's writes.
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(bar, nk * 8u + nnz * 4u);
        if (cnt) {
            const Desc &d = descs[it.plot];
            bulk_g2s(b ? YK : XK, d.b_keys + (uint64_t)it.f * d.cap2, nk * 8u, bar);
            bulk_g2s(b ? YN : XN, d.b_nonces + (uint64_t)it.f * d.cap2, nnz * 4u, bar);
        }
        s_plot = it.plot;
        s_f = it.f;
        s_n = cnt;
        s_valid = valid ? 1 : 0;
    };
    if (threadIdx.x == 0) {
        mbar_init(bar, 1);
        if (blockIdx.x < items) {
            const Item i0 = take_item<EMIT>(descs, nplots, tile_start, blockIdx.x);
            const uint32_t n0 = i0.f < (1u << descs[i0.plot].p) ? descs[i0.plot].cnt2[i0.f] : 0u;
            if (blockIdx.x + G < items) nx = take_item<EMIT>(descs, nplots, tile_start, blockIdx.x + G);
            launch_copy(i0, min(n0, descs[i0.plot].cap2), 0);
        }
    }
    __syncthreads();
    uint32_t phase = 0;
    int rb = 0;  // buffer holding the current item's slot, then its sorted records
    for (uint32_t t = blockIdx.x; t < items; t += G, phase ^= 1u, rb ^= 1) {
        const int plot = s_plot;
        const uint32_t f = s_f, n = s_n;
        const bool valid = s_valid != 0;
        const Desc &d = descs[plot];
        if (threadIdx.x == 0) {
            if (nx.ok) {
                const Desc &dn = descs[nx.plot];
                nx_n = nx.f < (1u << dn.p) ? min(dn.cnt2[nx.f], dn.cap2) : 0u;
            }
            if (t + 2 * G < items) nn = take_item<EMIT>(descs, nplots, tile_start, t + 2 * G);
        }
        const uint32_t ndig = 1u << d.dbits;
        if (ndig % 4u == 0) {
            uint4 *D4 = reinterpret_cast<uint4 *>(A.DC);
            for (uint32_t i = threadIdx.x; i < ndig / 4u; i += NT) D4[i] = make_uint4(0u, 0u, 0u, 0u);
        } else {
            for (uint32_t i = threadIdx.x; i < ndig; i += NT) A.DC[i] = 0u;
        }
        const uint64_t off = valid ? d.t1off[f] : 0ull;
        // The slot copy was started during the previous item (or above).
        if (!__syncthreads_and(mbar_wait(bar, phase, d.spin_limit))) {
            if (threadIdx.x == 0) atomicOr(d.status, kStTimeout);
            mbar_wait(bar, phase, d.spin_limit);  // let it land before the CTA exits
            return;
        }
        A.SK = rb ? YK : XK;
        A.SN = rb ? YN : XN;
        // One more digit bit in the same counter words where they allow it.
        const int shift = 64 - d.pk - d.dbits;
        // The previous item's staged pairs leave the buffer this item
        // places its records into while the sort counts its digits.
        constexpr bool DR = SLOTS_MODE(MODE);
        if (valid && n < 0x10000u && rows_shape<NT, 8>(ndig))
            sort_pingpong<NT, true, DR>(A, A.SK, A.SN, rb ? XK : YK, rb ? XN : YN, n, shift - 1, ndig << 1);
        else if (valid)
            sort_pingpong<NT, false, DR>(A, A.SK, A.SN, rb ? XK : YK, rb ? XN : YN, n, shift, ndig);
        // The other buffer is free: start the next item's copy into it
        // (after the staged pairs' reads, already over unless no sort ran).
        if (threadIdx.x == 0) {
            if (DR) bulk_wait_all<true>();
            if (nx.ok) launch_copy(nx, nx_n, rb ^ 1);
            nx = nn;
            nn.ok = false;
        }
        if (valid) {
            match_and_write<MODE, HALO, NT>(d, f, n, off, A, &s_base, &s_ok);
        } else {
            __syncthreads();
        }
    }
    if (SLOTS_MODE(MODE) && threadIdx.x == 0) bulk_wait_all<false>();
}

// ------------------------------------- one CTA per partition front end
template <int MODE, bool HALO>
__global__ void __launch_bounds__(kGlThreads, MODE == kSortHash ? 2 : 3)
    k_sortmatch_gl(const Desc *__restrict__ descs, int nplots, const uint32_t *__restrict__ tile_start)
{
    constexpr bool EMIT = MODE == kSortHash || MODE == kSortEmit;
    constexpr int NT = kGlThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ uint32_t s_f;
    __shared__ uint64_t s_base;
    __shared__ int s_ok;
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    if (EMIT) {
        if (threadIdx.x == 0) s_f = atomicAdd(d.ticket, 1u);
        __syncthreads();
    }
    const uint32_t f = EMIT ? s_f : (blockIdx.x - tile_start[plot]);
    if (f >= (1u << d.p)) {  // only if the ticket was not reset: report, never index with it
        if (threadIdx.x == 0) atomicOr(d.status, kStBadTicket);
        return;
    }
    const uint32_t cap = d.cap2;
    const SMLayout L(cap + (HALO ? d.hcap : 0u), d.dbits, MODE == kSortHash, false);
    const Part A = part_arrays(smem_raw, L);
    const uint32_t ndig = 1u << d.dbits;
    for (uint32_t i = threadIdx.x; i < ndig; i += NT) A.DC[i] = 0u;
    // Warm L2 with the filled part of the slot kSlotPrefetchAhead tickets
    // ahead, so that its CTA's reads hit L2.
    const uint64_t fa = (uint64_t)f + kSlotPrefetchAhead;
    if (threadIdx.x == 0 && fa < (1ull << d.p)) prefetch_slot_l2(d, (uint32_t)fa);
    const uint32_t n = min(d.cnt2[f], cap);
    const uint64_t off = d.t1off[f];
    __syncthreads();
    sort_generic<NT>(A, n, 64 - d.pk - d.dbits, ndig,
                     GlobalSrc<MODE != kSortSlots>{d.b_keys + (uint64_t)f * cap, d.b_nonces + (uint64_t)f * cap});
    match_and_write<MODE, HALO, NT>(d, f, n, off, A, &s_base, &s_ok);
    if (SLOTS_MODE(MODE) && threadIdx.x == 0) bulk_wait_all<false>();
}

size_t sortmatch_smem_bytes(uint32_t cap, int dbits) { return SMLayout(cap, dbits, true, false).bytes; }

uint32_t sortmatch_max_cap() { return 16384u; }

template <int MODE, bool HALO>
static cudaError_t launch_sm(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits)
{
    if (total_tiles == 0) return cudaSuccess;
    const size_t pipe = SMLayout(max_cap, max_dbits, MODE == kSortHash, true).bytes;
    if (pipe <= kMaxSmemPerCta) {
        auto fn = k_sortmatch_pipe<MODE, HALO>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pipe);
        if (e != cudaSuccess) return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPipeThreads, pipe)) != cudaSuccess)
            return e;
        const uint64_t want = (uint64_t)(per_sm > 0 ? per_sm : 1) * (uint64_t)sms;
        const uint32_t grid = (uint32_t)(want < total_tiles ? want : total_tiles);
        fn<<<grid, kPipeThreads, pipe, s>>>(descs, nplots, tile_start, total_tiles, max_cap, max_dbits);
        return cudaGetLastError();
    }
    const size_t smem = SMLayout(max_cap, max_dbits, MODE == kSortHash, false).bytes;
    auto fn = k_sortmatch_gl<MODE, HALO>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<total_tiles, kGlThreads, smem, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

template <int MODE>
static cudaError_t launch_sm2(const Desc *descs, int nplots, const uint32_t *tile_start,
                              uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                              bool halo)
{
    // HALO instances carry the cross-bucket code; plain launches do not.
    return halo ? launch_sm<MODE, true>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits)
                : launch_sm<MODE, false>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits);
}

cudaError_t launch_sortmatch(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                             SortMatchOut out, bool halo)
{
    if (out == kOutLookbackHashed)
        return launch_sm2<kSortHash>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits, halo);
    if (out == kOutSlots)
        return launch_sm2<kSortSlots>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits, halo);
    return launch_sm2<kSortEmit>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits, halo);
}

cudaError_t launch_sort(const Desc *descs, int nplots, const uint32_t *tile_start,
                        uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                        bool halo)
{
    return launch_sm2<kSortCount>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits, halo);
}

}  // namespace vx
