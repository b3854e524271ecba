// k_sort2.cu -- Table 2 sorted by its hash (hash2), for lookups by a prover.
//
// Paper: a plot is searched by hash value (Sec. I-B, the VaultX prover); the
// paper's Table 2 stays in pair order.  This pass orders the same 16-byte
// records {a, b, hash2} by (key2, a, b), key2 = big-endian u64 of hash2,
// with the Table-1 machinery applied to 16-byte records: a first scatter
// level by the top p1 bits of key2, a second level by the next p2 bits into
// 2^p Poisson-sized partitions, a scan of the partition counts, and a
// shared-memory sort of every partition (counting sort on the next
// dbits + 1 key bits, each record ranked inside its digit run by warp
// shuffles) that writes its records straight back into the Table-2 buffer
// at their places.  Table 2 is read completely by
// the first level before anything writes it.
#include "vx_internal.cuh"
#include "vx_plan.h"

namespace vx {

constexpr int kS2Threads = 512;              // first level: 512 threads x 8 records
constexpr int kS2PerThread = 8;
constexpr uint32_t kS2Tile1 = kS2Threads * kS2PerThread;
static_assert(kS2Tile1 == kPlanS2Tile1, "planner and first-level sort tiles differ");
constexpr int kS2BThreads = 512;             // second level: 512 threads x 8 records
constexpr uint32_t kS2Tile2 = 4096;
constexpr int kS2SortThreads = 256;

__device__ __forceinline__ uint64_t sort2_key(uint4 r)
{
    return ((uint64_t)bswap32(r.z) << 32) | bswap32(r.w);
}

// ------------------------------------------------------------------ setup
__global__ void k_s2_setup(Sort2Desc *dp)
{
    Sort2Desc &d = *dp;
    const uint64_t n1 = d.p2 > 0 ? (1ull << d.p1) : 0ull;
    const uint64_t n2 = 1ull << d.p;
    const uint64_t nchunks = (n2 + kScanChunk - 1) / kScanChunk;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) *d.ticket = 0u;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n2; i += stride) {
        d.cnt2[i] = 0u;
        if (i < n1) d.cnt1[i] = 0u;
        if (i < nchunks) d.lbs[i] = 0ull;
    }
}

// ---------------------------------------------------- first scatter level
// A CTA takes kS2Tile1 consecutive Table-2 records, ranks them in shared memory
// by their level bin, claims one run per (CTA, bin) with a global atomic,
// and writes them bin by bin (key2 and the packed pair (a << 32 | b)).
struct S2Smem1 {
    uint64_t keys[kS2Tile1];
    uint64_t vals[kS2Tile1];
    uint32_t hist[1 << kMaxCoarseBits];
    uint32_t loff[1 << kMaxCoarseBits];
    uint32_t gbase[1 << kMaxCoarseBits];
    uint32_t ws[kS2Threads / 32 + 1];
};

__global__ void __launch_bounds__(kS2Threads) k_s2_scatter1(const Sort2Desc *__restrict__ dp)
{
    constexpr int NT = kS2Threads, PER = kS2PerThread;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S2Smem1 &sm = *reinterpret_cast<S2Smem1 *>(smem_raw);
    const Sort2Desc &d = *dp;
    const uint64_t n = *d.count;
    const uint64_t base = (uint64_t)blockIdx.x * kS2Tile1;
    if (base >= n) return;
    const bool two_level = d.p2 > 0;
    const int bits = two_level ? d.p1 : d.p;
    const int nbins = 1 << bits;
    const uint32_t cap = two_level ? d.cap1 : d.cap2;
    uint64_t *okeys = two_level ? d.a_keys : d.b_keys;
    uint64_t *ovals = two_level ? d.a_vals : d.b_vals;
    uint32_t *cnt = two_level ? d.cnt1 : d.cnt2;
    for (int b = threadIdx.x; b < nbins; b += NT) sm.hist[b] = 0u;
    __syncthreads();
    uint64_t key[PER], val[PER];
    uint32_t rank[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t i = base + (uint64_t)j * NT + threadIdx.x;
        const bool valid = i < n;
        const uint4 r = valid ? d.t2[i] : make_uint4(0u, 0u, 0u, 0u);
        key[j] = sort2_key(r);
        val[j] = ((uint64_t)r.x << 32) | r.y;
        const uint32_t bin = bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u;
        rank[j] = valid ? atomicAdd(&sm.hist[bin], 1u) : 0u;
    }
    __syncthreads();
    constexpr int PB = ((1 << kMaxCoarseBits) + NT - 1) / NT;  // most bins a thread owns
    const int per = (nbins + NT - 1) / NT;
    const int b0 = threadIdx.x * per;
    uint32_t claim[PB];
    {
        uint32_t loc = 0;
        for (int k = 0; k < per; ++k)
            if (b0 + k < nbins) loc += sm.hist[b0 + k];
        uint32_t total;
        uint32_t run = block_exclusive_scan_u32<NT>(loc, sm.ws, &total);
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int b = b0 + k;
            claim[k] = 0u;
            if (k < per && b < nbins) {
                const uint32_t h = sm.hist[b];
                sm.loff[b] = run;
                run += h;
                if (h) claim[k] = atomicAdd(&cnt[b], h);  // result first needed after the restage
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint64_t i = base + (uint64_t)j * NT + threadIdx.x;
        if (i < n) {
            const uint32_t bin = bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u;
            const uint32_t pos = sm.loff[bin] + rank[j];
            sm.keys[pos] = key[j];
            sm.vals[pos] = val[j];
        }
    }
#pragma unroll
    for (int k = 0; k < PB; ++k)
        if (k < per && b0 + k < nbins) sm.gbase[b0 + k] = claim[k];
    __syncthreads();
    const uint32_t count = (uint32_t)(n - base < kS2Tile1 ? n - base : kS2Tile1);
    bool overflow = false;
    // unrolled over the thread's PER records so that their dependent
    // shared-memory reads (key, then its bin's bases) overlap
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        if (i >= count) break;
        const uint64_t k = sm.keys[i];
        const uint32_t bin = bits ? (uint32_t)(k >> (64 - bits)) : 0u;
        const uint32_t g = sm.gbase[bin] + (i - sm.loff[bin]);
        if (g < cap) {
            const uint64_t at = (uint64_t)bin * cap + g;
            okeys[at] = k;
            ovals[at] = sm.vals[i];
        } else {
            overflow = true;
        }
    }
    if (overflow) atomicOr(d.status, kStSort2);
}

// --------------------------------------------------- second scatter level
// One CTA per tile of up to 4096 records of a first-level slot: two TMA bulk
// copies (keys, packed pairs) into shared memory, ranks by the fine bin,
// claims issued before the in-place restage and read after it, coalesced
// runs out.
struct S2Smem2 {
    uint64_t keys[kS2Tile2];
    uint64_t vals[kS2Tile2];
    uint32_t hist[1 << kMaxFineBits];
    uint32_t loff[1 << kMaxFineBits];
    uint32_t gbase[1 << kMaxFineBits];
    uint32_t ws[kS2BThreads / 32 + 1];
    uint64_t bar;
};

__global__ void __launch_bounds__(kS2BThreads) k_s2_scatter2(const Sort2Desc *__restrict__ dp)
{
    constexpr int NT = kS2BThreads;
    constexpr int PER = kS2Tile2 / NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    S2Smem2 &sm = *reinterpret_cast<S2Smem2 *>(smem_raw);
    const Sort2Desc &d = *dp;
    const uint32_t c = blockIdx.x / d.chunks1;
    const uint32_t part = blockIdx.x - c * d.chunks1;
    const uint32_t filled = min(d.cnt1[c], d.cap1);
    const uint32_t start = part * kS2Tile2;
    if (start >= filled) return;
    const uint32_t count = min(kS2Tile2, filled - start);
    const int p2 = d.p2;
    const int nbins = 1 << p2;
    const int shift = 64 - d.p;
    const uint32_t bin_mask = (uint32_t)nbins - 1u;
    const uint32_t ncopy = (count + 1u) & ~1u;  // 16-byte multiples; cap1 is even
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        mbar_expect_tx(&sm.bar, ncopy * 16u);
        bulk_g2s(sm.keys, d.a_keys + (uint64_t)c * d.cap1 + start, ncopy * 8u, &sm.bar);
        bulk_g2s(sm.vals, d.a_vals + (uint64_t)c * d.cap1 + start, ncopy * 8u, &sm.bar);
    }
    for (int b = threadIdx.x; b < nbins; b += NT) sm.hist[b] = 0u;
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(&sm.bar, 0, d.spin_limit))) {  // one answer for all threads
        if (threadIdx.x == 0) atomicOr(d.status, kStTimeout);
        mbar_wait(&sm.bar, 0, d.spin_limit);  // let the copy land before leaving
        return;
    }
    uint64_t key[PER], val[PER];
    uint32_t rank[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        const bool valid = i < count;
        key[j] = valid ? sm.keys[i] : 0ull;
        val[j] = valid ? sm.vals[i] : 0ull;
        const uint32_t bin = (uint32_t)(key[j] >> shift) & bin_mask;
        rank[j] = valid ? atomicAdd(&sm.hist[bin], 1u) : 0u;
    }
    __syncthreads();
    constexpr int PB = ((1 << kMaxFineBits) + NT - 1) / NT;
    const int per = (nbins + NT - 1) / NT;
    const int b0 = threadIdx.x * per;
    uint32_t claim[PB];
    {
        uint32_t loc = 0;
        for (int k = 0; k < per; ++k)
            if (b0 + k < nbins) loc += sm.hist[b0 + k];
        uint32_t total;
        uint32_t run = block_exclusive_scan_u32<NT>(loc, sm.ws, &total);
#pragma unroll
        for (int k = 0; k < PB; ++k) {
            const int b = b0 + k;
            claim[k] = 0u;
            if (k < per && b < nbins) {
                const uint32_t h = sm.hist[b];
                sm.loff[b] = run;
                run += h;
                if (h) claim[k] = atomicAdd(&d.cnt2[((uint64_t)c << p2) + b], h);
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        if (i < count) {
            const uint32_t bin = (uint32_t)(key[j] >> shift) & bin_mask;
            const uint32_t pos = sm.loff[bin] + rank[j];
            sm.keys[pos] = key[j];
            sm.vals[pos] = val[j];
        }
    }
#pragma unroll
    for (int k = 0; k < PB; ++k)
        if (k < per && b0 + k < nbins) sm.gbase[b0 + k] = claim[k];
    __syncthreads();
    const uint32_t cap = d.cap2;
    bool overflow = false;
#pragma unroll
    for (int j = 0; j < (int)(kS2Tile2 / kS2BThreads); ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        if (i >= count) break;
        const uint64_t k = sm.keys[i];
        const uint32_t bin = (uint32_t)(k >> shift) & bin_mask;
        const uint32_t g = sm.gbase[bin] + (i - sm.loff[bin]);
        if (g < cap) {
            const uint64_t at = (((uint64_t)c << p2) + bin) * cap + g;
            d.b_keys[at] = k;
            d.b_vals[at] = sm.vals[i];
        } else {
            overflow = true;
        }
    }
    if (overflow) atomicOr(d.status, kStSort2);
}

// --------------------------------------------------------- offsets scan
// Exclusive prefix of the 2^p partition counts (clipped to the slot), 4096
// counters per CTA, chunks chained by decoupled look-back in ticket order;
// the last chunk checks that every record arrived.
__global__ void __launch_bounds__(256) k_s2_scan(const Sort2Desc *__restrict__ dp)
{
    constexpr int NT = 256;
    constexpr uint32_t PER = kScanChunk / NT;
    __shared__ uint32_t ws[NT / 32 + 1];
    __shared__ uint32_t s_c;
    __shared__ uint64_t s_base;
    __shared__ int s_ok;
    const Sort2Desc &d = *dp;
    if (threadIdx.x == 0) s_c = atomicAdd(d.ticket, 1u);
    __syncthreads();
    const uint32_t c = s_c;
    const uint64_t np = 1ull << d.p;
    const uint32_t nchunks = (uint32_t)((np + kScanChunk - 1) / kScanChunk);
    if (c >= nchunks) {
        if (threadIdx.x == 0) atomicOr(d.status, kStBadTicket);
        return;
    }
    const uint64_t b0 = (uint64_t)c * kScanChunk + (uint64_t)threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t loc = 0;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        v[k] = b0 + k < np ? min(d.cnt2[b0 + k], d.cap2) : 0u;
        loc += v[k];
    }
    uint32_t total;
    const uint32_t run = block_exclusive_scan_u32<NT>(loc, ws, &total);
    if (threadIdx.x < 32) {
        uint64_t excl = 0;
        const int ok = lookback_warp(d.lbs, c, total, d.status, d.spin_limit, false, &excl) ? 1 : 0;
        if (threadIdx.x == 0) {
            s_ok = ok;
            s_base = excl;
        }
    }
    __syncthreads();
    if (!s_ok) return;
    uint64_t at = s_base + run;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        if (b0 + k < np) d.off[b0 + k] = at;
        at += v[k];
    }
    if (c + 1 == nchunks && threadIdx.x == 0) {
        const uint64_t all = s_base + total;
        d.off[np] = all;
        if (all != *d.count) atomicOr(d.status, kStSort2);
    }
}

// In-place exclusive scan of 2M digit counters of 16 bits, two to a word
// (digit 2w in the low half of word w, 2w + 1 in the high half; every
// count and start below 2^16), by a CTA of NT threads: each word's two
// counts become their starts.  Warp w takes a contiguous run of the words,
// 32 at a time; `ws` holds NT/32 words.  Ends with a __syncthreads.
template <int NT>
__device__ __forceinline__ void block_scan_packed16(uint32_t *A, uint32_t M, uint32_t *ws)
{
    constexpr int NW = NT / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t chunk = (M + NW - 1) / NW;
    const uint32_t lo = min(M, (uint32_t)warp * chunk), hi = min(M, lo + chunk);
    uint32_t sum = 0;
    for (uint32_t i = lo + lane; i < hi; i += 32) sum += (A[i] & 0xFFFFu) + (A[i] >> 16);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (lane == 0) ws[warp] = sum;
    __syncthreads();
    uint32_t carry = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) carry += w < warp ? ws[w] : 0u;
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t i = base + lane;
        const uint32_t a = i < hi ? A[i] : 0u, l = a & 0xFFFFu, v = l + (a >> 16);
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t P = carry + incl - v;
        if (i < hi) A[i] = P | ((P + l) << 16);
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    __syncthreads();
}

// ------------------------------------------------------- partition sort
// One CTA per partition: counting sort on the dbits key bits below the
// partition prefix, then each record ranked inside its digit run by
// (key2, a, b) with warp shuffles and written straight to its place at the
// partition's offset as {a, b, hash2}.  Shared memory holds each record's
// key and its index in the slot (12 B with the digit rank); the packed pair
// is read from the slot (L2) when the record is written out, or when two
// keys tie.
constexpr uint32_t kS2PrefetchAhead = 384;  // partitions ahead: ~half the resident CTAs

struct S2SortLayout {
    size_t idx, rank, dcnt, ws, bytes;
    __host__ __device__ S2SortLayout(uint32_t cap, int dbits)
    {
        idx = (size_t)cap * 8;
        rank = idx + (size_t)((cap + 1) & ~1u) * 2;
        dcnt = rank + (size_t)((cap + 1) & ~1u) * 2;
        ws = dcnt + ((size_t)1 << dbits) * 4;
        bytes = ws + 40 * 4;
    }
};

__global__ void __launch_bounds__(kS2SortThreads, 5) k_s2_sort(const Sort2Desc *__restrict__ dp)
{
    constexpr int NT = kS2SortThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Sort2Desc &d = *dp;
    if (*d.status & (kStSort2 | kStTimeout | kStBadTicket)) return;  // offsets not trusted
    const uint32_t f = blockIdx.x;
    const uint32_t cap = d.cap2;
    const int dbits = d.dbits;
    const uint32_t ndig = 1u << dbits;
    const S2SortLayout L(cap, dbits);
    uint64_t *SK = reinterpret_cast<uint64_t *>(smem_raw);
    uint16_t *SI = reinterpret_cast<uint16_t *>(smem_raw + L.idx);
    uint16_t *RK = reinterpret_cast<uint16_t *>(smem_raw + L.rank);
    uint32_t *DC = reinterpret_cast<uint32_t *>(smem_raw + L.dcnt);
    uint32_t *WS = reinterpret_cast<uint32_t *>(smem_raw + L.ws);
    const uint32_t n = min(d.cnt2[f], cap);
    const uint64_t o = d.off[f];
    const uint64_t *__restrict__ ik = d.b_keys + (uint64_t)f * cap;
    const uint64_t *__restrict__ iv = d.b_vals + (uint64_t)f * cap;
    // one more digit bit than the plan's in the same counter words: 16-bit
    // counters, two to a word (n < 2^16), runs of about half the records
    const int shift = 64 - d.p - dbits - 1;
    const uint32_t pdig = ndig << 1, dmask = pdig - 1u;
    const uint16_t *DC16 = reinterpret_cast<const uint16_t *>(DC);
    // the filled part of the slot kS2PrefetchAhead partitions ahead goes to
    // L2 after step 1 (its fill count is read now)
    const uint64_t fa = (uint64_t)f + kS2PrefetchAhead;
    const uint32_t nfa = (threadIdx.x == 0 && fa < (1ull << d.p)) ? min(d.cnt2[fa], cap) : 0u;
    for (uint32_t i = threadIdx.x; i < ndig; i += NT) DC[i] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t g = (uint32_t)(__ldg(ik + i) >> shift) & dmask, h = (g & 1u) << 4;
        RK[i] = (uint16_t)(atomicAdd(&DC[g >> 1], 1u << h) >> h);
    }
    if (nfa) {
        const uint32_t nb = ((nfa + 1u) & ~1u) * 8u;  // 16-byte multiple (cap is even)
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_keys + fa * cap), "r"(nb)
                     : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_vals + fa * cap), "r"(nb)
                     : "memory");
    }
    __syncthreads();
    block_scan_packed16<NT>(DC, ndig, WS);
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint64_t k = __ldg(ik + i);
        const uint32_t pos = DC16[(uint32_t)(k >> shift) & dmask] + RK[i];
        SK[pos] = k;
        SI[pos] = (uint16_t)i;
    }
    __syncthreads();
    // DC16[g] is the start of run g (records of digit g in arrival order);
    // the run ends at DC16[g + 1] (n for the last digit).  Every position, 32
    // per warp step and one per lane, finds its record's rank inside its run
    // and the record goes straight to its place in the sorted table.  A
    // run's records sit in neighbouring lanes, so each lane compares with
    // the lanes up to the longest run's length away (shuffles, every lane
    // in step) on a 32-bit compare key: the key bits below the digit, or
    // their top 32 (records of a run agree above them).  A lane whose run
    // leaves its chunk, or that meets an equal compare key, ranks itself
    // from shared memory on full keys, then on the packed pairs (a << 32 |
    // b) for equal keys.  Two chunks per step so that their work overlaps.
    uint4 *__restrict__ out = d.t2 + o;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr uint32_t NW = NT / 32;
    const uint32_t nch = (n + 31u) >> 5;
    const int cs = shift > 32 ? shift - 32 : 0;
    auto run_bounds = [&](uint64_t k, uint32_t &s0, uint32_t &s1) {
        const uint32_t g = (uint32_t)(k >> shift) & dmask;
        s0 = DC16[g];
        s1 = g + 1 < pdig ? DC16[g + 1] : n;
    };
    // place of the record (k, slot index ix) among the run [s0, s1)
    auto rank_slow = [&](uint64_t k, uint16_t ix, uint32_t s0, uint32_t s1) -> uint32_t {
        uint32_t r = s0;
        uint64_t v = 0;
        bool have_v = false;
        for (uint32_t q = s0; q < s1; ++q) {
            const uint64_t kq = SK[q];
            if (kq < k) {
                ++r;
            } else if (kq == k && SI[q] != ix) {
                if (!have_v) {
                    v = __ldg(iv + ix);
                    have_v = true;
                }
                r += __ldg(iv + SI[q]) < v ? 1u : 0u;
            }
        }
        return r;
    };
    for (uint32_t c = warp; c < nch; c += 2 * NW) {
        const uint32_t pa = 32u * c + lane, pb = pa + 32u * NW;
        const bool va = pa < n, vb = pb < n;
        const uint32_t xa = va ? pa : 0u, xb = vb ? pb : 0u;
        const uint64_t ka = SK[xa], kb = SK[xb];
        const uint16_t ia = SI[xa], ib = SI[xb];
        uint32_t sa, ea, sb, eb;
        run_bounds(ka, sa, ea);
        run_bounds(kb, sb, eb);
        if (!va) sa = ea = 0u;
        if (!vb) sb = eb = 0u;
        const uint32_t lmax = __reduce_max_sync(0xffffffffu, max(ea - sa, eb - sb));
        uint32_t da = sa, db = sb;
        if (lmax > 1) {
            const uint32_t qa = (uint32_t)(ka >> cs), qb = (uint32_t)(kb >> cs);
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
            if (va && slow_a) da = rank_slow(ka, ia, sa, ea);
            if (vb && slow_b) db = rank_slow(kb, ib, sb, eb);
        }
        if (va) {
            const uint64_t v = __ldg(iv + ia);
            out[da] = make_uint4((uint32_t)(v >> 32), (uint32_t)v, bswap32((uint32_t)(ka >> 32)),
                                 bswap32((uint32_t)ka));
        }
        if (vb) {
            const uint64_t v = __ldg(iv + ib);
            out[db] = make_uint4((uint32_t)(v >> 32), (uint32_t)v, bswap32((uint32_t)(kb >> 32)),
                                 bswap32((uint32_t)kb));
        }
    }
}

size_t sort2_smem_bytes(uint32_t cap, int dbits) { return S2SortLayout(cap, dbits).bytes; }

cudaError_t launch_sort2(const Sort2Desc *d_desc, const Sort2Launch &g, cudaStream_t s)
{
    cudaError_t e;
    k_s2_setup<<<64, 256, 0, s>>>(const_cast<Sort2Desc *>(d_desc));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (g.tiles1) {
        const size_t sm1 = sizeof(S2Smem1);
        if ((e = cudaFuncSetAttribute(k_s2_scatter1, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm1)) != cudaSuccess)
            return e;
        k_s2_scatter1<<<g.tiles1, kS2Threads, sm1, s>>>(d_desc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (g.tiles2) {
        const size_t sm2 = sizeof(S2Smem2);
        if ((e = cudaFuncSetAttribute(k_s2_scatter2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)sm2)) != cudaSuccess)
            return e;
        k_s2_scatter2<<<g.tiles2, kS2BThreads, sm2, s>>>(d_desc);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    k_s2_scan<<<g.tiles_scan, 256, 0, s>>>(d_desc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const size_t sm3 = sort2_smem_bytes(g.cap2, g.dbits);
    if ((e = cudaFuncSetAttribute(k_s2_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3)) !=
        cudaSuccess)
        return e;
    k_s2_sort<<<g.parts, kS2SortThreads, sm3, s>>>(d_desc);
    return cudaGetLastError();
}

}  // namespace vx
