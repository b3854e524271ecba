// k_sort.cu -- second bucketing scatter level, prefix scans, and the
// logical bucket offsets of Table 1.
//
// Paper: Sec. III-A/III-B (Table 1 bucketed by hash prefix, 2^24 buckets).
// The partition sort itself lives in k_sortmatch.cu.
#include "vx_internal.cuh"

namespace vx {

// ------------------------------------------------ second scatter level
// One CTA takes a tile of up to kScatterTile records of one first-level
// slot.  The tile's keys and nonces are contiguous, so two TMA bulk copies
// bring them into shared memory (one mbarrier, bounded wait); ranks within
// the second-level bins come from shared-memory atomics; one global atomic
// per (CTA, bin) claims a run of the final partition slot; records are
// restaged in bin order in place (through registers) and written out so
// that consecutive threads store consecutive addresses of each run.
// FB: the most second-level bits the instance handles (10; 11 for the
// 2^21 partitions of K = 32).
template <int FB>
struct Scatter2Smem {
    uint64_t keys[kScatterTile];
    uint32_t nonces[kScatterTile];
    uint32_t hist[1 << FB];
    uint32_t loff[1 << FB];
    uint32_t gbase[1 << FB];
    uint32_t ws[kScatterThreads / 32 + 1];
    uint64_t bar;
};

template <bool HALO, int FB>
__global__ void __launch_bounds__(kScatterThreads) k_scatter2(const Desc *__restrict__ descs,
                                                             int nplots,
                                                             const uint32_t *__restrict__ tile_start,
                                                             int chunk)
{
    constexpr int NT = kScatterThreads;
    constexpr int PER = kScatterTile / NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    Scatter2Smem<FB> &sm = *reinterpret_cast<Scatter2Smem<FB> *>(smem_raw);

    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    const uint32_t local = blockIdx.x - tile_start[plot];
    const uint32_t c = local / d.chunks1;              // level-1 bin of this nonce chunk
    const uint32_t part = local - c * d.chunks1;       // tile of the slot
    const uint64_t cs = ((uint64_t)chunk << d.p1) + c; // the slot
    const uint32_t filled = min(d.cnt1[cs], d.cap1);
    const uint32_t start = part * (uint32_t)kScatterTile;
    if (start >= filled) return;
    const uint32_t count = min((uint32_t)kScatterTile, filled - start);
    const int p2 = d.p2;
    const int nbins = 1 << p2;
    const int shift = 64 - d.pk;                       // fine index = key >> shift
    const uint32_t bin_mask = (uint32_t)nbins - 1u;
    // Copy a multiple of 4 records: the slot (cap1 % 4 == 0) always holds them.
    const uint32_t ncopy = (count + 3u) & ~3u;
    if (threadIdx.x == 0) {
        mbar_init(&sm.bar, 1);
        mbar_expect_tx(&sm.bar, ncopy * 12u);
        bulk_g2s(sm.keys, d.a_keys + cs * d.cap1 + start, ncopy * 8u, &sm.bar);
        bulk_g2s(sm.nonces, d.a_nonces + cs * d.cap1 + start, ncopy * 4u, &sm.bar);
    }
    for (int b = threadIdx.x; b < nbins; b += NT) sm.hist[b] = 0u;
    __syncthreads();
    if (!__syncthreads_and(mbar_wait(&sm.bar, 0, d.spin_limit))) {  // one answer for all threads
        // The copy did not land in time: report, give it one more bounded
        // wait so it does not write into a successor's shared memory, stop.
        if (threadIdx.x == 0) atomicOr(d.status, kStTimeout);
        mbar_wait(&sm.bar, 0, d.spin_limit);
        return;
    }

    uint64_t key[PER];
    uint32_t nonce[PER], rank[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        const bool valid = i < count;
        key[j] = valid ? sm.keys[i] : 0ull;
        nonce[j] = valid ? sm.nonces[i] : 0u;
        const uint32_t bin = (uint32_t)(key[j] >> shift) & bin_mask;
        rank[j] = valid ? atomicAdd(&sm.hist[bin], 1u) : 0u;
    }
    __syncthreads();
    constexpr int PB = ((1 << FB) + NT - 1) / NT;  // most bins a thread owns
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
                // the claim's result is first needed after the restage below
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
            sm.nonces[pos] = nonce[j];
        }
    }
#pragma unroll
    for (int k = 0; k < PB; ++k)
        if (k < per && b0 + k < nbins) sm.gbase[b0 + k] = claim[k];
    __syncthreads();
    const uint32_t cap = d.cap2;
    bool overflow = false, hover = false;
    // unrolled over the thread's PER records so that their dependent
    // shared-memory reads (key, then its bin's bases) overlap
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        if (i >= count) break;
        const uint64_t k = sm.keys[i];
        const uint32_t bin = (uint32_t)(k >> shift) & bin_mask;
        const uint32_t g = sm.gbase[bin] + (i - sm.loff[bin]);
        const uint64_t part = ((uint64_t)c << p2) + bin;
        if (g < cap) {
            const uint64_t at = part * cap + g;
            d.b_keys[at] = k;
            d.b_nonces[at] = sm.nonces[i];
        } else {
            overflow = true;
        }
        if (HALO) halo_add(d, part, k, sm.nonces[i], hover);
    }
    if (overflow) atomicOr(d.status, kStSlot2Overflow);
    if (hover) atomicOr(d.status, kStHaloOverflow);
}

cudaError_t launch_scatter2(const Desc *descs, int nplots, const uint32_t *tile_start,
                            uint32_t total_tiles, int chunk, cudaStream_t s, bool halo,
                            int fine_bits)
{
    if (total_tiles == 0) return cudaSuccess;
    const bool wide = fine_bits > kMaxFineBits;
    const size_t smem = wide ? sizeof(Scatter2Smem<kMaxFineBitsWide>) : sizeof(Scatter2Smem<kMaxFineBits>);
    auto fn = wide ? (halo ? k_scatter2<true, kMaxFineBitsWide> : k_scatter2<false, kMaxFineBitsWide>)
                   : (halo ? k_scatter2<true, kMaxFineBits> : k_scatter2<false, kMaxFineBits>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<total_tiles, kScatterThreads, smem, s>>>(descs, nplots, tile_start, chunk);
    return cudaGetLastError();
}

// ------------------------------- Table-1 / Table-2 offsets (counts scan)
// Exclusive prefix of 2^p per-partition counts in chunks of kScanChunk
// counters, one CTA per chunk (taken in ticket order), the chunks chained by
// decoupled look-back.
constexpr int kScanCtaThreads = 256;

// SRC 0: level-2 fill counters (clipped to the slot) -> Table-1 offsets,
// chunk ticket ticket_s, look-back words lbs; the last chunk checks that
// every nonce arrived.
// SRC 1: per-partition pair counts of the slot placement -> Table-2
// offsets, chunk ticket `ticket` and look-back words `lb` (both unused by
// the slot sort, zeroed by the key setup); counts are clipped to one more
// than a pair slot holds (a larger count has already failed the plot), and
// the last chunk checks the Table-2 capacity.
template <int SRC>
__global__ void __launch_bounds__(kScanCtaThreads) k_scan_counts(const Desc *__restrict__ descs,
                                                                 int nplots,
                                                                 const uint32_t *__restrict__ tile_start)
{
    constexpr int NT = kScanCtaThreads;
    constexpr uint32_t PER = kScanChunk / NT;
    __shared__ uint32_t ws[NT / 32 + 1];
    __shared__ uint32_t s_c;
    __shared__ uint64_t s_base;
    __shared__ int s_ok;
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    uint32_t *ticket = SRC == 0 ? d.ticket_s : d.ticket;
    uint64_t *lb = SRC == 0 ? d.lbs : d.lb;
    uint64_t *out = SRC == 0 ? d.t1off : d.t2off;
    if (threadIdx.x == 0) s_c = atomicAdd(ticket, 1u);
    __syncthreads();
    const uint32_t c = s_c;
    const uint64_t n = 1ull << d.p;
    const uint32_t nchunks = (uint32_t)((n + kScanChunk - 1) / kScanChunk);
    if (c >= nchunks) {  // only if the ticket was not reset: report, never index with it
        if (threadIdx.x == 0) atomicOr(d.status, kStBadTicket);
        return;
    }
    const uint32_t clip = SRC == 0 ? d.cap2 : d.cap2 + d.cap2 / 2u + 1u;
    const uint64_t b0 = (uint64_t)c * kScanChunk + (uint64_t)threadIdx.x * PER;
    uint32_t v[PER];
    uint32_t loc = 0;
#pragma unroll
    for (uint32_t k = 0; k < PER; ++k) {
        uint32_t x = 0;
        if (b0 + k < n) {
            if (SRC == 0) {
                x = min(d.cnt2[b0 + k], clip);
            } else {
                const uint64_t y = d.pairs[b0 + k];
                x = y < clip ? (uint32_t)y : clip;
            }
        }
        v[k] = x;
        loc += x;
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan_u32<NT>(loc, ws, &total);
    if (threadIdx.x < 32) {
        uint64_t excl = 0;
        // VX_TEST_WITHHOLD_PREFIX: chunk 0 of the pair-count scan never
        // publishes, so every later chunk's bounded wait runs out.
        const bool withhold = SRC == 1 && (d.test_flags & 1u) != 0;
        const int ok = lookback_warp(lb, c, total, d.status, d.spin_limit, withhold, &excl) ? 1 : 0;
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
        if (b0 + k < n) out[b0 + k] = at;
        at += v[k];
    }
    if (c + 1 == nchunks && threadIdx.x == 0) {
        const uint64_t all = s_base + total;
        out[n] = all;
        if (SRC == 0) {
            // Every nonce exactly once; a window's share is random (the
            // windows of one plot add up to 2^K, checked by their caller).
            if (d.wbits == 0 && all != d.N) atomicOr(d.status, kStCountMismatch);
        } else {
            if (all > d.t2cap) atomicOr(d.status, kStT2Capacity);
        }
    }
}

cudaError_t launch_scan_counts(const Desc *descs, int nplots, const uint32_t *tile_start,
                               uint32_t total_tiles, cudaStream_t s)
{
    k_scan_counts<0><<<total_tiles, kScanCtaThreads, 0, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

cudaError_t launch_scan_pair_counts(const Desc *descs, int nplots, const uint32_t *tile_start,
                                    uint32_t total_tiles, cudaStream_t s)
{
    k_scan_counts<1><<<total_tiles, kScanCtaThreads, 0, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

// ------------------------------------------------------ pair-offset scan
// One CTA per plot: exclusive prefix of the 2^p per-partition pair counts
// -> Table-2 offsets (split vx_table1 / vx_match path), with the Table-2
// capacity check.
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads) k_scan_pairs(const Desc *__restrict__ descs)
{
    constexpr int NT = kScanThreads, NW = NT / 32, PER = 4;
    __shared__ uint64_t ws[NW];
    __shared__ uint64_t s_tile;
    const Desc &d = descs[blockIdx.x];
    const uint64_t n = 1ull << d.p;
    uint64_t *out = d.t2off;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // tiles of NT * PER consecutive counts, PER per thread (coalesced),
    // block-scanned one after the other with the running total carried
    uint64_t carry = 0;
    for (uint64_t t0 = 0; t0 < n; t0 += (uint64_t)NT * PER) {
        const uint64_t b0 = t0 + (uint64_t)threadIdx.x * PER;
        uint64_t v[PER], local = 0;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            v[k] = b0 + k < n ? d.pairs[b0 + k] : 0ull;
            local += v[k];
        }
        uint64_t incl = local;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) ws[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint64_t x = lane < NW ? ws[lane] : 0ull;
            uint64_t wi = x;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += y;
            }
            if (lane < NW) ws[lane] = wi - x;  // exclusive warp prefixes
            if (lane == NW - 1) s_tile = wi;
        }
        __syncthreads();
        uint64_t at = carry + ws[warp] + incl - local;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (b0 + k < n) out[b0 + k] = at;
            at += v[k];
        }
        carry += s_tile;
        __syncthreads();  // ws and s_tile are reused by the next tile
    }
    if (threadIdx.x == 0) {
        out[n] = carry;
        // A re-run of the match (e.g. after a larger Table-2 buffer was
        // bound) re-decides the capacity bit.
        if (carry > d.t2cap) atomicOr(d.status, kStT2Capacity);
        else atomicAnd(d.status, ~kStT2Capacity);
    }
}

cudaError_t launch_scan_pairs(const Desc *descs, int nplots, cudaStream_t s)
{
    k_scan_pairs<<<nplots, kScanThreads, 0, s>>>(descs);
    return cudaGetLastError();
}

// ----------------------------------------------- logical bucket offsets
// offsets[b] = first Table-1 record of logical bucket b, found by a binary
// search inside the physical partition that holds bucket b.  A window's
// Table 1 holds buckets [w0, w0 + 2^(24 - wbits)) only: buckets below get
// offset 0, buckets above the window's record count.
__global__ void k_bucket_offsets(const Desc *__restrict__ dp, uint64_t *__restrict__ out)
{
    const Desc &d = *dp;
    const uint32_t nb = 1u << kBucketBits;
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    const uint64_t np = 1ull << d.p;
    if (b == nb) {
        out[nb] = d.wbits ? d.t1off[np] : d.N;
        return;
    }
    const int wb = kBucketBits - (int)d.wbits;  // bucket bits inside the window
    const uint32_t w0 = d.win << wb;
    if (b < w0) {
        out[b] = 0;
        return;
    }
    if (b - w0 >= (1u << wb)) {
        out[b] = d.t1off[np];
        return;
    }
    const uint32_t f = d.p ? ((b - w0) >> (wb - d.p)) : 0u;
    uint64_t lo = d.t1off[f], hi = d.t1off[f + 1];
    const uint32_t *t1w = reinterpret_cast<const uint32_t *>(d.t1);
    while (lo < hi) {   // first record whose bucket >= b
        const uint64_t mid = (lo + hi) >> 1;
        const uint32_t hb = bswap32(t1w[3 * mid + 1]) >> 8;   // key64 >> 40
        if (hb < b) lo = mid + 1; else hi = mid;
    }
    out[b] = lo;
}

cudaError_t launch_bucket_offsets(const Desc *desc, uint64_t *out, cudaStream_t s)
{
    const uint32_t n = (1u << kBucketBits) + 1;
    k_bucket_offsets<<<(n + 255) / 256, 256, 0, s>>>(desc, out);
    return cudaGetLastError();
}

}  // namespace vx
