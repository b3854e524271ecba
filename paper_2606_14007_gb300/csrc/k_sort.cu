// k_sort.cu -- second bucketing scatter level, prefix scans, the
// in-partition shared-memory sort that finishes Table 1, and the logical
// bucket offsets.
//
// Paper: Sec. III-A/III-B.  The paper sorts each of its 2^24 buckets with a
// single-thread insertion sort inside its fused Sort+Match kernel (Sec. I-A
// and V name this O(n^2) sort as the K=31 bottleneck and propose a parallel
// radix sort).  Here a physical partition (a run of whole logical buckets,
// a few thousand records) is sorted by one CTA in shared memory: one
// counting-sort pass on the next `dbits` key bits below the partition
// prefix spreads the records over ~1 per digit, then each thread finishes
// its digits with an insertion sort on (key64, nonce).  Deterministic: the
// result is the unique (key64, nonce) order whatever order the scatter
// atomics left the slot in.
#include "vx_internal.cuh"

namespace vx {

// ------------------------------------------------ second scatter level
struct Scatter2Smem {
    uint64_t keys[kScatterTile];
    uint32_t nonces[kScatterTile];
    uint32_t hist[1 << kMaxFineBits];
    uint32_t loff[1 << kMaxFineBits];
    uint32_t gbase[1 << kMaxFineBits];
    uint32_t ws[kScatterThreads / 32 + 1];
};

__global__ void __launch_bounds__(kScatterThreads) k_scatter2(const Desc *__restrict__ descs,
                                                             int nplots,
                                                             const uint32_t *__restrict__ tile_start)
{
    constexpr int NT = kScatterThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Scatter2Smem &sm = *reinterpret_cast<Scatter2Smem *>(smem_raw);

    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    const uint32_t local = blockIdx.x - tile_start[plot];
    const uint32_t c = local / d.chunks1;              // level-1 slot
    const uint32_t chunk = local - c * d.chunks1;
    const uint32_t filled = min(d.cnt1[c], d.cap1);
    const uint32_t start = chunk * (uint32_t)kScatterTile;
    if (start >= filled) return;
    const uint32_t count = min((uint32_t)kScatterTile, filled - start);
    const int p2 = d.p2;
    const int nbins = 1 << p2;
    const int shift = 64 - d.p;                        // fine index = key >> shift
    const uint32_t bin_mask = (uint32_t)nbins - 1u;
    const uint64_t *__restrict__ ikeys = d.a_keys + (uint64_t)c * d.cap1 + start;
    const uint32_t *__restrict__ inonces = d.a_nonces + (uint64_t)c * d.cap1 + start;

    for (int b = threadIdx.x; b < nbins; b += NT) sm.hist[b] = 0u;
    __syncthreads();

    // Records held in registers between the histogram and the staging pass.
    constexpr int PER = kScatterTile / NT;
    uint64_t key[PER];
    uint32_t nonce[PER], rank[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const uint32_t i = (uint32_t)j * NT + threadIdx.x;
        const bool valid = i < count;
        key[j] = valid ? ikeys[i] : 0ull;
        nonce[j] = valid ? inonces[i] : 0u;
        const uint32_t bin = (uint32_t)(key[j] >> shift) & bin_mask;
        rank[j] = valid ? atomicAdd(&sm.hist[bin], 1u) : 0u;
    }
    __syncthreads();
    {
        const int per = (nbins + NT - 1) / NT;
        const int b0 = threadIdx.x * per;
        uint32_t loc = 0;
        for (int k = 0; k < per; ++k)
            if (b0 + k < nbins) loc += sm.hist[b0 + k];
        uint32_t total;
        uint32_t run = block_exclusive_scan_u32<NT>(loc, sm.ws, &total);
        for (int k = 0; k < per; ++k) {
            const int b = b0 + k;
            if (b < nbins) {
                const uint32_t h = sm.hist[b];
                sm.loff[b] = run;
                run += h;
                sm.gbase[b] = h ? atomicAdd(&d.cnt2[((uint64_t)c << p2) + b], h) : 0u;
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
    __syncthreads();
    const uint32_t cap = d.cap2;
    bool overflow = false;
    for (uint32_t i = threadIdx.x; i < count; i += NT) {
        const uint64_t k = sm.keys[i];
        const uint32_t bin = (uint32_t)(k >> shift) & bin_mask;
        const uint32_t g = sm.gbase[bin] + (i - sm.loff[bin]);
        if (g < cap) {
            const uint64_t at = (((uint64_t)c << p2) + bin) * cap + g;
            d.b_keys[at] = k;
            d.b_nonces[at] = sm.nonces[i];
        } else {
            overflow = true;
        }
    }
    if (overflow) atomicOr(d.status, kStSlot2Overflow);
}

cudaError_t launch_scatter2(const Desc *descs, int nplots, const uint32_t *tile_start,
                            uint32_t total_tiles, cudaStream_t s)
{
    if (total_tiles == 0) return cudaSuccess;
    const size_t smem = sizeof(Scatter2Smem);
    cudaError_t e = cudaFuncSetAttribute(k_scatter2, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_scatter2<<<total_tiles, kScatterThreads, smem, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

// ------------------------------------------------------------- scans
// One CTA per plot: exclusive prefix of 2^p per-partition counts.  COUNTS:
// level-2 fill counters (clipped to the slot capacity) -> Table-1 offsets,
// with a check that every nonce arrived.  Otherwise: pair counts -> Table-2
// offsets.
constexpr int kScanThreads = 1024;

template <bool COUNTS>
__global__ void __launch_bounds__(kScanThreads) k_scan(const Desc *__restrict__ descs)
{
    __shared__ uint64_t ws[kScanThreads / 32 + 1];
    __shared__ uint64_t carry_s;
    const Desc &d = descs[blockIdx.x];
    const uint64_t n = 1ull << d.p;
    uint64_t *out = COUNTS ? d.t1off : d.t2off;
    const uint64_t per = (n + kScanThreads - 1) / kScanThreads;
    const uint64_t b0 = (uint64_t)threadIdx.x * per;
    const uint64_t b1 = min(n, b0 + per);
    auto val = [&](uint64_t i) -> uint64_t {
        return COUNTS ? (uint64_t)min(d.cnt2[i], d.cap2) : d.pairs[i];
    };
    uint64_t local = 0;
    for (uint64_t i = b0; i < b1; ++i) local += val(i);
    // block exclusive scan of `local` (u64)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t incl = local;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t run = 0;
        for (int w = 0; w < kScanThreads / 32; ++w) {
            uint64_t t = ws[w];
            ws[w] = run;
            run += t;
        }
        carry_s = run;
    }
    __syncthreads();
    uint64_t run = ws[warp] + incl - local;
    for (uint64_t i = b0; i < b1; ++i) {
        out[i] = run;
        run += val(i);
    }
    if (threadIdx.x == 0) {
        out[n] = carry_s;
        if (COUNTS && carry_s != d.N) atomicOr(d.status, kStCountMismatch);
        // A re-run of the match (e.g. after a larger Table-2 buffer was
        // bound) re-decides the capacity bit.
        if (!COUNTS) {
            if (carry_s > d.t2cap) atomicOr(d.status, kStT2Capacity);
            else atomicAnd(d.status, ~kStT2Capacity);
        }
    }
}

cudaError_t launch_scan_counts(const Desc *descs, int nplots, cudaStream_t s)
{
    k_scan<true><<<nplots, kScanThreads, 0, s>>>(descs);
    return cudaGetLastError();
}

cudaError_t launch_scan_pairs(const Desc *descs, int nplots, cudaStream_t s)
{
    k_scan<false><<<nplots, kScanThreads, 0, s>>>(descs);
    return cudaGetLastError();
}

// ------------------------------------------------------ partition sort
// Pairs of record i (r-th in sorted order) with later records of the same
// logical bucket closer than D: the Table-2 count this partition owes.
__device__ __forceinline__ uint32_t pair_run(const uint64_t *keys, const uint16_t *perm,
                                             uint32_t r, uint32_t n, uint64_t D)
{
    const uint64_t k = keys[perm[r]];
    const uint64_t bucket = k >> 40;
    uint32_t c = 0;
    for (uint32_t r2 = r + 1; r2 < n; ++r2) {
        const uint64_t k2 = keys[perm[r2]];
        if ((k2 >> 40) != bucket || k2 - k >= D) break;
        ++c;
    }
    return c;
}

// Shared layout (dynamic), cap a multiple of 4: keys[cap] u64 | nonces[cap]
// u32 | perm[cap] u16 | rank[cap] u16 | digit counters [2^dbits] u32 |
// ws u32 [NT/32 + 2] | ws64 u64 [NT/32 + 1].  perm[r] = input index of the
// r-th record in sorted order.
struct SortLayout {
    size_t nonces, perm, rank, dcnt, ws, ws64, bytes;
    __host__ __device__ SortLayout(uint32_t cap, int dbits)
    {
        nonces = (size_t)cap * 8;
        perm = nonces + (size_t)cap * 4;
        rank = perm + (size_t)cap * 2;
        dcnt = rank + (size_t)cap * 2;
        ws = dcnt + ((size_t)1 << dbits) * 4;
        ws64 = (ws + (kSortThreads / 32 + 2) * 4 + 7) & ~(size_t)7;
        bytes = ws64 + (kSortThreads / 32 + 1) * 8;
    }
};
__global__ void __launch_bounds__(kSortThreads) k_sort(const Desc *__restrict__ descs, int nplots,
                                                       const uint32_t *__restrict__ tile_start)
{
    constexpr int NT = kSortThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    const uint32_t f = blockIdx.x - tile_start[plot];
    const uint32_t cap = d.cap2;
    const int dbits = d.dbits;
    const uint32_t ndig = 1u << dbits;
    const SortLayout L(cap, dbits);
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *nonces = reinterpret_cast<uint32_t *>(smem_raw + L.nonces);
    uint16_t *perm = reinterpret_cast<uint16_t *>(smem_raw + L.perm);
    uint16_t *rank = reinterpret_cast<uint16_t *>(smem_raw + L.rank);
    uint32_t *dcnt = reinterpret_cast<uint32_t *>(smem_raw + L.dcnt);
    uint32_t *ws = reinterpret_cast<uint32_t *>(smem_raw + L.ws);
    uint64_t *ws64 = reinterpret_cast<uint64_t *>(smem_raw + L.ws64);

    const uint32_t n = min(d.cnt2[f], cap);
    const uint64_t off = d.t1off[f];
    const uint64_t *__restrict__ ikeys = d.b_keys + (uint64_t)f * cap;
    const uint32_t *__restrict__ inonces = d.b_nonces + (uint64_t)f * cap;
    const int shift = 64 - d.p - dbits;
    const uint32_t dmask = ndig - 1u;

    for (uint32_t i = threadIdx.x; i < ndig; i += NT) dcnt[i] = 0u;
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        keys[i] = ikeys[i];
        nonces[i] = inonces[i];
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t dg = (uint32_t)(keys[i] >> shift) & dmask;
        rank[i] = (uint16_t)atomicAdd(&dcnt[dg], 1u);
    }
    __syncthreads();
    {   // exclusive scan of the digit counters; each thread owns a run
        const uint32_t per = (ndig + NT - 1) / NT;
        const uint32_t b0 = threadIdx.x * per;
        uint32_t loc = 0;
        for (uint32_t k = 0; k < per; ++k)
            if (b0 + k < ndig) loc += dcnt[b0 + k];
        uint32_t total;
        uint32_t run = block_exclusive_scan_u32<NT>(loc, ws, &total);
        for (uint32_t k = 0; k < per; ++k)
            if (b0 + k < ndig) {
                const uint32_t h = dcnt[b0 + k];
                dcnt[b0 + k] = run;
                run += h;
            }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t dg = (uint32_t)(keys[i] >> shift) & dmask;
        perm[dcnt[dg] + rank[i]] = (uint16_t)i;
    }
    __syncthreads();
    // Finish each digit run with an insertion sort on (key64, nonce).
    for (uint32_t dg = threadIdx.x; dg < ndig; dg += NT) {
        const uint32_t s0 = dcnt[dg];
        const uint32_t s1 = dg + 1 < ndig ? dcnt[dg + 1] : n;
        for (uint32_t a = s0 + 1; a < s1; ++a) {
            const uint16_t x = perm[a];
            const uint64_t kx = keys[x];
            const uint32_t nx = nonces[x];
            uint32_t b = a;
            while (b > s0) {
                const uint16_t y = perm[b - 1];
                const uint64_t ky = keys[y];
                if (ky < kx || (ky == kx && nonces[y] < nx)) break;
                perm[b] = y;
                --b;
            }
            perm[b] = x;
        }
    }
    __syncthreads();
    // Table-1 words {nonce, h0, h1}: consecutive threads store consecutive
    // 4-byte words of the partition's byte range.
    uint32_t *__restrict__ t1w = reinterpret_cast<uint32_t *>(d.t1) + 3 * off;
    for (uint32_t w = threadIdx.x; w < 3 * n; w += NT) {
        const uint32_t r = w / 3, q = w - 3 * r;
        const uint16_t x = perm[r];
        const uint64_t k = keys[x];
        t1w[w] = q == 0 ? nonces[x] : bswap32(q == 1 ? (uint32_t)(k >> 32) : (uint32_t)k);
    }
    // Pairs this partition contributes to Table 2.
    uint64_t mine = 0;
    const uint64_t D = d.D;
    for (uint32_t r = threadIdx.x; r < n; r += NT) mine += pair_run(keys, perm, r, n, D);
    const uint64_t tot = block_sum_u64<NT>(mine, ws64);
    if (threadIdx.x == 0) d.pairs[f] = tot;
}

size_t sort_smem_bytes(uint32_t cap, int dbits) { return SortLayout(cap, dbits).bytes; }

cudaError_t launch_sort(const Desc *descs, int nplots, const uint32_t *tile_start,
                        uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits)
{
    const size_t smem = sort_smem_bytes(max_cap, max_dbits);
    cudaError_t e = cudaFuncSetAttribute(k_sort, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_sort<<<total_tiles, kSortThreads, smem, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

// ----------------------------------------------- logical bucket offsets
// offsets[b] = first Table-1 record of logical bucket b, found by a binary
// search inside the physical partition that holds bucket b.
__global__ void k_bucket_offsets(const Desc *__restrict__ dp, uint64_t *__restrict__ out)
{
    const Desc &d = *dp;
    const uint32_t nb = 1u << kBucketBits;
    const uint32_t b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nb) return;
    if (b == nb) {
        out[nb] = d.N;
        return;
    }
    const uint32_t f = d.p ? (b >> (kBucketBits - d.p)) : 0u;
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
