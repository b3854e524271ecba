// k_sortmatch.cu -- partition sort fused with the match stage.
//
// Paper: Sec. I-B / III-A / III-B fuse sort and Table-2 generation into one
// kernel that keeps each bucket in shared memory, one block per bucket,
// with a single-thread insertion sort; Sec. V names that O(n^2) sort as the
// K=31 bottleneck and proposes a parallel radix sort.  Kept here: the
// fusion (a partition never leaves shared memory between sort and match).
// Changed: one CTA per physical partition (a run of whole logical buckets,
// ~2048 records), a counting-sort pass on the key bits below the partition
// prefix followed by per-digit insertion sorts (about one record per digit),
// pairs listed in shared memory so all lanes hash back to back, and the
// partition's Table-2 base found by a decoupled look-back over the
// partitions before it (partition order comes from a ticket counter, so
// every partition a CTA waits on is already running; every wait is bounded
// and a timeout poisons the chain instead of hanging).
//
// MODE kSortCount: the sort alone (Table 1 + per-partition pair counts),
// used by the split vx_table1 / vx_match path.
// MODE kSortHash: everything in one kernel, pairs hashed here.
// MODE kSortEmit: Table 1, then each pair written as a Table-2 record
// {a, b, 0, 0} at its final offset; the streaming pair-hash kernel fills in
// the hashes (no barriers, full occupancy: the ALU-bound part runs apart
// from the latency-bound sort).
#include "vx_internal.cuh"

namespace vx {

constexpr int kSMThreads = 256;
enum { kSortCount = 0, kSortHash = 1, kSortEmit = 2 };
constexpr uint32_t kSMList = 2048;            // pair-list window (entries)

struct SMLayout {
    size_t sn, rank, dcnt, start, list, ws, bytes;
    __host__ __device__ SMLayout(uint32_t cap, int dbits, bool with_list)
    {
        sn = (size_t)cap * 8;                    // sorted key64 [cap] at 0
        rank = sn + (size_t)cap * 4;             // sorted nonce [cap]
        dcnt = rank + (size_t)((cap + 1) & ~1u) * 2;  // rank within digit, u16 [cap]
        start = dcnt + ((size_t)1 << dbits) * 4; // digit counters -> starts [2^dbits]
        list = start + (size_t)cap * 4;          // per-record pair count -> start [cap]
        ws = list + (with_list ? (size_t)kSMList * 4 : 0);  // pair list window
        bytes = ws + (kSMThreads / 32 + 2) * 4 + 16;
    }
};

template <int MODE>
__global__ void __launch_bounds__(kSMThreads, MODE == kSortHash ? 3 : 4)
    k_sortmatch(const Desc *__restrict__ descs, int nplots, const uint32_t *__restrict__ tile_start)
{
    constexpr bool EMIT = MODE != kSortCount;
    constexpr int NT = kSMThreads;
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
    const int dbits = d.dbits;
    const uint32_t ndig = 1u << dbits;
    const SMLayout L(cap, dbits, MODE == kSortHash);
    uint64_t *SK = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *SN = reinterpret_cast<uint32_t *>(smem_raw + L.sn);
    uint16_t *RK = reinterpret_cast<uint16_t *>(smem_raw + L.rank);
    uint32_t *DC = reinterpret_cast<uint32_t *>(smem_raw + L.dcnt);
    uint32_t *ST = reinterpret_cast<uint32_t *>(smem_raw + L.start);
    uint32_t *LS = reinterpret_cast<uint32_t *>(smem_raw + L.list);
    uint32_t *WS = reinterpret_cast<uint32_t *>(smem_raw + L.ws);

    const uint32_t n = min(d.cnt2[f], cap);
    const uint64_t off = d.t1off[f];
    const uint64_t *__restrict__ ikeys = d.b_keys + (uint64_t)f * cap;
    const uint32_t *__restrict__ inonces = d.b_nonces + (uint64_t)f * cap;
    const int shift = 64 - d.p - dbits;
    const uint32_t dmask = ndig - 1u;

    // 1. digit histogram (rank of each record within its digit)
    for (uint32_t i = threadIdx.x; i < ndig; i += NT) DC[i] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t dg = (uint32_t)(__ldg(ikeys + i) >> shift) & dmask;
        RK[i] = (uint16_t)atomicAdd(&DC[dg], 1u);
    }
    __syncthreads();
    {   // 2. exclusive scan of the digit counters (contiguous run per thread)
        const uint32_t per = (ndig + NT - 1) / NT;
        const uint32_t b0 = threadIdx.x * per;
        uint32_t loc = 0;
        for (uint32_t k = 0; k < per; ++k)
            if (b0 + k < ndig) loc += DC[b0 + k];
        uint32_t total;
        uint32_t run = block_exclusive_scan_u32<NT>(loc, WS, &total);
        for (uint32_t k = 0; k < per; ++k)
            if (b0 + k < ndig) {
                const uint32_t h = DC[b0 + k];
                DC[b0 + k] = run;
                run += h;
            }
    }
    __syncthreads();
    // 3. place records at their digit position (second read hits L1/L2)
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint64_t k = __ldg(ikeys + i);
        const uint32_t pos = DC[(uint32_t)(k >> shift) & dmask] + RK[i];
        SK[pos] = k;
        SN[pos] = __ldg(inonces + i);
    }
    __syncthreads();
    // 4. finish every digit run by insertion sort on (key64, nonce)
    for (uint32_t dg = threadIdx.x; dg < ndig; dg += NT) {
        const uint32_t s0 = DC[dg];
        const uint32_t s1 = dg + 1 < ndig ? DC[dg + 1] : n;
        for (uint32_t a = s0 + 1; a < s1; ++a) {
            const uint64_t kx = SK[a];
            const uint32_t nx = SN[a];
            uint32_t b = a;
            while (b > s0) {
                const uint64_t ky = SK[b - 1];
                const uint32_t ny = SN[b - 1];
                if (ky < kx || (ky == kx && ny < nx)) break;
                SK[b] = ky;
                SN[b] = ny;
                --b;
            }
            SK[b] = kx;
            SN[b] = nx;
        }
    }
    __syncthreads();
    // 5. Table-1 words {nonce, h0, h1}, consecutive threads on consecutive words
    uint32_t *__restrict__ t1w = reinterpret_cast<uint32_t *>(d.t1) + 3 * off;
    for (uint32_t w = threadIdx.x; w < 3 * n; w += NT) {
        const uint32_t r = w / 3, q = w - 3 * r;
        const uint64_t k = SK[r];
        t1w[w] = q == 0 ? SN[r] : bswap32(q == 1 ? (uint32_t)(k >> 32) : (uint32_t)k);
    }
    // 6. pairs starting at each record: later records of its logical bucket
    //    closer than D
    const uint64_t D = d.D;
    for (uint32_t r = threadIdx.x; r < n; r += NT) {
        const uint64_t k = SK[r];
        const uint64_t bucket = k >> 40;
        uint32_t c = 0;
        for (uint32_t r2 = r + 1; r2 < n; ++r2) {
            const uint64_t k2 = SK[r2];
            if ((k2 >> 40) != bucket || k2 - k >= D) break;
            ++c;
        }
        ST[r] = c;
    }
    __syncthreads();
    uint32_t P;
    {   // exclusive scan of the counts -> per-record Table-2 offsets
        const uint32_t per = (n + NT - 1) / NT;
        const uint32_t b0 = min(n, threadIdx.x * per), b1 = min(n, b0 + per);
        uint32_t loc = 0;
        for (uint32_t r = b0; r < b1; ++r) loc += ST[r];
        uint32_t run = block_exclusive_scan_u32<NT>(loc, WS, &P);
        for (uint32_t r = b0; r < b1; ++r) {
            const uint32_t c = ST[r];
            ST[r] = run;
            run += c;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) d.pairs[f] = P;  // lets vx_match re-run the match alone
    if (!EMIT) return;
    const uint64_t np = 1ull << d.p;
    if (MODE == kSortEmit) {
        // Table-2 base by look-back, then {a, b, 0, 0} records in (i, j) order.
        if (threadIdx.x < 32) {
            uint64_t excl = 0;
            int ok = lookback_warp(d.lb, f, P, d.status, d.spin_limit, (d.test_flags & 1u) != 0,
                                   &excl) ? 1 : 0;
            if (threadIdx.x == 0) {
                if (ok) {
                    d.t2off[f] = excl;
                    if (f + 1 == np) d.t2off[np] = excl + P;
                    if (excl + P > d.t2cap) {
                        atomicOr(d.status, kStT2Capacity);
                        ok = 0;
                    }
                }
                s_base = excl;
                s_ok = ok;
            }
        }
        __syncthreads();
        if (!s_ok) return;
        uint4 *__restrict__ out = reinterpret_cast<uint4 *>(d.t2) + s_base;
        for (uint32_t r = threadIdx.x; r < n; r += NT) {
            const uint32_t s0 = ST[r];
            const uint32_t s1 = r + 1 < n ? ST[r + 1] : P;
            const uint32_t a = SN[r];
            for (uint32_t k = s0; k < s1; ++k) out[k] = make_uint4(a, SN[r + 1 + (k - s0)], 0u, 0u);
        }
        return;
    }
    // 7. Table-2 base by look-back (after the first window is listed, to
    //    give the partitions before this one time to publish)
    uint32_t g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
    bool first = true;
    uint32_t w0 = 0;
    do {
        const uint32_t w1 = min(P, w0 + kSMList);
        for (uint32_t r = threadIdx.x; r < n; r += NT) {
            const uint32_t s = ST[r];
            const uint32_t e = r + 1 < n ? ST[r + 1] : P;
            const uint32_t lo = max(s, w0), hi = min(e, w1);
            for (uint32_t k = lo; k < hi; ++k) LS[k - w0] = r | ((r + 1 + (k - s)) << 16);
        }
        if (first) {
            if (threadIdx.x < 32) {
                uint64_t excl = 0;
                int ok = lookback_warp(d.lb, f, P, d.status, d.spin_limit,
                                       (d.test_flags & 1u) != 0, &excl) ? 1 : 0;
                if (threadIdx.x == 0) {
                    if (ok) {
                        d.t2off[f] = excl;
                        if (f + 1 == np) d.t2off[np] = excl + P;
                        if (excl + P > d.t2cap) {
                            atomicOr(d.status, kStT2Capacity);
                            ok = 0;
                        }
                    }
                    s_base = excl;
                    s_ok = ok;
                }
            }
            first = false;
        }
        __syncthreads();
        if (!s_ok) return;
        uint4 *__restrict__ out = reinterpret_cast<uint4 *>(d.t2) + s_base;
        for (uint32_t q = threadIdx.x; q < w1 - w0; q += NT) {
            const uint32_t e = LS[q];
            const uint32_t a = SN[e & 0xffffu], b = SN[e >> 16];
            uint32_t h0, h1;
            b3_finish<true>(g, a, b, h0, h1);
            out[w0 + q] = make_uint4(a, b, h0, h1);
        }
        __syncthreads();
        w0 = w1;
    } while (w0 < P);
}

size_t sortmatch_smem_bytes(uint32_t cap, int dbits) { return SMLayout(cap, dbits, true).bytes; }

template <int MODE>
static cudaError_t launch_sm(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits)
{
    if (total_tiles == 0) return cudaSuccess;
    const size_t smem = SMLayout(max_cap, max_dbits, MODE == kSortHash).bytes;
    auto fn = k_sortmatch<MODE>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<total_tiles, kSMThreads, smem, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

cudaError_t launch_sortmatch(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits,
                             bool fused_hash)
{
    if (fused_hash)
        return launch_sm<kSortHash>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits);
    return launch_sm<kSortEmit>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits);
}

cudaError_t launch_sort(const Desc *descs, int nplots, const uint32_t *tile_start,
                        uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits)
{
    return launch_sm<kSortCount>(descs, nplots, tile_start, total_tiles, s, max_cap, max_dbits);
}

}  // namespace vx
