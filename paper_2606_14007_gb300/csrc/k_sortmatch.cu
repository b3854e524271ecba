// k_sortmatch.cu -- partition sort fused with the match stage.
//
// Paper: Sec. I-B / III-A / III-B fuse sort and Table-2 generation into one
// kernel that keeps each bucket in shared memory, one block per bucket,
// with a single-thread insertion sort; Sec. V names that O(n^2) sort as the
// K=31 bottleneck and proposes a parallel radix sort.  Kept here: the
// fusion (a partition never leaves shared memory between sort and match).
// Changed: one CTA per physical partition (a run of whole logical buckets,
// ~2048 records; five CTAs per SM), a counting-sort pass on the key bits
// below the partition prefix followed by per-digit insertion sorts (about
// one record per digit), and the partition's Table-2 base found by a
// decoupled look-back over the partitions before it (partition order comes
// from a ticket counter, so every partition a CTA waits on is already
// running; every wait is bounded and a timeout poisons the chain instead of
// hanging).  With the cross-bucket match (HALO instances) the next
// partition's halo is sorted in behind the partition's records.
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
constexpr uint32_t kSMList = 2048;  // pair-list window (entries), kSortHash only
constexpr int kSMThreads = 256;
// Tickets between a CTA and the partition whose slot it prefetches into L2:
// about half of the CTAs resident at once (152 SMs x 5).  Measured at K=31:
// 38.7 ms for 190..380, 39.0 ms for 760, 41.0 ms (no gain) from 1520 up.
// Only the filled part is fetched (the whole slot cost 27% extra DRAM
// reads), its fill count loaded at CTA start and used after step 1 so the
// load's latency hides under the histogram.
constexpr uint32_t kSlotPrefetchAhead = 384;

// Shared layout: sorted key64 [cap] | sorted nonce [cap] | rank within the
// digit, u16 [cap] + digit counters [2^dbits], later overlaid by the
// per-record pair count -> Table-2 offset [cap] | pair list (kSortHash) |
// scan workspace.  The latency-bound sort runs five CTAs per SM (48
// registers): measured 41.0 ms at K=31 against 44.8 ms with four.
struct SMLayout {
    size_t sn, rank, dcnt, start, list, ws, bytes;
    __host__ __device__ SMLayout(uint32_t cap, int dbits, bool with_list)
    {
        sn = (size_t)cap * 8;
        rank = sn + (size_t)cap * 4;
        dcnt = rank + (size_t)((cap + 1) & ~1u) * 2;
        // The per-record pair counts (step 5 on) reuse the rank and digit-
        // counter space, dead after step 4: 43.8 KiB at the default 2608-
        // record slot, so five CTAs fit an SM's 228 KiB.
        start = rank;
        const size_t rd_end = dcnt + ((size_t)1 << dbits) * 4;
        const size_t st_end = start + (size_t)cap * 4;
        list = rd_end > st_end ? rd_end : st_end;
        ws = list + (with_list ? (size_t)kSMList * 4 : 0);
        bytes = ws + 40 * 4;
    }
};

template <int MODE, bool HALO>
__global__ void __launch_bounds__(kSMThreads, MODE == kSortHash ? 3 : 5)
    k_sortmatch(const Desc *__restrict__ descs, int nplots, const uint32_t *__restrict__ tile_start)
{
    constexpr bool EMIT = MODE == kSortHash || MODE == kSortEmit;  // look-back placement
    constexpr bool SLOTS = MODE == kSortSlots;
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
    // Warm L2 with the filled part of the slot of the partition
    // kSlotPrefetchAhead tickets (CTAs) ahead, so that its CTA's first reads
    // (steps 1, 3) hit L2; its fill count is read now and used after step 1.
    const uint64_t fa = (uint64_t)f + kSlotPrefetchAhead;
    const uint32_t nfa = (threadIdx.x == 0 && fa < (1ull << d.p)) ? min(d.cnt2[fa], cap) : 0u;
    const uint32_t ndig = 1u << dbits;
    const uint32_t hcap = HALO ? d.hcap : 0u;
    const SMLayout L(cap + hcap, dbits, MODE == kSortHash);  // + the next partition's halo
    uint64_t *SK = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *SN = reinterpret_cast<uint32_t *>(smem_raw + L.sn);
    uint16_t *RK = reinterpret_cast<uint16_t *>(smem_raw + L.rank);
    uint32_t *DC = reinterpret_cast<uint32_t *>(smem_raw + L.dcnt);
    uint32_t *ST = reinterpret_cast<uint32_t *>(smem_raw + L.start);
    uint32_t *LS = reinterpret_cast<uint32_t *>(smem_raw + L.list);
    uint32_t *WS = reinterpret_cast<uint32_t *>(smem_raw + L.ws);

    const uint32_t n = min(d.cnt2[f], cap);
    const uint64_t off = d.t1off[f];
    // The slot is read through the read-only path unless this kernel later
    // overwrites it with the partition's pairs.
    const uint64_t *ikeys = d.b_keys + (uint64_t)f * cap;
    const uint32_t *inonces = d.b_nonces + (uint64_t)f * cap;
    auto key_at = [&](uint32_t i) -> uint64_t { return SLOTS ? ikeys[i] : __ldg(ikeys + i); };
    auto nonce_at = [&](uint32_t i) -> uint32_t { return SLOTS ? inonces[i] : __ldg(inonces + i); };
    const int shift = 64 - d.pk - dbits;
    const uint32_t dmask = ndig - 1u;

    // 1. digit histogram (rank of each record within its digit)
    for (uint32_t i = threadIdx.x; i < ndig; i += NT) DC[i] = 0u;
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint32_t dg = (uint32_t)(key_at(i) >> shift) & dmask;
        RK[i] = (uint16_t)atomicAdd(&DC[dg], 1u);
    }
    if (nfa) {
        const uint32_t nk = (nfa + 1u) & ~1u, nn = (nfa + 3u) & ~3u;  // 16-byte multiples
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_keys + fa * cap),
                     "r"(nk * 8u)
                     : "memory");
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(d.b_nonces + fa * cap),
                     "r"(nn * 4u)
                     : "memory");
    }
    __syncthreads();
    // 2. digit counters -> digit start positions
    block_scan_inplace_u32<NT>(DC, ndig, WS);
    // 3. place records at their digit position (the second read of the
    //    slot hits L1/L2)
    for (uint32_t i = threadIdx.x; i < n; i += NT) {
        const uint64_t k = key_at(i);
        const uint32_t pos = DC[(uint32_t)(k >> shift) & dmask] + RK[i];
        SK[pos] = k;
        SN[pos] = nonce_at(i);
    }
    __syncthreads();
    // 4. finish every digit run (about one record each) by insertion sort on
    //    (key64, nonce)
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
    // 4b. cross-bucket match: the next partition's halo (its records within
    //     D of its lower edge, collected while the slots were filled) goes
    //     sorted right after this partition's records, so the pair scan
    //     below runs on into it; records n .. nt - 1 start no pairs here.
    uint32_t nt = n;
    if (HALO && hcap) {
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
                for (; b > n && (SK[b - 1] > kx || (SK[b - 1] == kx && SN[b - 1] > nx)); --b) {
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
    // 5. pairs starting at each record r: the later records up to
    //    lim = min(last key of r's logical bucket, key_r + D - 1), or
    //    key_r + D - 1 for the cross-bucket match; four probes per step
    //    (key64 sorted ascending)
    const uint64_t D = d.D;
    const bool global = HALO && d.scope != 0;
    for (uint32_t r = threadIdx.x; r < n; r += NT) {
        const uint64_t k = SK[r];
        const uint64_t last_in_bucket = global ? ~0ull : (k | ((1ull << 40) - 1));
        uint64_t reach = k + (D - 1);
        if (reach < k) reach = ~0ull;  // saturate
        const uint64_t lim = reach < last_in_bucket ? reach : last_in_bucket;
        uint32_t c = 0;
        for (uint32_t q = r + 1; q < nt; q += 4) {
            const bool m0 = SK[q] <= lim;
            const bool m1 = m0 && q + 1 < nt && SK[q + 1] <= lim;
            const bool m2 = m1 && q + 2 < nt && SK[q + 2] <= lim;
            const bool m3 = m2 && q + 3 < nt && SK[q + 3] <= lim;
            c += (uint32_t)m0 + (uint32_t)m1 + (uint32_t)m2 + (uint32_t)m3;
            if (!m3) break;
        }
        ST[r] = c;
    }
    __syncthreads();
    // 6. counts -> per-record Table-2 offsets; the partition's pair count
    //    is published at once so later partitions are not held up
    const uint32_t P = block_scan_inplace_u32<NT>(ST, n, WS);
    const bool withhold = (d.test_flags & 1u) != 0;
    if (threadIdx.x == 0) {
        d.pairs[f] = P;  // lets vx_match re-run the match alone
        if (EMIT) lb_publish(d.lb, f, P, withhold);
    }
    // 7. Table 1.  Records 12 B each: the head up to a 16-byte boundary and
    //    the tail go word by word; the body goes as groups of 4 records =
    //    three 16-byte stores per thread.  (Resolving the look-back in warp 0
    //    while the other warps write Table 1 measured slower than this
    //    order: 45.2 vs 44.8 ms at K=31.)
    const uint64_t np = 1ull << d.p;
    {
        constexpr uint32_t NW = NT;  // Table-1 writers
        const uint32_t tw = threadIdx.x;
        uint32_t *__restrict__ t1w = reinterpret_cast<uint32_t *>(d.t1) + 3 * off;
        const uint32_t head = min(n, (uint32_t)((4u - (uint32_t)(off & 3u)) & 3u));
        const uint32_t groups = (n - head) / 4u;
        const uint32_t tail0 = head + 4u * groups;
        for (uint32_t r = tw; r < head + (n - tail0); r += NW) {
            const uint32_t rr = r < head ? r : tail0 + (r - head);
            const uint64_t k = SK[rr];
            t1w[3 * rr] = SN[rr];
            t1w[3 * rr + 1] = bswap32((uint32_t)(k >> 32));
            t1w[3 * rr + 2] = bswap32((uint32_t)k);
        }
        uint4 *__restrict__ body = reinterpret_cast<uint4 *>(t1w + 3 * head);
        for (uint32_t g = tw; g < groups; g += NW) {
            const uint32_t r = head + 4u * g;
            uint32_t w[12];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t k = SK[r + j];
                w[3 * j] = SN[r + j];
                w[3 * j + 1] = bswap32((uint32_t)(k >> 32));
                w[3 * j + 2] = bswap32((uint32_t)k);
            }
            body[3 * g] = make_uint4(w[0], w[1], w[2], w[3]);
            body[3 * g + 1] = make_uint4(w[4], w[5], w[6], w[7]);
            body[3 * g + 2] = make_uint4(w[8], w[9], w[10], w[11]);
        }
    }
    if (SLOTS) {
        // 8. pairs into the slot (its records were read before the
        //    barriers above)
        const uint32_t capA = cap, capB = cap / 2u;
        if (P > capA + capB) {
            if (threadIdx.x == 0) atomicOr(d.status, kStPairSlot);
            return;
        }
        uint2 *__restrict__ pa = reinterpret_cast<uint2 *>(d.b_keys + (uint64_t)f * cap);
        uint2 *__restrict__ pb = reinterpret_cast<uint2 *>(d.b_nonces + (uint64_t)f * cap);
        for (uint32_t r = threadIdx.x; r < n; r += NT) {
            const uint32_t s0 = ST[r];
            const uint32_t s1 = r + 1 < n ? ST[r + 1] : P;
            const uint32_t a = SN[r];
            for (uint32_t k = s0; k < s1; ++k) {
                const uint2 v = make_uint2(a, SN[r + 1 + (k - s0)]);
                if (k < capA)
                    pa[k] = v;
                else
                    pb[k - capA] = v;
            }
        }
        return;
    }
    if (!EMIT) return;
    // 8. Table-2 base: resolve the look-back (warp 0)
    if (threadIdx.x < 32) {
        uint64_t excl = 0;
        int ok = lb_resolve(d.lb, f, P, d.status, d.spin_limit, withhold, &excl) ? 1 : 0;
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
    if (MODE == kSortEmit) {
        // 9a. {a, b, 0, 0} records in (i, j) order; hashes come later
        for (uint32_t r = threadIdx.x; r < n; r += NT) {
            const uint32_t s0 = ST[r];
            const uint32_t s1 = r + 1 < n ? ST[r + 1] : P;
            const uint32_t a = SN[r];
            for (uint32_t k = s0; k < s1; ++k) out[k] = make_uint4(a, SN[r + 1 + (k - s0)], 0u, 0u);
        }
        return;
    }
    // 9b. hash here: list the pairs window by window, every lane hashes
    uint32_t g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
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

size_t sortmatch_smem_bytes(uint32_t cap, int dbits) { return SMLayout(cap, dbits, true).bytes; }

uint32_t sortmatch_max_cap() { return 16384u; }

template <int MODE, bool HALO>
static cudaError_t launch_sm(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, cudaStream_t s, uint32_t max_cap, int max_dbits)
{
    if (total_tiles == 0) return cudaSuccess;
    const size_t smem = SMLayout(max_cap, max_dbits, MODE == kSortHash).bytes;
    auto fn = k_sortmatch<MODE, HALO>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<total_tiles, kSMThreads, smem, s>>>(descs, nplots, tile_start);
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
