// k_match.cu -- the match stage and Table 2.
//
// Paper: Sec. II-B (pairwise match against a matching-factor threshold ->
// Table 2) and Sec. III-A (match half of the fused Sort+Match kernel, one
// bucket per block, data kept in shared memory).  Here one CTA takes one
// physical partition (a run of whole logical buckets) of the sorted Table 1
// into shared memory, counts for every record i the later records j of its
// logical bucket with key64_j - key64_i < D, turns the counts into
// positions with a block prefix sum, lists the pairs in shared memory in
// (i, j) order, and then every lane hashes list entries back to back, so
// the one-compression-per-pair work never idles lanes on records without a
// partner.  Table-2 placement comes from the per-partition pair counts of
// the sort kernel and an exclusive scan: deterministic, no atomics.
#include "vx_internal.cuh"

namespace vx {

// Shared layout for slots of at most `cap` records (with the halo): key64
// [cap] | nonce [cap] | pair offset [cap] | scan workspace.  Once the pairs
// are counted the keys are dead and their space holds the pair list, in
// windows of 2 * cap entries (2 x u16 each).
struct MatchLayout {
    size_t nonces, start, ws, bytes;
    __host__ __device__ MatchLayout(uint32_t cap)
    {
        nonces = (size_t)cap * 8;
        start = nonces + (size_t)cap * 4;
        ws = start + (size_t)cap * 4;
        bytes = ws + (kMatchThreads / 32 + 1) * 4;
    }
};

__global__ void __launch_bounds__(kMatchThreads) k_match(const Desc *__restrict__ descs, int nplots,
                                                         const uint32_t *__restrict__ tile_start)
{
    constexpr int NT = kMatchThreads;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    const uint32_t f = blockIdx.x - tile_start[plot];
    const uint64_t np = 1ull << d.p;
    if (d.t2off[np] > d.t2cap) return;  // capacity exceeded: the scan flagged it
    const uint64_t pbase = d.t2off[f];
    const uint32_t P = (uint32_t)(d.t2off[f + 1] - pbase);
    if (P == 0) return;
    const uint64_t off = d.t1off[f];
    const uint32_t n = (uint32_t)(d.t1off[f + 1] - off);
    const MatchLayout L(d.cap2 + d.hcap);  // + the next partition's halo
    uint64_t *keys = reinterpret_cast<uint64_t *>(smem_raw);
    uint32_t *nonces = reinterpret_cast<uint32_t *>(smem_raw + L.nonces);
    uint32_t *start = reinterpret_cast<uint32_t *>(smem_raw + L.start);
    uint32_t *list = reinterpret_cast<uint32_t *>(smem_raw);  // over the keys, after the counts
    const uint32_t kPairList = 2u * (d.cap2 + d.hcap);
    uint32_t *ws = reinterpret_cast<uint32_t *>(smem_raw + L.ws);

    // Table-1 words {nonce, h0, h1} -> nonce[], key64[] (key64 = BE of h).
    const uint32_t *__restrict__ t1w = reinterpret_cast<const uint32_t *>(d.t1) + 3 * off;
    uint32_t *khalf = reinterpret_cast<uint32_t *>(keys);
    for (uint32_t w = threadIdx.x; w < 3 * n; w += NT) {
        const uint32_t r = w / 3, q = w - 3 * r;
        const uint32_t v = t1w[w];
        if (q == 0) nonces[r] = v;
        else khalf[2 * r + (q == 1 ? 1 : 0)] = bswap32(v);
    }
    // Cross-bucket match: the next partition's first records within D of
    // its lower edge (a prefix of its sorted Table-1 run) follow this
    // partition's records, so the pair scan runs on into them.
    const uint64_t D = d.D;
    uint32_t nt = n;
    if (d.hcap && f + 1 < np) {
        const uint64_t hoff = d.t1off[f + 1];
        const uint64_t hrun = d.t1off[f + 2] - hoff;
        const uint32_t hn = (uint32_t)(hrun < d.hcap ? hrun : d.hcap);
        const uint64_t edge = (uint64_t)(f + 1) << (64 - d.p);
        bool in = false;
        uint32_t nv = 0;
        uint64_t kv = 0;
        if (threadIdx.x < hn) {
            const uint32_t *w = reinterpret_cast<const uint32_t *>(d.t1) + 3 * (hoff + threadIdx.x);
            nv = w[0];
            kv = ((uint64_t)bswap32(w[1]) << 32) | bswap32(w[2]);
            in = kv - edge < D;
        }
        const uint32_t hc = (uint32_t)__syncthreads_count(in);  // a prefix: keys ascend
        if (in) {
            keys[n + threadIdx.x] = kv;
            nonces[n + threadIdx.x] = nv;
        }
        nt = n + hc;
    }
    __syncthreads();

    // Per-record pair counts, chunks of 32 sorted records (one per lane),
    // warp w over chunks [c0, c1): the later records up to lim =
    // min(last key of r's logical bucket, key_r + D - 1), or key_r + D - 1
    // for the cross-bucket match (four probes, then one by one while all
    // four match), and their warp scans.  Probes may read up to four
    // entries past the records: inside the shared allocation, and masked.
    const bool global = d.scope != 0;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr uint32_t NW = NT / 32;
    const uint32_t nch = (n + 31u) >> 5;
    const uint32_t c0 = warp * nch / NW, c1 = (warp + 1) * nch / NW;
    uint32_t carry = 0;  // the warp's pairs before the current chunk
    for (uint32_t c = c0; c < c1; ++c) {
        const uint32_t r = 32u * c + lane;
        uint32_t cnt = 0;
        if (r < n) {
            const uint64_t k = keys[r];
            const uint64_t last = global ? ~0ull : (k | ((1ull << 40) - 1));
            uint64_t lim = k + (D - 1);
            if (lim < k) lim = ~0ull;  // saturate
            if (lim > last) lim = last;
            const uint64_t k1 = keys[r + 1], k2 = keys[r + 2], k3 = keys[r + 3], k4 = keys[r + 4];
            const bool m1 = r + 1 < nt && k1 <= lim;
            const bool m2 = m1 && r + 2 < nt && k2 <= lim;
            const bool m3 = m2 && r + 3 < nt && k3 <= lim;
            const bool m4 = m3 && r + 4 < nt && k4 <= lim;
            cnt = (uint32_t)m1 + (uint32_t)m2 + (uint32_t)m3 + (uint32_t)m4;
            if (m4)
                for (uint32_t q = r + 5; q < nt && keys[q] <= lim; ++q) ++cnt;
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        if (r < n) start[r] = carry + incl - cnt;
        carry += __shfl_sync(0xffffffffu, incl, 31);
    }
    if (lane == 0) ws[warp] = carry;
    __syncthreads();
    uint32_t wbase = 0, total = 0;
#pragma unroll
    for (uint32_t w = 0; w < NW; ++w) {
        const uint32_t t = ws[w];
        wbase += w < warp ? t : 0u;
        total += t;
    }
    if (total != P && threadIdx.x == 0) atomicOr(d.status, kStCountMismatch);
    // the warp's pairs end here (a record's count is the gap to the next
    // record's offset; the warp's total after its last record)
    const uint32_t rend = min(32u * c1, n);
    uint32_t g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
    uint4 *__restrict__ out = reinterpret_cast<uint4 *>(d.t2) + pbase;
    const uint32_t limit = min(total, P);
    for (uint32_t w0 = 0; w0 < limit; w0 += kPairList) {
        const uint32_t w1 = min(limit, w0 + kPairList);
        // List the pairs whose Table-2 position falls in [w0, w1): each lane
        // its records' pairs (r, r + 1 + j) at the warp base plus the
        // record's offset.
        for (uint32_t c = c0; c < c1; ++c) {
            const uint32_t r = 32u * c + lane;
            if (r < n) {
                const uint32_t s = wbase + start[r];
                const uint32_t e = wbase + (r + 1 < rend ? start[r + 1] : carry);
                const uint32_t lo = max(s, w0), hi = min(e, w1);
                for (uint32_t k = lo; k < hi; ++k) list[k - w0] = r | ((r + 1 + (k - s)) << 16);
            }
        }
        __syncthreads();
        for (uint32_t q = threadIdx.x; q < w1 - w0; q += NT) {
            const uint32_t e = list[q];
            const uint32_t a = nonces[e & 0xffffu], b = nonces[e >> 16];
            uint32_t h0, h1;
            b3_finish<true>(g, a, b, h0, h1);
            out[w0 + q] = make_uint4(a, b, h0, h1);
        }
        __syncthreads();
    }
}

size_t match_smem_bytes(uint32_t cap) { return MatchLayout(cap).bytes; }

cudaError_t launch_match(const Desc *descs, int nplots, const uint32_t *tile_start,
                         uint32_t total_tiles, cudaStream_t s, uint32_t max_cap)
{
    const size_t smem = match_smem_bytes(max_cap);
    cudaError_t e = cudaFuncSetAttribute(k_match, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_match<<<total_tiles, kMatchThreads, smem, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

}  // namespace vx
