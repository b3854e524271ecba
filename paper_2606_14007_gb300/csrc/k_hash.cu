// k_hash.cu -- key setup, Table-1 hashing fused with the first bucketing
// scatter (also for one window of a plot: filtering every nonce's key, or
// hashing the window's listed nonces), the window-id and window-list passes
// of tiled plots, and the stand-alone hash / pair-hash kernels.
//
// Paper: Sec. III-A/III-B (one keyed BLAKE3 per nonce, little-endian nonce,
// bucket index from the hash prefix).  The paper's kernel claims one bucket
// slot per nonce with a global atomicAdd; here a CTA hashes a tile of
// nonces, histograms them by the leading hash bits in shared memory
// (warp-aggregated with __match_any_sync where bins are few), claims one
// contiguous run per (CTA, bin) with a single global atomic, and writes the
// records partition-ordered so that consecutive threads store consecutive
// addresses.  Order inside a partition is irrelevant: the partition sort
// orders records by (key64, nonce), a total order.
#include "vx_internal.cuh"

namespace vx {

// ------------------------------------------------------------ key setup
// One CTA row per plot: thread 0 of block x == 0 derives the per-key hash
// states; every CTA zeroes a share of the plot's fill counters and the
// status word.
__global__ void k_key_setup(Desc *descs)
{
    Desc &d = descs[blockIdx.y];
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        uint32_t pre[16];
        b3_key_setup(d.key, 4u, pre);
        for (int i = 0; i < 16; ++i) d.pre1[i] = pre[i];
        b3_key_setup(d.key, 8u, pre);
        for (int i = 0; i < 16; ++i) d.pre2[i] = pre[i];
        *d.status = 0u;
        *d.ticket = 0u;
        *d.ticket_s = 0u;
        if (d.wcount) *d.wcount = 0u;
    }
    const uint64_t n1 = d.p2 > 0 ? ((uint64_t)d.hchunks << d.p1) : 0ull;
    const uint64_t n2 = 1ull << d.p;
    const uint64_t nchunks = (n2 + kScanChunk - 1) / kScanChunk;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t nz = n2 > n1 ? n2 : n1;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nz; i += stride) {
        if (i < n2) {
            d.cnt2[i] = 0u;
            d.lb[i] = 0ull;
            if (d.hcap) d.halo_cnt[i] = 0u;
        }
        if (i < n1) d.cnt1[i] = 0u;
        if (i < nchunks) d.lbs[i] = 0ull;
    }
}

cudaError_t launch_key_setup(Desc *descs, int nplots, cudaStream_t s)
{
    dim3 grid(64, nplots);
    k_key_setup<<<grid, 256, 0, s>>>(descs);
    return cudaGetLastError();
}

// --------------------------------------------- hash + first-level scatter
// Shared layout of one tile: staged key64[T], nonce[T], then per-bin
// histogram, local offset and claimed global base (kMaxCoarseBits bins).
template <int NT, int NPT>
struct HashSmem {
    static constexpr int T = NT * NPT;
    uint64_t keys[T];
    uint32_t nonces[T];
    uint32_t hist[1 << kMaxCoarseBits];
    uint32_t loff[1 << kMaxCoarseBits];
    uint32_t gbase[1 << kMaxCoarseBits];
    uint32_t ws[NT / 32 + 1];
};

// Rank of this lane's record within its bin's run of the tile.
template <bool AGG>
__device__ __forceinline__ uint32_t bin_rank(uint32_t *hist, uint32_t bin, bool valid)
{
    if (AGG) {
        const uint32_t peers = __match_any_sync(0xffffffffu, valid ? bin : 0xffffffffu);
        const int leader = __ffs(peers) - 1;
        const int lane = threadIdx.x & 31;
        uint32_t base = 0;
        if (lane == leader && valid) base = atomicAdd(&hist[bin], (uint32_t)__popc(peers));
        base = __shfl_sync(0xffffffffu, base, leader);
        return base + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    } else {
        return valid ? atomicAdd(&hist[bin], 1u) : 0u;
    }
}

// Exclusive scan of hist[0..nbins) into loff, and one global claim per
// non-empty bin: gbase[b] = atomicAdd(&cnt[bin_base + b], hist[b]).
template <int NT>
__device__ __forceinline__ void scan_and_claim(uint32_t *hist, uint32_t *loff, uint32_t *gbase,
                                               uint32_t *ws, int nbins, uint32_t *cnt,
                                               uint32_t bin_base)
{
    const int per = (nbins + NT - 1) / NT;  // <= 4 for 1024 bins and 256 threads
    const int b0 = threadIdx.x * per;
    uint32_t local = 0;
    for (int k = 0; k < per; ++k)
        if (b0 + k < nbins) local += hist[b0 + k];
    uint32_t total;
    uint32_t run = block_exclusive_scan_u32<NT>(local, ws, &total);
    for (int k = 0; k < per; ++k) {
        const int b = b0 + k;
        if (b < nbins) {
            const uint32_t h = hist[b];
            loff[b] = run;
            run += h;
            gbase[b] = h ? atomicAdd(&cnt[bin_base + b], h) : 0u;
        }
    }
}

// Windowed plots keep the keys whose top wbits equal win and bin them by the
// bits after those.  kWinFilter instances hash every nonce and test its key
// (a plot without a window, wbits 0, keeps every key, so one such launch may
// also carry whole plots); kWinList instances hash only the nonces listed
// for the window (Desc::wlist, from a pass that stored every nonce's window).
enum { kWinNone = 0, kWinFilter = 1, kWinList = 2 };

// Window bits plus bin bits are at most the 21 partition bits, so both tests
// read only the key's high word.
template <bool WIN>
__device__ __forceinline__ bool in_window(const Desc &d, uint64_t key)
{
    const uint32_t hi = (uint32_t)(key >> 32);
    return !WIN || ((hi >> 1) >> (31 - d.wbits)) == d.win;  // wbits 0: always
}

template <bool WIN>
__device__ __forceinline__ uint32_t key_bin(const Desc &d, uint64_t key, int bits)
{
    const uint32_t hi = (uint32_t)(key >> 32);
    return bits ? (WIN ? hi << d.wbits : hi) >> (32 - bits) : 0u;
}

template <int NT, int NPT, bool AGG, bool HALO, int WM>
__global__ void __launch_bounds__(NT) k_hash_scatter(const Desc *__restrict__ descs, int nplots,
                                                     const uint32_t *__restrict__ tile_start,
                                                     int chunk)
{
    using S = HashSmem<NT, NPT>;
    constexpr int T = S::T;
    constexpr bool WIN = WM != kWinNone;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    S &sm = *reinterpret_cast<S *>(smem_raw);

    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    uint64_t lo, N;  // this chunk's nonces: [lo, N), or (list) list entries [0, N)
    nonce_chunk(d, chunk, lo, N);
    if (WM == kWinList) N = min(*d.wcount, d.listcap);
    const uint64_t base = lo + (uint64_t)(blockIdx.x - tile_start[plot]) * T;
    if (WM == kWinList && base >= N) return;  // the grid covers the list's capacity
    const bool two_level = d.p2 > 0;
    const int bits = two_level ? d.p1 : d.p;
    const int nbins = 1 << bits;
    const uint32_t cap = two_level ? d.cap1 : d.cap2;
    // Two levels: this chunk's own level-1 slots; one level: the final slots.
    const uint64_t slot0 = two_level ? ((uint64_t)chunk << d.p1) : 0ull;
    uint64_t *__restrict__ okeys = two_level ? d.a_keys + slot0 * cap : d.b_keys;
    uint32_t *__restrict__ ononces = two_level ? d.a_nonces + slot0 * cap : d.b_nonces;
    uint32_t *cnt = two_level ? d.cnt1 + slot0 : d.cnt2;

    uint32_t pre[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) pre[i] = d.pre1[i];

    for (int b = threadIdx.x; b < nbins; b += NT) sm.hist[b] = 0u;
    __syncthreads();

    uint64_t key[NPT];
    uint32_t rank[NPT];
    uint32_t count;  // records the tile keeps
    if constexpr (!WIN) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const uint64_t nonce = base + (uint64_t)j * NT + threadIdx.x;
            const bool valid = nonce < N;
            uint32_t h0, h1;
            b3_finish<false>(pre, (uint32_t)nonce, 0u, h0, h1);
            key[j] = key64_of(h0, h1);
            const uint32_t bin = bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u;
            rank[j] = bin_rank<AGG>(sm.hist, bin, valid);
        }
        __syncthreads();
        scan_and_claim<NT>(sm.hist, sm.loff, sm.gbase, sm.ws, nbins, cnt, 0u);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const uint64_t nonce = base + (uint64_t)j * NT + threadIdx.x;
            if (nonce < N) {
                const uint32_t bin = bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u;
                const uint32_t pos = sm.loff[bin] + rank[j];
                sm.keys[pos] = key[j];
                sm.nonces[pos] = (uint32_t)nonce;
            }
        }
        __syncthreads();
        count = (uint32_t)((N - base) < (uint64_t)T ? (N - base) : (uint64_t)T);
    } else {
        uint32_t keep = 0;  // bit j: record j's nonce exists and its key is in the window
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const uint64_t idx = base + (uint64_t)j * NT + threadIdx.x;
            uint32_t nonce;
            if constexpr (WM == kWinList) nonce = idx < N ? d.wlist[idx] : 0u;
            else nonce = (uint32_t)idx;
            uint32_t h0, h1;
            b3_finish<false>(pre, nonce, 0u, h0, h1);
            key[j] = key64_of(h0, h1);
            const bool valid = idx < N && (WM != kWinFilter || in_window<true>(d, key[j]));
            keep |= (valid ? 1u : 0u) << j;
            rank[j] = bin_rank<AGG>(sm.hist, key_bin<true>(d, key[j], bits), valid);
        }
        __syncthreads();
        scan_and_claim<NT>(sm.hist, sm.loff, sm.gbase, sm.ws, nbins, cnt, 0u);
        __syncthreads();
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            if (keep >> j & 1u) {
                const uint64_t idx = base + (uint64_t)j * NT + threadIdx.x;
                const uint32_t pos = sm.loff[key_bin<true>(d, key[j], bits)] + rank[j];
                sm.keys[pos] = key[j];
                sm.nonces[pos] = WM == kWinList ? d.wlist[idx] : (uint32_t)idx;
            }
        }
        __syncthreads();
        count = sm.loff[nbins - 1] + sm.hist[nbins - 1];  // the histogram's total
    }
    bool overflow = false, hover = false;
    for (uint32_t i = threadIdx.x; i < count; i += NT) {
        const uint64_t k = sm.keys[i];
        const uint32_t bin = WIN ? key_bin<true>(d, k, bits) : (bits ? (uint32_t)(k >> (64 - bits)) : 0u);
        const uint32_t g = sm.gbase[bin] + (i - sm.loff[bin]);
        if (g < cap) {
            const uint64_t at = (uint64_t)bin * cap + g;
            okeys[at] = k;
            ononces[at] = sm.nonces[i];
        } else {
            overflow = true;
        }
        if (HALO && !two_level) halo_add(d, bin, k, sm.nonces[i], hover);  // final partitions
    }
    if (overflow) atomicOr(d.status, two_level ? kStSlot1Overflow : kStSlot2Overflow);
    if (hover) atomicOr(d.status, kStHaloOverflow);
}

template <int NT, int NPT, bool AGG, bool HALO, int WM>
static cudaError_t launch_hs(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, int chunk, cudaStream_t s)
{
    const size_t smem = sizeof(HashSmem<NT, NPT>);
    auto fn = k_hash_scatter<NT, NPT, AGG, HALO, WM>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<total_tiles, NT, smem, s>>>(descs, nplots, tile_start, chunk);
    return cudaGetLastError();
}

// AGG (warp-aggregated ranks) pays off when a warp's 32 records fall into
// few bins; the host picks it from the smallest bin count in the launch.
// HALO instances carry the cross-bucket halo code and window instances the
// window filter or the nonce list; plain launches carry neither.  A list
// launch holds one windowed plot (never cross-bucket).
// Whole plots may take 4 or 16 nonces per thread instead of 8 (a tuning
// choice: more nonces per thread, more independent hashes in flight per
// thread but fewer resident CTAs); windows always take 8.
template <bool HALO, int WM, int P>
static cudaError_t launch_hs_npt(const Desc *descs, int nplots, const uint32_t *tile_start,
                                 uint32_t total_tiles, bool agg, int chunk, cudaStream_t s)
{
    constexpr int T = kHashThreads;
    return agg ? launch_hs<T, P, true, HALO, WM>(descs, nplots, tile_start, total_tiles, chunk, s)
               : launch_hs<T, P, false, HALO, WM>(descs, nplots, tile_start, total_tiles, chunk, s);
}

template <bool HALO, int WM>
static cudaError_t launch_hs_agg(const Desc *descs, int nplots, const uint32_t *tile_start,
                                 uint32_t total_tiles, bool agg, int chunk, cudaStream_t s, int npt)
{
    if (WM == kWinNone && npt == 4)
        return launch_hs_npt<HALO, kWinNone, 4>(descs, nplots, tile_start, total_tiles, agg, chunk, s);
    if (WM == kWinNone && npt == 16)
        return launch_hs_npt<HALO, kWinNone, 16>(descs, nplots, tile_start, total_tiles, agg, chunk, s);
    if (npt != kHashNoncesPerThread) return cudaErrorInvalidValue;
    return launch_hs_npt<HALO, WM, kHashNoncesPerThread>(descs, nplots, tile_start, total_tiles, agg, chunk, s);
}

cudaError_t launch_hash_scatter(const Desc *descs, int nplots, const uint32_t *tile_start,
                                uint32_t total_tiles, HashCfg cfg, int chunk, cudaStream_t s)
{
    if (total_tiles == 0) return cudaSuccess;
    const int npt = cfg.npt;
    if (cfg.list)
        return cfg.halo ? cudaErrorInvalidValue
                        : launch_hs_agg<false, kWinList>(descs, nplots, tile_start, total_tiles, cfg.agg, chunk, s, npt);
    if (cfg.win)
        return cfg.halo ? launch_hs_agg<true, kWinFilter>(descs, nplots, tile_start, total_tiles, cfg.agg, chunk, s, npt)
                        : launch_hs_agg<false, kWinFilter>(descs, nplots, tile_start, total_tiles, cfg.agg, chunk, s, npt);
    return cfg.halo ? launch_hs_agg<true, kWinNone>(descs, nplots, tile_start, total_tiles, cfg.agg, chunk, s, npt)
                    : launch_hs_agg<false, kWinNone>(descs, nplots, tile_start, total_tiles, cfg.agg, chunk, s, npt);
}

// ------------------------------------------------- hash + direct scatter
// The other bucketing strategy (the paper's, Sec. III-B: an atomicAdd slot
// claim per nonce), here straight into the final partitions: every thread
// hashes NPT nonces, then claims one slot per record in its partition with
// a global atomic and stores key64 and nonce there.  No shared memory and
// no second scatter pass; the claims and scattered stores run on the LSU
// and L2 while the ALU pipe -- the kernel's bound -- keeps hashing.
template <int NT, int NPT, bool HALO, int WM>
__global__ void __launch_bounds__(NT) k_hash_direct(const Desc *__restrict__ descs, int nplots,
                                                    const uint32_t *__restrict__ tile_start,
                                                    int chunk)
{
    constexpr bool WIN = WM != kWinNone;
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    uint64_t lo, N;  // this chunk's nonces: [lo, N), or (list) list entries [0, N)
    nonce_chunk(d, chunk, lo, N);
    if (WM == kWinList) N = min(*d.wcount, d.listcap);
    const uint64_t base = lo + (uint64_t)(blockIdx.x - tile_start[plot]) * (NT * NPT);
    if (WM == kWinList && base >= N) return;  // the grid covers the list's capacity
    const int bits = d.p;
    const uint32_t cap = d.cap2;
    uint32_t pre[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) pre[i] = d.pre1[i];
    // the nonce of entry idx: the entry itself, or (list) the listed nonce
    auto nonce_of = [&](uint64_t idx) -> uint32_t {
        return WM == kWinList ? (idx < N ? d.wlist[idx] : 0u) : (uint32_t)idx;
    };
    uint64_t key[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        uint32_t h0, h1;
        b3_finish<false>(pre, nonce_of(base + (uint64_t)j * NT + threadIdx.x), 0u, h0, h1);
        key[j] = key64_of(h0, h1);
    }
    uint32_t slot[NPT];
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const uint64_t nonce = base + (uint64_t)j * NT + threadIdx.x;
        const uint32_t bin = WIN ? key_bin<true>(d, key[j], bits) : (bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u);
        // A record outside the window claims no slot: its slot reads as "none".
        slot[j] = (nonce < N && in_window<WM == kWinFilter>(d, key[j])) ? atomicAdd(&d.cnt2[bin], 1u)
                                                                         : 0xffffffffu;
    }
    bool overflow = false, hover = false;
#pragma unroll
    for (int j = 0; j < NPT; ++j) {
        const uint64_t nonce = base + (uint64_t)j * NT + threadIdx.x;
        if (nonce >= N) continue;
        if (WIN && slot[j] == 0xffffffffu) continue;
        const uint32_t bin = WIN ? key_bin<true>(d, key[j], bits) : (bits ? (uint32_t)(key[j] >> (64 - bits)) : 0u);
        if (slot[j] < cap) {
            const uint64_t at = (uint64_t)bin * cap + slot[j];
            d.b_keys[at] = key[j];
            d.b_nonces[at] = nonce_of(nonce);
        } else {
            overflow = true;
        }
        if (HALO) halo_add(d, bin, key[j], nonce_of(nonce), hover);
    }
    if (overflow) atomicOr(d.status, kStSlot2Overflow);
    if (hover) atomicOr(d.status, kStHaloOverflow);
}

template <bool HALO, int WM>
static cudaError_t launch_hd(const Desc *descs, int nplots, const uint32_t *tile_start,
                             uint32_t total_tiles, int chunk, cudaStream_t s)
{
    k_hash_direct<kHashThreads, kHashNoncesPerThread, HALO, WM><<<total_tiles, kHashThreads, 0, s>>>(
        descs, nplots, tile_start, chunk);
    return cudaGetLastError();
}

cudaError_t launch_hash_direct(const Desc *descs, int nplots, const uint32_t *tile_start,
                               uint32_t total_tiles, int chunk, cudaStream_t s, HashCfg cfg)
{
    if (total_tiles == 0) return cudaSuccess;
    if (cfg.list)
        return cfg.halo ? cudaErrorInvalidValue
                        : launch_hd<false, kWinList>(descs, nplots, tile_start, total_tiles, chunk, s);
    if (cfg.win)
        return cfg.halo ? launch_hd<true, kWinFilter>(descs, nplots, tile_start, total_tiles, chunk, s)
                        : launch_hd<false, kWinFilter>(descs, nplots, tile_start, total_tiles, chunk, s);
    return cfg.halo ? launch_hd<true, kWinNone>(descs, nplots, tile_start, total_tiles, chunk, s)
                    : launch_hd<false, kWinNone>(descs, nplots, tile_start, total_tiles, chunk, s);
}

// ------------------------------------------------ Table-2 pair hashing
// Fills hash2 of the Table-2 records {a, b, 0, 0} the sort wrote at their
// final offsets: a streaming, barrier-free pass (one compression per
// record, all lanes busy).  One launch covers one chunk of partitions --
// the records between the look-back prefixes at the chunk's ends -- so it
// can run on a second stream while the sort works on the next chunk.  A
// plot's CTAs stride over its range.  Skips plots whose Table 2 is invalid
// (capacity exceeded, a wait timed out).
constexpr int kT2HashThreads = 256;
constexpr int kT2HashPer = 8;  // records per thread of the look-back pair hash's grid

__global__ void __launch_bounds__(kT2HashThreads) k_t2_hash(const Desc *__restrict__ descs,
                                                            int nplots,
                                                            const uint32_t *__restrict__ tile_start,
                                                            int chunk)
{
    constexpr int NT = kT2HashThreads;
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    if (*d.status & (kStT2Capacity | kStTimeout | kStBadTicket)) return;
    // Records of this partition chunk: [prefix before its first partition,
    // inclusive prefix of its last), from the sort's look-back words.
    const uint64_t np = 1ull << d.p;
    const uint64_t fa = np * (uint64_t)chunk / (uint64_t)d.pchunks;
    const uint64_t fb = np * (uint64_t)(chunk + 1) / (uint64_t)d.pchunks;
    if (fa >= fb) return;
    const uint64_t w = ld_acquire_u64(d.lb + (fb - 1));
    if ((w & ~kLbMask) != kLbIncl) return;  // chain broken: status says why
    const uint64_t lo = fa == 0 ? 0ull : d.t2off[fa];
    uint64_t hi = w & kLbMask;
    if (hi > d.t2cap) hi = d.t2cap;
    const uint32_t me = blockIdx.x - tile_start[plot];
    const uint32_t ctas = tile_start[plot + 1] - tile_start[plot];
    uint32_t g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
    uint4 *__restrict__ t2 = reinterpret_cast<uint4 *>(d.t2);
    // One record per iteration, loop kept rolled: the body is one
    // compression, small enough for the instruction cache even when the
    // warps (no barrier here) drift apart; unrolling several compressions
    // made the warps stall on instruction fetch.
#pragma unroll 1
    for (uint64_t q = lo + (uint64_t)me * NT + threadIdx.x; q < hi; q += (uint64_t)ctas * NT) {
        const uint4 v = t2[q];
        uint32_t h0, h1;
        b3_finish<true>(g, v.x, v.y, h0, h1);
        t2[q] = make_uint4(v.x, v.y, h0, h1);
    }
}

cudaError_t launch_t2_hash(const Desc *descs, int nplots, const uint32_t *tile_start,
                           uint32_t total_tiles, int chunk, cudaStream_t s)
{
    if (total_tiles == 0) return cudaSuccess;
    k_t2_hash<<<total_tiles, kT2HashThreads, 0, s>>>(descs, nplots, tile_start, chunk);
    return cudaGetLastError();
}

// Pair hash of the slot placement (Sec. III-A, Table 2): CTA b takes
// partitions [8b, 8b + 8) of one plot, whose pairs the sort left in the
// partitions' level-2 slots (pair k of partition f: key array of slot f
// for k < cap2, nonce array for k >= cap2) and whose Table-2 offsets the
// pair-count scan wrote; the CTA walks the group's pairs as one run, so
// every warp reads consecutive pairs and writes consecutive records.
__global__ void __launch_bounds__(kT2HashThreads) k_t2_hash_slots(const Desc *__restrict__ descs,
                                                                  int nplots,
                                                                  const uint32_t *__restrict__ tile_start)
{
    constexpr int NT = kT2HashThreads;
    constexpr uint32_t G = kT2SlotGroup;
    static_assert(G == 8, "the search below is written for groups of 8");
    __shared__ uint32_t s_rel[G + 1];  // pair offsets relative to the group's first
    __shared__ uint64_t s_base;
    const int plot = find_plot(tile_start, nplots, blockIdx.x);
    const Desc &d = descs[plot];
    if (*d.status & (kStT2Capacity | kStTimeout | kStBadTicket | kStPairSlot)) return;
    const uint64_t np = 1ull << d.p;
    const uint64_t fa = (uint64_t)(blockIdx.x - tile_start[plot]) * G;
    if (fa >= np) return;
    // The offsets exist only if the scan's chain reached its last chunk
    // (a broken chain has set a status bit, except for a withheld chunk 0
    // in a one-chunk scan).
    const uint64_t nchunks = (np + kScanChunk - 1) / kScanChunk;
    if ((ld_acquire_u64(d.lb + (nchunks - 1)) & ~kLbMask) != kLbIncl) return;
    const uint32_t ng = (uint32_t)(np - fa < G ? np - fa : G);
    if (threadIdx.x == 0) s_base = d.t2off[fa];
    __syncthreads();
    if (threadIdx.x <= G) {
        // partitions past the plot's last read as "never reached"
        s_rel[threadIdx.x] = threadIdx.x <= ng ? (uint32_t)(d.t2off[fa + threadIdx.x] - s_base)
                                               : 0xFFFFFFFFu;
    }
    __syncthreads();
    const uint32_t total = s_rel[ng];
    const uint32_t cap = d.cap2;
    if (s_base + total > d.t2cap) return;  // the scan flags this; never write past Table 2
    uint32_t g[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) g[i] = d.pre2[i];
    uint4 *__restrict__ t2 = reinterpret_cast<uint4 *>(d.t2) + s_base;
#pragma unroll 1
    for (uint32_t q = threadIdx.x; q < total; q += NT) {  // one compression per iteration
        // partition of pair q: the last t with s_rel[t] <= q
        uint32_t t = s_rel[4] <= q ? 4u : 0u;
        t += s_rel[t + 2] <= q ? 2u : 0u;
        t += s_rel[t + 1] <= q ? 1u : 0u;
        const uint32_t k = q - s_rel[t];
        const uint64_t f = fa + t;
        if (k >= cap + cap / 2u) break;  // past the pair slot (the sort flags this)
        const uint2 ab = k < cap ? reinterpret_cast<const uint2 *>(d.b_keys + f * cap)[k]
                                 : reinterpret_cast<const uint2 *>(d.b_nonces + f * cap)[k - cap];
        uint32_t h0, h1;
        b3_finish<true>(g, ab.x, ab.y, h0, h1);
        t2[q] = make_uint4(ab.x, ab.y, h0, h1);
    }
}

cudaError_t launch_t2_hash_slots(const Desc *descs, int nplots, const uint32_t *tile_start,
                                 uint32_t total_tiles, cudaStream_t s)
{
    if (total_tiles == 0) return cudaSuccess;
    k_t2_hash_slots<<<total_tiles, kT2HashThreads, 0, s>>>(descs, nplots, tile_start);
    return cudaGetLastError();
}

// ------------------------------------------------ tiled plots: windows
// The first pass of a tiled plot: the window (top c <= 8 bits of key64) of
// every nonce, one byte each; four nonces per thread and one 32-bit store.
__global__ void __launch_bounds__(256) k_window_ids(uint32_t k0, uint32_t k1, uint32_t k2,
                                                    uint32_t k3, uint32_t k4, uint32_t k5,
                                                    uint32_t k6, uint32_t k7, uint64_t N, int c,
                                                    uint32_t *__restrict__ ids4)
{
    const uint32_t key[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    uint32_t pre[16];
    b3_key_setup(key, 4u, pre);
    const uint64_t words = (N + 3) / 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += stride) {
        uint32_t packed = 0;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint64_t nonce = 4 * i + j;
            uint32_t h0, h1;
            b3_finish<false>(pre, (uint32_t)nonce, 0u, h0, h1);
            const uint32_t id = bswap32(h0) >> (32 - c);  // key64's top c bits
            packed |= (nonce < N ? id : 0u) << (8 * j);
        }
        ids4[i] = packed;
    }
}

cudaError_t launch_window_ids(const uint32_t key[8], uint64_t N, int c, uint8_t *ids, cudaStream_t s)
{
    if (N == 0 || c < 1 || c > 8) return cudaErrorInvalidValue;
    uint64_t blocks = ((N + 3) / 4 + 255) / 256;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_window_ids<<<(unsigned)blocks, 256, 0, s>>>(key[0], key[1], key[2], key[3], key[4], key[5],
                                                  key[6], key[7], N, c,
                                                  reinterpret_cast<uint32_t *>(ids));
    return cudaGetLastError();
}

// A window's nonces (wids[n] == win) listed into wlist in any order (the
// partition sort orders records by (key64, nonce)): each CTA reads 4096
// window ids, 16 per thread, ranks its matches with one block scan and
// claims their places with one atomic on wcount.  Entries past the list's
// capacity are dropped and reported.
constexpr int kListThreads = 256;
constexpr int kListPerThread = 16;

__global__ void __launch_bounds__(kListThreads) k_window_list(const Desc *__restrict__ dp, uint64_t N)
{
    __shared__ uint32_t ws[kListThreads / 32 + 1];
    __shared__ uint32_t s_base;
    const Desc &d = *dp;
    const uint64_t n0 = ((uint64_t)blockIdx.x * kListThreads + threadIdx.x) * kListPerThread;
    uint4 v = make_uint4(0u, 0u, 0u, 0u);
    if (n0 < N) v = *reinterpret_cast<const uint4 *>(d.wids + n0);  // ids rounded up to 16 bytes
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
    uint32_t match = 0;  // bit b: nonce n0 + b is in the window
#pragma unroll
    for (int b = 0; b < kListPerThread; ++b) {
        const bool m = n0 + b < N && ((w[b >> 2] >> (8 * (b & 3))) & 0xffu) == d.win;
        match |= (m ? 1u : 0u) << b;
    }
    uint32_t total;
    const uint32_t r = block_exclusive_scan_u32<kListThreads>((uint32_t)__popc(match), ws, &total);
    if (threadIdx.x == 0) s_base = total ? atomicAdd(d.wcount, total) : 0u;
    __syncthreads();
    uint32_t at = s_base + r;
    bool over = false;
    for (int b = 0; b < kListPerThread; ++b) {
        if (!(match >> b & 1u)) continue;
        if (at < d.listcap) d.wlist[at] = (uint32_t)(n0 + b);
        else over = true;
        ++at;
    }
    if (over) atomicOr(d.status, kStWinList);
}

cudaError_t launch_window_list(const Desc *desc, uint64_t N, cudaStream_t s)
{
    const uint64_t per = (uint64_t)kListThreads * kListPerThread;
    const uint64_t blocks = (N + per - 1) / per;
    if (blocks == 0 || blocks > 0x7FFFFFFFull) return cudaErrorInvalidValue;
    k_window_list<<<(unsigned)blocks, kListThreads, 0, s>>>(desc, N);
    return cudaGetLastError();
}

// --------------------------------------------------- stand-alone hashing
// Records {nonce, h0, h1} of nonces nonce0 .. nonce0+count-1, nonce order.
__global__ void __launch_bounds__(256) k_hash_records(uint32_t k0, uint32_t k1, uint32_t k2,
                                                      uint32_t k3, uint32_t k4, uint32_t k5,
                                                      uint32_t k6, uint32_t k7, uint64_t nonce0,
                                                      uint64_t count, uint32_t *__restrict__ out)
{
    const uint32_t key[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    uint32_t pre[16];
    b3_key_setup(key, 4u, pre);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint32_t nonce = (uint32_t)(nonce0 + i);
        uint32_t h0, h1;
        b3_finish<false>(pre, nonce, 0u, h0, h1);
        out[3 * i] = nonce;
        out[3 * i + 1] = h0;
        out[3 * i + 2] = h1;
    }
}

cudaError_t launch_hash_records(const uint32_t key[8], uint64_t nonce0, uint64_t count,
                                uint32_t *out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_hash_records<<<(unsigned)blocks, 256, 0, s>>>(key[0], key[1], key[2], key[3], key[4],
                                                      key[5], key[6], key[7], nonce0, count, out);
    return cudaGetLastError();
}

// Hash-only ceiling of the Table-1 hash: keyed BLAKE3 of nonces nonce0 ..
// nonce0 + count - 1 in the Table-1 kernel's shape (256 threads, 8 nonces
// per thread and step, key state from the per-key setup), with no record
// stores: each thread folds its hash words into one word, stored once.  It
// measures how fast the integer pipes run this instruction mix with no
// memory work beside it.  Grid-stride over tiles of 2048 nonces.
__global__ void __launch_bounds__(256) k_hash_peak(uint32_t k0, uint32_t k1, uint32_t k2,
                                                   uint32_t k3, uint32_t k4, uint32_t k5,
                                                   uint32_t k6, uint32_t k7, uint64_t nonce0,
                                                   uint64_t count, uint32_t *__restrict__ fold)
{
    constexpr int NPT = kHashNoncesPerThread;
    constexpr uint64_t T = (uint64_t)kHashThreads * NPT;
    const uint32_t key[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    uint32_t pre[16];
    b3_key_setup(key, 4u, pre);
    uint32_t acc = 0;
    const uint64_t tiles = (count + T - 1) / T;
    for (uint64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
#pragma unroll
        for (int j = 0; j < NPT; ++j) {
            const uint64_t i = t * T + (uint64_t)j * kHashThreads + threadIdx.x;
            uint32_t h0, h1;
            b3_finish<false>(pre, (uint32_t)(nonce0 + i), 0u, h0, h1);
            acc ^= i < count ? (h0 ^ h1) : 0u;
        }
    }
    fold[(uint64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

cudaError_t launch_hash_peak(const uint32_t key[8], uint64_t nonce0, uint64_t count, uint32_t *fold,
                             uint32_t blocks, cudaStream_t s)
{
    if (blocks == 0) return cudaErrorInvalidValue;
    k_hash_peak<<<blocks, kHashThreads, 0, s>>>(key[0], key[1], key[2], key[3], key[4], key[5],
                                                key[6], key[7], nonce0, count, fold);
    return cudaGetLastError();
}

// Table-2 records {a, b, g0, g1} of the pairs (a, b).
__global__ void __launch_bounds__(256) k_pair_hash(uint32_t k0, uint32_t k1, uint32_t k2,
                                                   uint32_t k3, uint32_t k4, uint32_t k5,
                                                   uint32_t k6, uint32_t k7,
                                                   const uint2 *__restrict__ pairs, uint64_t count,
                                                   uint4 *__restrict__ out)
{
    const uint32_t key[8] = {k0, k1, k2, k3, k4, k5, k6, k7};
    uint32_t pre[16];
    b3_key_setup(key, 8u, pre);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
        const uint2 ab = pairs[i];
        uint32_t g0, g1;
        b3_finish<true>(pre, ab.x, ab.y, g0, g1);
        out[i] = make_uint4(ab.x, ab.y, g0, g1);
    }
}

cudaError_t launch_pair_hash(const uint32_t key[8], const uint32_t *pairs, uint64_t count,
                             uint4 *out, cudaStream_t s)
{
    if (count == 0) return cudaSuccess;
    uint64_t blocks = (count + 255) / 256;
    if (blocks > 152ull * 64) blocks = 152ull * 64;
    k_pair_hash<<<(unsigned)blocks, 256, 0, s>>>(key[0], key[1], key[2], key[3], key[4], key[5],
                                                   key[6], key[7],
                                                   reinterpret_cast<const uint2 *>(pairs), count,
                                                   out);
    return cudaGetLastError();
}

}  // namespace vx
