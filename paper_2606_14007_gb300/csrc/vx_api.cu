// vx_api.cu -- host engine behind include/vaultx.h: the plot planner (how
// many physical partitions, slot capacities, buffer sizes), device-memory
// binding, the launch sequences of vx_table1 / vx_match, the batch path
// (grouped launches recorded into a CUDA graph), status mapping and the
// Table-2 file writer.
//
// Paper: Sec. III-A (pipeline: Table 1 in VRAM -> sort+match -> Table 2 ->
// D2H -> flat binary file in 4 MB chunks), Sec. III-B (pinned 256 MB
// staging buffer), Sec. III-C (allocation-size admission check).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include <cerrno>
#include <fcntl.h>
#include <unistd.h>

#include "../../include/vaultx.h"
#include "vx_internal.cuh"
#include "vx_plan.h"
#include "vx_engine.h"

using vx::Desc;
using vx::LaunchSet;

namespace vx {
static_assert(kPlanHashTile == (uint64_t)kHashTile, "planner and hash kernel tiles differ");
static_assert(kPlanScanChunk == (uint64_t)kScanChunk, "planner and scan kernel chunks differ");
static_assert(kPlanScatterTile == (uint64_t)kScatterTile, "planner and scatter kernel tiles differ");
static_assert(kPlanT2HashTile == kT2HashTile, "planner and pair-hash kernel tiles differ");
static_assert(kPlanT2SlotGroup == (uint64_t)kT2SlotGroup, "planner and slot pair-hash groups differ");
static_assert(kHashThreads == kPlanHashThreads && kHashNoncesPerThread == kPlanNoncesPerThread,
              "hash shape the planner accepts");
static_assert(kMatchThreads >= 256, "k_match loads a halo (<= 256 records) one per thread");
static_assert(sizeof(Desc) + 64 <= kStageTilesOffset, "descriptor overlaps staged tiles");
static_assert(kStageTilesOffset + kTileArrays * 2 * sizeof(uint32_t) <= kStageResultOffset &&
                  kStageResultOffset + 24 <= kStageBytes,
              "staged tiles overlap the result block");
int make_plan(int K, const vx_opts *o, Plan *pl, const char **why)
{
    int rc = make_plan_sized(K, o, pl, why, sizeof(Desc));
    if (rc != VX_OK) return rc;
    const uint32_t held = pl->cap2 + pl->hcap;  // a partition plus the next one's halo
    if (held > sortmatch_max_cap() || sortmatch_smem_bytes(held, pl->dbits) > kMaxSmemPerCta ||
        match_smem_bytes(held) > kMaxSmemPerCta) {
        *why = "partition slot too large for shared memory";
        return VX_EINVAL;
    }
    return VX_OK;
}
}  // namespace vx

namespace {

void forget_batches(vx_plot *p);  // drops cached batch graphs that use p
std::mutex g_mu;
int g_fail_allocs = 0;  // test hook: the next N device allocations fail

void set_err(vx_plot *p, const std::string &s)
{
    if (p) p->err = s;
}

int cuda_fail(vx_plot *p, const char *what, cudaError_t e)
{
    set_err(p, std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return VX_ECUDA;
}

#define VX_TRY(p, call)                                \
    do {                                               \
        cudaError_t e_ = (call);                       \
        if (e_ != cudaSuccess) return cuda_fail(p, #call, e_); \
    } while (0)

bool aligned(const void *ptr, size_t a) { return ((uintptr_t)ptr % a) == 0; }

void key_words(const uint8_t key[32], uint32_t w[8])
{
    for (int i = 0; i < 8; ++i)
        w[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) |
               ((uint32_t)key[4 * i + 2] << 16) | ((uint32_t)key[4 * i + 3] << 24);
}

cudaError_t dev_alloc(void **p, size_t bytes)
{
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_fail_allocs > 0) {
            --g_fail_allocs;
            *p = nullptr;
            return cudaErrorMemoryAllocation;
        }
    }
    return cudaMalloc(p, bytes);
}

void free_owned(vx_plot *p)
{
    if (p->owned) {
        cudaFree(p->d_t1);
        cudaFree(p->d_t2);
        cudaFree(p->d_scratch);
    }
    p->d_t1 = p->d_t2 = p->d_scratch = nullptr;
    p->owned = false;
    p->desc_dirty = true;
    p->stage = 0;
    p->t2_known = false;
    p->t1_known = false;
}

// Descriptor of a bound plot (host copy).
void fill_desc(const vx_plot *p, Desc *d)
{
    const vx::Plan &pl = p->plan;
    memset(d, 0, sizeof(*d));
    d->N = pl.N;
    d->D = pl.D;
    d->t2cap = p->t2cap;
    d->K = pl.K;
    d->p = pl.p;
    d->p1 = pl.p1;
    d->p2 = pl.p2;
    d->dbits = pl.dbits;
    d->cap1 = pl.cap1;
    d->cap2 = pl.cap2;
    d->chunks1 = pl.chunks1;
    d->spin_limit = pl.spin_limit;
    d->test_flags = pl.test_flags;
    d->hchunks = pl.hchunks;
    d->pchunks = pl.pchunks;
    d->scope = (uint32_t)pl.scope;
    d->hcap = pl.hcap;
    d->pk = pl.pk;
    d->wbits = pl.wbits;
    d->win = pl.win;
    if (p->wids && pl.wbits) {
        d->wids = p->wids;
        d->listcap = pl.listcap;
        d->wlist = reinterpret_cast<uint32_t *>(p->d_t2);  // free until the sort writes pairs
        d->wcount = reinterpret_cast<uint32_t *>(p->d_scratch + pl.o_wcount);
    }
    if (pl.p2 > 0) {
        d->a_keys = reinterpret_cast<uint64_t *>(p->d_t1);
        d->a_nonces = reinterpret_cast<uint32_t *>(p->d_t1 + pl.regionA_keys);
    }
    uint8_t *s = p->d_scratch;
    d->b_keys = reinterpret_cast<uint64_t *>(s + pl.o_regionB);
    d->b_nonces = reinterpret_cast<uint32_t *>(s + pl.o_regionB + pl.regionB_keys);
    d->status = reinterpret_cast<uint32_t *>(s + pl.o_status);
    d->cnt1 = reinterpret_cast<uint32_t *>(s + pl.o_cnt1);
    d->cnt2 = reinterpret_cast<uint32_t *>(s + pl.o_cnt2);
    d->t1off = reinterpret_cast<uint64_t *>(s + pl.o_t1off);
    d->pairs = reinterpret_cast<uint64_t *>(s + pl.o_pairs);
    d->t2off = reinterpret_cast<uint64_t *>(s + pl.o_t2off);
    d->lb = reinterpret_cast<uint64_t *>(s + pl.o_lb);
    d->ticket = reinterpret_cast<uint32_t *>(s + pl.o_ticket);
    d->lbs = reinterpret_cast<uint64_t *>(s + pl.o_lbs);
    d->ticket_s = reinterpret_cast<uint32_t *>(s + pl.o_ticket_s);
    if (pl.hcap) {
        d->halo_cnt = reinterpret_cast<uint32_t *>(s + pl.o_halo_cnt);
        d->halo_keys = reinterpret_cast<uint64_t *>(s + pl.o_halo_keys);
        d->halo_nonces = reinterpret_cast<uint32_t *>(s + pl.o_halo_nonces);
    }
    d->t1 = p->d_t1;
    d->t2 = p->d_t2;
    key_words(p->key, d->key);
}

Desc *dev_desc(vx_plot *p) { return reinterpret_cast<Desc *>(p->d_scratch + p->plan.o_desc); }
uint32_t *dev_tiles(vx_plot *p) { return reinterpret_cast<uint32_t *>(p->d_scratch + p->plan.o_tiles); }

// Tile prefixes (exclusive prefix of per-plot CTA counts) of every launch of
// a run over plots[0..n), written to h (host) for upload to d (device), and
// the launch set pointing at d.  Arrays of n + 1 entries in the order
// staged[8] direct[8] s2[8] pchunk[8] t2h[8] scan part.  Nonce chunk g and
// partition chunk c exist for a plot while g < its hchunks, c < its pchunks.
// Pair-hash grids follow the bound Table-2 capacity (a caller may bind a
// larger buffer than planned) and stride over their records.
int build_tiles(vx_plot *const *plots, int n, uint32_t *h, const uint32_t *d, LaunchSet *L)
{
    using namespace vx;
    const int W = n + 1;
    enum { A_STG = 0, A_DIR = 8, A_S2 = 16, A_PC = 24, A_T2H = 32, A_SCAN = 40, A_PART = 41 };
    static_assert(A_PART + 1 == vx::kTileArrays, "tile arrays");
    bool fuse = true, slots = true, halo = false, win = false, list = false;
    L->G = L->C = 1;
    L->max_cap2 = 0;
    L->max_dbits = 1;
    L->max_p2 = 0;
    int min_bits = 64;
    // One staged hash launch takes one shape: the plots' common nonces per
    // thread, else the default (any shape gives the same records).
    int npt = n > 0 && plots[0] ? plots[0]->plan.npt : kPlanNoncesPerThread;
    for (int i = 0; i < n; ++i)
        if (plots[i] && plots[i]->plan.npt != npt) npt = kPlanNoncesPerThread;
    for (int i = 0; i < n; ++i) {
        if (!plots[i] || !plots[i]->d_t1) return VX_EINVAL;
        const Plan &pl = plots[i]->plan;
        fuse = fuse && pl.fuse_pair_hash;
        slots = slots && pl.pair_slots;
        halo = halo || pl.scope != 0;
        win = win || pl.wbits != 0;
        if (plots[i]->wids && pl.wbits) {
            // a listed window runs alone, its hash in one nonce chunk
            if (n != 1 || pl.hchunks != 1) return VX_EINVAL;
            list = true;
        }
        L->G = std::max(L->G, pl.hchunks);
        L->C = std::max(L->C, pl.pchunks);
        L->max_cap2 = std::max(L->max_cap2, pl.cap2 + pl.hcap);
        L->max_dbits = std::max(L->max_dbits, pl.dbits);
        L->max_p2 = std::max(L->max_p2, pl.p2);
        if (pl.mode == kScatterStaged) min_bits = std::min(min_bits, pl.p2 > 0 ? pl.p1 : pl.p);
    }
    uint64_t acc[vx::kTileArrays] = {};
    for (int a = 0; a < vx::kTileArrays; ++a) h[a * W] = 0;
    for (int i = 0; i < n; ++i) {
        const Plan &pl = plots[i]->plan;
        uint64_t cnt[vx::kTileArrays] = {};
        const bool staged = pl.mode == kScatterStaged;
        for (int g = 0; g < vx::kMaxChunks && g < pl.hchunks; ++g) {
            cnt[(staged ? A_STG : A_DIR) + g] =
                list ? pl.tiles_list : staged ? vx::hash_tiles(pl.N / pl.hchunks, npt) : pl.tiles_hash;
            if (staged && pl.p2 > 0) cnt[A_S2 + g] = pl.tiles_s2;
        }
        const uint64_t np = 1ull << pl.p;
        for (int c = 0; c < vx::kMaxChunks && c < pl.pchunks; ++c) {
            cnt[A_PC + c] = np * (c + 1) / pl.pchunks - np * c / pl.pchunks;
            if (slots) {
                cnt[A_T2H + c] = pl.tiles_t2s;  // pchunks == 1
            } else if (!fuse) {
                const uint64_t per = (plots[i]->t2cap / pl.pchunks + kPlanT2HashTile - 1) / kPlanT2HashTile;
                cnt[A_T2H + c] = per ? per : 1;
            }
        }
        cnt[A_SCAN] = pl.tiles_scan;
        cnt[A_PART] = pl.tiles_part;
        for (int a = 0; a < vx::kTileArrays; ++a) {
            acc[a] += cnt[a];
            if (acc[a] > 0x7FFFFFFFull) return VX_EINVAL;
            h[a * W + i + 1] = (uint32_t)acc[a];
        }
    }
    L->n = n;
    L->agg = min_bits <= kAggMaxBits;
    L->npt = npt;
    L->fuse_pair_hash = fuse;
    L->pair_slots = slots;
    L->halo = halo;
    L->win = win;
    L->list = list;
    L->list_N = list ? plots[0]->plan.N : 0;
    for (int g = 0; g < vx::kMaxChunks; ++g) {
        L->t_staged[g] = d + (A_STG + g) * W;
        L->t_direct[g] = d + (A_DIR + g) * W;
        L->t_s2[g] = d + (A_S2 + g) * W;
        L->t_pchunk[g] = d + (A_PC + g) * W;
        L->t_t2h[g] = d + (A_T2H + g) * W;
        L->n_staged[g] = (uint32_t)acc[A_STG + g];
        L->n_direct[g] = (uint32_t)acc[A_DIR + g];
        L->n_s2[g] = (uint32_t)acc[A_S2 + g];
        L->n_pchunk[g] = (uint32_t)acc[A_PC + g];
        L->n_t2h[g] = (uint32_t)acc[A_T2H + g];
    }
    L->t_scan = d + A_SCAN * W;
    L->t_part = d + A_PART * W;
    L->n_scan = (uint32_t)acc[A_SCAN];
    L->n_part = (uint32_t)acc[A_PART];
    return VX_OK;
}

// Uploads the descriptor and the single-plot tile prefixes if they changed
// and caches the single-plot launch set.
int upload_desc(vx_plot *p, cudaStream_t s)
{
    if (!p->desc_dirty) return VX_OK;
    if (!p->h_stage) {
        void *h = nullptr;
        VX_TRY(p, cudaMallocHost(&h, vx::kStageBytes));
        p->h_stage = reinterpret_cast<Desc *>(h);
        VX_TRY(p, cudaEventCreateWithFlags(&p->ev_stage, cudaEventDisableTiming));
    }
    if (p->ev_pending) VX_TRY(p, cudaEventSynchronize(p->ev_stage));
    fill_desc(p, p->h_stage);
    uint32_t *t = reinterpret_cast<uint32_t *>(reinterpret_cast<uint8_t *>(p->h_stage) +
                                               vx::kStageTilesOffset);
    vx_plot *one[1] = {p};
    if (build_tiles(one, 1, t, dev_tiles(p), &p->single) != VX_OK) {
        set_err(p, "grid too large");
        return VX_EINVAL;
    }
    p->single.descs = dev_desc(p);
    // Only the host-filled part: pre1/pre2 are derived on the device by the
    // key-setup kernel and must survive a re-upload after vx_plot_bind.
    VX_TRY(p, cudaMemcpyAsync(dev_desc(p), p->h_stage, offsetof(Desc, pre1), cudaMemcpyHostToDevice, s));
    VX_TRY(p, cudaMemcpyAsync(dev_tiles(p), t, vx::kTileArrays * 2 * sizeof(uint32_t),
                              cudaMemcpyHostToDevice, s));
    VX_TRY(p, cudaEventRecord(p->ev_stage, s));
    p->ev_pending = true;
    p->desc_dirty = false;
    return VX_OK;
}

int ensure_memory(vx_plot *p)
{
    if (p->d_t1) return VX_OK;
    return vx_plot_alloc(p);
}

int map_status(uint32_t st)
{
    if (st & vx::kStTimeout) return VX_ETIMEDOUT;
    if (st & vx::kStBadTicket) return VX_ECUDA;
    if (st & (vx::kStSlot1Overflow | vx::kStSlot2Overflow | vx::kStCountMismatch |
              vx::kStPartitionTooBig | vx::kStPairSlot | vx::kStHaloOverflow | vx::kStSort2 |
              vx::kStWinList))
        return VX_EOVERFLOW;
    if (st & vx::kStT2Capacity) return VX_ENOMEM;
    return VX_OK;
}

std::string status_text(uint32_t st)
{
    std::string s;
    if (st & vx::kStSlot1Overflow) s += "first-level partition slot overflow; ";
    if (st & vx::kStSlot2Overflow) s += "second-level partition slot overflow; ";
    if (st & vx::kStCountMismatch) s += "records lost before the sort (count mismatch); ";
    if (st & vx::kStPartitionTooBig) s += "partition larger than shared memory; ";
    if (st & vx::kStT2Capacity) s += "Table 2 exceeds its capacity; ";
    if (st & vx::kStPairSlot) s += "a partition's pairs exceed its pair slot (use t2_placement 1); ";
    if (st & vx::kStHaloOverflow) s += "a partition's cross-bucket halo exceeds its capacity; ";
    if (st & vx::kStSort2) s += "sorting Table 2: a slot overflowed or records were lost; ";
    if (st & vx::kStWinList) s += "a window's nonce list exceeded its capacity; ";
    if (st & vx::kStTimeout) s += "device wait timed out; ";
    if (st & vx::kStBadTicket) s += "work ticket out of range (state not reset); ";
    return s;
}

// ----------------------------------------------------- kernel sequences
// Tracing ids (vx_kernel_name order).
enum { KID_SETUP = 0, KID_STAGED, KID_DIRECT, KID_S2, KID_SCAN, KID_SORT, KID_SCANP, KID_MATCH,
       KID_SORTMATCH, KID_PAIRHASH };

int tr_begin(const vx::Trace *T, int kid, cudaStream_t s)
{
    if (!T || *T->used >= vx::kProfLaunches) return -1;
    const int i = (*T->used)++;
    T->kid[i] = (int8_t)kid;
    cudaEventRecord(T->ev[2 * i], s);
    return i;
}

void tr_end(const vx::Trace *T, int i, cudaStream_t s)
{
    if (T && i >= 0) cudaEventRecord(T->ev[2 * i + 1], s);
}

#define VX_LAUNCH(kid, st, call)                 \
    do {                                         \
        const int i_ = tr_begin(T, kid, st);     \
        const cudaError_t e_ = (call);           \
        tr_end(T, i_, st);                       \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

// Key setup, hashing + bucketing, Table-1 offsets.  With an aux stream the
// second scatter level of nonce chunk g runs on it while chunk g+1 hashes.
cudaError_t launch_front(const LaunchSet &L, const vx::Lanes &ln, const vx::Trace *T)
{
    const cudaStream_t A = ln.main, B = ln.aux;
    VX_LAUNCH(KID_SETUP, A, vx::launch_key_setup(L.descs, L.n, A));
    if (L.list) {  // the window's nonces, listed from the window ids
        const cudaError_t e = vx::launch_window_list(L.descs, L.list_N, A);
        if (e != cudaSuccess) return e;
    }
    bool any_s2 = false;
    for (int g = 0; g < L.G; ++g) any_s2 = any_s2 || L.n_s2[g] > 0;
    const bool ov = B && L.G > 1 && any_s2;
    for (int g = 0; g < L.G; ++g) {
        if (L.n_staged[g])
            VX_LAUNCH(KID_STAGED, A, vx::launch_hash_scatter(L.descs, L.n, L.t_staged[g], L.n_staged[g],
                                                             vx::HashCfg{L.agg, L.halo, L.win, L.list, L.npt}, g, A));
        if (L.n_direct[g])
            VX_LAUNCH(KID_DIRECT, A, vx::launch_hash_direct(L.descs, L.n, L.t_direct[g], L.n_direct[g], g, A,
                                                            vx::HashCfg{L.agg, L.halo, L.win, L.list, L.npt}));
        if (L.n_s2[g]) {
            if (ov) {
                cudaEventRecord(ln.sync[g], A);
                cudaStreamWaitEvent(B, ln.sync[g], 0);
                VX_LAUNCH(KID_S2, B, vx::launch_scatter2(L.descs, L.n, L.t_s2[g], L.n_s2[g], g, B, L.halo,
                                                         L.max_p2));
            } else {
                VX_LAUNCH(KID_S2, A, vx::launch_scatter2(L.descs, L.n, L.t_s2[g], L.n_s2[g], g, A, L.halo,
                                                         L.max_p2));
            }
        }
    }
    if (ov) {
        cudaEventRecord(ln.sync[vx::kMaxChunks], B);
        cudaStreamWaitEvent(A, ln.sync[vx::kMaxChunks], 0);
    }
    VX_LAUNCH(KID_SCAN, A, vx::launch_scan_counts(L.descs, L.n, L.t_scan, L.n_scan, A));
    return cudaSuccess;
}

// Split path, Table 1: front + partition sort (Table 1 and pair counts).
cudaError_t launch_table1(const LaunchSet &L, const vx::Lanes &ln, const vx::Trace *T)
{
    const cudaError_t e = launch_front(L, ln, T);
    if (e != cudaSuccess) return e;
    const cudaStream_t A = ln.main;
    VX_LAUNCH(KID_SORT, A, vx::launch_sort(L.descs, L.n, L.t_part, L.n_part, A, L.max_cap2, L.max_dbits,
                                           L.halo));
    return cudaSuccess;
}

// Split path, Table 2: pair-offset scan + match.
cudaError_t launch_match_seq(const LaunchSet &L, cudaStream_t A, const vx::Trace *T)
{
    VX_LAUNCH(KID_SCANP, A, vx::launch_scan_pairs(L.descs, L.n, A));
    VX_LAUNCH(KID_MATCH, A, vx::launch_match(L.descs, L.n, L.t_part, L.n_part, A, L.max_cap2));
    return cudaSuccess;
}

// One-pass path: front, then sort + match per partition chunk (ticket order
// chains the chunks' Table-2 offsets), and the pair hash of chunk c on the
// aux stream while chunk c+1 sorts.
cudaError_t launch_fused(const LaunchSet &L, const vx::Lanes &ln, const vx::Trace *T)
{
    cudaError_t e = launch_front(L, ln, T);
    if (e != cudaSuccess) return e;
    const cudaStream_t A = ln.main, B = ln.aux_lo;
    if (L.pair_slots) {
        // slot placement: sort + match, pair-count scan, slot pair hash
        VX_LAUNCH(KID_SORTMATCH, A, vx::launch_sortmatch(L.descs, L.n, L.t_pchunk[0], L.n_pchunk[0], A,
                                                         L.max_cap2, L.max_dbits, vx::kOutSlots, L.halo));
        VX_LAUNCH(KID_SCANP, A, vx::launch_scan_pair_counts(L.descs, L.n, L.t_scan, L.n_scan, A));
        VX_LAUNCH(KID_PAIRHASH, A, vx::launch_t2_hash_slots(L.descs, L.n, L.t_t2h[0], L.n_t2h[0], A));
        return cudaSuccess;
    }
    const bool ph = !L.fuse_pair_hash;
    const bool ov = B && L.C > 1 && ph;
    for (int c = 0; c < L.C; ++c) {
        if (L.n_pchunk[c])
            VX_LAUNCH(KID_SORTMATCH, A, vx::launch_sortmatch(L.descs, L.n, L.t_pchunk[c], L.n_pchunk[c], A,
                                                             L.max_cap2, L.max_dbits,
                                                             L.fuse_pair_hash ? vx::kOutLookbackHashed
                                                                              : vx::kOutLookback,
                                                             L.halo));
        if (ph && L.n_t2h[c]) {
            if (ov) {
                cudaEventRecord(ln.sync[vx::kMaxChunks + 1 + c], A);
                cudaStreamWaitEvent(B, ln.sync[vx::kMaxChunks + 1 + c], 0);
                VX_LAUNCH(KID_PAIRHASH, B, vx::launch_t2_hash(L.descs, L.n, L.t_t2h[c], L.n_t2h[c], c, B));
            } else {
                VX_LAUNCH(KID_PAIRHASH, A, vx::launch_t2_hash(L.descs, L.n, L.t_t2h[c], L.n_t2h[c], c, A));
            }
        }
    }
    if (ov) {
        cudaEventRecord(ln.sync[2 * vx::kMaxChunks + 1], B);
        cudaStreamWaitEvent(A, ln.sync[2 * vx::kMaxChunks + 1], 0);
    }
    return cudaSuccess;
}

// Lanes of a single plot: its aux stream when its plan pipelines.
int plot_lanes(vx_plot *p, cudaStream_t s, vx::Lanes *ln)
{
    ln->main = s;
    ln->aux = ln->aux_lo = nullptr;
    ln->sync = p->sync_ev;
    if (p->plan.hchunks > 1 || p->plan.pchunks > 1) {
        if (!p->aux) VX_TRY(p, vx::make_lanes(&p->aux, &p->aux_lo, p->sync_ev));
        ln->aux = p->aux;
        ln->aux_lo = p->aux_lo;
    }
    return VX_OK;
}

// Trace of the plot's next run, if tracing is on and a slot is left.
vx::Trace *next_trace(vx_plot *p, vx::Trace *T)
{
    if (p->prof_slots <= 0 || p->prof_runs >= p->prof_slots) return nullptr;
    const int r = p->prof_runs;
    T->ev = p->prof_ev + (size_t)r * vx::kProfLaunches * 2;
    T->kid = p->prof_kid + (size_t)r * vx::kProfLaunches;
    T->used = p->prof_used + r;
    return T;
}

}  // namespace

// ================================================================ C ABI
extern "C" {

int vx_version(void) { return (1 << 16) | 0; }

int vx_opts_default(vx_opts *o)
{
    if (!o) return VX_EINVAL;
    memset(o, 0, sizeof(*o));
    o->size = sizeof(vx_opts);
    o->coarse_bits = -1;
    return VX_OK;
}

const char *vx_strerror(int st)
{
    switch (st) {
    case VX_OK: return "ok";
    case VX_EINVAL: return "invalid argument";
    case VX_ENOMEM: return "out of memory or Table-2 capacity exceeded";
    case VX_ECUDA: return "CUDA runtime error";
    case VX_ETIMEDOUT: return "device wait timed out";
    case VX_EBUSY: return "busy";
    case VX_ENOTREADY: return "not ready";
    case VX_EOVERFLOW: return "partition slot overflow";
    case VX_EIO: return "plot file I/O error";
    default: return "unknown status";
    }
}

const char *vx_last_error(const vx_plot *p) { return p ? p->err.c_str() : ""; }

int vx_plot_required_bytes(int K, const vx_opts *opts, uint64_t *t1, uint64_t *t2,
                           uint64_t *scratch)
{
    vx::Plan pl;
    const char *why = nullptr;
    if (vx::make_plan(K, opts, &pl, &why) != VX_OK) return VX_EINVAL;
    if (t1) *t1 = pl.t1_bytes;
    if (t2) *t2 = pl.t2_bytes;
    if (scratch) *scratch = pl.scratch_bytes;
    return VX_OK;
}

int vx_plot_create(int K, const uint8_t key[32], const vx_opts *opts, vx_plot **out)
{
    if (!out || !key) return VX_EINVAL;
    *out = nullptr;
    vx::Plan pl;
    const char *why = nullptr;
    if (vx::make_plan(K, opts, &pl, &why) != VX_OK) return VX_EINVAL;
    vx_plot *p = new (std::nothrow) vx_plot();
    if (!p) return VX_ENOMEM;
    p->K = K;
    memcpy(p->key, key, 32);
    if (opts) memcpy(&p->opts, opts, std::min<size_t>(sizeof(vx_opts), opts->size ? opts->size : sizeof(vx_opts)));
    else vx_opts_default(&p->opts);
    p->plan = pl;
    p->t2cap = pl.t2cap;
    *out = p;
    return VX_OK;
}

int vx_plot_bind(vx_plot *p, void *d_t1, void *d_t2, void *d_scratch, uint64_t t2_capacity)
{
    if (!p || !d_t1 || !d_t2 || !d_scratch) return VX_EINVAL;
    if (!aligned(d_t1, 256) || !aligned(d_t2, 256) || !aligned(d_scratch, 256)) {
        set_err(p, "bound buffers must be 256-byte aligned");
        return VX_EINVAL;
    }
    if (p->ev_pending) cudaEventSynchronize(p->ev_stage);
    // Re-binding only the Table-2 buffer (e.g. a larger one after VX_ENOMEM)
    // keeps a finished Table 1: vx_match may run again without vx_table1.
    const bool keep_t1 = !p->owned && p->d_t1 == (uint8_t *)d_t1 &&
                         p->d_scratch == (uint8_t *)d_scratch && p->stage >= 1;
    if (p->have_last) cudaStreamSynchronize(p->last);
    free_owned(p);
    if (keep_t1) p->stage = 1;
    p->d_t1 = (uint8_t *)d_t1;
    p->d_t2 = (uint8_t *)d_t2;
    p->d_scratch = (uint8_t *)d_scratch;
    p->owned = false;
    p->t2cap = t2_capacity ? t2_capacity : p->plan.t2cap;
    p->desc_dirty = true;
    return VX_OK;
}

int vx_plot_alloc(vx_plot *p)
{
    if (!p) return VX_EINVAL;
    if (p->d_t1) return VX_OK;
    void *a = nullptr, *b = nullptr, *c = nullptr;
    cudaError_t e = dev_alloc(&a, p->plan.t1_bytes);
    if (e == cudaSuccess) e = dev_alloc(&b, p->plan.t2_bytes);
    if (e == cudaSuccess) e = dev_alloc(&c, p->plan.scratch_bytes);
    if (e != cudaSuccess) {
        cudaFree(a);
        cudaFree(b);
        cudaFree(c);
        cudaGetLastError();
        set_err(p, std::string("device allocation failed: ") + cudaGetErrorName(e));
        return e == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA;
    }
    p->d_t1 = (uint8_t *)a;
    p->d_t2 = (uint8_t *)b;
    p->d_scratch = (uint8_t *)c;
    p->owned = true;
    p->t2cap = p->plan.t2cap;
    p->desc_dirty = true;
    return VX_OK;
}

int vx_table1(vx_plot *p, void *stream)
{
    if (!p) return VX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_memory(p);
    if (rc) return rc;
    if ((rc = upload_desc(p, s))) return rc;
    vx::Trace tr;
    const vx::Trace *T = next_trace(p, &tr);
    p->prof_cur = T ? p->prof_runs : -1;  // vx_match closes this traced run
    vx::Lanes ln{s, nullptr, nullptr, p->sync_ev};
    cudaError_t e = launch_table1(p->single, ln, T);
    if (e != cudaSuccess) return cuda_fail(p, "Table-1 launch", e);
    p->stage = 1;
    p->t2_known = false;
    p->t1_known = false;
    p->last = s;
    p->have_last = true;
    p->res_pending = false;
    return VX_OK;
}

int vx_match(vx_plot *p, void *stream)
{
    if (!p) return VX_EINVAL;
    if (p->stage < 1) {
        set_err(p, "vx_match before vx_table1");
        return VX_ENOTREADY;
    }
    cudaStream_t s = (cudaStream_t)stream;
    int rc = upload_desc(p, s);
    if (rc) return rc;
    vx::Trace tr;
    const vx::Trace *T = nullptr;
    if (p->prof_cur >= 0 && p->prof_cur == p->prof_runs) {
        T = next_trace(p, &tr);
        p->prof_runs += 1;
    }
    p->prof_cur = -1;
    cudaError_t e = launch_match_seq(p->single, s, T);
    if (e != cudaSuccess) return cuda_fail(p, "match launch", e);
    p->stage = 2;
    p->t2_known = false;
    p->t1_known = false;
    p->last = s;
    p->have_last = true;
    p->res_pending = false;
    return VX_OK;
}

namespace {
// Copies the plot's status word and Table-2 count into its pinned result
// block behind its kernels and records ev_done, so that vx_sync waits for
// this plot alone and reads what this plot produced, even when a plot
// queued later on the same stream reuses the scratch buffer.
int record_result(vx_plot *p, cudaStream_t s)
{
    uint8_t *h = reinterpret_cast<uint8_t *>(p->h_stage) + vx::kStageResultOffset;
    if (!p->ev_done) VX_TRY(p, cudaEventCreateWithFlags(&p->ev_done, cudaEventDisableTiming));
    VX_TRY(p, cudaMemcpyAsync(h, p->d_scratch + p->plan.o_status, 4, cudaMemcpyDeviceToHost, s));
    VX_TRY(p, cudaMemcpyAsync(h + 8, p->d_scratch + p->plan.o_t2off + 8 * (1ull << p->plan.p), 8,
                              cudaMemcpyDeviceToHost, s));
    VX_TRY(p, cudaMemcpyAsync(h + 16, p->d_scratch + p->plan.o_t1off + 8 * (1ull << p->plan.p), 8,
                              cudaMemcpyDeviceToHost, s));
    VX_TRY(p, cudaEventRecord(p->ev_done, s));
    p->res_pending = true;
    return VX_OK;
}
}  // namespace

int vx_plot_run(vx_plot *p, void *stream)
{
    if (!p) return VX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    int rc = ensure_memory(p);
    if (rc) return rc;
    if ((rc = upload_desc(p, s))) return rc;
    vx::Lanes ln;
    if ((rc = plot_lanes(p, s, &ln))) return rc;
    vx::Trace tr;
    const vx::Trace *T = next_trace(p, &tr);
    if (T) p->prof_runs += 1;
    p->prof_cur = -1;
    cudaError_t e = launch_fused(p->single, ln, T);
    if (e != cudaSuccess) return cuda_fail(p, "plot launch", e);
    p->stage = 2;
    p->t2_known = false;
    p->t1_known = false;
    p->last = s;
    p->have_last = true;
    p->res_pending = false;
    return record_result(p, s);
}

int vx_sync(vx_plot *p)
{
    if (!p) return VX_EINVAL;
    if (p->stage == 0) return VX_ENOTREADY;
    if (p->res_pending) {
        VX_TRY(p, cudaEventSynchronize(p->ev_done));
        const uint8_t *h = reinterpret_cast<const uint8_t *>(p->h_stage) + vx::kStageResultOffset;
        uint32_t st = 0;
        uint64_t total = 0, t1 = 0;
        memcpy(&st, h, 4);
        memcpy(&total, h + 8, 8);
        memcpy(&t1, h + 16, 8);
        p->status = st;
        p->t2_count = total;
        p->t2_known = true;
        p->t1_count = t1;
        p->t1_known = true;
        const int rc = map_status(st);
        if (rc != VX_OK) set_err(p, status_text(st));
        return rc;
    }
    if (p->have_last) VX_TRY(p, cudaStreamSynchronize(p->last));
    uint32_t st = 0;
    VX_TRY(p, cudaMemcpy(&st, p->d_scratch + p->plan.o_status, 4, cudaMemcpyDeviceToHost));
    p->status = st;
    if (p->stage >= 1) {
        uint64_t t1 = 0;
        VX_TRY(p, cudaMemcpy(&t1, p->d_scratch + p->plan.o_t1off + 8 * (1ull << p->plan.p), 8,
                             cudaMemcpyDeviceToHost));
        p->t1_count = t1;
        p->t1_known = true;
    }
    if (p->stage >= 2) {
        uint64_t total = 0;
        VX_TRY(p, cudaMemcpy(&total, p->d_scratch + p->plan.o_t2off + 8 * (1ull << p->plan.p), 8,
                             cudaMemcpyDeviceToHost));
        p->t2_count = total;
        p->t2_known = true;
    }
    const int rc = map_status(st);
    if (rc != VX_OK) set_err(p, status_text(st));
    return rc;
}

// --------------------------------------------------- sorted Table 2
namespace {
int sort2_plan(const vx_plot *p, vx::Sort2Plan *sp)
{
    if (p->stage < 2 || !p->t2_known || p->status != 0) return VX_ENOTREADY;
    if (vx::make_sort2_plan(p->t2_count, sp, sizeof(vx::Sort2Desc)) != VX_OK) return VX_EINVAL;
    return VX_OK;
}
}  // namespace

int vx_sort_table2_work_bytes(const vx_plot *p, uint64_t *bytes)
{
    if (!p || !bytes) return VX_EINVAL;
    vx::Sort2Plan sp;
    const int rc = sort2_plan(p, &sp);
    if (rc != VX_OK) return rc;
    *bytes = sp.bytes;
    return VX_OK;
}

int vx_sort_table2(vx_plot *p, void *d_work, uint64_t work_bytes, void *stream)
{
    if (!p || !d_work || ((uintptr_t)d_work % 256) != 0) return VX_EINVAL;
    vx::Sort2Plan sp;
    int rc = sort2_plan(p, &sp);
    if (rc != VX_OK) return rc;
    if (work_bytes < sp.bytes) {
        set_err(p, "work buffer smaller than vx_sort_table2_work_bytes");
        return VX_EINVAL;
    }
    if (p->t2_count == 0) return VX_OK;
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t *w = (uint8_t *)d_work;
    const vx::Plan &pl = p->plan;
    vx::Sort2Desc d;
    memset(&d, 0, sizeof(d));
    d.count = reinterpret_cast<const uint64_t *>(p->d_scratch + pl.o_t2off + 8 * (1ull << pl.p));
    d.p = sp.p;
    d.p1 = sp.p1;
    d.p2 = sp.p2;
    d.dbits = sp.dbits;
    d.cap1 = sp.cap1;
    d.cap2 = sp.cap2;
    d.chunks1 = sp.chunks1;
    d.spin_limit = pl.spin_limit;
    d.t2 = reinterpret_cast<uint4 *>(p->d_t2);
    d.a_keys = reinterpret_cast<uint64_t *>(w + sp.o_akeys);
    d.a_vals = reinterpret_cast<uint64_t *>(w + sp.o_avals);
    d.b_keys = reinterpret_cast<uint64_t *>(w + sp.o_bkeys);
    d.b_vals = reinterpret_cast<uint64_t *>(w + sp.o_bvals);
    d.cnt1 = reinterpret_cast<uint32_t *>(w + sp.o_cnt1);
    d.cnt2 = reinterpret_cast<uint32_t *>(w + sp.o_cnt2);
    d.off = reinterpret_cast<uint64_t *>(w + sp.o_off);
    d.lbs = reinterpret_cast<uint64_t *>(w + sp.o_lbs);
    d.ticket = reinterpret_cast<uint32_t *>(w + sp.o_ticket);
    d.status = reinterpret_cast<uint32_t *>(p->d_scratch + pl.o_status);
    vx::Sort2Desc *dd = reinterpret_cast<vx::Sort2Desc *>(w + sp.o_desc);
    VX_TRY(p, cudaMemcpyAsync(dd, &d, sizeof(d), cudaMemcpyHostToDevice, s));
    const vx::Sort2Launch g{sp.tiles1, sp.tiles2, sp.tiles_scan, sp.parts, sp.cap2, sp.dbits};
    cudaError_t e = vx::launch_sort2(dd, g, s);
    if (e != cudaSuccess) return cuda_fail(p, "sort Table 2", e);
    p->last = s;
    p->have_last = true;
    p->res_pending = false;
    return record_result(p, s);  // vx_sync now waits for the sort and reads its status
}

int vx_autotune(int K, const vx_opts *base, vx_opts *best, double *best_ms, void *stream)
{
    if (!best || K < 1 || K > 32) return VX_EINVAL;
    vx_opts b0;
    vx_opts_default(&b0);
    if (base) {
        if (base->size != 0 && base->size < sizeof(vx_opts)) return VX_EINVAL;
        memcpy(&b0, base, sizeof(b0));
        b0.size = sizeof(vx_opts);
    }
    cudaStream_t s = (cudaStream_t)stream;
    uint8_t key[32];
    for (int i = 0; i < 32; ++i) key[i] = (uint8_t)(0xA5 ^ (i * 7));
    struct Seen { int p, p1, p2, mode, npt; uint32_t cap2; int dbits; };
    std::vector<Seen> seen;
    double best_t = 0;
    bool found = false;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return VX_ECUDA;
    }
    // candidates: partition size x bucketing strategy x nonces per hash
    // thread (4, 8, 16 for the staged hash; the direct one takes 8)
    for (int part = 9; part <= 13; ++part) {
        for (int cand = 0; cand < 4; ++cand) {
            const uint32_t mode = cand < 3 ? (uint32_t)vx::kScatterStaged : (uint32_t)vx::kScatterDirect;
            vx_opts o = b0;
            o.partition_log2 = part;
            o.scatter_mode = mode;
            o.nonces_per_thread = cand == 0 ? 4u : cand == 2 ? 16u : 8u;
            vx::Plan pl;
            const char *why = nullptr;
            if (make_plan(K, &o, &pl, &why) != VX_OK) continue;
            const Seen me{pl.p, pl.p1, pl.p2, pl.mode, pl.npt, pl.cap2, pl.dbits};
            bool dup = false;
            for (const Seen &x : seen)
                dup = dup || (x.p == me.p && x.p1 == me.p1 && x.p2 == me.p2 && x.mode == me.mode &&
                              x.npt == me.npt && x.cap2 == me.cap2 && x.dbits == me.dbits);
            if (dup) continue;  // the planner clamped it to a plan already timed
            seen.push_back(me);
            vx_plot *p = nullptr;
            if (vx_plot_create(K, key, &o, &p) != VX_OK) continue;
            bool ok = vx_plot_alloc(p) == VX_OK && vx_plot_run(p, stream) == VX_OK &&
                      vx_sync(p) == VX_OK;
            float ms = 0;
            if (ok) {
                ok = cudaEventRecord(e0, s) == cudaSuccess;
                for (int r = 0; ok && r < 3; ++r) ok = vx_plot_run(p, stream) == VX_OK;
                ok = ok && cudaEventRecord(e1, s) == cudaSuccess && vx_sync(p) == VX_OK &&
                     cudaEventSynchronize(e1) == cudaSuccess &&
                     cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
            }
            vx_plot_destroy(p);
            if (!ok) {
                cudaGetLastError();  // a failed candidate (e.g. out of memory) is skipped
                continue;
            }
            const double t = ms / 3.0;
            if (!found || t < best_t) {
                found = true;
                best_t = t;
                *best = o;
                // report the partition size the planner actually used
                if (pl.p > 0) best->partition_log2 = K - pl.p;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (!found) return VX_ENOMEM;
    if (best_ms) *best_ms = best_t;
    return VX_OK;
}

int vx_table_info(const vx_plot *p, int which, const void **dptr, uint64_t *nrec,
                  uint32_t *rec_bytes)
{
    if (!p || (which != VX_TABLE1 && which != VX_TABLE2)) return VX_EINVAL;
    if (which == VX_TABLE1) {
        if (p->stage < 1) return VX_ENOTREADY;
        // A window's record count is known once vx_sync has read it.
        if (p->plan.wbits && !p->t1_known) return VX_ENOTREADY;
        if (dptr) *dptr = p->d_t1;
        if (nrec) *nrec = p->plan.wbits ? p->t1_count : p->plan.N;
        if (rec_bytes) *rec_bytes = 12;
        return VX_OK;
    }
    if (p->stage < 2 || !p->t2_known) return VX_ENOTREADY;
    if (dptr) *dptr = p->d_t2;
    if (nrec) *nrec = p->t2_count;
    if (rec_bytes) *rec_bytes = 16;
    return p->t2_count > p->t2cap ? VX_ENOMEM : VX_OK;
}

int vx_table1_offsets(vx_plot *p, void *d_out, void *stream)
{
    if (!p || !d_out || !aligned(d_out, 8)) return VX_EINVAL;
    if (p->stage < 1) return VX_ENOTREADY;
    int rc = upload_desc(p, (cudaStream_t)stream);
    if (rc) return rc;
    cudaError_t e = vx::launch_bucket_offsets(dev_desc(p), (uint64_t *)d_out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(p, "offsets launch", e);
    return VX_OK;
}

int vx_table_copy(vx_plot *p, int which, uint64_t offset, void *host_dst, uint64_t bytes,
                  void *stream)
{
    if (!p || !host_dst) return VX_EINVAL;
    const void *src = nullptr;
    uint64_t n = 0;
    uint32_t rb = 0;
    int rc = vx_table_info(p, which, &src, &n, &rb);
    if (rc != VX_OK) return rc;
    if (offset > n * rb || bytes > n * rb - offset) return VX_EINVAL;
    if (bytes == 0) return VX_OK;
    VX_TRY(p, cudaMemcpyAsync(host_dst, (const uint8_t *)src + offset, bytes, cudaMemcpyDeviceToHost,
                              (cudaStream_t)stream));
    return VX_OK;
}

void vx_plot_destroy(vx_plot *p)
{
    if (!p) return;
    forget_batches(p);
    if (p->res_pending)
        cudaEventSynchronize(p->ev_done);
    else if (p->have_last)
        cudaStreamSynchronize(p->last);
    if (p->ev_pending) cudaEventSynchronize(p->ev_stage);
    if (p->release) p->release(p->release_ctx, p);
    free_owned(p);
    if (p->h_stage) cudaFreeHost(p->h_stage);
    if (p->ev_stage) cudaEventDestroy(p->ev_stage);
    if (p->ev_done) cudaEventDestroy(p->ev_done);
    vx_plot_profile(p, 0);
    if (p->aux) vx::free_lanes(p->aux, p->aux_lo, p->sync_ev);
    delete p;
}

// -------------------------------------------------------------- tracing
const char *vx_kernel_name(int k)
{
    static const char *names[vx::kProfKernels] = {"key_setup",  "hash_staged", "hash_direct",
                                                  "scatter2",   "scan_counts", "sort",
                                                  "scan_pairs", "match",       "sortmatch",
                                                  "pairhash"};
    return (k >= 0 && k < vx::kProfKernels) ? names[k] : "";
}

int vx_plot_kernel_mask(const vx_plot *p, int split, uint32_t *mask)
{
    if (!p || !mask) return VX_EINVAL;
    const vx::Plan &pl = p->plan;
    uint32_t m = 1u << 0 | 1u << 4;                         // key_setup, scan_counts
    m |= pl.mode == vx::kScatterStaged ? 1u << 1 : 1u << 2;  // hash_staged / hash_direct
    if (pl.mode == vx::kScatterStaged && pl.p2 > 0) m |= 1u << 3;  // scatter2
    if (split) m |= 1u << 5 | 1u << 6 | 1u << 7;           // sort, scan_pairs, match
    else m |= 1u << 8 | (pl.fuse_pair_hash ? 0u : 1u << 9) |  // sortmatch, pairhash
              (pl.pair_slots ? 1u << 6 : 0u);                  // scan_pairs (pair-count scan)
    *mask = m;
    return VX_OK;
}

int vx_plot_profile(vx_plot *p, int runs)
{
    if (!p || runs < 0 || runs > 10000) return VX_EINVAL;
    if (p->prof_ev) {
        if (p->have_last) cudaStreamSynchronize(p->last);
        for (int i = 0; i < p->prof_slots * vx::kProfLaunches * 2; ++i) cudaEventDestroy(p->prof_ev[i]);
        delete[] p->prof_ev;
        delete[] p->prof_kid;
        delete[] p->prof_used;
        p->prof_ev = nullptr;
        p->prof_kid = nullptr;
        p->prof_used = nullptr;
    }
    p->prof_slots = p->prof_runs = 0;
    p->prof_cur = -1;
    if (runs == 0) return VX_OK;
    const size_t nev = (size_t)runs * vx::kProfLaunches * 2;
    p->prof_ev = new (std::nothrow) cudaEvent_t[nev]();
    p->prof_kid = new (std::nothrow) int8_t[(size_t)runs * vx::kProfLaunches];
    p->prof_used = new (std::nothrow) int[runs]();
    if (!p->prof_ev || !p->prof_kid || !p->prof_used) {
        delete[] p->prof_ev;
        delete[] p->prof_kid;
        delete[] p->prof_used;
        p->prof_ev = nullptr;
        p->prof_kid = nullptr;
        p->prof_used = nullptr;
        return VX_ENOMEM;
    }
    for (size_t i = 0; i < nev; ++i) {
        cudaError_t e = cudaEventCreate(&p->prof_ev[i]);
        if (e != cudaSuccess) {
            for (size_t j = 0; j < i; ++j) cudaEventDestroy(p->prof_ev[j]);
            delete[] p->prof_ev;
            delete[] p->prof_kid;
            delete[] p->prof_used;
            p->prof_ev = nullptr;
            p->prof_kid = nullptr;
            p->prof_used = nullptr;
            return cuda_fail(p, "cudaEventCreate", e);
        }
    }
    p->prof_slots = runs;
    return VX_OK;
}

int vx_plot_profile_read(vx_plot *p, double *ms, int cap, int *nkernels, int *nruns)
{
    if (!p || !ms || cap < vx::kProfKernels) return VX_EINVAL;
    for (int k = 0; k < vx::kProfKernels; ++k) ms[k] = 0.0;
    if (nkernels) *nkernels = vx::kProfKernels;
    if (nruns) *nruns = p->prof_runs;
    for (int r = 0; r < p->prof_runs; ++r) {
        const cudaEvent_t *ev = p->prof_ev + (size_t)r * vx::kProfLaunches * 2;
        const int8_t *kid = p->prof_kid + (size_t)r * vx::kProfLaunches;
        for (int i = 0; i < p->prof_used[r]; ++i) {
            VX_TRY(p, cudaEventSynchronize(ev[2 * i + 1]));
            float t = 0.f;
            VX_TRY(p, cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]));
            if (kid[i] >= 0 && kid[i] < vx::kProfKernels) ms[kid[i]] += t;
        }
    }
    return VX_OK;
}

// ------------------------------------------------------ stand-alone rows
int vx_hash_nonces(const uint8_t key[32], uint64_t nonce0, uint64_t count, void *d_out,
                   void *stream)
{
    if (!key || (!d_out && count) || !aligned(d_out, 4)) return VX_EINVAL;
    if (count > (1ull << 32) || nonce0 + count > (1ull << 32)) return VX_EINVAL;
    uint32_t w[8];
    key_words(key, w);
    cudaError_t e = vx::launch_hash_records(w, nonce0, count, (uint32_t *)d_out, (cudaStream_t)stream);
    return e == cudaSuccess ? VX_OK : VX_ECUDA;
}

int vx_hash_peak(const uint8_t key[32], uint64_t nonce0, uint64_t count, void *d_fold,
                 uint32_t fold_words, void *stream)
{
    if (!key || !d_fold || !aligned(d_fold, 4) || fold_words == 0 || fold_words % 256 != 0)
        return VX_EINVAL;
    if (count > (1ull << 32) || nonce0 + count > (1ull << 32)) return VX_EINVAL;
    uint32_t w[8];
    key_words(key, w);
    cudaError_t e = vx::launch_hash_peak(w, nonce0, count, (uint32_t *)d_fold, fold_words / 256,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? VX_OK : VX_ECUDA;
}

int vx_pair_hash(const uint8_t key[32], const void *d_pairs, uint64_t count, void *d_out,
                 void *stream)
{
    if (!key || ((!d_pairs || !d_out) && count) || !aligned(d_pairs, 8) || !aligned(d_out, 16))
        return VX_EINVAL;
    uint32_t w[8];
    key_words(key, w);
    cudaError_t e = vx::launch_pair_hash(w, (const uint32_t *)d_pairs, count, (uint4 *)d_out,
                                         (cudaStream_t)stream);
    return e == cudaSuccess ? VX_OK : VX_ECUDA;
}

// Test hook: the next `count` device allocations made by the library fail
// with cudaErrorMemoryAllocation (host-side fault injection).
int vx_test_fail_next_allocs(int count)
{
    std::lock_guard<std::mutex> lk(g_mu);
    g_fail_allocs = count < 0 ? 0 : count;
    return VX_OK;
}

}  // extern "C"

// ------------------------------------------------------------- batch
namespace {

// A batch's device workspace and its recorded graph, cached by the exact
// sequence of plot handles (and their buffers) it was built for.
struct BatchEntry {
    std::vector<vx_plot *> plots;
    std::vector<uint8_t *> bufs;
    uint8_t *d_ws = nullptr;
    uint8_t *h_ws = nullptr;
    size_t ws_bytes = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaStream_t aux = nullptr, aux_lo = nullptr;  // other branches of the recorded graph
    cudaEvent_t sync[vx::kSyncEvents] = {};
    // the second lane: its own stream and branches, and the fork / join
    cudaStream_t lane2 = nullptr, aux2 = nullptr, aux_lo2 = nullptr;
    cudaEvent_t sync2[vx::kSyncEvents] = {};
    cudaEvent_t fork = nullptr, join = nullptr;
};

std::mutex g_batch_mu;
std::vector<BatchEntry *> g_batches;

BatchEntry *find_batch(vx_plot *const *plots, int n)
{
    for (BatchEntry *b : g_batches) {
        if ((int)b->plots.size() != n) continue;
        bool same = true;
        for (int i = 0; i < n && same; ++i)
            same = b->plots[i] == plots[i] && b->bufs[i] == plots[i]->d_scratch;
        if (same) return b;
    }
    return nullptr;
}

void drop_batch(BatchEntry *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    vx::free_lanes(b->aux, b->aux_lo, b->sync);
    if (b->lane2) cudaStreamDestroy(b->lane2);
    vx::free_lanes(b->aux2, b->aux_lo2, b->sync2);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->join) cudaEventDestroy(b->join);
    cudaFree(b->d_ws);
    cudaFreeHost(b->h_ws);
    delete b;
}

}  // namespace

namespace vx {

void fill_desc_ext(const vx_plot *p, Desc *d) { fill_desc(p, d); }

int build_tiles_ext(vx_plot *const *plots, int n, uint32_t *h, const uint32_t *d, LaunchSet *L)
{
    return build_tiles(plots, n, h, d, L);
}

int map_status_ext(uint32_t st) { return map_status(st); }

size_t batch_ws_bytes(int n)
{
    const size_t o_tiles = ((size_t)n * sizeof(Desc) + 255) & ~(size_t)255;
    return o_tiles + (size_t)kTileArrays * (size_t)(n + 1) * 4;
}

int batch_prepare(vx_plot *const *plots, int n, uint8_t *h_ws, uint8_t *d_ws, LaunchSet *L)
{
    const size_t o_tiles = ((size_t)n * sizeof(Desc) + 255) & ~(size_t)255;
    Desc *hd = reinterpret_cast<Desc *>(h_ws);
    for (int i = 0; i < n; ++i) {
        if (!plots[i] || !plots[i]->d_t1) return VX_EINVAL;
        fill_desc(plots[i], hd + i);
    }
    const int rc = build_tiles(plots, n, reinterpret_cast<uint32_t *>(h_ws + o_tiles),
                               reinterpret_cast<const uint32_t *>(d_ws + o_tiles), L);
    L->descs = reinterpret_cast<Desc *>(d_ws);
    return rc;
}

cudaError_t launch_plot_seq(const LaunchSet &L, const Lanes &lanes)
{
    return launch_fused(L, lanes, nullptr);
}

cudaError_t make_lanes(cudaStream_t *aux, cudaStream_t *aux_lo, cudaEvent_t *sync)
{
    int lo = 0, hi = 0;  // numerically lower = higher priority
    cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(aux, cudaStreamNonBlocking, hi);
    if (e == cudaSuccess) e = cudaStreamCreateWithPriority(aux_lo, cudaStreamNonBlocking, lo);
    for (int i = 0; i < kSyncEvents && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&sync[i], cudaEventDisableTiming);
    return e;
}

void free_lanes(cudaStream_t aux, cudaStream_t aux_lo, cudaEvent_t *sync)
{
    if (aux) cudaStreamSynchronize(aux);
    if (aux_lo) cudaStreamSynchronize(aux_lo);
    for (int i = 0; i < kSyncEvents; ++i)
        if (sync[i]) cudaEventDestroy(sync[i]);
    if (aux) cudaStreamDestroy(aux);
    if (aux_lo) cudaStreamDestroy(aux_lo);
}

void mark_issued(vx_plot *const *plots, int n, cudaStream_t s)
{
    for (int i = 0; i < n; ++i) {
        vx_plot *p = plots[i];
        p->stage = 2;
        p->t2_known = false;
        p->t1_known = false;
        p->last = s;
        p->have_last = true;
        p->res_pending = false;
    }
}

int ensure_memory_ext(vx_plot *p) { return ensure_memory(p); }

}  // namespace vx

extern "C" int vx_plot_batch(vx_plot *const *plots, int n, void *stream)
{
    if (!plots || n <= 0) return VX_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < n; ++i) {
        if (!plots[i]) return VX_EINVAL;
        int rc = ensure_memory(plots[i]);
        if (rc) return rc;
    }
    std::lock_guard<std::mutex> lk(g_batch_mu);
    BatchEntry *b = find_batch(plots, n);
    if (!b) {
        b = new BatchEntry();
        b->plots.assign(plots, plots + n);
        for (int i = 0; i < n; ++i) b->bufs.push_back(plots[i]->d_scratch);
        // Two lanes of grouped launches, balanced by nonces (largest plots
        // first, each to the lighter lane), recorded on two branches of the
        // graph so that one lane's kernels can run beside the other's.
        std::vector<int> order(n);
        for (int i = 0; i < n; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return plots[x]->plan.N > plots[y]->plan.N; });
        std::vector<vx_plot *> lane[2];
        uint64_t load[2] = {0, 0};
        for (int i : order) {
            const int l = n >= 2 && load[1] < load[0] ? 1 : 0;
            lane[l].push_back(plots[i]);
            load[l] += plots[i]->plan.N;
        }
        const int nl = lane[1].empty() ? 1 : 2;
        const size_t ws0 = (vx::batch_ws_bytes((int)lane[0].size()) + 255) & ~(size_t)255;
        b->ws_bytes = ws0 + (nl == 2 ? vx::batch_ws_bytes((int)lane[1].size()) : 0);
        if (cudaMallocHost((void **)&b->h_ws, b->ws_bytes) != cudaSuccess ||
            dev_alloc((void **)&b->d_ws, b->ws_bytes) != cudaSuccess) {
            cudaGetLastError();
            drop_batch(b);
            return VX_ENOMEM;
        }
        LaunchSet L[2];
        for (int l = 0; l < nl; ++l) {
            const size_t at = l ? ws0 : 0;
            if (vx::batch_prepare(lane[l].data(), (int)lane[l].size(), b->h_ws + at, b->d_ws + at, &L[l]) !=
                VX_OK) {
                drop_batch(b);
                return VX_EINVAL;
            }
        }
        // The workspace is uploaded once; replays of the graph reuse it.
        cudaError_t e = cudaMemcpy(b->d_ws, b->h_ws, b->ws_bytes, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = vx::make_lanes(&b->aux, &b->aux_lo, b->sync);
        if (e == cudaSuccess && nl == 2) {
            e = cudaStreamCreateWithFlags(&b->lane2, cudaStreamNonBlocking);
            if (e == cudaSuccess) e = vx::make_lanes(&b->aux2, &b->aux_lo2, b->sync2);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join, cudaEventDisableTiming);
        }
        cudaGraph_t g = nullptr;
        if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = cudaSuccess;
            if (nl == 2) {
                e1 = cudaEventRecord(b->fork, b->cap_stream);
                if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(b->lane2, b->fork, 0);
            }
            if (e1 == cudaSuccess)
                e1 = vx::launch_plot_seq(L[0], vx::Lanes{b->cap_stream, b->aux, b->aux_lo, b->sync});
            if (e1 == cudaSuccess && nl == 2) {
                e1 = vx::launch_plot_seq(L[1], vx::Lanes{b->lane2, b->aux2, b->aux_lo2, b->sync2});
                if (e1 == cudaSuccess) e1 = cudaEventRecord(b->join, b->lane2);
                if (e1 == cudaSuccess) e1 = cudaStreamWaitEvent(b->cap_stream, b->join, 0);
            }
            e = cudaStreamEndCapture(b->cap_stream, &g);
            if (e == cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            drop_batch(b);
            for (int i = 0; i < n; ++i) set_err(plots[i], std::string("batch graph: ") + cudaGetErrorName(e));
            return VX_ECUDA;
        }
        g_batches.push_back(b);
        while (g_batches.size() > 16) {  // bounded cache
            drop_batch(g_batches.front());
            g_batches.erase(g_batches.begin());
        }
    }
    cudaError_t e = cudaGraphLaunch(b->exec, s);
    if (e != cudaSuccess) {
        for (int i = 0; i < n; ++i) set_err(plots[i], std::string("batch launch: ") + cudaGetErrorName(e));
        return VX_ECUDA;
    }
    vx::mark_issued(plots, n, s);
    return VX_OK;
}

namespace {
// Forgets cached batch graphs that reference plot p (called on destroy).
void forget_batches(vx_plot *p)
{
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (size_t i = 0; i < g_batches.size();) {
        BatchEntry *b = g_batches[i];
        if (std::find(b->plots.begin(), b->plots.end(), p) != b->plots.end()) {
            drop_batch(b);
            g_batches.erase(g_batches.begin() + i);
        } else {
            ++i;
        }
    }
}
}  // namespace

// --------------------------------------------------------- file write
namespace {
std::mutex g_stage_mu;
uint8_t *g_stage = nullptr;      // pinned staging, two halves
cudaStream_t g_copy_stream = nullptr;
cudaEvent_t g_copy_ev[2] = {nullptr, nullptr};
}  // namespace

namespace vx {

// Appends plot p's Table 2 (synced) to the open file fd through the pinned
// staging buffer: double-buffered half-buffer copies on the library's copy
// stream, each written as sequential 4 MB chunks.  *d2h (may be null) gets
// the seconds spent waiting for copies.  VX_OK, VX_ECUDA or VX_EIO (a
// failed write, errno text on p).
int write_table2_fd(vx_plot *p, int fd, double *d2h_out)
{
    const void *src = nullptr;
    uint64_t nrec = 0;
    uint32_t rb = 0;
    int rc = vx_table_info(p, VX_TABLE2, &src, &nrec, &rb);
    if (rc != VX_OK) return rc;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    if (!g_stage) {
        VX_TRY(p, cudaMallocHost((void **)&g_stage, vx::kWriteStageBytes));
        VX_TRY(p, cudaStreamCreateWithFlags(&g_copy_stream, cudaStreamNonBlocking));
        VX_TRY(p, cudaEventCreateWithFlags(&g_copy_ev[0], cudaEventDisableTiming));
        VX_TRY(p, cudaEventCreateWithFlags(&g_copy_ev[1], cudaEventDisableTiming));
    }
    const uint64_t total = nrec * rb;
    const uint64_t half = vx::kWriteStageBytes / 2;
    double d2h = 0;
    uint64_t done = 0;
    int slot = 0;
    // Double buffering: copy block k+1 while block k is written.
    uint64_t pending_bytes[2] = {0, 0};
    auto issue = [&](int sl, uint64_t at) -> cudaError_t {
        const uint64_t n = std::min(half, total - at);
        pending_bytes[sl] = n;
        cudaError_t e = cudaMemcpyAsync(g_stage + sl * half, (const uint8_t *)src + at, n,
                                        cudaMemcpyDeviceToHost, g_copy_stream);
        if (e == cudaSuccess) e = cudaEventRecord(g_copy_ev[sl], g_copy_stream);
        return e;
    };
    bool ok = true;
    int werr = 0;  // errno of a failed write
    if (total > 0) {
        if (issue(0, 0) != cudaSuccess) ok = false;
        uint64_t next = std::min(half, total);
        while (ok && done < total) {
            const auto c0 = std::chrono::steady_clock::now();
            if (cudaEventSynchronize(g_copy_ev[slot]) != cudaSuccess) { ok = false; break; }
            d2h += std::chrono::duration<double>(std::chrono::steady_clock::now() - c0).count();
            if (next < total) {
                if (issue(slot ^ 1, next) != cudaSuccess) { ok = false; break; }
                next += pending_bytes[slot ^ 1];
            }
            const uint8_t *buf = g_stage + slot * half;
            uint64_t left = pending_bytes[slot];
            while (left > 0 && ok) {   // sequential 4 MB writes
                const size_t chunk = (size_t)std::min<uint64_t>(left, vx::kWriteChunkBytes);
                ssize_t w = ::write(fd, buf, chunk);
                if (w <= 0) {
                    werr = w < 0 ? errno : ENOSPC;
                    ok = false;
                    break;
                }
                buf += w;
                left -= (uint64_t)w;
            }
            done += pending_bytes[slot];
            slot ^= 1;
        }
    }
    cudaStreamSynchronize(g_copy_stream);
    if (!ok) {
        if (werr) {
            set_err(p, std::string("Table-2 write failed: ") + strerror(werr));
            return VX_EIO;
        }
        set_err(p, "Table-2 copy to the staging buffer failed");
        return VX_ECUDA;
    }
    if (d2h_out) *d2h_out = d2h;
    return VX_OK;
}

}  // namespace vx

extern "C" int vx_plot_write(vx_plot *p, const char *path, double *sec_d2h, double *sec_total)
{
    if (!p || !path) return VX_EINVAL;
    int rc = vx_sync(p);
    if (rc != VX_OK) return rc;
    const auto t0 = std::chrono::steady_clock::now();
    int fd = open(path, O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (fd < 0) {
        set_err(p, std::string("cannot open ") + path + ": " + strerror(errno));
        return VX_EIO;
    }
    double d2h = 0;
    rc = vx::write_table2_fd(p, fd, &d2h);
    if (close(fd) != 0 && rc == VX_OK) {  // deferred write-back errors surface here
        set_err(p, std::string("closing ") + path + ": " + strerror(errno));
        rc = VX_EIO;
    }
    if (rc != VX_OK) return rc;
    if (sec_d2h) *sec_d2h = d2h;
    if (sec_total) *sec_total = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return VX_OK;
}
