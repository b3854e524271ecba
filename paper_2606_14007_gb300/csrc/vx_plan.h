// vx_plan.h -- the plot planner: from (K, options) to partition counts, slot
// capacities, buffer sizes and kernel grid sizes.  Host only, no CUDA calls,
// so it can be checked on a machine without a GPU.
//
// Paper basis: Table 1 has 2^K records in 2^24 buckets (Sec. I-A, III-B);
// the paper's per-bucket capacity RPB (Sec. III-B) is replaced by physical
// partitions (runs of 2^(24-p) whole logical buckets) with Poisson-sized
// slots; Table 2 gets a capacity from the expected pair count.
#pragma once

#include <cmath>
#include <cstdint>
#include <cstring>
#include <string>

#include "../../include/vaultx.h"

namespace vx {

constexpr int kDefaultPartLog2 = 11;       // mean records per physical partition: 2048
constexpr int kSort2PartLog2 = 10;         // the same for the sort of Table 2 by hash2
constexpr uint32_t kDefaultSlackSigma = 12;
constexpr int kMaxPartBits = 21;           // scatter levels of <= 10 and <= 11 bits
constexpr int kAggMaxBits = 6;             // warp-aggregate ranks up to 64 bins
constexpr size_t kStageBytes = 4096;       // pinned staging: Desc + tile prefixes
constexpr size_t kStageTilesOffset = 3584;
constexpr size_t kStageResultOffset = 4064;  // status u32 at +0, Table-2 count u64 at +8
constexpr uint64_t kWriteStageBytes = 256ull << 20;  // Sec. III-B: 256 MB pinned staging
constexpr uint64_t kWriteChunkBytes = 4ull << 20;    // Sec. III-A: 4 MB sequential chunks
constexpr uint64_t kPlanHashTile = 2048;   // nonces per hash CTA (threads x nonces/thread)
constexpr int kPlanHashThreads = 256;      // threads per hash CTA
constexpr int kPlanNoncesPerThread = 8;    // default nonces per hash thread

// Table-1 hash CTAs over n nonces with npt nonces per thread.
inline uint32_t hash_tiles(uint64_t n, int npt)
{
    const uint64_t tile = (uint64_t)kPlanHashThreads * (uint64_t)npt;
    return (uint32_t)((n + tile - 1) / tile);
}
constexpr uint64_t kPlanScanChunk = 4096;  // counters per Table-1 offset-scan CTA
constexpr uint64_t kPlanScatterTile = 4096; // records per second-level scatter CTA
constexpr uint64_t kPlanT2HashTile = 2048; // Table-2 records per pair-hash CTA
constexpr uint64_t kPlanS2Tile1 = 4096;    // Table-2 records per first-level CTA of the sort by hash2
constexpr uint64_t kPlanT2SlotGroup = 8;   // partitions per pair-hash CTA reading pair slots

enum { kScatterAuto = 0, kScatterStaged = 1, kScatterDirect = 2 };
enum { kPlaceAuto = 0, kPlaceLookback = 1, kPlaceSlots = 2 };

struct Plan {
    int K, s, p, p1, p2, dbits;
    int pk;                                // partition bits in key space: p + wbits
    uint32_t wbits, win;                   // window: top wbits of key64 == win (wbits 0: whole plot)
    int mode;                              // kScatterStaged or kScatterDirect
    int npt;                               // nonces per thread of the Table-1 hash (4, 8, 16)
    uint32_t test_flags, spin_limit;
    bool fuse_pair_hash;
    bool pair_slots;                       // pairs staged in the partition slots (t2_placement 2)
    int scope;                             // 0 bucket-scope match, 1 cross-bucket
    uint32_t hcap;                         // halo records per partition (scope 1, p > 0)
    int hchunks;                           // nonce chunks of the hash / second-scatter pipeline
    int pchunks;                           // partition chunks of the sort / pair-hash pipeline
    uint64_t N, D, t2cap;
    uint32_t cap1, cap2, chunks1;
    bool agg;
    uint32_t tiles_hash, tiles_s2, tiles_part;
    uint32_t tiles_staged, tiles_direct;   // tiles_hash of the kernel the mode uses, 0 for the other
    uint32_t tiles_scan, tiles_t2h;        // Table-1 offset scan chunks, pair-hash CTAs
    uint32_t tiles_t2s;                    // pair-hash CTAs reading pair slots
    uint32_t listcap, tiles_list;          // window nonce list: capacity, hash CTAs over it
    uint64_t regionA_keys, regionB_keys;   // byte offset of the nonce array in each slot region
    uint64_t regionA_bytes, regionB_bytes;
    uint64_t t1_bytes, t2_bytes, scratch_bytes;
    uint64_t o_status, o_ticket, o_ticket_s, o_cnt1, o_cnt2, o_t1off, o_pairs, o_t2off, o_lb, o_lbs,
        o_desc, o_tiles;
    uint64_t o_regionB;                    // final-partition slots (scratch buffer)
    uint64_t o_halo_cnt, o_halo_keys, o_halo_nonces;  // scope 1 halos (scratch buffer)
    uint64_t o_wcount;                     // window nonce list entry counter (scratch buffer)
};

inline uint64_t round_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Capacity of a slot expecting `avg` records (Poisson): avg + slack * sd,
// rounded up to a multiple of 4 records.
inline uint64_t slot_capacity(double avg, uint32_t slack)
{
    return round_up((uint64_t)std::ceil(avg + slack * std::sqrt(avg) + 16.0), 4);
}

// Expected Table-2 pairs: 2^24 buckets of Poisson(lambda) records, key64
// uniform over a bucket of width 2^40; a pair matches with probability
// 2u - u^2 (u = D / 2^40, all pairs when u >= 1).
inline double expected_pairs(uint64_t N, uint64_t D)
{
    const double lam = (double)N / 16777216.0;
    const double u = (double)D / 1099511627776.0;
    const double q = u >= 1.0 ? 1.0 : 2.0 * u - u * u;
    return 16777216.0 * lam * lam / 2.0 * q;
}

// Expected pairs of the cross-bucket match: N uniform key64 values, a pair
// within D with probability 2u - u^2, u = D / 2^64.
inline double expected_pairs_global(uint64_t N, uint64_t D)
{
    const double u = (double)D / 18446744073709551616.0;
    const double q = u >= 1.0 ? 1.0 : 2.0 * u - u * u;
    return (double)N * ((double)N - 1.0) / 2.0 * q;
}

inline int make_plan_sized(int K, const vx_opts *o, Plan *pl, const char **why, size_t desc_bytes)
{
    if (K < 1 || K > 32) {
        *why = "K must be in 1..32";
        return VX_EINVAL;
    }
    vx_opts opts;
    memset(&opts, 0, sizeof(opts));
    opts.coarse_bits = -1;
    if (o) {
        if (o->size != 0 && o->size < sizeof(vx_opts)) {
            *why = "vx_opts.size too small";
            return VX_EINVAL;
        }
        memcpy(&opts, o, sizeof(opts));
    }
    Plan P;
    memset(&P, 0, sizeof(P));
    P.K = K;
    P.N = 1ull << K;
    P.D = opts.match_distance ? opts.match_distance : (1ull << (64 - K));
    P.s = opts.partition_log2 ? opts.partition_log2 : kDefaultPartLog2;
    if (P.s < 6 || P.s > 13) {
        *why = "partition_log2 must be in 6..13";
        return VX_EINVAL;
    }
    const uint32_t slack = opts.slack_sigma ? opts.slack_sigma : kDefaultSlackSigma;
    if (opts.test_flags & ~1u) {
        *why = "unknown test_flags bit";
        return VX_EINVAL;
    }
    P.test_flags = opts.test_flags;
    for (int i = 0; i < 2; ++i)
        if (opts.reserved[i]) {
            *why = "reserved vx_opts fields must be zero";
            return VX_EINVAL;
        }
    // The hash kernels run 256 threads per CTA with 8 nonces per thread;
    // the plain staged Table-1 hash is also compiled for 4 and 16.
    if ((opts.hash_block != 0 && opts.hash_block != 256) ||
        (opts.nonces_per_thread != 0 && opts.nonces_per_thread != 4 && opts.nonces_per_thread != 8 &&
         opts.nonces_per_thread != 16)) {
        *why = "hash_block must be 0 or 256 and nonces_per_thread 0, 4, 8 or 16";
        return VX_EINVAL;
    }
    P.npt = opts.nonces_per_thread ? (int)opts.nonces_per_thread : kPlanNoncesPerThread;
    P.fuse_pair_hash = opts.fuse_pair_hash != 0;
    const uint32_t pc = opts.pipeline_chunks;
    if (pc != 0 && pc != 1 && pc != 2 && pc != 4 && pc != 8) {
        *why = "pipeline_chunks must be 0, 1, 2, 4 or 8";
        return VX_EINVAL;
    }
    // ~1 us per poll: ~4 s in normal use (never reached unless a partition
    // fails to publish), ~4 ms when a test withholds a prefix on purpose.
    P.spin_limit = opts.test_flags ? (1u << 12) : (1u << 22);
    P.p = K - P.s;
    if (P.p < 0) P.p = 0;
    if (P.p > kMaxPartBits) P.p = kMaxPartBits;
    // A window keeps the 2^(p - c) partitions whose top c key bits are its
    // index; every shift into the key uses pk = p, every array 2^(p - c).
    P.pk = P.p;
    P.wbits = opts.window_bits;
    P.win = opts.window;
    if (P.wbits > 16 || (int)P.wbits > P.p) {
        *why = "window_bits must be at most 16 and at most the partition bits K - partition_log2";
        return VX_EINVAL;
    }
    if (P.win >> P.wbits) {
        *why = "window must be below 2^window_bits";
        return VX_EINVAL;
    }
    if (P.wbits && opts.match_scope != 0) {
        *why = "window_bits needs match_scope 0 (a window holds no halo of the next one)";
        return VX_EINVAL;
    }
    P.p -= (int)P.wbits;
    if (opts.scatter_mode > kScatterDirect) {
        *why = "scatter_mode must be 0 (auto), 1 (staged) or 2 (direct)";
        return VX_EINVAL;
    }
    // Automatic = staged: on GB300 the per-record slot claims of the direct
    // strategy cost more L2 atomic throughput than the second scatter pass.
    P.mode = opts.scatter_mode == kScatterDirect ? kScatterDirect : kScatterStaged;
    if (P.npt != kPlanNoncesPerThread && (P.mode != kScatterStaged || P.wbits)) {
        *why = "nonces_per_thread 4 or 16 needs the staged bucketing and a whole plot (no window)";
        return VX_EINVAL;
    }
    if (P.mode == kScatterDirect) {
        P.p1 = P.p;  // one level: the hash kernel claims final-partition slots
    } else if (opts.coarse_bits >= 0) {
        P.p1 = opts.coarse_bits < P.p ? opts.coarse_bits : P.p;
    } else {
        P.p1 = P.p <= 10 ? P.p : P.p / 2;
    }
    P.p2 = P.p - P.p1;
    if (P.mode == kScatterStaged && (P.p1 > 10 || P.p2 > 11)) {
        *why = "coarse_bits leaves a scatter level wider than 10 (first) or 11 (second) bits";
        return VX_EINVAL;
    }
    // Pipeline chunks, only where a second kernel exists to overlap (the
    // second scatter level; the separate pair hash).  Off unless asked for:
    // measured on GB300 at K=31 it does not pay, because each kernel of a
    // pair alone fills an SM's register file (the latency-bound sort needs
    // four resident CTAs, the ALU-bound hashes need ~24 warps), so the two
    // streams take turns instead of sharing SMs.
    const int want = pc == 0 ? 1 : (int)pc;
    P.hchunks = (P.mode == kScatterStaged && P.p2 > 0) ? want : 1;
    while (P.hchunks > 1 && ((1ull << K) < (uint64_t)P.hchunks)) P.hchunks >>= 1;
    P.pchunks = P.fuse_pair_hash ? 1 : want;
    while (P.pchunks > 1 && (1ull << P.p) < (uint64_t)P.pchunks) P.pchunks >>= 1;
    // Records of the plot (of the window: Binomial(2^K, 2^-c), Poisson-like).
    const double wrec = std::ldexp((double)P.N, -(int)P.wbits);
    const double avg2 = std::ldexp((double)P.N, -P.pk);
    uint64_t cap2 = (P.pk == 0) ? round_up(P.N, 4) : slot_capacity(avg2, slack);
    if (cap2 > round_up(P.N, 4)) cap2 = round_up(P.N, 4);
    if (cap2 > 16384) {
        *why = "partition slot larger than the sort's shared-memory capacity";
        return VX_EINVAL;
    }
    P.cap2 = (uint32_t)cap2;
    if (P.p2 > 0) {
        const double avg1 = wrec / (double)P.hchunks / (double)(1ull << P.p1);
        // One level-1 bin of a whole plot holds every record: exact.
        uint64_t cap1 = (P.p1 == 0 && !P.wbits) ? round_up(P.N, 4) : slot_capacity(avg1, slack);
        if (cap1 > round_up(P.N / P.hchunks, 4)) cap1 = round_up(P.N / P.hchunks, 4);
        if (cap1 > 0xFFFFFF00ull) {
            *why = "first-level slot too large";
            return VX_EINVAL;
        }
        P.cap1 = (uint32_t)cap1;
        P.chunks1 = (uint32_t)((cap1 + kPlanScatterTile - 1) / kPlanScatterTile);
    }
    int db = K - P.pk;
    if (db < 1) db = 1;
    if (db > 13) db = 13;
    P.dbits = db;
    P.agg = (P.p2 > 0 ? P.p1 : P.p) <= kAggMaxBits;

    // Table-2 placement: look-back (pairs at their final offsets, each
    // partition waiting for the pair counts of the ones before it) or slots
    // (pairs staged in the partition's own slot, no waits, a scan and the
    // slot pair hash place them).  Automatic takes the slots whenever a
    // partition's pairs fit its pair slot with a wide margin (decided below,
    // once the expected pair count is known): the slots move 8 bytes per
    // pair less each way and the sort never waits on another partition.
    if (opts.t2_placement > kPlaceSlots) {
        *why = "t2_placement must be 0 (auto), 1 (look-back) or 2 (slots)";
        return VX_EINVAL;
    }
    if (opts.t2_placement == kPlaceSlots && (P.fuse_pair_hash || P.pchunks != 1)) {
        *why = "t2_placement 2 (slots) needs fuse_pair_hash 0 and pipeline_chunks 0 or 1";
        return VX_EINVAL;
    }
    P.pair_slots = opts.t2_placement == kPlaceSlots;

    // Cross-bucket match: partition f's pairs reach into partition f + 1
    // only (D at most one partition wide), through the records of f + 1
    // within D of its lower edge, Poisson with mean avg2 * D / 2^(64-p).
    if (opts.match_scope > 1) {
        *why = "match_scope must be 0 (bucket) or 1 (cross-bucket)";
        return VX_EINVAL;
    }
    P.scope = (int)opts.match_scope;
    P.hcap = 0;
    if (P.scope == 1 && P.p > 0) {  // wbits == 0 here: p == pk
        const double W = std::ldexp(1.0, 64 - P.p);
        if ((double)P.D > W) {
            *why = "match_scope 1 needs match_distance <= 2^(64-p), one partition";
            return VX_EINVAL;
        }
        const uint64_t hc = slot_capacity(avg2 * (double)P.D / W, slack);
        if (hc > 256) {
            *why = "match_scope 1: match distance gives a halo of more than 256 records";
            return VX_EINVAL;
        }
        P.hcap = (uint32_t)hc;
    }

    const double E = (P.scope ? expected_pairs_global(P.N, P.D) : expected_pairs(P.N, P.D)) /
                     std::ldexp(1.0, (int)P.wbits);
    if (opts.t2_capacity) {
        P.t2cap = opts.t2_capacity;
    } else {
        P.t2cap = round_up((uint64_t)std::ceil(E + 24.0 * std::sqrt(E) + 4096.0), 256);
    }
    if (opts.t2_placement == kPlaceAuto && !P.fuse_pair_hash && P.pchunks == 1) {
        // A partition's pairs sum over its buckets' pairs, more spread than
        // Poisson: the margin takes 12 sigma of a variance four times the mean.
        const double Ep = E / std::ldexp(1.0, P.p);
        P.pair_slots = Ep + 12.0 * std::sqrt(4.0 * Ep) + 64.0 <= (double)(P.cap2 + P.cap2 / 2u);
    }
    // Grids (tile sizes are the kernels' compile-time tiles).
    // Grids per chunk (a chunk of the hash covers 2^K / hchunks nonces).
    P.tiles_hash = hash_tiles(P.N / P.hchunks, P.npt);
    P.tiles_staged = P.mode == kScatterStaged ? P.tiles_hash : 0u;
    P.tiles_direct = P.mode == kScatterDirect ? P.tiles_hash : 0u;
    P.tiles_s2 = P.p2 > 0 ? (uint32_t)(((uint64_t)1 << P.p1) * P.chunks1) : 0u;
    P.tiles_part = (uint32_t)(1ull << P.p);
    P.tiles_scan = (uint32_t)(((1ull << P.p) + kPlanScanChunk - 1) / kPlanScanChunk);
    P.tiles_t2h = (uint32_t)((P.t2cap / P.pchunks + kPlanT2HashTile - 1) / kPlanT2HashTile);
    if (P.tiles_t2h == 0) P.tiles_t2h = 1;
    P.tiles_t2s = (uint32_t)(((1ull << P.p) + kPlanT2SlotGroup - 1) / kPlanT2SlotGroup);

    // Slot regions (SoA: key64 array, then nonce array).
    if (P.p2 > 0) {
        const uint64_t recs = ((uint64_t)P.hchunks << P.p1) * P.cap1;
        P.regionA_keys = recs * 8;
        P.regionA_bytes = recs * 12;
    }
    {
        const uint64_t recs = ((uint64_t)1 << P.p) * P.cap2;
        P.regionB_keys = recs * 8;
        P.regionB_bytes = recs * 12;
    }
    // Buffers.  The first-level slots alias the Table-1 buffer (they are
    // consumed by the second scatter level before any Table-1 write).  The
    // final-partition slots get their own region in the scratch buffer: the
    // fused sort + match reads them while it writes both tables.
    // A window's record count is random: its Table 1 takes the most its
    // partition slots can hold, so no write can pass the buffer's end.
    const uint64_t t1_rec = P.wbits ? std::min<uint64_t>(P.N, ((uint64_t)1 << P.p) * P.cap2) : P.N;
    const uint64_t t1_tab = 12 * t1_rec;
    // A window of a tiled plot may hash from a list of its nonces (as many
    // as its Table 1 can hold), kept in its Table-2 buffer until the sort.
    P.listcap = P.wbits ? (uint32_t)std::min<uint64_t>(t1_rec, 0xFFFFFFFFull) : 0u;
    P.tiles_list = (uint32_t)(((uint64_t)P.listcap + kPlanHashTile - 1) / kPlanHashTile);
    const uint64_t t2_tab = std::max<uint64_t>(16 * P.t2cap, 4 * (uint64_t)P.listcap);
    P.t1_bytes = round_up((t1_tab > P.regionA_bytes ? t1_tab : P.regionA_bytes) + 256, 256);
    P.t2_bytes = round_up(t2_tab + 256, 256);
    // Scratch layout.
    const uint64_t np = 1ull << P.p;
    uint64_t at = 0;
    P.o_status = at;
    P.o_ticket = at + 64;
    P.o_ticket_s = at + 128;
    at += 256;
    P.o_cnt1 = at; at = round_up(at + 4 * ((uint64_t)P.hchunks << P.p1), 256);
    P.o_cnt2 = at; at = round_up(at + 4 * np, 256);
    P.o_t1off = at; at = round_up(at + 8 * (np + 1), 256);
    P.o_pairs = at; at = round_up(at + 8 * np, 256);
    P.o_t2off = at; at = round_up(at + 8 * (np + 1), 256);
    P.o_lb = at; at = round_up(at + 8 * np, 256);
    P.o_lbs = at; at = round_up(at + 8 * (uint64_t)P.tiles_scan, 256);
    P.o_desc = at; at = round_up(at + desc_bytes, 256);
    P.o_tiles = at; at = round_up(at + 512, 256);
    P.o_regionB = at; at = round_up(at + P.regionB_bytes, 256);
    const uint64_t nh = P.hcap ? np : 0;
    P.o_halo_cnt = at; at = round_up(at + 4 * nh, 256);
    P.o_halo_keys = at; at = round_up(at + 8 * nh * P.hcap, 256);
    P.o_halo_nonces = at; at = round_up(at + 4 * nh * P.hcap, 256);
    P.o_wcount = at; at = round_up(at + 4, 256);
    P.scratch_bytes = at;
    *pl = P;
    return VX_OK;
}

// Table 2 sorted by hash2 (vx_sort_table2): partitions of ~2^11 of the n
// Table-2 records by the top p bits of key2 (uniform hash bits, so slot
// fills are Poisson), two scatter levels of <= 10 bits, and a work buffer
// holding both levels' slots (16 B per record) and the counters.
struct Sort2Plan {
    int p, p1, p2, dbits;
    uint32_t cap1, cap2, chunks1;
    uint32_t tiles1, tiles2, tiles_scan, parts;
    uint64_t o_desc, o_ticket, o_cnt1, o_cnt2, o_off, o_lbs, o_akeys, o_avals, o_bkeys, o_bvals;
    uint64_t bytes;
};

inline int make_sort2_plan(uint64_t n, Sort2Plan *out, size_t desc_bytes)
{
    Sort2Plan S;
    memset(&S, 0, sizeof(S));
    int lg = 0;
    while (lg < 63 && (2ull << lg) <= n) ++lg;  // floor(log2(n)), 0 for n <= 1
    S.p = lg - kSort2PartLog2;
    if (S.p < 0) S.p = 0;
    if (S.p > 20) S.p = 20;  // its second level keeps to <= 10 bits
    S.p1 = S.p <= 10 ? S.p : S.p / 2;
    S.p2 = S.p - S.p1;
    const double avg2 = (double)n / (double)(1ull << S.p);
    uint64_t cap2 = S.p == 0 ? round_up(n, 4) : slot_capacity(avg2, kDefaultSlackSigma);
    if (cap2 < 4) cap2 = 4;
    if (cap2 > 16384) return VX_EINVAL;
    S.cap2 = (uint32_t)cap2;
    int db = lg - S.p;
    if (db < 1) db = 1;
    if (db > 13) db = 13;
    S.dbits = db;
    if (S.p2 > 0) {
        const uint64_t cap1 = slot_capacity((double)n / (double)(1ull << S.p1), kDefaultSlackSigma);
        if (cap1 > 0xFFFFFF00ull) return VX_EINVAL;
        S.cap1 = (uint32_t)cap1;
        S.chunks1 = (uint32_t)((cap1 + 4095) / 4096);
        S.tiles2 = (uint32_t)((1u << S.p1) * S.chunks1);
    }
    S.tiles1 = (uint32_t)((n + kPlanS2Tile1 - 1) / kPlanS2Tile1);
    S.parts = 1u << S.p;
    S.tiles_scan = (uint32_t)((S.parts + kPlanScanChunk - 1) / kPlanScanChunk);
    const uint64_t np = S.parts, n1 = S.p2 > 0 ? (1ull << S.p1) : 0ull;
    uint64_t at = 0;
    S.o_desc = at; at = round_up(at + desc_bytes, 256);
    S.o_ticket = at; at = round_up(at + 4, 256);
    S.o_cnt1 = at; at = round_up(at + 4 * n1, 256);
    S.o_cnt2 = at; at = round_up(at + 4 * np, 256);
    S.o_off = at; at = round_up(at + 8 * (np + 1), 256);
    S.o_lbs = at; at = round_up(at + 8 * (uint64_t)S.tiles_scan, 256);
    S.o_akeys = at; at = round_up(at + 8 * n1 * S.cap1, 256);
    S.o_avals = at; at = round_up(at + 8 * n1 * S.cap1, 256);
    S.o_bkeys = at; at = round_up(at + 8 * np * S.cap2, 256);
    S.o_bvals = at; at = round_up(at + 8 * np * S.cap2, 256);
    S.bytes = at;
    *out = S;
    return VX_OK;
}

}  // namespace vx
