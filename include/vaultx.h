/*
 * vaultx.h -- C ABI of the GB300 (sm_103a) VaultxGPU plotting path.
 *
 * A plot is the paper's unit of work (Sec. III-A): for a K and a 256-bit
 * plot key, hash every nonce 0 .. 2^K-1 with keyed BLAKE3 into Table 1,
 * bucket and sort Table 1 by hash prefix, pair its entries under the match
 * threshold and hash every pair into Table 2.  All compute runs in this
 * library's CUDA kernels; the Python binding only marshals arguments.
 *
 * Layouts (readings of the paper, which leaves them unstated):
 *   Table 1 record, 12 bytes: LE u32 nonce, then hash bytes 0..7 of
 *     BLAKE3-keyed(key, LE32(nonce)).  Sorted by key64 = big-endian u64 of
 *     the 8 hash bytes, ties by nonce; logical bucket = key64 >> 40, so the
 *     2^24 buckets of Sec. I-A / III-B come out concatenated in order.
 *   Table 2 record, 16 bytes: LE u32 a, LE u32 b, then hash bytes 0..7 of
 *     BLAKE3-keyed(key, LE32(a) || LE32(b)); (a, b) ranges over pairs of
 *     Table-1 records i < j in the same logical bucket with
 *     key64_j - key64_i < D (Sec. II-B "matching factor threshold",
 *     Sec. III-A "expected distance threshold"); D = 2^(64-K) by default.
 *     Order: bucket, then i, then j.
 *
 * Conventions.
 *   - Every call returns an int status: VX_OK (0) or a negative VX_E* code.
 *     No call aborts the process, and no kernel traps: device-side failures
 *     set bits in a per-plot status word that vx_sync() reads and maps.
 *   - Streams are cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Compute calls are asynchronous on that stream.
 *   - Device pointers are plain CUDA device addresses (e.g. a torch
 *     tensor's data_ptr()).  Buffers given to vx_plot_bind stay owned by
 *     the caller; the library never frees them.
 *   - A vx_plot is owned by the caller from vx_plot_create until
 *     vx_plot_destroy; it may be used from one host thread at a time.
 */
#ifndef VAULTX_H
#define VAULTX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status */
enum {
    VX_OK = 0,
    VX_EINVAL = -1,     /* bad argument (K, key, opts, pointer, alignment, size)   */
    VX_ENOMEM = -2,     /* allocation failed, or Table 2 exceeds its capacity      */
    VX_ECUDA = -3,      /* a CUDA runtime call failed (detail in vx_last_error)    */
    VX_ETIMEDOUT = -4,  /* a bounded device-side wait gave up                      */
    VX_EBUSY = -5,      /* server full / resource in use                           */
    VX_ENOTREADY = -6,  /* result not produced yet (call order, or still running)  */
    VX_EOVERFLOW = -7,  /* a partition slot overflowed its capacity: the tables are
                           incomplete; re-run with a larger opts.slack_sigma       */
    VX_EIO = -8         /* a plot file could not be opened, written or closed (the
                           system's reason, errno text, in vx_last_error)          */
};

/* Table selectors. */
enum { VX_TABLE1 = 1, VX_TABLE2 = 2 };

/* vx_opts.test_flags bits. */
enum { VX_TEST_WITHHOLD_PREFIX = 1 };

/* Plot states reported by the server. */
enum { VX_QUEUED = 0, VX_RUNNING = 1, VX_DONE = 2, VX_FAILED = 3 };

/* Tuning and semantics options.  Zero-initialised fields take defaults;
 * always set .size = sizeof(vx_opts) (vx_opts_default does). */
typedef struct vx_opts {
    uint32_t size;              /* sizeof(vx_opts)                                   */
    uint32_t test_flags;        /* fault injection for tests, 0 in normal use:
                                   VX_TEST_WITHHOLD_PREFIX makes partition 0 of the
                                   fused sort + match (look-back placement), or
                                   chunk 0 of the pair-count scan (slot placement),
                                   never publish its Table-2 prefix, so every later
                                   bounded wait runs out (short limit) and vx_sync
                                   returns VX_ETIMEDOUT; the paper has no
                                   counterpart                                       */
    uint64_t match_distance;    /* D of the match predicate; 0 = 2^(64-K)            */
    int32_t partition_log2;     /* log2 of the mean records per physical partition
                                   (6..13); 0 = default (11).  Partitions are runs
                                   of whole logical buckets; at most 2^24 of them.  */
    int32_t coarse_bits;        /* bits of the first scatter level (0..10);
                                   -1 = automatic                                     */
    uint32_t slack_sigma;       /* partition-slot slack in standard deviations of a
                                   Poisson count; 0 = default (12)                   */
    uint32_t hash_block;        /* threads per block of the hash kernels: 0 or 256
                                   (the one shape built; others are VX_EINVAL)      */
    uint32_t nonces_per_thread; /* nonces each Table-1 hash thread handles: 0 (= 8),
                                   4, 8 or 16 with the staged bucketing of a whole
                                   plot; 8 with the direct bucketing or a window;
                                   others VX_EINVAL.  Same tables for every value. */
    uint32_t scatter_mode;      /* bucketing of hashed records: 0 = automatic
                                   (staged), 1 = staged (shared-memory histogram per CTA, one
                                   claim per (CTA, bin), two levels), 2 = direct
                                   (one slot claim per record into the final
                                   partition)                                          */
    uint64_t t2_capacity;       /* Table-2 capacity in records; 0 = default bound    */
    uint32_t fuse_pair_hash;    /* vx_plot_run: 1 = hash the pairs inside the sort +
                                   match kernel; 0 = (default) the sort writes {a, b}
                                   records and a streaming pass hashes them         */
    uint32_t pipeline_chunks;   /* vx_plot_run / batches: the hash and the second
                                   scatter level, and the sort and the pair hash,
                                   run in this many chunks on two streams, each
                                   memory-bound chunk overlapping the next ALU-bound
                                   one; 0 = automatic (currently no overlap: on
                                   GB300 the kernel pairs take turns on the SMs
                                   rather than share them), 1 = no overlap; else
                                   2, 4 or 8                                          */
    uint32_t t2_placement;      /* vx_plot_run / batches (not fused, not pipelined):
                                   how each partition's pairs reach their Table-2
                                   offset.  1 = the sort + match kernel chains the
                                   partitions by a decoupled look-back and writes
                                   {a, b} records at their final offsets; 2 = it
                                   writes each partition's {a, b} pairs into that
                                   partition's own sort slot (1.5x its record
                                   capacity), a scan of the per-partition pair
                                   counts gives the offsets, and the pair hash
                                   moves the pairs to Table 2 (no waiting between
                                   partitions; more pairs than the slot holds fail
                                   the plot with VX_EOVERFLOW: at K >= 26 with the
                                   default D a partition expects ~2040 +- 100 pairs
                                   against 3910 places); 0 = automatic = 1 (the
                                   faster on GB300 at K=31)                        */
    uint32_t match_scope;       /* 0 = (default) pairs inside one logical bucket
                                   (the fused Sort+Match kernel of Sec. III-A holds
                                   one bucket); 1 = cross-bucket: every pair i < j
                                   of the whole Table-1 order with key64_j - key64_i
                                   < D.  The few records within D of the next
                                   physical partition's lower edge (a "halo", mean
                                   2^11 * D / 2^(64-p) records) are collected while
                                   the partitions are filled; needs D <= 2^(64-p)
                                   and a halo of at most 256 records             */
    uint32_t window_bits;       /* c: 0 = (default) the whole plot.  c >= 1 makes
                                   this plot window `window` of 2^c: only the
                                   records whose key64 has top c bits == window
                                   (2^(24-c) consecutive logical buckets), their
                                   sorted Table 1 and their Table-2 pairs; the
                                   2^c windows concatenated in window order are
                                   the whole plot's tables.  Every nonce is still
                                   hashed (the hash decides the window); buffers
                                   shrink by ~2^c.  Chunked device-memory tiling
                                   (Sec. V future work).  Needs match_scope 0 and
                                   c <= the partition bits (K - partition_log2,
                                   at most 21); c <= 16                            */
    uint32_t window;            /* the window index, < 2^window_bits                 */
    uint32_t reserved[2];       /* must be zero                                      */
} vx_opts;

typedef struct vx_plot vx_plot;

/* Fills *opts with the defaults.  Returns VX_EINVAL on NULL.  Library
 * housekeeping: the paper has no counterpart. */
int vx_opts_default(vx_opts *opts);

/* Short static description of a status code.  The paper has no counterpart. */
const char *vx_strerror(int status);

/* Detail of the last failure on this plot (static empty string if none or
 * plot is NULL).  Valid until the next call on the plot.  The paper has no
 * counterpart. */
const char *vx_last_error(const vx_plot *plot);

/* Library version, (major << 16) | minor.  The paper has no counterpart. */
int vx_version(void);

/* Device memory one plot needs (Sec. I-A: Table 1 stays resident in VRAM).
 *   t1_bytes:      Table-1 buffer (>= 12 * 2^K; a staged two-level scatter
 *                  also uses it for its first level, so it may be larger)
 *   t2_bytes:      Table-2 buffer (16 * Table-2 capacity, + 256)
 *   scratch_bytes: counters, offsets, the plot descriptor, and the partition
 *                  slots the hashed records are bucketed into (about
 *                  12 * 2^K * 1.3 bytes)
 * Any output pointer may be NULL.  1 <= K <= 32.  No allocation. */
int vx_plot_required_bytes(int K, const vx_opts *opts, uint64_t *t1_bytes,
                           uint64_t *t2_bytes, uint64_t *scratch_bytes);

/* Creates a plot for (K, key) (Sec. III-B: the 256-bit plot key).  key is 32
 * host bytes, copied.  opts may be NULL.  Allocates host state only. */
int vx_plot_create(int K, const uint8_t key[32], const vx_opts *opts, vx_plot **out);

/* Gives the plot caller-owned device buffers of at least the sizes
 * vx_plot_required_bytes reports, each 256-byte aligned.  t2_capacity is the
 * number of 16-byte Table-2 records d_t2 can hold (0 = t2_bytes / 16 of the
 * default plan).  Replaces any earlier binding; frees library-owned memory.
 * Both tables live in device memory for the whole plot (Sec. I-A); that the
 * caller owns the buffers has no counterpart in the paper, whose plotter
 * allocates them itself. */
int vx_plot_bind(vx_plot *plot, void *d_t1, void *d_t2, void *d_scratch, uint64_t t2_capacity);

/* Allocates library-owned device buffers (cudaMalloc) if none are bound:
 * the paper's own arrangement, Table 1 and Table 2 in device memory
 * (Sec. I-A, III-A). */
int vx_plot_alloc(vx_plot *plot);

/* Table 1 (Sec. III-A hash stage; sort half of the fused Sort+Match kernel):
 * key setup, keyed BLAKE3 of every nonce, two-level bucketing scatter by
 * hash prefix, in-partition shared-memory sort.  Allocates (vx_plot_alloc)
 * if nothing is bound.  Asynchronous on stream. */
int vx_table1(vx_plot *plot, void *stream);

/* Table 2 (Sec. III-A match half of the fused Sort+Match kernel): pair
 * counting, deterministic placement by prefix sums, pair hashing.  Requires
 * vx_table1 earlier on the same stream.  If the pairs exceed the Table-2
 * capacity nothing is written and vx_sync returns VX_ENOMEM; the needed
 * count is then in vx_table_info(VX_TABLE2).nrec.  Asynchronous. */
int vx_match(vx_plot *plot, void *stream);

/* Table 1 and Table 2 in one pass (Sec. III-A pipeline): key setup, keyed
 * BLAKE3 of every nonce fused with the first bucketing scatter level, the
 * second level, then the fused partition sort + match kernel.  That kernel
 * sorts each partition in shared memory and writes it to Table 1; its pairs
 * {a, b} go either into Table 2 at the offset a decoupled look-back over
 * the earlier partitions gives (t2_placement 1; a streaming pass then
 * hashes them in place) or into the partition's own slot (t2_placement 2,
 * the automatic choice when they fit; a scan of the pair counts and the
 * slot pair hash then write Table 2).  fuse_pair_hash hashes inside the
 * sort kernel instead.  Same tables as vx_table1 + vx_match.  Ends with a
 * 12-byte copy of the status and the Table-2 count to pinned host memory
 * and an event that vx_sync waits on.  Allocates if nothing is bound.
 * Asynchronous.  One plot's runs must not overlap on the GPU (two runs of
 * the same plot on different streams race on its buffers): different plots
 * may run concurrently. */
int vx_plot_run(vx_plot *plot, void *stream);

/* Waits for the plot's work, reads its status word and Table-2 count, and
 * maps the status to VX_OK / VX_EOVERFLOW / VX_ENOMEM / VX_ETIMEDOUT.
 * Synchronous.  After vx_plot_run it waits on an event recorded behind that
 * run (vx_plot_run ends with a 12-byte device-to-host copy of the status and
 * count into the handle's pinned block), so work queued later on the same
 * stream is not waited for, and the values are this run's even when a later
 * plot on the stream reuses the same Table-1 and scratch buffers.  After
 * vx_table1, vx_match or vx_plot_batch it synchronises the whole stream and
 * reads the scratch buffer.  The paper's host likewise waits for the device
 * before Table 2 leaves it (Sec. III-A); the status codes (capacity
 * overflow, bounded-wait timeout) have no counterpart there. */
int vx_sync(vx_plot *plot);

/* Zero-copy view of a table: device pointer, record count, record size.
 * Table-2 counts are known after vx_sync following vx_match (VX_ENOTREADY
 * before).  The tables are the ones Sec. III-A keeps in device memory; the
 * view itself has no counterpart in the paper. */
int vx_table_info(const vx_plot *plot, int which, const void **dptr, uint64_t *nrec,
                  uint32_t *rec_bytes);

/* Autotuner: times every distinct plan for K that the candidate options give
 * (partition size 2^9 .. 2^13 records, i.e. the physical partition count and
 * the sort tile; the staged bucketing with 4, 8 or 16 nonces per hash
 * thread, i.e. threads per nonce 1/4, 1/8, 1/16; the direct bucketing with
 * 8) on this device.  Each candidate runs one warm-up and three timed plots
 * with a fixed synthetic key in library-owned memory on stream (CUDA
 * events).  *best gets base (defaults if null) with the fastest candidate's
 * partition_log2, scatter_mode and nonces_per_thread, *best_ms its mean
 * plot time.
 * Synchronous; a candidate that cannot be planned or allocated is skipped
 * (VX_ENOMEM if none ran).  The Python binding keeps an on-disk cache of the
 * result keyed by device and K.  The paper has no counterpart (its kernels
 * use a fixed block size, Sec. III-B). */
int vx_autotune(int K, const vx_opts *base, vx_opts *best, double *best_ms, void *stream);

/* Writes the 2^24 + 1 logical-bucket offsets of Table 1 (u64, offsets[b] =
 * records in buckets < b) to d_out (device, 8-byte aligned): the 2^24
 * buckets Table 1 is organised into (Sec. I-A, III-B), which this library
 * stores concatenated rather than at fixed per-bucket capacity.
 * Asynchronous. */
int vx_table1_offsets(vx_plot *plot, void *d_out, void *stream);

/* Copies bytes [offset, offset + bytes) of a table to host memory (pinned
 * memory makes it asynchronous on stream).  The range must lie within
 * nrec * rec_bytes.  The device-to-host transfer of Sec. III-A, for any
 * byte range of either table. */
int vx_table_copy(vx_plot *plot, int which, uint64_t offset, void *host_dst, uint64_t bytes,
                  void *stream);

/* Table 2 sorted by its hash, for lookups by hash value (the VaultX prover
 * searches a plot by hash, Sec. I-B; the paper's Table 2 stays in pair
 * order).  Reorders the plot's Table 2 in place into ascending (key2, a, b),
 * key2 = big-endian u64 of the record's hash2 bytes; records are unchanged.
 * Needs the plot complete and synced (vx_sync returned VX_OK; VX_ENOTREADY
 * otherwise) and a caller-owned device work buffer of at least
 * vx_sort_table2_work_bytes (256-byte aligned; about 36.5 B per Table-2
 * record: two scatter levels of 16-byte records; the library never frees
 * it).  Asynchronous on stream; vx_sync then reports VX_EOVERFLOW if a slot
 * overflowed (Table 2 is then left partly rewritten). */
int vx_sort_table2_work_bytes(const vx_plot *plot, uint64_t *bytes);
int vx_sort_table2(vx_plot *plot, void *d_work, uint64_t work_bytes, void *stream);

/* Writes Table 2 as a flat binary file (Sec. III-A / III-B: D2H through a
 * 256 MB pinned staging buffer on the library's own copy stream, sequential
 * 4 MB chunks; no header).  The device copy of one 128 MB half overlaps the
 * write of the other.  Waits for the plot's own work first (vx_sync), so it
 * may run on a host thread while later plots compute.  Returns after the
 * data is handed to the file system (no fsync); seconds_d2h = time spent
 * waiting for device copies, seconds_total = the whole call.  Synchronous.
 * VX_EIO when the file cannot be opened, a write fails or the close reports
 * a deferred write error (errno text in vx_last_error); VX_ECUDA when a
 * device copy fails. */
int vx_plot_write(vx_plot *plot, const char *path, double *seconds_d2h, double *seconds_total);

/* ------------------------------------------- chunked device-memory tiling */

/* Memory vx_plot_tiled needs for 2^K nonces in 2^window_bits windows
 * (vx_opts.window_bits; opts' own window fields must be zero):
 *   device_bytes:  two windows' buffers (one window computes while the other's
 *                  tables are copied out; one window if window_bits is 0),
 *                  plus one byte per nonce of window ids for 1..8 window bits
 *   host_t1_bytes: 12 * 2^K, Table 1 exactly
 *   host_t2_bytes: the windows' Table-2 capacities, 16 B per record (a bound)
 * Any output pointer may be NULL.  Host only.  VX_EINVAL for a combination
 * the planner rejects (see vx_opts.window_bits). */
int vx_plot_tiled_bytes(int K, const vx_opts *opts, int window_bits, uint64_t *device_bytes,
                        uint64_t *host_t1_bytes, uint64_t *host_t2_bytes);

/* How many times vx_plot_tiled hashes every nonce at window_bits c, into
 * *passes: 1 for c = 0 (the whole plot), 2 for 1 <= c <= 8 without nonce
 * chunks (a first pass stores one window-id byte per nonce, then each window
 * hashes only its own nonces), else 2^c (each window hashes every nonce and
 * keeps its share: at K=31 a hash pass takes ~51 ms, so c = 9 costs ~26 s).
 * The cost to weigh against vx_plot_tiled_bytes' footprint: above 8 bits
 * the id bytes are gone (K=31: 2.93 GB at c = 8, 0.39 GB at c = 9) but the
 * hashing grows 256-fold.  VX_EINVAL as vx_plot_tiled_bytes.  Host only.
 * The paper has no counterpart. */
int vx_plot_tiled_hash_passes(int K, const vx_opts *opts, int window_bits, uint32_t *passes);

/* The fewest window bits (0 .. 16) whose vx_plot_tiled_bytes device_bytes
 * fit budget_bytes and whose vx_plot_tiled_hash_passes are at most
 * max_hash_passes (>= 1), into *window_bits.  VX_ENOMEM if none does (the
 * partition bits bound the window bits), VX_EINVAL for bad arguments.  Host
 * only.  The paper has no counterpart. */
int vx_plot_tiled_window_bits_capped(int K, const vx_opts *opts, uint64_t budget_bytes,
                                     uint32_t max_hash_passes, int *window_bits);

/* vx_plot_tiled_window_bits_capped with at most 2 hash passes: the window-id
 * path only, never the window counts above 8 bits that hash the whole plot
 * once per window (a budget below that path's footprint gets VX_ENOMEM; a
 * caller who accepts 2^c passes asks the capped call).  Host only. */
int vx_plot_tiled_window_bits(int K, const vx_opts *opts, uint64_t budget_bytes, int *window_bits);

/* A whole plot in device memory of about 2^(1 - window_bits) of its
 * footprint (chunked VRAM tiling, Sec. V future work): the 2^window_bits
 * windows of vx_opts.window_bits are built one after the other in two
 * window buffer sets on `stream` -- cut from d_work, caller-owned device
 * memory of at least vx_plot_tiled_bytes' device_bytes (256-byte aligned,
 * never freed by the library), or allocated for the call and freed before
 * it returns when d_work is NULL -- and each finished window's
 * tables are copied, on a copy stream of the library's own and overlapped
 * with the next window's kernels, to their places in host memory: Table 1
 * (12-byte records, 2^K of them; host_t1 may be NULL to skip it, else it
 * holds at least 12 * 2^K bytes) and Table 2 (16-byte records) at host_t2,
 * host_t2_bytes long.  The host tables equal the whole plot's (vx_plot_run
 * without windows) byte for byte.  Pinned host memory (cudaHostAlloc) makes
 * the copies asynchronous; pageable memory works but serialises them.
 * With 1..8 window bits a first pass hashes every nonce and stores its
 * window (one byte), and each window hashes only the nonces listed for it:
 * two hashes of every nonce in all.  With more window bits, or the hash
 * split into nonce chunks (vx_opts.pipeline_chunks), each window hashes
 * every nonce and keeps its share.  *t1_count / *t2_count (may be
 * NULL) get the record counts.  Returns VX_OK; VX_ENOMEM if Table 2 did not
 * fit host_t2_bytes (*t2_count is then the size needed; Table 1 is
 * complete) or a window buffer could not be allocated; a window's
 * VX_EOVERFLOW / VX_ETIMEDOUT stops the plot; VX_EINVAL for window bits the
 * planner rejects, opts that already name a window, a d_work shorter than
 * device_bytes or not 256-byte aligned, or a host_t1 shorter than 12 * 2^K.
 * Synchronous.  The paper names the direction; the window scheme is this
 * library's. */
int vx_plot_tiled(int K, const uint8_t key[32], const vx_opts *opts, int window_bits,
                  void *d_work, uint64_t work_bytes, void *host_t1, uint64_t host_t1_bytes,
                  void *host_t2, uint64_t host_t2_bytes, uint64_t *t1_count, uint64_t *t2_count,
                  void *stream);

/* vx_plot_tiled with Table 2 written as a flat plot file at `path` (created
 * or truncated; the bytes of vx_plot_write of the whole plot) instead of
 * into host memory: each finished window's Table 2 is appended through the
 * library's 256 MB pinned staging buffer in sequential 4 MB chunks
 * (Sec. III-A, III-B) while the next window computes, so no host buffer of
 * the table's size is needed.  d_work and host_t1 as in vx_plot_tiled (both
 * may be NULL).
 * *seconds (may be NULL) gets the call's wall time.  On an error the file
 * holds the windows written so far.  Synchronous.  VX_EIO when the file
 * cannot be opened, a write fails or the close reports a deferred write
 * error; VX_ECUDA when a device step fails. */
int vx_plot_tiled_write(int K, const uint8_t key[32], const vx_opts *opts, int window_bits,
                        void *d_work, uint64_t work_bytes, const char *path, void *host_t1,
                        uint64_t host_t1_bytes, uint64_t *t1_count, uint64_t *t2_count,
                        double *seconds, void *stream);

/* Runs vx_table1 + vx_match for n plots as one batch: every stage is one
 * grouped launch over all plots' work (mixed K and keys), recorded once into
 * a CUDA graph per batch shape and replayed.  Each plot must be bound or
 * allocatable.  Per-plot status via vx_sync on each plot (the batch records
 * the stream on every plot).  Asynchronous.  The paper plots one K at a time
 * and has no counterpart. */
int vx_plot_batch(vx_plot *const *plots, int n, void *stream);

/* Frees library-owned memory and the handle.  NULL is a no-op.  The paper
 * has no counterpart. */
void vx_plot_destroy(vx_plot *plot);

/* ------------------------------------------------- no-allocation path */

/* Bytes of the library's static device scratch array (64 MiB). */
#define VX_NOALLOC_SCRATCH_BYTES (64ull << 20)

/* vx_plot_run without any allocation, for callers that cannot call
 * cudaMalloc: callers whose device memory belongs to another allocator
 * under a fixed budget (a framework's caching allocator, a pre-reserved
 * pool) that must not be bypassed, and latency-critical callers that must
 * not take the implicit device-wide synchronisation cudaMalloc can cause.
 * The paper has no counterpart.
 *
 * The caller passes the key (32 host bytes) and both table buffers: d_t1 and
 * d_t2 (device, 256-byte aligned) of at least the t1_bytes / t2_bytes that
 * vx_plot_required_bytes(K, opts) reports; t2_capacity is d_t2's record
 * capacity (0 = the planned one).  Everything else -- partition slots,
 * counters, offsets, the plot descriptor -- lives in one static device array
 * of VX_NOALLOC_SCRATCH_BYTES that every GPU loading the library holds until
 * the process exits; plots whose scratch (vx_plot_required_bytes'
 * scratch_bytes) does not fit, e.g. K > 22 with default options, are
 * rejected with VX_EINVAL.  No cudaMalloc, cudaFree, pinned or library
 * allocation is made.
 *
 * The first call on a device looks up the array's device address (once per
 * device; make that first call before any stream capture).  All calls share
 * the one array, which keeps the last call's contents (each run clears what
 * it reads before use): calls that overlap on the GPU -- on other streams
 * or other host threads -- race and corrupt each other.  The kernels run one
 * after the other on `stream`; the call then waits for them and returns
 * VX_OK / VX_EOVERFLOW / VX_ENOMEM / VX_ETIMEDOUT like vx_sync, with the
 * Table-2 record count in *t2_count (if not NULL).  Synchronous. */
int vx_plot_run_noalloc(int K, const uint8_t key[32], const vx_opts *opts, void *d_t1, void *d_t2,
                        uint64_t t2_capacity, void *stream, uint64_t *t2_count);

/* ------------------------------------------------------------ tracing */

/* Records CUDA events around every kernel of this plot's next `runs` runs
 * (a run is vx_plot_run, or vx_table1 followed by vx_match; single-plot
 * path; the paper's per-stage timing of Sec. IV-C at kernel granularity).  runs = 0 turns tracing off
 * and frees the events.  Adds one event record per kernel, no sync. */
int vx_plot_profile(vx_plot *plot, int runs);

/* Sums the traced runs: ms[k] = total milliseconds of kernel k, k <
 * *nkernels (cap must be >= 9); *nruns = runs recorded.  Waits for them.
 * The per-stage times of Sec. IV-C, summed per kernel. */
int vx_plot_profile_read(vx_plot *plot, double *ms, int cap, int *nkernels, int *nruns);

/* Which kernel slots (bit k = kernel k of vx_kernel_name) one run of this
 * plot launches: split != 0 for vx_table1 + vx_match, else vx_plot_run.
 * Host only.  The paper has no counterpart. */
int vx_plot_kernel_mask(const vx_plot *plot, int split, uint32_t *mask);

/* Name of traced kernel k ("key_setup", "hash_staged", "hash_direct",
 * "scatter2", "scan_counts", "sort", "scan_pairs", "match", "sortmatch"),
 * or "" if out of range.  Kernels a run does not use time as zero.  The
 * paper has no counterpart. */
const char *vx_kernel_name(int k);

/* ------------------------------------------------ stand-alone stages */

/* Keyed BLAKE3 of nonces nonce0 .. nonce0+count-1 into 12-byte Table-1
 * records in nonce order (no bucketing), at d_out (device, 4-byte aligned,
 * 12*count bytes).  The hash row of the path on its own: one keyed hash of
 * each little-endian nonce with the plot key (Sec. III-B), without the
 * bucket insertion.  Asynchronous. */
int vx_hash_nonces(const uint8_t key[32], uint64_t nonce0, uint64_t count, void *d_out,
                   void *stream);

/* Measurement of the hash's ceiling, not a step of the path: keyed BLAKE3
 * of nonces nonce0 .. nonce0+count-1 in the Table-1 hash kernel's shape
 * (256 threads, 8 nonces per thread and step), with no record stores; each
 * thread folds its hash words into one u32 of d_fold (device, 4-byte
 * aligned, fold_words words, a nonzero multiple of 256: the grid is
 * fold_words / 256 CTAs).  Timing it gives the integer-issue rate this
 * instruction mix reaches with no memory work beside it, the ceiling the
 * Table-1 hash (Sec. III-B) is compared with.  VX_EINVAL for a bad size or
 * a nonce range beyond 2^32.  Asynchronous.  The paper has no counterpart. */
int vx_hash_peak(const uint8_t key[32], uint64_t nonce0, uint64_t count, void *d_fold,
                 uint32_t fold_words, void *stream);

/* Pair hash of Table 2 on its own: for each of `count` pairs (a, b) at
 * d_pairs (device, 2 LE u32 each, 8-byte aligned) writes the 16-byte
 * Table-2 record {a, b, hash2[0..7]} to d_out (16-byte aligned),
 * hash2 = keyed hash of LE32(a) || LE32(b) with the plot key.  The paper
 * produces Table-2 records from matched pairs (Sec. II-B, III-A) but does
 * not state their content; this is the reading the whole library uses.
 * Asynchronous. */
int vx_pair_hash(const uint8_t key[32], const void *d_pairs, uint64_t count, void *d_out,
                 void *stream);

/* Test hook (host-side fault injection, no GPU fault): the next `count`
 * device allocations the library makes fail as if cudaMalloc had returned
 * cudaErrorMemoryAllocation, so callers' VX_ENOMEM paths can be exercised.
 * The paper has no counterpart.  count <= 0 clears it. */
int vx_test_fail_next_allocs(int count);

/* ------------------------------------------------------------ server */

typedef struct vx_server vx_server;

typedef struct vx_serve_opts {
    uint32_t size;           /* sizeof(vx_serve_opts)                                  */
    uint32_t max_inflight;   /* plots admitted and not yet fetched by vx_serve_poll
                                (queued on the device, running, or done and waiting);
                                0 = 4 (more plots in flight crowd each other out of
                                L2: 64 served 10% fewer nonces/s).  A fetched plot
                                no longer counts; its memory stays charged to the
                                budget until vx_plot_destroy                           */
    uint64_t memory_budget;  /* bytes of device memory the server may hold; 0 = 80% of
                                free memory at creation                                 */
    uint32_t streams;        /* concurrent waves in flight; 0 = 2                      */
    uint32_t max_wave;       /* plots per wave (one batch launch); 0 = 32              */
    vx_opts plot_opts;       /* options for every plot (size 0 = defaults)            */
} vx_serve_opts;

/* Creates a continuous-batching plot server on the current device.  The
 * vx_serve_* calls have no counterpart in the paper, which plots one K at a
 * time. */
int vx_serve_create(const vx_serve_opts *opts, vx_server **out);

/* Queues a plot request; *ticket identifies it.  VX_EINVAL for a bad K or a
 * plot larger than the memory budget.  Never blocks. */
int vx_serve_submit(vx_server *srv, int K, const uint8_t key[32], uint64_t *ticket);

/* Advances the server (admits queued requests whose footprint fits the free
 * budget, launches waves, retires finished ones) and reports the ticket's
 * state.  When *state == VX_DONE and out != NULL, the plot handle is handed
 * to the caller (tables on the device, count synced), who must
 * vx_plot_destroy it; that frees its share of the budget.  VX_EINVAL for an
 * unknown ticket. */
int vx_serve_poll(vx_server *srv, uint64_t ticket, int *state, vx_plot **out);

/* Advances the server without asking about a ticket; returns the number of
 * requests not yet handed out. */
int vx_serve_step(vx_server *srv);

/* Submit-to-done latency of a finished ticket in seconds. */
int vx_serve_latency(vx_server *srv, uint64_t ticket, double *seconds);

/* Waits for all waves, frees every plot not handed out, frees the server. */
void vx_serve_destroy(vx_server *srv);

#ifdef __cplusplus
}
#endif
#endif /* VAULTX_H */
