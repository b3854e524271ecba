// vx_engine.h -- internal host-side state shared by the C ABI (vx_api.cu)
// and the plot server (vx_serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/vaultx.h"
#include "vx_internal.cuh"
#include "vx_plan.h"

namespace vx {
constexpr int kMaxChunks = 8;             // pipeline chunks per stage
// Kernels a run may launch (tracing ids, vx_kernel_name order).
constexpr int kProfKernels = 10;
constexpr int kProfLaunches = 64;         // traced launches per run (upper bound)
// Fork/join events of one pipelined run: hash->scatter2 per chunk, its
// join, sort->pair-hash per chunk, its join.
constexpr int kSyncEvents = 2 * kMaxChunks + 2;
// Tile-prefix arrays of a launch: staged[8] direct[8] s2[8] pchunk[8]
// t2h[8] scan part, each nplots + 1 entries.
constexpr int kTileArrays = 5 * kMaxChunks + 2;
}  // namespace vx

namespace vx {
// Kernel sequence of one or many plots sharing a descriptor array.
struct LaunchSet {
    Desc *descs;
    int n;
    int G, C;  // nonce chunks, partition chunks of the launch (max over plots)
    const uint32_t *t_staged[kMaxChunks], *t_direct[kMaxChunks], *t_s2[kMaxChunks];
    const uint32_t *t_pchunk[kMaxChunks], *t_t2h[kMaxChunks];
    const uint32_t *t_scan, *t_part;  // device tile prefixes
    uint32_t n_staged[kMaxChunks], n_direct[kMaxChunks], n_s2[kMaxChunks];
    uint32_t n_pchunk[kMaxChunks], n_t2h[kMaxChunks];
    uint32_t n_scan, n_part;          // total CTAs
    bool agg;
    int npt;                 // nonces per thread of the staged Table-1 hash launch
    bool fuse_pair_hash;
    bool pair_slots;   // every plot uses the slot placement (t_t2h[0] = slot pair-hash grid)
    bool halo;         // some plot matches across buckets: kernels with the halo code
    bool win;          // some plot is a window: hash kernels with the window filter
    bool list;         // the one plot hashes its window's nonce list (tiled plots)
    uint64_t list_N;   // its nonce count (the list kernel's input)
    uint32_t max_cap2;
    int max_dbits;
    int max_p2;        // widest second scatter level of the launch
};

// Records the (kernel, start, end) events of one run; null = not traced.
struct Trace {
    cudaEvent_t *ev;
    int8_t *kid;
    int *used;
};

// Streams and fork/join events a pipelined run uses; aux = nullptr runs
// everything on `main` one kernel after the other.  aux (high priority)
// takes the second scatter level so its CTAs get SM slots ahead of the
// ALU-bound hash; aux_lo (low priority) takes the pair hash so it only
// fills what the sort leaves.
struct Lanes {
    cudaStream_t main, aux, aux_lo;
    cudaEvent_t *sync;  // kSyncEvents
};

}  // namespace vx

// -------------------------------------------------------------- handle
struct vx_plot {
    int K = 0;
    uint8_t key[32] = {};
    vx_opts opts{};
    vx::Plan plan{};
    uint8_t *d_t1 = nullptr, *d_t2 = nullptr, *d_scratch = nullptr;
    bool owned = false;
    uint64_t t2cap = 0;            // records the bound Table-2 buffer holds
    bool desc_dirty = true;        // descriptor needs an upload
    vx::Desc *h_stage = nullptr;   // pinned staging: Desc + tile prefixes
    cudaEvent_t ev_stage = nullptr;
    bool ev_pending = false;
    cudaStream_t last = nullptr;
    bool have_last = false;
    cudaEvent_t ev_done = nullptr;  // behind vx_plot_run's kernels and result copy
    bool res_pending = false;       // vx_sync reads the pinned result block after ev_done
    int stage = 0;                 // 0 created, 1 Table 1 issued, 2 match issued
    bool t2_known = false;
    uint64_t t2_count = 0;
    bool t1_known = false;          // a window's Table-1 count, read by vx_sync
    uint64_t t1_count = 0;
    const uint8_t *wids = nullptr;  // window id of every nonce (tiled plots): the
                                    // window hashes its listed nonces only
    uint32_t status = 0;
    std::string err;
    // Second streams and fork/join events of the pipelined run.
    cudaStream_t aux = nullptr, aux_lo = nullptr;
    cudaEvent_t sync_ev[vx::kSyncEvents] = {};
    // Called by vx_plot_destroy instead of freeing bound buffers itself when
    // set (the server hands out plots whose memory it accounts for).
    void (*release)(void *ctx, vx_plot *p) = nullptr;
    void *release_ctx = nullptr;
    vx::LaunchSet single{};         // launch set of vx_plot_run on this plot alone
    // Tracing: per run, up to kProfLaunches (kernel id, start, end) records.
    int prof_slots = 0, prof_runs = 0, prof_cur = -1;
    cudaEvent_t *prof_ev = nullptr;   // [slots][kProfLaunches][2]
    int8_t *prof_kid = nullptr;       // [slots][kProfLaunches], -1 = unused
    int *prof_used = nullptr;         // [slots]
};

namespace vx {

// Batch workspace: descs[n] | kTileArrays tile prefixes of n + 1 entries.
size_t batch_ws_bytes(int n);
// Fills the host workspace for plots[0..n) (each bound) and the launch set
// that reads it from d_ws.  Returns VX_OK or VX_EINVAL.
int batch_prepare(vx_plot *const *plots, int n, uint8_t *h_ws, uint8_t *d_ws, LaunchSet *L);
// Whole-plot kernel sequence (sort + match path, pipelined when lanes.aux).
cudaError_t launch_plot_seq(const LaunchSet &L, const Lanes &lanes);
// Creates the two aux streams (highest / lowest priority, non-blocking) and
// kSyncEvents events (timing disabled).
cudaError_t make_lanes(cudaStream_t *aux, cudaStream_t *aux_lo, cudaEvent_t *sync);
void free_lanes(cudaStream_t aux, cudaStream_t aux_lo, cudaEvent_t *sync);
// Marks plots as issued on stream s (vx_sync waits on it).
void mark_issued(vx_plot *const *plots, int n, cudaStream_t s);
int ensure_memory_ext(vx_plot *p);
// Planner with the descriptor size of this build; *why gets a static text.
int make_plan(int K, const vx_opts *o, Plan *pl, const char **why);
// Descriptor of a bound plot; tile prefixes + launch set of plots[0..n)
// (kTileArrays arrays of n + 1 entries at h, read on the device from d).
void fill_desc_ext(const vx_plot *p, Desc *d);
int build_tiles_ext(vx_plot *const *plots, int n, uint32_t *h, const uint32_t *d, LaunchSet *L);
int map_status_ext(uint32_t st);
// Appends plot p's Table 2 (synced) to the open file fd through the pinned
// staging buffer (double-buffered, sequential 4 MB writes); synchronous.
// *d2h (may be null): seconds waiting for device copies.
int write_table2_fd(vx_plot *p, int fd, double *d2h);

}  // namespace vx
