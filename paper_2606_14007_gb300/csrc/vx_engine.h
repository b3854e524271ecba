// vx_engine.h -- internal host-side state shared by the C ABI (vx_api.cu)
// and the plot server (vx_serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "../../include/vaultx.h"
#include "vx_internal.cuh"
#include "vx_plan.h"

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
    vx::Desc *h_stage = nullptr;       // pinned staging: Desc + tile prefixes
    cudaEvent_t ev_stage = nullptr;
    bool ev_pending = false;
    cudaStream_t last = nullptr;
    bool have_last = false;
    int stage = 0;                 // 0 created, 1 Table 1 issued, 2 match issued
    bool t2_known = false;
    uint64_t t2_count = 0;
    uint32_t status = 0;
    std::string err;
    // Called by vx_plot_destroy instead of freeing bound buffers itself when
    // set (the server hands out plots whose memory it accounts for).
    void (*release)(void *ctx, vx_plot *p) = nullptr;
    void *release_ctx = nullptr;
    // Tracing: kProfEvents events per run, `prof_slots` runs.
    int prof_slots = 0, prof_next = 0, prof_runs = 0, prof_cur = -1;
    cudaEvent_t *prof_ev = nullptr;
};

namespace vx {
// Kernels a single-plot run may launch, in launch order (tracing names).
constexpr int kProfKernels = 10;
constexpr int kProfEvents = kProfKernels + 1;
}  // namespace vx


namespace vx {

// Kernel sequence of one or many plots sharing a descriptor array.
struct LaunchSet {
    Desc *descs;
    int n;
    const uint32_t *t_hash, *t_direct, *t_s2, *t_part, *t_scan, *t_t2h;  // tile prefixes (device)
    uint32_t n_hash, n_direct, n_s2, n_part, n_scan, n_t2h;            // n_hash: staged hash CTAs
    bool fuse_pair_hash;
    bool agg;
    uint32_t max_cap2;
    int max_dbits;
};


// Batch workspace: descs[n] | tile prefixes staged[n+1] | direct[n+1] |
// s2[n+1] | part[n+1] | scan[n+1] | t2h[n+1].
size_t batch_ws_bytes(int n);
// Fills the host workspace for plots[0..n) (each bound) and the launch set
// that reads it from d_ws.  Returns VX_OK or VX_EINVAL.
int batch_prepare(vx_plot *const *plots, int n, uint8_t *h_ws, uint8_t *d_ws, LaunchSet *L);
// Whole-plot kernel sequence (fused sort + match) of a launch set.
cudaError_t launch_plot_seq(const LaunchSet &L, cudaStream_t s);
// Marks plots as issued on stream s (vx_sync waits on it).
void mark_issued(vx_plot *const *plots, int n, cudaStream_t s);
int ensure_memory_ext(vx_plot *p);

}  // namespace vx
