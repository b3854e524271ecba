// vx_noalloc.cu -- vx_plot_run_noalloc: a whole plot (Table 1 and Table 2)
// without any allocation, for callers that cannot call cudaMalloc: code
// whose device memory is owned by another allocator under a fixed budget
// (a framework's caching allocator, a pre-reserved pool) and may not be
// bypassed, and latency-critical callers that must not take the implicit
// device-wide synchronisation cudaMalloc can cause.  The caller passes the
// key and the two table buffers; the library's scratch (partition slots,
// counters, offsets, look-back words, the plot descriptor) comes from the
// static device array below instead of vx_plot_bind / vx_plot_alloc.
//
// The paper has no counterpart.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <mutex>

#include "vx_engine.h"

namespace {

// Every GPU that loads the library holds this array until the process
// exits.  64 MiB covers a plot of K <= 22 with the default options.
constexpr size_t kNoAllocScratchBytes = 64ull << 20;
static_assert(kNoAllocScratchBytes == (size_t)VX_NOALLOC_SCRATCH_BYTES, "header and array differ");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};  // device address of the array, per device

// Device address of the array on the current device (in host code the
// array's name is only a host-side stand-in).  Looked up once per device.
cudaError_t scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = ptr;
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int vx_plot_run_noalloc(int K, const uint8_t key[32], const vx_opts *opts, void *d_t1,
                                   void *d_t2, uint64_t t2_capacity, void *stream,
                                   uint64_t *t2_count)
{
    if (!key || !d_t1 || !d_t2) return VX_EINVAL;
    if (((uintptr_t)d_t1 | (uintptr_t)d_t2) % 256 != 0) return VX_EINVAL;
    // A stack handle: no heap, no device allocation.
    vx_plot p;
    const char *why = nullptr;
    if (vx::make_plan(K, opts, &p.plan, &why) != VX_OK) return VX_EINVAL;
    if (p.plan.scratch_bytes > kNoAllocScratchBytes) return VX_EINVAL;  // plot too large
    void *scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) return VX_ECUDA;
    p.K = K;
    memcpy(p.key, key, 32);
    p.d_t1 = (uint8_t *)d_t1;
    p.d_t2 = (uint8_t *)d_t2;
    p.d_scratch = (uint8_t *)scratch;
    p.t2cap = t2_capacity ? t2_capacity : p.plan.t2cap;
    cudaStream_t s = (cudaStream_t)stream;

    // Descriptor and tile prefixes into the array (the array keeps the last
    // call's contents; the key-setup kernel clears every counter, ticket and
    // look-back word a run reads before writing).
    vx::Desc desc;
    vx::fill_desc_ext(&p, &desc);
    uint32_t tiles[vx::kTileArrays * 2];
    vx::LaunchSet L;
    vx_plot *one[1] = {&p};
    const uint32_t *d_tiles = reinterpret_cast<const uint32_t *>(p.d_scratch + p.plan.o_tiles);
    if (vx::build_tiles_ext(one, 1, tiles, d_tiles, &L) != VX_OK) return VX_EINVAL;
    L.descs = reinterpret_cast<vx::Desc *>(p.d_scratch + p.plan.o_desc);
    cudaError_t e = cudaMemcpyAsync(L.descs, &desc, sizeof(desc), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync((void *)d_tiles, tiles, sizeof(tiles), cudaMemcpyHostToDevice, s);
    // One stream, one kernel after the other (no second stream, no events).
    if (e == cudaSuccess) e = vx::launch_plot_seq(L, vx::Lanes{s, nullptr, nullptr, nullptr});
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    uint32_t st = 0;
    uint64_t total = 0;
    if (e == cudaSuccess)
        e = cudaMemcpy(&st, p.d_scratch + p.plan.o_status, sizeof(st), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess)
        e = cudaMemcpy(&total, p.d_scratch + p.plan.o_t2off + 8 * (1ull << p.plan.p), sizeof(total),
                       cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return VX_ECUDA;
    if (t2_count) *t2_count = total;
    return vx::map_status_ext(st);
}
