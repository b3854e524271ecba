// vx_tiled.cu -- a whole plot built one window at a time in device memory
// (chunked VRAM tiling, the paper's third direction of future work, Sec. V).
//
// A window is a run of whole logical buckets: the records whose key64 has
// its top c bits equal to the window index.  The bucket-scope match never
// leaves a bucket, so each window's Table 1 and Table 2 are exactly the
// whole plot's tables restricted to its buckets, and the windows in index
// order concatenate to the whole plot's tables (Table 1 in (key64, nonce)
// order, Table 2 in bucket order).  Each window hashes every nonce again and
// keeps its own share: on GB300 hashing 2^31 nonces takes ~51 ms, less than
// moving the 26 GB of unsorted records across the host link once, so
// recomputing beats spilling the records and reading them back.
//
// A first pass hashes every nonce once and stores its window (one byte);
// each window then lists its own nonces from those bytes and hashes only
// them, so a plot of 2^c windows costs two hashes of every nonce, not 2^c.
// (Without the byte array -- more than 8 window bits, or the hash split
// into nonce chunks -- each window hashes every nonce and keeps its share.)
//
// Two window plots alternate: while one computes on the caller's stream, the
// other's tables go to the host -- into the caller's memory on a copy stream
// of the library's own, or (Table 2) appended to a flat plot file through
// the pinned staging buffer, as vx_plot_write does for a whole plot
// (Sec. III-A, III-B: 4 MB sequential chunks, 256 MB pinned staging).
#include <cuda_runtime.h>
#include <fcntl.h>
#include <unistd.h>

#include <chrono>
#include <cstring>

#include "vx_engine.h"

namespace {

int window_opts(const vx_opts *opts, int window_bits, vx_opts *o)
{
    if (window_bits < 0 || window_bits > 16) return VX_EINVAL;
    if (opts) {
        if (opts->size != 0 && opts->size < sizeof(vx_opts)) return VX_EINVAL;
        memcpy(o, opts, sizeof(vx_opts));
        if (o->window_bits || o->window) return VX_EINVAL;  // the argument sets them
    } else {
        vx_opts_default(o);
    }
    o->size = sizeof(vx_opts);
    o->window_bits = (uint32_t)window_bits;
    o->window = 0;
    return VX_OK;
}

// Where each window's Table 2 goes: host memory (t2, t2_bytes long; copied
// asynchronously) or the open file fd (written before the next window's
// buffers are reused).
struct Sink {
    uint8_t *t2 = nullptr;
    uint64_t t2_bytes = 0;
    int fd = -1;
};

// Whether a tiled plot stores window ids (one byte per nonce) and lists
// each window's nonces from them.
bool use_ids(const vx::Plan &pl) { return pl.wbits >= 1 && pl.wbits <= 8 && pl.hchunks == 1; }

uint64_t ids_bytes(const vx::Plan &pl) { return use_ids(pl) ? vx::round_up(pl.N, 256) : 0; }

int tiled_run(int K, const uint8_t key[32], const vx_opts *opts, int window_bits, void *d_work,
              uint64_t work_bytes, void *host_t1, uint64_t host_t1_bytes, const Sink &sink,
              uint64_t *t1_count, uint64_t *t2_count, void *stream)
{
    if (!key) return VX_EINVAL;
    vx_opts o;
    if (window_opts(opts, window_bits, &o) != VX_OK) return VX_EINVAL;
    vx::Plan pl;
    const char *why = nullptr;
    if (vx::make_plan(K, &o, &pl, &why) != VX_OK) return VX_EINVAL;
    const uint64_t N = 1ull << K;
    if (host_t1 && host_t1_bytes < 12 * N) return VX_EINVAL;
    const uint32_t nw = 1u << window_bits;
    const int nbuf = nw > 1 ? 2 : 1;
    // Window buffers: caller-owned work memory cut into nbuf sets of
    // (Table 1, Table 2, scratch) and the window ids, or library-owned ones
    // for this call.
    const uint64_t one = pl.t1_bytes + pl.t2_bytes + pl.scratch_bytes;
    const uint64_t idb = ids_bytes(pl);
    if (d_work && (work_bytes < one * nbuf + idb || ((uintptr_t)d_work & 255u))) return VX_EINVAL;
    uint8_t *ids = nullptr;
    bool own_ids = false;

    vx_plot *P[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    cudaEvent_t copied[2] = {nullptr, nullptr};
    int rc = VX_OK;
    for (int i = 0; i < nbuf && rc == VX_OK; ++i) {
        rc = vx_plot_create(K, key, &o, &P[i]);
        if (rc != VX_OK) break;
        if (d_work) {
            uint8_t *b = (uint8_t *)d_work + one * i;  // plan sizes are multiples of 256
            rc = vx_plot_bind(P[i], b, b + pl.t1_bytes, b + pl.t1_bytes + pl.t2_bytes, 0);
        } else {
            rc = vx_plot_alloc(P[i]);
        }
    }
    if (rc == VX_OK && cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) rc = VX_ECUDA;
    for (int i = 0; i < nbuf && rc == VX_OK; ++i)
        if (cudaEventCreateWithFlags(&copied[i], cudaEventDisableTiming) != cudaSuccess) rc = VX_ECUDA;

    cudaStream_t s = (cudaStream_t)stream;
    if (rc == VX_OK && idb) {
        if (d_work) {
            ids = (uint8_t *)d_work + one * nbuf;
        } else if (cudaMalloc((void **)&ids, idb) == cudaSuccess) {
            own_ids = true;
        } else {
            cudaGetLastError();
            rc = VX_ENOMEM;
        }
        if (rc == VX_OK) {
            uint32_t kw[8];
            for (int i = 0; i < 8; ++i)
                kw[i] = (uint32_t)key[4 * i] | ((uint32_t)key[4 * i + 1] << 8) |
                        ((uint32_t)key[4 * i + 2] << 16) | ((uint32_t)key[4 * i + 3] << 24);
            if (vx::launch_window_ids(kw, N, window_bits, ids, s) != cudaSuccess) rc = VX_ECUDA;
            for (int i = 0; i < nbuf; ++i) P[i]->wids = ids;
        }
    }
    uint64_t off1 = 0, off2 = 0;
    bool t2_full = false;
    // Waits for window plot X (its own completion event only, so the window
    // queued behind it keeps the GPU busy), then sends its tables on: Table 1
    // (and Table 2 into host memory) as copies on the copy stream, Table 2
    // into the file through the staging buffer.
    auto drain = [&](int slot) -> int {
        vx_plot *X = P[slot];
        int r = vx_sync(X);
        if (r != VX_OK) return r;
        const uint64_t n1 = X->t1_count, n2 = X->t2_count;
        if (off1 + n1 > N) return VX_EOVERFLOW;  // more records than nonces: never in a valid run
        if (host_t1 && n1 &&
            cudaMemcpyAsync((uint8_t *)host_t1 + 12 * off1, X->d_t1, 12 * n1, cudaMemcpyDeviceToHost,
                            cs) != cudaSuccess)
            return VX_ECUDA;
        if (sink.fd >= 0) {
            if ((r = vx::write_table2_fd(X, sink.fd, nullptr)) != VX_OK) return r;
        } else {
            if (16 * (off2 + n2) > sink.t2_bytes) t2_full = true;
            if (!t2_full && n2 &&
                cudaMemcpyAsync(sink.t2 + 16 * off2, X->d_t2, 16 * n2, cudaMemcpyDeviceToHost, cs) !=
                    cudaSuccess)
                return VX_ECUDA;
        }
        off1 += n1;
        off2 += n2;
        return cudaEventRecord(copied[slot], cs) == cudaSuccess ? VX_OK : VX_ECUDA;
    };
    for (uint32_t w = 0; w < nw && rc == VX_OK; ++w) {
        const int slot = (int)(w & 1u);
        vx_plot *X = P[slot];
        // The buffers of window w - 2 are free once its copies are done.
        if (w >= 2 && cudaStreamWaitEvent(s, copied[slot], 0) != cudaSuccess) {
            rc = VX_ECUDA;
            break;
        }
        X->plan.win = w;
        X->opts.window = w;
        X->desc_dirty = true;
        rc = vx_plot_run(X, s);
        if (rc == VX_OK && w >= 1) rc = drain(slot ^ 1);
    }
    if (rc == VX_OK) rc = drain((int)((nw - 1) & 1u));
    if (cs && cudaStreamSynchronize(cs) != cudaSuccess && rc == VX_OK) rc = VX_ECUDA;
    if (rc == VX_OK && off1 != N) rc = VX_EOVERFLOW;  // every nonce in exactly one window
    if (rc == VX_OK && t2_full) rc = VX_ENOMEM;     // *t2_count says how much is needed
    if (t1_count) *t1_count = off1;
    if (t2_count) *t2_count = off2;

    // Nothing of this call may still run when it returns (the caller owns
    // d_work): the window plots wait for their own work, the stream for the
    // id pass queued before them.
    for (int i = 0; i < 2; ++i) {
        if (copied[i]) cudaEventDestroy(copied[i]);
        vx_plot_destroy(P[i]);
    }
    if (ids) cudaStreamSynchronize(s);
    if (own_ids) cudaFree(ids);
    if (cs) cudaStreamDestroy(cs);
    return rc;
}

}  // namespace

extern "C" int vx_plot_tiled_bytes(int K, const vx_opts *opts, int window_bits,
                                   uint64_t *device_bytes, uint64_t *host_t1_bytes,
                                   uint64_t *host_t2_bytes)
{
    vx_opts o;
    if (window_opts(opts, window_bits, &o) != VX_OK) return VX_EINVAL;
    vx::Plan pl;
    const char *why = nullptr;
    if (vx::make_plan(K, &o, &pl, &why) != VX_OK) return VX_EINVAL;
    const uint64_t nw = 1ull << window_bits;
    const uint64_t one = pl.t1_bytes + pl.t2_bytes + pl.scratch_bytes;
    if (device_bytes) *device_bytes = one * (nw > 1 ? 2 : 1) + ids_bytes(pl);
    if (host_t1_bytes) *host_t1_bytes = 12ull << K;
    if (host_t2_bytes) *host_t2_bytes = 16 * pl.t2cap * nw;
    return VX_OK;
}

extern "C" int vx_plot_tiled_hash_passes(int K, const vx_opts *opts, int window_bits, uint32_t *passes)
{
    if (!passes) return VX_EINVAL;
    vx_opts o;
    if (window_opts(opts, window_bits, &o) != VX_OK) return VX_EINVAL;
    vx::Plan pl;
    const char *why = nullptr;
    if (vx::make_plan(K, &o, &pl, &why) != VX_OK) return VX_EINVAL;
    // whole plot: once; window ids: the id pass and the window's own list;
    // else every window hashes every nonce and keeps its share
    *passes = window_bits == 0 ? 1u : use_ids(pl) ? 2u : (1u << window_bits);
    return VX_OK;
}

extern "C" int vx_plot_tiled_window_bits_capped(int K, const vx_opts *opts, uint64_t budget_bytes,
                                                uint32_t max_hash_passes, int *window_bits)
{
    if (!window_bits || max_hash_passes == 0) return VX_EINVAL;
    // Fewest windows first: the device footprint falls with every extra bit
    // (one bit is the exception: two half-plot buffers are no smaller than one
    // whole plot), and each extra window costs a little time.
    for (int c = 0; c <= 16; ++c) {
        uint64_t dev = 0;
        uint32_t passes = 0;
        if (vx_plot_tiled_bytes(K, opts, c, &dev, nullptr, nullptr) != VX_OK) break;
        if (vx_plot_tiled_hash_passes(K, opts, c, &passes) != VX_OK) break;
        if (dev <= budget_bytes && passes <= max_hash_passes) {
            *window_bits = c;
            return VX_OK;
        }
    }
    return VX_ENOMEM;
}

extern "C" int vx_plot_tiled_window_bits(int K, const vx_opts *opts, uint64_t budget_bytes,
                                         int *window_bits)
{
    // At most two hashes of every nonce (the window-id path): above 8 window
    // bits each window would hash the whole plot again.
    return vx_plot_tiled_window_bits_capped(K, opts, budget_bytes, 2, window_bits);
}

extern "C" int vx_plot_tiled(int K, const uint8_t key[32], const vx_opts *opts, int window_bits,
                             void *d_work, uint64_t work_bytes, void *host_t1,
                             uint64_t host_t1_bytes, void *host_t2, uint64_t host_t2_bytes,
                             uint64_t *t1_count, uint64_t *t2_count, void *stream)
{
    if (!host_t2) return VX_EINVAL;
    Sink sink;
    sink.t2 = (uint8_t *)host_t2;
    sink.t2_bytes = host_t2_bytes;
    return tiled_run(K, key, opts, window_bits, d_work, work_bytes, host_t1, host_t1_bytes, sink,
                     t1_count, t2_count, stream);
}

extern "C" int vx_plot_tiled_write(int K, const uint8_t key[32], const vx_opts *opts,
                                   int window_bits, void *d_work, uint64_t work_bytes,
                                   const char *path, void *host_t1, uint64_t host_t1_bytes,
                                   uint64_t *t1_count, uint64_t *t2_count, double *seconds,
                                   void *stream)
{
    if (!path) return VX_EINVAL;
    vx_opts o;  // reject bad arguments before the file is created
    if (!key || window_opts(opts, window_bits, &o) != VX_OK) return VX_EINVAL;
    const auto t0 = std::chrono::steady_clock::now();
    Sink sink;
    sink.fd = open(path, O_WRONLY | O_CREAT | O_TRUNC, 0644);
    if (sink.fd < 0) return VX_EIO;
    int rc = tiled_run(K, key, opts, window_bits, d_work, work_bytes, host_t1, host_t1_bytes, sink,
                       t1_count, t2_count, stream);
    if (close(sink.fd) != 0 && rc == VX_OK) rc = VX_EIO;  // deferred write-back errors
    if (seconds)
        *seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return rc;
}
