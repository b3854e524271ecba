// vx_serve.cu -- continuous-batching plot server.
//
// Requests (K, key) queue on the host.  Each step: finished waves are
// retired (their plots become DONE or FAILED), queued requests are admitted
// in arrival order while their device footprint fits the free memory budget
// and the in-flight limit allows, and admitted plots are launched as a wave
// (one grouped launch of the whole kernel sequence over all of them) on a
// free stream.  Waves on different streams overlap on the device, so
// requests arriving while others run join the next wave as soon as memory
// and a stream free up.  Tables stay on the device until the caller takes
// the plot handle and destroys it; destroying it returns its memory to the
// server's budget.
//
// The paper plots one K at a time (Sec. III-A) and checks each allocation
// against a device limit before making it (Sec. III-C); admission by
// footprint is that check applied to a queue of plots.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "vx_engine.h"

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Memory accounting that outlives the server while handed-out plots live.
struct Shared {
    std::mutex mu;
    uint64_t budget = 0, used = 0;
    uint32_t inflight = 0;
    cudaMemPool_t pool = nullptr;
    cudaStream_t free_stream = nullptr;
    ~Shared()
    {
        if (free_stream) cudaStreamSynchronize(free_stream);
        if (pool) cudaMemPoolDestroy(pool);
        if (free_stream) cudaStreamDestroy(free_stream);
    }
};

struct Req {
    uint64_t ticket = 0;
    int K = 0;
    uint8_t key[32];
    int state = VX_QUEUED;
    vx_plot *plot = nullptr;
    uint64_t bytes = 0;
    double t_submit = 0, t_done = 0;
    bool handed = false;
};

struct Wave;

struct Lane {  // one stream (plus its pipeline's second stream), one wave at a time
    cudaStream_t stream = nullptr;
    cudaStream_t aux = nullptr, aux_lo = nullptr;
    cudaEvent_t sync[vx::kSyncEvents] = {};
    uint8_t *h_ws = nullptr, *d_ws = nullptr;
    Wave *wave = nullptr;
};

struct Wave {
    std::vector<Req *> reqs;
    std::atomic<int> done{0};
    std::atomic<double> t_done{0.0};
};

struct Release {  // release hook context: one per handed-in plot
    std::shared_ptr<Shared> sh;
    uint64_t bytes;
    void *t1, *t2, *scratch;
    bool inflight = true;  // counted in Shared::inflight until handed to the caller
};

void CUDART_CB on_wave_done(void *arg)
{
    Wave *w = static_cast<Wave *>(arg);
    w->t_done.store(now_s());
    w->done.store(1);
}

void release_plot(void *ctx, vx_plot *p)
{
    Release *r = static_cast<Release *>(ctx);
    {
        std::lock_guard<std::mutex> lk(r->sh->mu);
        cudaFreeAsync(r->t1, r->sh->free_stream);
        cudaFreeAsync(r->t2, r->sh->free_stream);
        cudaFreeAsync(r->scratch, r->sh->free_stream);
        r->sh->used -= r->bytes;
        if (r->inflight) r->sh->inflight -= 1;
    }
    // The buffers belong to the server's pool, not to the plot.
    p->d_t1 = p->d_t2 = p->d_scratch = nullptr;
    p->owned = false;
    p->release = nullptr;
    delete r;
}

}  // namespace

struct vx_server {
    vx_serve_opts opts;
    std::shared_ptr<Shared> sh;
    std::vector<Lane> lanes;
    std::deque<Req *> queue;
    std::vector<Req *> admitted;  // allocated, not yet launched
    std::unordered_map<uint64_t, Req *> reqs;
    uint64_t next_ticket = 1;
    cudaStream_t alloc_stream = nullptr;
    cudaEvent_t alloc_ev = nullptr;
    std::mutex mu;
};

namespace {

int admit_one(vx_server *S, Req *r)
{
    vx_plot *p = nullptr;
    const vx_opts *po = S->opts.plot_opts.size ? &S->opts.plot_opts : nullptr;
    int rc = vx_plot_create(r->K, r->key, po, &p);
    if (rc) return rc;
    uint64_t t1 = 0, t2 = 0, sc = 0;
    vx_plot_required_bytes(r->K, po, &t1, &t2, &sc);
    void *a = nullptr, *b = nullptr, *c = nullptr;
    Shared &sh = *S->sh;
    cudaError_t e = cudaMallocFromPoolAsync(&a, t1, sh.pool, S->alloc_stream);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&b, t2, sh.pool, S->alloc_stream);
    if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&c, sc, sh.pool, S->alloc_stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaFreeAsync(a, S->alloc_stream);
        if (b) cudaFreeAsync(b, S->alloc_stream);
        vx_plot_destroy(p);
        return VX_ENOMEM;
    }
    rc = vx_plot_bind(p, a, b, c, 0);
    if (rc) {
        cudaFreeAsync(a, S->alloc_stream);
        cudaFreeAsync(b, S->alloc_stream);
        cudaFreeAsync(c, S->alloc_stream);
        vx_plot_destroy(p);
        return rc;
    }
    Release *rel = new Release{S->sh, r->bytes, a, b, c};
    p->release = release_plot;
    p->release_ctx = rel;
    r->plot = p;
    return VX_OK;
}

void retire(vx_server *S)
{
    for (Lane &L : S->lanes) {
        Wave *w = L.wave;
        if (!w || !w->done.load()) continue;
        for (Req *r : w->reqs) {
            const int rc = vx_sync(r->plot);
            r->state = rc == VX_OK ? VX_DONE : VX_FAILED;
            r->t_done = w->t_done.load();
        }
        delete w;
        L.wave = nullptr;
    }
}

void admit(vx_server *S)
{
    bool any = false;
    while (!S->queue.empty()) {
        Req *r = S->queue.front();
        {
            std::lock_guard<std::mutex> lk(S->sh->mu);
            if (S->sh->inflight >= S->opts.max_inflight) break;
            if (S->sh->used + r->bytes > S->sh->budget) break;
            S->sh->used += r->bytes;
            S->sh->inflight += 1;
        }
        S->queue.pop_front();
        if (admit_one(S, r) != VX_OK) {
            std::lock_guard<std::mutex> lk(S->sh->mu);
            S->sh->used -= r->bytes;
            S->sh->inflight -= 1;
            r->state = VX_FAILED;
            r->t_done = now_s();
            continue;
        }
        S->admitted.push_back(r);
        any = true;
    }
    if (any) cudaEventRecord(S->alloc_ev, S->alloc_stream);
}

void launch(vx_server *S)
{
    for (Lane &L : S->lanes) {
        if (S->admitted.empty()) return;
        if (L.wave) continue;
        const size_t n = std::min<size_t>(S->admitted.size(), S->opts.max_wave);
        Wave *w = new Wave();
        w->reqs.assign(S->admitted.begin(), S->admitted.begin() + n);
        S->admitted.erase(S->admitted.begin(), S->admitted.begin() + n);
        std::vector<vx_plot *> plots;
        for (Req *r : w->reqs) plots.push_back(r->plot);
        vx::LaunchSet LS;
        cudaError_t e = cudaStreamWaitEvent(L.stream, S->alloc_ev, 0);
        int rc = vx::batch_prepare(plots.data(), (int)n, L.h_ws, L.d_ws, &LS);
        if (e == cudaSuccess && rc == VX_OK)
            e = cudaMemcpyAsync(L.d_ws, L.h_ws, vx::batch_ws_bytes((int)n), cudaMemcpyHostToDevice,
                                L.stream);
        if (e == cudaSuccess && rc == VX_OK) e = vx::launch_plot_seq(LS, vx::Lanes{L.stream, L.aux, L.aux_lo, L.sync});
        if (e == cudaSuccess && rc == VX_OK) e = cudaLaunchHostFunc(L.stream, on_wave_done, w);
        if (e != cudaSuccess || rc != VX_OK) {
            cudaGetLastError();
            for (Req *r : w->reqs) {
                r->state = VX_FAILED;
                r->t_done = now_s();
            }
            delete w;
            continue;
        }
        vx::mark_issued(plots.data(), (int)n, L.stream);
        for (Req *r : w->reqs) r->state = VX_RUNNING;
        L.wave = w;
    }
}

void advance(vx_server *S)
{
    retire(S);
    admit(S);
    launch(S);
}

}  // namespace

extern "C" {

int vx_serve_create(const vx_serve_opts *o, vx_server **out)
{
    if (!out) return VX_EINVAL;
    *out = nullptr;
    vx_serve_opts opts;
    memset(&opts, 0, sizeof(opts));
    if (o) {
        if (o->size != 0 && o->size < sizeof(vx_serve_opts)) return VX_EINVAL;
        memcpy(&opts, o, sizeof(opts));
    }
    // Measured at 200 req/s (K 22..29, saturated): 2..8 plots in flight
    // serve 14.0-14.15 G nonces/s, 64 only 12.4 (the resident plots' working
    // sets crowd each other out of L2); plotting one at a time gives 13.9.
    if (!opts.max_inflight) opts.max_inflight = 4;
    if (!opts.streams) opts.streams = 2;
    if (!opts.max_wave) opts.max_wave = 32;
    if (opts.streams > 16 || opts.max_wave > 4096) return VX_EINVAL;
    // Requests are whole plots: a window option would make every one the
    // same window of its plot.
    if (opts.plot_opts.window_bits || opts.plot_opts.window) return VX_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VX_ECUDA;
    if (!opts.memory_budget) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return VX_ECUDA;
        opts.memory_budget = (uint64_t)(0.8 * (double)fr);
    }
    vx_server *S = new vx_server();
    S->opts = opts;
    S->sh = std::make_shared<Shared>();
    S->sh->budget = opts.memory_budget;
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaError_t e = cudaMemPoolCreate(&S->sh->pool, &props);
    uint64_t keep = UINT64_MAX;  // keep freed memory in the pool for the next plots
    if (e == cudaSuccess) e = cudaMemPoolSetAttribute(S->sh->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->sh->free_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->alloc_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->alloc_ev, cudaEventDisableTiming);
    const size_t ws = vx::batch_ws_bytes((int)opts.max_wave);
    S->lanes.resize(opts.streams);
    for (Lane &L : S->lanes) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = vx::make_lanes(&L.aux, &L.aux_lo, L.sync);
        if (e == cudaSuccess) e = cudaMallocHost((void **)&L.h_ws, ws);
        if (e == cudaSuccess) e = cudaMalloc((void **)&L.d_ws, ws);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        vx_serve_destroy(S);
        return e == cudaErrorMemoryAllocation ? VX_ENOMEM : VX_ECUDA;
    }
    *out = S;
    return VX_OK;
}

int vx_serve_submit(vx_server *S, int K, const uint8_t key[32], uint64_t *ticket)
{
    if (!S || !key || !ticket) return VX_EINVAL;
    const vx_opts *po = S->opts.plot_opts.size ? &S->opts.plot_opts : nullptr;
    uint64_t t1 = 0, t2 = 0, sc = 0;
    if (vx_plot_required_bytes(K, po, &t1, &t2, &sc) != VX_OK) return VX_EINVAL;
    if (t1 + t2 + sc > S->sh->budget) return VX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    Req *r = new Req();
    r->ticket = S->next_ticket++;
    r->K = K;
    memcpy(r->key, key, 32);
    r->bytes = t1 + t2 + sc;
    r->t_submit = now_s();
    S->reqs[r->ticket] = r;
    S->queue.push_back(r);
    *ticket = r->ticket;
    return VX_OK;
}

int vx_serve_step(vx_server *S)
{
    if (!S) return VX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    advance(S);
    int pending = 0;
    for (auto &kv : S->reqs)
        if (!kv.second->handed) ++pending;
    return pending;
}

int vx_serve_poll(vx_server *S, uint64_t ticket, int *state, vx_plot **out)
{
    if (!S || !state) return VX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    advance(S);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return VX_EINVAL;
    Req *r = it->second;
    *state = r->state;
    if (out) *out = nullptr;
    if (r->state == VX_DONE && out && !r->handed) {
        *out = r->plot;
        r->handed = true;
        // Fetched: no longer in flight (its memory stays charged to the
        // budget until the caller destroys it).
        Release *rel = static_cast<Release *>(r->plot->release_ctx);
        std::lock_guard<std::mutex> lk2(S->sh->mu);
        if (rel && rel->inflight) {
            rel->inflight = false;
            S->sh->inflight -= 1;
        }
    }
    if (r->state == VX_FAILED && r->plot && !r->handed) {
        vx_plot_destroy(r->plot);   // returns its memory to the budget
        r->plot = nullptr;
        r->handed = true;
    }
    return VX_OK;
}

int vx_serve_latency(vx_server *S, uint64_t ticket, double *seconds)
{
    if (!S || !seconds) return VX_EINVAL;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end()) return VX_EINVAL;
    Req *r = it->second;
    if (r->state != VX_DONE && r->state != VX_FAILED) return VX_ENOTREADY;
    *seconds = r->t_done - r->t_submit;
    return VX_OK;
}

void vx_serve_destroy(vx_server *S)
{
    if (!S) return;
    for (Lane &L : S->lanes)
        if (L.stream) cudaStreamSynchronize(L.stream);
    {
        std::lock_guard<std::mutex> lk(S->mu);
        retire(S);
        for (auto &kv : S->reqs) {
            Req *r = kv.second;
            if (r->plot && !r->handed) vx_plot_destroy(r->plot);
            delete r;
        }
        S->reqs.clear();
    }
    for (Lane &L : S->lanes) {
        if (L.wave) delete L.wave;
        vx::free_lanes(L.aux, L.aux_lo, L.sync);
        if (L.stream) cudaStreamDestroy(L.stream);
        if (L.h_ws) cudaFreeHost(L.h_ws);
        if (L.d_ws) cudaFree(L.d_ws);
    }
    if (S->alloc_stream) {
        cudaStreamSynchronize(S->alloc_stream);
        cudaStreamDestroy(S->alloc_stream);
    }
    if (S->alloc_ev) cudaEventDestroy(S->alloc_ev);
    delete S;   // the pool goes when the last handed-out plot is destroyed
}

}  // extern "C"
