// Request server: continuous batching of independent TTN propagations on one
// device (declarations and documentation in include/ttn.h).
//
// Each request is a context plus (dt, nsteps).  Requests wait in a FIFO
// queue on the host, holding no device memory.  A request runs on the
// number of thread blocks its context asks for (ttn_get_cluster): one lane
// per block count (1, 2, 4, 8, 16), each lane with its own stream, launch
// table and CUDA graph, so small requests share launches one block each
// while large ones get a cluster, and the lanes' launches overlap on the
// device.  A request is admitted to its lane when a slot is free there and
// its footprint (operator and state arenas, from its plan) fits in the
// budget beside every admitted one; admission allocates from the
// stream-ordered pool and builds the environments on a side stream, so it
// overlaps the launches in flight.  Every launch runs each admitted context
// of the lane for one slice of device time; a context runs whole steps of
// its own dt until the slice is used up or its steps are done, so its
// arithmetic does not depend on which other contexts share the launch.
// After a lane's launch the server retires its finished contexts (time
// stamps read, tensors copied to the host, memory returned to the pool) and
// admits waiting ones before the lane's next launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <thread>
#include <vector>

#include "../../include/ttn.h"
#include "ttn_ctx.hpp"
#include "ttn_launch.h"

namespace {

struct Request {
    int64_t ticket = 0;
    ttn_ctx* ctx = nullptr;
    cudaStream_t user_stream = nullptr;
    double dt = 0.0;
    int nsteps = 0;
    int left = 0;
    size_t footprint = 0;
    double est_step_ns = 0.0;
};

}  // namespace

namespace {

// One lane: every admitted context of one block count, launched together.
struct Lane {
    int cluster = 1;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    std::vector<Request> running;     // admitted, in launch order
    TtnLaunchHdr* h_hdr = nullptr;    // pinned host copies of what a launch reads / writes
    TtnInstance* h_table = nullptr;
    TtnRepOut* h_rep = nullptr;
    TtnLaunchHdr* d_hdr = nullptr;
    TtnInstance* d_table = nullptr;
    TtnRepOut* d_rep = nullptr;
    cudaGraphExec_t graph = nullptr;
    int inflight = 0;                 // contexts in the launch in flight (prefix of `running`)
};

constexpr int kLanes = 5;             // block counts 1, 2, 4, 8, 16

int lane_of(int cluster) {
    int i = 0;
    while ((1 << i) < cluster && i + 1 < kLanes) ++i;
    return i;
}

}  // namespace

struct ttn_server {
    int precision = 0;
    int device = 0;
    int sms = 0;
    size_t budget = 0;
    int max_slots = 0;                // one-block lane; cluster lanes hold what fits at once
    long long slice_ns = 0;
    bool use_graph = false;
    cudaStream_t side_stream = nullptr;

    std::deque<Request> queue;
    Lane lanes[kLanes];
    std::vector<std::pair<int64_t, ttn_status>> finished;
    std::vector<double> lat_ms;

    int64_t next_ticket = 1;
    ttn_server_stats st{};
    std::string err;
};

namespace {

ttn_status srv_fail(ttn_server* s, ttn_status code, const std::string& msg) {
    s->err = msg;
    return code;
}

ttn_status srv_cuda(ttn_server* s, cudaError_t e, const char* what) {
    return srv_fail(s, TTN_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define SCK(call, what)                                       \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return srv_cuda(s, e_, what);  \
    } while (0)

ttn_status status_of(int device_status) {
    if (device_status == 0) return TTN_OK;
    if (device_status == 4) return TTN_E_NOCONV;
    if (device_status == 5) return TTN_E_TIMEOUT;
    return TTN_E_CUDA;
}

// Issue one launch of a lane: table and header in, kernel, per-instance results out.
ttn_status issue(ttn_server* s, Lane& L) {
    SCK(cudaMemcpyAsync(L.d_table, L.h_table, sizeof(TtnInstance) * L.max_slots, cudaMemcpyHostToDevice, L.stream),
        "table upload");
    SCK(cudaMemcpyAsync(L.d_hdr, L.h_hdr, sizeof(TtnLaunchHdr), cudaMemcpyHostToDevice, L.stream), "header upload");
    int e = ttn_launch_program_ex(s->precision, L.cluster, L.d_table, L.d_hdr, L.max_slots, 0.0, -1, 0, L.d_rep,
                                  L.stream);
    if (e) return srv_cuda(s, (cudaError_t)e, "kernel launch");
    SCK(cudaMemcpyAsync(L.h_rep, L.d_rep, sizeof(TtnRepOut) * L.max_slots, cudaMemcpyDeviceToHost, L.stream),
        "result copy");
    return TTN_OK;
}

ttn_status build_graph(ttn_server* s, Lane& L) {
    int e = ttn_program_init();
    if (e) return srv_cuda(s, (cudaError_t)e, "kernel attributes");
    SCK(cudaStreamBeginCapture(L.stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    ttn_status r = issue(s, L);
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamEndCapture(L.stream, &g);
    if (r) { if (g) cudaGraphDestroy(g); return r; }
    if (ce != cudaSuccess) return srv_cuda(s, ce, "end capture");
    ce = cudaGraphInstantiate(&L.graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) return srv_cuda(s, ce, "graph instantiate");
    return TTN_OK;
}

// Create a lane's stream, buffers and graph on first use.  A cluster lane
// holds as many contexts as clusters of its size fit on the device at once.
ttn_status lane_open(ttn_server* s, int li) {
    Lane& L = s->lanes[li];
    if (L.stream) return TTN_OK;
    L.cluster = 1 << li;
    if (L.cluster == 1) {
        L.max_slots = s->max_slots;
    } else {
        int active = 0;
        int e = ttn_cluster_capacity(s->precision, L.cluster, &active);
        if (e) return srv_cuda(s, (cudaError_t)e, "cluster occupancy");
        if (active < 1) return srv_fail(s, TTN_E_INVALID, "clusters of " + std::to_string(L.cluster) +
                                                          " blocks cannot be scheduled on this device");
        L.max_slots = std::min(active, s->max_slots);
    }
    bool ok = cudaStreamCreateWithFlags(&L.stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaHostAlloc((void**)&L.h_hdr, sizeof(TtnLaunchHdr), cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc((void**)&L.h_table, sizeof(TtnInstance) * L.max_slots, cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc((void**)&L.h_rep, sizeof(TtnRepOut) * L.max_slots, cudaHostAllocDefault) == cudaSuccess &&
              cudaMalloc((void**)&L.d_hdr, sizeof(TtnLaunchHdr)) == cudaSuccess &&
              cudaMalloc((void**)&L.d_table, sizeof(TtnInstance) * L.max_slots) == cudaSuccess &&
              cudaMalloc((void**)&L.d_rep, sizeof(TtnRepOut) * L.max_slots) == cudaSuccess;
    if (!ok) return srv_fail(s, TTN_E_OOM, "lane allocation failed");
    std::memset(L.h_table, 0, sizeof(TtnInstance) * L.max_slots);
    std::memset(L.h_hdr, 0, sizeof(TtnLaunchHdr));
    if (s->use_graph) return build_graph(s, L);
    return TTN_OK;
}

void lane_close(Lane& L) {
    if (L.stream) cudaStreamSynchronize(L.stream);
    if (L.graph) cudaGraphExecDestroy(L.graph);
    if (L.h_hdr) cudaFreeHost(L.h_hdr);
    if (L.h_table) cudaFreeHost(L.h_table);
    if (L.h_rep) cudaFreeHost(L.h_rep);
    if (L.d_hdr) cudaFree(L.d_hdr);
    if (L.d_table) cudaFree(L.d_table);
    if (L.d_rep) cudaFree(L.d_rep);
    if (L.stream) cudaStreamDestroy(L.stream);
    L = Lane();
}

// Per-step latencies of a finished request from its device time stamps.
void record_latencies(ttn_server* s, Request& r) {
    int64_t steps = 0;
    const int cap = 4096;
    std::vector<uint64_t> stamps(cap);
    int n = 0;
    if (ttn_step_stats(r.ctx, &steps, nullptr, stamps.data(), std::min(cap, r.nsteps), &n) != TTN_OK) return;
    for (int i = 1; i < n; ++i)
        if (stamps[i] >= stamps[i - 1]) s->lat_ms.push_back((double)(stamps[i] - stamps[i - 1]) * 1e-6);
}

// Finished or failed: stamps, tensors to the host, memory back to the pool.
void retire(ttn_server* s, Request& r, ttn_status code) {
    if (code == TTN_OK) record_latencies(s, r);
    r.ctx->stream = s->side_stream;
    const ttn_status ev = ttn::ctx_evict(r.ctx);
    if (code == TTN_OK && ev != TTN_OK) code = ev;
    if (code != TTN_OK) {
        ttn::ctx_fail(r.ctx, code, "request failed on the device (status " + std::to_string((int)code) + ")");
        r.ctx->failed = true;
    }
    r.ctx->stream = r.user_stream;
    s->st.bytes_in_use -= std::min(s->st.bytes_in_use, r.footprint);
    s->finished.emplace_back(r.ticket, code);
    if (code == TTN_OK) s->st.completed++;
    else s->st.failed++;
}

// Admit queued requests (in arrival order, each to its lane) while a slot is
// free in that lane and the footprint fits in the budget.
ttn_status admit(ttn_server* s) {
    for (auto it = s->queue.begin(); it != s->queue.end();) {
        Request& r = *it;
        Lane& L = s->lanes[lane_of(ttn::ctx_cluster(r.ctx))];
        if (r.footprint > s->budget) {
            s->finished.emplace_back(r.ticket, TTN_E_OOM);
            ttn::ctx_fail(r.ctx, TTN_E_OOM, "request footprint exceeds the server's device-memory budget");
            s->st.failed++;
            it = s->queue.erase(it);
            continue;
        }
        if ((int)L.running.size() >= L.max_slots) { ++it; continue; }      // lane full: later lanes may admit
        if (s->st.bytes_in_use + r.footprint > s->budget) break;
        r.ctx->stream = s->side_stream;
        ttn_status m = ttn::ctx_materialize(r.ctx);
        r.ctx->stream = r.user_stream;
        bool any_running = false;
        for (auto& l : s->lanes) any_running |= !l.running.empty();
        if (m == TTN_E_OOM && any_running) break;   // pool fragmented: retry after retirements
        if (m != TTN_OK) {
            s->finished.emplace_back(r.ticket, m);
            s->st.failed++;
            it = s->queue.erase(it);
            continue;
        }
        s->st.bytes_in_use += r.footprint;
        s->st.peak_bytes = std::max(s->st.peak_bytes, s->st.bytes_in_use);
        L.running.push_back(r);
        it = s->queue.erase(it);
    }
    int64_t run = 0;
    for (auto& l : s->lanes) run += (int64_t)l.running.size();
    s->st.peak_running = std::max<int64_t>(s->st.peak_running, run);
    return TTN_OK;
}

// Account for what a finished launch of a lane did.
ttn_status complete(ttn_server* s, Lane& L) {
    if (!L.inflight) return TTN_OK;
    SCK(cudaStreamSynchronize(L.stream), "launch");
    const int n = L.inflight;
    L.inflight = 0;
    std::vector<Request> keep;
    keep.reserve(L.running.size());
    for (int i = 0; i < (int)L.running.size(); ++i) {
        Request& r = L.running[i];
        if (i >= n) { keep.push_back(r); continue; }
        const TtnRepOut o = L.h_rep[i];
        r.left -= o.reps;
        s->st.steps += o.reps;
        if (o.reps > 0) r.est_step_ns = (double)o.elapsed_ns / o.reps;
        const ttn_status code = status_of(o.status);
        if (code != TTN_OK) retire(s, r, code);
        else if (r.left <= 0) retire(s, r, TTN_OK);
        else keep.push_back(r);
    }
    L.running.swap(keep);
    return TTN_OK;
}

ttn_status launch(ttn_server* s, Lane& L) {
    const int n = (int)L.running.size();
    if (n == 0 || L.inflight) return TTN_OK;
    double longest = 0.0;
    for (int i = 0; i < n; ++i) {
        Request& r = L.running[i];
        TtnInstance in = ttn::make_instance(r.ctx, r.ctx->step_p);
        in.nrep = r.left;
        in.dt = r.dt;
        L.h_table[i] = in;
        longest = std::max(longest, r.est_step_ns);
    }
    // a slice holds at least one step of the slowest admitted context
    L.h_hdr->n = n;
    L.h_hdr->slice_ns = std::max(s->slice_ns, (long long)(1.25 * longest));
    if (s->use_graph) {
        SCK(cudaGraphLaunch(L.graph, L.stream), "graph launch");
    } else {
        ttn_status r = issue(s, L);
        if (r) return r;
    }
    L.inflight = n;
    s->st.launches++;
    return TTN_OK;
}

// Block until some lane's launch has finished (none in flight: return).
void wait_any(ttn_server* s) {
    for (;;) {
        bool any = false;
        for (auto& L : s->lanes) {
            if (!L.inflight) continue;
            any = true;
            if (cudaStreamQuery(L.stream) != cudaErrorNotReady) return;
        }
        if (!any) return;
        std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

ttn_status ttn_server_create(int precision, const ttn_server_opts* opts, ttn_server** out) {
    if (!out) return TTN_E_INVALID;
    *out = nullptr;
    if (precision != TTN_FP64 && precision != TTN_MIXED) return TTN_E_INVALID;
    ttn_server* s = new (std::nothrow) ttn_server();
    if (!s) return TTN_E_OOM;
    cudaGetDevice(&s->device);
    cudaDeviceGetAttribute(&s->sms, cudaDevAttrMultiProcessorCount, s->device);
    size_t free_b = 0, total_b = 0;
    cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { delete s; return TTN_E_CUDA; }
    s->precision = precision;
    s->budget = opts && opts->hbm_budget ? opts->hbm_budget : (size_t)(0.9 * (double)free_b);
    s->max_slots = opts && opts->max_slots > 0 ? opts->max_slots : std::max(1, 2 * s->sms);
    const double ms = opts && opts->slice_ms > 0 ? opts->slice_ms : 20.0;
    s->slice_ns = (long long)(ms * 1e6);
    s->use_graph = opts ? opts->use_graph != 0 : true;
    if (cudaStreamCreateWithFlags(&s->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        lane_open(s, 0) != TTN_OK) {
        ttn_server_destroy(s);
        return TTN_E_CUDA;
    }
    *out = s;
    return TTN_OK;
}

ttn_status ttn_server_submit(ttn_server* s, ttn_ctx* ctx, double dt, int nsteps, const ttn_step_opts* opts,
                             int64_t* ticket) {
    if (!s || !ctx) return TTN_E_INVALID;
    if (ctx->failed) return srv_fail(s, TTN_E_STATE, "context is in a failed state");
    if (!ctx->has_h) return srv_fail(s, TTN_E_STATE, "context has no Hamiltonian");
    if (ctx->precision != s->precision) return srv_fail(s, TTN_E_INVALID, "context precision differs from the server's");
    if (ctx->device != s->device) return srv_fail(s, TTN_E_INVALID, "context lives on another device");
    if (nsteps < 1 || !std::isfinite(dt)) return srv_fail(s, TTN_E_INVALID, "nsteps must be >= 1 and dt finite");
    if (opts) {
        if (opts->expand) return srv_fail(s, TTN_E_INVALID, "the server runs fixed bond dimensions (expand = 0)");
        if (opts->krylov_maxdim > TTN_KMAX) return srv_fail(s, TTN_E_INVALID, "krylov_maxdim must be <= 32");
    }
    for (const Request& r : s->queue)
        if (r.ctx == ctx) return srv_fail(s, TTN_E_INVALID, "context already submitted");
    for (const Lane& L : s->lanes)
        for (const Request& r : L.running)
            if (r.ctx == ctx) return srv_fail(s, TTN_E_INVALID, "context already submitted");
    cudaSetDevice(s->device);
    {
        ttn_status le = lane_open(s, lane_of(ttn::ctx_cluster(ctx)));
        if (le) return le;
    }
    if (ctx->resident) {
        // queued requests hold no device memory
        ttn_status e = ttn::ctx_evict(ctx);
        if (e) return srv_fail(s, e, "could not move the context to the host: " + ctx->err);
    }
    if (opts) {
        ctx->ktol = opts->krylov_tol;
        ctx->qtol = opts->qr_rank_tol;
        ctx->kmax = opts->krylov_maxdim > 0 ? opts->krylov_maxdim : TTN_KMAX;
    }
    ctx->pooled = true;
    Request r;
    r.ticket = s->next_ticket++;
    r.ctx = ctx;
    r.user_stream = ctx->stream;
    r.dt = dt;
    r.nsteps = r.left = nsteps;
    r.footprint = ttn::ctx_footprint(ctx);
    s->queue.push_back(r);
    s->st.submitted++;
    if (ticket) *ticket = r.ticket;
    return TTN_OK;
}

ttn_status ttn_server_pump(ttn_server* s, int* n_running, int* n_queued) {
    if (!s) return TTN_E_INVALID;
    cudaSetDevice(s->device);
    ttn_status r = admit(s);            // overlaps the launches in flight
    if (!r) {
        wait_any(s);
        for (auto& L : s->lanes) {
            if (r) break;
            if (L.inflight && cudaStreamQuery(L.stream) != cudaErrorNotReady) r = complete(s, L);
        }
    }
    if (!r) r = admit(s);               // memory released by retirements
    for (auto& L : s->lanes) {
        if (r) break;
        if (L.stream) r = launch(s, L);
    }
    int running = 0;
    for (auto& L : s->lanes) running += (int)L.running.size();
    if (n_running) *n_running = running;
    if (n_queued) *n_queued = (int)s->queue.size();
    return r;
}

ttn_status ttn_server_drain(ttn_server* s) {
    if (!s) return TTN_E_INVALID;
    for (;;) {
        bool busy = !s->queue.empty();
        for (auto& L : s->lanes) busy |= !L.running.empty() || L.inflight;
        if (!busy) return TTN_OK;
        ttn_status r = ttn_server_pump(s, nullptr, nullptr);
        if (r) return r;
    }
}

ttn_status ttn_server_poll(ttn_server* s, int max, int64_t* tickets, ttn_status* status, int* n) {
    if (!s || !n || max < 0 || (max > 0 && (!tickets || !status))) return TTN_E_INVALID;
    const int k = std::min<int>(max, (int)s->finished.size());
    for (int i = 0; i < k; ++i) {
        tickets[i] = s->finished[i].first;
        status[i] = s->finished[i].second;
    }
    s->finished.erase(s->finished.begin(), s->finished.begin() + k);
    *n = k;
    return TTN_OK;
}

ttn_status ttn_server_get_stats(ttn_server* s, ttn_server_stats* out) {
    if (!s || !out) return TTN_E_INVALID;
    ttn_server_stats st = s->st;
    st.queued = (int64_t)s->queue.size();
    st.running = 0;
    for (auto& L : s->lanes) st.running += (int64_t)L.running.size();
    st.n_latencies = (int64_t)s->lat_ms.size();
    st.p50_step_ms = st.p99_step_ms = 0.0;
    if (!s->lat_ms.empty()) {
        std::vector<double> v = s->lat_ms;
        auto q = [&](double f) {
            size_t i = (size_t)std::min<double>((double)v.size() - 1, std::floor(f * (double)(v.size() - 1) + 0.5));
            std::nth_element(v.begin(), v.begin() + i, v.end());
            return v[i];
        };
        st.p50_step_ms = q(0.50);
        st.p99_step_ms = q(0.99);
    }
    *out = st;
    return TTN_OK;
}

ttn_status ttn_server_latencies(ttn_server* s, double* out_ms, int64_t max, int64_t* n) {
    if (!s || !n || max < 0 || (max > 0 && !out_ms)) return TTN_E_INVALID;
    const int64_t k = std::min<int64_t>(max, (int64_t)s->lat_ms.size());
    std::copy(s->lat_ms.begin(), s->lat_ms.begin() + k, out_ms);
    *n = k;
    return TTN_OK;
}

const char* ttn_server_last_error(const ttn_server* s) { return s ? s->err.c_str() : ""; }

void ttn_server_destroy(ttn_server* s) {
    if (!s) return;
    cudaSetDevice(s->device);
    for (auto& L : s->lanes) {
        if (L.stream) cudaStreamSynchronize(L.stream);
        L.inflight = 0;
        // admitted contexts go back to the host, unfinished
        for (Request& r : L.running) {
            r.ctx->stream = s->side_stream;
            ttn::ctx_evict(r.ctx);
            r.ctx->stream = r.user_stream;
        }
        L.running.clear();
    }
    if (s->side_stream) cudaStreamSynchronize(s->side_stream);
    for (auto& L : s->lanes) lane_close(L);
    if (s->side_stream) cudaStreamDestroy(s->side_stream);
    delete s;
}

}  // extern "C"
