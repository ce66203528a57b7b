#include <chrono>
// Context, error reporting and device allocation helpers of the C ABI.
#include <cudaTypedefs.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <mutex>
#include <thread>

#include "host_pool.h"
#include "internal.h"

namespace pb {

static thread_local char g_err[1024] = "";
static std::atomic<int64_t> g_launches{0};
static thread_local StepGraph* t_capture = nullptr;
static std::atomic<uint64_t> g_ws_gen{1};

uint64_t ws_generation(const uint64_t* d0, const uint64_t* d1) {
    return g_ws_gen.load() + (d0 ? *d0 : 0) + (d1 ? *d1 : 0);
}
void ws_bump() { g_ws_gen.fetch_add(1); }

void count_launch(int n) {
    if (t_capture) t_capture->launches += n;  // runs once per replay, counted then
    else g_launches.fetch_add(n, std::memory_order_relaxed);
}

StepGraph* capturing() { return t_capture; }

void graph_free(StepGraph& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    for (auto& t : g.timers) {
        cudaEventDestroy(t.e0);
        cudaEventDestroy(t.e1);
    }
    g = StepGraph();
}

int graph_capture(StepGraph& g, cudaStream_t s, const std::function<int()>& body, const uint64_t* d0,
                  const uint64_t* d1) {
    graph_free(g);
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        cudaGetLastError();
        g.failed = true;
        return PB_OK;
    }
    const uint64_t gen = ws_generation(d0, d1);
    t_capture = &g;
    const int rc = body();
    t_capture = nullptr;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc == PB_OK && e == cudaSuccess && graph) e = cudaGraphInstantiate(&g.exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (rc != PB_OK || e != cudaSuccess || !g.exec) {
        // nothing of the body ran: the caller runs it directly (a capture that
        // was invalidated reports its error through the body as well)
        cudaGetLastError();
        graph_free(g);
        g.failed = true;
        return PB_OK;
    }
    if (ws_generation(d0, d1) != gen) {  // the body moved a workspace while it was captured
        graph_free(g);
        g.failed = true;
        return PB_OK;
    }
    g.gen = gen;
    return PB_OK;
}

void graph_check(StepGraph& g, const uint64_t* d0, const uint64_t* d1) {
    if (g.exec && g.gen != ws_generation(d0, d1)) graph_free(g);
}

int graph_replay(StepGraph& g, cudaStream_t s) {
    PB_CUDA(cudaGraphLaunch(g.exec, s));
    g_launches.fetch_add(g.launches, std::memory_order_relaxed);
    return PB_OK;
}

int graph_credit(pb_ctx* ctx, StepGraph& g, int j) {
    for (auto& t : g.timers) {
        float ms = 0.0f;
        PB_CUDA(cudaEventElapsedTime(&ms, t.e0, t.e1));
        KernelStats& st = ctx->stats[t.id];
        const double p = t.pairs + t.pairs_j * (double)(j + 1);
        st.ms += ms;
        st.launches += 1;
        st.pairs += p;
        st.ops += p * t.ops;
    }
    return PB_OK;
}

int& arnoldi_j() {
    static thread_local int j = 0;
    return j;
}

int set_error(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

namespace {
HostPool& host_pool() {
    // never destroyed: the workers wait on the pool until the process ends
    static HostPool* pool = new HostPool(host_threads() - 1);
    return *pool;
}
}  // namespace

int host_threads() {
    static const int n = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    return n;
}

void host_parallel(int n, const std::function<void(int)>& f) { host_pool().run(n, f); }

static bool trace_enabled() {
    static const bool on = getenv("PBBEM_TRACE") != nullptr;
    return on;
}

static double wall_ms() {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

PhaseTrace::PhaseTrace(const char* s) : scope(s), t0(0.0), on(trace_enabled()) {
    if (on) {
        cudaDeviceSynchronize();
        t0 = wall_ms();
    }
}

void PhaseTrace::lap(const char* label) {
    if (!on) return;
    cudaDeviceSynchronize();
    const double t = wall_ms();
    fprintf(stderr, "[pbbem] %s/%s %.3f ms\n", scope, label, t - t0);
    t0 = t;
}

void PhaseTrace::note(const char* label, double value) const {
    if (on) fprintf(stderr, "[pbbem] %s/%s %.3e\n", scope, label, value);
}

int dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return PB_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        *p = nullptr;
        cudaGetLastError();
        return set_error(e == cudaErrorMemoryAllocation ? PB_ENOMEM : PB_ECUDA,
                         "cudaMalloc(%zu bytes) failed: %s", bytes, cudaGetErrorString(e));
    }
    return PB_OK;
}

int ws_reserve(Workspace& w, size_t bytes) {
    if (bytes <= w.bytes) return PB_OK;
    if (w.gen) ++*w.gen;
    else g_ws_gen.fetch_add(1);
    ws_free(w);
    PB_TRY(dev_alloc(&w.ptr, bytes));
    w.bytes = bytes;
    return PB_OK;
}

void ws_free(Workspace& w) {
    if (w.ptr) {
        if (w.gen) ++*w.gen;
        else g_ws_gen.fetch_add(1);
    }
    if (w.ptr) cudaFree(w.ptr);
    w.ptr = nullptr;
    w.bytes = 0;
}

}  // namespace pb

using namespace pb;

extern "C" const char* pb_last_error(void) { return g_err; }

extern "C" const char* pb_version(void) { return "pbbem 0.1 sm_103a"; }

extern "C" int pb_init(int device, pb_ctx** out) {
    if (!out) return set_error(PB_EINVAL, "pb_init: out is NULL");
    *out = nullptr;
    int n = 0;
    PB_CUDA(cudaGetDeviceCount(&n));
    if (device < 0 || device >= n) return set_error(PB_EINVAL, "pb_init: device %d of %d", device, n);
    PB_CUDA(cudaSetDevice(device));
    pb_ctx* c = new pb_ctx();
    c->device = device;
    cudaDeviceProp prop;
    cudaError_t e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete c;
        return set_error(PB_ECUDA, "cudaGetDeviceProperties: %s", cudaGetErrorString(e));
    }
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
        delete c;
        return set_error(PB_ECUDA, "cuTensorMapEncodeTiled entry point unavailable");
    }
    c->encode_tiled = fn;
    const char* pk = getenv("PBBEM_PAIR_KERNEL");
    if (pk && pk[0] == '1') c->pair_kernel = 1;
    const char* gr = getenv("PBBEM_GRAPHS");
    if (gr && gr[0] == '0') c->graphs = 0;
    const char* tc = getenv("PBBEM_TREECODE");
    if (tc && tc[0] == '0') c->tree_enable = 0;
    *out = c;
    return PB_OK;
}

static void reset_stats(pb_ctx* ctx) {
    for (auto& st : ctx->stats) {
        for (auto& e : st.events) {
            cudaEventDestroy(e.first);
            cudaEventDestroy(e.second);
        }
        st = KernelStats();
    }
}

extern "C" int pb_free_ctx(pb_ctx* ctx) {
    if (ctx) reset_stats(ctx);
    delete ctx;
    return PB_OK;
}

extern "C" int pb_profile(pb_ctx* ctx, int enable) {
    if (!ctx) return set_error(PB_EINVAL, "pb_profile: NULL context");
    reset_stats(ctx);
    ctx->profile = enable ? 1 : 0;
    return PB_OK;
}

extern "C" int pb_profile_read(pb_ctx* ctx, int kernel, int64_t* launches, double* total_ms, double* pairs,
                               double* ops) {
    if (!ctx || kernel < 0 || kernel >= PB_KERNEL_COUNT) return set_error(PB_EINVAL, "pb_profile_read: bad argument");
    KernelStats& st = ctx->stats[kernel];
    for (auto& e : st.events) {
        float ms = 0.0f;
        PB_CUDA(cudaEventSynchronize(e.second));
        PB_CUDA(cudaEventElapsedTime(&ms, e.first, e.second));
        st.ms += ms;
        cudaEventDestroy(e.first);
        cudaEventDestroy(e.second);
    }
    st.events.clear();
    if (launches) *launches = st.launches;
    if (total_ms) *total_ms = st.ms;
    if (pairs) *pairs = st.pairs;
    if (ops) *ops = st.ops;
    return PB_OK;
}

extern "C" int64_t pb_launch_count(void) { return g_launches.load(); }

extern "C" int pb_set_treecode(pb_ctx* ctx, int enable, int order, double theta, int64_t min_points) {
    if (!ctx) return set_error(PB_EINVAL, "pb_set_treecode: NULL context");
    if (order < 2 || order > 7 || !(theta > 0.0 && theta <= 1.0) || min_points < 0)
        return set_error(PB_EINVAL, "pb_set_treecode: need order in 2..7, theta in (0, 1], min_points >= 0");
    ctx->tree_enable = enable ? 1 : 0;
    ctx->tree_order = order;
    ctx->tree_theta = theta;
    ctx->tree_min_points = min_points;
    return PB_OK;
}

extern "C" int pb_tree_info(const pb_mesh* m, int64_t out[6]) {
    if (!m || !out) return set_error(PB_EINVAL, "pb_tree_info: NULL argument");
    return tree_info(m, out);
}

extern "C" int pb_set_graphs(pb_ctx* ctx, int enable) {
    if (!ctx) return set_error(PB_EINVAL, "pb_set_graphs: NULL context");
    ctx->graphs = enable ? 1 : 0;
    return PB_OK;
}
