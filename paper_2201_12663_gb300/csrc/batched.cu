// batched.cu -- many independent canonical tensors in one call (rhosvd_c2t_batched).
//
// A reduction is a chain of ~60 launches, several of them single-block factorisations that
// leave most SMs idle.  Independent tensors fill the GPU by running side by side: a host-side
// scheduler assigns the tensors to L stream lanes by longest-processing-time first (cost model:
// the two passes over U, 3 n R, plus a fixed term for the sequential small factorisations), each
// lane running its tensors in order on its own slice of the workspace.  The whole fork/join
// sequence is captured once into a CUDA graph (relaxed capture mode) and the executable graph is
// cached under the call's arguments, so a repeated batch is one graph launch.  With lanes <= 0
// the lane count is autotuned on the first call for a batch shape: candidates are launched and
// timed once each (4, 8, 16, 32 below the maximum, and the maximum; a synchronising step), and
// the fastest is remembered for that shape.
// Optional per-tensor completion events (rhosvd_batch_latency_*) give latency percentiles.
#include "internal.cuh"

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

namespace {

constexpr int LANES_MAX = 32;
constexpr size_t ALIGN = 256;

size_t up_align(size_t b) { return (b + ALIGN - 1) / ALIGN * ALIGN; }

struct Lanes {
    int device = -1;
    cudaStream_t origin = nullptr;
    cudaStream_t s[LANES_MAX] = {};
    cudaEvent_t fork = nullptr, after = nullptr, before = nullptr;
    cudaEvent_t join[LANES_MAX] = {};
    cudaEvent_t t0 = nullptr;
    std::vector<cudaEvent_t> done;
};

struct Cached {
    cudaGraphExec_t exec = nullptr;
    int count = 0;
};

std::mutex g_mu;
Lanes g_lanes;
std::map<std::string, Cached> g_graphs;       // key: the call's arguments
std::map<std::string, int> g_tuned;           // key: the batch shape -> lane count
bool g_latency = false;
int g_latency_count = 0;

int ensure_lanes(int count)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (g_lanes.device != dev) {
        // streams and events of another device are abandoned (one device per process here)
        g_lanes = Lanes();
        g_lanes.device = dev;
        if (cudaStreamCreateWithFlags(&g_lanes.origin, cudaStreamNonBlocking) != cudaSuccess) return RHOSVD_ERR_CUDA;
        for (int i = 0; i < LANES_MAX; ++i) {
            if (cudaStreamCreateWithFlags(&g_lanes.s[i], cudaStreamNonBlocking) != cudaSuccess) return RHOSVD_ERR_CUDA;
            if (cudaEventCreateWithFlags(&g_lanes.join[i], cudaEventDisableTiming) != cudaSuccess)
                return RHOSVD_ERR_CUDA;
        }
        if (cudaEventCreateWithFlags(&g_lanes.fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g_lanes.after, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g_lanes.before, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&g_lanes.t0) != cudaSuccess)
            return RHOSVD_ERR_CUDA;
    }
    while ((int)g_lanes.done.size() < count) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return RHOSVD_ERR_CUDA;
        g_lanes.done.push_back(e);
    }
    return 0;
}

double cost_of(const rhosvd_cp& cp)
{
    const double nsum = (double)cp.n[0] + cp.n[1] + cp.n[2];
    return 3.0 * nsum * (cp.R > 0 ? cp.R : 1) + 4.0e6;   // two passes over U + small factorisations
}

struct Schedule {
    std::vector<std::vector<int>> order;   // tensors of each lane, in launch order
    std::vector<size_t> offset;            // workspace offset of each lane
};

// longest processing time first: each tensor (by decreasing cost) to the least-loaded lane
int make_schedule(int count, const rhosvd_cp* cps, int lanes, size_t slot, Schedule* s)
{
    std::vector<int> idx(count);
    for (int i = 0; i < count; ++i) idx[i] = i;
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost_of(cps[a]) > cost_of(cps[b]); });
    std::vector<double> load(lanes, 0.0);
    s->order.assign(lanes, std::vector<int>());
    for (int t : idx) {
        int best = 0;
        for (int l = 1; l < lanes; ++l)
            if (load[l] < load[best]) best = l;
        load[best] += cost_of(cps[t]);
        s->order[best].push_back(t);
    }
    s->offset.resize(lanes);
    for (int l = 0; l < lanes; ++l) s->offset[l] = (size_t)l * slot;
    return 0;
}

size_t slot_size(int count, const rhosvd_cp* cps, const rhosvd_opts* opts)
{
    size_t mx = 0;
    for (int i = 0; i < count; ++i) {
        const size_t w = rhosvd_c2t_workspace_size(&cps[i], &opts[i]);
        if (w == 0) return 0;
        mx = std::max(mx, w);
    }
    return up_align(mx);
}

int default_lanes(int count) { return std::max(1, std::min(count, LANES_MAX)); }

std::string key_of(int count, const rhosvd_cp* cps, const rhosvd_opts* opts, const rhosvd_tucker* outs,
                   const void* ws, size_t bytes, int lanes, bool latency)
{
    std::string k;
    k.append((const char*)&count, sizeof(count));
    k.append((const char*)cps, sizeof(rhosvd_cp) * count);
    k.append((const char*)opts, sizeof(rhosvd_opts) * count);
    k.append((const char*)outs, sizeof(rhosvd_tucker) * count);
    k.append((const char*)&ws, sizeof(ws));
    k.append((const char*)&bytes, sizeof(bytes));
    k.append((const char*)&lanes, sizeof(lanes));
    k.push_back(latency ? 1 : 0);
    k.append((const char*)&g_lanes.device, sizeof(int));
    return k;
}

std::string shape_of(int count, const rhosvd_cp* cps, const rhosvd_opts* opts)
{
    std::string k;
    for (int i = 0; i < count; ++i) {
        k.append((const char*)cps[i].n, sizeof(cps[i].n));
        k.append((const char*)&cps[i].R, sizeof(int));
        k.append((const char*)&opts[i].r_max, sizeof(int));
        k.append((const char*)&opts[i].oversample, sizeof(int));
        k.append((const char*)&opts[i].precision, sizeof(int));
    }
    return k;
}

// capture the batch with `lanes` lanes into an executable graph
int build_graph(int count, const rhosvd_cp* cps, const rhosvd_opts* opts, const rhosvd_tucker* outs, char* ws,
                size_t slot, int lanes, bool latency, cudaGraphExec_t* exec)
{
    Schedule sch;
    make_schedule(count, cps, lanes, slot, &sch);
    const int prof = rhosvd_profile_enable(0);     // no tracing events inside a graph
    cudaStream_t o = g_lanes.origin;
    if (cudaStreamBeginCapture(o, cudaStreamCaptureModeRelaxed) != cudaSuccess) {
        rhosvd_profile_enable(prof);
        return RHOSVD_ERR_CUDA;
    }
    int rc = 0;
    if (cudaEventRecord(g_lanes.fork, o) != cudaSuccess) rc = RHOSVD_ERR_CUDA;
    if (!rc && latency && cudaEventRecordWithFlags(g_lanes.t0, o, cudaEventRecordExternal) != cudaSuccess)
        rc = RHOSVD_ERR_CUDA;
    for (int l = 0; l < lanes && !rc; ++l) {
        cudaStream_t s = g_lanes.s[l];
        if (cudaStreamWaitEvent(s, g_lanes.fork, 0) != cudaSuccess) { rc = RHOSVD_ERR_CUDA; break; }
        for (int t : sch.order[l]) {
            rc = rhosvd_c2t(&cps[t], &opts[t], &outs[t], ws + sch.offset[l], slot, s);
            if (rc) break;
            if (latency && cudaEventRecordWithFlags(g_lanes.done[t], s, cudaEventRecordExternal) != cudaSuccess) {
                rc = RHOSVD_ERR_CUDA;
                break;
            }
        }
        if (rc) break;
        if (cudaEventRecord(g_lanes.join[l], s) != cudaSuccess || cudaStreamWaitEvent(o, g_lanes.join[l], 0) != cudaSuccess)
            rc = RHOSVD_ERR_CUDA;
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(o, &g);
    rhosvd_profile_enable(prof);
    if (!rc && ec != cudaSuccess) rc = RHOSVD_ERR_CUDA;
    if (!rc && cudaGraphInstantiate(exec, g, 0) != cudaSuccess) rc = RHOSVD_ERR_CUDA;
    if (g) cudaGraphDestroy(g);
    return rc;
}

int launch_graph(cudaGraphExec_t exec, cudaStream_t stream)
{
    cudaStream_t o = g_lanes.origin;
    if (cudaEventRecord(g_lanes.before, stream) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (cudaStreamWaitEvent(o, g_lanes.before, 0) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (cudaGraphLaunch(exec, o) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (cudaEventRecord(g_lanes.after, o) != cudaSuccess) return RHOSVD_ERR_CUDA;
    if (cudaStreamWaitEvent(stream, g_lanes.after, 0) != cudaSuccess) return RHOSVD_ERR_CUDA;
    return 0;
}

}  // namespace

extern "C" size_t rhosvd_c2t_batched_workspace_size(int count, const rhosvd_cp* cps, const rhosvd_opts* opts,
                                                    int lanes)
{
    if (count < 1 || !cps || !opts) return 0;
    const size_t slot = slot_size(count, cps, opts);
    if (slot == 0) return 0;
    const int L = lanes > 0 ? std::min(lanes, LANES_MAX) : default_lanes(count);
    return slot * (size_t)L;
}

extern "C" int rhosvd_c2t_batched(int count, const rhosvd_cp* cps, const rhosvd_opts* opts,
                                  const rhosvd_tucker* outs, void* workspace, size_t bytes, int lanes,
                                  void* stream_)
{
    cudaStream_t stream = (cudaStream_t)stream_;
    if (count < 1 || !cps || !opts || !outs || !workspace) return RHOSVD_ERR_INVALID_ARG;
    const size_t slot = slot_size(count, cps, opts);
    if (slot == 0) return RHOSVD_ERR_INVALID_ARG;
    const int Lmax = lanes > 0 ? std::min(lanes, LANES_MAX) : default_lanes(count);
    if (bytes < slot * (size_t)Lmax) return RHOSVD_ERR_WORKSPACE;
    std::lock_guard<std::mutex> lk(g_mu);
    int rc = ensure_lanes(count);
    if (rc) return rc;
    char* ws = (char*)workspace;
    int L = lanes > 0 ? Lmax : 0;
    if (L == 0) {
        const std::string shape = shape_of(count, cps, opts);
        auto it = g_tuned.find(shape);
        if (it != g_tuned.end() && it->second <= Lmax) {
            L = it->second;
        } else {
            // autotune: time each candidate lane count once (synchronises), keep the fastest
            float best = 0.f;
            std::vector<int> cands;
            for (int c : {4, 8, 16, 32})
                if (c < Lmax) cands.push_back(c);
            cands.push_back(Lmax);
            for (int c : cands) {
                cudaGraphExec_t ex = nullptr;
                rc = build_graph(count, cps, opts, outs, ws, slot, c, false, &ex);
                if (rc) return rc;
                cudaEvent_t a = nullptr, b = nullptr;
                cudaEventCreate(&a);
                cudaEventCreate(&b);
                cudaEventRecord(a, g_lanes.origin);
                const cudaError_t e1 = cudaGraphLaunch(ex, g_lanes.origin);
                cudaEventRecord(b, g_lanes.origin);
                const cudaError_t e2 = cudaEventSynchronize(b);
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                cudaEventDestroy(a);
                cudaEventDestroy(b);
                cudaGraphExecDestroy(ex);
                if (e1 != cudaSuccess || e2 != cudaSuccess) return RHOSVD_ERR_CUDA;
                if (L == 0 || ms < best) { best = ms; L = c; }
            }
            g_tuned[shape] = L;
        }
    }
    const std::string key = key_of(count, cps, opts, outs, workspace, bytes, L, g_latency);
    auto it = g_graphs.find(key);
    if (it == g_graphs.end()) {
        if (g_graphs.size() >= 8) {
            for (auto& kv : g_graphs) cudaGraphExecDestroy(kv.second.exec);
            g_graphs.clear();
        }
        Cached c;
        c.count = count;
        rc = build_graph(count, cps, opts, outs, ws, slot, L, g_latency, &c.exec);
        if (rc) return rc;
        it = g_graphs.emplace(key, c).first;
    }
    rc = launch_graph(it->second.exec, stream);
    if (rc) return rc;
    if (g_latency) g_latency_count = count;
    return 0;
}

extern "C" int rhosvd_batch_latency_enable(int on)
{
    std::lock_guard<std::mutex> lk(g_mu);
    const int prev = g_latency ? 1 : 0;
    g_latency = on != 0;
    return prev;
}

extern "C" int rhosvd_batch_latency_read(float* ms, int count)
{
    std::lock_guard<std::mutex> lk(g_mu);
    if (!ms || count < 1 || count > g_latency_count) return RHOSVD_ERR_INVALID_ARG;
    for (int t = 0; t < count; ++t) {
        if (cudaEventSynchronize(g_lanes.done[t]) != cudaSuccess) return RHOSVD_ERR_CUDA;
        if (cudaEventElapsedTime(&ms[t], g_lanes.t0, g_lanes.done[t]) != cudaSuccess) return RHOSVD_ERR_CUDA;
    }
    return 0;
}
