// capi.cu -- the C ABI declared in include/sta.h.
//
// Execution model: one handle per netlist keeps every array resident on the
// device.  A forward pass is a sequence of kernels (net RC over every net,
// then one launch per level, then the endpoint reduction, then one launch per
// level in reverse for required times); the gradient pass is one launch per
// level in reverse.  Each sequence is captured once into a CUDA graph and
// replayed, so the per-level launches cost a graph node each, not a host
// launch.  The required-time sweep runs on a stream of the handle's own that
// waits for the arrival-time pass only, so the caller's stream is free as
// soon as arrival times exist and a gradient sweep queued there overlaps the
// required-time sweep on the GPU: the GB300 counterpart of the paper's
// two-stream operation fusion (Section 3.2).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "sta_internal.h"

using namespace sta;

namespace {

thread_local std::string g_err;

StaStatus set_err(StaStatus st, const std::string& msg) {
    g_err = msg;
    return st;
}

#define CUDA_TRY(expr)                                                                       \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return set_err(e_ == cudaErrorMemoryAllocation ? STA_ERR_OOM : STA_ERR_CUDA,     \
                           std::string(#expr) + ": " + cudaGetErrorString(e_));              \
    } while (0)

}  // namespace

namespace {
// 16-byte host-visible words for the handles' stream-ordered readbacks, carved
// from pinned pages kept for the life of the process: creating and destroying
// a handle never calls cudaMallocHost / cudaFreeHost (which waits for the
// whole device)
std::mutex g_pin_mu;
std::vector<int32_t*> g_pin_free;

int32_t* pinned_acquire() {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    if (g_pin_free.empty()) {
        int32_t* page = nullptr;
        if (cudaMallocHost(&page, 4096) != cudaSuccess) return nullptr;
        for (int k = 4096 / 16 - 1; k >= 0; --k) g_pin_free.push_back(page + 4 * k);
    }
    int32_t* p = g_pin_free.back();
    g_pin_free.pop_back();
    p[0] = p[1] = p[2] = p[3] = 0;
    return p;
}

void pinned_release(int32_t* p) {
    if (!p) return;
    std::lock_guard<std::mutex> lk(g_pin_mu);
    g_pin_free.push_back(p);
}
}  // namespace

namespace sta {
// lets other translation units of the library report through sta_last_error()
void set_last_error_text(const std::string& msg) { g_err = msg; }
}  // namespace sta

struct StaHandle {
    explicit StaHandle(std::shared_ptr<Layout> l) : lay_sp(std::move(l)), lay(*lay_sp) {}
    std::shared_ptr<Layout> lay_sp;  // the host layout, possibly shared with other handles of the netlist
    Layout& lay;
    DevNet g{};
    DevState s{};
    DfState d{};
    int schedule = STA_SCHED_DATAFLOW;
    int grid_fwd = 0, grid_bwd = 0;  // dataflow grids (blocks)
    int grid_bwd_w = 0;  // batched: the lane-per-placement backward sweeps' grid
    int grid_fwd_w = 0;  // batched: the lane-per-placement forward sweep's grid
    // batched schedule: B placements, lane per placement
    int B = 1;
    int bsweep = STA_BATCH_LEVELS;
    // independent placements of the single-placement schedule (StaOptions
    // batch_sweep = STA_BATCH_LANES): lanes, each with its own state slab
    int nl = 1;
    int active = 1, active_next = 1;  // lanes the current / the next positions' calls run
    BatchState bs{};
    const int32_t* pin_int = nullptr;  // [P] internal index of each original pin
    BigChunks bload;  // batched: the large nets' sinks in chunks, whose loads k_bload computes
    float* qscratch = nullptr;         // device scratch of the batched pin-slack query
    size_t qscratch_bytes = 0;
    bool batch() const { return schedule == STA_SCHED_BATCH; }
    std::vector<std::pair<void*, size_t>> allocs;  // device allocations and their sizes
    size_t dev_bytes = 0;
    int device = 0;
    bool use_graphs = true;
    // forward calls begun.  A pooled handle (a server's resident copy, often
    // evicted after a request or two) launches directly on its first request and
    // captures its graphs from the second on: a capture and instantiation costs
    // the server's worker thread more than one request's direct launches.
    long long nforward = 0;
    bool graphs_now() const { return use_graphs && (!pool || nforward >= 2); }
    bool have_pos = false, have_fwd = false, have_lse = false, have_rat = false;
    float gamma_fwd = 1.f;
    cudaEvent_t ev_at = nullptr;    // arrival-time pass of the latest forward done
    cudaEvent_t ev_fwd = nullptr;   // whole latest forward (required times included) done
    cudaEvent_t ev_bwd = nullptr;   // latest gradient sweep done
    cudaStream_t cap = nullptr;     // private stream used for graph capture
    cudaStream_t side = nullptr;    // required-time sweep
    cudaStream_t fork = nullptr;    // the batched sweeps' resets beside the position transpose
    cudaEvent_t ev_fork[2] = {nullptr, nullptr};
    cudaEvent_t ev_pool = nullptr;  // pooled handle: legacy-stream allocations -> the caller's stream
    // batched dataflow handles: the words the next forward and fused gradient
    // sweeps poll were reset by sta_set_positions (on `fork`, done at ev_fork[1]);
    // a forward without new positions resets them itself
    bool pre_reset = false;
    // graph cache
    cudaGraphExec_t gx_fwd[2] = {nullptr, nullptr};  // [lse]
    float gx_fwd_gamma[2] = {0.f, 0.f};
    cudaGraphExec_t gx_rat = nullptr;
    float gx_rat_gamma = 0.f;
    cudaGraphExec_t gx_adj = nullptr;
    float gx_adj_gamma = 0.f;
    cudaGraphExec_t gx_fused = nullptr;  // dataflow: required times + adjoint in one sweep
    float gx_fused_gamma = 0.f;
    // dataflow: the required-time sweep of the latest forward is deferred until a
    // gradient sweep can carry it or a query needs it
    bool rat_pending = false;
    bool last_fused = false;
    // host-visible words: [0] expiry flag read back, [1] [2] dependency count of the
    // task a requested wait expiry stalls (raised, original)
    int32_t* pinned = nullptr;
    bool expire_next = false;  // the next forward sweep runs one wait into its budget
    int stall_task = -1;       // single-placement dataflow forward: the task whose wait never succeeds
    // staging for host inputs / outputs
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // profiling: event pairs around every launch of each sequence
    bool profile = false;
    struct Prof {
        std::vector<cudaEvent_t> ev;  // 2 per launch
        std::vector<int> kind;        // 1 per launch
        size_t next = 0;
    } prof_pos, prof_fwd, prof_rat, prof_adj, prof_out;

    // device memory from a stream-ordered pool (handles of a server, created and
    // destroyed while other requests run: no device-wide synchronization), else
    // cudaMalloc.  Pool allocations, uploads and creation-time fills are queued
    // on the legacy stream; events recorded there order every later call after
    // them, so creation does not wait for them on the host.  A pooled handle is
    // destroyed only once none of its work is in flight.
    cudaMemPool_t pool = nullptr;
    cudaError_t dev_malloc(void** q, size_t bytes) {
        return pool ? cudaMallocFromPoolAsync(q, bytes, pool, 0) : cudaMalloc(q, bytes);
    }
    void dev_free(void* q) {
        if (pool) cudaFreeAsync(q, 0);
        else cudaFree(q);
    }
    template <typename T>
    StaStatus alloc(T*& p, size_t n) {
        void* q = nullptr;
        const size_t bytes = (n ? n : 1) * sizeof(T);
        cudaError_t e = dev_malloc(&q, bytes);
        if (e != cudaSuccess) return set_err(STA_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        allocs.emplace_back(q, bytes);
        dev_bytes += bytes;
        p = static_cast<T*>(q);
        return STA_OK;
    }
    // free one allocation made by alloc()/upload()
    void release(const void* p) {
        for (size_t i = 0; i < allocs.size(); ++i)
            if (allocs[i].first == p) {
                dev_free(allocs[i].first);
                dev_bytes -= allocs[i].second;
                allocs.erase(allocs.begin() + (long)i);
                return;
            }
    }
    void drop_graphs() {
        for (cudaGraphExec_t* gx : {&gx_fwd[0], &gx_fwd[1], &gx_rat, &gx_adj, &gx_fused})
            if (*gx) {
                cudaGraphExecDestroy(*gx);
                *gx = nullptr;
            }
    }
    template <typename T>
    StaStatus upload(const T*& dst, const std::vector<T>& src) {
        T* p = nullptr;
        StaStatus st = alloc(p, src.size());
        if (st != STA_OK) return st;
        // a pooled handle's uploads are queued on the legacy stream (page-locked
        // sources: plain DMA, overlapping other requests' work)
        if (!src.empty() && pool)
            CUDA_TRY(cudaMemcpyAsync(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, 0));
        else if (!src.empty())
            CUDA_TRY(cudaMemcpy(p, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
        dst = p;
        return STA_OK;
    }
    // host-input / host-output staging of at least `bytes`, for work on `st`.
    // A pooled buffer is allocated on the legacy stream; `st` waits for that
    // (an event, not a host synchronization: the server's worker thread keeps
    // dispatching meanwhile).
    StaStatus staging(size_t bytes, cudaStream_t st) {
        if (bytes <= stage_bytes) return STA_OK;
        if (stage && pool) {  // the buffer's last use on `st` before it goes back to the pool
            CUDA_TRY(cudaEventRecord(ev_pool, st));
            CUDA_TRY(cudaStreamWaitEvent(0, ev_pool, 0));
        }
        if (stage) dev_free(stage);
        stage = nullptr;
        stage_bytes = 0;
        CUDA_TRY(dev_malloc(&stage, bytes));
        if (pool) {
            CUDA_TRY(cudaEventRecord(ev_pool, 0));
            CUDA_TRY(cudaStreamWaitEvent(st, ev_pool, 0));
        }
        stage_bytes = bytes;
        return STA_OK;
    }
    // creation-time copies and fills: a pooled handle queues them on the legacy
    // stream (ordered after its allocations and uploads; every later call waits
    // for them through the events recorded there at the end of creation)
    cudaError_t init_h2d(void* dst, const void* src, size_t n) {
        return pool ? cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, 0)
                    : cudaMemcpy(dst, src, n, cudaMemcpyHostToDevice);
    }
    cudaError_t init_zero(void* p, size_t n) { return pool ? cudaMemsetAsync(p, 0, n, 0) : cudaMemset(p, 0, n); }
    ~StaHandle() {
        for (auto* gx : {gx_fwd[0], gx_fwd[1], gx_rat, gx_adj, gx_fused})
            if (gx) cudaGraphExecDestroy(gx);
        for (auto& a : allocs) dev_free(a.first);
        if (stage) dev_free(stage);
        if (qscratch) cudaFree(qscratch);
        pinned_release(pinned);
        for (auto* ev : {ev_at, ev_fwd, ev_bwd, ev_fork[0], ev_fork[1], ev_pool})
            if (ev) cudaEventDestroy(ev);
        for (Prof* pr : {&prof_pos, &prof_fwd, &prof_rat, &prof_adj, &prof_out})
            for (cudaEvent_t e : pr->ev) cudaEventDestroy(e);
        if (cap) cudaStreamDestroy(cap);
        if (side) cudaStreamDestroy(side);
        if (fork) cudaStreamDestroy(fork);
    }
};

namespace {

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

// ---- sequences (also what the graphs capture) ----
// With profiling on, every launch is bracketed by an event pair (event record
// nodes when captured).  Events are created on first use.
struct ProfScope {
    StaHandle::Prof* pr;
    cudaStream_t st;
    size_t i;
    ProfScope(StaHandle* h, StaHandle::Prof* p, int kind, cudaStream_t s) : pr(h->profile ? p : nullptr), st(s), i(0) {
        if (!pr || 2 * pr->next + 1 >= pr->ev.size()) {  // events are made at creation
            pr = nullptr;
            return;
        }
        i = pr->next++;
        pr->kind[i] = kind;
        record(pr->ev[2 * i]);
    }
    ~ProfScope() {
        if (pr) record(pr->ev[2 * i + 1]);
    }
    // under stream capture an event-record node needs the External flag; outside
    // capture that flag is not accepted, so a plain record is used
    void record(cudaEvent_t e) const {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        cudaStreamIsCapturing(st, &cs);
        if (cs == cudaStreamCaptureStatusActive) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
        else cudaEventRecord(e, st);
    }
};

void enqueue_forward_dataflow(StaHandle* h, int lse, float gamma, cudaStream_t st) {
    const Layout& L = h->lay;
    cudaMemsetAsync(h->d.heads, 0, sizeof(int32_t), st);
    cudaMemsetAsync(h->d.abort_word, 0, sizeof(int32_t), st);
    {
        // load and wire RC of the nets > 32 pins, and the reset of the words the
        // sweep's tasks poll, in one launch
        ProfScope ps(h, &h->prof_fwd, STA_PROF_NET_RC, st);
        launch_fwd_prologue(h->g, h->s, h->d, L.P, st);
    }
    {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_FORWARD, st);
        launch_fwd_dataflow(h->g, h->s, h->d, h->grid_fwd, gamma, lse, h->stall_task, st);
    }
    {
        // the endpoints, and the reset of the words the next fused gradient sweep
        // polls (a fused sweep always follows a forward directly, so it needs no
        // reset of its own), in one launch
        ProfScope ps(h, &h->prof_fwd, STA_PROF_ENDPOINTS, st);
        launch_endpoints(h->g, h->s, gamma, lse, st, &h->d, L.P);
    }
}

void enqueue_backward_dataflow(StaHandle* h, int mode, float gamma, cudaStream_t st) {
    const Layout& L = h->lay;
    StaHandle::Prof* pr = (mode & 2) ? &h->prof_adj : &h->prof_rat;
    pr->next = 0;
    // every lane's counters (lane l's sit l * lane_bytes after lane 0's)
    cudaMemset2DAsync((mode & 2) ? h->d.acnt : h->d.rcnt, h->s.lane_bytes, 0, sizeof(int32_t) * (L.TB ? L.TB : 1),
                      h->nl, st);  // (every lane: the count a call runs is on the device)
    cudaMemsetAsync(h->d.heads + ((mode & 2) ? 2 : 1), 0, sizeof(int32_t), st);
    if (mode != 3) {  // the fused sweep's words were reset by the forward before it
        ProfScope ps(h, pr, STA_PROF_RESET, st);
        launch_bwd_reset(h->s, h->d, L.P, mode, st);  // the words the sweep's tasks poll
    }
    if ((mode & 2) && h->g.ep_clk) {
        ProfScope ps(h, pr, STA_PROF_SEED, st);
        launch_cap_seed(h->g, h->s, gamma, st);
    }
    ProfScope ps(h, pr, (mode & 2) ? STA_PROF_ADJOINT : STA_PROF_REQUIRED, st);
    launch_bwd_dataflow(h->g, h->s, h->d, h->grid_bwd, gamma, mode, st);
}

// Launches of a level-synchronous batched backward sweep: per level (deepest
// first) the partial chunks and packed nets of the level with the gradient
// chunks of the level above, then the driver steps of the level's large nets;
// finally the gradient chunks of level 0.  Each entry holds up to three task ranges.
void batch_bwd_phases(const Layout& L, int mode, std::vector<std::array<int, 6>>& out) {
    out.clear();
    for (int l = L.L - 1; l >= 0; --l) {
        const int* s = &L.lvl_bsec[(size_t)l * 5];
        std::array<int, 6> a = {s[0], s[1], s[2], s[3], 0, 0};
        if ((mode & 2) && l + 1 < L.L) {
            const int* u = &L.lvl_bsec[(size_t)(l + 1) * 5];
            a[4] = u[3];
            a[5] = u[4];
        }
        if (a[1] > a[0] || a[3] > a[2] || a[5] > a[4]) out.push_back(a);
        if (s[2] > s[1]) out.push_back({s[1], s[2], 0, 0, 0, 0});
    }
    if ((mode & 2) && L.L > 0 && L.lvl_bsec[4] > L.lvl_bsec[3]) out.push_back({L.lvl_bsec[3], L.lvl_bsec[4], 0, 0, 0, 0});
}

int batch_fwd_levels(const Layout& L) {
    int n = 0;
    for (int l = 0; l < L.L; ++l) n += L.lvl_ftask[l + 1] > L.lvl_ftask[l] ? 1 : 0;
    return n;
}

void enqueue_forward_batch(StaHandle* h, int lse, float gamma, cudaStream_t st) {
    const Layout& L = h->lay;
    if (h->bsweep == STA_BATCH_LEVELS) {
        {
            ProfScope ps(h, &h->prof_fwd, STA_PROF_NET_RC, st);
            launch_batch_load(h->g, h->bs, h->bload, st);
            launch_batch_load_small(h->g, h->bs, L.shape.big, st);
        }
        for (int l = 0; l < L.L; ++l) {
            if (L.lvl_ftask[l + 1] == L.lvl_ftask[l]) continue;
            ProfScope ps(h, &h->prof_fwd, STA_PROF_FORWARD, st);
            launch_batch_fwd_level(h->g, h->bs, h->d, L.lvl_ftask[l], L.lvl_ftask[l + 1], gamma, lse, st);
        }
        ProfScope ps(h, &h->prof_fwd, STA_PROF_ENDPOINTS, st);
        launch_batch_endpoints(h->g, h->bs, gamma, lse, st);
        return;
    }
    cudaMemsetAsync(h->d.heads, 0, sizeof(int32_t), st);
    cudaMemsetAsync(h->d.abort_word, 0, sizeof(int32_t), st);
    // (the words the sweeps poll were reset before: enqueue_batch_resets)
    if (h->bload.n) {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_NET_RC, st);
        launch_batch_load(h->g, h->bs, h->bload, st);
    }
    {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_FORWARD, st);
        // (STA_BATCH_WIDE: a lane per placement in both sweeps; the forward
        // measured 10% faster than the 8-placement one, bit-identical results)
        if (h->bsweep == STA_BATCH_WIDE)
            launch_batch_fwd_wide(h->g, h->bs, h->d, h->grid_fwd_w, gamma, lse, h->stall_task, st);
        else launch_batch_fwd(h->g, h->bs, h->d, h->grid_fwd, gamma, lse, h->stall_task, st);
    }
    {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_ENDPOINTS, st);
        launch_batch_endpoints(h->g, h->bs, gamma, lse, st);
    }
}

// The batched dataflow sweeps' polled words, set to kUnwritten before a forward:
// the forward's (arrival / slew / LSE arrival of cell-input pins) and those of
// the fused gradient sweep that follows it (required times, adjoints, large
// nets' partial records).  Bandwidth-bound writes: sta_set_positions runs them
// on the fork stream beside its position transpose (the previous positions'
// results cannot be queried any more), a forward without new positions on its
// own stream, the autotuner inside each candidate step.
bool batch_resets_needed(const StaHandle* h) { return h->batch() && h->bsweep != STA_BATCH_LEVELS; }

void enqueue_batch_resets(StaHandle* h, StaHandle::Prof* pr, cudaStream_t st) {
    ProfScope ps(h, pr, STA_PROF_RESET, st);
    launch_batch_reset(h->bs, h->d, h->lay.P, 0, st);
    launch_batch_reset(h->bs, h->d, h->lay.P, 3, st);
}

void enqueue_backward_batch(StaHandle* h, int mode, float gamma, cudaStream_t st) {
    const Layout& L = h->lay;
    StaHandle::Prof* pr = (mode & 2) ? &h->prof_adj : &h->prof_rat;
    pr->next = 0;
    if ((mode & 2) && h->g.ep_clk) {
        ProfScope ps(h, pr, STA_PROF_SEED, st);
        launch_batch_cap_seed(h->g, h->bs, gamma, st);
    }
    if (h->bsweep == STA_BATCH_LEVELS) {
        std::vector<std::array<int, 6>> ph;
        batch_bwd_phases(L, mode, ph);
        for (const auto& r : ph) {
            ProfScope ps(h, pr, (mode & 2) ? STA_PROF_ADJOINT : STA_PROF_REQUIRED, st);
            launch_batch_bwd_level(h->g, h->bs, h->d, r.data(), gamma, mode, st);
        }
        return;
    }
    cudaMemsetAsync((mode & 2) ? h->d.acnt : h->d.rcnt, 0, sizeof(int32_t) * (L.TB ? L.TB * (size_t)h->bs.GT : 1), st);
    cudaMemsetAsync(h->d.heads + ((mode & 2) ? 2 : 1), 0, sizeof(int32_t), st);
    if (mode != 3) {  // the fused sweep's words were reset by the forward before it
        ProfScope ps(h, pr, STA_PROF_RESET, st);
        launch_batch_reset(h->bs, h->d, L.P, mode, st);  // the words the sweep's tasks poll
    }
    ProfScope ps(h, pr, (mode & 2) ? STA_PROF_ADJOINT : STA_PROF_REQUIRED, st);
    if (h->bsweep == STA_BATCH_WIDE) launch_batch_bwd_wide(h->g, h->bs, h->d, h->grid_bwd_w, gamma, mode, st);
    else launch_batch_bwd(h->g, h->bs, h->d, h->grid_bwd, gamma, mode, st);
}

void enqueue_forward(StaHandle* h, int lse, float gamma, cudaStream_t st) {
    if (h->batch()) {
        h->prof_fwd.next = 0;
        enqueue_forward_batch(h, lse, gamma, st);
        return;
    }
    if (h->schedule == STA_SCHED_DATAFLOW) {
        h->prof_fwd.next = 0;
        enqueue_forward_dataflow(h, lse, gamma, st);
        return;
    }
    const Layout& L = h->lay;
    h->prof_fwd.next = 0;
    {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_NET_RC, st);
        launch_rc(h->g, h->s, L.lvl_wtask[L.L], st);
    }
    for (int l = 0; l < L.L; ++l) {
        ProfScope ps(h, &h->prof_fwd, STA_PROF_FORWARD, st);
        launch_fwd_level(h->g, h->s, L.lvl_wtask[l], L.lvl_wtask[l + 1] - L.lvl_wtask[l], L.lvl_ctask[l],
                         L.lvl_ctask[l + 1] - L.lvl_ctask[l], gamma, lse, st);
    }
    ProfScope ps(h, &h->prof_fwd, STA_PROF_ENDPOINTS, st);
    launch_endpoints(h->g, h->s, gamma, lse, st);
}

void enqueue_backward(StaHandle* h, int mode, float gamma, cudaStream_t st) {
    if (h->batch()) {
        enqueue_backward_batch(h, mode, gamma, st);
        return;
    }
    if (h->schedule == STA_SCHED_DATAFLOW) {
        enqueue_backward_dataflow(h, mode, gamma, st);
        return;
    }
    const Layout& L = h->lay;
    StaHandle::Prof* pr = (mode & 2) ? &h->prof_adj : &h->prof_rat;
    pr->next = 0;
    if (mode & 2) {
        ProfScope ps(h, pr, STA_PROF_SEED, st);
        launch_seed(h->g, h->s, gamma, st);
    }
    if ((mode & 2) && h->g.ep_clk) {
        ProfScope ps(h, pr, STA_PROF_SEED, st);
        launch_cap_seed(h->g, h->s, gamma, st);
    }
    for (int l = L.L - 1; l >= 0; --l) {
        ProfScope ps(h, pr, (mode & 2) ? STA_PROF_ADJOINT : STA_PROF_REQUIRED, st);
        launch_bwd_level(h->g, h->s, L.lvl_wtask[l], L.lvl_wtask[l + 1] - L.lvl_wtask[l], L.lvl_ctask[l],
                         L.lvl_ctask[l + 1] - L.lvl_ctask[l], gamma, mode, st);
    }
}

template <typename F>
StaStatus capture(StaHandle* h, cudaGraphExec_t* out, F&& body) {
    if (*out) {
        cudaGraphExecDestroy(*out);
        *out = nullptr;
    }
    cudaGraph_t graph = nullptr;
    CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    body(h->cap);
    cudaError_t e = cudaStreamEndCapture(h->cap, &graph);
    if (e != cudaSuccess) return set_err(STA_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return set_err(STA_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
    return STA_OK;
}

StaStatus launch_graph_or_direct(StaHandle* h, cudaGraphExec_t* gx, float* key, float gamma, int mode,
                                 cudaStream_t st);

// Launch the deferred required-time sweep (dataflow schedule) on the handle's
// stream, after the latest arrival-time pass.
StaStatus flush_rat(StaHandle* h) {
    if (!h->rat_pending) return STA_OK;
    h->rat_pending = false;
    if (cudaStreamWaitEvent(h->side, h->ev_at, 0) != cudaSuccess) return set_err(STA_ERR_CUDA, "cudaStreamWaitEvent");
    StaStatus st = launch_graph_or_direct(h, &h->gx_rat, &h->gx_rat_gamma, 1.f, 1, h->side);
    if (st != STA_OK) return st;
    if (cudaEventRecord(h->ev_fwd, h->side) != cudaSuccess) return set_err(STA_ERR_CUDA, "cudaEventRecord");
    return STA_OK;
}

StaStatus check_launch() {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(STA_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return STA_OK;
}

// Synchronize `st` and report a bounded device-side wait that expired since the
// last report (the sticky word is read in stream order, then cleared).
StaStatus sync_checked(StaHandle* h, cudaStream_t st) {
    CUDA_TRY(cudaMemcpyAsync(h->pinned, h->d.abort_word + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (h->pinned[0] != 0) {
        CUDA_TRY(cudaMemsetAsync(h->d.abort_word + 1, 0, sizeof(int32_t), st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return set_err(STA_ERR_TIMEOUT,
                       "a dependency wait of the dataflow schedule exceeded its 1 s budget; the results of "
                       "the sweeps since the previous report are invalid");
    }
    return STA_OK;
}

// A backward sweep of the given mode, as a cached graph (re-captured when
// gamma changes) or as direct launches.
StaStatus launch_graph_or_direct(StaHandle* h, cudaGraphExec_t* gx, float* key, float gamma, int mode,
                                 cudaStream_t st) {
    if (h->graphs_now()) {
        if (!*gx || *key != gamma) {
            StaStatus s2 = capture(h, gx, [&](cudaStream_t c) { enqueue_backward(h, mode, gamma, c); });
            if (s2 != STA_OK) return s2;
            *key = gamma;
        }
        CUDA_TRY(cudaGraphLaunch(*gx, st));
        return STA_OK;
    }
    enqueue_backward(h, mode, gamma, st);
    return check_launch();
}

// The large nets' sink chunks of the batched handle's task shape, their chunk
// sums and their per-net counters (zero).
StaStatus upload_big_chunks(StaHandle* h) {
    const Layout& L = h->lay;
    const std::vector<int32_t> rec = big_chunk_list(L.big_nets, L.net_ptr);
    const int32_t* cp = nullptr;
    StaStatus st = h->upload(cp, rec);
    if (st != STA_OK) return st;
    h->bload.rec = reinterpret_cast<const int4*>(cp);
    h->bload.n = (int)(rec.size() / 4);
    st = h->alloc(h->bload.part, (size_t)h->bload.n * h->bs.Bp);
    if (st != STA_OK) return st;
    st = h->alloc(h->bload.cnt, (size_t)h->bload.n * h->bs.G);
    if (st != STA_OK) return st;
    const size_t bytes = sizeof(int32_t) * (h->bload.n ? (size_t)h->bload.n * h->bs.G : 1);
    CUDA_TRY(h->pool ? cudaMemsetAsync(h->bload.cnt, 0, bytes, 0) : cudaMemset(h->bload.cnt, 0, bytes));
    return STA_OK;
}

// Device state of the batched schedule: per-placement arrays, the inverse pin
// permutation, the prologue's chunk list, constant state broadcast to every
// placement.
StaStatus init_batch(StaHandle* h) {
    const Layout& L = h->lay;
    BatchState& b = h->bs;
    b.B = h->B;
    b.Bp = (h->B + 31) / 32 * 32;
    b.G = b.Bp / 32;
    // sweep task groups of 8 placements: only the groups that hold placements
    // (the padding lanes of the last group ride along; whole padding groups are
    // not swept)
    b.GT = (h->B + kPlacePerWarp - 1) / kPlacePerWarp;
    const size_t P = L.P, N = L.N, E = L.E, Bp = b.Bp;
    StaStatus st = STA_OK;
#define BSTEP(x)                  \
    do {                          \
        st = (x);                 \
        if (st != STA_OK) return st; \
    } while (0)
    BSTEP(h->alloc(b.xy, P * Bp));
    BSTEP(h->alloc(b.load, N * Bp));
    BSTEP(h->alloc(b.at, 4 * P * Bp));
    BSTEP(h->alloc(b.slew, 4 * P * Bp));
    BSTEP(h->alloc(b.ats, 2 * P * Bp));
    BSTEP(h->alloc(b.rat, 4 * P * Bp));
    BSTEP(h->alloc(b.g_ats, 2 * P * Bp));
    BSTEP(h->alloc(b.g_slew, 2 * P * Bp));
    BSTEP(h->alloc(b.grad, P * Bp));
    BSTEP(h->alloc(b.ep_slack, E * Bp));
    BSTEP(h->alloc(b.summary, STA_SUM_COUNT * Bp));
    BSTEP(h->alloc(b.red, kRedBlocks * Bp * (kBatchEpBytes / sizeof(double))));
    BSTEP(h->alloc(b.params, 2 * Bp));
    BSTEP(h->alloc(b.part, (size_t)L.npart * kPartFloats * Bp));
    BSTEP(h->alloc(b.rpart, (size_t)L.npart * kPartFloats * Bp));
    BSTEP(h->alloc(b.net_gload, N * Bp));
    b.cap_seed = nullptr;
    if (!L.ep_clk.empty()) {
        BSTEP(h->alloc(b.cap_seed, P * Bp));
        if (cudaMemset(b.cap_seed, 0, P * Bp * 4) != cudaSuccess) return set_err(STA_ERR_CUDA, "cudaMemset failed");
    }
    std::vector<int32_t> inv(P);
    for (size_t i = 0; i < P; ++i) inv[L.pin_orig[i]] = (int32_t)i;
    BSTEP(h->upload(h->pin_int, inv));
    BSTEP(upload_big_chunks(h));
#undef BSTEP
    auto zero = [&](void* p, size_t bytes) { return cudaMemset(p, 0, bytes); };
    if (zero(b.xy, P * Bp * 8) || zero(b.load, N * Bp * 4) || zero(b.g_ats, 2 * P * Bp * 4) ||
        zero(b.g_slew, 2 * P * Bp * 4) || zero(b.grad, P * Bp * 8) || zero(b.summary, STA_SUM_COUNT * Bp * 8) ||
        zero(b.params, 2 * Bp * 4) || zero(b.net_gload, N * Bp * 4))
        return set_err(STA_ERR_CUDA, "cudaMemset failed");
    // asserted arrival / slew and required-time constraints, the same for every placement
    if (P) {
        st = h->staging(P * 16, 0);
        if (st != STA_OK) return st;
        float* tmp = static_cast<float*>(h->stage);
        const std::pair<float*, const std::vector<float>*> init[] = {{b.at, &L.at0}, {b.slew, &L.slew0},
                                                                       {b.rat, &L.rat0}};
        for (const auto& it : init) {
            CUDA_TRY(cudaMemcpy(tmp, it.second->data(), P * 16, cudaMemcpyHostToDevice));
            launch_batch_broadcast(it.first, tmp, (long long)P * 4, (int)Bp, 0);
            CUDA_TRY(cudaDeviceSynchronize());
        }
        launch_batch_init_ats(b, (int)P, 0);
    }
    CUDA_TRY(cudaGetLastError());
    return STA_OK;
}

// Replace the dataflow task lists of a handle (batched schedule) by those of
// another task shape: rebuild them on the host, free the old device copies,
// upload the new ones and drop every captured graph.
StaStatus set_tasks(StaHandle* h, const TaskShape& sh) {
    Layout& L = h->lay;
    try {
        std::string err;
        StaStatus st = build_tasks(L, sh, err);
        if (st != STA_OK) return set_err(st, err);
    } catch (const std::bad_alloc&) {
        return set_err(STA_ERR_OOM, "host allocation failed");
    }
    const long long GT = h->bs.GT;
    if ((long long)L.TF * GT >= (1ll << 31) || (long long)L.TB * GT >= (1ll << 31))
        return set_err(STA_ERR_INVALID_ARG, "num_placements too large for this netlist");
    DfState& d = h->d;
    for (const void* p : {(const void*)d.ftask, (const void*)d.arc_prod, (const void*)d.btask, (const void*)d.baux,
                          (const void*)d.pin_cons, (const void*)d.b_indeg, (const void*)d.b_out_ptr,
                          (const void*)d.b_out, (const void*)d.rcnt, (const void*)d.acnt, (const void*)h->bs.part,
                          (const void*)h->bs.rpart, (const void*)h->bload.rec, (const void*)h->bload.part,
                          (const void*)h->bload.cnt})
        h->release(p);
    StaStatus st = STA_OK;
#define TSTEP(x)                     \
    do {                             \
        st = (x);                    \
        if (st != STA_OK) return st; \
    } while (0)
    const int32_t* cp = nullptr;
    TSTEP(h->upload(cp, L.ftask));
    d.ftask = reinterpret_cast<const int4*>(cp);
    TSTEP(h->upload(d.arc_prod, L.arc_prod));
    TSTEP(h->upload(cp, L.btask));
    d.btask = reinterpret_cast<const int4*>(cp);
    TSTEP(h->upload(d.baux, L.baux));
    TSTEP(h->upload(d.pin_cons, L.pin_cons));
    TSTEP(h->upload(d.b_indeg, L.b_indeg));
    TSTEP(h->upload(d.b_out_ptr, L.b_out_ptr));
    TSTEP(h->upload(d.b_out, L.b_out));
    TSTEP(h->alloc(d.rcnt, (size_t)L.TB * GT));
    TSTEP(h->alloc(d.acnt, (size_t)L.TB * GT));
    TSTEP(h->alloc(h->bs.part, (size_t)L.npart * kPartFloats * h->bs.Bp));
    TSTEP(h->alloc(h->bs.rpart, (size_t)L.npart * kPartFloats * h->bs.Bp));
    TSTEP(upload_big_chunks(h));
#undef TSTEP
    d.TF = L.TF;
    d.TB = L.TB;
    d.npart = L.npart;
    h->drop_graphs();
    h->have_fwd = h->have_lse = h->have_rat = false;
    h->rat_pending = false;
    h->pre_reset = false;  // new partial-record buffers: the next forward resets them
    return STA_OK;
}

}  // namespace

extern "C" {

int sta_abi_version(void) { return STA_ABI_VERSION; }

StaStatus sta_measure_latency(int64_t bytes, int32_t steps, double* ns_per_load) {
    if (!ns_per_load || bytes < 64 || bytes > (int64_t(1) << 33) || steps < 1 || steps > 10000000)
        return set_err(STA_ERR_INVALID_ARG, "sta_measure_latency: bytes in [64, 2^33], steps in [1, 1e7]");
    const int64_t n = bytes / 4;
    // Sattolo's algorithm: a uniformly random cyclic permutation (one cycle through every index)
    std::vector<int32_t> next((size_t)n);
    for (int64_t i = 0; i < n; ++i) next[(size_t)i] = (int32_t)i;
    uint64_t x = 0x9e3779b97f4a7c15ull;
    for (int64_t i = n - 1; i > 0; --i) {
        x ^= x << 13;
        x ^= x >> 7;
        x ^= x << 17;
        const int64_t j = (int64_t)(x % (uint64_t)i);  // j < i
        std::swap(next[(size_t)i], next[(size_t)j]);
    }
    int32_t* d = nullptr;
    if (cudaMalloc(&d, (size_t)(n + 1) * sizeof(int32_t)) != cudaSuccess)
        return set_err(STA_ERR_OOM, "sta_measure_latency: cudaMalloc failed");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    float ms = 0.f;
    cudaError_t ce = cudaMemcpy(d, next.data(), (size_t)n * sizeof(int32_t), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) {
        launch_touch(d, n, d + n, 0);
        launch_chase(d, std::min<int64_t>(steps, 64), d + n, 0);  // warm the launch path
        cudaEventRecord(e0, 0);
        launch_chase(d, steps, d + n, 0);
        cudaEventRecord(e1, 0);
        ce = cudaEventSynchronize(e1);
    }
    if (ce == cudaSuccess) ce = cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(d);
    if (ce != cudaSuccess) return set_err(STA_ERR_CUDA, std::string("sta_measure_latency: ") + cudaGetErrorString(ce));
    *ns_per_load = 1e6 * (double)ms / steps;
    return STA_OK;
}

const char* sta_last_error(void) { return g_err.c_str(); }

StaStatus sta_levelize(const StaNetlistDesc* nl, int32_t* net_level, int32_t* num_levels, int32_t* net_order,
                       int32_t* pin_order) {
    if (!nl || !net_level || !num_levels) return set_err(STA_ERR_INVALID_ARG, "null argument");
    try {
        std::vector<int32_t> lv, order, pins;
        int32_t L = 0;
        std::string err;
        StaStatus st = ordering(*nl, lv, L, order, pins, err);
        if (st != STA_OK) return set_err(st, err);
        std::memcpy(net_level, lv.data(), lv.size() * sizeof(int32_t));
        *num_levels = L;
        if (net_order) std::memcpy(net_order, order.data(), order.size() * sizeof(int32_t));
        if (pin_order) std::memcpy(pin_order, pins.data(), pins.size() * sizeof(int32_t));
        return STA_OK;
    } catch (const std::bad_alloc&) {
        return set_err(STA_ERR_OOM, "host allocation failed");
    }
}

}  // extern "C"

namespace {
StaStatus create_handle(std::shared_ptr<const Layout> shared, const StaNetlistDesc* nl, const StaLibrary* lib,
                        const StaOptions* opts, cudaMemPool_t pool, StaHandle** out);
}  // namespace

extern "C" StaStatus sta_create(const StaNetlistDesc* nl, const StaLibrary* lib, const StaOptions* opts,
                                StaHandle** out) {
    if (!nl || !lib || !out) return set_err(STA_ERR_INVALID_ARG, "null argument");
    return create_handle(nullptr, nl, lib, opts, nullptr, out);
}

StaStatus sta_create_from_layout(std::shared_ptr<const Layout> lay, const StaOptions* opts, void* pool,
                                 StaHandle** out) {
    if (!lay || !out) return set_err(STA_ERR_INVALID_ARG, "null argument");
    return create_handle(std::move(lay), nullptr, nullptr, opts, static_cast<cudaMemPool_t>(pool), out);
}

extern "C" StaStatus sta_create_multi(const StaNetlistDesc* const* nls, int32_t count, const StaLibrary* lib,
                                      const StaOptions* opts, StaHandle** out) {
    if (!nls || !lib || !out) return set_err(STA_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (opts && opts->schedule != STA_SCHED_DATAFLOW)
        return set_err(STA_ERR_INVALID_ARG, "sta_create_multi: the DATAFLOW schedule only");
    auto lay = std::make_shared<Layout>();
    try {
        UnionNetlist u;
        std::string err;
        StaStatus st = build_union(nls, count, u, err);
        if (st != STA_OK) return set_err(st, err);
        st = build_layout(u.nl, *lib, *lay, err);
        if (st != STA_OK) return set_err(st, err);
        if (count > 1) set_groups(*lay, u);
    } catch (const std::bad_alloc&) {
        return set_err(STA_ERR_OOM, "host allocation failed");
    }
    return create_handle(std::move(lay), nullptr, nullptr, opts, nullptr, out);
}

namespace {
// The handle of sta_create (nl, lib: build the layout) or of
// sta_create_from_layout (shared: a built layout, shared unless the options
// make a batched handle with its own task lists, which gets a copy).
StaStatus create_handle(std::shared_ptr<const Layout> shared, const StaNetlistDesc* nl, const StaLibrary* lib,
                        const StaOptions* opts, cudaMemPool_t pool, StaHandle** out) {
    *out = nullptr;
    StaHandle* h = nullptr;
    const bool own_tasks = opts && opts->schedule == STA_SCHED_BATCH && opts->batch_sweep != STA_BATCH_LANES;
    try {
        std::shared_ptr<Layout> lay;
        if (!shared) lay = std::make_shared<Layout>();
        else if (own_tasks) lay = std::make_shared<Layout>(*shared);
        else lay = std::const_pointer_cast<Layout>(shared);  // never modified: no task re-planning
        h = new StaHandle(std::move(lay));
        h->pool = pool;
    } catch (const std::bad_alloc&) {
        return set_err(STA_ERR_OOM, "host allocation failed");
    }
    auto fail = [&](StaStatus st) {
        std::string keep = g_err;
        delete h;
        g_err = keep;
        return st;
    };
    if (pool && cudaEventCreateWithFlags(&h->ev_pool, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_err(STA_ERR_CUDA, "cudaEventCreate failed"));
    if (!shared) {
        try {
            std::string err;
            StaStatus st = build_layout(*nl, *lib, h->lay, err);
            if (st != STA_OK) return fail(set_err(st, err));
        } catch (const std::bad_alloc&) {
            return fail(set_err(STA_ERR_OOM, "host allocation failed"));
        }
    }
    if (opts) {
        h->use_graphs = opts->use_graphs != 0;
        h->profile = opts->profile != 0;
        if (opts->grid_blocks < 0) return fail(set_err(STA_ERR_INVALID_ARG, "StaOptions.grid_blocks must be >= 0"));
        if (opts->schedule != STA_SCHED_DATAFLOW && opts->schedule != STA_SCHED_LEVELS &&
            opts->schedule != STA_SCHED_BATCH)
            return fail(set_err(STA_ERR_INVALID_ARG, "StaOptions.schedule must be DATAFLOW, LEVELS or BATCH"));
        h->schedule = opts->schedule;
        if (h->batch() && opts->batch_sweep == STA_BATCH_LANES) {
            // B placements as lanes of the single-placement dataflow sweeps
            if (opts->num_placements < 0 || opts->num_placements > 1024)
                return fail(set_err(STA_ERR_INVALID_ARG, "StaOptions: num_placements in [0, 1024] for LANES"));
            h->schedule = STA_SCHED_DATAFLOW;
            h->B = h->nl = opts->num_placements > 0 ? opts->num_placements : 1;
            h->bsweep = STA_BATCH_LANES;
            if ((long long)h->lay.TF * h->nl >= (1ll << 31) || (long long)h->lay.TB * h->nl >= (1ll << 31))
                return fail(set_err(STA_ERR_INVALID_ARG, "num_placements too large for this netlist"));
        } else if (h->batch()) {
            if (opts->num_placements < 0 || opts->num_placements > (1 << 16) || opts->tile_pins < 0 ||
                opts->chunk < 0)
                return fail(set_err(STA_ERR_INVALID_ARG, "StaOptions: num_placements in [0, 65536], tile_pins, "
                                                         "chunk >= 0"));
            h->B = opts->num_placements > 0 ? opts->num_placements : 1;
            TaskShape sh;
            sh.pack_pins = opts->tile_pins > 0 ? opts->tile_pins : 4;
            sh.pack_nets = 1 << 20;
            sh.chunk = opts->chunk > 0 ? opts->chunk : 16;
            if (opts->batch_sweep != STA_BATCH_LEVELS && opts->batch_sweep != STA_BATCH_DATAFLOW &&
                opts->batch_sweep != STA_BATCH_WIDE)
                return fail(set_err(STA_ERR_INVALID_ARG,
                                    "StaOptions.batch_sweep must be LEVELS, DATAFLOW, LANES or WIDE"));
            h->bsweep = opts->batch_sweep;
            sh.big = sh.chunk + 1;  // a driver and `chunk` sinks still form one task
            try {
                std::string err;
                StaStatus st = build_tasks(h->lay, sh, err);
                if (st != STA_OK) return fail(set_err(st, err));
                const long long G = (h->B + 31) / 32 * (32 / kPlacePerWarp);
                if ((long long)h->lay.TF * G >= (1ll << 31) || (long long)h->lay.TB * G >= (1ll << 31) ||
                    (long long)h->lay.P * 4 * G * 32 >= (1ll << 40))
                    return fail(set_err(STA_ERR_INVALID_ARG, "num_placements too large for this netlist"));
            } catch (const std::bad_alloc&) {
                return fail(set_err(STA_ERR_OOM, "host allocation failed"));
            }
        }
    }
    const Layout& L = h->lay;
    cudaError_t ce = cudaGetDevice(&h->device);
    if (ce != cudaSuccess) return fail(set_err(STA_ERR_CUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(ce)));

    DevNet& g = h->g;
    DevState& s = h->s;
    StaStatus st = STA_OK;
#define STEP(x)                      \
    do {                             \
        st = (x);                    \
        if (st != STA_OK) return fail(st); \
    } while (0)
    STEP(h->upload(g.net_ptr, L.net_ptr));
    STEP(h->upload(g.net_drv, L.net_drv));
    STEP(h->upload(g.net_arc_ptr, L.net_arc_ptr));
    STEP(h->upload(g.arc_pin, L.arc_pin));
    STEP(h->upload(g.pin_orig, L.pin_orig));
    STEP(h->upload(g.pin_cap, L.pin_cap));
    STEP(h->upload(g.wtask, L.wtask));
    STEP(h->upload(g.ctask, L.ctask));
    {
        const int32_t* cp = nullptr;
        STEP(h->upload(cp, L.rc_chunk));
        g.rc_chunk = reinterpret_cast<const int4*>(cp);
        STEP(h->upload(cp, L.rc_net));
        g.rc_net = reinterpret_cast<const int2*>(cp);
        g.nrc = (int32_t)(L.rc_chunk.size() / 4);
    }
    STEP(h->upload(g.lib_idx, L.lib_idx));
    STEP(h->upload(g.lib_inv, L.lib_inv));
    STEP(h->upload(g.lib_unate, L.lib_unate));
    STEP(h->upload(g.lib_tab, L.lib_tab));
    {
        const float* cp = nullptr;
        STEP(h->upload(cp, L.lib_cell));
        g.lib_cell = reinterpret_cast<const float4*>(cp);
        STEP(h->upload(cp, L.lib_col));
        g.lib_col = reinterpret_cast<const float4*>(cp);
    }
    {
        const int32_t* dp = nullptr;
        STEP(h->upload(dp, L.net_desc));
        g.net_desc = reinterpret_cast<const int4*>(dp);
    }
    STEP(h->upload(g.ep_pin, L.ep_pin));
    STEP(h->upload(g.ep_rat, L.ep_rat));
    g.ep_clk = nullptr;
    if (!L.ep_clk.empty()) STEP(h->upload(g.ep_clk, L.ep_clk));
    g.r = L.r_per_um;
    g.c = L.c_per_um;
    g.P = L.P;
    g.Pnet = L.Pnet;
    g.N = L.N;
    g.E = L.E;
    g.G = L.G;
    g.ep_gx = kEpBlocks;
    g.grp_ep = g.pin_grp = nullptr;
    if (L.G > 1) {  // several netlists: per-netlist endpoint ranges and pin owners
        if (h->batch() || h->schedule != STA_SCHED_DATAFLOW || h->nl > 1)
            return fail(set_err(STA_ERR_INVALID_ARG, "sta_create_multi: the DATAFLOW schedule only"));
        STEP(h->upload(g.grp_ep, L.grp_ep));
        STEP(h->upload(g.pin_grp, L.pin_grp));
        // blocks per netlist: every endpoint of the largest one at one thread (at
        // most kEpBlocks), so each netlist reduces in the order it has alone
        int32_t emax = 0;
        for (int32_t k = 0; k < L.G; ++k) emax = std::max(emax, L.grp_ep[k + 1] - L.grp_ep[k]);
        g.ep_gx = std::max(1, std::min(kEpBlocks, (emax + kBlock - 1) / kBlock));
    }

    const size_t P = L.P;
    const bool bat = h->batch();
    DfState& d = h->d;
    {
        const int32_t* cp = nullptr;
        STEP(h->upload(cp, L.ftask));
        d.ftask = reinterpret_cast<const int4*>(cp);
        STEP(h->upload(d.arc_prod, L.arc_prod));
        STEP(h->upload(cp, L.btask));
        d.btask = reinterpret_cast<const int4*>(cp);
        STEP(h->upload(d.baux, L.baux));
        STEP(h->upload(d.pin_cons, L.pin_cons));
        STEP(h->upload(d.pin_keep, L.pin_keep));
        d.pin_grp = g.pin_grp;
        {
            const uint8_t* mp = nullptr;
            STEP(h->upload(mp, L.pin_mask));
            d.pin_mask = reinterpret_cast<const uchar4*>(mp);
        }
        STEP(h->upload(d.b_indeg, L.b_indeg));
        STEP(h->upload(d.b_out_ptr, L.b_out_ptr));
        STEP(h->upload(d.b_out, L.b_out));
    }
    STEP(h->alloc(d.heads, 4));
    STEP(h->alloc(d.abort_word, 2));
    d.TF = L.TF;
    d.TB = L.TB;
    d.npart = L.npart;
    if (bat) {
        const size_t G = (size_t)(h->B + 31) / 32 * (32 / kPlacePerWarp);
        STEP(h->alloc(d.rcnt, L.TB * G));
        STEP(h->alloc(d.acnt, L.TB * G));
        STEP(h->alloc(d.rpart, 1));
        STEP(h->alloc(d.apart, 1));
        STEP(h->alloc(d.net_gload, 1));
        STEP(init_batch(h));
    } else {
        // The per-placement state: one slab per lane (a single placement: one),
        // every array at the same offset in each slab, so that lane l's state is
        // lane 0's shifted by l * lane_bytes (lane_state, lane_df).
        struct Carve {
            size_t bytes = 0;
            size_t add(size_t n, size_t elem) {
                const size_t off = (bytes + 255) / 256 * 256;
                bytes = off + std::max<size_t>(n, 1) * elem;
                return off;
            }
        } cv;
        const size_t NS = (size_t)std::max(L.rc_slots, 1), NP = (size_t)L.npart * kPartFloats;
        const size_t o_xy = cv.add(P, 8), o_load = cv.add(L.N, 4), o_wdi = cv.add(P, 8), o_at = cv.add(4 * P, 4),
                     o_slew = cv.add(4 * P, 4), o_ats = cv.add(2 * P, 4), o_adel = cv.add(4 * (size_t)L.A, 4),
                     o_rat = cv.add(4 * P, 4), o_gats = cv.add(2 * P, 4), o_gslew = cv.add(2 * P, 4),
                     o_grad = cv.add(P, 8), o_eps = cv.add(L.E, 8), o_red = cv.add(std::max<size_t>((size_t)kEpBlocks * 8, (size_t)L.G * g.ep_gx * 6), 8),
                     o_sum = cv.add((size_t)STA_SUM_COUNT * L.G, 8), o_par = cv.add(2 * (size_t)L.G + 2, 4), o_rcp = cv.add(NS, 4),
                     o_rcc = cv.add(NS, 4), o_epc = cv.add(L.G, 4), o_cap = L.ep_clk.empty() ? 0 : cv.add(P, 4),
                     o_rcnt = cv.add(L.TB, 4), o_acnt = cv.add(L.TB, 4), o_rpart = cv.add(NP, 4),
                     o_apart = cv.add(NP, 4), o_gload = cv.add(L.N, 4), o_brec = cv.add(8 * (size_t)L.N, 16);
        const size_t lb = (cv.bytes + 255) / 256 * 256;
        char* slab = nullptr;
        STEP(h->alloc(slab, lb * (size_t)h->nl));
        if (h->init_zero(slab, lb * (size_t)h->nl) != cudaSuccess) return fail(set_err(STA_ERR_CUDA, "cudaMemset failed"));
        s.xy = reinterpret_cast<float2*>(slab + o_xy);
        s.load = reinterpret_cast<float*>(slab + o_load);
        s.wdi = reinterpret_cast<float2*>(slab + o_wdi);
        s.at = reinterpret_cast<float*>(slab + o_at);
        s.slew = reinterpret_cast<float*>(slab + o_slew);
        s.ats = reinterpret_cast<float*>(slab + o_ats);
        s.adel = reinterpret_cast<float*>(slab + o_adel);
        s.rat = reinterpret_cast<float*>(slab + o_rat);
        s.g_ats = reinterpret_cast<float*>(slab + o_gats);
        s.g_slew = reinterpret_cast<float*>(slab + o_gslew);
        s.grad = reinterpret_cast<float2*>(slab + o_grad);
        s.ep_slack = reinterpret_cast<float2*>(slab + o_eps);
        s.red = reinterpret_cast<double*>(slab + o_red);
        s.summary = reinterpret_cast<double*>(slab + o_sum);
        s.params = reinterpret_cast<float*>(slab + o_par);
        s.rc_part = reinterpret_cast<float*>(slab + o_rcp);
        s.rc_count = reinterpret_cast<int32_t*>(slab + o_rcc);
        s.ep_count = reinterpret_cast<int32_t*>(slab + o_epc);
        s.cap_seed = L.ep_clk.empty() ? nullptr : reinterpret_cast<float*>(slab + o_cap);
        d.rcnt = reinterpret_cast<int32_t*>(slab + o_rcnt);
        d.acnt = reinterpret_cast<int32_t*>(slab + o_acnt);
        d.rpart = reinterpret_cast<float*>(slab + o_rpart);
        d.apart = reinterpret_cast<float*>(slab + o_apart);
        d.net_gload = reinterpret_cast<float*>(slab + o_gload);
        d.brec = reinterpret_cast<float4*>(slab + o_brec);
        s.lane_bytes = lb;
        s.nl = h->nl;
        s.active = nullptr;
        h->active = h->active_next = h->nl;
        if (h->nl > 1) {
            STEP(h->alloc(s.active, 1));
            // (pooled and under 256 lanes: two fills, the count as its low,
            // little-endian byte, instead of a copy from pageable memory, which
            // would first wait for the legacy stream's uploads)
            const bool fill = h->pool && h->nl < 256;
            if ((fill ? (cudaMemsetAsync(s.active, 0, sizeof(int32_t), 0) != cudaSuccess ||
                         cudaMemsetAsync(s.active, h->nl, 1, 0) != cudaSuccess)
                      : cudaMemcpy(s.active, &h->nl, sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess))
                return fail(set_err(STA_ERR_CUDA, "initial state upload failed"));
        }
        // constant state of every lane: asserted AT/slew (and LSE AT = late AT),
        // required-time seeds
        for (int l = 0; l < h->nl; ++l) {
            const DevState sl = lane_state(s, l);
            if (h->init_h2d(sl.at, L.at0.data(), P * 16) != cudaSuccess ||
                h->init_h2d(sl.slew, L.slew0.data(), P * 16) != cudaSuccess ||
                h->init_h2d(sl.rat, L.rat0.data(), P * 16) != cudaSuccess)
                return fail(set_err(STA_ERR_CUDA, "initial state upload failed"));
            launch_init_ats(sl, L.P, 0);
        }
    }
    if (h->init_zero(d.abort_word, 8) != cudaSuccess || h->init_zero(d.heads, 16) != cudaSuccess)
        return fail(set_err(STA_ERR_CUDA, "cudaMemset failed"));
#undef STEP
    if (!(h->pinned = pinned_acquire())) return fail(set_err(STA_ERR_OOM, "cudaMallocHost failed"));
    if (cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&h->fork, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fork[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_at, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_fwd, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&h->ev_bwd, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_err(STA_ERR_CUDA, "stream/event creation failed"));
    {   // dataflow grids: every block that fits (a required-time sweep flushed for a
        // query and an adjoint sweep on another stream then run one after the other)
        const int fmax = bat ? batch_max_blocks(1) : dataflow_max_blocks(1, h->nl > 1);
        const int bmax = bat ? batch_max_blocks(0) : dataflow_max_blocks(0, h->nl > 1);
        h->grid_fwd = fmax > 0 ? fmax : 1;
        h->grid_bwd = bmax > 0 ? bmax : 1;
        if (bat) {  // (sta_autotune may switch to them)
            h->grid_bwd_w = std::max(1, batch_wide_max_blocks());
            h->grid_fwd_w = std::max(1, batch_wide_fwd_max_blocks());
        }
        if (opts && opts->grid_blocks > 0) {
            h->grid_fwd = std::min(h->grid_fwd, (int)opts->grid_blocks);
            h->grid_bwd = std::min(h->grid_bwd, (int)opts->grid_blocks);
            h->grid_bwd_w = std::min(h->grid_bwd_w, (int)opts->grid_blocks);
            h->grid_fwd_w = std::min(h->grid_fwd_w, (int)opts->grid_blocks);
        }
        if (cudaGetLastError() != cudaSuccess) return fail(set_err(STA_ERR_CUDA, "occupancy query failed"));
    }
    if (h->profile) {  // event pairs for every launch of each sequence, made before any capture
        const size_t nl = (size_t)L.L;
        const std::pair<StaHandle::Prof*, size_t> sizes[] = {
            {&h->prof_pos, 3}, {&h->prof_fwd, nl + 5}, {&h->prof_rat, 2 * nl + 2}, {&h->prof_adj, 2 * nl + 3},
            {&h->prof_out, 1}};
        for (const auto& ps : sizes) {
            ps.first->kind.assign(ps.second, 0);
            for (size_t k = 0; k < 2 * ps.second; ++k) {
                cudaEvent_t e = nullptr;
                if (cudaEventCreate(&e) != cudaSuccess) return fail(set_err(STA_ERR_CUDA, "cudaEventCreate failed"));
                ps.first->ev.push_back(e);
            }
        }
    }
    // A pooled handle (the server's) does not wait for its creation work: its
    // allocations, uploads and fills are queued on the legacy stream, and the
    // events recorded there below order every later call after them (each call
    // waits for ev_fwd / ev_bwd / ev_at before touching the handle's memory).
    ce = pool ? cudaGetLastError() : cudaDeviceSynchronize();
    if (ce != cudaSuccess) return fail(set_err(STA_ERR_CUDA, std::string("init: ") + cudaGetErrorString(ce)));
    cudaEventRecord(h->ev_at, 0);
    cudaEventRecord(h->ev_fwd, 0);
    cudaEventRecord(h->ev_bwd, 0);
    *out = h;
    return STA_OK;
}
}  // namespace

extern "C" {

void sta_destroy(StaHandle* h) {
    if (!h) return;
    if (!h->pool) cudaDeviceSynchronize();  // (a pooled handle's owner knows it idle)
    delete h;
}

StaStatus sta_set_positions(StaHandle* h, const float* xy, int on_device, void* stream) {
    if (!h || (!xy && h->lay.P > 0)) return set_err(STA_ERR_INVALID_ARG, "null argument");
    if (on_device && reinterpret_cast<uintptr_t>(xy) % 8)  // read as float2 by the gather kernels
        return set_err(STA_ERR_INVALID_ARG, "sta_set_positions: device xy must be 8-byte aligned");
    cudaStream_t st = as_stream(stream);
    // do not overwrite positions that a pending sweep still reads
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_bwd, 0));
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    const float2* src = reinterpret_cast<const float2*>(xy);
    if (!h->batch()) h->active = h->active_next;  // lanes: the placements of this and the following calls
    const size_t bytes = (size_t)h->lay.P * 8 * (h->batch() ? h->B : h->active);
    if (!on_device) {
        StaStatus s2 = h->staging(bytes, st);
        if (s2 != STA_OK) return s2;
        if (bytes) CUDA_TRY(cudaMemcpyAsync(h->stage, xy, bytes, cudaMemcpyHostToDevice, st));
        src = static_cast<const float2*>(h->stage);
    }
    h->prof_pos.next = 0;
    if (batch_resets_needed(h)) {  // beside the transpose: the next forward waits for them
        CUDA_TRY(cudaEventRecord(h->ev_fork[0], st));
        CUDA_TRY(cudaStreamWaitEvent(h->fork, h->ev_fork[0], 0));
        enqueue_batch_resets(h, &h->prof_pos, h->fork);
        CUDA_TRY(cudaEventRecord(h->ev_fork[1], h->fork));
    }
    {
        ProfScope ps(h, &h->prof_pos, STA_PROF_POSITIONS, st);
        if (h->batch()) launch_batch_xy_in(h->bs, h->pin_int, h->lay.P, src, st);
        else launch_gather_xy(h->g, h->s, src, h->active, st);
    }
    StaStatus s3 = check_launch();
    if (s3 != STA_OK) return s3;
    h->pre_reset = batch_resets_needed(h);
    h->have_pos = true;
    h->have_fwd = h->have_lse = h->have_rat = false;
    h->rat_pending = false;  // its results could no longer be queried
    return STA_OK;
}

StaStatus sta_forward(StaHandle* h, uint32_t flags, float gamma, void* stream) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    if (!h->have_pos) return set_err(STA_ERR_STATE, "sta_set_positions must come before sta_forward");
    const int lse = (flags & STA_FWD_LSE) ? 1 : 0;
    if (lse && !(std::isfinite(gamma) && gamma > 0.f)) return set_err(STA_ERR_INVALID_ARG, "gamma must be > 0");
    if (!lse) gamma = 1.f;
    ++h->nforward;
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_bwd, 0));
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    if (batch_resets_needed(h)) {  // the sweeps' polled words: reset with the positions, or now
        if (h->pre_reset) CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fork[1], 0));
        else enqueue_batch_resets(h, &h->prof_pos, st);
        h->pre_reset = false;
    }
    if (h->expire_next) {
        // one forward task waits for a producer that never comes: its wait runs
        // into the budget, the sweep ends early and the expiry is reported
        h->expire_next = false;
        const Layout& L = h->lay;
        // (the levels schedules reject the hook: they never wait)
        if (L.TF == 0) return set_err(STA_ERR_STATE, "no forward task");
        h->stall_task = L.TF - 1;  // its wait for its fanin words never succeeds
        enqueue_forward(h, lse, gamma, st);
        h->stall_task = -1;
        StaStatus s2 = check_launch();
        if (s2 != STA_OK) return s2;
    } else if (h->graphs_now()) {
        if (!h->gx_fwd[lse] || h->gx_fwd_gamma[lse] != gamma) {
            StaStatus s2 = capture(h, &h->gx_fwd[lse], [&](cudaStream_t c) { enqueue_forward(h, lse, gamma, c); });
            if (s2 != STA_OK) return s2;
            h->gx_fwd_gamma[lse] = gamma;
        }
        CUDA_TRY(cudaGraphLaunch(h->gx_fwd[lse], st));
    } else {
        enqueue_forward(h, lse, gamma, st);
        StaStatus s2 = check_launch();
        if (s2 != STA_OK) return s2;
    }
    CUDA_TRY(cudaEventRecord(h->ev_at, st));
    h->rat_pending = false;
    if ((flags & STA_FWD_RAT) && h->schedule != STA_SCHED_LEVELS && !(flags & STA_FWD_RAT_EAGER)) {
        // deferred: carried by the next gradient sweep, or launched when queried
        h->rat_pending = true;
        CUDA_TRY(cudaEventRecord(h->ev_fwd, st));
    } else if ((flags & STA_FWD_RAT) && h->schedule != STA_SCHED_LEVELS) {
        StaStatus s2 = launch_graph_or_direct(h, &h->gx_rat, &h->gx_rat_gamma, 1.f, 1, st);
        if (s2 != STA_OK) return s2;
        CUDA_TRY(cudaEventRecord(h->ev_fwd, st));
    } else if (flags & STA_FWD_RAT) {
        CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_at, 0));
        StaStatus s2 = launch_graph_or_direct(h, &h->gx_rat, &h->gx_rat_gamma, 1.f, 1, h->side);
        if (s2 != STA_OK) return s2;
        CUDA_TRY(cudaEventRecord(h->ev_fwd, h->side));
    } else {
        CUDA_TRY(cudaEventRecord(h->ev_fwd, st));
    }
    h->have_fwd = true;
    h->have_lse = lse != 0;
    h->have_rat = (flags & STA_FWD_RAT) != 0;
    h->gamma_fwd = gamma;
    return STA_OK;
}

StaStatus sta_backward_grad(StaHandle* h, const float* w, int w_on_device, float* grad_xy, int on_device,
                            void* stream) {
    if (!h || !w || (!grad_xy && h->lay.P > 0)) return set_err(STA_ERR_INVALID_ARG, "null argument");
    if ((on_device && reinterpret_cast<uintptr_t>(grad_xy) % 8) || (w_on_device && reinterpret_cast<uintptr_t>(w) % 4))
        return set_err(STA_ERR_INVALID_ARG, "sta_backward_grad: device grad_xy must be 8-byte, w 4-byte aligned");
    if (!h->have_lse) return set_err(STA_ERR_STATE, "sta_forward with STA_FWD_LSE must come before sta_backward_grad");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_at, 0));
    if (h->batch()) {  // one weight pair per placement
        CUDA_TRY(cudaMemcpyAsync(h->bs.params, w, sizeof(float) * 2 * h->B,
                                 w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else if (h->lay.G > 1) {  // several netlists: one weight pair each
        CUDA_TRY(cudaMemcpyAsync(h->s.params, w, sizeof(float) * 2 * h->lay.G,
                                 w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else if (h->nl > 1) {  // lanes: pair l into lane l's parameters
        CUDA_TRY(cudaMemcpy2DAsync(h->s.params, h->s.lane_bytes, w, 2 * sizeof(float), 2 * sizeof(float), h->active,
                                   w_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st));
    } else {
        launch_set_weights(h->s, w_on_device ? w : nullptr, w_on_device ? 0.f : w[0], w_on_device ? 0.f : w[1], st);
    }
    const float gamma = h->gamma_fwd;
    h->last_fused = h->rat_pending;
    if (h->rat_pending) {  // one sweep for the required times and the adjoint
        h->rat_pending = false;
        StaStatus s2 = launch_graph_or_direct(h, &h->gx_fused, &h->gx_fused_gamma, gamma, 3, st);
        if (s2 != STA_OK) return s2;
        CUDA_TRY(cudaEventRecord(h->ev_fwd, st));
    } else {
        StaStatus s2 = launch_graph_or_direct(h, &h->gx_adj, &h->gx_adj_gamma, gamma, 2, st);
        if (s2 != STA_OK) return s2;
    }
    if (h->batch()) {  // internal [P][Bp] -> the caller's [B][P][2]
        const size_t bytes = (size_t)h->lay.P * 8 * h->B;
        float2* dst = reinterpret_cast<float2*>(grad_xy);
        if (!on_device) {
            StaStatus s2 = h->staging(bytes, st);
            if (s2 != STA_OK) return s2;
            dst = static_cast<float2*>(h->stage);
        }
        {
            h->prof_out.next = 0;
            ProfScope ps(h, &h->prof_out, STA_PROF_OUTPUT, st);
            launch_batch_out2(h->bs, h->pin_int, h->lay.P, h->bs.grad, dst, st);
        }
        StaStatus s3 = check_launch();
        if (s3 != STA_OK) return s3;
        if (!on_device && bytes) CUDA_TRY(cudaMemcpyAsync(grad_xy, dst, bytes, cudaMemcpyDeviceToHost, st));
    } else {
        // lane l's gradient (caller's pin order) to [l][P][2]
        const size_t bytes = (size_t)h->lay.P * 8;
        if (bytes) {
            CUDA_TRY(cudaMemcpy2DAsync(grad_xy, bytes, h->s.grad, h->s.lane_bytes, bytes, h->active,
                                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        }
    }
    CUDA_TRY(cudaEventRecord(h->ev_bwd, st));
    return on_device ? STA_OK : sync_checked(h, st);
}

StaStatus sta_set_active(StaHandle* h, int32_t lanes) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    if (h->nl <= 1) return set_err(STA_ERR_STATE, "sta_set_active: handles with STA_BATCH_LANES only");
    if (lanes < 1 || lanes > h->nl) return set_err(STA_ERR_INVALID_ARG, "sta_set_active: lanes in [1, num_placements]");
    h->active_next = lanes;
    return STA_OK;
}

StaStatus sta_stream_wait(StaHandle* h, void* stream) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_bwd, 0));
    return STA_OK;
}

StaStatus sta_synchronize(StaHandle* h) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_fwd, 0));
    CUDA_TRY(cudaStreamWaitEvent(h->side, h->ev_bwd, 0));
    return sync_checked(h, h->side);
}

StaStatus sta_debug_expire_wait(StaHandle* h) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    if (h->schedule == STA_SCHED_LEVELS || (h->batch() && h->bsweep == STA_BATCH_LEVELS))
        return set_err(STA_ERR_STATE, "level-synchronous sweeps have no waits");
    h->expire_next = true;
    return STA_OK;
}

StaStatus sta_autotune(StaHandle* h, const int32_t* tile_pins, int32_t n_tile, const int32_t* chunks,
                       int32_t n_chunk, const int32_t* sweeps, int32_t n_sweep, int32_t reps, float gamma, float* ms,
                       int32_t* best) {
    if (!h || !tile_pins || !chunks || !sweeps || n_tile < 1 || n_chunk < 1 || n_sweep < 1 || reps < 1 || !best)
        return set_err(STA_ERR_INVALID_ARG, "sta_autotune: null or empty candidate lists");
    if (!h->batch()) return set_err(STA_ERR_STATE, "sta_autotune: the batched schedule only");
    if (!h->have_pos) return set_err(STA_ERR_STATE, "sta_autotune: sta_set_positions first");
    if (!(std::isfinite(gamma) && gamma > 0.f)) return set_err(STA_ERR_INVALID_ARG, "gamma must be > 0");
    for (int32_t i = 0; i < n_tile; ++i)
        if (tile_pins[i] < 1) return set_err(STA_ERR_INVALID_ARG, "tile_pins must be >= 1");
    for (int32_t i = 0; i < n_chunk; ++i)
        if (chunks[i] < 1) return set_err(STA_ERR_INVALID_ARG, "chunk must be >= 1");
    for (int32_t i = 0; i < n_sweep; ++i)
        if (sweeps[i] != STA_BATCH_LEVELS && sweeps[i] != STA_BATCH_DATAFLOW && sweeps[i] != STA_BATCH_WIDE)
            return set_err(STA_ERR_INVALID_ARG, "sweeps: STA_BATCH_LEVELS, STA_BATCH_DATAFLOW or STA_BATCH_WIDE");
    CUDA_TRY(cudaDeviceSynchronize());
    cudaStream_t st = h->side;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    float best_ms = 0.f;
    int32_t bi = -1;
    StaStatus status = STA_OK;
    for (int32_t i = 0; i < n_tile && status == STA_OK; ++i)
        for (int32_t j = 0; j < n_chunk && status == STA_OK; ++j)
            for (int32_t k = 0; k < n_sweep && status == STA_OK; ++k) {
                TaskShape sh;
                sh.pack_pins = tile_pins[i];
                sh.pack_nets = 1 << 20;
                sh.chunk = chunks[j];
                sh.big = chunks[j] + 1;
                h->bsweep = sweeps[k];
                if ((status = set_tasks(h, sh)) != STA_OK) break;
                // one step (forward with LSE and required times, fused gradient sweep) as a graph
                cudaGraphExec_t gx = nullptr;
                status = capture(h, &gx, [&](cudaStream_t c) {
                    if (batch_resets_needed(h)) enqueue_batch_resets(h, nullptr, c);
                    enqueue_forward(h, 1, gamma, c);
                    enqueue_backward(h, 3, gamma, c);
                });
                if (status != STA_OK) break;
                float t = 0.f;
                cudaError_t e = cudaGraphLaunch(gx, st);  // warm-up
                if (e == cudaSuccess) e = cudaEventRecord(e0, st);
                for (int32_t r = 0; r < reps && e == cudaSuccess; ++r) e = cudaGraphLaunch(gx, st);
                if (e == cudaSuccess) e = cudaEventRecord(e1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
                cudaGraphExecDestroy(gx);
                if (e != cudaSuccess) {
                    status = set_err(STA_ERR_CUDA, std::string("sta_autotune: ") + cudaGetErrorString(e));
                    break;
                }
                t /= (float)reps;
                if (ms) ms[((size_t)i * n_chunk + j) * n_sweep + k] = t;
                if (bi < 0 || t < best_ms) {
                    best_ms = t;
                    bi = (int32_t)(((size_t)i * n_chunk + j) * n_sweep + k);
                    best[0] = tile_pins[i];
                    best[1] = chunks[j];
                    best[2] = sweeps[k];
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (status != STA_OK) return status;
    StaStatus s2 = sync_checked(h, st);  // a dataflow candidate whose wait expired
    if (s2 != STA_OK) return s2;
    TaskShape sh;
    sh.pack_pins = best[0];
    sh.pack_nets = 1 << 20;
    sh.chunk = best[1];
    sh.big = best[1] + 1;
    h->bsweep = best[2];
    return set_tasks(h, sh);
}

StaStatus sta_ablation_net_rc(StaHandle* h, int32_t scheme, int32_t reps, float* ms) {
    if (!h || reps < 1 || (scheme != STA_RC_PIN && scheme != STA_RC_CTE))
        return set_err(STA_ERR_INVALID_ARG, "sta_ablation_net_rc: scheme PIN or CTE, reps >= 1");
    if (h->batch()) return set_err(STA_ERR_STATE, "sta_ablation_net_rc: single-placement schedules only");
    if (!h->have_pos) return set_err(STA_ERR_STATE, "sta_ablation_net_rc: sta_set_positions first");
    const Layout& L = h->lay;
    cudaStream_t st = h->side;
    CUDA_TRY(cudaDeviceSynchronize());
    auto launch = [&] {
        if (scheme == STA_RC_CTE) launch_rc_cte(h->g, h->s, 0, L.N, st);
        else launch_rc(h->g, h->s, L.lvl_wtask[L.L], st);
    };
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    launch();  // warm-up
    cudaEventRecord(e0, st);
    for (int32_t r = 0; r < reps; ++r) launch();
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return set_err(STA_ERR_CUDA, std::string("sta_ablation_net_rc: ") + cudaGetErrorString(e));
    if (ms) *ms = t / (float)reps;
    h->have_fwd = h->have_lse = h->have_rat = false;  // the loads were rewritten: run sta_forward again
    h->rat_pending = false;
    return STA_OK;
}

StaStatus sta_query_net_rc(StaHandle* h, float* load, float* wdelay, float* impulse) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    if (h->batch()) return set_err(STA_ERR_STATE, "sta_query_net_rc: single-placement schedules only");
    const Layout& L = h->lay;
    CUDA_TRY(cudaDeviceSynchronize());
    if (load) {
        std::vector<float> v(L.N);
        if (L.N) CUDA_TRY(cudaMemcpy(v.data(), h->s.load, (size_t)L.N * 4, cudaMemcpyDeviceToHost));
        for (int32_t i = 0; i < L.N; ++i)
            if (L.net_orig[i] >= 0) load[L.net_orig[i]] = v[i];
    }
    if (wdelay || impulse) {
        std::vector<float2> v(L.P);
        if (L.P) CUDA_TRY(cudaMemcpy(v.data(), h->s.wdi, (size_t)L.P * 8, cudaMemcpyDeviceToHost));
        std::vector<char> sink(L.P, 0);
        for (int32_t n = 0; n < L.N; ++n)
            for (int32_t p = L.net_ptr[n] + 1; p < L.net_ptr[n + 1]; ++p) sink[p] = 1;
        for (int32_t p = 0; p < L.P; ++p) {
            const int32_t o = L.pin_orig[p];
            if (wdelay) wdelay[o] = sink[p] ? v[p].x : 0.f;
            if (impulse) impulse[o] = sink[p] ? v[p].y : 0.f;
        }
    }
    return STA_OK;
}

StaStatus sta_query_summary(StaHandle* h, double* out, int on_device, void* stream) {
    if (!h || !out) return set_err(STA_ERR_INVALID_ARG, "null argument");
    if (!h->have_fwd) return set_err(STA_ERR_STATE, "no forward pass yet");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (h->batch()) {
        CUDA_TRY(cudaMemcpyAsync(out, h->bs.summary, STA_SUM_COUNT * sizeof(double) * h->B, kind, st));
    } else if (h->lay.G > 1) {  // several netlists: netlist k's summary to out[k]
        CUDA_TRY(cudaMemcpyAsync(out, h->s.summary, STA_SUM_COUNT * sizeof(double) * h->lay.G, kind, st));
    } else {  // lane l's summary to out[l]
        CUDA_TRY(cudaMemcpy2DAsync(out, STA_SUM_COUNT * sizeof(double), h->s.summary, h->s.lane_bytes,
                                   STA_SUM_COUNT * sizeof(double), h->active, kind, st));
    }
    return on_device ? STA_OK : sync_checked(h, st);
}

namespace {

StaStatus deliver(StaHandle* h, const float* internal, int k, float* out, int on_device, cudaStream_t st) {
    const size_t bytes = (size_t)h->lay.P * k * sizeof(float) * (h->batch() ? h->B : h->active);
    if (!bytes) return STA_OK;
    float* dst = out;
    if (!on_device) {
        StaStatus s2 = h->staging(bytes, st);
        if (s2 != STA_OK) return s2;
        dst = static_cast<float*>(h->stage);
    }
    if (h->batch()) {
        launch_batch_out(h->bs, h->pin_int, h->lay.P, internal, k, dst, st);
    } else {  // lane l (internal points at lane 0's array) to out[l]
        for (int l = 0; l < h->active; ++l)
            launch_scatter(h->g, lane_ptr(internal, (size_t)l * h->s.lane_bytes), dst + (size_t)l * h->lay.P * k, k,
                           h->lay.P, st);
    }
    StaStatus s3 = check_launch();
    if (s3 != STA_OK) return s3;
    if (!on_device) {
        CUDA_TRY(cudaMemcpyAsync(out, dst, bytes, cudaMemcpyDeviceToHost, st));
        return sync_checked(h, st);
    }
    return STA_OK;
}

}  // namespace

StaStatus sta_query_pins(StaHandle* h, float* at, float* slew, float* rat, float* ats, float* slack, int on_device,
                         void* stream) {
    if (!h) return set_err(STA_ERR_INVALID_ARG, "null handle");
    if (on_device) {  // written by kernels: floats, and the slack pairs as float2
        for (const float* q : {at, slew, rat, ats})
            if (reinterpret_cast<uintptr_t>(q) % 4)
                return set_err(STA_ERR_INVALID_ARG, "sta_query_pins: device outputs must be 4-byte aligned");
        if (reinterpret_cast<uintptr_t>(slack) % 8)
            return set_err(STA_ERR_INVALID_ARG, "sta_query_pins: device slack must be 8-byte aligned");
    }
    if (!h->have_fwd) return set_err(STA_ERR_STATE, "no forward pass yet");
    if ((rat || slack) && !h->have_rat) return set_err(STA_ERR_STATE, "required times need STA_FWD_RAT");
    if (ats && !h->have_lse) return set_err(STA_ERR_STATE, "LSE arrival times need STA_FWD_LSE");
    if (rat || slack) {
        StaStatus s1 = flush_rat(h);
        if (s1 != STA_OK) return s1;
    }
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    StaStatus s2 = STA_OK;
    const bool bat = h->batch();
    if (at && (s2 = deliver(h, bat ? h->bs.at : h->s.at, 4, at, on_device, st)) != STA_OK) return s2;
    if (slew && (s2 = deliver(h, bat ? h->bs.slew : h->s.slew, 4, slew, on_device, st)) != STA_OK) return s2;
    if (rat && (s2 = deliver(h, bat ? h->bs.rat : h->s.rat, 4, rat, on_device, st)) != STA_OK) return s2;
    if (ats && (s2 = deliver(h, bat ? h->bs.ats : h->s.ats, 2, ats, on_device, st)) != STA_OK) return s2;
    if (slack && bat) {
        const size_t need = (size_t)h->lay.P * 2 * h->bs.Bp * sizeof(float);
        if (need > h->qscratch_bytes) {
            if (h->qscratch) cudaFree(h->qscratch);
            h->qscratch = nullptr;
            h->qscratch_bytes = 0;
            CUDA_TRY(cudaMalloc(&h->qscratch, need));
            h->qscratch_bytes = need;
        }
        if (need) {
            launch_batch_pin_slack(h->bs, h->lay.P, h->qscratch, st);
            if ((s2 = check_launch()) != STA_OK) return s2;
            if ((s2 = deliver(h, h->qscratch, 2, slack, on_device, st)) != STA_OK) return s2;
        }
    } else if (slack) {
        const size_t bytes = (size_t)h->lay.P * 8 * h->active;
        if (bytes) {
            float* dst = slack;
            if (!on_device) {
                if ((s2 = h->staging(bytes, st)) != STA_OK) return s2;
                dst = static_cast<float*>(h->stage);
            }
            for (int l = 0; l < h->active; ++l)
                launch_pin_slack(h->g, lane_state(h->s, l), dst + (size_t)l * h->lay.P * 2, st);
            if ((s2 = check_launch()) != STA_OK) return s2;
            if (!on_device) {
                CUDA_TRY(cudaMemcpyAsync(slack, dst, bytes, cudaMemcpyDeviceToHost, st));
                if ((s2 = sync_checked(h, st)) != STA_OK) return s2;
            }
        }
    }
    return STA_OK;
}

StaStatus sta_query_endpoints(StaHandle* h, float* slack, int on_device, void* stream) {
    if (!h || (!slack && h->lay.E > 0)) return set_err(STA_ERR_INVALID_ARG, "null argument");
    if (!h->have_fwd) return set_err(STA_ERR_STATE, "no forward pass yet");
    cudaStream_t st = as_stream(stream);
    CUDA_TRY(cudaStreamWaitEvent(st, h->ev_fwd, 0));
    if (h->lay.E && h->batch()) {
        const size_t bytes = (size_t)h->lay.E * 8 * h->B;
        float2* dst = reinterpret_cast<float2*>(slack);
        if (!on_device) {
            StaStatus s2 = h->staging(bytes, st);
            if (s2 != STA_OK) return s2;
            dst = static_cast<float2*>(h->stage);
        }
        launch_batch_ep_out(h->bs, h->lay.E, dst, st);
        StaStatus s3 = check_launch();
        if (s3 != STA_OK) return s3;
        if (!on_device) {
            CUDA_TRY(cudaMemcpyAsync(slack, dst, bytes, cudaMemcpyDeviceToHost, st));
            return sync_checked(h, st);
        }
    } else if (h->lay.E) {  // lane l's endpoint slacks to slack[l]
        CUDA_TRY(cudaMemcpy2DAsync(slack, (size_t)h->lay.E * 8, h->s.ep_slack, h->s.lane_bytes, (size_t)h->lay.E * 8,
                                   h->active, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
        if (!on_device) return sync_checked(h, st);
    }
    return STA_OK;
}

StaStatus sta_query_profile(StaHandle* h, double* ms, int32_t* launches) {
    if (!h || !launches) return set_err(STA_ERR_INVALID_ARG, "null argument");
    const Layout& L = h->lay;
    // launches of one step, by kind (levels with no task launch nothing)
    int32_t nonempty = 0;
    for (int l = 0; l < L.L; ++l)
        nonempty += (L.lvl_wtask[l + 1] > L.lvl_wtask[l] || L.lvl_ctask[l + 1] > L.lvl_ctask[l]) ? 1 : 0;
    const int32_t nw = L.lvl_wtask.empty() ? 0 : L.lvl_wtask.back(), nc = L.lvl_ctask.empty() ? 0 : L.lvl_ctask.back();
    launches[STA_PROF_POSITIONS] = L.P > 0 ? 1 : 0;
    launches[STA_PROF_ENDPOINTS] = h->batch() ? 2 : 1;
    launches[STA_PROF_OUTPUT] = (h->batch() && L.P > 0) ? 1 : 0;
    launches[STA_PROF_RESET] = 0;
    if (h->batch() && h->bsweep == STA_BATCH_LEVELS) {
        std::vector<std::array<int, 6>> ph;
        batch_bwd_phases(L, 3, ph);
        const int32_t nb = (int32_t)ph.size();
        batch_bwd_phases(L, 1, ph);
        launches[STA_PROF_NET_RC] = (h->bload.n > 0 ? 1 : 0) + (L.N > 0 ? 1 : 0);
        launches[STA_PROF_FORWARD] = batch_fwd_levels(L);
        launches[STA_PROF_REQUIRED] = h->last_fused ? 0 : (int32_t)ph.size();
        launches[STA_PROF_SEED] = 1 + (h->g.ep_clk ? 1 : 0);
        launches[STA_PROF_ADJOINT] = nb;
    } else if (h->batch()) {
        // each sweep is preceded by the reset of the words its tasks poll
        launches[STA_PROF_NET_RC] = h->bload.n > 0 ? 1 : 0;
        launches[STA_PROF_FORWARD] = L.TF > 0 ? 1 : 0;
        launches[STA_PROF_REQUIRED] = (L.TB > 0 && !h->last_fused) ? 1 : 0;
        launches[STA_PROF_SEED] = 1 + (h->g.ep_clk ? 1 : 0);  // weights (+ capture-clock seeds)
        launches[STA_PROF_ADJOINT] = L.TB > 0 ? 1 : 0;
        // the forward's polled words and the fused sweep's, reset with the positions
        launches[STA_PROF_RESET] = 2 + (h->last_fused ? 0 : launches[STA_PROF_REQUIRED] + launches[STA_PROF_ADJOINT]);
    } else if (h->schedule == STA_SCHED_DATAFLOW) {
        // the prologue (large-net RC + reset of the forward's polled words) is one
        // launch; the endpoint launch also resets the fused sweep's polled words
        launches[STA_PROF_NET_RC] = (nc > 0 || L.P > 0) ? 1 : 0;
        launches[STA_PROF_FORWARD] = L.TF > 0 ? 1 : 0;
        launches[STA_PROF_REQUIRED] = (L.TB > 0 && !h->last_fused) ? 1 : 0;  // fused into the adjoint sweep
        launches[STA_PROF_SEED] = 1 + (h->g.ep_clk ? 1 : 0);  // weights (+ capture-clock seeds)
        launches[STA_PROF_ADJOINT] = L.TB > 0 ? 1 : 0;
        // a separate required-time or adjoint sweep resets its own words
        const int32_t br = (L.P > 0 || L.npart > 0) ? 1 : 0;
        launches[STA_PROF_RESET] = h->last_fused ? 0 : br * (launches[STA_PROF_REQUIRED] + launches[STA_PROF_ADJOINT]);
    } else {
        launches[STA_PROF_NET_RC] = (nw + nc) > 0 ? 1 : 0;
        launches[STA_PROF_FORWARD] = nonempty;
        launches[STA_PROF_REQUIRED] = nonempty;
        launches[STA_PROF_SEED] = 1 + (L.E > 0 ? 1 : 0) + (h->g.ep_clk ? 1 : 0);  // weights + seeds
        launches[STA_PROF_ADJOINT] = nonempty;
    }
    if (!ms) return STA_OK;
    for (int k = 0; k < STA_PROF_KINDS; ++k) ms[k] = 0.0;
    if (!h->profile) return set_err(STA_ERR_STATE, "handle was created without StaOptions.profile");
    CUDA_TRY(cudaDeviceSynchronize());
    for (StaHandle::Prof* pr : {&h->prof_pos, &h->prof_fwd, &h->prof_rat, &h->prof_adj, &h->prof_out}) {
        for (size_t i = 0; i < pr->next && 2 * i + 1 < pr->ev.size(); ++i) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, pr->ev[2 * i], pr->ev[2 * i + 1]) == cudaSuccess) ms[pr->kind[i]] += t;
            else cudaGetLastError();
        }
    }
    return STA_OK;
}

StaStatus sta_plan_tasks(const StaNetlistDesc* nl, const StaLibrary* lib, int32_t tile_pins, int32_t tile_nets,
                         int32_t chunk, int64_t* o) {
    if (!nl || !lib || !o) return set_err(STA_ERR_INVALID_ARG, "null argument");
    try {
        Layout L;
        std::string err;
        StaStatus st = build_layout(*nl, *lib, L, err);
        if (st != STA_OK) return set_err(st, err);
        TaskShape sh;
        sh.pack_pins = tile_pins;
        sh.pack_nets = tile_nets;
        sh.chunk = chunk;
        sh.big = chunk + 1;
        st = build_tasks(L, sh, err);
        if (st != STA_OK) return set_err(st, err);
        int64_t chunks = 0, max_pins = 0, max_nets = 0, edges_f = (int64_t)L.f_out.size();
        for (int32_t t = 0; t < L.TF; ++t) {
            const int32_t nn = L.ftask[4 * t + 1];
            if (nn < 0) {
                ++chunks;
                continue;
            }
            max_nets = std::max<int64_t>(max_nets, nn);
            max_pins = std::max<int64_t>(max_pins, L.ftask[4 * t + 3]);
        }
        o[0] = L.TF;
        o[1] = L.TB;
        o[2] = L.npart;
        o[3] = chunks;
        o[4] = max_pins;
        o[5] = max_nets;
        o[6] = edges_f;
        o[7] = (int64_t)L.big_nets.size();
        return STA_OK;
    } catch (const std::bad_alloc&) {
        return set_err(STA_ERR_OOM, "host allocation failed");
    }
}

StaStatus sta_query_slack(StaHandle* h, float* wns_tns, float* pin_slack, float* endpoint_slack) {
    if (!h || !wns_tns) return set_err(STA_ERR_INVALID_ARG, "null argument");
    if (h->batch() || h->nl > 1 || h->lay.G > 1)
        return set_err(STA_ERR_STATE, "sta_query_slack: single-placement, single-netlist handles (use the queries)");
    double sum[STA_SUM_COUNT];
    StaStatus st = sta_query_summary(h, sum, 0, nullptr);
    if (st != STA_OK) return st;
    wns_tns[0] = (float)sum[STA_SUM_WNS_EARLY];
    wns_tns[1] = (float)sum[STA_SUM_TNS_EARLY];
    wns_tns[2] = (float)sum[STA_SUM_WNS_LATE];
    wns_tns[3] = (float)sum[STA_SUM_TNS_LATE];
    if (pin_slack && (st = sta_query_pins(h, nullptr, nullptr, nullptr, nullptr, pin_slack, 0, nullptr)) != STA_OK)
        return st;
    if (endpoint_slack && (st = sta_query_endpoints(h, endpoint_slack, 0, nullptr)) != STA_OK) return st;
    return STA_OK;
}

StaStatus sta_query_sizes(const StaHandle* h, int64_t* o) {
    if (!h || !o) return set_err(STA_ERR_INVALID_ARG, "null argument");
    const Layout& L = h->lay;
    o[0] = L.P;
    o[1] = L.N;
    o[2] = L.L;
    o[3] = L.A;
    o[4] = L.E;
    o[5] = L.lvl_wtask.empty() ? 0 : L.lvl_wtask.back();
    o[6] = L.lvl_ctask.empty() ? 0 : L.lvl_ctask.back();
    o[7] = (int64_t)h->dev_bytes;
    return STA_OK;
}

}  // extern "C"
