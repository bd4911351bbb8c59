// serve.cu -- a request loop over resident netlists (continuous batching).
//
// The server keeps netlists resident on the device under a memory budget and
// runs STA / gradient requests on a pool of CUDA streams ("slots").  A worker
// thread admits requests as slots and memory free up: a request whose netlist
// is resident and idle starts on a free slot at once, whatever the requests
// before it wait for, so the work of requests on different netlists overlaps
// on the device.  Requests of one netlist run one after another (they share
// the netlist's device state), or concurrently on its copies (replicas).
// When the budget binds, requests of resident netlists go first; a netlist
// that is not resident is brought in by evicting least recently used idle
// netlists without pending requests (any idle one once the oldest request has
// waited 20 ms), and it serves its queue before it can be evicted; bringing it
// in allocates and uploads the host layout built once at registration.
// Every request's result is that of the same request run alone: the kernels
// are deterministic and a netlist's state is only touched by its own requests.
//
// With merge = M > 0, pending requests of one netlist with the same gamma and
// kind run together, up to M at a time, as the lanes of one call of a lanes
// handle (STA_BATCH_LANES: independent placements of the single-placement
// sweeps), which runs only the lanes it is given; each lane's results are those
// of the same placement alone.
//
// With sequential = 1 the server is the plain one-request-per-launch loop:
// one slot, strict arrival order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "sta.h"
#include "sta_internal.h"

namespace sta {
void set_last_error_text(const std::string& msg);
}

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// how long the oldest pending request may wait before an admission for it may
// evict netlists that still have pending requests
constexpr double kStarveS = 0.02;

// Host copy of a netlist description and library (the caller's arrays are
// only borrowed during sta_server_add_netlist).
struct HostNetlist {
    std::vector<int32_t> net_ptr, net_pins, cell_type, cell_in_ptr, cell_in_pins, cell_out_pin, start_pins, end_pins,
        end_clock;
    std::vector<float> pin_cap, start_at, start_slew, end_rat;
    std::vector<int32_t> type_num_arcs;
    std::vector<int8_t> arc_unate;
    std::vector<float> slew_index, load_index, delay_tab, slew_tab;
    StaNetlistDesc nl{};
    StaLibrary lib{};
};

template <typename T>
void copy_in(std::vector<T>& v, const T* p, size_t n) {
    v.assign(p, p + n);
}

// One resident copy of a netlist: a handle and its request scratch.  A netlist
// may have several (StaServerOptions.replicas), so that its requests run
// concurrently, each on its own state.
struct Rep {
    StaHandle* h = nullptr;
    size_t bytes = 0;           // device bytes (the handle's allocations and the scratch)
    bool busy = false;
    double last_use = 0.0;
    float* grad_dev = nullptr;  // [M][P][2] device gradient of the request(s) in flight (M = 1 unmerged)
    double* sum_dev = nullptr;  // [M][STA_SUM_COUNT]
    float* xy_dev = nullptr;    // merged: [M][P][2] positions of the placements in flight
    float* w_host = nullptr;    // merged: pinned [M][2] loss weights of the placements in flight
    bool pooled = false;        // the scratch (and the handle's memory) came from the server's pool
    cudaEvent_t ready = nullptr;  // pooled: the copy's allocations and uploads (legacy stream) done
};

struct Net {
    HostNetlist host;
    std::shared_ptr<const sta::Layout> layout;  // built once at registration; every copy is created from it
    std::vector<const void*> pinned;            // layout arrays page-locked for the copies' uploads
    ~Net() {
        for (const void* p : pinned) cudaHostUnregister(const_cast<void*>(p));
    }
    std::vector<Rep*> reps;     // resident copies
    size_t rep_bytes = 0;       // measured bytes of one copy (0: not created yet, estimate)
    int32_t P = 0;
};

struct Req {
    StaServerRequest r;
    int64_t id;
    double t_arrival;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    bool busy = false;
    std::vector<Req> reqs;       // the request(s) in flight (several when merged)
    Rep* rep = nullptr;          // the netlist copy they run on
    double t_start = 0.0;
    double* sum_host = nullptr;  // pinned [M][STA_SUM_COUNT]
};

}  // namespace

struct StaServer {
    StaServerOptions opt{};
    int device = 0;
    std::vector<Net*> nets;
    std::vector<Slot> slots;
    size_t resident_bytes = 0;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Req> incoming;  // submitted, not yet seen by the worker
    std::vector<StaServerCompletion> done;
    int64_t next_id = 0;
    int64_t admissions = 0, evictions = 0;
    // during an admission round: pending requests per netlist, and whether an
    // eviction may take a netlist that still has some (the oldest request has
    // waited kStarveS)
    std::vector<int32_t> npend;
    bool evict_pending = true;
    // device memory of the resident copies: a stream-ordered pool that keeps
    // up to the budget, so that admissions and evictions while other requests
    // run neither go to the driver's allocator nor wait for the whole device
    cudaMemPool_t pool = nullptr;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::string fatal;  // first worker error, reported by later calls

    ~StaServer();
    void run();
};

namespace {

StaStatus fail(const std::string& msg, StaStatus st = STA_ERR_INVALID_ARG) {
    sta::set_last_error_text(msg);
    return st;
}

// Copy a description (and library) into host-owned arrays.
StaStatus copy_netlist(const StaNetlistDesc& d, const StaLibrary& l, HostNetlist& o) {
    if (d.num_pins < 0 || d.num_nets < 0 || d.num_cells < 0 || d.num_start < 0 || d.num_end < 0 || l.num_types < 1)
        return fail("sta_server_add_netlist: negative sizes");
    if ((d.num_nets > 0 && (!d.net_ptr || !d.net_pins)) || (d.num_cells > 0 && (!d.cell_type || !d.cell_in_ptr ||
                                                                               !d.cell_out_pin)) ||
        (d.num_pins > 0 && !d.pin_cap) || (d.num_start > 0 && (!d.start_pins || !d.start_at || !d.start_slew)) ||
        (d.num_end > 0 && (!d.end_pins || !d.end_rat)) || !l.type_num_arcs || !l.arc_unate || !l.slew_index ||
        !l.load_index || !l.delay_tab || !l.slew_tab)
        return fail("sta_server_add_netlist: null array");
    const size_t N = d.num_nets, C = d.num_cells, T = l.num_types;
    copy_in(o.net_ptr, d.net_ptr, N + 1);
    copy_in(o.net_pins, d.net_pins, N ? (size_t)std::max(o.net_ptr[N], 0) : 0);
    copy_in(o.cell_type, d.cell_type, C);
    copy_in(o.cell_in_ptr, d.cell_in_ptr, C + 1);
    copy_in(o.cell_in_pins, d.cell_in_pins, C ? (size_t)std::max(o.cell_in_ptr[C], 0) : 0);
    copy_in(o.cell_out_pin, d.cell_out_pin, C);
    copy_in(o.pin_cap, d.pin_cap, (size_t)d.num_pins);
    copy_in(o.start_pins, d.start_pins, (size_t)d.num_start);
    copy_in(o.start_at, d.start_at, (size_t)d.num_start * 4);
    copy_in(o.start_slew, d.start_slew, (size_t)d.num_start * 4);
    copy_in(o.end_pins, d.end_pins, (size_t)d.num_end);
    copy_in(o.end_rat, d.end_rat, (size_t)d.num_end * 4);
    if (d.end_clock) copy_in(o.end_clock, d.end_clock, (size_t)d.num_end);
    copy_in(o.type_num_arcs, l.type_num_arcs, T);
    copy_in(o.arc_unate, l.arc_unate, T * STA_MAX_ARCS);
    copy_in(o.slew_index, l.slew_index, T * STA_LUT);
    copy_in(o.load_index, l.load_index, T * STA_LUT);
    copy_in(o.delay_tab, l.delay_tab, T * STA_MAX_ARCS * 2 * STA_LUT * STA_LUT);
    copy_in(o.slew_tab, l.slew_tab, T * STA_MAX_ARCS * 2 * STA_LUT * STA_LUT);
    o.nl = d;
    o.nl.net_ptr = o.net_ptr.data();
    o.nl.net_pins = o.net_pins.data();
    o.nl.cell_type = o.cell_type.data();
    o.nl.cell_in_ptr = o.cell_in_ptr.data();
    o.nl.cell_in_pins = o.cell_in_pins.data();
    o.nl.cell_out_pin = o.cell_out_pin.data();
    o.nl.pin_cap = o.pin_cap.data();
    o.nl.start_pins = o.start_pins.data();
    o.nl.start_at = o.start_at.data();
    o.nl.start_slew = o.start_slew.data();
    o.nl.end_pins = o.end_pins.data();
    o.nl.end_rat = o.end_rat.data();
    o.nl.end_clock = d.end_clock ? o.end_clock.data() : nullptr;
    o.lib = l;
    o.lib.type_num_arcs = o.type_num_arcs.data();
    o.lib.arc_unate = o.arc_unate.data();
    o.lib.slew_index = o.slew_index.data();
    o.lib.load_index = o.load_index.data();
    o.lib.delay_tab = o.delay_tab.data();
    o.lib.slew_tab = o.slew_tab.data();
    return STA_OK;
}

}  // namespace

// (only for a copy none of whose work is in flight)
static void release_rep(Rep* r) {
    if (r->h) sta_destroy(r->h);
    for (void* p : {(void*)r->grad_dev, (void*)r->sum_dev, (void*)r->xy_dev})
        if (p) {
            if (r->pooled) cudaFreeAsync(p, 0);
            else cudaFree(p);
        }
    if (r->w_host) cudaFreeHost(r->w_host);
    if (r->ready) cudaEventDestroy(r->ready);
    delete r;
}

StaServer::~StaServer() {
    stop = true;
    cv.notify_all();
    if (worker.joinable()) worker.join();
    for (Slot& s : slots) {
        if (s.st) cudaStreamSynchronize(s.st);
        if (s.done) cudaEventDestroy(s.done);
        if (s.st) cudaStreamDestroy(s.st);
        if (s.sum_host) cudaFreeHost(s.sum_host);
    }
    for (Net* n : nets) {
        for (Rep* r : n->reps) release_rep(r);
        delete n;
    }
    if (pool) {
        cudaDeviceSynchronize();  // the stream-ordered frees above
        cudaMemPoolDestroy(pool);
    }
}

namespace {

// Upper bound of the device bytes of a netlist's handle plus the server's
// scratch, from the description alone (used until it has been created once):
// per pin the per-pin state, staging and gradient scratch (132 B); per net or
// cell output the per-net arrays and the task lists (120 B); per arc the arc
// delays and dependency edges (32 B); per endpoint 28 B; with a propagated
// clock 4 B more per pin (clock seeds) and per endpoint (its clock pin).
// A lanes handle of M placements (merged requests) holds M copies of the
// per-placement state (at most the whole single-placement estimate each).
size_t estimate_bytes(const HostNetlist& hn, int merge) {
    const StaNetlistDesc& d = hn.nl;
    const size_t A = d.num_cells ? (size_t)hn.cell_in_ptr[d.num_cells] : 0;
    const size_t clk = d.end_clock ? 4 : 0;
    const size_t base = (size_t)d.num_pins * (132 + clk) + ((size_t)d.num_nets + d.num_cells) * 120 + A * 32 +
                        (size_t)d.num_end * (28 + clk) + (1u << 20);
    return merge <= 0 ? base : base * (size_t)merge;
}

}  // namespace

// Evict the least recently used idle copy (not `keep`) of a netlist with no
// pending request -- of any netlist if S->evict_pending; false if there is none.
static bool evict_one(StaServer* S, const Rep* keep) {
    Net* vn = nullptr;
    size_t vi = 0;
    for (size_t k = 0; k < S->nets.size(); ++k) {
        Net* m = S->nets[k];
        if (!S->evict_pending && k < S->npend.size() && S->npend[k] > 0) continue;
        for (size_t i = 0; i < m->reps.size(); ++i) {
            Rep* r = m->reps[i];
            if (r == keep || r->busy) continue;
            if (!vn || r->last_use < vn->reps[vi]->last_use) {
                vn = m;
                vi = i;
            }
        }
    }
    if (!vn) return false;
    Rep* r = vn->reps[vi];
    S->resident_bytes -= r->bytes;
    release_rep(r);
    vn->reps.erase(vn->reps.begin() + (long)vi);
    ++S->evictions;
    return true;
}

// An idle resident copy of netlist k for a request: an idle one if there is
// one; otherwise a new copy -- the first one evicting idle copies of other
// netlists in least-recently-used order if the budget needs it, further ones
// (up to StaServerOptions.replicas) only while the budget allows without
// evicting.  nullptr: none now (the request waits); err set: never.
static Rep* create_rep(StaServer* S, Net* n, std::string& err);

static int max_copies(const StaServer* S) { return S->opt.merge > 0 ? 1 : std::max(S->opt.replicas, 1); }

static Rep* admit(StaServer* S, int k, std::string& err) {
    Net* n = S->nets[k];
    for (Rep* r : n->reps)
        if (!r->busy) return r;
    if ((int)n->reps.size() >= max_copies(S)) return nullptr;
    return create_rep(S, n, err);
}

// A new resident copy of netlist n (see admit).
static Rep* create_rep(StaServer* S, Net* n, std::string& err) {
    const size_t need = n->rep_bytes ? n->rep_bytes : estimate_bytes(n->host, S->opt.merge);
    const size_t budget = (size_t)S->opt.budget_bytes;
    if (need > budget) {
        err = "netlist larger than the memory budget";
        return nullptr;
    }
    const bool first = n->reps.empty();
    while (S->resident_bytes + need > budget)
        if (!first || !evict_one(S, nullptr)) return nullptr;  // wait
    const int M = S->opt.merge > 0 ? S->opt.merge : 1;
    StaOptions o{};
    o.use_graphs = 1;
    o.schedule = S->opt.merge > 0 ? STA_SCHED_BATCH : STA_SCHED_DATAFLOW;
    if (S->opt.merge > 0) {  // M placements as lanes of the single-placement sweeps
        o.num_placements = M;
        o.batch_sweep = STA_BATCH_LANES;
    }
    // a netlist's persistent sweeps use a grid in proportion to its size, so the
    // sweeps of small netlists leave room for others on the device
    o.grid_blocks = S->opt.sequential ? 0 : std::max(8, n->P / 4000);
    Rep* r = new (std::nothrow) Rep();
    if (!r) {
        err = "host allocation failed";
        return nullptr;
    }
    // from the layout built at registration: an evicted netlist comes back
    // with allocations and uploads only, no host rebuild
    if (sta_create_from_layout(n->layout, &o, S->pool, &r->h) != STA_OK) {
        err = std::string("sta_create: ") + sta_last_error();
        r->h = nullptr;
        release_rep(r);
        return nullptr;
    }
    const size_t P1 = (size_t)std::max(n->P, 1);
    r->pooled = S->pool != nullptr;
    auto dmalloc = [&](auto** p, size_t bytes) {
        void** q = reinterpret_cast<void**>(p);
        return (S->pool ? cudaMallocFromPoolAsync(q, bytes, S->pool, 0) : cudaMalloc(q, bytes)) == cudaSuccess;
    };
    if (!dmalloc(&r->grad_dev, M * P1 * 8) || !dmalloc(&r->sum_dev, M * STA_SUM_COUNT * sizeof(double)) ||
        (S->opt.merge > 0 && (!dmalloc(&r->xy_dev, M * P1 * 8) ||
                              cudaMallocHost(&r->w_host, M * 2 * sizeof(float)) != cudaSuccess)) ||
        // pool: the slot stream of the copy's first request waits for this event
        // (its allocations, uploads and fills on the legacy stream), so the
        // worker dispatches other requests while the copy loads
        (S->pool && (cudaEventCreateWithFlags(&r->ready, cudaEventDisableTiming) != cudaSuccess ||
                     cudaEventRecord(r->ready, 0) != cudaSuccess))) {
        err = "cudaMalloc of request scratch failed";
        release_rep(r);
        return nullptr;
    }
    int64_t sz[8];
    sta_query_sizes(r->h, sz);
    // measured size (the handle's allocations, its host-input staging, the scratch)
    r->bytes = (size_t)sz[7] + (S->opt.merge > 0 ? 3 : 2) * M * P1 * 8 + M * STA_SUM_COUNT * sizeof(double);
    n->rep_bytes = r->bytes;
    n->reps.push_back(r);
    S->resident_bytes += r->bytes;
    ++S->admissions;
    while (S->resident_bytes > budget) {  // the estimate was low: make room, or give up
        if (first && evict_one(S, r)) continue;
        S->resident_bytes -= r->bytes;
        n->reps.pop_back();
        release_rep(r);
        ++S->evictions;
        if (n->rep_bytes > budget) err = "netlist larger than the memory budget";
        return nullptr;
    }
    return r;
}

// Queue one request's work on a slot's stream: positions in, forward, gradient
// if asked, results out; an event marks its end.
// a pooled copy's requests wait on the device for its loading (legacy stream)
static StaStatus wait_loaded(const Rep* rp, cudaStream_t st) {
    return (rp->ready && cudaStreamWaitEvent(st, rp->ready, 0) != cudaSuccess) ? STA_ERR_CUDA : STA_OK;
}

static StaStatus dispatch(StaServer* S, Slot& sl, Net* n) {
    const StaServerRequest& r = sl.reqs[0].r;
    Rep* rp = sl.rep;
    StaHandle* h = rp->h;
    void* st = sl.st;
    StaStatus s = wait_loaded(rp, sl.st);
    if (s == STA_OK) s = sta_set_positions(h, r.xy, 0, st);
    if (s == STA_OK)
        s = sta_forward(h, STA_FWD_LSE | STA_FWD_RAT | (r.gradient ? 0u : STA_FWD_RAT_EAGER), r.gamma, st);
    if (s == STA_OK && r.gradient) {
        const float w[2] = {r.w_tns, r.w_wns};
        s = sta_backward_grad(h, w, 0, rp->grad_dev, 1, st);
        if (s == STA_OK && r.grad &&
            cudaMemcpyAsync(r.grad, rp->grad_dev, (size_t)n->P * 8, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
            s = STA_ERR_CUDA;
    }
    if (s == STA_OK) s = sta_query_summary(h, rp->sum_dev, 1, st);
    if (s == STA_OK && cudaMemcpyAsync(sl.sum_host, rp->sum_dev, STA_SUM_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                       sl.st) != cudaSuccess)
        s = STA_ERR_CUDA;
    if (s == STA_OK && cudaEventRecord(sl.done, sl.st) != cudaSuccess) s = STA_ERR_CUDA;
    (void)S;
    return s;
}

// Merged: the slot's k requests (same netlist, gamma and kind) are lanes
// 0..k-1 of one call of the netlist's lanes handle, which runs those k lanes
// only (sta_set_active).  Each request's gradient and summary are copied out of
// its own lane.
static StaStatus dispatch_merged(StaServer* S, Slot& sl, Net* n) {
    const int M = (int)sl.reqs.size(), k = M;
    (void)S;
    const StaServerRequest& r0 = sl.reqs[0].r;
    const size_t P = (size_t)n->P;
    Rep* rp = sl.rep;
    cudaStream_t cst = sl.st;
    void* st = sl.st;
    StaStatus s = wait_loaded(rp, cst);
    if (s == STA_OK) s = sta_set_active(rp->h, k);
    for (int b = 0; b < k && s == STA_OK && P; ++b)
        if (cudaMemcpyAsync(rp->xy_dev + b * P * 2, sl.reqs[b].r.xy, P * 8, cudaMemcpyHostToDevice, cst) != cudaSuccess)
            s = STA_ERR_CUDA;
    if (s == STA_OK) s = sta_set_positions(rp->h, rp->xy_dev, 1, st);
    if (s == STA_OK)
        s = sta_forward(rp->h, STA_FWD_LSE | STA_FWD_RAT | (r0.gradient ? 0u : STA_FWD_RAT_EAGER), r0.gamma, st);
    if (s == STA_OK && r0.gradient) {
        for (int b = 0; b < M; ++b) {
            rp->w_host[2 * b] = b < k ? sl.reqs[b].r.w_tns : 0.f;
            rp->w_host[2 * b + 1] = b < k ? sl.reqs[b].r.w_wns : 0.f;
        }
        s = sta_backward_grad(rp->h, rp->w_host, 0, rp->grad_dev, 1, st);
        for (int b = 0; b < k && s == STA_OK; ++b)
            if (sl.reqs[b].r.grad && P &&
                cudaMemcpyAsync(sl.reqs[b].r.grad, rp->grad_dev + b * P * 2, P * 8, cudaMemcpyDeviceToHost, cst) !=
                    cudaSuccess)
                s = STA_ERR_CUDA;
    }
    if (s == STA_OK) s = sta_query_summary(rp->h, rp->sum_dev, 1, st);
    if (s == STA_OK && cudaMemcpyAsync(sl.sum_host, rp->sum_dev, (size_t)k * STA_SUM_COUNT * sizeof(double),
                                       cudaMemcpyDeviceToHost, cst) != cudaSuccess)
        s = STA_ERR_CUDA;
    if (s == STA_OK && cudaEventRecord(sl.done, cst) != cudaSuccess) s = STA_ERR_CUDA;
    return s;
}

void StaServer::run() {
    cudaSetDevice(device);
    std::vector<Req> pending;
    std::unique_lock<std::mutex> lk(mu);  // held except while waiting
    while (true) {
        bool any_busy = false;
        for (const Slot& s : slots) any_busy = any_busy || s.busy;
        if (incoming.empty() && pending.empty() && !any_busy) {
            if (stop) break;
            cv.wait_for(lk, std::chrono::milliseconds(50));
            continue;
        }
        while (!incoming.empty()) {
            pending.push_back(incoming.front());
            incoming.pop_front();
        }
        // completions
        bool finished = false;
        for (Slot& s : slots) {
            if (!s.busy) continue;
            const cudaError_t q = cudaEventQuery(s.done);
            if (q == cudaErrorNotReady) continue;
            StaStatus status = q == cudaSuccess ? STA_OK : STA_ERR_CUDA;
            if (status == STA_OK) status = sta_synchronize(s.rep->h);  // a bounded wait that expired
            const double t_done = now_s();
            for (size_t b = 0; b < s.reqs.size(); ++b) {
                const Req& rq = s.reqs[b];
                StaServerCompletion c{};
                c.id = rq.id;
                c.netlist = rq.r.netlist;
                c.t_submit = rq.t_arrival;
                c.t_start = s.t_start;
                c.t_done = t_done;
                c.status = status;
                c.merged = (int32_t)s.reqs.size();
                if (rq.r.summary)
                    std::memcpy(rq.r.summary, s.sum_host + b * STA_SUM_COUNT, STA_SUM_COUNT * sizeof(double));
                done.push_back(c);
            }
            s.rep->busy = false;
            s.rep->last_use = t_done;
            s.rep = nullptr;
            s.busy = false;
            finished = true;
        }
        // admissions, residency first: pass 0 starts, in arrival order, the
        // pending requests whose netlist has an idle resident copy; pass 1 the
        // rest in arrival order, making copies -- evicting least recently used
        // idle netlists that have no pending request (any idle one once the
        // oldest request has waited kStarveS), so an admitted netlist serves its
        // queue before it can go.  A request waits while its netlist is busy or
        // cannot be admitted; later ones go ahead, except in the sequential
        // loop, which keeps strict arrival order on one slot (one pass).  With
        // merging, the later pending requests of the same netlist, gamma and
        // kind join it, up to `merge` of them, in arrival order.
        npend.assign(nets.size(), 0);
        for (const Req& r : pending) ++npend[r.r.netlist];
        evict_pending = !pending.empty() && now_s() - pending.front().t_arrival > kStarveS;
        for (int pass = opt.sequential ? 1 : 0; pass < 2; ++pass)
        for (size_t i = 0; i < pending.size();) {
            int free_slot = -1;
            for (int k = 0; k < (int)slots.size(); ++k)
                if (!slots[k].busy) {
                    free_slot = k;
                    break;
                }
            if (free_slot < 0) break;
            Req& rq = pending[i];
            Net* n = nets[rq.r.netlist];
            if (pass == 0 && std::none_of(n->reps.begin(), n->reps.end(), [](const Rep* r) { return !r->busy; })) {
                ++i;
                continue;
            }
            std::string err;
            Rep* rep = admit(this, rq.r.netlist, err);
            if (!rep) {
                if (!err.empty()) {  // can never run
                    StaServerCompletion c{};
                    c.id = rq.id;
                    c.netlist = rq.r.netlist;
                    c.t_submit = rq.t_arrival;
                    c.t_start = c.t_done = now_s();
                    c.status = STA_ERR_OOM;
                    c.merged = 1;
                    done.push_back(c);
                    finished = true;
                    pending.erase(pending.begin() + (long)i);
                    continue;
                }
                if (opt.sequential) break;
                ++i;
                continue;
            }
            Slot& sl = slots[free_slot];
            sl.reqs.clear();
            sl.reqs.push_back(rq);
            pending.erase(pending.begin() + (long)i);
            if (opt.merge > 0) {
                for (size_t j = i; j < pending.size() && (int)sl.reqs.size() < opt.merge;) {
                    const StaServerRequest& a = sl.reqs[0].r;
                    const StaServerRequest& b = pending[j].r;
                    if (b.netlist == a.netlist && b.gradient == a.gradient && b.gamma == a.gamma) {
                        sl.reqs.push_back(pending[j]);
                        pending.erase(pending.begin() + (long)j);
                    } else {
                        ++j;
                    }
                }
            }
            sl.t_start = now_s();
            sl.rep = rep;
            rep->busy = true;
            sl.busy = true;
            const StaStatus s = opt.merge > 0 ? dispatch_merged(this, sl, n) : dispatch(this, sl, n);
            if (s != STA_OK) {  // report at once, after what was queued has run
                cudaStreamSynchronize(sl.st);
                const double t_done = now_s();
                for (const Req& r : sl.reqs) {
                    StaServerCompletion c{};
                    c.id = r.id;
                    c.netlist = r.r.netlist;
                    c.t_submit = r.t_arrival;
                    c.t_start = sl.t_start;
                    c.t_done = t_done;
                    c.status = s;
                    c.merged = (int32_t)sl.reqs.size();
                    done.push_back(c);
                }
                finished = true;
                rep->busy = false;
                sl.rep = nullptr;
                sl.busy = false;
            }
        }
        if (finished) cv.notify_all();
        any_busy = false;
        for (const Slot& s : slots) any_busy = any_busy || s.busy;
        if (any_busy || !pending.empty()) {  // poll the slots' events again shortly
            lk.unlock();
            std::this_thread::yield();
            lk.lock();
        }
    }
}

extern "C" {

double sta_server_clock(void) { return now_s(); }

StaStatus sta_server_create(const StaServerOptions* opt, StaServer** out) {
    if (!out) return fail("sta_server_create: null argument");
    *out = nullptr;
    StaServerOptions o{};
    if (opt) o = *opt;
    if (o.slots < 0 || o.slots > 64 || o.budget_bytes < 0 || o.merge < 0 || o.merge > 64 || (o.merge && o.sequential) ||
        o.replicas < 0 || o.replicas > 64 || (o.replicas > 1 && (o.sequential || o.merge)))
        return fail("sta_server_create: slots in [0, 64], budget >= 0, merge and replicas in [0, 64], "
                    "neither with sequential, not both");
    if (o.slots == 0) o.slots = 4;
    if (o.sequential) o.slots = 1;
    if (o.budget_bytes == 0) o.budget_bytes = 150ll << 30;
    StaServer* S = nullptr;
    try {
        S = new StaServer();
    } catch (const std::bad_alloc&) {
        return fail("host allocation failed", STA_ERR_OOM);
    }
    S->opt = o;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return fail("cudaGetDevice failed", STA_ERR_CUDA);
    }
    {
        cudaMemPoolProps pp{};
        pp.allocType = cudaMemAllocationTypePinned;
        pp.location.type = cudaMemLocationTypeDevice;
        pp.location.id = S->device;
        uint64_t keep = (uint64_t)o.budget_bytes;  // freed memory stays in the pool up to the budget
        if (cudaMemPoolCreate(&S->pool, &pp) != cudaSuccess ||
            cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
            delete S;
            return fail("cudaMemPoolCreate failed", STA_ERR_CUDA);
        }
    }
    S->slots.resize(o.slots);
    for (Slot& s : S->slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.sum_host, (size_t)std::max(o.merge, 1) * STA_SUM_COUNT * sizeof(double)) != cudaSuccess) {
            delete S;
            return fail("stream / event / pinned allocation failed", STA_ERR_CUDA);
        }
    }
    try {
        S->worker = std::thread([S] { S->run(); });
    } catch (...) {
        delete S;
        return fail("could not start the worker thread", STA_ERR_STATE);
    }
    *out = S;
    return STA_OK;
}

StaStatus sta_server_add_netlist(StaServer* S, const StaNetlistDesc* nl, const StaLibrary* lib, int32_t preload,
                                 int32_t* id) {
    if (!S || !nl || !lib || !id) return fail("sta_server_add_netlist: null argument");
    Net* n = nullptr;
    try {
        n = new Net();
        StaStatus st = copy_netlist(*nl, *lib, n->host);
        if (st != STA_OK) {
            delete n;
            return st;
        }
        // the host layout, once (outside the server's lock: the worker runs on)
        std::string err;
        st = sta::build_layout_shared(n->host.nl, n->host.lib, n->layout, err);
        if (st != STA_OK) {
            delete n;
            return fail("sta_server_add_netlist: " + err, st);
        }
        // page-lock the arrays every copy uploads (best effort: a refusal leaves
        // an array pageable, and its uploads slower)
        for (const auto& buf : layout_host_buffers(*n->layout))
            if (buf.second >= (64u << 10) &&
                cudaHostRegister(const_cast<void*>(buf.first), buf.second, cudaHostRegisterDefault) == cudaSuccess)
                n->pinned.push_back(buf.first);
        cudaGetLastError();  // (clear a refusal)
    } catch (const std::bad_alloc&) {
        delete n;
        return fail("host allocation failed", STA_ERR_OOM);
    }
    n->P = nl->num_pins;
    std::lock_guard<std::mutex> lk(S->mu);  // the worker touches nets only while holding the lock
    S->nets.push_back(n);
    *id = (int32_t)S->nets.size() - 1;
    if (preload) {
        // the first copy, or an error; then the further copies (replicas) while
        // the budget allows, so that none is built while requests wait
        S->evict_pending = true;  // (the worker sets it again for its next round)
        std::string err;
        if (!admit(S, *id, err)) {
            if (err.empty()) err = "over the memory budget";
            return fail("sta_server_add_netlist: preload: " + err, STA_ERR_OOM);
        }
        while ((int)n->reps.size() < max_copies(S) && create_rep(S, n, err)) {
        }
    }
    return STA_OK;
}

StaStatus sta_server_submit(StaServer* S, const StaServerRequest* r, int64_t* id) {
    if (!S || !r) return fail("sta_server_submit: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (r->netlist < 0 || r->netlist >= (int32_t)S->nets.size()) return fail("sta_server_submit: unknown netlist");
    if (!r->xy && S->nets[r->netlist]->P > 0) return fail("sta_server_submit: null positions");
    if (!(r->gamma > 0.f)) return fail("sta_server_submit: gamma must be > 0");
    Req q;
    q.r = *r;
    q.id = S->next_id++;
    q.t_arrival = now_s();
    S->incoming.push_back(q);
    if (id) *id = q.id;
    S->cv.notify_all();
    return STA_OK;
}

StaStatus sta_server_poll(StaServer* S, StaServerCompletion* out, int32_t max, int32_t* n, int32_t wait_ms) {
    if (!S || !n || (max > 0 && !out)) return fail("sta_server_poll: null argument");
    std::unique_lock<std::mutex> lk(S->mu);
    if (S->done.empty() && wait_ms > 0)
        S->cv.wait_for(lk, std::chrono::milliseconds(wait_ms), [S] { return !S->done.empty(); });
    const int32_t k = (int32_t)std::min<size_t>(S->done.size(), (size_t)std::max(max, 0));
    for (int32_t i = 0; i < k; ++i) out[i] = S->done[i];
    S->done.erase(S->done.begin(), S->done.begin() + k);
    *n = k;
    return STA_OK;
}

StaStatus sta_server_netlist_bytes(StaServer* S, int32_t id, int64_t* bytes) {
    if (!S || !bytes) return fail("sta_server_netlist_bytes: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    if (id < 0 || id >= (int32_t)S->nets.size()) return fail("sta_server_netlist_bytes: unknown netlist");
    const Net* n = S->nets[id];
    *bytes = (int64_t)(n->rep_bytes ? n->rep_bytes : estimate_bytes(n->host, S->opt.merge));
    return STA_OK;
}

StaStatus sta_server_stats(StaServer* S, int64_t* out4) {
    if (!S || !out4) return fail("sta_server_stats: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t res = 0;
    for (Net* n : S->nets) res += n->reps.empty() ? 0 : 1;
    out4[0] = res;
    out4[1] = (int64_t)S->resident_bytes;
    out4[2] = S->admissions;
    out4[3] = S->evictions;
    return STA_OK;
}

void sta_server_destroy(StaServer* S) { delete S; }

}  // extern "C"
