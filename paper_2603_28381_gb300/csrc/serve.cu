// serve.cu -- a request loop over resident netlists (continuous batching).
//
// The server keeps netlists resident on the device under a memory budget and
// runs STA / gradient requests on a pool of CUDA streams ("slots").  A worker
// thread admits requests as slots and memory free up: a request whose netlist
// is resident and idle starts on a free slot at once, whatever the requests
// before it wait for, so the work of requests on different netlists overlaps
// on the device.  Requests of one netlist run one after another (they share
// the netlist's device state).  A netlist that is not resident is created
// when the budget allows, evicting the least recently used idle netlists.
// Every request's result is that of the same request run alone: the kernels
// are deterministic and a netlist's state is only touched by its own requests.
//
// With sequential = 1 the server is the plain one-request-per-launch loop:
// one slot, strict arrival order.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
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

struct Net {
    HostNetlist host;
    StaHandle* h = nullptr;
    size_t bytes = 0;        // device bytes while resident (estimate before the first creation)
    bool busy = false;
    double last_use = 0.0;
    int32_t P = 0;
    float* grad_dev = nullptr;  // [P][2] device gradient of the request in flight
    double* sum_dev = nullptr;  // [STA_SUM_COUNT]
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
    Req req{};
    double t_start = 0.0;
    double* sum_host = nullptr;  // pinned [STA_SUM_COUNT]
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
        if (n->h) sta_destroy(n->h);
        if (n->grad_dev) cudaFree(n->grad_dev);
        if (n->sum_dev) cudaFree(n->sum_dev);
        delete n;
    }
}

namespace {

// Upper bound of the device bytes of a netlist's handle plus the server's
// scratch, from the description alone (used until it has been created once):
// per pin the per-pin state, staging and gradient scratch (132 B); per net or
// cell output the per-net arrays and the task lists (120 B); per arc the arc
// delays and dependency edges (32 B); per endpoint 28 B; with a propagated
// clock 4 B more per pin (clock seeds) and per endpoint (its clock pin).
size_t estimate_bytes(const HostNetlist& hn) {
    const StaNetlistDesc& d = hn.nl;
    const size_t A = d.num_cells ? (size_t)hn.cell_in_ptr[d.num_cells] : 0;
    const size_t clk = d.end_clock ? 4 : 0;
    return (size_t)d.num_pins * (132 + clk) + ((size_t)d.num_nets + d.num_cells) * 120 + A * 32 +
           (size_t)d.num_end * (28 + clk) + (1u << 20);
}

}  // namespace

// Make netlist k resident (create its handle) if the budget allows, evicting
// idle netlists in least-recently-used order.  Returns false if it cannot be
// admitted now (the request waits).
static bool admit(StaServer* S, int k, std::string& err) {
    Net* n = S->nets[k];
    if (n->h) return true;
    const size_t need = n->bytes ? n->bytes : estimate_bytes(n->host);
    const size_t budget = (size_t)S->opt.budget_bytes;
    if (need > budget) {
        err = "netlist larger than the memory budget";
        return false;
    }
    while (S->resident_bytes + need > budget) {
        int victim = -1;
        for (int i = 0; i < (int)S->nets.size(); ++i) {
            Net* m = S->nets[i];
            if (m->h && !m->busy && (victim < 0 || m->last_use < S->nets[victim]->last_use)) victim = i;
        }
        if (victim < 0) return false;  // everything resident is busy: wait
        Net* m = S->nets[victim];
        sta_destroy(m->h);
        m->h = nullptr;
        cudaFree(m->grad_dev);
        cudaFree(m->sum_dev);
        m->grad_dev = nullptr;
        m->sum_dev = nullptr;
        S->resident_bytes -= m->bytes;
        ++S->evictions;
    }
    StaOptions o{};
    o.use_graphs = 1;
    o.schedule = STA_SCHED_DATAFLOW;
    // a netlist's persistent sweeps use a grid in proportion to its size, so the
    // sweeps of small netlists leave room for others on the device
    o.grid_blocks = S->opt.sequential ? 0 : std::max(8, n->P / 4000);
    StaStatus st = sta_create(&n->host.nl, &n->host.lib, &o, &n->h);
    if (st != STA_OK) {
        err = std::string("sta_create: ") + sta_last_error();
        n->h = nullptr;
        return false;
    }
    if (cudaMalloc(&n->grad_dev, (size_t)std::max(n->P, 1) * 8) != cudaSuccess ||
        cudaMalloc(&n->sum_dev, STA_SUM_COUNT * sizeof(double)) != cudaSuccess) {
        err = "cudaMalloc of request scratch failed";
        sta_destroy(n->h);
        n->h = nullptr;
        return false;
    }
    int64_t sz[8];
    sta_query_sizes(n->h, sz);
    // measured size (the handle's allocations, its host-input staging, the scratch)
    n->bytes = (size_t)sz[7] + 2 * (size_t)std::max(n->P, 1) * 8 + STA_SUM_COUNT * sizeof(double);
    S->resident_bytes += n->bytes;
    ++S->admissions;
    while (S->resident_bytes > budget) {  // the estimate was low: make room, or give up
        int victim = -1;
        for (int i = 0; i < (int)S->nets.size(); ++i) {
            Net* m = S->nets[i];
            if (m != n && m->h && !m->busy && (victim < 0 || m->last_use < S->nets[victim]->last_use)) victim = i;
        }
        Net* m = victim >= 0 ? S->nets[victim] : n;
        sta_destroy(m->h);
        m->h = nullptr;
        cudaFree(m->grad_dev);
        cudaFree(m->sum_dev);
        m->grad_dev = nullptr;
        m->sum_dev = nullptr;
        S->resident_bytes -= m->bytes;
        ++S->evictions;
        if (m == n) {
            if (n->bytes > budget) err = "netlist larger than the memory budget";
            return false;
        }
    }
    return true;
}

// Queue one request's work on a slot's stream: positions in, forward, gradient
// if asked, results out; an event marks its end.
static StaStatus dispatch(StaServer* S, Slot& sl, Net* n) {
    const StaServerRequest& r = sl.req.r;
    StaHandle* h = n->h;
    void* st = sl.st;
    StaStatus s = sta_set_positions(h, r.xy, 0, st);
    if (s == STA_OK)
        s = sta_forward(h, STA_FWD_LSE | STA_FWD_RAT | (r.gradient ? 0u : STA_FWD_RAT_EAGER), r.gamma, st);
    if (s == STA_OK && r.gradient) {
        const float w[2] = {r.w_tns, r.w_wns};
        s = sta_backward_grad(h, w, 0, n->grad_dev, 1, st);
        if (s == STA_OK && r.grad &&
            cudaMemcpyAsync(r.grad, n->grad_dev, (size_t)n->P * 8, cudaMemcpyDeviceToHost, sl.st) != cudaSuccess)
            s = STA_ERR_CUDA;
    }
    if (s == STA_OK) s = sta_query_summary(h, n->sum_dev, 1, st);
    if (s == STA_OK && cudaMemcpyAsync(sl.sum_host, n->sum_dev, STA_SUM_COUNT * sizeof(double), cudaMemcpyDeviceToHost,
                                       sl.st) != cudaSuccess)
        s = STA_ERR_CUDA;
    if (s == STA_OK && cudaEventRecord(sl.done, sl.st) != cudaSuccess) s = STA_ERR_CUDA;
    (void)S;
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
            Net* n = nets[s.req.r.netlist];
            StaServerCompletion c{};
            c.id = s.req.id;
            c.netlist = s.req.r.netlist;
            c.t_submit = s.req.t_arrival;
            c.t_start = s.t_start;
            c.t_done = now_s();
            c.status = q == cudaSuccess ? STA_OK : STA_ERR_CUDA;
            if (c.status == STA_OK) c.status = sta_synchronize(n->h);  // a bounded wait that expired
            if (s.req.r.summary) std::memcpy(s.req.r.summary, s.sum_host, STA_SUM_COUNT * sizeof(double));
            n->busy = false;
            n->last_use = c.t_done;
            s.busy = false;
            done.push_back(c);
            finished = true;
        }
        // admissions: the earliest pending request first; later ones go ahead
        // while it waits for its netlist (busy, or not yet admitted), except in
        // the sequential loop, which keeps strict arrival order on one slot
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
            std::string err;
            if (n->busy || !admit(this, rq.r.netlist, err)) {
                if (!err.empty()) {  // can never run
                    StaServerCompletion c{};
                    c.id = rq.id;
                    c.netlist = rq.r.netlist;
                    c.t_submit = rq.t_arrival;
                    c.t_start = c.t_done = now_s();
                    c.status = STA_ERR_OOM;
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
            sl.req = rq;
            sl.t_start = now_s();
            n->busy = true;
            sl.busy = true;
            const StaStatus s = dispatch(this, sl, n);
            if (s != STA_OK) {  // report at once, after what was queued has run
                cudaStreamSynchronize(sl.st);
                StaServerCompletion c{};
                c.id = rq.id;
                c.netlist = rq.r.netlist;
                c.t_submit = rq.t_arrival;
                c.t_start = sl.t_start;
                c.t_done = now_s();
                c.status = s;
                done.push_back(c);
                finished = true;
                n->busy = false;
                sl.busy = false;
            }
            pending.erase(pending.begin() + (long)i);
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
    if (o.slots < 0 || o.slots > 64 || o.budget_bytes < 0) return fail("sta_server_create: slots in [0, 64], budget >= 0");
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
    S->slots.resize(o.slots);
    for (Slot& s : S->slots) {
        if (cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost(&s.sum_host, STA_SUM_COUNT * sizeof(double)) != cudaSuccess) {
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
    } catch (const std::bad_alloc&) {
        delete n;
        return fail("host allocation failed", STA_ERR_OOM);
    }
    n->P = nl->num_pins;
    std::lock_guard<std::mutex> lk(S->mu);  // the worker touches nets only while holding the lock
    S->nets.push_back(n);
    *id = (int32_t)S->nets.size() - 1;
    if (preload) {
        std::string err;
        if (!admit(S, *id, err)) {
            if (err.empty()) err = "over the memory budget";
            return fail("sta_server_add_netlist: preload: " + err, STA_ERR_OOM);
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
    *bytes = (int64_t)(n->bytes ? n->bytes : estimate_bytes(n->host));
    return STA_OK;
}

StaStatus sta_server_stats(StaServer* S, int64_t* out4) {
    if (!S || !out4) return fail("sta_server_stats: null argument");
    std::lock_guard<std::mutex> lk(S->mu);
    int64_t res = 0;
    for (Net* n : S->nets) res += n->h ? 1 : 0;
    out4[0] = res;
    out4[1] = (int64_t)S->resident_bytes;
    out4[2] = S->admissions;
    out4[3] = S->evictions;
    return STA_OK;
}

void sta_server_destroy(StaServer* S) { delete S; }

}  // extern "C"
