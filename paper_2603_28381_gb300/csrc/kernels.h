// kernels.h -- device views of a handle's buffers and the kernel launchers.
#pragma once

#include <cuda_runtime.h>

#include "sta_internal.h"

namespace sta {

// Read-only topology, library and constraints (internal order).
struct DevNet {
    const int32_t* net_ptr;      // [N+1]
    const int32_t* net_drv;      // [N]
    const int32_t* net_arc_ptr;  // [N+1]
    const int32_t* arc_pin;      // [A]
    const int32_t* pin_orig;     // [P]
    const float* pin_cap;        // [P]
    const int32_t* wtask;        // [2W]
    const int32_t* ctask;        // [Cb]
    const int4* rc_chunk;        // [K] RC chunks of the nets > 32 pins (Layout::rc_chunk)
    const int2* rc_net;          // [K]
    const float* lib_idx;        // [T*16]
    const float* lib_inv;        // [T*16]
    const int32_t* lib_unate;    // [T]
    const float* lib_tab;        // [T*4*2*98]
    const float4* lib_cell;      // [T*4*2*36*2] corner-packed cells (delay float4, slew float4)
    const float4* lib_col;       // [T*4*2*6*7] slew rows of each load segment (Layout::lib_col)
    const int4* net_desc;        // [N*2] per-net driver-cell record (see Layout::net_desc)
    const int32_t* ep_pin;       // [E]
    const float* ep_rat;         // [E*4]
    const int32_t* ep_clk;       // [E] capturing clock pin (propagated clock), -1 none; null: ideal clock
    float r, c;                  // Ohm/um, fF/um
    int32_t P, Pnet, N, E;
    int32_t nrc;                 // RC chunks
    // several netlists in one handle (sta_create_multi; G = 1 and nulls otherwise):
    // per netlist its endpoint range, summary, loss weights and reduction counter
    const int32_t* grp_ep;       // [G+1] endpoint range of each netlist
    const int32_t* pin_grp;      // [P] netlist of each pin
    int32_t G;                   // netlists
    int32_t ep_gx;               // endpoint-reduction blocks per netlist
};

// Mutable per-call state (internal order unless stated).
struct DevState {
    float2* xy;        // [P] positions
    float* load;       // [N] net load (Eq. 1 at the driver)
    float2* wdi;       // [P] (wire delay, impulse) at sink pins (Eqs. 2-3)
    float* at;         // [P*4]
    float* slew;       // [P*4]
    float* ats;        // [P*2] late rise/fall LSE arrival time (Eq. 4)
    float* adel;       // [A*4] cell-arc delays
    float* rat;        // [P*4]
    float* g_ats;      // [P*2] adjoint of ats
    float* g_slew;     // [P*2] adjoint of the late slews
    float2* grad;      // [P] d loss / d (x, y), ORIGINAL pin order
    float2* ep_slack;  // [E] (early, late)
    double* red;       // [G][ep_gx] endpoint-reduction partials (scratch, 48 bytes each)
    double* summary;   // [G][STA_SUM_COUNT]
    float* params;     // [G][2] w_tns, w_wns (padded to 4 floats)
    float* cap_seed;   // [P] d loss / d (rising arrival) of capturing clock pins, 0 elsewhere;
                       // null without a propagated clock
    float* rc_part;    // [rc_slots] partial loads of the nets split into several RC chunks
    int32_t* rc_count; // [rc_slots] chunks done (0 between launches: the last chunk resets it)
    int32_t* ep_count; // [G] endpoint blocks done (0 between launches)
    // Independent placements ("lanes") of one handle: every array above of lane
    // l sits l * lane_bytes after lane 0's (one slab per lane, same layout).
    size_t lane_bytes;
    int32_t nl;        // lanes (1: a single placement)
    int32_t* active;   // lanes handles: device word, the lanes [0, *active) a call runs (set by the
                       // position gather); null for a single placement.  Not per lane.
};

template <typename T>
__host__ __device__ inline T* lane_ptr(T* p, size_t off) {
    return p ? reinterpret_cast<T*>(reinterpret_cast<uintptr_t>(p) + off) : p;
}

// The per-placement state of lane l.
__host__ __device__ inline DevState lane_state(const DevState& s, int l) {
    const size_t off = (size_t)l * s.lane_bytes;
    DevState r = s;
    r.xy = lane_ptr(s.xy, off);
    r.load = lane_ptr(s.load, off);
    r.wdi = lane_ptr(s.wdi, off);
    r.at = lane_ptr(s.at, off);
    r.slew = lane_ptr(s.slew, off);
    r.ats = lane_ptr(s.ats, off);
    r.adel = lane_ptr(s.adel, off);
    r.rat = lane_ptr(s.rat, off);
    r.g_ats = lane_ptr(s.g_ats, off);
    r.g_slew = lane_ptr(s.g_slew, off);
    r.grad = lane_ptr(s.grad, off);
    r.ep_slack = lane_ptr(s.ep_slack, off);
    r.red = lane_ptr(s.red, off);
    r.summary = lane_ptr(s.summary, off);
    r.params = lane_ptr(s.params, off);
    r.cap_seed = lane_ptr(s.cap_seed, off);
    r.rc_part = lane_ptr(s.rc_part, off);
    r.rc_count = lane_ptr(s.rc_count, off);
    r.ep_count = lane_ptr(s.ep_count, off);
    return r;
}

// Dataflow schedule: task lists, the counters of the large nets' gradient
// chunks, queue heads.  Tasks wait on the data words they read (reset to
// kUnwritten before each sweep); only a gradient chunk waits on a counter,
// which its net's driver step releases.
struct DfState {
    const int4* ftask;       // [TF]
    const int32_t* arc_prod; // [A]
    const int4* btask;       // [TB]
    const int32_t* baux;     // [TB]
    const int32_t* pin_cons; // [P]
    const int32_t* b_indeg;  // [TB] producers of each backward task (a gradient chunk: its driver step)
    const int32_t* b_out_ptr;// [TB+1]
    const int32_t* b_out;    // consumers each backward task would signal (driver steps do)
    int32_t* rcnt;           // [TB x groups] arrived producers, required-time sweep
    int32_t* acnt;           // [TB x groups] arrived producers, adjoint sweep
    int32_t* heads;          // [4] queue heads: forward, required time, adjoint
    float* rpart;            // [npart * kPartFloats] partials, required-time sweep
    float* apart;            // [npart * kPartFloats] partials, adjoint sweep
    float* net_gload;        // [N] d loss / d load of large nets
    int32_t* abort_word;     // [2] [0] a bounded wait of the current sweep expired, [1] sticky copy
    const uint8_t* pin_keep; // [P] 1: the forward sweep does not write the pin (asserted values)
    const int32_t* pin_grp;  // [P] several netlists: each pin's (DevNet::pin_grp), else null
    const uchar4* pin_mask;  // [P/4 rounded up] Layout::pin_mask (read a byte per pin)
    int32_t TF, TB;
    int32_t npart;           // partial records of the backward sweeps
    float4* brec;            // [N*2*4] per (net, late output transition): the adjoint terms of the
                             // driver cell the forward sweep computed (see fwd_brec)
    // rcnt, acnt, rpart, apart, net_gload and brec are per lane (in the lane's slab,
    // DevState::lane_bytes apart); the task lists, queue heads and abort words are
    // shared: a sweep's queue holds task t of lane l at index t * nl + l
};

// The dataflow bookkeeping of lane l.
__host__ __device__ inline DfState lane_df(const DfState& d, int l, size_t lane_bytes) {
    const size_t off = (size_t)l * lane_bytes;
    DfState r = d;
    r.rcnt = lane_ptr(d.rcnt, off);
    r.acnt = lane_ptr(d.acnt, off);
    r.rpart = lane_ptr(d.rpart, off);
    r.apart = lane_ptr(d.apart, off);
    r.net_gload = lane_ptr(d.net_gload, off);
    r.brec = lane_ptr(d.brec, off);
    return r;
}

// Batched schedule (many placements of one netlist; lane = placement).
// Per-placement state is pin-major, placement-minor: value[(row) * Bp + b].
struct BatchState {
    int32_t B, Bp, G;    // placements, padded to a multiple of 32, groups of 32
    int32_t GT;          // task groups of kPlacePerWarp placements (Bp / 8)
    float2* xy;          // [P][Bp]
    float* load;         // [N][Bp]
    float* at;           // [P*4][Bp]
    float* slew;         // [P*4][Bp]
    float* ats;          // [P*2][Bp]
    float* rat;          // [P*4][Bp]
    float* g_ats;        // [P*2][Bp]
    float* g_slew;       // [P*2][Bp]
    float2* grad;        // [P][Bp], internal pin order
    float2* ep_slack;    // [E][Bp]
    double* summary;     // [Bp][STA_SUM_COUNT]
    double* red;         // [kRedBlocks][Bp] endpoint partials (48 bytes each)
    float* params;       // [Bp][2] w_tns, w_wns of each placement
    float* part;         // [npart * kPartFloats][Bp] partials of large nets, adjoint sweeps
    float* rpart;        // the same for required-time sweeps (which may overlap an adjoint sweep)
    float* net_gload;    // [N][Bp] d loss / d load of large nets
    float* cap_seed;     // [P][Bp] as DevState::cap_seed; null without a propagated clock
};
constexpr size_t kBatchEpBytes = 48;  // one endpoint partial
constexpr int kPlacePerWarp = 8;       // sweep tasks: 8 placements x 4 conditions per warp

int batch_max_blocks(int fwd);
// the batched sweeps with a lane per placement (batch_wide.cu)
int batch_wide_max_blocks();
int batch_wide_fwd_max_blocks();
void launch_batch_fwd_wide(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int lse,
                           int stall_task, cudaStream_t st);
void launch_batch_bwd_wide(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int mode,
                           cudaStream_t st);
// the large nets' sinks in chunks of at most kLoadChunk (k_bload): per chunk an
// int4 {net, first sink, the net's first chunk, sinks | (chunks of the net << 16)}
constexpr int kLoadChunk = 256;
struct BigChunks {
    const int4* rec = nullptr;  // [n]
    int n = 0;
    float* part = nullptr;      // [n][Bp] chunk sums
    int32_t* cnt = nullptr;     // [n][G] finished chunks of a net (at its first chunk), zero between launches
};
std::vector<int32_t> big_chunk_list(const std::vector<int32_t>& big_nets, const std::vector<int32_t>& net_ptr);
void launch_batch_load(const DevNet& g, const BatchState& bs, const BigChunks& c, cudaStream_t st);
void launch_batch_fwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int lse,
                      int stall_task, cudaStream_t st);
void launch_batch_endpoints(const DevNet& g, const BatchState& bs, float gamma, int lse, cudaStream_t st);
// level-synchronous batched sweeps
void launch_batch_load_small(const DevNet& g, const BatchState& bs, int big, cudaStream_t st);
void launch_batch_fwd_level(const DevNet& g, const BatchState& bs, const DfState& d, int t0, int t1, float gamma,
                            int lse, cudaStream_t st);
// r6: up to three backward task ranges [r6[0], r6[1]), [r6[2], r6[3]), [r6[4], r6[5])
void launch_batch_bwd_level(const DevNet& g, const BatchState& bs, const DfState& d, const int* r6, float gamma,
                            int mode, cudaStream_t st);
void launch_batch_bwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int mode,
                      cudaStream_t st);
// marks the words a batched dataflow sweep polls (what: 0 forward, else the backward mode)
void launch_batch_reset(const BatchState& bs, const DfState& d, int P, int what, cudaStream_t st);
void launch_batch_xy_in(const BatchState& bs, const int32_t* pin_int, int P, const float2* xy_user, cudaStream_t st);
void launch_batch_out(const BatchState& bs, const int32_t* pin_int, int P, const float* in, int K, float* out,
                      cudaStream_t st);
void launch_batch_out2(const BatchState& bs, const int32_t* pin_int, int P, const float2* in, float2* out,
                       cudaStream_t st);
void launch_batch_pin_slack(const BatchState& bs, int P, float* scratch, cudaStream_t st);
void launch_batch_ep_out(const BatchState& bs, int E, float2* out, cudaStream_t st);
void launch_batch_broadcast(float* dst, const float* src, long long rows, int Bp, cudaStream_t st);
void launch_batch_init_ats(const BatchState& bs, int P, cudaStream_t st);

// stall_task >= 0: that task's wait never succeeds (test hook for the bounded wait)
void launch_fwd_dataflow(const DevNet& g, const DevState& s, const DfState& d, int grid, float gamma, int lse,
                         int stall_task, cudaStream_t st);
// marks the words a dataflow backward sweep of this mode writes as not yet written
void launch_bwd_reset(const DevState& s, const DfState& d, int P, int mode, cudaStream_t st);
void launch_bwd_dataflow(const DevNet& g, const DevState& s, const DfState& d, int grid, float gamma, int mode,
                         cudaStream_t st);
// largest co-resident grid of the dataflow kernels on the current device (lanes:
// the variants of a handle with several independent placements)
int dataflow_max_blocks(int fwd, int lanes);

// net RC in the CTE scheme of Algorithm 2 (ablation), nets [n0, n1)
void launch_rc_cte(const DevNet& g, const DevState& s, int n0, int n1, cudaStream_t st);

// positions of `lanes` placements ([lanes][P][2], caller's pin order); a lanes
// handle's following calls run those lanes
void launch_gather_xy(const DevNet& g, const DevState& s, const float2* xy_user, int lanes, cudaStream_t st);
// net RC: the first nw warp tasks (packed small nets) and every large-net chunk
void launch_rc(const DevNet& g, const DevState& s, int nw, cudaStream_t st);
// dataflow forward prologue: large-net RC chunks and the reset of the sweep's polled words
void launch_fwd_prologue(const DevNet& g, const DevState& s, const DfState& d, int P, cudaStream_t st);
void launch_fwd_level(const DevNet& g, const DevState& s, int w0, int nw, int c0, int nc, float gamma,
                      int lse, cudaStream_t st);
// endpoint slacks and the summary in one launch; with d non-null it also marks the words
// the next fused (mode 3) dataflow backward sweep polls
void launch_endpoints(const DevNet& g, const DevState& s, float gamma, int lse, cudaStream_t st,
                      const DfState* d = nullptr, int P = 0);
// mode bit 1 = required times, bit 2 = adjoint
void launch_bwd_level(const DevNet& g, const DevState& s, int w0, int nw, int c0, int nc, float gamma,
                      int mode, cudaStream_t st);
void launch_set_weights(const DevState& s, const float* w_dev, float w0, float w1, cudaStream_t st);
void launch_seed(const DevNet& g, const DevState& s, float gamma, cudaStream_t st);
// memory latency probe: read a buffer once; follow next[] from index 0 for `steps` loads
void launch_touch(const int32_t* a, long long n, int32_t* sink, cudaStream_t st);
void launch_chase(const int32_t* next, int steps, int32_t* sink, cudaStream_t st);
// propagated clock: d loss / d (early rising arrival) of each capturing clock pin
void launch_cap_seed(const DevNet& g, const DevState& s, float gamma, cudaStream_t st);
void launch_batch_cap_seed(const DevNet& g, const BatchState& bs, float gamma, cudaStream_t st);
// out[orig(p)*k + q] = in[p*k + q] for the first `np` internal pins
void launch_scatter(const DevNet& g, const float* in, float* out, int k, int np, cudaStream_t st);
void launch_pin_slack(const DevNet& g, const DevState& s, float* out, cudaStream_t st);
void launch_init_ats(const DevState& s, int P, cudaStream_t st);

}  // namespace sta
