// dataflow.cu -- persistent, dependency-driven schedule of the level sweeps.
//
// The level-synchronous scheme of the paper launches one kernel per level
// (Section 3.1.2), so a sweep costs (levels) x (launch + the longest chain of
// dependent loads of the level).  Here each sweep is ONE kernel: the builder
// lists the warp-sized tasks of the sweep in a topological order (the levels
// in order, or reversed), every warp takes the next task from a queue
// (atomicAdd on a head) and waits only for the data it reads: the words its
// producers write (arrival / slew / LSE arrival of its fanin pins in the
// forward; required times and adjoints of its sinks, or a large net's partial
// records, in the backward).  Those words are reset to a NaN marker before the
// sweep and written once with strong relaxed stores, so the waiting warp polls
// them directly (strong relaxed loads, the whole warp together) and needs no
// counter, release fence or acquire.  Work of different levels overlaps; no
// grid-wide barrier exists.  A waiting warp only ever waits for tasks with
// smaller indices, which warps that are already running hold, so the sweep
// always progresses; every wait is nevertheless bounded in time and reports
// expiry through an abort word instead of spinning forever.
//
// Tasks are one warp each: packed small nets (as in the level schedule), and,
// for nets of more than 32 pins, 32-sink chunks.  In the forward pass a chunk
// re-evaluates the net's driver cell (cheap) with the load computed by a
// prologue kernel; in the backward pass a large net becomes partial-reduction
// chunks, one driver task that combines them in a fixed order, and gradient
// chunks (which wait on a counter the driver task releases), so every
// reduction stays deterministic.
#include <mutex>

#include "dataflow_sync.cuh"
#include "device_common.cuh"

namespace sta {
namespace {

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

// What a driver-cell lane (net n, condition c) can load before its inputs
// exist: cell type, arcs, input pins and transitions, the load's table segment.
struct FwdPre {
    int t;    // cell type, -1 if the driver is asserted
    int a0, na;
    int pin[STA_MAX_ARCS];
    int rfi;  // bit k: input transition of arc k
    int dyn;  // bit k: arc k's input pin is written during the sweep (not asserted)
    int jl;   // load segment and fraction
    float ul, inv_l;
    float sidx[6], sinv[6];  // slew index points 0..5 of the type and 1/width of each segment
};

// slew segment and fraction from registers (same result as axis_seg)
__device__ __forceinline__ void slew_seg(const float* sidx, const float* sinv, float v, int& is, float& ts) {
    float base = sidx[0], inv = sinv[0];
    is = 0;
#pragma unroll
    for (int j = 1; j <= 5; ++j)
        if (sidx[j] <= v) {
            base = sidx[j];
            inv = sinv[j];
            is = j;
        }
    ts = (v - base) * inv;
}

__device__ __forceinline__ FwdPre fwd_pre(const DevNet& g, const DfState& d, int n, int c, float ld) {
    FwdPre f;
    f.t = g.net_drv[n];
    f.a0 = f.na = f.rfi = f.jl = f.dyn = 0;
    f.ul = f.inv_l = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) f.pin[k] = 0;
#pragma unroll
    for (int j = 0; j < 6; ++j) f.sidx[j] = f.sinv[j] = 0.f;
    if (f.t < 0) return f;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        f.sidx[j] = __ldg(g.lib_idx + f.t * kLibStride + j);
        f.sinv[j] = __ldg(g.lib_inv + f.t * kLibStride + j);
    }
    f.a0 = g.net_arc_ptr[n];
    f.na = g.net_arc_ptr[n + 1] - f.a0;
    const int un = g.lib_unate[f.t], rf = c & 1;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
        if (k < f.na) {
            f.pin[k] = g.arc_pin[f.a0 + k];
            f.rfi |= (rf ^ ((un >> k) & 1)) << k;
            f.dyn |= (d.arc_prod[f.a0 + k] >= 0 ? 1 : 0) << k;
        }
    const float* li = g.lib_idx + f.t * kLibStride + 8;
    f.jl = axis_seg(li, ld);
    f.inv_l = __ldg(g.lib_inv + f.t * kLibStride + 8 + f.jl);
    f.ul = (ld - __ldg(li + f.jl)) * f.inv_l;
    return f;
}

// Shared memory of the forward sweep: per warp, per arc k and slew row i of the
// NLDM tables, (delay, slew) of each lane's cell already interpolated along the
// load axis at the lane's known load -- [k][i][lane] as float2.
constexpr int kColPerWarp = STA_MAX_ARCS * STA_LUT * 32;
constexpr size_t kFwdSmem = sizeof(float2) * kColPerWarp * kWarpsPerBlock;

__device__ __forceinline__ float2* df_cols() {
    extern __shared__ float2 df_smem[];
    return df_smem + (threadIdx.x >> 5) * kColPerWarp;
}

// Before the wait: the lane's slew columns.  Row i of arc k holds
//   D_i = fma(ul, T_delay(i, j+1) - T_delay(i, j), T_delay(i, j)), S_i likewise,
// the same first interpolation step (along load, segment j) that a bilinear
// lookup takes, so the lookup after the wait (along slew, from two rows) gives
// bit-identical results with a shared-memory access instead of a dependent
// global one.
__device__ __forceinline__ void fwd_cols(const DevNet& g, const FwdPre& f, int rf, float2* col, int lane) {
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < f.na) {
            const float4* q = g.lib_col + ((((size_t)f.t * STA_MAX_ARCS + k) * 2 + rf) * 6 + f.jl) * STA_LUT;
#pragma unroll
            for (int i = 0; i < STA_LUT; ++i) {
                const float4 v = __ldg(q + i);
                col[(k * STA_LUT + i) * 32 + lane] =
                    make_float2(fmaf(f.ul, v.y - v.x, v.x), fmaf(f.ul, v.w - v.z, v.z));
            }
        }
    }
}

// After the wait: NLDM lookups from the shared-memory columns, late max / early
// min and the LSE of Eq. 4.  The code is branch-free across lanes (unused arcs
// read a harmless row of the lane's own columns; results are selected), so a
// warp never splits.  The arc delays go to D for the caller to store.

// The wait of a forward task: the fanin arrival / slew / LSE arrival words this
// lane reads, polled (strong relaxed loads, all lanes together) until every one
// that is written during the sweep holds its value; a word is written once per
// sweep and reset to kUnwritten before it, so no counter or release fence is
// needed.  Returns the values.  Bounded like wait_ready: after kWaitBudgetNs or
// once any wait of the launch has expired it sets the abort word and returns.
// `stall` makes the wait never succeed (test hook for the bounded wait).
template <bool lse>
__device__ __forceinline__ void fwd_fanin(const DevState& s, const FwdPre& f, int dp, int c, float* ain, float* sin,
                                          float* zin, bool stall, int32_t* abort_word) {
    const int el = c >> 1;
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        bool ok = !stall;
#pragma unroll
        for (int k = 0; k < STA_MAX_ARCS; ++k) {
            // every lane issues the same loads (unused arcs read the driver's own
            // words, a valid address; their values are not used): no branch, so
            // the warp stays converged.  Loading only the cell's own arcs, as
            // predicated loads, was measured slower.
            const int pin = k < f.na ? f.pin[k] : dp;
            const int r = (f.rfi >> k) & 1;
            const int q = 4 * pin + 2 * el + r;
            sin[k] = ld_relaxed_f(s.slew + q);
            ain[k] = ld_relaxed_f(s.at + q);
            zin[k] = lse ? ld_relaxed_f(s.ats + 2 * pin + r) : 0.f;
            const bool need = k < f.na && ((f.dyn >> k) & 1);
            ok = ok && (!need || (written(sin[k]) && written(ain[k]) && (!lse || !el || written(zin[k]))));
        }
        if (__all_sync(kFull, ok)) return;
        __nanosleep(STA_POLL_NS);
        if ((it & 63) == 63) {
            if (__any_sync(kFull, ld_relaxed(abort_word) != 0)) return;
            const unsigned long long now = __shfl_sync(kFull, global_ns(), 0);
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitBudgetNs) {
                if ((threadIdx.x & 31) == 0) {
                    atomicExch(abort_word, 1);
                    atomicExch(abort_word + 1, 1);
                }
                __syncwarp();
                return;
            }
        }
    }
}

__device__ __forceinline__ void st_relaxed_f4(float* p, float4 v) {
    asm volatile("st.relaxed.gpu.global.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
                 "f"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_relaxed_f2(float* p, float2 v) {
    asm volatile("st.relaxed.gpu.global.v2.f32 [%0], {%1, %2};" ::"l"(p), "f"(v.x), "f"(v.y) : "memory");
}

// a sink's arrival / slew / LSE arrival, the words its consumers poll
__device__ __forceinline__ void store_sink_polled(const DevState& s, int p, const float* A, const float* S, float z0,
                                                  float z1, float2 wdi, bool lse) {
    const float i2 = wdi.y * wdi.y;
    st_relaxed_f4(s.at + 4 * p, make_float4(A[0] + wdi.x, A[1] + wdi.x, A[2] + wdi.x, A[3] + wdi.x));
    st_relaxed_f4(s.slew + 4 * p, make_float4(sqrtf(fmaf(S[0], S[0], i2)), sqrtf(fmaf(S[1], S[1], i2)),
                                              sqrtf(fmaf(S[2], S[2], i2)), sqrtf(fmaf(S[3], S[3], i2))));
    if (lse) st_relaxed_f2(s.ats + 2 * p, make_float2(z0 + wdi.x, z1 + wdi.x));
}

__device__ __forceinline__ DrvOut fwd_eval(const DevState& s, const FwdPre& f, int dp, int c, float gamma, bool lse,
                                           const float* ain, const float* sin, const float* zin, const float2* col,
                                           int lane, float* D, bool asserted) {
    const int el = c >> 1, rf = c & 1;
    float best_at = el ? -kInf : kInf, best_sl = el ? -kInf : kInf, m = -kInf;
    float cand[STA_MAX_ARCS];
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        const bool use = k < f.na;
        int is;
        float ts;
        slew_seg(f.sidx, f.sinv, sin[k], is, ts);
        const float2 lo = col[(k * STA_LUT + is) * 32 + lane], hi = col[(k * STA_LUT + is + 1) * 32 + lane];
        D[k] = fmaf(ts, hi.x - lo.x, lo.x);
        const float S = fmaf(ts, hi.y - lo.y, lo.y);
        const float v = ain[k] + D[k];
        const float ba = el ? fmaxf(best_at, v) : fminf(best_at, v);
        const float bs = el ? fmaxf(best_sl, S) : fminf(best_sl, S);
        best_at = use ? ba : best_at;
        best_sl = use ? bs : best_sl;
        cand[k] = use ? zin[k] + D[k] : -kInf;
        m = fmaxf(m, cand[k]);
    }
    const float lse_v = lse_arcs(cand, f.na, f.na > 0 ? m : 0.f, gamma);
    DrvOut o;
    o.at = best_at;
    o.slew = best_sl;
    o.ats = (el && lse) ? lse_v : 0.f;
    if (asserted) {  // an asserted driver (level-0 tasks only): its constants, set at creation
        o.at = __ldcg(s.at + 4 * dp + c);
        o.slew = __ldcg(s.slew + 4 * dp + c);
        o.ats = (el && lse) ? __ldcg(s.ats + 2 * dp + rf) : 0.f;
    }
    return o;
}

// After a late lane's critical stores: the terms the backward sweep needs for
// this (net, output transition), which depend on forward results only -- per
// arc the LSE weight w_k = exp((LSE-AT_in + delay - LSE-AT_out) / gamma) (Eq. 4's
// softmax), the bilinear partials of the delay along slew and load, and, for
// the arc attaining the late output slew (first one on ties), the slew
// partials.  Same operations as a lookup from the raw tables, so the backward
// reads bit-identical values in one record instead of recomputing them from
// scattered loads before its wait.
__device__ __forceinline__ void fwd_brec(const DevNet& g, const DfState& d, const FwdPre& f, int n, int rf,
                                         const float* sin, const float* zin, const float* D, float ats_out,
                                         float gamma) {
    float w[STA_MAX_ARCS], dds[STA_MAX_ARCS], ddl[STA_MAX_ARCS];
    float best = -kInf, dss = 0.f, dsl = 0.f;
    int amax = -1;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        w[k] = dds[k] = ddl[k] = 0.f;
        if (k < f.na) {
            int is;
            float ts;
            slew_seg(f.sidx, f.sinv, sin[k], is, ts);
            const float inv_s = f.sinv[is];
            const float4* q = g.lib_col + ((((size_t)f.t * STA_MAX_ARCS + k) * 2 + rf) * 6 + f.jl) * STA_LUT + is;
            const float4 r0 = __ldg(q), r1 = __ldg(q + 1);  // rows is, is+1: delay (j, j+1), slew (j, j+1)
            float dSs, dSl;
            lerp_cell_grad(make_float4(r0.x, r0.y, r1.x, r1.y), ts, f.ul, inv_s, f.inv_l, dds[k], ddl[k]);
            const float S = lerp_cell_grad(make_float4(r0.z, r0.w, r1.z, r1.w), ts, f.ul, inv_s, f.inv_l, dSs, dSl);
            w[k] = expf((zin[k] + D[k] - ats_out) / gamma);
            if (S > best) {
                best = S;
                amax = k;
                dss = dSs;
                dsl = dSl;
            }
        }
    }
    float4* r = d.brec + ((size_t)n * 2 + rf) * 4;
    r[0] = make_float4(w[0], w[1], w[2], w[3]);
    r[1] = make_float4(dds[0], dds[1], dds[2], dds[3]);
    r[2] = make_float4(ddl[0], ddl[1], ddl[2], ddl[3]);
    r[3] = make_float4(dss, dsl, __int_as_float(amax), 0.f);
}

// Packed small nets: net RC (Eqs. 1-3) of the task's own pins and every
// static load first; then the wait; then the driver cells (4 lanes per net)
// and the wire step to every sink.
template <bool lse>
__device__ void fwd_df_warp(const DevNet& g, const DevState& s, const DfState& d, int t, int n0, int nn,
                            float gamma, int stall_task) {
    const WarpGeom w = warp_geom(g, n0, nn);
    const int p = w.pin0 + w.lane;
    const bool sink = w.valid && w.lane != w.hd;
    const float2 xy = w.valid ? s.xy[p] : make_float2(0.f, 0.f);
    const float cap = w.valid ? g.pin_cap[p] : 0.f;
    const float2 xyd = make_float2(__shfl_sync(kFull, xy.x, w.hd), __shfl_sync(kFull, xy.y, w.hd));
    float v = cap;
    float2 wdi = make_float2(0.f, 0.f);
    if (sink) {
        const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
        const float R = g.r * dist;
        const float C = fmaf(0.5f * g.c, dist, cap);
        const float D = R * C * kKrc;
        const float m = 2.f * R * C * D * kKrc - D * D;
        wdi = make_float2(D, sqrtf(fmaxf(m, 0.f)));
        s.wdi[p] = wdi;
        v = fmaf(g.c, dist, cap);
    }
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float u = __shfl_up_sync(kFull, v, off);
        v = (w.lane - off >= w.hd) ? v + u : v;
    }
    if (w.valid && w.lane == w.last) s.load[n0 + w.j] = v;

    const int j1 = w.lane >> 2, c = w.lane & 3;
    const int hj = __shfl_sync(kFull, w.h, j1);
    const int lastj = __shfl_sync(kFull, w.h, j1 + 1) - 1;
    const float ldj = __shfl_sync(kFull, v, lastj & 31);
    FwdPre f = fwd_pre(g, d, n0 + min(j1, nn - 1), c, ldj);
    if (j1 >= nn) {  // idle lanes evaluate a dummy: no arcs, results unused
        f.t = -1;
        f.na = 0;
    }
    const int dp = w.pin0 + (j1 < nn ? hj : 0);
    float2* col = df_cols();
    fwd_cols(g, f, c & 1, col, w.lane);

    float ain[STA_MAX_ARCS], sin[STA_MAX_ARCS], zin[STA_MAX_ARCS];
    fwd_fanin<lse>(s, f, dp, c, ain, sin, zin, t == stall_task, d.abort_word);

    float D[STA_MAX_ARCS];
    const DrvOut o = fwd_eval(s, f, dp, c, gamma, lse, ain, sin, zin, col, w.lane, D, j1 < nn && f.t < 0);
    const int src = 4 * max(w.j, 0);
    float A[4], S[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = __shfl_sync(kFull, o.at, src + k);
        S[k] = __shfl_sync(kFull, o.slew, src + k);
    }
    const float z0 = __shfl_sync(kFull, o.ats, src + 2), z1 = __shfl_sync(kFull, o.ats, src + 3);
    // the sinks' words first: consumers poll them; the driver's words and the arc
    // delays are read only after the sweep
    if (sink) store_sink_polled(s, p, A, S, z0, z1, wdi, lse);
    if (j1 < nn && f.t >= 0) {
        s.at[4 * dp + c] = o.at;
        s.slew[4 * dp + c] = o.slew;
        if (lse && c >= 2) s.ats[2 * dp + c - 2] = o.ats;
#pragma unroll
        for (int k = 0; k < STA_MAX_ARCS; ++k)
            if (k < f.na) s.adel[4 * (f.a0 + k) + c] = D[k];
        if (lse && c >= 2) fwd_brec(g, d, f, n0 + j1, c & 1, sin, zin, D, o.ats, gamma);
    }
}

// A 32-sink chunk of a large net: the net's load and wire RC come from the
// prologue kernel; lanes 0-3 evaluate the driver (the first chunk also stores it).
template <bool lse>
__device__ void fwd_df_chunk(const DevNet& g, const DevState& s, const DfState& d, int t, int n, int p0, int cnt,
                             float gamma, int stall_task) {
    const int lane = threadIdx.x & 31;
    const int dp = g.net_ptr[n];
    const bool first = p0 == dp + 1;
    FwdPre f = fwd_pre(g, d, n, lane & 3, s.load[n]);
    if (lane >= 4) {  // lanes 4-31 evaluate a dummy: no arcs, results unused
        f.t = -1;
        f.na = 0;
    }
    float2 wdi = make_float2(0.f, 0.f);
    if (lane < cnt) wdi = s.wdi[p0 + lane];
    float2* col = df_cols();
    fwd_cols(g, f, lane & 1, col, lane);

    float ain[STA_MAX_ARCS], sin[STA_MAX_ARCS], zin[STA_MAX_ARCS];
    fwd_fanin<lse>(s, f, dp, lane & 3, ain, sin, zin, t == stall_task, d.abort_word);

    float D[STA_MAX_ARCS];
    const DrvOut o = fwd_eval(s, f, dp, lane & 3, gamma, lse, ain, sin, zin, col, lane, D, lane < 4 && f.t < 0);
    float A[4], S[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = __shfl_sync(kFull, o.at, k);
        S[k] = __shfl_sync(kFull, o.slew, k);
    }
    const float z0 = __shfl_sync(kFull, o.ats, 2), z1 = __shfl_sync(kFull, o.ats, 3);
    if (lane < cnt) store_sink_polled(s, p0 + lane, A, S, z0, z1, wdi, lse);
    if (lane < 4 && first && f.t >= 0) {  // the first chunk stores the driver and its arc delays
        s.at[4 * dp + lane] = o.at;
        s.slew[4 * dp + lane] = o.slew;
        if (lse && lane >= 2) s.ats[2 * dp + lane - 2] = o.ats;
#pragma unroll
        for (int k = 0; k < STA_MAX_ARCS; ++k)
            if (k < f.na) s.adel[4 * (f.a0 + k) + lane] = D[k];
        if (lse && lane >= 2) fwd_brec(g, d, f, n, lane & 1, sin, zin, D, o.ats, gamma);
    }
}

// With several lanes (independent placements) queue index q is task q / nl of
// lane q % nl: a task only waits for tasks of its own lane with smaller task
// indices, which have smaller queue indices, so the sweep still progresses.
// (kLanes: the lane variant; the single-placement one carries no lane arithmetic)
template <bool lse, bool kLanes>
__global__ void __launch_bounds__(kBlock) k_fwd_df(DevNet g, DevState s, DfState d, float gamma, int stall_task) {
    const int nl = kLanes ? *s.active : 1;  // the lanes this call runs
    int q = grab(d.heads + 0);
    while (q < d.TF * nl) {
        const int t = kLanes ? q / nl : q, l = kLanes ? q - t * nl : 0;
        const DevState sl = kLanes ? lane_state(s, l) : s;
        const DfState dl = kLanes ? lane_df(d, l, s.lane_bytes) : d;
        const int4 task = d.ftask[t];
        const int stall = l == 0 ? stall_task : -1;
        if (task.y > 0) fwd_df_warp<lse>(g, sl, dl, t, task.x, task.y, gamma, stall);
        else fwd_df_chunk<lse>(g, sl, dl, t, task.x, task.z, task.w, gamma, stall);
        // the next task only once this one is done: a task reserved while this one
        // waits could not start when its own data arrives (head-of-line blocking)
        q = grab(d.heads + 0);
    }
}

// Before a backward sweep: the required-time (mode 1) and adjoint (mode 2)
// words of every cell-input pin, which the sweep writes once, are set to kUnwritten.
__global__ void __launch_bounds__(kBlock) k_bwd_reset(DevState s0, const int32_t* __restrict__ pin_cons, int P,
                                                      int mode, float* part0, int npart_words) {
    if (s0.active && (int)blockIdx.y >= *s0.active) return;  // a lane this call does not run
    const DevState s = lane_state(s0, blockIdx.y);            // one lane per grid row
    float* part = lane_ptr(part0, (size_t)blockIdx.y * s0.lane_bytes);
    const float u = __uint_as_float(kUnwritten);
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < npart_words; i += gridDim.x * kBlock) part[i] = u;
    for (int p = blockIdx.x * kBlock + threadIdx.x; p < P; p += gridDim.x * kBlock) {
        if (pin_cons[p] < 0) continue;
        if (mode & 1) reinterpret_cast<float4*>(s.rat)[p] = make_float4(u, u, u, u);
        if (mode & 2) {
            reinterpret_cast<float2*>(s.g_ats)[p] = make_float2(u, u);
            reinterpret_cast<float2*>(s.g_slew)[p] = make_float2(u, u);
        }
    }
}

// Before a forward sweep, in one launch: the RC of the large nets (one chunk of
// sinks per block, see rc_chunk), and, on every block, a grid-stride share of
// the reset of the words that forward tasks poll -- the arrival / slew /
// LSE-arrival words of the cell-input pins the sweep writes -- to kUnwritten
// (asserted pins keep their constants; sinks that feed no cell are only written).
__global__ void __launch_bounds__(kBlock) k_fwd_prologue(DevNet g, DevState s0, const uchar4* __restrict__ mask,
                                                         int P) {
    if (s0.active && (int)blockIdx.y >= *s0.active) return;  // a lane this call does not run
    const DevState s = lane_state(s0, blockIdx.y);            // one lane per grid row
    if ((int)blockIdx.x < g.nrc) rc_chunk(g, s, g.rc_chunk[blockIdx.x], g.rc_net[blockIdx.x]);
    const float u = __uint_as_float(kUnwritten);
    const float4 u4 = make_float4(u, u, u, u);
    // four grid strides per step: the four mask bytes are loaded together, and
    // consecutive threads store consecutive pins
    const int stride = gridDim.x * kBlock;
    const uint8_t* mk = reinterpret_cast<const uint8_t*>(mask);
    for (int p0 = blockIdx.x * kBlock + threadIdx.x; p0 < P; p0 += 4 * stride) {
        unsigned m[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) m[j] = p0 + j * stride < P ? mk[p0 + j * stride] : 0u;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (m[j] & 1) {
                const int p = p0 + j * stride;
                reinterpret_cast<float4*>(s.at)[p] = u4;
                reinterpret_cast<float4*>(s.slew)[p] = u4;
                reinterpret_cast<float2*>(s.ats)[p] = make_float2(u, u);
            }
    }
}

// ---------------------------------------------------------------------------
// Backward (mode 1 required times, mode 2 adjoint, 3 both)
// ---------------------------------------------------------------------------
struct SeedCtx {
    float W, wt, ww;  // WNS_gamma, w_tns, w_wns
};

// What a sink lane can load before the wait.  Cell-input sinks get their
// required time and adjoints from the task that does their cell's arc step
// (read after the wait); other sinks are constant: an endpoint carries its
// constraint and, in the adjoint, the seed d loss / d LSE-AT =
// -(w_tns dTNS_g/ds + w_wns dWNS_g/ds); a dangling sink has +-inf required
// times and zero adjoints.
struct SinkPre {
    int cons;
    float2 wdi, sl;  // wire (delay, impulse), late slews (rise, fall)
    float4 rat;      // constant required times
    float2 ga;       // constant adjoint of the LSE arrival
};

__device__ __forceinline__ SinkPre sink_pre(const DevState& s, const DfState& d, int p, int mode, float gamma,
                                            const SeedCtx& sc) {
    SinkPre q;
    q.cons = d.pin_cons[p];
    q.wdi = s.wdi[p];
    q.sl = (mode & 2) ? reinterpret_cast<const float2*>(s.slew)[2 * p + 1] : make_float2(0.f, 0.f);
    q.rat = make_float4(0.f, 0.f, 0.f, 0.f);
    q.ga = make_float2(0.f, 0.f);
    if (q.cons < 0) {
        q.rat = reinterpret_cast<const float4*>(s.rat)[p];
        if ((mode & 2) && isfinite(q.rat.z)) {
            SeedCtx c = sc;
            if (d.pin_grp) {  // several netlists: the endpoint's own WNS_gamma and weights
                const int gi = d.pin_grp[p];
                c.W = (float)s.summary[(size_t)gi * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
                c.wt = s.params[2 * gi];
                c.ww = s.params[2 * gi + 1];
            }
            const float2 z = reinterpret_cast<const float2*>(s.ats)[p];
            const float sr = q.rat.z - z.x, sf = q.rat.w - z.y;
            const float te = softmin3(sr, sf, gamma);
            float gr = c.wt * expf(-(sr - te) / gamma), gf = c.wt * expf(-(sf - te) / gamma);
            if (isfinite(c.W)) {
                gr += c.ww * expf(-(sr - c.W) / gamma);
                gf += c.ww * expf(-(sf - c.W) / gamma);
            }
            q.ga = make_float2(-gr, -gf);
        }
    }
    return q;
}

// The words a cell-input sink's backward terms read: its required times and
// adjoints, written by the task of the cell it feeds.
struct SinkWords {
    float4 rat;
    float2 ga, gs;
};

__device__ __forceinline__ float4 ld_relaxed_f4(const float* p) {
    float4 v;
    asm volatile("ld.relaxed.gpu.global.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}

__device__ __forceinline__ float2 ld_relaxed_f2(const float* p) {
    float2 v;
    asm volatile("ld.relaxed.gpu.global.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "l"(p) : "memory");
    return v;
}

// The wait of a backward task over its sinks: every lane whose sink is a cell
// input (`need`) polls that sink's words (strong relaxed loads, the warp
// together) until all of them hold this sweep's values; the words are reset to
// kUnwritten before the sweep and written once.  Bounded like wait_ready.
template <int mode>
__device__ __forceinline__ SinkWords sink_wait(const DevState& s, int p, bool need, int32_t* abort_word) {
    SinkWords w;
    w.rat = make_float4(0.f, 0.f, 0.f, 0.f);
    w.ga = w.gs = make_float2(0.f, 0.f);
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        bool ok = true;
        if (mode & 1) {
            w.rat = ld_relaxed_f4(s.rat + 4 * p);
            ok = ok && written(w.rat.x) && written(w.rat.y) && written(w.rat.z) && written(w.rat.w);
        }
        if (mode & 2) {
            w.ga = ld_relaxed_f2(s.g_ats + 2 * p);
            w.gs = ld_relaxed_f2(s.g_slew + 2 * p);
            ok = ok && written(w.ga.x) && written(w.ga.y) && written(w.gs.x) && written(w.gs.y);
        }
        if (__all_sync(kFull, ok || !need)) return w;
        __nanosleep(STA_POLL_NS);
        if ((it & 63) == 63) {
            if (__any_sync(kFull, ld_relaxed(abort_word) != 0)) return w;
            const unsigned long long now = __shfl_sync(kFull, global_ns(), 0);
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitBudgetNs) {
                if ((threadIdx.x & 31) == 0) {
                    atomicExch(abort_word, 1);
                    atomicExch(abort_word + 1, 1);
                }
                __syncwarp();
                return w;
            }
        }
    }
}

// After the wait: the sink's terms of the backward reductions (see sink_bwd),
// from the polled words of a cell-input sink or the constants of another sink.
__device__ __forceinline__ SinkBwd sink_post(const SinkWords& wd, const SinkPre& q, float2 sld, int mode) {
    const bool dyn = q.cons >= 0;
    float4 rat = q.rat;
    float2 ga = q.ga, gs = make_float2(0.f, 0.f);
    if (mode & 1) rat = dyn ? wd.rat : q.rat;
    if (mode & 2) {
        ga = dyn ? wd.ga : q.ga;
        gs = dyn ? wd.gs : make_float2(0.f, 0.f);
    }
    SinkBwd b;
    if (mode & 1) {
        b.r[0] = rat.x - q.wdi.x;
        b.r[1] = rat.y - q.wdi.x;
        b.r[2] = rat.z - q.wdi.x;
        b.r[3] = rat.w - q.wdi.x;
    } else {
        b.r[0] = b.r[1] = -kInf;
        b.r[2] = b.r[3] = kInf;
    }
    b.ga[0] = b.ga[1] = b.gs[0] = b.gs[1] = b.gwire = 0.f;
    if (mode & 2) {
        const float q0 = q.sl.x > 0.f ? gs.x / q.sl.x : 0.f;
        const float q1 = q.sl.y > 0.f ? gs.y / q.sl.y : 0.f;
        b.ga[0] = ga.x;
        b.ga[1] = ga.y;
        b.gs[0] = q0 * sld.x;
        b.gs[1] = q1 * sld.y;
        b.gwire = ga.x + ga.y + (q0 + q1) * q.wdi.y;
    }
    return b;
}

// identity terms of a lane that carries no sink
__device__ __forceinline__ SinkBwd sink_none() {
    SinkBwd b;
    b.r[0] = b.r[1] = -kInf;
    b.r[2] = b.r[3] = kInf;
    b.ga[0] = b.ga[1] = b.gs[0] = b.gs[1] = b.gwire = 0.f;
    return b;
}

// select between two term sets without branching
__device__ __forceinline__ SinkBwd sink_pick(bool take, const SinkBwd& a, const SinkBwd& b) {
    SinkBwd r;
#pragma unroll
    for (int k = 0; k < 4; ++k) r.r[k] = take ? a.r[k] : b.r[k];
    r.ga[0] = take ? a.ga[0] : b.ga[0];
    r.ga[1] = take ? a.ga[1] : b.ga[1];
    r.gs[0] = take ? a.gs[0] : b.gs[0];
    r.gs[1] = take ? a.gs[1] : b.gs[1];
    r.gwire = take ? a.gwire : b.gwire;
    return r;
}

// What a driver-cell lane (net n, condition c) of the backward sweep can
// compute from forward results before the wait: its arc delays (required
// times) and, for the late conditions, the LSE weights of the arcs, the
// bilinear partials of delay and slew, and the arc that attains the late
// slew (first one on ties).
struct BwdPre {
    int t, a0, na, rfi;
    int pin[STA_MAX_ARCS];
    float adel[STA_MAX_ARCS];
    float w[STA_MAX_ARCS], dDs[STA_MAX_ARCS], dDl[STA_MAX_ARCS];
    int amax;
    float dSs, dSl;
    float cs;  // propagated clock: the setup seed of a one-input cell's clock pin (rising lane)
};

// a lane with no driver cell (asserted driver or idle lane)
__device__ __forceinline__ BwdPre bwd_none() {
    BwdPre b;
    b.t = -1;
    b.a0 = b.na = b.rfi = 0;
    b.amax = -1;
    b.dSs = b.dSl = b.cs = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        b.pin[k] = 0;
        b.adel[k] = b.w[k] = b.dDs[k] = b.dDl[k] = 0.f;
    }
    return b;
}

__device__ __forceinline__ BwdPre bwd_pre(const DevNet& g, const DevState& s, const DfState& d, int n, int c,
                                          int mode) {
    BwdPre b;
    b.t = g.net_drv[n];
    b.a0 = b.na = b.rfi = 0;
    b.amax = -1;
    b.dSs = b.dSl = b.cs = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        b.pin[k] = 0;
        b.adel[k] = b.w[k] = b.dDs[k] = b.dDl[k] = 0.f;
    }
    if (b.t < 0) return b;
    const int el = c >> 1, rf = c & 1;
    b.a0 = g.net_arc_ptr[n];
    b.na = g.net_arc_ptr[n + 1] - b.a0;
    const int un = g.lib_unate[b.t];
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
        if (k < b.na) {
            b.pin[k] = g.arc_pin[b.a0 + k];
            b.rfi |= (rf ^ ((un >> k) & 1)) << k;
            if (mode & 1) b.adel[k] = s.adel[4 * (b.a0 + k) + c];
        }
    // a capturing clock pin is the input of a one-input cell; its seed is read
    // here, before the wait, and added to the rising adjoint it writes
    if ((mode & 2) && el == 1 && s.cap_seed && b.na == 1 && (b.rfi & 1) == 0) b.cs = __ldcg(s.cap_seed + b.pin[0]);
    if ((mode & 2) && el == 1) {  // the terms the forward sweep stored for (net, rf)
        const float4* r = d.brec + ((size_t)n * 2 + rf) * 4;
        const float4 w = r[0], dds = r[1], ddl = r[2], x = r[3];
        b.w[0] = w.x, b.w[1] = w.y, b.w[2] = w.z, b.w[3] = w.w;
        b.dDs[0] = dds.x, b.dDs[1] = dds.y, b.dDs[2] = dds.z, b.dDs[3] = dds.w;
        b.dDl[0] = ddl.x, b.dDl[1] = ddl.y, b.dDl[2] = ddl.z, b.dDl[3] = ddl.w;
        b.dSs = x.x;
        b.dSl = x.y;
        b.amax = __float_as_int(x.z);
    }
    return b;
}

// After the wait: required times of the cell's inputs (R = the output's
// required time for this condition) and, for the late conditions, the adjoint
// through the LSE, the NLDM partials and the late-slew max; returns this
// transition's d loss / d load.
__device__ __forceinline__ float bwd_apply(const DevState& s, const BwdPre& b, int c, float R, float GA, float GS,
                                           int mode) {
    const int el = c >> 1;
    const bool adj = (mode & 2) && el == 1;
    float gl = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        const bool use = k < b.na;  // na = 0 for asserted drivers and idle lanes
        const int r = (b.rfi >> k) & 1;
        const int qr = 4 * b.pin[k] + 2 * el + r, qa = 2 * b.pin[k] + r;
        const float rv = R - b.adel[k];
        const float gD = GA * b.w[k];
        const float gsv = fmaf(gD, b.dDs[k], k == b.amax ? GS * b.dSs : 0.f);
        if ((mode & 1) && use) st_relaxed_f(s.rat + qr, rv);  // words the sink's own task polls
        // a capturing clock pin also carries its endpoint's setup term
        if (adj && use) st_relaxed_f(s.g_ats + qa, (s.cap_seed && k == 0) ? gD + b.cs : gD);
        if (adj && use) st_relaxed_f(s.g_slew + qa, gsv);
        gl = (adj && use) ? fmaf(gD, b.dDl[k], gl) : gl;
    }
    return (adj && b.amax >= 0) ? fmaf(GS, b.dSl, gl) : gl;
}

template <int mode>
__device__ void bwd_df_warp(const DevNet& g, const DevState& s, const DfState& d, int32_t* cnt, int t, int n0,
                            int nn, float gamma, const SeedCtx& sc) {
    const WarpGeom w = warp_geom(g, n0, nn);
    const int p = w.pin0 + w.lane;
    const bool sink = w.valid && w.lane != w.hd;
    // static part
    float2 sld = make_float2(0.f, 0.f);
    if (mode & 2) {
        const float2 sl = w.valid ? reinterpret_cast<const float2*>(s.slew)[2 * p + 1] : make_float2(0.f, 0.f);
        sld = make_float2(__shfl_sync(kFull, sl.x, w.hd), __shfl_sync(kFull, sl.y, w.hd));
    }
    const int pl = w.valid ? p : w.pin0;  // a valid pin for every lane
    SinkPre q = sink_pre(s, d, pl, mode, gamma, sc);
    const int j1 = w.lane >> 2, c = w.lane & 3;
    const int hj = __shfl_sync(kFull, w.h, j1);
    const int lastj = (__shfl_sync(kFull, w.h, j1 + 1) - 1) & 31;
    const BwdPre bp = j1 < nn ? bwd_pre(g, s, d, n0 + j1, c, mode) : bwd_none();
    float2 xy = make_float2(0.f, 0.f), xyd = make_float2(0.f, 0.f);
    float cap = 0.f;
    int orig = 0;
    if (mode & 2) {
        xy = s.xy[pl];
        xyd = make_float2(__shfl_sync(kFull, xy.x, w.hd), __shfl_sync(kFull, xy.y, w.hd));
        cap = g.pin_cap[pl];
        orig = g.pin_orig[pl];
    }

    const SinkWords wd = sink_wait<mode>(s, pl, sink && q.cons >= 0, d.abort_word);
    const SinkBwd b = sink_pick(sink, sink_post(wd, q, sld, mode), sink_none());
    float r0 = b.r[0], r1 = b.r[1], r2 = b.r[2], r3 = b.r[3];
    float ga0 = b.ga[0], ga1 = b.ga[1], gs0 = b.gs[0], gs1 = b.gs[1];
    // segmented inclusive scans; updates are selects, not branches, so the
    // warp stays converged between the shuffles
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const bool take = w.lane - off >= w.hd;
        if (mode & 1) {
            const float u0 = __shfl_up_sync(kFull, r0, off), u1 = __shfl_up_sync(kFull, r1, off);
            const float u2 = __shfl_up_sync(kFull, r2, off), u3 = __shfl_up_sync(kFull, r3, off);
            r0 = take ? fmaxf(r0, u0) : r0;
            r1 = take ? fmaxf(r1, u1) : r1;
            r2 = take ? fminf(r2, u2) : r2;
            r3 = take ? fminf(r3, u3) : r3;
        }
        if (mode & 2) {
            const float u0 = __shfl_up_sync(kFull, ga0, off), u1 = __shfl_up_sync(kFull, ga1, off);
            const float u2 = __shfl_up_sync(kFull, gs0, off), u3 = __shfl_up_sync(kFull, gs1, off);
            ga0 = take ? ga0 + u0 : ga0;
            ga1 = take ? ga1 + u1 : ga1;
            gs0 = take ? gs0 + u2 : gs0;
            gs1 = take ? gs1 + u3 : gs1;
        }
    }
    if ((mode & 1) && w.valid && w.lane == w.last)
        reinterpret_cast<float4*>(s.rat)[w.pin0 + w.hd] = make_float4(r0, r1, r2, r3);
    const float R0 = __shfl_sync(kFull, r0, lastj), R1 = __shfl_sync(kFull, r1, lastj);
    const float R2 = __shfl_sync(kFull, r2, lastj), R3 = __shfl_sync(kFull, r3, lastj);
    const float GA0 = __shfl_sync(kFull, ga0, lastj), GA1 = __shfl_sync(kFull, ga1, lastj);
    const float GS0 = __shfl_sync(kFull, gs0, lastj), GS1 = __shfl_sync(kFull, gs1, lastj);
    const float Rc = c == 0 ? R0 : c == 1 ? R1 : c == 2 ? R2 : R3;
    float gl = bwd_apply(s, bp, c, Rc, (c & 1) ? GA1 : GA0, (c & 1) ? GS1 : GS0, mode);
    if (mode & 2) {
        gl += __shfl_down_sync(kFull, gl, 1);
        const float gload = __shfl_sync(kFull, gl, (4 * max(w.j, 0) + 2) & 31);
        const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
        const float gd = fmaf(gload, g.c, b.gwire * kKrc * g.r * fmaf(g.c, fabsf(dx) + fabsf(dy), cap));
        const float2 gxy = sink ? make_float2(gd * ((dx > 0.f) - (dx < 0.f)), gd * ((dy > 0.f) - (dy < 0.f)))
                                : make_float2(0.f, 0.f);
        if (sink) s.grad[orig] = gxy;
        float sx = gxy.x, sy = gxy.y;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float u = __shfl_up_sync(kFull, sx, off), v = __shfl_up_sync(kFull, sy, off);
            const bool take = w.lane - off >= w.hd;
            sx = take ? sx + u : sx;
            sy = take ? sy + v : sy;
        }
        const int orig_d = __shfl_sync(kFull, orig, w.hd);
        if (w.valid && w.lane == w.last) s.grad[orig_d] = make_float2(-sx, -sy);
    }
}

// fixed-order butterfly reductions across a warp
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(kFull, v, off);
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, off));
    return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fminf(v, __shfl_xor_sync(kFull, v, off));
    return v;
}

// Partial chunk of a large net: 12 partial terms over up to 32 sinks,
//   0-3 max/max/min/min of RAT_s - Delay_s, 4-5 sums of g_ats, 6-7 sums of
//   g_slew * slew_d / slew_s, 8-9 sums of sign(x_s - x_d), sign(y_s - y_d),
//   10-11 sums of sign * g_wire * dDelay/dd (the driver's gradient is
//   -(gload * c * sums 8-9 + sums 10-11)).
template <int mode>
__device__ void bwd_df_part(const DevNet& g, const DevState& s, const DfState& d, int32_t* cnt_arr, int t, int n,
                            int p0, int cnt, float gamma, const SeedCtx& sc, float* part) {
    const int lane = threadIdx.x & 31;
    const int dp = g.net_ptr[n];
    const float2 sld = (mode & 2) ? reinterpret_cast<const float2*>(s.slew)[2 * dp + 1] : make_float2(0.f, 0.f);
    const int p = p0 + (lane < cnt ? lane : 0);  // a valid pin for every lane
    const SinkPre q = sink_pre(s, d, p, mode, gamma, sc);
    float sx = 0.f, sy = 0.f, fd = 0.f;
    if (lane < cnt) {
        if (mode & 2) {
            const float2 xy = s.xy[p], xyd = s.xy[dp];
            const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
            sx = (dx > 0.f) - (dx < 0.f);
            sy = (dy > 0.f) - (dy < 0.f);
            fd = kKrc * g.r * fmaf(g.c, fabsf(dx) + fabsf(dy), g.pin_cap[p]);
        }
    }

    const SinkWords wd = sink_wait<mode>(s, p, lane < cnt && q.cons >= 0, d.abort_word);
    const SinkBwd b = sink_pick(lane < cnt, sink_post(wd, q, sld, mode), sink_none());
    float v[kPartFloats];
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = b.r[k];
    v[4] = b.ga[0];
    v[5] = b.ga[1];
    v[6] = b.gs[0];
    v[7] = b.gs[1];
    const float h = b.gwire * fd;
    v[8] = sx;
    v[9] = sy;
    v[10] = sx * h;
    v[11] = sy * h;
    v[0] = warp_max(v[0]);
    v[1] = warp_max(v[1]);
    v[2] = warp_min(v[2]);
    v[3] = warp_min(v[3]);
#pragma unroll
    for (int k = 4; k < kPartFloats; ++k) v[k] = warp_sum(v[k]);
    if (lane < kPartFloats) {
        float out = v[0];
#pragma unroll
        for (int k = 1; k < kPartFloats; ++k)
            if (lane == k) out = v[k];
        st_relaxed_f(part + lane, out);  // the driver step polls these words
    }
}

// Driver step of a large net: combine its partial chunks in a fixed order, then
// required times / adjoint through the driver cell and the driver's gradient.
template <int mode>
__device__ void bwd_df_driver(const DevNet& g, const DevState& s, const DfState& d, int32_t* cnt, int t, int n,
                              const float* part, int slot0, int nch, float gamma) {
    const int lane = threadIdx.x & 31;
    const int dp = g.net_ptr[n];
    const BwdPre bp = lane < 4 ? bwd_pre(g, s, d, n, lane, mode) : bwd_none();

    // the wait: poll the chunks' partial words (reset to kUnwritten before the
    // sweep, written once by the partial tasks) until all are written; bounded
    // like wait_ready
    // the lane's chunks lane, lane + 32, ... combined in that order during each poll;
    // the successful poll's values are final (every word is written once per sweep)
    float v[kPartFloats];
    {
        unsigned long long t0 = 0;
        for (unsigned it = 0;; ++it) {
            bool ok = true;
            v[0] = v[1] = -kInf;
            v[2] = v[3] = kInf;
#pragma unroll
            for (int j = 4; j < kPartFloats; ++j) v[j] = 0.f;
            for (int k = lane; k < nch; k += 32) {
                const float* q = part + (size_t)(slot0 + k) * kPartFloats;
                float x[kPartFloats];
#pragma unroll
                for (int j = 0; j < kPartFloats; ++j) {
                    x[j] = ld_relaxed_f(q + j);
                    ok &= written(x[j]);
                }
                v[0] = fmaxf(v[0], x[0]);
                v[1] = fmaxf(v[1], x[1]);
                v[2] = fminf(v[2], x[2]);
                v[3] = fminf(v[3], x[3]);
#pragma unroll
                for (int j = 4; j < kPartFloats; ++j) v[j] += x[j];
            }
            if (__all_sync(kFull, ok)) break;
            __nanosleep(STA_POLL_NS);
            if ((it & 63) == 63) {
                if (__any_sync(kFull, ld_relaxed(d.abort_word) != 0)) break;
                const unsigned long long now = __shfl_sync(kFull, global_ns(), 0);
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > kWaitBudgetNs) {
                    if (lane == 0) {
                        atomicExch(d.abort_word, 1);
                        atomicExch(d.abort_word + 1, 1);
                    }
                    __syncwarp();
                    break;
                }
            }
        }
    }
    v[0] = warp_max(v[0]);
    v[1] = warp_max(v[1]);
    v[2] = warp_min(v[2]);
    v[3] = warp_min(v[3]);
#pragma unroll
    for (int k = 4; k < kPartFloats; ++k) v[k] = warp_sum(v[k]);
    if ((mode & 1) && lane == 0) reinterpret_cast<float4*>(s.rat)[dp] = make_float4(v[0], v[1], v[2], v[3]);
    const int c = lane & 3;
    const float Rc = c == 0 ? v[0] : c == 1 ? v[1] : c == 2 ? v[2] : v[3];
    float gl = bwd_apply(s, bp, c, Rc, (c & 1) ? v[5] : v[4], (c & 1) ? v[7] : v[6], mode);
    if (mode & 2) {
        gl += __shfl_down_sync(kFull, gl, 1);
        const float gload = __shfl_sync(kFull, gl, 2);
        if (lane == 0) {
            d.net_gload[n] = gload;
            s.grad[g.pin_orig[dp]] = make_float2(-fmaf(gload * g.c, v[8], v[10]), -fmaf(gload * g.c, v[9], v[11]));
        }
    }
}

// Gradient chunk of a large net: d loss / d (x, y) of up to 32 sinks, once the
// driver task has published d loss / d load.  No task waits for these.
__device__ void bwd_df_grad(const DevNet& g, const DevState& s, const DfState& d, int32_t* cnt_arr, int t, int n,
                            int p0, int cnt, float gamma, const SeedCtx& sc) {
    const int lane = threadIdx.x & 31;
    const int dp = g.net_ptr[n];
    wait_ready(cnt_arr, t, d.b_indeg[t], d.abort_word);
    const float gload = __ldcg(d.net_gload + n);
    if (lane < cnt) {
        const int p = p0 + lane;
        const float2 sld = reinterpret_cast<const float2*>(s.slew)[2 * dp + 1];
        const SinkPre q = sink_pre(s, d, p, 2, gamma, sc);
        SinkWords wd;
        wd.rat = make_float4(0.f, 0.f, 0.f, 0.f);
        wd.ga = ld_relaxed_f2(s.g_ats + 2 * p);  // final: the driver task saw every partial after its sinks'
        wd.gs = ld_relaxed_f2(s.g_slew + 2 * p);
        const SinkBwd b = sink_post(wd, q, sld, 2);
        s.grad[g.pin_orig[p]] = sink_grad(g, s, p, s.xy[p], s.xy[dp], b.gwire, gload);
    }
}

template <int mode, bool kLanes>
// 3 blocks per SM (80 registers, no spills): more warps hold backward tasks
// ahead of the front, so a task's pre-wait loads are done when its data arrives
__global__ void __launch_bounds__(kBlock, 3) k_bwd_df(DevNet g, DevState s, DfState d, float gamma) {
    int32_t* head = d.heads + ((mode & 2) ? 2 : 1);
    const int nl = kLanes ? *s.active : 1;  // the lanes this call runs
    int q = grab(head);
    while (q < d.TB * nl) {  // queue index q: task q / nl of lane q % nl (see k_fwd_df)
        const int t = kLanes ? q / nl : q, l = kLanes ? q - t * nl : 0;
        const DevState sl = kLanes ? lane_state(s, l) : s;
        const DfState dl = kLanes ? lane_df(d, l, s.lane_bytes) : d;
        int32_t* cnt = (mode & 2) ? dl.acnt : dl.rcnt;
        float* part = (mode & 2) ? dl.apart : dl.rpart;
        SeedCtx sc;
        sc.W = (float)sl.summary[STA_SUM_WNS_GAMMA];
        sc.wt = sl.params[0];
        sc.ww = sl.params[1];
        const int4 task = d.btask[t];
        if (task.y > 0) {
            bwd_df_warp<mode>(g, sl, dl, cnt, t, task.x, task.y, gamma, sc);
        } else if (task.y == -1) {
            bwd_df_part<mode>(g, sl, dl, cnt, t, task.x, task.z, task.w, gamma, sc,
                              part + (size_t)d.baux[t] * kPartFloats);
        } else if (task.y == -2) {
            bwd_df_driver<mode>(g, sl, dl, cnt, t, task.x, part, task.z, task.w, gamma);
        } else if (mode & 2) {
            bwd_df_grad(g, sl, dl, cnt, t, task.x, task.z, task.w, gamma, sc);
        }
        // every task's consumers poll the words it wrote, except the gradient
        // chunks of a large net, which wait on a counter that its driver step releases
        if (task.y == -2) signal_consumers(cnt, d.b_out_ptr, d.b_out, t);
        q = grab(head);
    }
}

}  // namespace

// Co-resident blocks of a sweep: the smallest count over every variant the
// sweep may launch (they share one grid size).  Also grants the forward kernels
// their dynamic shared memory (above the default 48 KB), once per device.
// (the result depends on the device and the kernels only: it is computed once
// per device and variant, since a server creates handles at request rate)
static int dataflow_max_blocks_query(int fwd, int lanes);

int dataflow_max_blocks(int fwd, int lanes) {
    constexpr int kDevs = 64;
    static std::mutex mu;
    static int cache[kDevs][2][2] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const int f = fwd ? 1 : 0, l = lanes ? 1 : 0;
    if (dev < 0 || dev >= kDevs) return dataflow_max_blocks_query(fwd, lanes);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (cache[dev][f][l] > 0) return cache[dev][f][l];
    }
    const int v = dataflow_max_blocks_query(fwd, lanes);
    if (cudaPeekAtLastError() == cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu);
        cache[dev][f][l] = v;
    }
    return v;
}

static int dataflow_max_blocks_query(int fwd, int lanes) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int per_sm = 1 << 20;
    auto take = [&](auto kernel, size_t smem) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, kBlock, smem);
        per_sm = n < per_sm ? n : per_sm;
    };
    if (fwd && lanes) {
        cudaFuncSetAttribute(k_fwd_df<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        cudaFuncSetAttribute(k_fwd_df<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        take(k_fwd_df<true, true>, kFwdSmem);
        take(k_fwd_df<false, true>, kFwdSmem);
    } else if (fwd) {
        cudaFuncSetAttribute(k_fwd_df<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        cudaFuncSetAttribute(k_fwd_df<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem);
        take(k_fwd_df<true, false>, kFwdSmem);
        take(k_fwd_df<false, false>, kFwdSmem);
        // one placement: 2 blocks per SM hold enough tasks ahead of the front
        // (about 3 levels) and poll a third less than 3 (measured 1-2% faster;
        // 1 block per SM is 55% slower); several lanes keep the occupancy limit
        per_sm = per_sm < 2 ? per_sm : 2;
    } else if (lanes) {
        take(k_bwd_df<1, true>, 0);
        take(k_bwd_df<2, true>, 0);
        take(k_bwd_df<3, true>, 0);
    } else {
        take(k_bwd_df<1, false>, 0);
        take(k_bwd_df<2, false>, 0);
        take(k_bwd_df<3, false>, 0);
    }
    return sms * (per_sm > 0 ? per_sm : 1);
}

void launch_fwd_dataflow(const DevNet& g, const DevState& s, const DfState& d, int grid, float gamma, int lse,
                         int stall_task, cudaStream_t st) {
    if (d.TF == 0) return;
    if (s.nl > 1) {
        if (lse) launch_coop(k_fwd_df<true, true>, grid, kBlock, kFwdSmem, st, g, s, d, gamma, stall_task);
        else launch_coop(k_fwd_df<false, true>, grid, kBlock, kFwdSmem, st, g, s, d, gamma, stall_task);
    } else {
        if (lse) launch_coop(k_fwd_df<true, false>, grid, kBlock, kFwdSmem, st, g, s, d, gamma, stall_task);
        else launch_coop(k_fwd_df<false, false>, grid, kBlock, kFwdSmem, st, g, s, d, gamma, stall_task);
    }
}

void launch_bwd_reset(const DevState& s, const DfState& d, int P, int mode, cudaStream_t st) {
    if (P == 0 && d.npart == 0) return;
    int blocks = (P + kBlock - 1) / kBlock;
    if (blocks > 152 * 8) blocks = 152 * 8;
    k_bwd_reset<<<dim3(blocks, s.nl), kBlock, 0, st>>>(s, d.pin_cons, P, mode, (mode & 2) ? d.apart : d.rpart,
                                                       d.npart * kPartFloats);
}

void launch_fwd_prologue(const DevNet& g, const DevState& s, const DfState& d, int P, cudaStream_t st) {
    int blocks = (P + kBlock - 1) / kBlock;
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < g.nrc) blocks = g.nrc;
    if (blocks == 0) return;
    k_fwd_prologue<<<dim3(blocks, s.nl), kBlock, 0, st>>>(g, s, d.pin_mask, P);
}

void launch_bwd_dataflow(const DevNet& g, const DevState& s, const DfState& d, int grid, float gamma, int mode,
                         cudaStream_t st) {
    if (d.TB == 0) return;
    if (s.nl > 1) {
        if (mode == 1) launch_coop(k_bwd_df<1, true>, grid, kBlock, 0, st, g, s, d, gamma);
        else if (mode == 2) launch_coop(k_bwd_df<2, true>, grid, kBlock, 0, st, g, s, d, gamma);
        else launch_coop(k_bwd_df<3, true>, grid, kBlock, 0, st, g, s, d, gamma);
    } else {
        if (mode == 1) launch_coop(k_bwd_df<1, false>, grid, kBlock, 0, st, g, s, d, gamma);
        else if (mode == 2) launch_coop(k_bwd_df<2, false>, grid, kBlock, 0, st, g, s, d, gamma);
        else launch_coop(k_bwd_df<3, false>, grid, kBlock, 0, st, g, s, d, gamma);
    }
}

}  // namespace sta
