// batch.cu -- many placements of one netlist in one sweep.
//
// Every placement runs the same timing graph, so the batched schedule maps
// LANES TO (PLACEMENT, CONDITION) PAIRS: a warp takes one task (a net, or a
// chunk of a large net's sinks) for 8 placements x 4 timing conditions and
// each lane runs the per-net algorithm for its placement and condition.  All
// lanes follow the same control flow (the topology is shared), and every
// per-pin access of a warp is four full 32-byte sectors: per-placement state
// is stored pin-major, placement-minor, value[(pin * k + component) * Bp + b]
// with Bp = the batch rounded up to a multiple of 32.  Topology, capacitances
// and tables are read once per warp for 8 placements.
//
// The sweeps are the dependency-driven persistent kernels of the
// single-placement schedule with queue index q = task * GT + group (GT = Bp / 8
// placement groups): task t of group g waits only for its producers in group
// g, whose queue indices are smaller.  Every placement's arithmetic is the
// same whatever the batch size or its position in the batch, so a placement's
// results are bit-identical alone and in a batch.
#include <algorithm>

#include "batch_common.cuh"

namespace sta {
namespace {

// ---------------------------------------------------------------------------
// Lanes: 8 placements x 4 timing conditions per warp (lane = 4 * placement +
// condition), so each lane evaluates one condition of its placement; the 4
// lanes of a placement ("quad") exchange values with xor shuffles 1 and 2.
// Every branch below depends on the task only (warp-uniform), never on data.
// ---------------------------------------------------------------------------
struct Lane {
    int lane, c, el, rf, b;
};

__device__ __forceinline__ Lane lane_of(int gq) {
    Lane L;
    L.lane = threadIdx.x & 31;
    L.c = L.lane & 3;
    L.el = L.c >> 1;
    L.rf = L.c & 1;
    L.b = gq * kPlacePerWarp + (L.lane >> 2);
    return L;
}

// fixed-order sum over the quad: (l0 + l1) + (l2 + l3), the same bits on all 4 lanes
__device__ __forceinline__ float quad_sum(float v) {
    v += __shfl_xor_sync(kFull, v, 1);
    return v + __shfl_xor_sync(kFull, v, 2);
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

// What a lane loads before the wait: the driver cell, its arcs' input pins and
// input transitions for this lane's output transition, the type's slew axis,
// and the load segment of this placement.
struct FCell {
    int t, na, a0, rfi;
    int dyn;  // bit k: arc k's input pin is written during the sweep
    int pin[STA_MAX_ARCS];
    int jl;
    float ul;
    float sidx[6], sinv[6];
};

// the driver cell's record: type, arcs, input pins, input transitions
__device__ __forceinline__ FCell fcell_topo(const DevNet& g, int n, int rf) {
    FCell f;
    const int4 q0 = __ldg(g.net_desc + 2 * n), q1 = __ldg(g.net_desc + 2 * n + 1);  // one record
    f.t = q0.x;
    f.a0 = q0.y;
    f.na = q0.z;
    f.rfi = 0;
    f.dyn = q0.w & 15;
    f.jl = 0;
    f.ul = 0.f;
    f.pin[0] = q1.x;
    f.pin[1] = q1.y;
    f.pin[2] = q1.z;
    f.pin[3] = q1.w;
#pragma unroll
    for (int j = 0; j < 6; ++j) f.sidx[j] = f.sinv[j] = 0.f;
    if (f.t < 0) return f;
    const int un = q0.w >> 4;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
        if (k < f.na) f.rfi |= (rf ^ ((un >> k) & 1)) << k;
    return f;
}

// the type's slew axis and the load's table segment and fraction
__device__ __forceinline__ void fcell_lib(const DevNet& g, FCell& f, float ld) {
    if (f.t < 0) return;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        f.sidx[j] = __ldg(g.lib_idx + f.t * kLibStride + j);
        f.sinv[j] = __ldg(g.lib_inv + f.t * kLibStride + j);
    }
    const float* li = g.lib_idx + f.t * kLibStride + 8;
    f.jl = axis_seg(li, ld);
    f.ul = (ld - __ldg(li + f.jl)) * __ldg(g.lib_inv + f.t * kLibStride + 8 + f.jl);
}

struct FOut {
    float at, sl, z;  // arrival, slew, LSE arrival (late conditions) of this lane's condition
};

// The fanin arrival / slew / LSE-arrival words of the lane's arcs, all
// together (through L2: other warps of this sweep wrote them).  Returns
// whether every word written during the sweep holds its value; the dataflow
// sweep issues this first round as soon as the cell's record is known and
// repeats it in the wait only if a word was missing.
struct FIn {
    float ain[STA_MAX_ARCS], sin[STA_MAX_ARCS], zin[STA_MAX_ARCS];
};

template <bool kPoll>
__device__ __forceinline__ bool fcell_fanin(const BatchState& bs, const FCell& f, const Lane& L, bool lse, bool stall,
                                            FIn& in) {
    const int Bp = bs.Bp, b = L.b, el = L.el;
    bool ok = !stall;  // the test hook's stalled task never sees its inputs
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        in.ain[k] = in.sin[k] = in.zin[k] = 0.f;
        if (f.t >= 0 && k < f.na) {
            const int r = (f.rfi >> k) & 1;
            const int row = 4 * f.pin[k] + 2 * el + r;
            in.ain[k] = kPoll ? ld_poll(bs.at + ix(row, Bp, b)) : __ldcg(bs.at + ix(row, Bp, b));
            in.sin[k] = kPoll ? ld_poll(bs.slew + ix(row, Bp, b)) : __ldcg(bs.slew + ix(row, Bp, b));
            if (lse && el)
                in.zin[k] = kPoll ? ld_poll(bs.ats + ix(2 * f.pin[k] + r, Bp, b))
                                  : __ldcg(bs.ats + ix(2 * f.pin[k] + r, Bp, b));
            if ((f.dyn >> k) & 1)
                ok &= written(in.ain[k]) & written(in.sin[k]) & (!(lse && el) || written(in.zin[k]));
        }
    }
    return ok;
}

// Driver-cell evaluation for one condition (late max / early min over the
// arcs, worst slew, Eq. 4 LSE for the late conditions) from the fanin words
// of fcell_fanin; `ok` is its first round's result, and in the dataflow sweep
// the wait repeats the round until every lane has all its words.
template <bool kPoll>
__device__ __forceinline__ FOut fcell_eval(const DevNet& g, const BatchState& bs, const FCell& f, int dp,
                                           const Lane& L, float gamma, bool lse, int32_t* abort_word, bool stall,
                                           FIn& in, bool ok) {
    const int Bp = bs.Bp, b = L.b, el = L.el, rf = L.rf;
    FOut o;
    if (f.t < 0) {  // asserted driver: constant values set at creation
        o.at = bs.at[ix(4 * dp + L.c, Bp, b)];
        o.sl = bs.slew[ix(4 * dp + L.c, Bp, b)];
        o.z = (el && lse) ? bs.ats[ix(2 * dp + rf, Bp, b)] : 0.f;
        return o;
    }
    if constexpr (kPoll) {
        if (!__all_sync(kFull, ok)) poll_words([&]() { return fcell_fanin<true>(bs, f, L, lse, stall, in); }, abort_word);
    }
    float best_at = el ? -kInf : kInf, best_sl = el ? -kInf : kInf, m = -kInf;
    float cand[STA_MAX_ARCS];
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        cand[k] = -kInf;
        if (k < f.na) {
            int is;
            float ts;
            seg_reg(f.sidx, f.sinv, in.sin[k], is, ts);
            float4 dq, sq;
            cell_corners(g, f.t, k, rf, is, f.jl, dq, sq);
            const float D = lerp_cell(dq, ts, f.ul);
            const float S = lerp_cell(sq, ts, f.ul);
            const float v = in.ain[k] + D;
            best_at = el ? fmaxf(best_at, v) : fminf(best_at, v);
            best_sl = el ? fmaxf(best_sl, S) : fminf(best_sl, S);
            cand[k] = in.zin[k] + D;
            m = fmaxf(m, cand[k]);
        }
    }
    o.at = best_at;
    o.sl = best_sl;
    o.z = 0.f;
    if (lse && el) {
        o.z = lse_arcs(cand, f.na, m, gamma);
    }
    return o;
}

__device__ __forceinline__ void store_pin(const BatchState& bs, int p, const Lane& L, float at, float sl, float z,
                                          bool lse) {
    const int Bp = bs.Bp;  // strong stores: words that other tasks of the sweep poll
    st_poll(bs.at + ix(4 * p + L.c, Bp, L.b), at);
    st_poll(bs.slew + ix(4 * p + L.c, Bp, L.b), sl);
    if (lse && L.el) st_poll(bs.ats + ix(2 * p + L.rf, Bp, L.b), z);
}

// wire step to the sinks [s0, s1): every lane its condition; the positions and
// capacitances of four sinks are loaded before their stores
__device__ __forceinline__ void store_sinks(const DevNet& g, const BatchState& bs, int s0, int s1, const Lane& L,
                                            float2 xyd, const FOut& o, bool lse) {
    for (int p0 = s0; p0 < s1; p0 += 4) {
        float2 xy[4];
        float cap[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = min(p0 + u, s1 - 1);
            xy[u] = bs.xy[ix(p, bs.Bp, L.b)];
            cap[u] = __ldg(g.pin_cap + p);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (p0 + u < s1) {
                const Wire w = wire(g, xy[u], xyd, cap[u]);
                store_pin(bs, p0 + u, L, o.at + w.D, sqrtf(fmaf(o.sl, o.sl, w.I * w.I)), o.z + w.D, lse);
            }
        }
    }
}

// net load (Eq. 1): lane c of the quad sums sinks c, c + 4, ..., then the quad
// sum and the driver's pin capacitance
__device__ __forceinline__ float net_load(const DevNet& g, const BatchState& bs, int dp, int s1, const Lane& L,
                                          float2 xyd) {
    float acc = 0.f;
#pragma unroll 4
    for (int p = dp + 1 + L.c; p < s1; p += 4) {
        const float2 xy = bs.xy[ix(p, bs.Bp, L.b)];
        const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
        acc += fmaf(g.c, dist, __ldg(g.pin_cap + p));
    }
    return __ldg(g.pin_cap + dp) + quad_sum(acc);
}

// kWait: dataflow sweep (wait for the producers; the net's load is computed
// here); otherwise a level-synchronous sweep (producers ran in earlier
// launches; every load comes from the prologue).  The first round of the
// wait is issued as soon as the cell's record is known, before the net's load
// and the table segment.
template <bool lse, bool kWait>
__device__ void bfwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int q, int n0, int nn,
                          const Lane& L, float gamma, bool stall = false) {
    const int Bp = bs.Bp;
    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = g.net_ptr[n], e = g.net_ptr[n + 1];
        FCell f = fcell_topo(g, n, L.rf);
        FIn in;
        const bool ok = fcell_fanin<kWait>(bs, f, L, lse, stall, in);
        const float2 xyd = bs.xy[ix(dp, Bp, L.b)];
        float ld;
        if constexpr (kWait) {
            ld = net_load(g, bs, dp, e, L, xyd);
            if (L.c == 0) bs.load[ix(n, Bp, L.b)] = ld;
        } else {
            ld = bs.load[ix(n, Bp, L.b)];
        }
        fcell_lib(g, f, ld);
        const FOut o = fcell_eval<kWait>(g, bs, f, dp, L, gamma, lse, d.abort_word, stall, in, ok);
        if (f.t >= 0) store_pin(bs, dp, L, o.at, o.sl, o.z, lse);
        store_sinks(g, bs, dp + 1, e, L, xyd, o, lse);
    }
}

// chunk of a large net: its load comes from the prologue; every chunk
// evaluates the driver cell, the first one stores it
template <bool lse, bool kWait>
__device__ void bfwd_chunk(const DevNet& g, const BatchState& bs, const DfState& d, int q, int n, int p0, int cnt,
                           const Lane& L, float gamma, bool stall = false) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    FCell f = fcell_topo(g, n, L.rf);
    FIn in;
    const bool ok = fcell_fanin<kWait>(bs, f, L, lse, stall, in);
    const float2 xyd = bs.xy[ix(dp, Bp, L.b)];
    fcell_lib(g, f, bs.load[ix(n, Bp, L.b)]);
    const FOut o = fcell_eval<kWait>(g, bs, f, dp, L, gamma, lse, d.abort_word, stall, in, ok);
    if (f.t >= 0 && p0 == dp + 1) store_pin(bs, dp, L, o.at, o.sl, o.z, lse);
    store_sinks(g, bs, p0, p0 + cnt, L, xyd, o, lse);
}

constexpr int kFwdGrab = 2;

template <bool lse>
__global__ void __launch_bounds__(kBlock, 4) k_bfwd(DevNet g, BatchState bs, DfState d, float gamma,
                                                    int stall_task) {
    const int GT = bs.GT;
    const int Q = d.TF * GT;
    // Two queue entries per grab (usually one task for two groups of 8
    // placements), taken in order: half the atomics on the queue head, which
    // at 64 placements sees a million grabs per sweep (measured 13% faster than
    // one entry, 4 and 8 entries slower again).  The smallest unfinished entry
    // is always the one its warp is running, and its producers have smaller
    // entries, so the sweep still progresses.
    int q0 = grab_n(d.heads + 0, kFwdGrab);
    while (q0 < Q) {
        for (int q = q0; q < q0 + kFwdGrab && q < Q; ++q) {
            const int t = q / GT, gq = q - t * GT;
            const Lane L = lane_of(gq);
            const int4 task = d.ftask[t];
            if (task.y > 0) bfwd_nets<lse, true>(g, bs, d, q, task.x, task.y, L, gamma, t == stall_task);
            else bfwd_chunk<lse, true>(g, bs, d, q, task.x, task.z, task.w, L, gamma, t == stall_task);
        }
        q0 = grab_n(d.heads + 0, kFwdGrab);  // the next entries only once these are done
    }
}

// Loads of the large nets (the chunk tasks read them), in chunks of at most
// kLoadChunk sinks: a block per (chunk, group of 32 placements).  Warp w sums
// the chunk's sinks w, w + 8, ..., the warps' sums are added in warp order,
// and the last block of a net to finish adds the driver's capacitance and the
// chunks' sums in chunk order, so the result is fixed (and a 20,000-sink net
// is 79 blocks, not one).  The per-net counters return to zero for the next
// launch.
__global__ void __launch_bounds__(kBlock) k_bload(DevNet g, BatchState bs, const int4* __restrict__ chunks,
                                                  float* __restrict__ part, int32_t* __restrict__ cnt) {
    __shared__ float sh[kWarpsPerBlock][32];
    __shared__ int last;
    // net, first sink, the net's first chunk, sinks | (chunks of the net << 16)
    const int4 c = chunks[blockIdx.x];
    const int n = c.x, p0 = c.y, first = c.z, np = c.w & 0xffff, nch = c.w >> 16;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane, Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    float acc = 0.f;
#pragma unroll 4
    for (int p = p0 + w; p < p0 + np; p += kWarpsPerBlock) {
        const float2 xy = bs.xy[ix(p, Bp, b)];
        const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
        acc += fmaf(g.c, dist, __ldg(g.pin_cap + p));
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        float v = 0.f;
#pragma unroll
        for (int k = 0; k < kWarpsPerBlock; ++k) v += sh[k][lane];
        part[(size_t)blockIdx.x * Bp + b] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int32_t* ct = cnt + (size_t)first * bs.G + blockIdx.y;
        last = atomicAdd(ct, 1) == nch - 1;
        if (last) *ct = 0;  // every chunk of this net and group has counted
    }
    __syncthreads();
    if (last && w == 0) {
        __threadfence();
        float ld = __ldg(g.pin_cap + dp);
        for (int k = 0; k < nch; ++k) ld += __ldcg(part + (size_t)(first + k) * Bp + b);
        bs.load[ix(n, Bp, b)] = ld;
    }
}

// ---------------------------------------------------------------------------
// Endpoints: slack, WNS, TNS and the smoothed TNS / WNS per placement (lane =
// placement); the same accumulator and merge order as the single-placement
// reduction, per lane.
// ---------------------------------------------------------------------------
struct BEp {
    double tns_e, tns_l, tns_g, viol;
    float wns_e, wns_l, wmin, wsum;
};

__device__ __forceinline__ BEp bep_identity() {
    BEp a;
    a.tns_e = a.tns_l = a.tns_g = a.viol = 0.0;
    a.wns_e = a.wns_l = a.wmin = kInf;
    a.wsum = 0.f;
    return a;
}

__device__ __forceinline__ void bep_merge(BEp& a, const BEp& b, float gamma) {
    a.tns_e += b.tns_e;
    a.tns_l += b.tns_l;
    a.tns_g += b.tns_g;
    a.viol += b.viol;
    a.wns_e = fminf(a.wns_e, b.wns_e);
    a.wns_l = fminf(a.wns_l, b.wns_l);
    const float m = fminf(a.wmin, b.wmin);
    float sum = 0.f;
    if (a.wsum > 0.f) sum += a.wsum * expf(-(a.wmin - m) / gamma);
    if (b.wsum > 0.f) sum += b.wsum * expf(-(b.wmin - m) / gamma);
    a.wsum = sum;
    a.wmin = m;
}

// Bounds of endpoint e in placement b (hold, hold, setup, setup); a propagated
// clock adds the capturing clock pin's late rising arrival to the hold bound
// and its early rising arrival to the setup bound.  Returns the clock pin or -1.
__device__ __forceinline__ int bep_bounds(const DevNet& g, const BatchState& bs, int e, int b, float4& con) {
    con = reinterpret_cast<const float4*>(g.ep_rat)[e];
    const int k = g.ep_clk ? g.ep_clk[e] : -1;
    if (k >= 0) {
        const float early = bs.at[ix(4 * k, bs.Bp, b)], late = bs.at[ix(4 * k + 2, bs.Bp, b)];
        con.x += late;
        con.y += late;
        con.z += early;
        con.w += early;
    }
    return k;
}

// Propagated clock, per placement: d loss / d (setup bound) of each clocked
// endpoint, which enters the adjoint of its clock pin's rising LSE arrival
// (the arc step that writes that word adds it).  grid (ceil(E / 8), G).
__global__ void __launch_bounds__(kBlock) k_bcap_seed(DevNet g, BatchState bs, float gamma) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane, Bp = bs.Bp;
    const int e = blockIdx.x * kWarpsPerBlock + w;
    if (e >= g.E) return;
    float4 con;
    const int k = bep_bounds(g, bs, e, b, con);
    if (k < 0) return;
    const int p = g.ep_pin[e];
    const float W = (float)bs.summary[(size_t)b * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
    const float wt = bs.params[2 * b], ww = bs.params[2 * b + 1];
    const float sr = con.z - bs.ats[ix(2 * p, Bp, b)], sf = con.w - bs.ats[ix(2 * p + 1, Bp, b)];
    const float te = softmin3(sr, sf, gamma);
    float gr = wt * expf(-(sr - te) / gamma), gf = wt * expf(-(sf - te) / gamma);
    if (isfinite(W)) {
        gr += ww * expf(-(sr - W) / gamma);
        gf += ww * expf(-(sf - W) / gamma);
    }
    bs.cap_seed[ix(k, Bp, b)] = gr + gf;
}

// A lane's own endpoints are summed in float (a handful per lane, so the sums
// stay within a few ulps), then the lanes' partials in double: double
// arithmetic runs at a small fraction of the float rate on this part.
struct BEpF {
    float tns_e, tns_l, tns_g, viol;
    float wns_e, wns_l, wmin, wsum;
};

__device__ __forceinline__ BEpF bepf_identity() {
    BEpF a;
    a.tns_e = a.tns_l = a.tns_g = a.viol = 0.f;
    a.wns_e = a.wns_l = a.wmin = kInf;
    a.wsum = 0.f;
    return a;
}

__device__ __forceinline__ void bepf_merge(BEpF& a, const BEpF& b, float gamma) {
    a.tns_e += b.tns_e;
    a.tns_l += b.tns_l;
    a.tns_g += b.tns_g;
    a.viol += b.viol;
    a.wns_e = fminf(a.wns_e, b.wns_e);
    a.wns_l = fminf(a.wns_l, b.wns_l);
    const float m = fminf(a.wmin, b.wmin);
    float sum = 0.f;
    if (a.wsum > 0.f) sum += a.wsum * expf(-(a.wmin - m) / gamma);
    if (b.wsum > 0.f) sum += b.wsum * expf(-(b.wmin - m) / gamma);
    a.wsum = sum;
    a.wmin = m;
}

// grid (kRedBlocks, G): block x takes endpoints x*8 + w, stepping by
// kRedBlocks*8; partial per (block, placement)
__global__ void __launch_bounds__(kBlock) k_bep1(DevNet g, BatchState bs, float gamma, int lse) {
    __shared__ BEp sh[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane, Bp = bs.Bp;
    BEpF accf = bepf_identity();
    for (int e = blockIdx.x * kWarpsPerBlock + w; e < g.E; e += gridDim.x * kWarpsPerBlock) {
        const int p = g.ep_pin[e];
        float4 con;
        // a clocked endpoint's bounds are this placement's required-time seeds
        if (bep_bounds(g, bs, e, b, con) >= 0) {
            bs.rat[ix(4 * p, Bp, b)] = con.x;
            bs.rat[ix(4 * p + 1, Bp, b)] = con.y;
            bs.rat[ix(4 * p + 2, Bp, b)] = con.z;
            bs.rat[ix(4 * p + 3, Bp, b)] = con.w;
        }
        const float a0 = bs.at[ix(4 * p, Bp, b)], a1 = bs.at[ix(4 * p + 1, Bp, b)];
        const float a2 = bs.at[ix(4 * p + 2, Bp, b)], a3 = bs.at[ix(4 * p + 3, Bp, b)];
        const float se = fminf(a0 - con.x, a1 - con.y);
        const float sl = fminf(con.z - a2, con.w - a3);
        bs.ep_slack[ix(e, Bp, b)] = make_float2(se, sl);
        BEpF v = bepf_identity();
        v.wns_e = se;
        v.wns_l = sl;
        v.tns_e = fminf(se, 0.f);
        v.tns_l = fminf(sl, 0.f);
        v.viol = sl < 0.f ? 1.f : 0.f;
        if (lse) {
            const float sr = con.z - bs.ats[ix(2 * p, Bp, b)], sf = con.w - bs.ats[ix(2 * p + 1, Bp, b)];
            v.tns_g = softmin3(sr, sf, gamma);
            v.wmin = fminf(sr, sf);
            v.wsum = expf(-(sr - v.wmin) / gamma) + expf(-(sf - v.wmin) / gamma);
        }
        bepf_merge(accf, v, gamma);
    }
    BEp acc;
    acc.tns_e = accf.tns_e;
    acc.tns_l = accf.tns_l;
    acc.tns_g = accf.tns_g;
    acc.viol = accf.viol;
    acc.wns_e = accf.wns_e;
    acc.wns_l = accf.wns_l;
    acc.wmin = accf.wmin;
    acc.wsum = accf.wsum;
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        for (int k = 1; k < kWarpsPerBlock; ++k) bep_merge(acc, sh[k][lane], gamma);
        reinterpret_cast<BEp*>(bs.red)[ix(blockIdx.x, Bp, b)] = acc;
    }
}

// warp per placement: lane l merges partials l, l + 32, ... in order, then a
// butterfly across the lanes (each merge is symmetric in its operands, so both
// lanes of a pair hold the same bits and the result is fixed)
__global__ void k_bep2(DevNet g, BatchState bs, float gamma, int lse, int nparts) {
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= bs.Bp) return;  // warp-uniform
    BEp acc = bep_identity();
    for (int k = lane; k < nparts; k += 32) bep_merge(acc, reinterpret_cast<const BEp*>(bs.red)[ix(k, bs.Bp, b)], gamma);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        BEp o;
        o.tns_e = __shfl_xor_sync(kFull, acc.tns_e, off);
        o.tns_l = __shfl_xor_sync(kFull, acc.tns_l, off);
        o.tns_g = __shfl_xor_sync(kFull, acc.tns_g, off);
        o.viol = __shfl_xor_sync(kFull, acc.viol, off);
        o.wns_e = __shfl_xor_sync(kFull, acc.wns_e, off);
        o.wns_l = __shfl_xor_sync(kFull, acc.wns_l, off);
        o.wmin = __shfl_xor_sync(kFull, acc.wmin, off);
        o.wsum = __shfl_xor_sync(kFull, acc.wsum, off);
        bep_merge(acc, o, gamma);
    }
    if (lane != 0) return;
    double* o = bs.summary + (size_t)b * STA_SUM_COUNT;
    o[STA_SUM_WNS_EARLY] = acc.wns_e;
    o[STA_SUM_TNS_EARLY] = acc.tns_e;
    o[STA_SUM_WNS_LATE] = acc.wns_l;
    o[STA_SUM_TNS_LATE] = acc.tns_l;
    o[STA_SUM_TNS_GAMMA] = lse ? acc.tns_g : 0.0;
    o[STA_SUM_WNS_GAMMA] =
        (lse && acc.wsum > 0.f) ? (double)acc.wmin - (double)gamma * log((double)acc.wsum) : (double)kInf;
    o[STA_SUM_LATE_VIOLATIONS] = acc.viol;
    o[STA_SUM_NUM_ENDPOINTS] = g.E;
}

// ---------------------------------------------------------------------------
// Backward (mode 1 required times, 2 adjoint, 3 both); lanes as in the forward.
// Every lane carries the required time of its condition; the late lanes (one
// per output transition) carry the adjoint.
// ---------------------------------------------------------------------------

// One lane's part of a driver cell's backward step, all from forward results:
// the arc delays of its condition (required times) and, on late lanes, the LSE
// weights, the delay partials, and the arc of the late slew (first one on ties)
// with its slew partials.
struct BCell {
    int t, na, rfi;
    int pin[STA_MAX_ARCS];
    float adel[STA_MAX_ARCS], w[STA_MAX_ARCS], dDs[STA_MAX_ARCS], dDl[STA_MAX_ARCS];
    int amax;
    float dSs, dSl;
    float cs;  // propagated clock: the setup seed of a one-input cell's clock pin (rising lane)
};

template <int mode>
__device__ __forceinline__ BCell bcell_pre(const DevNet& g, const BatchState& bs, int n, int dp, const Lane& L,
                                           float gamma) {
    const int Bp = bs.Bp, b = L.b, el = L.el, rf = L.rf;
    BCell bc;
    const int4 q0 = __ldg(g.net_desc + 2 * n), q1 = __ldg(g.net_desc + 2 * n + 1);  // one record
    bc.t = q0.x;
    bc.na = q0.z;
    const int dpin[STA_MAX_ARCS] = {q1.x, q1.y, q1.z, q1.w};
    bc.rfi = 0;
    bc.amax = -1;
    bc.dSs = bc.dSl = bc.cs = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        bc.pin[k] = 0;
        bc.adel[k] = bc.w[k] = bc.dDs[k] = bc.dDl[k] = 0.f;
    }
    if (bc.t < 0) return bc;
    const bool need = (mode & 1) || el;  // mode 2 needs the late lanes only
    const int t = bc.t;
    const int un = q0.w >> 4;
    const float ld = bs.load[ix(n, Bp, b)];
    const float* li = g.lib_idx + t * kLibStride + 8;
    const int jl = axis_seg(li, ld);
    const float inv_l = __ldg(g.lib_inv + t * kLibStride + 8 + jl);
    const float ul = (ld - __ldg(li + jl)) * inv_l;
    const float zd = ((mode & 2) && el) ? bs.ats[ix(2 * dp + rf, Bp, b)] : 0.f;
    float best = -kInf;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < bc.na) {
            bc.pin[k] = dpin[k];
            const int r = rf ^ ((un >> k) & 1);
            bc.rfi |= r << k;
            if (need) {
                const float sin = bs.slew[ix(4 * bc.pin[k] + 2 * el + r, Bp, b)];
                const float* si = g.lib_idx + t * kLibStride;
                const int is = axis_seg(si, sin);
                const float inv_s = __ldg(g.lib_inv + t * kLibStride + is);
                const float ts = (sin - __ldg(si + is)) * inv_s;
                float4 dq, sq;
                cell_corners(g, t, k, rf, is, jl, dq, sq);
                float dDs, dDl, dSs, dSl;
                const float D = lerp_cell_grad(dq, ts, ul, inv_s, inv_l, dDs, dDl);
                bc.adel[k] = D;
                if ((mode & 2) && el) {
                    const float S = lerp_cell_grad(sq, ts, ul, inv_s, inv_l, dSs, dSl);
                    bc.dDs[k] = dDs;
                    bc.dDl[k] = dDl;
                    bc.w[k] = expf((bs.ats[ix(2 * bc.pin[k] + r, Bp, b)] + D - zd) / gamma);
                    if (S > best) {
                        best = S;
                        bc.amax = k;
                        bc.dSs = dSs;
                        bc.dSl = dSl;
                    }
                }
            }
        }
    }
    // a capturing clock pin is the input of a one-input cell; its seed is read
    // here, before the wait, and added to the rising adjoint it writes
    if ((mode & 2) && el && bs.cap_seed && bc.na == 1 && (bc.rfi & 1) == 0)
        bc.cs = __ldcg(bs.cap_seed + ix(bc.pin[0], Bp, b));
    return bc;
}

// Required times of the cell's inputs (R = this lane's condition at the
// output) and, on late lanes, the adjoint through the LSE, the NLDM partials
// and the late-slew max; returns the lane's part of d loss / d load.
template <int mode>
__device__ __forceinline__ float bcell_apply(const BatchState& bs, const BCell& bc, const Lane& L, float R, float GA,
                                             float GS) {
    const int Bp = bs.Bp, b = L.b, el = L.el;
    float gl = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < bc.na) {
            const int r = (bc.rfi >> k) & 1;
            // strong stores: words that the sinks' tasks poll
            if (mode & 1) st_relaxed_f(bs.rat + ix(4 * bc.pin[k] + 2 * el + r, Bp, b), R - bc.adel[k]);
            if ((mode & 2) && el) {
                const float gD = GA * bc.w[k];
                // a capturing clock pin also carries its endpoint's setup term
                st_relaxed_f(bs.g_ats + ix(2 * bc.pin[k] + r, Bp, b), (bs.cap_seed && k == 0) ? gD + bc.cs : gD);
                st_relaxed_f(bs.g_slew + ix(2 * bc.pin[k] + r, Bp, b),
                             fmaf(gD, bc.dDs[k], k == bc.amax ? GS * bc.dSs : 0.f));
                gl = fmaf(gD, bc.dDl[k], gl);
            }
        }
    }
    if ((mode & 2) && el && bc.amax >= 0) gl = fmaf(GS, bc.dSl, gl);
    return gl;
}

// One sink's terms for this lane: r = RAT_s - Delay_s of its condition; on late
// lanes the sink's LSE-arrival adjoint ga, the slew term gs = g_slew_s *
// slew_d / slew_s, and this transition's part of the wire adjoint.
// Cell-input sinks read what their cell's task wrote (through L2); endpoints
// and dangling sinks are constant: the constraint (or +-inf) and the seed
// d loss / d LSE-AT = -(w_tns dTNS_g/ds + w_wns dWNS_g/ds).
struct BSink {
    float r, ga, gs, gw;
    Wire w;
};

// An endpoint sink's adjoint seed for output transition rf, from its slacks
// sr, sf: d loss / d LSE-arrival (the TNS soft-min with the zero term, and the
// WNS soft-min's share).  Out of line, like batch_wide.cu's: endpoints are a
// small share of the sinks, and the accurate exponentials inlined in every
// sink loop crowd the instruction cache.  Same operations, same bits.
__device__ __noinline__ float bsink_seed(float sr, float sf, int rf, float gamma, float W, float wt, float ww) {
    const float te = softmin3(sr, sf, gamma);
    const float sv = rf ? sf : sr;
    float gv = wt * expf(-(sv - te) / gamma);
    if (isfinite(W)) gv += ww * expf(-(sv - W) / gamma);
    return -gv;
}

template <int mode, bool kPoll>
__device__ __forceinline__ BSink bsink(const DevNet& g, const BatchState& bs, const DfState& d, int p, const Lane& L,
                                       float2 xyd, float sld, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp, b = L.b;
    BSink s;
    s.w = wire(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p));
    const bool dyn = d.pin_cons[p] >= 0;  // the same for every lane
    // the sink's words written by the task of the cell it feeds; in the
    // dataflow sweep this is the wait (repeated until written)
    float rr = 0.f, ga = 0.f, gs = 0.f;
    auto load = [&]() {
        bool ok = true;
        if (mode & 1) {
            rr = kPoll ? ld_relaxed_f(bs.rat + ix(4 * p + L.c, Bp, b)) : __ldcg(bs.rat + ix(4 * p + L.c, Bp, b));
            ok &= written(rr);
        }
        if ((mode & 2) && L.el && dyn) {
            ga = kPoll ? ld_relaxed_f(bs.g_ats + ix(2 * p + L.rf, Bp, b)) : __ldcg(bs.g_ats + ix(2 * p + L.rf, Bp, b));
            gs = kPoll ? ld_relaxed_f(bs.g_slew + ix(2 * p + L.rf, Bp, b))
                       : __ldcg(bs.g_slew + ix(2 * p + L.rf, Bp, b));
            ok &= written(ga) & written(gs);
        }
        return ok;
    };
    if (kPoll && dyn) poll_words(load, d.abort_word);
    else load();
    s.r = (mode & 1) ? rr - s.w.D : 0.f;
    s.ga = s.gs = s.gw = 0.f;
    if ((mode & 2) && L.el) {
        if (dyn) {
            // ga, gs loaded above
        } else {
            const float rl = bs.rat[ix(4 * p + 2, Bp, b)], rfl = bs.rat[ix(4 * p + 3, Bp, b)];
            if (isfinite(rl)) {
                const float sr = rl - bs.ats[ix(2 * p, Bp, b)], sf = rfl - bs.ats[ix(2 * p + 1, Bp, b)];
                ga = bsink_seed(sr, sf, L.rf, gamma, sd.W, sd.wt, sd.ww);
            }
        }
        const float sl = bs.slew[ix(4 * p + 2 + L.rf, Bp, b)];
        const float qv = sl > 0.f ? gs / sl : 0.f;
        s.ga = ga;
        s.gs = qv * sld;
        s.gw = fmaf(qv, s.w.I, ga);
    }
    return s;
}


__device__ __forceinline__ float late_slew_of_driver(const BatchState& bs, int dp, const Lane& L) {
    return L.el ? bs.slew[ix(4 * dp + 2 + L.rf, bs.Bp, L.b)] : 0.f;
}

template <int mode, bool kWait>
__device__ void bbwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n0, int nn,
                          const Lane& L, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp, b = L.b;
    const int dp0 = g.net_ptr[n0];
    BCell bc = bcell_pre<mode>(g, bs, n0, dp0, L, gamma);
    const float2 xyd0 = bs.xy[ix(dp0, Bp, b)];
    const float sld0 = (mode & 2) ? late_slew_of_driver(bs, dp0, L) : 0.f;

    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = j ? g.net_ptr[n] : dp0, e = g.net_ptr[n + 1];
        float2 xyd = xyd0;
        float sld = sld0;
        if (j) {
            bc = bcell_pre<mode>(g, bs, n, dp, L, gamma);
            xyd = bs.xy[ix(dp, Bp, b)];
            sld = (mode & 2) ? late_slew_of_driver(bs, dp, L) : 0.f;
        }
        float R = L.el ? kInf : -kInf, GA = 0.f, GS = 0.f;
#pragma unroll 2
        for (int p = dp + 1; p < e; ++p) {
            const BSink s = bsink<mode, kWait>(g, bs, d, p, L, xyd, sld, gamma, sd);
            R = L.el ? fminf(R, s.r) : fmaxf(R, s.r);
            GA += s.ga;
            GS += s.gs;
            if (mode & 2) {  // the sink's wire adjoint, both transitions; kept until d loss / d load is known
                const float gw = s.gw + __shfl_xor_sync(kFull, s.gw, 1);
                if (L.c == 2) bs.grad[ix(p, Bp, b)].x = gw;
            }
        }
        if (mode & 1) bs.rat[ix(4 * dp + L.c, Bp, b)] = R;
        const float gl = bcell_apply<mode>(bs, bc, L, R, GA, GS);
        if (mode & 2) {
            const float gload = quad_sum(gl);  // early lanes contribute 0
            __syncwarp();                      // the wire adjoints stored by lane 2 of each quad
            float sx = 0.f, sy = 0.f;
            for (int p = dp + 1 + L.c; p < e; p += 4) {
                const float gw = bs.grad[ix(p, Bp, b)].x;
                const float2 gxy = bsink_grad(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p), gw, gload);
                bs.grad[ix(p, Bp, b)] = gxy;
                sx += gxy.x;
                sy += gxy.y;
            }
            sx = quad_sum(sx);
            sy = quad_sum(sy);
            if (L.c == 0) bs.grad[ix(dp, Bp, b)] = make_float2(-sx, -sy);
        }
    }
}

// Partial chunk of a large net.  Slots of a partial record (per placement):
//   0-3 max/max/min/min of RAT_s - Delay_s, 4-5 sums of g_ats, 6-7 sums of
//   g_slew * slew_d / slew_s, 8-9 sums of sign(x_s - x_d), sign(y_s - y_d),
//   10-11 sums of sign * g_wire * dDelay/dd (the driver's gradient is
//   -(gload * c * sums 8-9 + sums 10-11)).
template <int mode, bool kWait>
__device__ void bbwd_part(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n, int p0,
                          int np, int slot, const Lane& L, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp, b = L.b;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float sld = (mode & 2) ? late_slew_of_driver(bs, dp, L) : 0.f;

    float R = L.el ? kInf : -kInf, GA = 0.f, GS = 0.f, sx = 0.f, sy = 0.f, hx = 0.f, hy = 0.f;
#pragma unroll 2
    for (int p = p0; p < p0 + np; ++p) {
        const BSink s = bsink<mode, kWait>(g, bs, d, p, L, xyd, sld, gamma, sd);
        R = L.el ? fminf(R, s.r) : fmaxf(R, s.r);
        GA += s.ga;
        GS += s.gs;
        if (mode & 2) {
            const float gw = s.gw + __shfl_xor_sync(kFull, s.gw, 1);
            const float2 xy = bs.xy[ix(p, Bp, b)];
            const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
            const float ex = (dx > 0.f) - (dx < 0.f), ey = (dy > 0.f) - (dy < 0.f);
            const float h = gw * (kKrc * g.r * fmaf(g.c, s.w.dist, __ldg(g.pin_cap + p)));
            sx += ex;
            sy += ey;
            hx += ex * h;
            hy += ey * h;
        }
    }
    float* part = (mode & 2) ? bs.part : bs.rpart;
    const int base = slot * kPartFloats;
    // strong stores: the driver step polls these words
    st_relaxed_f(part + ix(base + L.c, Bp, b), R);
    if ((mode & 2) && L.el) {
        st_relaxed_f(part + ix(base + 4 + L.rf, Bp, b), GA);
        st_relaxed_f(part + ix(base + 6 + L.rf, Bp, b), GS);
    }
    if ((mode & 2) && L.c == 2) {  // lane 2 holds the wire adjoints of both transitions
        st_relaxed_f(part + ix(base + 8, Bp, b), sx);
        st_relaxed_f(part + ix(base + 9, Bp, b), sy);
        st_relaxed_f(part + ix(base + 10, Bp, b), hx);
        st_relaxed_f(part + ix(base + 11, Bp, b), hy);
    }
}

template <int mode, bool kWait>
__device__ void bbwd_driver(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n,
                            int slot0, int nch, const Lane& L, float gamma) {
    const int Bp = bs.Bp, b = L.b;
    const int dp = g.net_ptr[n];
    const BCell bc = bcell_pre<mode>(g, bs, n, dp, L, gamma);

    const float* part = (mode & 2) ? bs.part : bs.rpart;
    float R = L.el ? kInf : -kInf, GA = 0.f, GS = 0.f, sx = 0.f, sy = 0.f, hx = 0.f, hy = 0.f;
    // The chunks' partials in chunk order.  Lane c of a quad reads slots c
    // (its required time), 4 + c and 8 + c of every chunk, loads of 8 chunks
    // issued together; the sums are then handed to the lanes that use them.
    constexpr int kU = 8;
    float v4 = 0.f, v8 = 0.f;
    for (int k0 = 0; k0 < nch; k0 += kU) {
        float vr[kU], va[kU], vb[kU];
        // in the dataflow sweep this is the wait: repeated until the 8 chunks'
        // words this lane reads are written
        auto load = [&]() {
            bool all = true;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int base = (slot0 + k0 + u) * kPartFloats;
                const bool ok = k0 + u < nch;
                vr[u] = ok ? (kWait ? ld_relaxed_f(part + ix(base + L.c, Bp, b)) : __ldcg(part + ix(base + L.c, Bp, b)))
                           : (L.el ? kInf : -kInf);
                va[u] = ((mode & 2) && ok)
                            ? (kWait ? ld_relaxed_f(part + ix(base + 4 + L.c, Bp, b)) : __ldcg(part + ix(base + 4 + L.c, Bp, b)))
                            : 0.f;
                vb[u] = ((mode & 2) && ok)
                            ? (kWait ? ld_relaxed_f(part + ix(base + 8 + L.c, Bp, b)) : __ldcg(part + ix(base + 8 + L.c, Bp, b)))
                            : 0.f;
                if (ok) all &= written(vr[u]) & (!(mode & 2) || (written(va[u]) & written(vb[u])));
            }
            return all;
        };
        if constexpr (kWait) poll_words(load, d.abort_word);
        else load();
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (k0 + u >= nch) break;
            R = L.el ? fminf(R, vr[u]) : fmaxf(R, vr[u]);
            v4 += va[u];
            v8 += vb[u];
        }
    }
    {
        // slot 4 + c: lanes 0, 1 hold the g_ats sums (rise, fall), lanes 2, 3 the
        // g_slew sums; slot 8 + c: sx, sy, hx, hy
        const int q0 = L.lane & ~3;
        const float ga_src = __shfl_sync(kFull, v4, q0 + (L.c & 1));
        const float sx_ = __shfl_sync(kFull, v8, q0 + 0), sy_ = __shfl_sync(kFull, v8, q0 + 1);
        const float hx_ = __shfl_sync(kFull, v8, q0 + 2), hy_ = __shfl_sync(kFull, v8, q0 + 3);
        GA = L.el ? ga_src : 0.f;
        GS = L.el ? v4 : 0.f;
        sx = sx_;
        sy = sy_;
        hx = hx_;
        hy = hy_;
    }
    if (mode & 1) bs.rat[ix(4 * dp + L.c, Bp, b)] = R;
    const float gl = bcell_apply<mode>(bs, bc, L, R, GA, GS);
    if (mode & 2) {
        const float gload = quad_sum(gl);
        if (L.c == 2) {
            bs.net_gload[ix(n, Bp, b)] = gload;
            bs.grad[ix(dp, Bp, b)] = make_float2(-fmaf(gload * g.c, sx, hx), -fmaf(gload * g.c, sy, hy));
        }
    }
}

// Gradient chunk of a large net: d loss / d (x, y) of its sinks once the
// driver task has published d loss / d load.  No task waits for these.
template <bool kWait>
__device__ void bbwd_grad(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n, int p0,
                          int np, const Lane& L, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp, b = L.b;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float sld = late_slew_of_driver(bs, dp, L);
    if constexpr (kWait) wait_ready(cnt, q, d.b_indeg[q / bs.GT], d.abort_word);
    const float gload = __ldcg(bs.net_gload + ix(n, Bp, b));
#pragma unroll 2
    for (int p = p0; p < p0 + np; ++p) {
        const BSink s = bsink<2, false>(g, bs, d, p, L, xyd, sld, gamma, sd);
        const float gw = s.gw + __shfl_xor_sync(kFull, s.gw, 1);
        if (L.c == 2)
            bs.grad[ix(p, Bp, b)] = bsink_grad(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p), gw, gload);
    }
}

template <int mode, bool kWait>
__device__ __forceinline__ void bbwd_task(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q,
                                          int t, const Lane& L, float gamma) {
    BSeed sd;
    sd.W = (float)bs.summary[(size_t)L.b * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
    sd.wt = bs.params[2 * L.b];
    sd.ww = bs.params[2 * L.b + 1];
    const int4 task = d.btask[t];
    if (task.y > 0) {
        bbwd_nets<mode, kWait>(g, bs, d, cnt, q, task.x, task.y, L, gamma, sd);
    } else if (task.y == -1) {
        bbwd_part<mode, kWait>(g, bs, d, cnt, q, task.x, task.z, task.w, d.baux[t], L, gamma, sd);
    } else if (task.y == -2) {
        bbwd_driver<mode, kWait>(g, bs, d, cnt, q, task.x, task.z, task.w, L, gamma);
    } else if (mode & 2) {
        bbwd_grad<kWait>(g, bs, d, cnt, q, task.x, task.z, task.w, L, gamma, sd);
    }  // gradient chunks have no work in the required-time sweep
}

template <int mode>
__global__ void __launch_bounds__(kBlock, 3) k_bbwd(DevNet g, BatchState bs, DfState d, float gamma) {
    int32_t* cnt = (mode & 2) ? d.acnt : d.rcnt;
    int32_t* head = d.heads + ((mode & 2) ? 2 : 1);
    const int GT = bs.GT;
    const int Q = d.TB * GT;
    int q = grab(head);
    while (q < Q) {
        const int t = q / GT, gq = q - t * GT;
        const Lane L = lane_of(gq);
        bbwd_task<mode, true>(g, bs, d, cnt, q, t, L, gamma);
        // every consumer polls the words its producers wrote, except the gradient
        // chunks of a large net, which wait on a counter that its driver step releases
        if (d.btask[t].y == -2) {
            __syncwarp();
            const int k1 = d.b_out_ptr[t + 1];
            for (int k = d.b_out_ptr[t] + L.lane; k < k1; k += 32) red_release_add(cnt + d.b_out[k] * GT + gq, 1);
        }
        q = grab(head);
    }
}

// ---------------------------------------------------------------------------
// Level-synchronous batched sweeps: one launch per level (per phase in the
// backward), replayed from a CUDA graph.  A launch runs every (task, group) of
// its task ranges, a warp each; kernel boundaries order the levels, so there
// are no counters, waits or release fences.
// ---------------------------------------------------------------------------
struct Ranges {
    int a0, a1, b0, b1, c0, c1;  // up to three task ranges, run as one
};

__device__ __forceinline__ int range_task(const Ranges& r, int i) {
    const int na = r.a1 - r.a0, nb = r.b1 - r.b0;
    return i < na ? r.a0 + i : (i < na + nb ? r.b0 + i - na : r.c0 + i - na - nb);
}

template <bool lse>
__global__ void __launch_bounds__(kBlock, 4) k_bfwd_lvl(DevNet g, BatchState bs, DfState d, int t0, int t1,
                                                      float gamma) {
    const int GT = bs.GT;
    const int nw = (t1 - t0) * GT;
    for (int i = (blockIdx.x * kBlock + threadIdx.x) >> 5; i < nw; i += gridDim.x * kWarpsPerBlock) {
        const int t = t0 + i / GT, gq = i - (i / GT) * GT;
        const Lane L = lane_of(gq);
        const int4 task = d.ftask[t];
        if (task.y > 0) bfwd_nets<lse, false>(g, bs, d, 0, task.x, task.y, L, gamma);
        else bfwd_chunk<lse, false>(g, bs, d, 0, task.x, task.z, task.w, L, gamma);
    }
}

template <int mode>
__global__ void __launch_bounds__(kBlock, 3) k_bbwd_lvl(DevNet g, BatchState bs, DfState d, Ranges r, float gamma) {
    const int GT = bs.GT;
    const int nw = ((r.a1 - r.a0) + (r.b1 - r.b0) + (r.c1 - r.c0)) * GT;
    for (int i = (blockIdx.x * kBlock + threadIdx.x) >> 5; i < nw; i += gridDim.x * kWarpsPerBlock) {
        const int k = i / GT, gq = i - k * GT;
        bbwd_task<mode, false>(g, bs, d, nullptr, 0, range_task(r, k), lane_of(gq), gamma);
    }
}

// Loads (Eq. 1) of every net of at most `big` pins, before a level-synchronous
// forward sweep: a warp per (net, 32 placements), lane = placement.  Sinks are
// summed in four interleaved partial sums combined as (s0 + s1) + (s2 + s3),
// the order of the quad sums of the dataflow sweep, so both sweeps give the
// same loads.
__global__ void __launch_bounds__(kBlock) k_bload_small(DevNet g, BatchState bs, int big) {
    const int lane = threadIdx.x & 31;
    const int nw = g.N * bs.G;
    for (int i = (blockIdx.x * kBlock + threadIdx.x) >> 5; i < nw; i += gridDim.x * kWarpsPerBlock) {
        const int n = i / bs.G, b = (i - n * bs.G) * 32 + lane;
        const int dp = g.net_ptr[n], e = g.net_ptr[n + 1];
        if (e - dp > big) continue;  // a large net: the block kernel
        const float2 xyd = bs.xy[ix(dp, bs.Bp, b)];
        float acc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int p = dp + 1; p < e; ++p) {
            const float2 xy = bs.xy[ix(p, bs.Bp, b)];
            const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
            const int k = (p - dp - 1) & 3;
            const float v = fmaf(g.c, dist, __ldg(g.pin_cap + p));
            acc[0] += k == 0 ? v : 0.f;
            acc[1] += k == 1 ? v : 0.f;
            acc[2] += k == 2 ? v : 0.f;
            acc[3] += k == 3 ? v : 0.f;
        }
        bs.load[ix(n, bs.Bp, b)] = __ldg(g.pin_cap + dp) + ((acc[0] + acc[1]) + (acc[2] + acc[3]));
    }
}

// ---------------------------------------------------------------------------
// Layout changes between the caller's placement-major arrays and the internal
// pin-major, placement-minor state.  A block moves a tile of 32 caller pins x
// 32 placements through shared memory so both sides are coalesced.
// ---------------------------------------------------------------------------

// xy_int[int(q)][b] = xy_user[b][q] for b < B (grid: pin tiles x groups)
__global__ void __launch_bounds__(kBlock) k_bxy_in(BatchState bs, const int32_t* __restrict__ pin_int, int P,
                                                   const float2* __restrict__ xy_user) {
    __shared__ float2 tile[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = blockIdx.y * 32;
    for (int q0 = blockIdx.x * 32; q0 < P; q0 += gridDim.x * 32) {
        for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = placement
            const int b = b0 + r, q = q0 + lane;
            tile[r][lane] = (b < bs.B && q < P) ? xy_user[(size_t)b * P + q] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = pin
            const int q = q0 + r, b = b0 + lane;
            if (q < P && b < bs.B) bs.xy[ix(pin_int[q], bs.Bp, b)] = tile[lane][r];
        }
        __syncthreads();
    }
}

// out[b][q] = in[int(q)][b] for b < B (float2 per pin and placement)
__global__ void __launch_bounds__(kBlock) k_bout2(BatchState bs, const int32_t* __restrict__ pin_int, int P,
                                                  const float2* __restrict__ in, float2* __restrict__ out) {
    __shared__ float2 tile[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = blockIdx.y * 32;
    for (int q0 = blockIdx.x * 32; q0 < P; q0 += gridDim.x * 32) {
        for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = pin
            const int q = q0 + r;
            tile[r][lane] = (q < P) ? in[ix(pin_int[q], bs.Bp, b0 + lane)] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = placement
            const int b = b0 + r, q = q0 + lane;
            if (q < P && b < bs.B) out[(size_t)b * P + q] = tile[lane][r];
        }
        __syncthreads();
    }
}

// out[b][q][k] = in[(int(q) * k + c) * Bp + b] for b < B, k components
__global__ void __launch_bounds__(kBlock) k_bout(BatchState bs, const int32_t* __restrict__ pin_int, int P,
                                                 const float* __restrict__ in, int K, float* __restrict__ out) {
    __shared__ float tile[32][33];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b0 = blockIdx.y * 32;
    for (int q0 = blockIdx.x * 32; q0 < P; q0 += gridDim.x * 32) {
        for (int c = 0; c < K; ++c) {
            for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = pin
                const int q = q0 + r, b = b0 + lane;
                tile[r][lane] = (q < P) ? in[ix(pin_int[q] * K + c, bs.Bp, b)] : 0.f;
            }
            __syncthreads();
            for (int r = w; r < 32; r += kWarpsPerBlock) {  // row = placement
                const int b = b0 + r, q = q0 + lane;
                if (q < P && b < bs.B) out[((size_t)b * P + q) * K + c] = tile[lane][r];
            }
            __syncthreads();
        }
    }
}

// per-pin slack (early, late): min over rise/fall, into internal scratch [P][2][Bp]
__global__ void __launch_bounds__(kBlock) k_bpin_slack(BatchState bs, int P, float* __restrict__ out) {
    const long long n = (long long)P * bs.Bp;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock) {
        const int p = (int)(i / bs.Bp), b = (int)(i - (long long)p * bs.Bp);
        float a[4], r[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            a[c] = bs.at[ix(4 * p + c, bs.Bp, b)];
            r[c] = bs.rat[ix(4 * p + c, bs.Bp, b)];
        }
        out[ix(2 * p, bs.Bp, b)] = fminf(a[0] - r[0], a[1] - r[1]);
        out[ix(2 * p + 1, bs.Bp, b)] = fminf(r[2] - a[2], r[3] - a[3]);
    }
}

// endpoint slacks [E][Bp] (float2) -> out[b][e][2]
__global__ void __launch_bounds__(kBlock) k_bep_out(BatchState bs, int E, float2* __restrict__ out) {
    const long long n = (long long)E * bs.B;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock) {
        const int b = (int)(i / E), e = (int)(i - (long long)b * E);
        out[i] = bs.ep_slack[ix(e, bs.Bp, b)];
    }
}

// constant state of every placement: dst[row][b] = src[row] (asserted values,
// required-time seeds); the LSE arrival starts as the late arrival
__global__ void __launch_bounds__(kBlock) k_bbroadcast(float* __restrict__ dst, const float* __restrict__ src,
                                                       long long rows, int Bp) {
    const long long n = rows * Bp;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock)
        dst[i] = src[i / Bp];
}

__global__ void __launch_bounds__(kBlock) k_binit_ats(BatchState bs, int P) {
    const long long n = (long long)P * bs.Bp;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock) {
        const int p = (int)(i / bs.Bp), b = (int)(i - (long long)p * bs.Bp);
        bs.ats[ix(2 * p, bs.Bp, b)] = bs.at[ix(4 * p + 2, bs.Bp, b)];
        bs.ats[ix(2 * p + 1, bs.Bp, b)] = bs.at[ix(4 * p + 3, bs.Bp, b)];
    }
}


// Before a batched dataflow sweep: the words its tasks poll are set to
// kUnwritten for every placement.  Forward: arrival / slew / LSE-arrival words
// of the cell-input pins the sweep writes.  Backward: required times (mode 1)
// and adjoints (mode 2) of cell-input pins, and the large nets' partial records.
__global__ void __launch_bounds__(kBlock) k_breset(BatchState bs, const uint8_t* __restrict__ keep,
                                                   const int32_t* __restrict__ pin_cons, int P, int what,
                                                   float* part, long long part_words) {
    const float u = __uint_as_float(kUnwritten);
    const int Bp = bs.Bp;
    const long long n = (long long)P * Bp;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < part_words; i += (long long)gridDim.x * kBlock)
        part[i] = u;
    for (long long i = (long long)blockIdx.x * kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock) {
        const int p = (int)(i / Bp), b = (int)(i - (long long)p * Bp);
        if (pin_cons[p] < 0) continue;
        if (what == 0) {  // forward
            if (keep[p]) continue;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                bs.at[ix(4 * p + c, Bp, b)] = u;
                bs.slew[ix(4 * p + c, Bp, b)] = u;
            }
            bs.ats[ix(2 * p, Bp, b)] = u;
            bs.ats[ix(2 * p + 1, Bp, b)] = u;
        } else {
            if (what & 1) {
#pragma unroll
                for (int c = 0; c < 4; ++c) bs.rat[ix(4 * p + c, Bp, b)] = u;
            }
            if (what & 2) {
                bs.g_ats[ix(2 * p, Bp, b)] = u;
                bs.g_ats[ix(2 * p + 1, Bp, b)] = u;
                bs.g_slew[ix(2 * p, Bp, b)] = u;
                bs.g_slew[ix(2 * p + 1, Bp, b)] = u;
            }
        }
    }
}

int bgrid(long long n) {
    long long b = (n + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

int pin_tiles(int P) {
    const int t = (P + 31) / 32;
    return t < 152 * 8 ? (t > 0 ? t : 1) : 152 * 8;
}

}  // namespace

int batch_max_blocks(int fwd) {
    int dev = 0, sms = 0, a = 0, b = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (fwd) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bfwd<true>, kBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bfwd<false>, kBlock, 0);
        c = a;
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bbwd<1>, kBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bbwd<2>, kBlock, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_bbwd<3>, kBlock, 0);
    }
    const int per_sm = std::min(a, std::min(b, c));
    return sms * (per_sm > 0 ? per_sm : 1);
}

void launch_batch_load(const DevNet& g, const BatchState& bs, const BigChunks& c, cudaStream_t st) {
    if (c.n == 0) return;
    k_bload<<<dim3(c.n, bs.G), kBlock, 0, st>>>(g, bs, c.rec, c.part, c.cnt);
}

std::vector<int32_t> big_chunk_list(const std::vector<int32_t>& big_nets, const std::vector<int32_t>& net_ptr) {
    std::vector<int32_t> rec;
    for (int32_t n : big_nets) {
        const int32_t dp = net_ptr[n], ns = net_ptr[n + 1] - dp - 1;
        const int32_t nch = (ns + kLoadChunk - 1) / kLoadChunk, first = (int32_t)(rec.size() / 4);
        for (int32_t k = 0; k < nch; ++k) {
            const int32_t cnt = std::min(kLoadChunk, ns - k * kLoadChunk);
            rec.insert(rec.end(), {n, dp + 1 + k * kLoadChunk, first, cnt | (nch << 16)});
        }
    }
    return rec;
}

void launch_batch_fwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int lse,
                      int stall_task, cudaStream_t st) {
    if (d.TF == 0) return;
    if (lse) launch_coop(k_bfwd<true>, grid, kBlock, 0, st, g, bs, d, gamma, stall_task);
    else launch_coop(k_bfwd<false>, grid, kBlock, 0, st, g, bs, d, gamma, stall_task);
}

void launch_batch_load_small(const DevNet& g, const BatchState& bs, int big, cudaStream_t st) {
    const long long nw = (long long)g.N * bs.G;
    if (nw == 0) return;
    k_bload_small<<<bgrid(nw * 32), kBlock, 0, st>>>(g, bs, big);
}

void launch_batch_fwd_level(const DevNet& g, const BatchState& bs, const DfState& d, int t0, int t1, float gamma,
                            int lse, cudaStream_t st) {
    const long long nw = (long long)(t1 - t0) * bs.GT;
    if (nw <= 0) return;
    const int grid = (int)((nw + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (lse) k_bfwd_lvl<true><<<grid, kBlock, 0, st>>>(g, bs, d, t0, t1, gamma);
    else k_bfwd_lvl<false><<<grid, kBlock, 0, st>>>(g, bs, d, t0, t1, gamma);
}

void launch_batch_bwd_level(const DevNet& g, const BatchState& bs, const DfState& d, const int* r6, float gamma,
                            int mode, cudaStream_t st) {
    Ranges r{r6[0], r6[1], r6[2], r6[3], r6[4], r6[5]};
    const long long nw = (long long)((r.a1 - r.a0) + (r.b1 - r.b0) + (r.c1 - r.c0)) * bs.GT;
    if (nw <= 0) return;
    const int grid = (int)((nw + kWarpsPerBlock - 1) / kWarpsPerBlock);
    if (mode == 1) k_bbwd_lvl<1><<<grid, kBlock, 0, st>>>(g, bs, d, r, gamma);
    else if (mode == 2) k_bbwd_lvl<2><<<grid, kBlock, 0, st>>>(g, bs, d, r, gamma);
    else k_bbwd_lvl<3><<<grid, kBlock, 0, st>>>(g, bs, d, r, gamma);
}

void launch_batch_cap_seed(const DevNet& g, const BatchState& bs, float gamma, cudaStream_t st) {
    if (g.E == 0 || !g.ep_clk) return;
    k_bcap_seed<<<dim3((g.E + kWarpsPerBlock - 1) / kWarpsPerBlock, bs.G), kBlock, 0, st>>>(g, bs, gamma);
}

void launch_batch_endpoints(const DevNet& g, const BatchState& bs, float gamma, int lse, cudaStream_t st) {
    k_bep1<<<dim3(kRedBlocks, bs.G), kBlock, 0, st>>>(g, bs, gamma, lse);
    k_bep2<<<(bs.Bp * 32 + 127) / 128, 128, 0, st>>>(g, bs, gamma, lse, kRedBlocks);
}

void launch_batch_reset(const BatchState& bs, const DfState& d, int P, int what, cudaStream_t st) {
    const long long pw = what == 0 ? 0 : (long long)d.npart * kPartFloats * bs.Bp;
    float* part = (what & 2) ? bs.part : bs.rpart;
    if ((long long)P * bs.Bp + pw == 0) return;
    k_breset<<<bgrid((long long)P * bs.Bp), kBlock, 0, st>>>(bs, d.pin_keep, d.pin_cons, P, what, part, pw);
}

void launch_batch_bwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int mode,
                      cudaStream_t st) {
    if (d.TB == 0) return;
    if (mode == 1) launch_coop(k_bbwd<1>, grid, kBlock, 0, st, g, bs, d, gamma);
    else if (mode == 2) launch_coop(k_bbwd<2>, grid, kBlock, 0, st, g, bs, d, gamma);
    else launch_coop(k_bbwd<3>, grid, kBlock, 0, st, g, bs, d, gamma);
}

void launch_batch_xy_in(const BatchState& bs, const int32_t* pin_int, int P, const float2* xy_user, cudaStream_t st) {
    if (P == 0) return;
    k_bxy_in<<<dim3(pin_tiles(P), bs.G), kBlock, 0, st>>>(bs, pin_int, P, xy_user);
}

void launch_batch_out(const BatchState& bs, const int32_t* pin_int, int P, const float* in, int K, float* out,
                      cudaStream_t st) {
    if (P == 0) return;
    k_bout<<<dim3(pin_tiles(P), bs.G), kBlock, 0, st>>>(bs, pin_int, P, in, K, out);
}

void launch_batch_out2(const BatchState& bs, const int32_t* pin_int, int P, const float2* in, float2* out,
                       cudaStream_t st) {
    if (P == 0) return;
    k_bout2<<<dim3(pin_tiles(P), bs.G), kBlock, 0, st>>>(bs, pin_int, P, in, out);
}

void launch_batch_pin_slack(const BatchState& bs, int P, float* scratch, cudaStream_t st) {
    if (P == 0) return;
    k_bpin_slack<<<bgrid((long long)P * bs.Bp), kBlock, 0, st>>>(bs, P, scratch);
}

void launch_batch_ep_out(const BatchState& bs, int E, float2* out, cudaStream_t st) {
    if (E == 0) return;
    k_bep_out<<<bgrid((long long)E * bs.B), kBlock, 0, st>>>(bs, E, out);
}

void launch_batch_broadcast(float* dst, const float* src, long long rows, int Bp, cudaStream_t st) {
    if (rows == 0) return;
    k_bbroadcast<<<bgrid(rows * Bp), kBlock, 0, st>>>(dst, src, rows, Bp);
}

void launch_batch_init_ats(const BatchState& bs, int P, cudaStream_t st) {
    if (P == 0) return;
    k_binit_ats<<<bgrid((long long)P * bs.Bp), kBlock, 0, st>>>(bs, P);
}

}  // namespace sta
