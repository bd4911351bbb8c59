// batch.cu -- many placements of one netlist in one sweep.
//
// Every placement runs the same timing graph, so the batched schedule maps
// LANES TO PLACEMENTS: a warp takes one task (a net, or a chunk of a large
// net's sinks) for 32 placements at once and each lane runs the scalar
// per-net algorithm for its placement.  All lanes follow the same control
// flow (the topology is shared), there are no shuffles or segmented scans,
// and every per-pin access is one coalesced 128-byte row: per-placement state
// is stored pin-major, placement-minor, value[(pin * k + component) * Bp + b]
// with Bp = the batch rounded up to a multiple of 32.  Topology, capacitances
// and tables are read once per warp for 32 placements.
//
// The sweeps are the dependency-driven persistent kernels of the
// single-placement schedule with queue index q = task * G + group (G = Bp / 32
// placement groups): task t of group g waits only for its producers in group
// g, whose queue indices are smaller.  Every placement's arithmetic is the
// same whatever the batch size or its position in the batch, so a placement's
// results are bit-identical alone and in a batch.
#include <algorithm>

#include "dataflow_sync.cuh"
#include "device_common.cuh"

namespace sta {
namespace {

__device__ __forceinline__ size_t ix(int row, int Bp, int b) { return (size_t)row * Bp + b; }

// ---------------------------------------------------------------------------
// Wire step of one sink (Eqs. 1-3 on a star) -- same arithmetic as the
// single-placement kernels.
// ---------------------------------------------------------------------------
struct Wire {
    float D, I, dist;  // Elmore delay, impulse, Manhattan distance
};

__device__ __forceinline__ Wire wire(const DevNet& g, float2 xy, float2 xyd, float cap) {
    Wire w;
    w.dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
    const float R = g.r * w.dist;
    const float C = fmaf(0.5f * g.c, w.dist, cap);
    w.D = R * C * kKrc;
    const float m = 2.f * R * C * w.D * kKrc - w.D * w.D;
    w.I = sqrtf(fmaxf(m, 0.f));
    return w;
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

// Static description of a driver cell (the same for every lane).
struct CellDesc {
    int t, a0, na, un;
    int pin[STA_MAX_ARCS];
};

__device__ __forceinline__ CellDesc cell_desc(const DevNet& g, int n) {
    CellDesc c;
    c.t = g.net_drv[n];
    c.a0 = g.net_arc_ptr[n];
    c.na = c.t >= 0 ? g.net_arc_ptr[n + 1] - c.a0 : 0;
    c.un = c.t >= 0 ? g.lib_unate[c.t] : 0;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) c.pin[k] = k < c.na ? g.arc_pin[c.a0 + k] : 0;
    return c;
}

__device__ __forceinline__ void load_seg(const DevNet& g, int t, float ld, int& jl, float& ul, float& inv_l) {
    const float* li = g.lib_idx + t * kLibStride + 8;
    jl = axis_seg(li, ld);
    inv_l = __ldg(g.lib_inv + t * kLibStride + 8 + jl);
    ul = (ld - __ldg(li + jl)) * inv_l;
}

__device__ __forceinline__ void slew_seg_g(const DevNet& g, int t, float v, int& is, float& ts, float& inv_s) {
    const float* si = g.lib_idx + t * kLibStride;
    is = axis_seg(si, v);
    inv_s = __ldg(g.lib_inv + t * kLibStride + is);
    ts = (v - __ldg(si + is)) * inv_s;
}

// Driver-cell results of one placement for the four conditions (late max /
// early min over the arcs, worst slew, LSE arrival of Eq. 4 for the late ones).
struct CellOut {
    float at[4], sl[4], z[2];
};

__device__ __forceinline__ CellOut eval_cell(const DevNet& g, const BatchState& bs, const CellDesc& cd, int dp,
                                             int b, float ld, float gamma, bool lse) {
    const int Bp = bs.Bp;
    CellOut o;
    if (cd.t < 0) {  // asserted driver: constant values set at creation
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            o.at[c] = bs.at[ix(4 * dp + c, Bp, b)];
            o.sl[c] = bs.slew[ix(4 * dp + c, Bp, b)];
        }
        o.z[0] = bs.ats[ix(2 * dp, Bp, b)];
        o.z[1] = bs.ats[ix(2 * dp + 1, Bp, b)];
        return o;
    }
    int jl;
    float ul, inv_l;
    load_seg(g, cd.t, ld, jl, ul, inv_l);
    o.at[0] = o.at[1] = o.sl[0] = o.sl[1] = kInf;
    o.at[2] = o.at[3] = o.sl[2] = o.sl[3] = -kInf;
    float cand[2][STA_MAX_ARCS], m[2] = {-kInf, -kInf};
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < cd.na) {
            const int pin = cd.pin[k];
            float ain[4], sin[4], zin[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                ain[q] = __ldcg(bs.at + ix(4 * pin + q, Bp, b));
                sin[q] = __ldcg(bs.slew + ix(4 * pin + q, Bp, b));
            }
            zin[0] = lse ? __ldcg(bs.ats + ix(2 * pin, Bp, b)) : 0.f;
            zin[1] = lse ? __ldcg(bs.ats + ix(2 * pin + 1, Bp, b)) : 0.f;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int el = c >> 1, rf = c & 1;
                const int rfi = rf ^ ((cd.un >> k) & 1);
                // selects, not a runtime index: the arrays stay in registers
                const float s_in = rfi ? sin[2 * el + 1] : sin[2 * el];
                const float a_in = rfi ? ain[2 * el + 1] : ain[2 * el];
                int is;
                float ts, inv_s;
                slew_seg_g(g, cd.t, s_in, is, ts, inv_s);
                float4 dq, sq;
                cell_corners(g, cd.t, k, rf, is, jl, dq, sq);
                const float D = lerp_cell(dq, ts, ul);
                const float S = lerp_cell(sq, ts, ul);
                const float v = a_in + D;
                if (el) {
                    o.at[c] = fmaxf(o.at[c], v);
                    o.sl[c] = fmaxf(o.sl[c], S);
                    cand[rf][k] = (rfi ? zin[1] : zin[0]) + D;
                    m[rf] = fmaxf(m[rf], cand[rf][k]);
                } else {
                    o.at[c] = fminf(o.at[c], v);
                    o.sl[c] = fminf(o.sl[c], S);
                }
            }
        }
    }
    o.z[0] = o.z[1] = 0.f;
    if (lse) {
#pragma unroll
        for (int rf = 0; rf < 2; ++rf) {
            float sum = 0.f;
#pragma unroll
            for (int k = 0; k < STA_MAX_ARCS; ++k)
                if (k < cd.na) sum += expf((cand[rf][k] - m[rf]) / gamma);
            o.z[rf] = m[rf] + gamma * logf(sum);
        }
    }
    return o;
}

__device__ __forceinline__ void store_driver(const BatchState& bs, int dp, int b, const CellOut& o, bool lse) {
    const int Bp = bs.Bp;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        bs.at[ix(4 * dp + c, Bp, b)] = o.at[c];
        bs.slew[ix(4 * dp + c, Bp, b)] = o.sl[c];
    }
    if (lse) {
        bs.ats[ix(2 * dp, Bp, b)] = o.z[0];
        bs.ats[ix(2 * dp + 1, Bp, b)] = o.z[1];
    }
}

// wire step to the sinks [s0, s1) of a net with driver values o
__device__ __forceinline__ void store_sinks(const DevNet& g, const BatchState& bs, int s0, int s1, int b, float2 xyd,
                                            const CellOut& o, bool lse) {
    const int Bp = bs.Bp;
#pragma unroll 2
    for (int p = s0; p < s1; ++p) {
        const Wire w = wire(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p));
        const float i2 = w.I * w.I;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            bs.at[ix(4 * p + c, Bp, b)] = o.at[c] + w.D;
            bs.slew[ix(4 * p + c, Bp, b)] = sqrtf(fmaf(o.sl[c], o.sl[c], i2));
        }
        if (lse) {
            bs.ats[ix(2 * p, Bp, b)] = o.z[0] + w.D;
            bs.ats[ix(2 * p + 1, Bp, b)] = o.z[1] + w.D;
        }
    }
}

// net load (Eq. 1): the driver's pin capacitance, then every sink in order
__device__ __forceinline__ float net_load(const DevNet& g, const BatchState& bs, int dp, int s1, int b, float2 xyd) {
    float ld = __ldg(g.pin_cap + dp);
#pragma unroll 4
    for (int p = dp + 1; p < s1; ++p) {
        const float2 xy = bs.xy[ix(p, bs.Bp, b)];
        const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
        ld += fmaf(g.c, dist, __ldg(g.pin_cap + p));
    }
    return ld;
}

template <bool lse>
__device__ void bfwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int q, int n0, int nn, int b,
                          float gamma) {
    const int Bp = bs.Bp;
    // before the wait: the first net's load (static) and its cell description
    const int dp0 = g.net_ptr[n0], e0 = g.net_ptr[n0 + 1];
    const float2 xyd0 = bs.xy[ix(dp0, Bp, b)];
    const float ld0 = net_load(g, bs, dp0, e0, b, xyd0);
    const CellDesc cd0 = cell_desc(g, n0);
    bs.load[ix(n0, Bp, b)] = ld0;

    wait_ready(d.fcnt, q, d.f_indeg[q / bs.G], d.abort_word);

    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = j ? g.net_ptr[n] : dp0, e = j ? g.net_ptr[n + 1] : e0;
        const float2 xyd = j ? bs.xy[ix(dp, Bp, b)] : xyd0;
        float ld = ld0;
        CellDesc cd = cd0;
        if (j) {
            ld = net_load(g, bs, dp, e, b, xyd);
            bs.load[ix(n, Bp, b)] = ld;
            cd = cell_desc(g, n);
        }
        const CellOut o = eval_cell(g, bs, cd, dp, b, ld, gamma, lse);
        if (cd.t >= 0) store_driver(bs, dp, b, o, lse);
        store_sinks(g, bs, dp + 1, e, b, xyd, o, lse);
    }
}

// chunk of a large net: its load comes from the prologue; every chunk
// evaluates the driver cell, the first one stores it
template <bool lse>
__device__ void bfwd_chunk(const DevNet& g, const BatchState& bs, const DfState& d, int q, int n, int p0, int cnt,
                           int b, float gamma) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float ld = bs.load[ix(n, Bp, b)];
    const CellDesc cd = cell_desc(g, n);

    wait_ready(d.fcnt, q, d.f_indeg[q / bs.G], d.abort_word);

    const CellOut o = eval_cell(g, bs, cd, dp, b, ld, gamma, lse);
    if (cd.t >= 0 && p0 == dp + 1) store_driver(bs, dp, b, o, lse);
    store_sinks(g, bs, p0, p0 + cnt, b, xyd, o, lse);
}

template <bool lse>
__global__ void __launch_bounds__(kBlock) k_bfwd(DevNet g, BatchState bs, DfState d, float gamma) {
    const int lane = threadIdx.x & 31;
    const int Q = d.TF * bs.G;
    int q = grab(d.heads + 0);
    while (q < Q) {
        const int next = grab(d.heads + 0);
        const int t = q / bs.G, b = (q - t * bs.G) * 32 + lane;
        const int4 task = d.ftask[t];
        if (task.y > 0) bfwd_nets<lse>(g, bs, d, q, task.x, task.y, b, gamma);
        else bfwd_chunk<lse>(g, bs, d, q, task.x, task.z, task.w, b, gamma);
        // consumers of (t, group) are (u, group): counter u * G + group
        __syncwarp();
        const int k1 = d.f_out_ptr[t + 1], gq = q - t * bs.G;
        for (int k = d.f_out_ptr[t] + lane; k < k1; k += 32) red_release_add(d.fcnt + d.f_out[k] * bs.G + gq, 1);
        q = next;
    }
}

// Loads of the large nets (the chunk tasks read them): a block per (net,
// placement group); warp w sums sinks w, w + 8, ... and the warps' sums are
// added in warp order, so the result is fixed.
__global__ void __launch_bounds__(kBlock) k_bload(DevNet g, BatchState bs, const int32_t* __restrict__ nets) {
    __shared__ float sh[kWarpsPerBlock][32];
    const int n = nets[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane, Bp = bs.Bp;
    const int dp = g.net_ptr[n], e = g.net_ptr[n + 1];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    float acc = 0.f;
#pragma unroll 4
    for (int p = dp + 1 + w; p < e; p += kWarpsPerBlock) {
        const float2 xy = bs.xy[ix(p, Bp, b)];
        const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
        acc += fmaf(g.c, dist, __ldg(g.pin_cap + p));
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        float ld = __ldg(g.pin_cap + dp);
#pragma unroll
        for (int k = 0; k < kWarpsPerBlock; ++k) ld += sh[k][lane];
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

// grid (kRedBlocks, G): block x takes endpoints x*8 + w, stepping by
// kRedBlocks*8; partial per (block, placement)
__global__ void __launch_bounds__(kBlock) k_bep1(DevNet g, BatchState bs, float gamma, int lse) {
    __shared__ BEp sh[kWarpsPerBlock][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int b = blockIdx.y * 32 + lane, Bp = bs.Bp;
    BEp acc = bep_identity();
    for (int e = blockIdx.x * kWarpsPerBlock + w; e < g.E; e += gridDim.x * kWarpsPerBlock) {
        const int p = g.ep_pin[e];
        const float4 con = reinterpret_cast<const float4*>(g.ep_rat)[e];
        const float a0 = bs.at[ix(4 * p, Bp, b)], a1 = bs.at[ix(4 * p + 1, Bp, b)];
        const float a2 = bs.at[ix(4 * p + 2, Bp, b)], a3 = bs.at[ix(4 * p + 3, Bp, b)];
        const float se = fminf(a0 - con.x, a1 - con.y);
        const float sl = fminf(con.z - a2, con.w - a3);
        bs.ep_slack[ix(e, Bp, b)] = make_float2(se, sl);
        BEp v = bep_identity();
        v.wns_e = se;
        v.wns_l = sl;
        v.tns_e = fminf(se, 0.f);
        v.tns_l = fminf(sl, 0.f);
        v.viol = sl < 0.f ? 1.0 : 0.0;
        if (lse) {
            const float sr = con.z - bs.ats[ix(2 * p, Bp, b)], sf = con.w - bs.ats[ix(2 * p + 1, Bp, b)];
            v.tns_g = softmin3(sr, sf, gamma);
            v.wmin = fminf(sr, sf);
            v.wsum = expf(-(sr - v.wmin) / gamma) + expf(-(sf - v.wmin) / gamma);
        }
        bep_merge(acc, v, gamma);
    }
    sh[w][lane] = acc;
    __syncthreads();
    if (w == 0) {
        for (int k = 1; k < kWarpsPerBlock; ++k) bep_merge(acc, sh[k][lane], gamma);
        reinterpret_cast<BEp*>(bs.red)[ix(blockIdx.x, Bp, b)] = acc;
    }
}

// thread per placement: the partials in block order
__global__ void k_bep2(DevNet g, BatchState bs, float gamma, int lse, int nparts) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= bs.Bp) return;
    BEp acc = bep_identity();
    for (int k = 0; k < nparts; ++k) bep_merge(acc, reinterpret_cast<const BEp*>(bs.red)[ix(k, bs.Bp, b)], gamma);
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
// Backward (mode 1 required times, 2 adjoint, 3 both)
// ---------------------------------------------------------------------------
struct BSeed {
    float W, wt, ww;  // WNS_gamma of this placement, w_tns, w_wns
};

// What one placement's driver cell contributes to the backward sweep, all from
// forward results: arc delays (required times) and, per late output transition
// rf, the LSE weights, the delay partials, and the arc of the late slew (first
// one on ties) with its slew partials.
struct BCell {
    float adel[STA_MAX_ARCS][4];
    float w[2][STA_MAX_ARCS], dDs[2][STA_MAX_ARCS], dDl[2][STA_MAX_ARCS];
    int amax[2];
    float dSs[2], dSl[2];
};

template <int mode>
__device__ __forceinline__ void bcell_pre(const DevNet& g, const BatchState& bs, const CellDesc& cd, int n, int dp,
                                          int b, float gamma, BCell& bc) {
    const int Bp = bs.Bp;
#pragma unroll
    for (int rf = 0; rf < 2; ++rf) {
        bc.amax[rf] = -1;
        bc.dSs[rf] = bc.dSl[rf] = 0.f;
#pragma unroll
        for (int k = 0; k < STA_MAX_ARCS; ++k) bc.w[rf][k] = bc.dDs[rf][k] = bc.dDl[rf][k] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
#pragma unroll
        for (int c = 0; c < 4; ++c) bc.adel[k][c] = 0.f;
    if (cd.t < 0) return;
    const float ld = bs.load[ix(n, Bp, b)];
    int jl;
    float ul, inv_l;
    load_seg(g, cd.t, ld, jl, ul, inv_l);
    const float zd0 = (mode & 2) ? bs.ats[ix(2 * dp, Bp, b)] : 0.f;
    const float zd1 = (mode & 2) ? bs.ats[ix(2 * dp + 1, Bp, b)] : 0.f;
    float best[2] = {-kInf, -kInf};
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < cd.na) {
            const int pin = cd.pin[k];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int el = c >> 1, rf = c & 1;
                if (!(mode & 1) && !el) continue;
                const int rfi = rf ^ ((cd.un >> k) & 1);
                const float sin = bs.slew[ix(4 * pin + 2 * el + rfi, Bp, b)];
                int is;
                float ts, inv_s;
                slew_seg_g(g, cd.t, sin, is, ts, inv_s);
                float4 dq, sq;
                cell_corners(g, cd.t, k, rf, is, jl, dq, sq);
                float dDs, dDl, dSs, dSl;
                const float D = lerp_cell_grad(dq, ts, ul, inv_s, inv_l, dDs, dDl);
                bc.adel[k][c] = D;
                if ((mode & 2) && el) {
                    const float S = lerp_cell_grad(sq, ts, ul, inv_s, inv_l, dSs, dSl);
                    bc.dDs[rf][k] = dDs;
                    bc.dDl[rf][k] = dDl;
                    bc.w[rf][k] = expf((bs.ats[ix(2 * pin + rfi, Bp, b)] + D - (rf ? zd1 : zd0)) / gamma);
                    if (S > best[rf]) {
                        best[rf] = S;
                        bc.amax[rf] = k;
                        bc.dSs[rf] = dSs;
                        bc.dSl[rf] = dSl;
                    }
                }
            }
        }
    }
}

// Required times of the cell's inputs and the adjoint through the LSE, the
// NLDM partials and the late-slew max; returns d loss / d load.
template <int mode>
__device__ __forceinline__ float bcell_apply(const BatchState& bs, const CellDesc& cd, const BCell& bc, int b,
                                             const float* R, const float* GA, const float* GS) {
    const int Bp = bs.Bp;
    float gl = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < cd.na) {
            const int pin = cd.pin[k];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int el = c >> 1, rf = c & 1;
                const int rfi = rf ^ ((cd.un >> k) & 1);
                if (mode & 1) bs.rat[ix(4 * pin + 2 * el + rfi, Bp, b)] = R[c] - bc.adel[k][c];
                if ((mode & 2) && el) {
                    const float gD = GA[rf] * bc.w[rf][k];
                    bs.g_ats[ix(2 * pin + rfi, Bp, b)] = gD;
                    bs.g_slew[ix(2 * pin + rfi, Bp, b)] = fmaf(gD, bc.dDs[rf][k], k == bc.amax[rf] ? GS[rf] * bc.dSs[rf] : 0.f);
                    gl = fmaf(gD, bc.dDl[rf][k], gl);
                }
            }
        }
    }
    if (mode & 2) {
#pragma unroll
        for (int rf = 0; rf < 2; ++rf)
            if (bc.amax[rf] >= 0) gl = fmaf(GS[rf], bc.dSl[rf], gl);
    }
    return gl;
}

// One sink's terms of the backward reductions.  Cell-input sinks read their
// required times / adjoints (written by their cell's task; through L2);
// endpoints and dangling sinks are constant: the constraint (or +-inf) and the
// adjoint seed d loss / d LSE-AT = -(w_tns dTNS_g/ds + w_wns dWNS_g/ds).
struct BSink {
    float r[4];    // RAT_s - Delay_s
    float ga[2];   // g_ats of the sink
    float gs[2];   // g_slew_s * slew_d / slew_s
    float gwire;   // d loss / d Delay_s + d loss / d Impulse_s
    Wire w;
};

template <int mode>
__device__ __forceinline__ BSink bsink(const DevNet& g, const BatchState& bs, const DfState& d, int p, int b,
                                       float2 xyd, const float* sld, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    BSink s;
    s.w = wire(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p));
    const bool dyn = d.pin_cons[p] >= 0;
    if (mode & 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) s.r[c] = __ldcg(bs.rat + ix(4 * p + c, Bp, b)) - s.w.D;
    }
    s.ga[0] = s.ga[1] = s.gs[0] = s.gs[1] = s.gwire = 0.f;
    if (mode & 2) {
        float ga0, ga1, gs0 = 0.f, gs1 = 0.f;
        if (dyn) {
            ga0 = __ldcg(bs.g_ats + ix(2 * p, Bp, b));
            ga1 = __ldcg(bs.g_ats + ix(2 * p + 1, Bp, b));
            gs0 = __ldcg(bs.g_slew + ix(2 * p, Bp, b));
            gs1 = __ldcg(bs.g_slew + ix(2 * p + 1, Bp, b));
        } else {
            ga0 = ga1 = 0.f;
            const float rr = bs.rat[ix(4 * p + 2, Bp, b)], rfl = bs.rat[ix(4 * p + 3, Bp, b)];
            if (isfinite(rr)) {
                const float sr = rr - bs.ats[ix(2 * p, Bp, b)], sf = rfl - bs.ats[ix(2 * p + 1, Bp, b)];
                const float te = softmin3(sr, sf, gamma);
                float gr = sd.wt * expf(-(sr - te) / gamma), gf = sd.wt * expf(-(sf - te) / gamma);
                if (isfinite(sd.W)) {
                    gr += sd.ww * expf(-(sr - sd.W) / gamma);
                    gf += sd.ww * expf(-(sf - sd.W) / gamma);
                }
                ga0 = -gr;
                ga1 = -gf;
            }
        }
        const float sl0 = bs.slew[ix(4 * p + 2, Bp, b)], sl1 = bs.slew[ix(4 * p + 3, Bp, b)];
        const float q0 = sl0 > 0.f ? gs0 / sl0 : 0.f;
        const float q1 = sl1 > 0.f ? gs1 / sl1 : 0.f;
        s.ga[0] = ga0;
        s.ga[1] = ga1;
        s.gs[0] = q0 * sld[0];
        s.gs[1] = q1 * sld[1];
        s.gwire = ga0 + ga1 + (q0 + q1) * s.w.I;
    }
    return s;
}

// d loss / d (x, y) of a sink from its wire adjoint and the net's d loss / d load
__device__ __forceinline__ float2 bsink_grad(const DevNet& g, float2 xy, float2 xyd, float cap, float gwire,
                                             float gload) {
    const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
    const float gd = fmaf(gload, g.c, gwire * kKrc * g.r * fmaf(g.c, fabsf(dx) + fabsf(dy), cap));
    return make_float2(gd * ((dx > 0.f) - (dx < 0.f)), gd * ((dy > 0.f) - (dy < 0.f)));
}

template <int mode>
__device__ void bbwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n0, int nn,
                          int b, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    const int dp0 = g.net_ptr[n0];
    const CellDesc cd0 = cell_desc(g, n0);
    BCell bc0;
    bcell_pre<mode>(g, bs, cd0, n0, dp0, b, gamma, bc0);

    wait_ready(cnt, q, d.b_indeg[q / bs.G], d.abort_word);

    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = j ? g.net_ptr[n] : dp0, e = g.net_ptr[n + 1];
        CellDesc cd = cd0;
        if (j) {
            cd = cell_desc(g, n);
            bcell_pre<mode>(g, bs, cd, n, dp, b, gamma, bc0);
        }
        const float2 xyd = bs.xy[ix(dp, Bp, b)];
        float sld[2] = {0.f, 0.f};
        if (mode & 2) {
            sld[0] = bs.slew[ix(4 * dp + 2, Bp, b)];
            sld[1] = bs.slew[ix(4 * dp + 3, Bp, b)];
        }
        float R[4] = {-kInf, -kInf, kInf, kInf}, GA[2] = {0.f, 0.f}, GS[2] = {0.f, 0.f};
        for (int p = dp + 1; p < e; ++p) {
            const BSink s = bsink<mode>(g, bs, d, p, b, xyd, sld, gamma, sd);
            if (mode & 1) {
                R[0] = fmaxf(R[0], s.r[0]);
                R[1] = fmaxf(R[1], s.r[1]);
                R[2] = fminf(R[2], s.r[2]);
                R[3] = fminf(R[3], s.r[3]);
            }
            if (mode & 2) {
                GA[0] += s.ga[0];
                GA[1] += s.ga[1];
                GS[0] += s.gs[0];
                GS[1] += s.gs[1];
                bs.grad[ix(p, Bp, b)].x = s.gwire;  // kept until d loss / d load is known
            }
        }
        if (mode & 1) {
#pragma unroll
            for (int c = 0; c < 4; ++c) bs.rat[ix(4 * dp + c, Bp, b)] = R[c];
        }
        const float gload = bcell_apply<mode>(bs, cd, bc0, b, R, GA, GS);
        if (mode & 2) {
            float sx = 0.f, sy = 0.f;
            for (int p = dp + 1; p < e; ++p) {
                const float gw = bs.grad[ix(p, Bp, b)].x;
                const float2 gxy = bsink_grad(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p), gw, gload);
                bs.grad[ix(p, Bp, b)] = gxy;
                sx += gxy.x;
                sy += gxy.y;
            }
            bs.grad[ix(dp, Bp, b)] = make_float2(-sx, -sy);
        }
    }
}

// Partial chunk of a large net: the 12 partial terms of the single-placement
// schedule over the chunk's sinks, per placement.
template <int mode>
__device__ void bbwd_part(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n, int p0,
                          int np, int slot, int b, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    float sld[2] = {0.f, 0.f};
    if (mode & 2) {
        sld[0] = bs.slew[ix(4 * dp + 2, Bp, b)];
        sld[1] = bs.slew[ix(4 * dp + 3, Bp, b)];
    }

    wait_ready(cnt, q, d.b_indeg[q / bs.G], d.abort_word);

    float v[kPartFloats];
    v[0] = v[1] = -kInf;
    v[2] = v[3] = kInf;
#pragma unroll
    for (int k = 4; k < kPartFloats; ++k) v[k] = 0.f;
    for (int p = p0; p < p0 + np; ++p) {
        const BSink s = bsink<mode>(g, bs, d, p, b, xyd, sld, gamma, sd);
        if (mode & 1) {
            v[0] = fmaxf(v[0], s.r[0]);
            v[1] = fmaxf(v[1], s.r[1]);
            v[2] = fminf(v[2], s.r[2]);
            v[3] = fminf(v[3], s.r[3]);
        }
        if (mode & 2) {
            v[4] += s.ga[0];
            v[5] += s.ga[1];
            v[6] += s.gs[0];
            v[7] += s.gs[1];
            const float2 xy = bs.xy[ix(p, Bp, b)];
            const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
            const float sx = (dx > 0.f) - (dx < 0.f), sy = (dy > 0.f) - (dy < 0.f);
            const float h = s.gwire * (kKrc * g.r * fmaf(g.c, s.w.dist, __ldg(g.pin_cap + p)));
            v[8] += sx;
            v[9] += sy;
            v[10] += sx * h;
            v[11] += sy * h;
        }
    }
    float* part = (mode & 2) ? bs.part : bs.rpart;
#pragma unroll
    for (int k = 0; k < kPartFloats; ++k) part[ix(slot * kPartFloats + k, Bp, b)] = v[k];
}

template <int mode>
__device__ void bbwd_driver(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n,
                            int slot0, int nch, int b, float gamma) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const CellDesc cd = cell_desc(g, n);
    BCell bc;
    bcell_pre<mode>(g, bs, cd, n, dp, b, gamma, bc);

    wait_ready(cnt, q, d.b_indeg[q / bs.G], d.abort_word);

    float v[kPartFloats];
    v[0] = v[1] = -kInf;
    v[2] = v[3] = kInf;
#pragma unroll
    for (int k = 4; k < kPartFloats; ++k) v[k] = 0.f;
    const float* part = (mode & 2) ? bs.part : bs.rpart;
    for (int k = 0; k < nch; ++k) {
        const int base = (slot0 + k) * kPartFloats;
        v[0] = fmaxf(v[0], __ldcg(part + ix(base + 0, Bp, b)));
        v[1] = fmaxf(v[1], __ldcg(part + ix(base + 1, Bp, b)));
        v[2] = fminf(v[2], __ldcg(part + ix(base + 2, Bp, b)));
        v[3] = fminf(v[3], __ldcg(part + ix(base + 3, Bp, b)));
#pragma unroll
        for (int j = 4; j < kPartFloats; ++j) v[j] += __ldcg(part + ix(base + j, Bp, b));
    }
    if (mode & 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) bs.rat[ix(4 * dp + c, Bp, b)] = v[c];
    }
    const float R[4] = {v[0], v[1], v[2], v[3]}, GA[2] = {v[4], v[5]}, GS[2] = {v[6], v[7]};
    const float gload = bcell_apply<mode>(bs, cd, bc, b, R, GA, GS);
    if (mode & 2) {
        bs.net_gload[ix(n, Bp, b)] = gload;
        bs.grad[ix(dp, Bp, b)] = make_float2(-fmaf(gload * g.c, v[8], v[10]), -fmaf(gload * g.c, v[9], v[11]));
    }
}

__device__ void bbwd_grad(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n, int p0,
                          int np, int b, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float sld[2] = {bs.slew[ix(4 * dp + 2, Bp, b)], bs.slew[ix(4 * dp + 3, Bp, b)]};
    wait_ready(cnt, q, d.b_indeg[q / bs.G], d.abort_word);
    const float gload = __ldcg(bs.net_gload + ix(n, Bp, b));
    for (int p = p0; p < p0 + np; ++p) {
        const BSink s = bsink<2>(g, bs, d, p, b, xyd, sld, gamma, sd);
        bs.grad[ix(p, Bp, b)] = bsink_grad(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p), s.gwire, gload);
    }
}

template <int mode>
__global__ void __launch_bounds__(kBlock) k_bbwd(DevNet g, BatchState bs, DfState d, float gamma) {
    const int lane = threadIdx.x & 31;
    int32_t* cnt = (mode & 2) ? d.acnt : d.rcnt;
    int32_t* head = d.heads + ((mode & 2) ? 2 : 1);
    const int Q = d.TB * bs.G;
    int q = grab(head);
    while (q < Q) {
        const int next = grab(head);
        const int t = q / bs.G, gq = q - t * bs.G, b = gq * 32 + lane;
        BSeed sd;
        sd.W = (float)bs.summary[(size_t)b * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
        sd.wt = bs.params[2 * b];
        sd.ww = bs.params[2 * b + 1];
        const int4 task = d.btask[t];
        if (task.y > 0) {
            bbwd_nets<mode>(g, bs, d, cnt, q, task.x, task.y, b, gamma, sd);
        } else if (task.y == -1) {
            bbwd_part<mode>(g, bs, d, cnt, q, task.x, task.z, task.w, d.baux[t], b, gamma, sd);
        } else if (task.y == -2) {
            bbwd_driver<mode>(g, bs, d, cnt, q, task.x, task.z, task.w, b, gamma);
        } else if (mode & 2) {
            bbwd_grad(g, bs, d, cnt, q, task.x, task.z, task.w, b, gamma, sd);
        }  // gradient chunks have no work in the required-time sweep
        __syncwarp();
        const int k1 = d.b_out_ptr[t + 1];
        for (int k = d.b_out_ptr[t] + lane; k < k1; k += 32) red_release_add(cnt + d.b_out[k] * bs.G + gq, 1);
        q = next;
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

void launch_batch_load(const DevNet& g, const BatchState& bs, const int32_t* big_nets, int nbig, cudaStream_t st) {
    if (nbig == 0) return;
    k_bload<<<dim3(nbig, bs.G), kBlock, 0, st>>>(g, bs, big_nets);
}

void launch_batch_fwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int lse,
                      cudaStream_t st) {
    if (d.TF == 0) return;
    if (lse) launch_coop(k_bfwd<true>, grid, kBlock, st, g, bs, d, gamma);
    else launch_coop(k_bfwd<false>, grid, kBlock, st, g, bs, d, gamma);
}

void launch_batch_endpoints(const DevNet& g, const BatchState& bs, float gamma, int lse, cudaStream_t st) {
    k_bep1<<<dim3(kRedBlocks, bs.G), kBlock, 0, st>>>(g, bs, gamma, lse);
    k_bep2<<<(bs.Bp + 127) / 128, 128, 0, st>>>(g, bs, gamma, lse, kRedBlocks);
}

void launch_batch_bwd(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int mode,
                      cudaStream_t st) {
    if (d.TB == 0) return;
    if (mode == 1) launch_coop(k_bbwd<1>, grid, kBlock, st, g, bs, d, gamma);
    else if (mode == 2) launch_coop(k_bbwd<2>, grid, kBlock, st, g, bs, d, gamma);
    else launch_coop(k_bbwd<3>, grid, kBlock, st, g, bs, d, gamma);
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
