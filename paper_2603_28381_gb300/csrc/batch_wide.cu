// batch_wide.cu -- the batched sweeps with a lane per placement.
//
// Same tasks, queue and polled data words as the batched dataflow sweeps of
// batch.cu, same per-placement layout value[row * Bp + b], but a warp takes a
// task for 32 placements and each lane runs all four timing conditions of its
// placement (early / late x rise / fall).  A warp task then carries four
// independent chains of memory round trips per lane instead of one, and its
// topology loads serve 32 placements instead of 8: the batched sweeps are
// bound by each warp's chain of dependent loads and by instruction issue, so
// this raises the memory parallelism per SM and issues fewer instructions per
// placement.  Queue index q = task * G + group (G = Bp / 32).  The per-arc
// terms live in a column of shared memory per lane, so the arc loops run
// rolled; loops unrolled over register arrays copied the cell's lookups for
// every arc and condition, and the kernels stalled on instruction fetch.
//
// Every value is computed with the same operations in the same order as in
// batch.cu: where the lanes of a quad exchanged values there (the net load's
// quad sum, the sink wire adjoints of the two late conditions, the quad sums
// of d loss / d load and of the driver's gradient), one lane now adds the same
// terms in the same association; with both files compiled without implicit
// multiply-add contraction the results are bit-identical to the narrow sweeps.
#include <algorithm>

#include "batch_common.cuh"

namespace sta {
namespace {

struct WLane {
    int lane, b;  // b = placement
};

__device__ __forceinline__ WLane wlane(int gw) {
    WLane L;
    L.lane = threadIdx.x & 31;
    L.b = gw * 32 + L.lane;
    return L;
}

// 128-thread blocks, 5 per SM: 20 warps per SM (with 256-thread blocks at 128
// registers 16 fitted; measured 5% slower)
constexpr int kWBlock = 128;

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

// The driver cell of net n: type, arcs, input pins, which arcs' input pins the
// sweep writes, unateness (bit k: arc k inverts), the type's slew axis and,
// once the load is known, the load's table segment and fraction.
struct WFCell {
    int t, na, dyn, un;
    int pin[STA_MAX_ARCS];
    int jl;
    float ul;
    float sidx[6], sinv[6];
};

__device__ __forceinline__ WFCell wfcell_topo(const DevNet& g, int n) {
    WFCell f;
    const int4 q0 = __ldg(g.net_desc + 2 * n), q1 = __ldg(g.net_desc + 2 * n + 1);  // one record
    f.t = q0.x;
    f.na = q0.z;
    f.dyn = q0.w & 15;
    f.un = q0.w >> 4;
    f.pin[0] = q1.x;
    f.pin[1] = q1.y;
    f.pin[2] = q1.z;
    f.pin[3] = q1.w;
    f.jl = 0;
    f.ul = 0.f;
#pragma unroll
    for (int j = 0; j < 6; ++j) f.sidx[j] = f.sinv[j] = 0.f;
    return f;
}

__device__ __forceinline__ void wfcell_lib(const DevNet& g, WFCell& f, float ld) {
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

// The fanin words of every arc for one placement: the input pin's four arrival
// and slew rows and its two LSE-arrival rows, all loaded together (polled:
// other warps of this sweep write them).  Returns whether every word written
// during the sweep holds its value.
struct WFIn {
    float a[STA_MAX_ARCS][4], s[STA_MAX_ARCS][4], z[STA_MAX_ARCS][2];
};

__device__ __forceinline__ bool wfcell_fanin(const BatchState& bs, const WFCell& f, int b, bool lse, bool stall,
                                             WFIn& in) {
    const int Bp = bs.Bp;
    bool ok = !stall;  // the test hook's stalled task never sees its inputs
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
#pragma unroll
        for (int j = 0; j < 4; ++j) in.a[k][j] = in.s[k][j] = 0.f;
        in.z[k][0] = in.z[k][1] = 0.f;
        if (f.t >= 0 && k < f.na) {
            bool w = true;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                in.a[k][j] = ld_poll(bs.at + ix(4 * f.pin[k] + j, Bp, b));
                in.s[k][j] = ld_poll(bs.slew + ix(4 * f.pin[k] + j, Bp, b));
                w &= written(in.a[k][j]) & written(in.s[k][j]);
            }
            if (lse) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    in.z[k][r] = ld_poll(bs.ats + ix(2 * f.pin[k] + r, Bp, b));
                    w &= written(in.z[k][r]);
                }
            }
            if ((f.dyn >> k) & 1) ok &= w;
        }
    }
    return ok;
}

// Word w of the lane's forward column: [w * kWBlock + threadIdx.x].  Per arc k:
// the input pin's four arrival rows and four slew rows (row 2 el + r: mode el,
// input transition r), its two LSE-arrival rows, and the LSE candidates of the
// two late output transitions.
struct WFArc {
    float* f;
    static constexpr int kAin = 0, kSin = 16, kZin = 32, kCand = 40, kWords = 48;
    __device__ __forceinline__ float& at(int w) const { return f[w * kWBlock + threadIdx.x]; }
};

__device__ __forceinline__ WFArc wfarc() {
    __shared__ float f[WFArc::kWords * kWBlock];
    WFArc a;
    a.f = f;
    return a;
}

// the wait's later rounds: the same words as wfcell_fanin, loaded straight
// into the column (no register copy of every word lives across the polls)
__device__ __forceinline__ bool wfcell_fanin_col(const BatchState& bs, const WFCell& f, int b, bool lse, bool stall,
                                                 const WFArc& A) {
    const int Bp = bs.Bp;
    bool ok = !stall;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (f.t >= 0 && k < f.na) {
            bool w = true;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const float a = ld_poll(bs.at + ix(4 * f.pin[k] + j, Bp, b));
                const float s = ld_poll(bs.slew + ix(4 * f.pin[k] + j, Bp, b));
                A.at(WFArc::kAin + 4 * k + j) = a;
                A.at(WFArc::kSin + 4 * k + j) = s;
                w &= written(a) & written(s);
            }
            if (lse) {
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const float z = ld_poll(bs.ats + ix(2 * f.pin[k] + r, Bp, b));
                    A.at(WFArc::kZin + 2 * k + r) = z;
                    w &= written(z);
                }
            }
            if ((f.dyn >> k) & 1) ok &= w;
        }
    }
    return ok;
}

// the first fanin round into the column (once the round's loads are back)
__device__ __forceinline__ void wfcell_to_col(const WFCell& f, const WFIn& in) {
    if (f.t < 0) return;
    const WFArc A = wfarc();
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < f.na) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                A.at(WFArc::kAin + 4 * k + j) = in.a[k][j];
                A.at(WFArc::kSin + 4 * k + j) = in.s[k][j];
            }
            A.at(WFArc::kZin + 2 * k) = in.z[k][0];
            A.at(WFArc::kZin + 2 * k + 1) = in.z[k][1];
        }
    }
}

struct WOut {
    float at[4], sl[4], z[2];  // by condition c = 2 el + rf; LSE arrival by rf (late)
};

// The driver cell for the four conditions of one placement (late max / early
// min over the arcs in arc order, worst slew, Eq. 4 for the late conditions),
// with the operations and order of batch.cu's fcell_eval, so the results are
// bit-identical.  `ok` is the first fanin round's result; in the dataflow sweep
// the wait repeats the round until every lane has all its words.  The arc loop
// runs rolled over the lane's shared-memory column (unrolled over register
// arrays, the cell's lookups would be copied for every arc and condition).
template <bool kPoll>
__device__ __forceinline__ WOut wfcell_eval(const DevNet& g, const BatchState& bs, const WFCell& f, int dp, int b,
                                            float gamma, bool lse, int32_t* abort_word, bool stall, bool ok) {
    const int Bp = bs.Bp;
    WOut o;
    if (f.t < 0) {  // asserted driver: constant values set at creation
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            o.at[c] = bs.at[ix(4 * dp + c, Bp, b)];
            o.sl[c] = bs.slew[ix(4 * dp + c, Bp, b)];
        }
        o.z[0] = lse ? bs.ats[ix(2 * dp, Bp, b)] : 0.f;
        o.z[1] = lse ? bs.ats[ix(2 * dp + 1, Bp, b)] : 0.f;
        return o;
    }
    const WFArc A = wfarc();
    if constexpr (kPoll) {
        if (!__all_sync(kFull, ok))
            poll_words([&]() { return wfcell_fanin_col(bs, f, b, lse, stall, A); }, abort_word);
    }
    float m[2] = {-kInf, -kInf};
#pragma unroll
    for (int c = 0; c < 4; ++c) o.at[c] = o.sl[c] = (c >> 1) ? -kInf : kInf;
#pragma unroll 1
    for (int k = 0; k < f.na; ++k) {
        const int u = (f.un >> k) & 1;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int el = c >> 1, rf = c & 1;
            const int row = 2 * el + (rf ^ u);  // the input transition of output transition rf
            int is;
            float ts;
            seg_reg(f.sidx, f.sinv, A.at(WFArc::kSin + 4 * k + row), is, ts);
            float4 dq, sq;
            cell_corners(g, f.t, k, rf, is, f.jl, dq, sq);
            const float D = lerp_cell(dq, ts, f.ul);
            const float S = lerp_cell(sq, ts, f.ul);
            const float v = A.at(WFArc::kAin + 4 * k + row) + D;
            o.at[c] = el ? fmaxf(o.at[c], v) : fminf(o.at[c], v);
            o.sl[c] = el ? fmaxf(o.sl[c], S) : fminf(o.sl[c], S);
            if (el) {
                const float cand = (lse ? A.at(WFArc::kZin + 2 * k + (rf ^ u)) : 0.f) + D;
                A.at(WFArc::kCand + 2 * k + rf) = cand;
                m[rf] = fmaxf(m[rf], cand);
            }
        }
    }
    // Eq. 4 over the arcs in arc order (lse_arcs' arithmetic: the terms of
    // absent arcs it adds are exact zeros)
    const float inv_g = 1.f / gamma;
#pragma unroll
    for (int rf = 0; rf < 2; ++rf) {
        o.z[rf] = 0.f;
        if (lse) {
            float sum = 0.f;
#pragma unroll 1
            for (int k = 0; k < f.na; ++k) sum += __expf((A.at(WFArc::kCand + 2 * k + rf) - m[rf]) * inv_g);
            o.z[rf] = m[rf] + gamma * __logf(f.na > 0 ? sum : 1.f);
        }
    }
    return o;
}

__device__ __forceinline__ void wstore_pin(const BatchState& bs, int p, int b, const float* at, const float* sl,
                                           const float* z, bool lse) {
    const int Bp = bs.Bp;  // strong stores: words that other tasks of the sweep poll
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        st_poll(bs.at + ix(4 * p + c, Bp, b), at[c]);
        st_poll(bs.slew + ix(4 * p + c, Bp, b), sl[c]);
    }
    if (lse) {
        st_poll(bs.ats + ix(2 * p, Bp, b), z[0]);
        st_poll(bs.ats + ix(2 * p + 1, Bp, b), z[1]);
    }
}

// wire step to the sinks [s0, s1), all four conditions; the positions and
// capacitances of two sinks are loaded before their stores
__device__ __forceinline__ void wstore_sinks(const DevNet& g, const BatchState& bs, int s0, int s1, int b, float2 xyd,
                                             const WOut& o, bool lse) {
#pragma unroll 1
    for (int p0 = s0; p0 < s1; p0 += 2) {
        float2 xy[2];
        float cap[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            const int p = min(p0 + u, s1 - 1);
            xy[u] = bs.xy[ix(p, bs.Bp, b)];
            cap[u] = __ldg(g.pin_cap + p);
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            if (p0 + u < s1) {
                const Wire w = wire(g, xy[u], xyd, cap[u]);
                float at[4], sl[4], z[2];
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    at[c] = o.at[c] + w.D;
                    sl[c] = sqrtf(fmaf(o.sl[c], o.sl[c], w.I * w.I));
                }
                z[0] = o.z[0] + w.D;
                z[1] = o.z[1] + w.D;
                wstore_pin(bs, p0 + u, b, at, sl, z, lse);
            }
        }
    }
}

// net load (Eq. 1): four interleaved partial sums over sinks c, c + 4, ...,
// added as (s0 + s1) + (s2 + s3), then the driver's pin capacitance (batch.cu's
// quad sum, in one lane); four sinks' loads per round
__device__ __forceinline__ float wnet_load(const DevNet& g, const BatchState& bs, int dp, int s1, int b, float2 xyd) {
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int p0 = dp + 1; p0 < s1; p0 += 4) {
        float2 xy[4];
        float cap[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int p = min(p0 + u, s1 - 1);
            xy[u] = bs.xy[ix(p, bs.Bp, b)];
            cap[u] = __ldg(g.pin_cap + p);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float dist = fabsf(xy[u].x - xyd.x) + fabsf(xy[u].y - xyd.y);
            if (p0 + u < s1) acc[u] += fmaf(g.c, dist, cap[u]);
        }
    }
    return __ldg(g.pin_cap + dp) + ((acc[0] + acc[1]) + (acc[2] + acc[3]));
}

// packed small nets; the first fanin round is issued as soon as the cell's
// record is known, before the net's load and the table segment
template <bool lse>
__device__ void wfwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int n0, int nn, int b,
                          float gamma, bool stall) {
    const int Bp = bs.Bp;
    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = g.net_ptr[n], e = g.net_ptr[n + 1];
        WFCell f = wfcell_topo(g, n);
        WFIn in;
        const bool ok = wfcell_fanin(bs, f, b, lse, stall, in);
        const float2 xyd = bs.xy[ix(dp, Bp, b)];
        const float ld = wnet_load(g, bs, dp, e, b, xyd);
        bs.load[ix(n, Bp, b)] = ld;
        wfcell_to_col(f, in);
        wfcell_lib(g, f, ld);
        const WOut o = wfcell_eval<true>(g, bs, f, dp, b, gamma, lse, d.abort_word, stall, ok);
        if (f.t >= 0) wstore_pin(bs, dp, b, o.at, o.sl, o.z, lse);
        wstore_sinks(g, bs, dp + 1, e, b, xyd, o, lse);
    }
}

// chunk of a large net: its load comes from the prologue; every chunk
// evaluates the driver cell, the first one stores it
template <bool lse>
__device__ void wfwd_chunk(const DevNet& g, const BatchState& bs, const DfState& d, int n, int p0, int cnt, int b,
                           float gamma, bool stall) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    WFCell f = wfcell_topo(g, n);
    WFIn in;
    const bool ok = wfcell_fanin(bs, f, b, lse, stall, in);
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float ld = bs.load[ix(n, Bp, b)];
    wfcell_to_col(f, in);
    wfcell_lib(g, f, ld);
    const WOut o = wfcell_eval<true>(g, bs, f, dp, b, gamma, lse, d.abort_word, stall, ok);
    if (f.t >= 0 && p0 == dp + 1) wstore_pin(bs, dp, b, o.at, o.sl, o.z, lse);
    wstore_sinks(g, bs, p0, p0 + cnt, b, xyd, o, lse);
}

// 4 blocks per SM (126 registers, no spills): measured faster than 5 (96
// registers with spills) and than a search of the slew axis per lookup
template <bool lse>
__global__ void __launch_bounds__(kWBlock, 4) k_bfwd_w(DevNet g, BatchState bs, DfState d, float gamma,
                                                       int stall_task) {
    const int G = bs.G;
    const int Q = d.TF * G;
    int q = grab(d.heads + 0);
    while (q < Q) {
        const int t = q / G, gw = q - t * G;
        const WLane L = wlane(gw);
        const int4 task = d.ftask[t];
        if (task.y > 0) wfwd_nets<lse>(g, bs, d, task.x, task.y, L.b, gamma, t == stall_task);
        else wfwd_chunk<lse>(g, bs, d, task.x, task.z, task.w, L.b, gamma, t == stall_task);
        q = grab(d.heads + 0);  // the next task only once this one is done
    }
}

// ---------------------------------------------------------------------------
// Backward
// ---------------------------------------------------------------------------

// The driver cell's backward terms for the four conditions of one placement,
// all from forward results (as BCell of batch.cu): arc delays of every
// condition (required times); for the late conditions (index rf) the LSE
// weights, the NLDM partials, the late-slew arc and its slew partials.  The
// per-arc terms live in the lane's column of shared memory (WArc), so the arc
// loops run rolled: loops unrolled over register arrays made four copies of
// the cell's lookups, and the kernel's instruction fetch stalled on them.
struct WBCell {
    int t, na;
    int rfi[2];
    int pin0;  // the first arc's input pin (a capturing clock pin's seed)
    int amax[2];
    float dSs[2], dSl[2];
    float cs[2];  // propagated clock: the setup seed of a one-input cell's clock pin (rising input)
};

// Word w of the lane's column: [w * kWBlock + threadIdx.x].  Per arc k: input
// pin, input slews of the four conditions, LSE arrivals of the two late input
// transitions, delays of the four conditions, and per late condition the LSE
// weight, d delay / d slew and d delay / d load.
struct WArc {
    int* pin;  // [k]
    float* f;  // kSin + 4k + c, kZin + 2k + rf, kDel + 4k + c, kW / kDs / kDl + 2k + rf
    static constexpr int kSin = 0, kZin = 16, kDel = 24, kW = 40, kDs = 48, kDl = 56, kWords = 64;
    __device__ __forceinline__ float& at(int w) const { return f[w * kWBlock + threadIdx.x]; }
    __device__ __forceinline__ int& pin_of(int k) const { return pin[k * kWBlock + threadIdx.x]; }
};

__device__ __forceinline__ WArc warc() {
    __shared__ float f[WArc::kWords * kWBlock];
    __shared__ int pin[STA_MAX_ARCS * kWBlock];
    WArc a;
    a.f = f;
    a.pin = pin;
    return a;
}

template <int mode>
__device__ __forceinline__ WBCell wbcell_pre(const DevNet& g, const BatchState& bs, int n, int dp, int b,
                                             float gamma) {
    const int Bp = bs.Bp;
    const WArc A = warc();
    WBCell bc;
    const int4 q0 = __ldg(g.net_desc + 2 * n), q1 = __ldg(g.net_desc + 2 * n + 1);  // one record
    bc.t = q0.x;
    bc.na = q0.z;
    bc.pin0 = q1.x;
#pragma unroll
    for (int rf = 0; rf < 2; ++rf) {
        bc.rfi[rf] = 0;
        bc.amax[rf] = -1;
        bc.dSs[rf] = bc.dSl[rf] = bc.cs[rf] = 0.f;
    }
    if (bc.t < 0) return bc;
    const int t = bc.t;
    const int un = q0.w >> 4;
    const int dpin[STA_MAX_ARCS] = {q1.x, q1.y, q1.z, q1.w};
    // the arcs' input words first, all loads in one round (unrolled: loads and
    // shared-memory stores only)
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (k < bc.na) {
            A.pin_of(k) = dpin[k];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int el = c >> 1, rf = c & 1;
                const int r = rf ^ ((un >> k) & 1);
                if (el == 0) bc.rfi[rf] |= r << k;
                if (!((mode & 1) || el)) continue;  // mode 2 needs the late conditions only
                A.at(WArc::kSin + 4 * k + c) = bs.slew[ix(4 * dpin[k] + 2 * el + r, Bp, b)];
                if ((mode & 2) && el) A.at(WArc::kZin + 2 * k + rf) = bs.ats[ix(2 * dpin[k] + r, Bp, b)];
            }
        }
    }
    const float ld = bs.load[ix(n, Bp, b)];
    const float* li = g.lib_idx + t * kLibStride + 8;
    const int jl = axis_seg(li, ld);
    const float inv_l = __ldg(g.lib_inv + t * kLibStride + 8 + jl);
    const float ul = (ld - __ldg(li + jl)) * inv_l;
    float zd[2] = {0.f, 0.f};
    if (mode & 2) {
        zd[0] = bs.ats[ix(2 * dp, Bp, b)];
        zd[1] = bs.ats[ix(2 * dp + 1, Bp, b)];
    }
    float best[2] = {-kInf, -kInf};
#pragma unroll 1
    for (int k = 0; k < bc.na; ++k) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int el = c >> 1, rf = c & 1;
            if (!((mode & 1) || el)) continue;
            const float sin = A.at(WArc::kSin + 4 * k + c);
            const float* si = g.lib_idx + t * kLibStride;
            const int is = axis_seg(si, sin);
            const float inv_s = __ldg(g.lib_inv + t * kLibStride + is);
            const float ts = (sin - __ldg(si + is)) * inv_s;
            float4 dq, sq;
            cell_corners(g, t, k, rf, is, jl, dq, sq);
            float dDs, dDl, dSs, dSl;
            const float D = lerp_cell_grad(dq, ts, ul, inv_s, inv_l, dDs, dDl);
            A.at(WArc::kDel + 4 * k + c) = D;
            if ((mode & 2) && el) {
                const float S = lerp_cell_grad(sq, ts, ul, inv_s, inv_l, dSs, dSl);
                A.at(WArc::kDs + 2 * k + rf) = dDs;
                A.at(WArc::kDl + 2 * k + rf) = dDl;
                A.at(WArc::kW + 2 * k + rf) = expf((A.at(WArc::kZin + 2 * k + rf) + D - zd[rf]) / gamma);
                if (S > best[rf]) {
                    best[rf] = S;
                    bc.amax[rf] = k;
                    bc.dSs[rf] = dSs;
                    bc.dSl[rf] = dSl;
                }
            }
        }
    }
    // a capturing clock pin is the input of a one-input cell; its seed is read
    // here, before the wait, and added to the rising adjoint it writes
    if ((mode & 2) && bs.cap_seed && bc.na == 1) {
#pragma unroll
        for (int rf = 0; rf < 2; ++rf)
            if ((bc.rfi[rf] & 1) == 0) bc.cs[rf] = __ldcg(bs.cap_seed + ix(bc.pin0, Bp, b));
    }
    return bc;
}

// Required times of the cell's inputs (R[c] at the output) and the adjoint of
// the late conditions; returns each condition's part of d loss / d load in gl
// (zero for the early ones).
template <int mode>
__device__ __forceinline__ void wbcell_apply(const BatchState& bs, const WBCell& bc, int b, const float* R,
                                             const float* GA, const float* GS, float* gl) {
    const int Bp = bs.Bp;
    const WArc A = warc();
#pragma unroll
    for (int c = 0; c < 4; ++c) gl[c] = 0.f;
    if (bc.t < 0) return;
#pragma unroll 1
    for (int k = 0; k < bc.na; ++k) {
        const int pin = A.pin_of(k);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int el = c >> 1, rf = c & 1;
            const int r = (bc.rfi[rf] >> k) & 1;
            // strong stores: words that the sinks' tasks poll
            if (mode & 1) st_poll(bs.rat + ix(4 * pin + 2 * el + r, Bp, b), R[c] - A.at(WArc::kDel + 4 * k + c));
            if ((mode & 2) && el) {
                const float gD = GA[rf] * A.at(WArc::kW + 2 * k + rf);
                // a capturing clock pin also carries its endpoint's setup term
                st_poll(bs.g_ats + ix(2 * pin + r, Bp, b), (bs.cap_seed && k == 0) ? gD + bc.cs[rf] : gD);
                st_poll(bs.g_slew + ix(2 * pin + r, Bp, b),
                        fmaf(gD, A.at(WArc::kDs + 2 * k + rf), k == bc.amax[rf] ? GS[rf] * bc.dSs[rf] : 0.f));
                gl[c] = fmaf(gD, A.at(WArc::kDl + 2 * k + rf), gl[c]);
            }
        }
    }
    if (mode & 2) {
#pragma unroll
        for (int rf = 0; rf < 2; ++rf)
            if (bc.amax[rf] >= 0) gl[2 + rf] = fmaf(GS[rf], bc.dSl[rf], gl[2 + rf]);
    }
}

// One sink's terms for the four conditions of one placement (as bsink of
// batch.cu): r[c] = RAT_s - Delay_s; for the late conditions (rf) the sink's
// LSE-arrival adjoint, the slew term and the wire adjoint.
struct WSink {
    float r[4], ga[2], gs[2], gw[2];
    Wire w;
};

// The adjoint seeds of an endpoint sink (a sink without a consumer task):
// d loss / d LSE-arrival of both transitions from its slacks sr, sf (the TNS
// soft-min with the zero term, and the WNS soft-min's share).  Out of line:
// endpoints are a small share of the sinks, and the accurate exponentials
// inlined in every sink loop crowded the instruction cache.
__device__ __noinline__ float2 wsink_seed(float sr, float sf, float gamma, float W, float wt, float ww) {
    const float te = softmin3(sr, sf, gamma);
    float g[2];
#pragma unroll
    for (int rf = 0; rf < 2; ++rf) {
        const float sv = rf ? sf : sr;
        float gv = wt * expf(-(sv - te) / gamma);
        if (isfinite(W)) gv += ww * expf(-(sv - W) / gamma);
        g[rf] = -gv;
    }
    return make_float2(g[0], g[1]);
}

template <int mode, bool kPoll>
__device__ __forceinline__ WSink wsink(const DevNet& g, const BatchState& bs, const DfState& d, int p, int b,
                                       float2 xyd, const float* sld, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    WSink s;
    // one round of loads: the sink's position, capacitance, consumer and late
    // slews (plain) together with the words its producers write (polled); the
    // wait repeats only the polled ones.  A sink without a consumer task
    // (pin_cons < 0, the same for every lane) holds no word of the sweep: its
    // adjoint loads are discarded and its seed computed below.
    const float2 xy = bs.xy[ix(p, Bp, b)];
    const float cap = __ldg(g.pin_cap + p);
    const int cons = d.pin_cons[p];
    float sl[2] = {0.f, 0.f};
    if (mode & 2) {
        sl[0] = bs.slew[ix(4 * p + 2, Bp, b)];
        sl[1] = bs.slew[ix(4 * p + 3, Bp, b)];
    }
    float rr[4] = {0.f, 0.f, 0.f, 0.f}, ga[2] = {0.f, 0.f}, gs[2] = {0.f, 0.f};
    auto load = [&]() {
        bool ok = true;
        if (mode & 1) {
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                rr[c] = kPoll ? ld_poll(bs.rat + ix(4 * p + c, Bp, b)) : __ldcg(bs.rat + ix(4 * p + c, Bp, b));
                ok &= written(rr[c]);
            }
        }
        if (mode & 2) {
#pragma unroll
            for (int rf = 0; rf < 2; ++rf) {
                ga[rf] = kPoll ? ld_poll(bs.g_ats + ix(2 * p + rf, Bp, b)) : __ldcg(bs.g_ats + ix(2 * p + rf, Bp, b));
                gs[rf] = kPoll ? ld_poll(bs.g_slew + ix(2 * p + rf, Bp, b)) : __ldcg(bs.g_slew + ix(2 * p + rf, Bp, b));
                ok &= written(ga[rf]) & written(gs[rf]);
            }
        }
        return ok;
    };
    const bool ok = load();
    const bool dyn = cons >= 0;  // the same for every lane
    if (kPoll && dyn && !__all_sync(kFull, ok)) poll_words(load, d.abort_word);
    s.w = wire(g, xy, xyd, cap);
#pragma unroll
    for (int c = 0; c < 4; ++c) s.r[c] = (mode & 1) ? rr[c] - s.w.D : 0.f;
#pragma unroll
    for (int rf = 0; rf < 2; ++rf) s.ga[rf] = s.gs[rf] = s.gw[rf] = 0.f;
    if (mode & 2) {
        if (!dyn) {
#pragma unroll
            for (int rf = 0; rf < 2; ++rf) ga[rf] = gs[rf] = 0.f;
            const float rl = (mode & 1) ? rr[2] : bs.rat[ix(4 * p + 2, Bp, b)];
            const float rfl = (mode & 1) ? rr[3] : bs.rat[ix(4 * p + 3, Bp, b)];
            if (isfinite(rl)) {
                const float sr = rl - bs.ats[ix(2 * p, Bp, b)], sf = rfl - bs.ats[ix(2 * p + 1, Bp, b)];
                const float2 gg = wsink_seed(sr, sf, gamma, sd.W, sd.wt, sd.ww);
                ga[0] = gg.x;
                ga[1] = gg.y;
            }
        }
#pragma unroll
        for (int rf = 0; rf < 2; ++rf) {
            const float qv = sl[rf] > 0.f ? gs[rf] / sl[rf] : 0.f;
            s.ga[rf] = ga[rf];
            s.gs[rf] = qv * sld[rf];
            s.gw[rf] = fmaf(qv, s.w.I, ga[rf]);
        }
    }
    return s;
}

// Packed small nets: per net the sinks' terms (the wait), the driver's arc
// step, then the sinks' and the driver's gradients.
template <int mode>
__device__ void wbwd_nets(const DevNet& g, const BatchState& bs, const DfState& d, int n0, int nn, int b,
                          float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    for (int j = 0; j < nn; ++j) {
        const int n = n0 + j;
        const int dp = g.net_ptr[n], e = g.net_ptr[n + 1];
        const WBCell bc = wbcell_pre<mode>(g, bs, n, dp, b, gamma);
        const float2 xyd = bs.xy[ix(dp, Bp, b)];
        float sld[2] = {0.f, 0.f};
        if (mode & 2) {
            sld[0] = bs.slew[ix(4 * dp + 2, Bp, b)];
            sld[1] = bs.slew[ix(4 * dp + 3, Bp, b)];
        }
        float R[4] = {kInf, kInf, kInf, kInf}, GA[2] = {0.f, 0.f}, GS[2] = {0.f, 0.f};
        R[0] = R[1] = -kInf;  // early conditions: max
// (not unrolled: the smaller loop body measured 6% faster, fewer instruction-fetch stalls)
#pragma unroll 1
        for (int p = dp + 1; p < e; ++p) {
            const WSink s = wsink<mode, true>(g, bs, d, p, b, xyd, sld, gamma, sd);
#pragma unroll
            for (int c = 0; c < 4; ++c) R[c] = (c >> 1) ? fminf(R[c], s.r[c]) : fmaxf(R[c], s.r[c]);
#pragma unroll
            for (int rf = 0; rf < 2; ++rf) {
                GA[rf] += s.ga[rf];
                GS[rf] += s.gs[rf];
            }
            // the sink's wire adjoint, both transitions; kept until d loss / d load is known
            if (mode & 2) bs.grad[ix(p, Bp, b)].x = s.gw[0] + s.gw[1];
        }
        if (mode & 1) {
#pragma unroll
            for (int c = 0; c < 4; ++c) bs.rat[ix(4 * dp + c, Bp, b)] = R[c];
        }
        float gl[4];
        wbcell_apply<mode>(bs, bc, b, R, GA, GS, gl);
        if (mode & 2) {
            const float gload = (gl[0] + gl[1]) + (gl[2] + gl[3]);  // early conditions contribute 0
            // sums over the sinks c, c + 4, ... (batch.cu's quad lanes), four
            // sinks' loads per round
            float sx[4] = {0.f, 0.f, 0.f, 0.f}, sy[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
            for (int p0 = dp + 1; p0 < e; p0 += 4) {
                float gw[4], cap[4];
                float2 xy[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int p = min(p0 + u, e - 1);
                    gw[u] = bs.grad[ix(p, Bp, b)].x;
                    xy[u] = bs.xy[ix(p, Bp, b)];
                    cap[u] = __ldg(g.pin_cap + p);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (p0 + u < e) {
                        const float2 gxy = bsink_grad(g, xy[u], xyd, cap[u], gw[u], gload);
                        bs.grad[ix(p0 + u, Bp, b)] = gxy;
                        sx[u] += gxy.x;
                        sy[u] += gxy.y;
                    }
                }
            }
            bs.grad[ix(dp, Bp, b)] = make_float2(-((sx[0] + sx[1]) + (sx[2] + sx[3])),
                                                 -((sy[0] + sy[1]) + (sy[2] + sy[3])));
        }
    }
}

// Partial chunk of a large net (slots as in batch.cu: 0-3 required times by
// condition, 4-5 sums of g_ats, 6-7 of g_slew * slew_d / slew_s, 8-11 the
// sign sums and sign-weighted wire adjoints of the driver's gradient).
template <int mode>
__device__ void wbwd_part(const DevNet& g, const BatchState& bs, const DfState& d, int n, int p0, int np, int slot,
                          int b, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    float sld[2] = {0.f, 0.f};
    if (mode & 2) {
        sld[0] = bs.slew[ix(4 * dp + 2, Bp, b)];
        sld[1] = bs.slew[ix(4 * dp + 3, Bp, b)];
    }
    float R[4] = {-kInf, -kInf, kInf, kInf}, GA[2] = {0.f, 0.f}, GS[2] = {0.f, 0.f};
    float sx = 0.f, sy = 0.f, hx = 0.f, hy = 0.f;
#pragma unroll 1
    for (int p = p0; p < p0 + np; ++p) {
        const WSink s = wsink<mode, true>(g, bs, d, p, b, xyd, sld, gamma, sd);
#pragma unroll
        for (int c = 0; c < 4; ++c) R[c] = (c >> 1) ? fminf(R[c], s.r[c]) : fmaxf(R[c], s.r[c]);
#pragma unroll
        for (int rf = 0; rf < 2; ++rf) {
            GA[rf] += s.ga[rf];
            GS[rf] += s.gs[rf];
        }
        if (mode & 2) {
            const float gw = s.gw[0] + s.gw[1];
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
#pragma unroll
    for (int c = 0; c < 4; ++c) st_poll(part + ix(base + c, Bp, b), R[c]);
    if (mode & 2) {
#pragma unroll
        for (int rf = 0; rf < 2; ++rf) {
            st_poll(part + ix(base + 4 + rf, Bp, b), GA[rf]);
            st_poll(part + ix(base + 6 + rf, Bp, b), GS[rf]);
        }
        st_poll(part + ix(base + 8, Bp, b), sx);
        st_poll(part + ix(base + 9, Bp, b), sy);
        st_poll(part + ix(base + 10, Bp, b), hx);
        st_poll(part + ix(base + 11, Bp, b), hy);
    }
}

// Driver step of a large net: the chunks' partials combined in chunk order,
// then the arc step and the driver's gradient; publishes d loss / d load.
template <int mode>
__device__ void wbwd_driver(const DevNet& g, const BatchState& bs, const DfState& d, int n, int slot0, int nch, int b,
                            float gamma) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const WBCell bc = wbcell_pre<mode>(g, bs, n, dp, b, gamma);
    const float* part = (mode & 2) ? bs.part : bs.rpart;
    constexpr int kS = (mode & 2) ? 12 : 4;  // slots read
    constexpr int kU = 2;                    // chunks per poll round
    float R[4] = {-kInf, -kInf, kInf, kInf}, v[12];
#pragma unroll
    for (int i = 0; i < 12; ++i) v[i] = 0.f;
    for (int k0 = 0; k0 < nch; k0 += kU) {
        float x[kU][kS];
        // in the dataflow sweep this is the wait: repeated until the chunks'
        // words are written
        auto load = [&]() {
            bool all = true;
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const int base = (slot0 + k0 + u) * kPartFloats;
                const bool ok = k0 + u < nch;
#pragma unroll
                for (int i = 0; i < kS; ++i) {
                    x[u][i] = ok ? ld_poll(part + ix(base + i, Bp, b)) : 0.f;
                    if (ok) all &= written(x[u][i]);
                }
            }
            return all;
        };
        poll_words(load, d.abort_word);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (k0 + u >= nch) break;
#pragma unroll
            for (int c = 0; c < 4; ++c) R[c] = (c >> 1) ? fminf(R[c], x[u][c]) : fmaxf(R[c], x[u][c]);
#pragma unroll
            for (int i = 4; i < kS; ++i) v[i] += x[u][i];
        }
    }
    if (mode & 1) {
#pragma unroll
        for (int c = 0; c < 4; ++c) bs.rat[ix(4 * dp + c, Bp, b)] = R[c];
    }
    const float GA[2] = {v[4], v[5]}, GS[2] = {v[6], v[7]};
    float gl[4];
    wbcell_apply<mode>(bs, bc, b, R, GA, GS, gl);
    if (mode & 2) {
        const float gload = (gl[0] + gl[1]) + (gl[2] + gl[3]);
        bs.net_gload[ix(n, Bp, b)] = gload;
        bs.grad[ix(dp, Bp, b)] = make_float2(-fmaf(gload * g.c, v[8], v[10]), -fmaf(gload * g.c, v[9], v[11]));
    }
}

// Gradient chunk of a large net: d loss / d (x, y) of its sinks once the
// driver step has published d loss / d load.  No task waits for these.
__device__ void wbwd_grad(const DevNet& g, const BatchState& bs, const DfState& d, int32_t* cnt, int q, int n, int p0,
                          int np, int b, float gamma, const BSeed& sd) {
    const int Bp = bs.Bp;
    const int dp = g.net_ptr[n];
    const float2 xyd = bs.xy[ix(dp, Bp, b)];
    const float sld[2] = {bs.slew[ix(4 * dp + 2, Bp, b)], bs.slew[ix(4 * dp + 3, Bp, b)]};
    wait_ready(cnt, q, d.b_indeg[q / bs.G], d.abort_word);
    const float gload = __ldcg(bs.net_gload + ix(n, Bp, b));
#pragma unroll 1
    for (int p = p0; p < p0 + np; ++p) {
        const WSink s = wsink<2, false>(g, bs, d, p, b, xyd, sld, gamma, sd);
        bs.grad[ix(p, Bp, b)] =
            bsink_grad(g, bs.xy[ix(p, Bp, b)], xyd, __ldg(g.pin_cap + p), s.gw[0] + s.gw[1], gload);
    }
}

template <int mode>
__global__ void __launch_bounds__(kWBlock, 5) k_bbwd_w(DevNet g, BatchState bs, DfState d, float gamma) {
    int32_t* cnt = (mode & 2) ? d.acnt : d.rcnt;
    int32_t* head = d.heads + ((mode & 2) ? 2 : 1);
    const int G = bs.G;
    const int Q = d.TB * G;
    int q = grab(head);
    while (q < Q) {
        const int t = q / G, gw = q - t * G;
        const WLane L = wlane(gw);
        BSeed sd;
        sd.W = (float)bs.summary[(size_t)L.b * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
        sd.wt = bs.params[2 * L.b];
        sd.ww = bs.params[2 * L.b + 1];
        const int4 task = d.btask[t];
        if (task.y > 0) wbwd_nets<mode>(g, bs, d, task.x, task.y, L.b, gamma, sd);
        else if (task.y == -1) wbwd_part<mode>(g, bs, d, task.x, task.z, task.w, d.baux[t], L.b, gamma, sd);
        else if (task.y == -2) wbwd_driver<mode>(g, bs, d, task.x, task.z, task.w, L.b, gamma);
        else if (mode & 2) wbwd_grad(g, bs, d, cnt, q, task.x, task.z, task.w, L.b, gamma, sd);
        // every consumer polls the words its producers wrote, except the gradient
        // chunks of a large net, which wait on a counter that its driver step releases
        if (task.y == -2) {
            __syncwarp();
            const int k1 = d.b_out_ptr[t + 1];
            for (int k = d.b_out_ptr[t] + L.lane; k < k1; k += 32) red_release_add(cnt + d.b_out[k] * G + gw, 1);
        }
        q = grab(head);
    }
}

}  // namespace

int batch_wide_fwd_max_blocks() {
    int dev = 0, sms = 0, a = 0, b = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bfwd_w<true>, kWBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bfwd_w<false>, kWBlock, 0);
    const int per_sm = std::min(a, b);
    return sms * (per_sm > 0 ? per_sm : 1);
}

void launch_batch_fwd_wide(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int lse,
                           int stall_task, cudaStream_t st) {
    if (d.TF == 0) return;
    if (lse) launch_coop(k_bfwd_w<true>, grid, kWBlock, 0, st, g, bs, d, gamma, stall_task);
    else launch_coop(k_bfwd_w<false>, grid, kWBlock, 0, st, g, bs, d, gamma, stall_task);
}

int batch_wide_max_blocks() {
    int dev = 0, sms = 0, a = 0, b = 0, c = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bbwd_w<1>, kWBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bbwd_w<2>, kWBlock, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_bbwd_w<3>, kWBlock, 0);
    const int per_sm = std::min(a, std::min(b, c));
    return sms * (per_sm > 0 ? per_sm : 1);
}

void launch_batch_bwd_wide(const DevNet& g, const BatchState& bs, const DfState& d, int grid, float gamma, int mode,
                           cudaStream_t st) {
    if (d.TB == 0) return;
    if (mode == 1) launch_coop(k_bbwd_w<1>, grid, kWBlock, 0, st, g, bs, d, gamma);
    else if (mode == 2) launch_coop(k_bbwd_w<2>, grid, kWBlock, 0, st, g, bs, d, gamma);
    else launch_coop(k_bbwd_w<3>, grid, kWBlock, 0, st, g, bs, d, gamma);
}

}  // namespace sta
