// kernels.cu -- sm_103a kernels of the levelized STA path.
//
// Work decomposition (replacing the paper's (4 x 8 x NETS_PER_BLOCK) thread
// layout of Algorithm 1): per level the builder packs consecutive nets of at
// most 32 pins, at most 8 of them, into one warp ("warp task"): lanes map to
// the task's pins, so a net of 3 pins uses 3 lanes and a warp stays busy
// whatever the fanout mix; the per-net reductions of Eq. 1 (load) and of the
// required-time / adjoint passes are segmented warp-shuffle scans, with no
// shared memory and no atomics.  The driver-cell evaluation of a task uses 4
// lanes per net, one per timing condition (cond = 2*el + rf).  Nets of more
// than 32 pins get a whole 256-thread block each ("block task") with a
// fixed-order block reduction.  Every reduction order depends on the netlist
// only, so results are bit-identical run to run.
#include "device_common.cuh"

namespace sta {
namespace {

// ---------------------------------------------------------------------------
// positions: internal order <- caller's pin order
// ---------------------------------------------------------------------------
// one lane per grid row: lane l reads the caller's placement l ([lanes][P][2]);
// the grid has a row per lane the following calls run, and it records that
// count for them (lanes handles)
__global__ void __launch_bounds__(kBlock) k_gather_xy(DevNet g, DevState s0, const float2* __restrict__ xy0) {
    if (s0.active && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *s0.active = (int)gridDim.y;
    const DevState s = lane_state(s0, blockIdx.y);
    const float2* xy = xy0 + (size_t)blockIdx.y * g.P;
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < g.P; p += gridDim.x * blockDim.x)
        s.xy[p] = xy[g.pin_orig[p]];
}

// ---------------------------------------------------------------------------
// Net RC, Eqs. 1-3 on a star: for a sink at Manhattan distance d,
//   R = r d, C = cap + c d / 2, Delay = R C, Impulse = sqrt(2 R C Delay - Delay^2)
// and the driver's Load = cap_driver + sum_sinks (cap + c d).
// ---------------------------------------------------------------------------
__device__ void rc_warp(const DevNet& g, const DevState& s, int n0, int nn) {
    const WarpGeom w = warp_geom(g, n0, nn);
    const int p = w.pin0 + w.lane;
    const float2 xy = w.valid ? s.xy[p] : make_float2(0.f, 0.f);
    const float cap = w.valid ? g.pin_cap[p] : 0.f;
    const float2 xyd = make_float2(__shfl_sync(kFull, xy.x, w.hd), __shfl_sync(kFull, xy.y, w.hd));
    float v = cap;
    if (w.valid && w.lane != w.hd) v = rc_sink(g, s, p, xy, xyd, cap);
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const float u = __shfl_up_sync(kFull, v, off);
        if (w.lane - off >= w.hd) v += u;
    }
    if (w.valid && w.lane == w.last) s.load[n0 + w.j] = v;
}

// blocks [0, nwb): 8 warp tasks each; the rest: one large-net RC chunk each
__global__ void __launch_bounds__(kBlock) k_rc(DevNet g, DevState s, int nw) {
    const int nwb = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if ((int)blockIdx.x < nwb) {
        const int t = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (t >= nw) return;
        rc_warp(g, s, g.wtask[2 * t], g.wtask[2 * t + 1]);
    } else {
        const int k = blockIdx.x - nwb;
        rc_chunk(g, s, g.rc_chunk[k], g.rc_net[k]);
    }
}

// ---------------------------------------------------------------------------
// Forward level: driver cells (4 lanes per net), then wire propagation to
// every sink: AT_s = AT_d + Delay_s, slew_s = sqrt(slew_d^2 + Impulse_s^2).
// ---------------------------------------------------------------------------
__device__ void fwd_warp(const DevNet& g, const DevState& s, int n0, int nn, float gamma, bool lse) {
    const WarpGeom w = warp_geom(g, n0, nn);
    const int j1 = w.lane >> 2, c = w.lane & 3;
    const int hj = __shfl_sync(kFull, w.h, j1);
    DrvOut o{0.f, 0.f, 0.f};
    if (j1 < nn) {
        const int n = n0 + j1, d = w.pin0 + hj;
        o = eval_driver<false>(g, s, n, d, c, s.load[n], gamma, lse);
        if (g.net_drv[n] >= 0) {
            s.at[4 * d + c] = o.at;
            s.slew[4 * d + c] = o.slew;
            if (lse && c >= 2) s.ats[2 * d + c - 2] = o.ats;
        }
    }
    const int src = 4 * max(w.j, 0);
    float A[4], S[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = __shfl_sync(kFull, o.at, src + k);
        S[k] = __shfl_sync(kFull, o.slew, src + k);
    }
    const float z0 = __shfl_sync(kFull, o.ats, src + 2), z1 = __shfl_sync(kFull, o.ats, src + 3);
    if (w.valid && w.lane != w.hd) store_sink(s, w.pin0 + w.lane, A, S, z0, z1, lse);
}

__device__ void fwd_block(const DevNet& g, const DevState& s, int n, float gamma, bool lse) {
    __shared__ float sh[12];
    const int d = g.net_ptr[n], e = g.net_ptr[n + 1];
    if (threadIdx.x < 4) {
        const int c = threadIdx.x;
        const DrvOut o = eval_driver<false>(g, s, n, d, c, s.load[n], gamma, lse);
        if (g.net_drv[n] >= 0) {
            s.at[4 * d + c] = o.at;
            s.slew[4 * d + c] = o.slew;
            if (lse && c >= 2) s.ats[2 * d + c - 2] = o.ats;
        }
        sh[c] = o.at;
        sh[4 + c] = o.slew;
        if (c >= 2) sh[8 + c - 2] = o.ats;
    }
    __syncthreads();
    float A[4], S[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = sh[k];
        S[k] = sh[4 + k];
    }
    const float z0 = sh[8], z1 = sh[9];
#pragma unroll 4
    for (int p = d + 1 + threadIdx.x; p < e; p += kBlock) store_sink(s, p, A, S, z0, z1, lse);
}

__global__ void __launch_bounds__(kBlock) k_fwd(DevNet g, DevState s, int w0, int nw, int c0, int nc, float gamma,
                                                int lse) {
    const int nwb = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if ((int)blockIdx.x < nwb) {
        const int t = w0 + blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (t >= w0 + nw) return;
        fwd_warp(g, s, g.wtask[2 * t], g.wtask[2 * t + 1], gamma, lse != 0);
    } else {
        fwd_block(g, s, g.ctask[c0 + blockIdx.x - nwb], gamma, lse != 0);
    }
}

// ---------------------------------------------------------------------------
// Backward level (reverse order).  mode & 1: required times
//   RAT_d = min over sinks (RAT_s - Delay_s) late / max early,
//   RAT_in = RAT_out - arc delay through each arc's unateness.
// mode & 2: adjoint of the smoothed loss through the wire step, the LSE cell
// step (softmax weights), the NLDM bilinear partials, the hard late-slew max
// (to the first arc attaining it) and the star RC, down to d/d(x, y).
// ---------------------------------------------------------------------------
__device__ void bwd_warp(const DevNet& g, const DevState& s, int n0, int nn, float gamma, int mode) {
    const WarpGeom w = warp_geom(g, n0, nn);
    const int p = w.pin0 + w.lane;
    const bool sink = w.valid && w.lane != w.hd;
    float2 sld = make_float2(0.f, 0.f);
    if (mode & 2) {
        const float2 sl = w.valid ? reinterpret_cast<const float2*>(s.slew)[2 * p + 1] : make_float2(0.f, 0.f);
        sld = make_float2(__shfl_sync(kFull, sl.x, w.hd), __shfl_sync(kFull, sl.y, w.hd));
    }
    SinkBwd b;
    if (sink) {
        b = sink_bwd(s, p, sld, mode);
    } else {
        b.r[0] = b.r[1] = -kInf;
        b.r[2] = b.r[3] = kInf;
        b.ga[0] = b.ga[1] = b.gs[0] = b.gs[1] = b.gwire = 0.f;
    }
    // segmented inclusive scans: totals land on the last pin of each net
    float r0 = b.r[0], r1 = b.r[1], r2 = b.r[2], r3 = b.r[3];
    float ga0 = b.ga[0], ga1 = b.ga[1], gs0 = b.gs[0], gs1 = b.gs[1];
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const bool take = w.lane - off >= w.hd;
        if (mode & 1) {
            const float u0 = __shfl_up_sync(kFull, r0, off), u1 = __shfl_up_sync(kFull, r1, off);
            const float u2 = __shfl_up_sync(kFull, r2, off), u3 = __shfl_up_sync(kFull, r3, off);
            if (take) {
                r0 = fmaxf(r0, u0);
                r1 = fmaxf(r1, u1);
                r2 = fminf(r2, u2);
                r3 = fminf(r3, u3);
            }
        }
        if (mode & 2) {
            const float u0 = __shfl_up_sync(kFull, ga0, off), u1 = __shfl_up_sync(kFull, ga1, off);
            const float u2 = __shfl_up_sync(kFull, gs0, off), u3 = __shfl_up_sync(kFull, gs1, off);
            if (take) {
                ga0 += u0;
                ga1 += u1;
                gs0 += u2;
                gs1 += u3;
            }
        }
    }
    if ((mode & 1) && w.valid && w.lane == w.last)
        reinterpret_cast<float4*>(s.rat)[w.pin0 + w.hd] = make_float4(r0, r1, r2, r3);

    // driver cell step: lane 4 j + c handles net j, condition c
    const int j1 = w.lane >> 2, c = w.lane & 3;
    const int hj = __shfl_sync(kFull, w.h, j1);
    const int lastj = __shfl_sync(kFull, w.h, j1 + 1) - 1;
    const float R0 = __shfl_sync(kFull, r0, lastj & 31), R1 = __shfl_sync(kFull, r1, lastj & 31);
    const float R2 = __shfl_sync(kFull, r2, lastj & 31), R3 = __shfl_sync(kFull, r3, lastj & 31);
    const float GA0 = __shfl_sync(kFull, ga0, lastj & 31), GA1 = __shfl_sync(kFull, ga1, lastj & 31);
    const float GS0 = __shfl_sync(kFull, gs0, lastj & 31), GS1 = __shfl_sync(kFull, gs1, lastj & 31);
    float gl = 0.f;
    if (j1 < nn) {
        const int n = n0 + j1, d = w.pin0 + hj, t = g.net_drv[n];
        if (t >= 0) {
            const int el = c >> 1, rf = c & 1;
            if (mode & 1) {
                const float Rc = c == 0 ? R0 : c == 1 ? R1 : c == 2 ? R2 : R3;
                const int a0 = g.net_arc_ptr[n], a1 = g.net_arc_ptr[n + 1], un = g.lib_unate[t];
                for (int a = a0; a < a1; ++a) {
                    const int rfi = rf ^ ((un >> (a - a0)) & 1);
                    s.rat[4 * g.arc_pin[a] + 2 * el + rfi] = Rc - s.adel[4 * a + c];
                }
            }
            if ((mode & 2) && el == 1)
                gl = arc_adjoint(g, s, n, d, t, rf, rf ? GA1 : GA0, rf ? GS1 : GS0, gamma);
        }
    }
    if (mode & 2) {
        gl += __shfl_down_sync(kFull, gl, 1);  // lane 4j+2: rise + fall
        const float gload = __shfl_sync(kFull, gl, (4 * max(w.j, 0) + 2) & 31);
        const float2 xy = w.valid ? s.xy[p] : make_float2(0.f, 0.f);
        const float2 xyd = make_float2(__shfl_sync(kFull, xy.x, w.hd), __shfl_sync(kFull, xy.y, w.hd));
        float2 gxy = make_float2(0.f, 0.f);
        if (sink) {
            gxy = sink_grad(g, s, p, xy, xyd, b.gwire, gload);
            s.grad[g.pin_orig[p]] = gxy;
        }
        float sx = gxy.x, sy = gxy.y;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float u = __shfl_up_sync(kFull, sx, off), v = __shfl_up_sync(kFull, sy, off);
            if (w.lane - off >= w.hd) {
                sx += u;
                sy += v;
            }
        }
        if (w.valid && w.lane == w.last) s.grad[g.pin_orig[w.pin0 + w.hd]] = make_float2(-sx, -sy);
    }
}

__device__ void bwd_block(const DevNet& g, const DevState& s, int n, float gamma, int mode) {
    __shared__ float sh[kWarpsPerBlock];
    __shared__ float bc[2];
    const int d = g.net_ptr[n], e = g.net_ptr[n + 1];
    const float2 sld = (mode & 2) ? reinterpret_cast<const float2*>(s.slew)[2 * d + 1] : make_float2(0.f, 0.f);
    float r0 = -kInf, r1 = -kInf, r2 = kInf, r3 = kInf, ga0 = 0.f, ga1 = 0.f, gs0 = 0.f, gs1 = 0.f;
#pragma unroll 2
    for (int p = d + 1 + threadIdx.x; p < e; p += kBlock) {
        const SinkBwd b = sink_bwd(s, p, sld, mode);
        r0 = fmaxf(r0, b.r[0]);
        r1 = fmaxf(r1, b.r[1]);
        r2 = fminf(r2, b.r[2]);
        r3 = fminf(r3, b.r[3]);
        ga0 += b.ga[0];
        ga1 += b.ga[1];
        gs0 += b.gs[0];
        gs1 += b.gs[1];
    }
    if (mode & 1) {
        r0 = block_reduce(r0, sh, OpMax());
        r1 = block_reduce(r1, sh, OpMax());
        r2 = block_reduce(r2, sh, OpMin());
        r3 = block_reduce(r3, sh, OpMin());
        if (threadIdx.x == 0) reinterpret_cast<float4*>(s.rat)[d] = make_float4(r0, r1, r2, r3);
    }
    if (mode & 2) {
        ga0 = block_reduce(ga0, sh, OpSum());
        ga1 = block_reduce(ga1, sh, OpSum());
        gs0 = block_reduce(gs0, sh, OpSum());
        gs1 = block_reduce(gs1, sh, OpSum());
    }
    const int t = g.net_drv[n];
    if (threadIdx.x < 4 && t >= 0) {
        const int c = threadIdx.x, el = c >> 1, rf = c & 1;
        if (mode & 1) {
            const float Rc = c == 0 ? r0 : c == 1 ? r1 : c == 2 ? r2 : r3;
            const int a0 = g.net_arc_ptr[n], a1 = g.net_arc_ptr[n + 1], un = g.lib_unate[t];
            for (int a = a0; a < a1; ++a) {
                const int rfi = rf ^ ((un >> (a - a0)) & 1);
                s.rat[4 * g.arc_pin[a] + 2 * el + rfi] = Rc - s.adel[4 * a + c];
            }
        }
        if ((mode & 2) && el == 1) bc[rf] = arc_adjoint(g, s, n, d, t, rf, rf ? ga1 : ga0, rf ? gs1 : gs0, gamma);
    }
    if (!(mode & 2)) return;
    __syncthreads();
    const float gload = t >= 0 ? bc[0] + bc[1] : 0.f;
    const float2 xyd = s.xy[d];
    float sx = 0.f, sy = 0.f;
#pragma unroll 2
    for (int p = d + 1 + threadIdx.x; p < e; p += kBlock) {
        const SinkBwd b = sink_bwd(s, p, sld, 2);
        const float2 gxy = sink_grad(g, s, p, s.xy[p], xyd, b.gwire, gload);
        s.grad[g.pin_orig[p]] = gxy;
        sx += gxy.x;
        sy += gxy.y;
    }
    sx = block_reduce(sx, sh, OpSum());
    sy = block_reduce(sy, sh, OpSum());
    if (threadIdx.x == 0) s.grad[g.pin_orig[d]] = make_float2(-sx, -sy);
}

__global__ void __launch_bounds__(kBlock) k_bwd(DevNet g, DevState s, int w0, int nw, int c0, int nc, float gamma,
                                                int mode) {
    const int nwb = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock;
    if ((int)blockIdx.x < nwb) {
        const int t = w0 + blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
        if (t >= w0 + nw) return;
        bwd_warp(g, s, g.wtask[2 * t], g.wtask[2 * t + 1], gamma, mode);
    } else {
        bwd_block(g, s, g.ctask[c0 + blockIdx.x - nwb], gamma, mode);
    }
}

// ---------------------------------------------------------------------------
// Endpoints: slack, WNS, TNS and the smoothed TNS_gamma / WNS_gamma, by a
// two-pass fixed-order reduction (partials per block in s.red).  Exponentials
// and logarithms are single precision (FP64 transcendentals are slow on this
// part); every sum over endpoints is accumulated in double.
//   TNS_gamma = sum_e softmin_gamma(s_rise, s_fall, 0),
//   WNS_gamma = softmin_gamma over every endpoint rise/fall slack,
//   softmin_gamma(x) = -LSE_gamma(-x), stabilised by the minimum (Eq. 4).
// ---------------------------------------------------------------------------
struct EpAcc {
    double tns_e, tns_l, tns_g, viol;  // sums in double (deterministic order)
    float wns_e, wns_l, wmin, wsum;    // wsum = sum exp(-(s - wmin) / gamma)
};

__device__ __forceinline__ void ep_merge(EpAcc& a, const EpAcc& b, float gamma) {
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

__device__ __forceinline__ EpAcc ep_identity() {
    EpAcc a;
    a.tns_e = a.tns_l = a.tns_g = a.viol = 0.0;
    a.wns_e = a.wns_l = a.wmin = kInf;
    a.wsum = 0.f;
    return a;
}

__device__ __forceinline__ EpAcc ep_shfl_down(const EpAcc& a, int off) {
    EpAcc b;
    b.tns_e = __shfl_down_sync(kFull, a.tns_e, off);
    b.tns_l = __shfl_down_sync(kFull, a.tns_l, off);
    b.tns_g = __shfl_down_sync(kFull, a.tns_g, off);
    b.viol = __shfl_down_sync(kFull, a.viol, off);
    b.wns_e = __shfl_down_sync(kFull, a.wns_e, off);
    b.wns_l = __shfl_down_sync(kFull, a.wns_l, off);
    b.wmin = __shfl_down_sync(kFull, a.wmin, off);
    b.wsum = __shfl_down_sync(kFull, a.wsum, off);
    return b;
}

// Fixed-order reduction of a block's accumulators, the result on thread 0: a
// shuffle tree within each warp (lane i takes lane i + 16, 8, 4, 2, 1), then
// warp 0 combines the warps' results the same way (one barrier; the
// shared-memory tree it replaces spent most of its time in eight of them).
// The first stage in single precision: a thread's endpoints and the warp's
// shuffle tree (a few dozen terms per partial, so float sums stay within a few
// ulps), converted to double once per warp.  Double arithmetic runs at a small
// fraction of the float rate on this part, and 608 blocks each reducing every
// lane in double kept the endpoint launch busy on it.
struct EpAccF {
    float tns_e, tns_l, tns_g, viol;
    float wns_e, wns_l, wmin, wsum;
};

__device__ __forceinline__ EpAccF epf_identity() {
    EpAccF a;
    a.tns_e = a.tns_l = a.tns_g = a.viol = 0.f;
    a.wns_e = a.wns_l = a.wmin = kInf;
    a.wsum = 0.f;
    return a;
}

__device__ __forceinline__ void epf_merge(EpAccF& a, const EpAccF& b, float gamma) {
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

__device__ __forceinline__ EpAccF epf_shfl_down(const EpAccF& a, int off) {
    EpAccF b;
    b.tns_e = __shfl_down_sync(kFull, a.tns_e, off);
    b.tns_l = __shfl_down_sync(kFull, a.tns_l, off);
    b.tns_g = __shfl_down_sync(kFull, a.tns_g, off);
    b.viol = __shfl_down_sync(kFull, a.viol, off);
    b.wns_e = __shfl_down_sync(kFull, a.wns_e, off);
    b.wns_l = __shfl_down_sync(kFull, a.wns_l, off);
    b.wmin = __shfl_down_sync(kFull, a.wmin, off);
    b.wsum = __shfl_down_sync(kFull, a.wsum, off);
    return b;
}

// block partial: warp trees in float, then the warps' partials in double
// (warp 0 holds the block's result)
__device__ void ep_block_reduce_f(EpAccF a, EpAcc& acc, float gamma) {
    __shared__ EpAcc shf[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const EpAccF b = epf_shfl_down(a, off);
        if (lane < off) epf_merge(a, b, gamma);
    }
    if (lane == 0) {
        EpAcc d;
        d.tns_e = a.tns_e;
        d.tns_l = a.tns_l;
        d.tns_g = a.tns_g;
        d.viol = a.viol;
        d.wns_e = a.wns_e;
        d.wns_l = a.wns_l;
        d.wmin = a.wmin;
        d.wsum = a.wsum;
        shf[w] = d;
    }
    __syncthreads();
    if (w == 0) {
        acc = lane < kWarpsPerBlock ? shf[lane] : ep_identity();
#pragma unroll
        for (int off = kWarpsPerBlock / 2; off > 0; off >>= 1) {
            const EpAcc b = ep_shfl_down(acc, off);
            if (lane < off) ep_merge(acc, b, gamma);
        }
    }
}

__device__ void ep_block_reduce(EpAcc& acc, float gamma) {
    __shared__ EpAcc sh[kWarpsPerBlock];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const EpAcc b = ep_shfl_down(acc, off);
        if (lane < off) ep_merge(acc, b, gamma);
    }
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (w == 0) {
        acc = lane < kWarpsPerBlock ? sh[lane] : ep_identity();
#pragma unroll
        for (int off = kWarpsPerBlock / 2; off > 0; off >>= 1) {
            const EpAcc b = ep_shfl_down(acc, off);
            if (lane < off) ep_merge(acc, b, gamma);
        }
    }
}

// Bounds of endpoint e: the constraint (early = hold, late = setup) and, with a
// propagated clock, the capturing clock pin's rising arrival: its late arrival
// moves the hold bound, its early arrival the setup bound.  Returns the clock
// pin, -1 without one.
__device__ __forceinline__ int ep_bounds(const DevNet& g, const DevState& s, int e, float4& con) {
    con = reinterpret_cast<const float4*>(g.ep_rat)[e];
    const int k = g.ep_clk ? g.ep_clk[e] : -1;
    if (k >= 0) {
        const float4 ak = reinterpret_cast<const float4*>(s.at)[k];
        con.x += ak.z;
        con.y += ak.z;
        con.z += ak.x;
        con.w += ak.x;
    }
    return k;
}

// d loss / d s of an endpoint's late rise / fall slacks s = bound - LSE arrival
// (TNS_gamma term and, when WNS_gamma is finite, its term)
__device__ __forceinline__ float2 ep_dloss(float4 con, float2 z, float gamma, float W, float wt, float ww) {
    const float sr = con.z - z.x, sf = con.w - z.y;
    const float te = softmin3(sr, sf, gamma);
    float gr = wt * expf(-(sr - te) / gamma), gf = wt * expf(-(sf - te) / gamma);
    if (isfinite(W)) {
        gr += ww * expf(-(sr - W) / gamma);
        gf += ww * expf(-(sf - W) / gamma);
    }
    return make_float2(gr, gf);
}

// partial of block b written by another block of the same launch: read through L2
__device__ __forceinline__ EpAcc ep_load_cg(const EpAcc* p) {
    static_assert(sizeof(EpAcc) == 48, "EpAcc layout");
    const double2* q = reinterpret_cast<const double2*>(p);
    const double2 a = __ldcg(q), b = __ldcg(q + 1);
    const float4 c = __ldcg(reinterpret_cast<const float4*>(q + 2));
    EpAcc r;
    r.tns_e = a.x;
    r.tns_l = a.y;
    r.tns_g = b.x;
    r.viol = b.y;
    r.wns_e = c.x;
    r.wns_l = c.y;
    r.wmin = c.z;
    r.wsum = c.w;
    return r;
}

// Endpoint slacks, WNS / TNS and the smoothed terms in one launch: each block
// reduces a grid-stride share of the endpoints in a fixed order and stores its
// partial; the last block to finish (a device-scope counter, reset by it for
// the next launch) merges the partials in block order, so the summary does not
// depend on which block finishes last.  With rs_cons non-null the blocks also
// mark the words the next fused dataflow backward sweep polls (the required-time
// and adjoint words of cell-input pins and the large nets' partial records).
__global__ void __launch_bounds__(kBlock) k_ep(DevNet g, DevState s0, float gamma, int lse,
                                               const uchar4* __restrict__ rs_mask, int P, float* rs_part0,
                                               int rs_part_words) {
    if (s0.active && (int)blockIdx.y >= *s0.active) return;  // a lane this call does not run
    // grid row: a lane (its own state), or with several netlists a netlist (its
    // endpoint range, partials, counter and summary; the reset is spread over
    // every block of the grid)
    const bool grp = g.G > 1;
    const int gi = grp ? (int)blockIdx.y : 0;
    DevState s = grp ? s0 : lane_state(s0, blockIdx.y);
    float* rs_part = grp ? rs_part0 : lane_ptr(rs_part0, (size_t)blockIdx.y * s0.lane_bytes);
    int e0 = 0, e1 = g.E;
    if (grp) {
        e0 = g.grp_ep[gi];
        e1 = g.grp_ep[gi + 1];
        s.red += (size_t)gi * gridDim.x * (sizeof(EpAcc) / sizeof(double));
        s.summary += (size_t)gi * STA_SUM_COUNT;
        s.ep_count += gi;
    }
    // (relative to the netlist's first endpoint: the same blocks and order as alone)
    EpAccF accf = epf_identity();
    for (int e = e0 + blockIdx.x * kBlock + threadIdx.x; e < e1; e += gridDim.x * kBlock) {
        const int p = g.ep_pin[e];
        float4 con;
        // a clocked endpoint's bounds are this analysis's required-time seeds
        if (ep_bounds(g, s, e, con) >= 0) reinterpret_cast<float4*>(s.rat)[p] = con;
        const float4 at = reinterpret_cast<const float4*>(s.at)[p];
        const float se = fminf(at.x - con.x, at.y - con.y);
        const float sl = fminf(con.z - at.z, con.w - at.w);
        s.ep_slack[e] = make_float2(se, sl);
        EpAccF b = epf_identity();
        b.wns_e = se;
        b.wns_l = sl;
        b.tns_e = fminf(se, 0.f);
        b.tns_l = fminf(sl, 0.f);
        b.viol = sl < 0.f ? 1.f : 0.f;
        if (lse) {
            const float2 z = reinterpret_cast<const float2*>(s.ats)[p];
            const float sr = con.z - z.x, sf = con.w - z.y;
            b.tns_g = softmin3(sr, sf, gamma);
            b.wmin = fminf(sr, sf);
            b.wsum = expf(-(sr - b.wmin) / gamma) + expf(-(sf - b.wmin) / gamma);
        }
        epf_merge(accf, b, gamma);
    }
    EpAcc acc = ep_identity();
    ep_block_reduce_f(accf, acc, gamma);
    __shared__ int last;
    if (threadIdx.x == 0) {
        reinterpret_cast<EpAcc*>(s.red)[blockIdx.x] = acc;
        __threadfence();
        last = atomicAdd(s.ep_count, 1) == (int)gridDim.x - 1;
    }
    if (rs_mask) {
        const float u = __uint_as_float(kUnwritten);
        const int bx = grp ? (int)(blockIdx.y * gridDim.x + blockIdx.x) : (int)blockIdx.x;
        const int stride = (grp ? (int)(gridDim.x * gridDim.y) : (int)gridDim.x) * kBlock;
        for (int i = bx * kBlock + threadIdx.x; i < rs_part_words; i += stride) rs_part[i] = u;
        // four grid strides per step: the four mask bytes are loaded together, and
        // consecutive threads store consecutive pins
        const uint8_t* mk = reinterpret_cast<const uint8_t*>(rs_mask);
        for (int p0 = bx * kBlock + threadIdx.x; p0 < P; p0 += 4 * stride) {
            unsigned m[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) m[j] = p0 + j * stride < P ? mk[p0 + j * stride] : 0u;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (m[j] & 2) {
                    const int p = p0 + j * stride;
                    reinterpret_cast<float4*>(s.rat)[p] = make_float4(u, u, u, u);
                    reinterpret_cast<float2*>(s.g_ats)[p] = make_float2(u, u);
                    reinterpret_cast<float2*>(s.g_slew)[p] = make_float2(u, u);
                }
        }
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    acc = ep_identity();
    // thread i merges partials i, i + 256, ... in order; then the fixed-order tree
    for (int k = threadIdx.x; k < (int)gridDim.x; k += kBlock)
        ep_merge(acc, ep_load_cg(reinterpret_cast<const EpAcc*>(s.red) + k), gamma);
    ep_block_reduce(acc, gamma);
    if (threadIdx.x == 0) {
        double* o = s.summary;
        o[STA_SUM_WNS_EARLY] = acc.wns_e;
        o[STA_SUM_TNS_EARLY] = acc.tns_e;
        o[STA_SUM_WNS_LATE] = acc.wns_l;
        o[STA_SUM_TNS_LATE] = acc.tns_l;
        o[STA_SUM_TNS_GAMMA] = lse ? acc.tns_g : 0.0;
        o[STA_SUM_WNS_GAMMA] =
            (lse && acc.wsum > 0.f) ? (double)acc.wmin - (double)gamma * log((double)acc.wsum) : (double)kInf;
        o[STA_SUM_LATE_VIOLATIONS] = acc.viol;
        o[STA_SUM_NUM_ENDPOINTS] = e1 - e0;
        *s.ep_count = 0;
    }
}

// Adjoint seeds at the endpoints: d loss / d ats = -(w_tns dTNS_g/ds + w_wns dWNS_g/ds).
__global__ void __launch_bounds__(kBlock) k_seed(DevNet g, DevState s, float gamma) {
    const float W = (float)s.summary[STA_SUM_WNS_GAMMA];
    const float wt = s.params[0], ww = s.params[1];
    for (int e = blockIdx.x * kBlock + threadIdx.x; e < g.E; e += gridDim.x * kBlock) {
        const int p = g.ep_pin[e];
        float4 con;
        ep_bounds(g, s, e, con);
        const float2 gl = ep_dloss(con, reinterpret_cast<const float2*>(s.ats)[p], gamma, W, wt, ww);
        reinterpret_cast<float2*>(s.g_ats)[p] = make_float2(-gl.x, -gl.y);
    }
}

// Propagated clock: the setup bound of a clocked endpoint holds its clock pin's
// early rising arrival, which (on a net driven by a startpoint) moves one for
// one with the pin's wire delay, so d loss / d bound enters the adjoint of the
// clock pin's rising LSE arrival, added where the arc step writes it.
__global__ void __launch_bounds__(kBlock) k_cap_seed(DevNet g, DevState s0, float gamma) {
    if (s0.active && (int)blockIdx.y >= *s0.active) return;  // a lane this call does not run
    const DevState s = lane_state(s0, blockIdx.y);            // one lane per grid row
    float W = (float)s.summary[STA_SUM_WNS_GAMMA];
    float wt = s.params[0], ww = s.params[1];
    for (int e = blockIdx.x * kBlock + threadIdx.x; e < g.E; e += gridDim.x * kBlock) {
        float4 con;
        const int k = ep_bounds(g, s, e, con);
        if (k < 0) continue;
        if (g.G > 1) {  // several netlists: the endpoint's own WNS_gamma and weights
            const int gi = g.pin_grp[g.ep_pin[e]];
            W = (float)s.summary[(size_t)gi * STA_SUM_COUNT + STA_SUM_WNS_GAMMA];
            wt = s.params[2 * gi];
            ww = s.params[2 * gi + 1];
        }
        const float2 gl = ep_dloss(con, reinterpret_cast<const float2*>(s.ats)[g.ep_pin[e]], gamma, W, wt, ww);
        s.cap_seed[k] = gl.x + gl.y;
    }
}

__global__ void k_set_weights(float* params, const float* w_dev, float w0, float w1) {
    if (w_dev) {
        params[0] = w_dev[0];
        params[1] = w_dev[1];
    } else {
        params[0] = w0;
        params[1] = w1;
    }
}

__global__ void __launch_bounds__(kBlock) k_scatter(DevNet g, const float* __restrict__ in, float* __restrict__ out,
                                                    int k, int np) {
    for (int i = blockIdx.x * kBlock + threadIdx.x; i < np * k; i += gridDim.x * kBlock) {
        const int p = i / k, q = i - p * k;
        out[(size_t)g.pin_orig[p] * k + q] = in[i];
    }
}

__global__ void __launch_bounds__(kBlock) k_pin_slack(DevNet g, DevState s, float2* __restrict__ out) {
    for (int p = blockIdx.x * kBlock + threadIdx.x; p < g.P; p += gridDim.x * kBlock) {
        const float4 at = reinterpret_cast<const float4*>(s.at)[p];
        const float4 rt = reinterpret_cast<const float4*>(s.rat)[p];
        out[g.pin_orig[p]] = make_float2(fminf(at.x - rt.x, at.y - rt.y), fminf(rt.z - at.z, rt.w - at.w));
    }
}

__global__ void __launch_bounds__(kBlock) k_init_ats(DevState s, int P) {
    for (int p = blockIdx.x * kBlock + threadIdx.x; p < P; p += gridDim.x * kBlock)
        reinterpret_cast<float2*>(s.ats)[p] = reinterpret_cast<const float2*>(s.at)[2 * p + 1];
}

int grid_for(long long n) {
    long long b = (n + kBlock - 1) / kBlock;
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

}  // namespace

void launch_gather_xy(const DevNet& g, const DevState& s, const float2* xy_user, int lanes, cudaStream_t st) {
    if (g.P == 0 && !s.active) return;
    k_gather_xy<<<dim3(grid_for(g.P), lanes), kBlock, 0, st>>>(g, s, xy_user);
}

void launch_rc(const DevNet& g, const DevState& s, int nw, cudaStream_t st) {
    const int blocks = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock + g.nrc;
    if (blocks == 0) return;
    k_rc<<<blocks, kBlock, 0, st>>>(g, s, nw);
}

void launch_fwd_level(const DevNet& g, const DevState& s, int w0, int nw, int c0, int nc, float gamma, int lse,
                      cudaStream_t st) {
    const int blocks = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock + nc;
    if (blocks == 0) return;
    k_fwd<<<blocks, kBlock, 0, st>>>(g, s, w0, nw, c0, nc, gamma, lse);
}

void launch_endpoints(const DevNet& g, const DevState& s, float gamma, int lse, cudaStream_t st, const DfState* d,
                      int P) {
    const dim3 grid = g.G > 1 ? dim3(g.ep_gx, g.G) : dim3(kEpBlocks, s.nl);
    if (d) k_ep<<<grid, kBlock, 0, st>>>(g, s, gamma, lse, d->pin_mask, P, d->apart, d->npart * kPartFloats);
    else k_ep<<<grid, kBlock, 0, st>>>(g, s, gamma, lse, nullptr, 0, nullptr, 0);
}

void launch_bwd_level(const DevNet& g, const DevState& s, int w0, int nw, int c0, int nc, float gamma, int mode,
                      cudaStream_t st) {
    const int blocks = (nw + kWarpsPerBlock - 1) / kWarpsPerBlock + nc;
    if (blocks == 0) return;
    k_bwd<<<blocks, kBlock, 0, st>>>(g, s, w0, nw, c0, nc, gamma, mode);
}

void launch_set_weights(const DevState& s, const float* w_dev, float w0, float w1, cudaStream_t st) {
    k_set_weights<<<1, 1, 0, st>>>(s.params, w_dev, w0, w1);
}

void launch_seed(const DevNet& g, const DevState& s, float gamma, cudaStream_t st) {
    if (g.E == 0) return;
    k_seed<<<grid_for(g.E), kBlock, 0, st>>>(g, s, gamma);
}

void launch_cap_seed(const DevNet& g, const DevState& s, float gamma, cudaStream_t st) {
    if (g.E == 0 || !g.ep_clk) return;
    k_cap_seed<<<dim3(grid_for(g.E), s.nl), kBlock, 0, st>>>(g, s, gamma);
}

void launch_scatter(const DevNet& g, const float* in, float* out, int k, int np, cudaStream_t st) {
    if (np == 0) return;
    k_scatter<<<grid_for((long long)np * k), kBlock, 0, st>>>(g, in, out, k, np);
}

void launch_pin_slack(const DevNet& g, const DevState& s, float* out, cudaStream_t st) {
    if (g.P == 0) return;
    k_pin_slack<<<grid_for(g.P), kBlock, 0, st>>>(g, s, reinterpret_cast<float2*>(out));
}

void launch_init_ats(const DevState& s, int P, cudaStream_t st) {
    if (P == 0) return;
    k_init_ats<<<grid_for(P), kBlock, 0, st>>>(s, P);
}

namespace {

// read every word once (brings a buffer smaller than L2 into L2)
__global__ void __launch_bounds__(kBlock) k_touch(const int32_t* __restrict__ a, long long n, int32_t* sink) {
    int32_t x = 0;
    for (long long i = blockIdx.x * (long long)kBlock + threadIdx.x; i < n; i += (long long)gridDim.x * kBlock)
        x ^= __ldcg(a + i);
    if (x == 0x7fffffff) *sink = x;  // keeps the loads
}

// one thread follows the cycle: every load's address is the previous load's value
__global__ void k_chase(const int32_t* __restrict__ next, int steps, int32_t* sink) {
    int32_t i = 0;
    for (int k = 0; k < steps; ++k) i = __ldcg(next + i);
    *sink = i;
}

}  // namespace

void launch_touch(const int32_t* a, long long n, int32_t* sink, cudaStream_t st) {
    if (n > 0) k_touch<<<grid_for(n), kBlock, 0, st>>>(a, n, sink);
}

void launch_chase(const int32_t* next, int steps, int32_t* sink, cudaStream_t st) {
    k_chase<<<1, 1, 0, st>>>(next, steps, sink);
}

}  // namespace sta
