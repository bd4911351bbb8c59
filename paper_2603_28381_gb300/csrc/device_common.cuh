// device_common.cuh -- device helpers shared by the level-by-level and the
// dataflow schedules (table lookup, driver-cell evaluation and adjoint,
// warp-task geometry, fixed-order reductions, wire step).
#pragma once

#include <cfloat>
#include <cmath>

#include "kernels.h"

namespace sta {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kInf = __builtin_huge_valf();

__device__ __forceinline__ unsigned lanes_upto(int lane) { return kFull >> (31 - lane); }

// largest k in [0,5] with idx[k] <= v (0 below the range): right-continuous
// segment of a 7-point table axis, extended linearly outside [idx0, idx6].
__device__ __forceinline__ int axis_seg(const float* __restrict__ idx, float v) {
    int k = 0;
#pragma unroll
    for (int j = 1; j <= 5; ++j) k += (__ldg(idx + j) <= v) ? 1 : 0;
    return k;
}

// bilinear inter/extrapolation of a 7x7 table [slew i][load j]
__device__ __forceinline__ float bilerp(const float* __restrict__ T, int i, int j, float ts, float ul) {
    const float* q = T + i * STA_LUT + j;
    const float t00 = __ldg(q), t01 = __ldg(q + 1), t10 = __ldg(q + STA_LUT), t11 = __ldg(q + STA_LUT + 1);
    const float r0 = fmaf(ul, t01 - t00, t00);
    const float r1 = fmaf(ul, t11 - t10, t10);
    return fmaf(ts, r1 - r0, r0);
}

__device__ __forceinline__ float bilerp_grad(const float* __restrict__ T, int i, int j, float ts, float ul,
                                             float inv_s, float inv_l, float& d_ds, float& d_dl) {
    const float* q = T + i * STA_LUT + j;
    const float t00 = __ldg(q), t01 = __ldg(q + 1), t10 = __ldg(q + STA_LUT), t11 = __ldg(q + STA_LUT + 1);
    const float r0 = fmaf(ul, t01 - t00, t00);
    const float r1 = fmaf(ul, t11 - t10, t10);
    d_ds = (r1 - r0) * inv_s;
    d_dl = fmaf(ts, (t11 - t10) - (t01 - t00), t01 - t00) * inv_l;
    return fmaf(ts, r1 - r0, r0);
}

// Corner-packed lookup: delay corners (t00, t01, t10, t11) and slew corners
// of cell (i, j) of the table of (type t, arc k, output transition rf), one
// 32-byte sector.
__device__ __forceinline__ void cell_corners(const DevNet& g, int t, int k, int rf, int i, int j, float4& dq,
                                             float4& sq) {
    const float4* c = g.lib_cell + ((((t * STA_MAX_ARCS + k) * 2 + rf) * 36 + i * 6 + j) * 2);
    dq = __ldg(c);
    sq = __ldg(c + 1);
}

// bilerp() on corners already loaded (same arithmetic, same result)
__device__ __forceinline__ float lerp_cell(float4 q, float ts, float ul) {
    const float r0 = fmaf(ul, q.y - q.x, q.x);
    const float r1 = fmaf(ul, q.w - q.z, q.z);
    return fmaf(ts, r1 - r0, r0);
}

__device__ __forceinline__ float lerp_cell_grad(float4 q, float ts, float ul, float inv_s, float inv_l, float& d_ds,
                                                float& d_dl) {
    const float r0 = fmaf(ul, q.y - q.x, q.x);
    const float r1 = fmaf(ul, q.w - q.z, q.z);
    d_ds = (r1 - r0) * inv_s;
    d_dl = fmaf(ts, (q.w - q.z) - (q.y - q.x), q.y - q.x) * inv_l;
    return fmaf(ts, r1 - r0, r0);
}

// Eq. 4 over a cell's arcs: m + gamma * log(sum_k exp((cand_k - m) / gamma)),
// stabilised by the maximum m of the na candidates (unused slots ignored).  The
// exponentials and the logarithm are the hardware base-2 forms (__expf, __logf)
// with the exponent scaled by 1/gamma: a few ulp of relative error, far below
// the parity tolerance, and a short chain of dependent instructions after a
// task's wait.  Every schedule evaluates it with these same operations.
__device__ __forceinline__ float lse_arcs(const float* cand, int na, float m, float gamma) {
    const float inv_g = 1.f / gamma;
    float sum = 0.f;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        const float e = __expf((cand[k] - m) * inv_g);
        sum += k < na ? e : 0.f;
    }
    return m + gamma * __logf(na > 0 ? sum : 1.f);
}

struct DrvOut {
    float at, slew, ats;
};

// Loads of values another warp of the same kernel produced go through L2
// only (ld.global.cg): an L1 line filled before the producer wrote would be
// stale.  Values produced by an earlier kernel use the ordinary path.
template <bool kCg>
__device__ __forceinline__ float ldx(const float* p) {
    if constexpr (kCg) return __ldcg(p);
    else return *p;
}

// Arrival time, slew and (late) LSE arrival time of net n's driver d for one
// condition c (Section 3.1.2; Eq. 4 for the LSE), given the net's load ld.
// Writes the arc delays if write_adel.
template <bool kCg>
__device__ DrvOut eval_driver(const DevNet& g, const DevState& s, int n, int d, int c, float ld, float gamma, bool lse,
                              bool write_adel = true) {
    DrvOut o;
    const int t = g.net_drv[n];
    if (t < 0) {  // asserted driver: constant values set at creation
        o.at = s.at[4 * d + c];
        o.slew = s.slew[4 * d + c];
        o.ats = c >= 2 ? s.ats[2 * d + c - 2] : 0.f;
        return o;
    }
    const int el = c >> 1, rf = c & 1;
    const int a0 = g.net_arc_ptr[n], a1 = g.net_arc_ptr[n + 1];
    const float* li = g.lib_idx + t * kLibStride + 8;
    const int jl = axis_seg(li, ld);
    const float ul = (ld - __ldg(li + jl)) * __ldg(g.lib_inv + t * kLibStride + 8 + jl);
    const float* si = g.lib_idx + t * kLibStride;
    const int un = g.lib_unate[t];
    float best_at = el ? -kInf : kInf, best_sl = el ? -kInf : kInf;
    float cand[STA_MAX_ARCS];
    float m = -kInf;
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        if (a0 + k < a1) {
            const int a = a0 + k, i = g.arc_pin[a];
            const int rfi = rf ^ ((un >> k) & 1);
            const float sin = ldx<kCg>(s.slew + 4 * i + 2 * el + rfi);
            const float ain = ldx<kCg>(s.at + 4 * i + 2 * el + rfi);
            const int is = axis_seg(si, sin);
            const float ts = (sin - __ldg(si + is)) * __ldg(g.lib_inv + t * kLibStride + is);
            const float* T = g.lib_tab + ((t * STA_MAX_ARCS + k) * 2 + rf) * kTabPerArcRf;
            const float D = bilerp(T, is, jl, ts, ul);
            const float S = bilerp(T + STA_LUT * STA_LUT, is, jl, ts, ul);
            if (write_adel) s.adel[4 * a + c] = D;
            if (el) {
                best_at = fmaxf(best_at, ain + D);
                best_sl = fmaxf(best_sl, S);
                if (lse) {
                    cand[k] = ldx<kCg>(s.ats + 2 * i + rfi) + D;
                    m = fmaxf(m, cand[k]);
                }
            } else {
                best_at = fminf(best_at, ain + D);
                best_sl = fminf(best_sl, S);
            }
        }
    }
    o.at = best_at;
    o.slew = best_sl;
    o.ats = 0.f;
    if (el && lse) {
        o.ats = lse_arcs(cand, a1 - a0, m, gamma);
    }
    return o;
}

// Adjoint of one late output transition rf of net n's driver cell.  Writes
// g_ats / g_slew of the cell's input pins (one writer per component) and
// returns this transition's contribution to d loss / d load.
__device__ float arc_adjoint(const DevNet& g, const DevState& s, int n, int d, int t, int rf, float GA, float GS,
                             float gamma) {
    const int a0 = g.net_arc_ptr[n], a1 = g.net_arc_ptr[n + 1];
    const float ld = s.load[n];
    const float* li = g.lib_idx + t * kLibStride + 8;
    const int jl = axis_seg(li, ld);
    const float inv_l = __ldg(g.lib_inv + t * kLibStride + 8 + jl);
    const float ul = (ld - __ldg(li + jl)) * inv_l;
    const float* si = g.lib_idx + t * kLibStride;
    const int un = g.lib_unate[t];
    const float atsd = s.ats[2 * d + rf];
    float best = -kInf, dss = 0.f, dsl = 0.f, gl = 0.f;
    int amax = -1;
    float gsl[STA_MAX_ARCS];
    int pin_c[STA_MAX_ARCS];
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k) {
        gsl[k] = 0.f;
        pin_c[k] = -1;
        if (a0 + k < a1) {
            const int a = a0 + k, i = g.arc_pin[a];
            const int rfi = rf ^ ((un >> k) & 1);
            const float sin = s.slew[4 * i + 2 + rfi];
            const int is = axis_seg(si, sin);
            const float inv_s = __ldg(g.lib_inv + t * kLibStride + is);
            const float ts = (sin - __ldg(si + is)) * inv_s;
            const float* T = g.lib_tab + ((t * STA_MAX_ARCS + k) * 2 + rf) * kTabPerArcRf;
            float dDs, dDl, dSs, dSl;
            bilerp_grad(T, is, jl, ts, ul, inv_s, inv_l, dDs, dDl);
            const float S = bilerp_grad(T + STA_LUT * STA_LUT, is, jl, ts, ul, inv_s, inv_l, dSs, dSl);
            const float D = s.adel[4 * a + 2 + rf];
            const float w = expf((s.ats[2 * i + rfi] + D - atsd) / gamma);
            const float gD = GA * w;
            // a capturing clock pin also carries its endpoint's setup term
            s.g_ats[2 * i + rfi] = (s.cap_seed && rfi == 0) ? gD + s.cap_seed[i] : gD;
            gsl[k] = gD * dDs;
            gl = fmaf(gD, dDl, gl);
            pin_c[k] = 2 * i + rfi;
            if (S > best) {
                best = S;
                amax = k;
                dss = dSs;
                dsl = dSl;
            }
        }
    }
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
        if (k == amax) gsl[k] = fmaf(GS, dss, gsl[k]);
    if (amax >= 0) gl = fmaf(GS, dsl, gl);
#pragma unroll
    for (int k = 0; k < STA_MAX_ARCS; ++k)
        if (pin_c[k] >= 0) s.g_slew[pin_c[k]] = gsl[k];
    return gl;
}

// ---------------------------------------------------------------------------
// Warp-task geometry: pins [pin0, pin0 + npins) of nets [n0, n0 + nn).
// ---------------------------------------------------------------------------
struct WarpGeom {
    int lane, pin0, npins, h;  // h: head offset of net `lane` (lane <= nn)
    unsigned heads;            // bit k set = pin0 + k is a driver
    int hd, j, last;           // for this lane's pin: driver offset, local net, last pin of its net
    bool valid;
};

__device__ __forceinline__ WarpGeom warp_geom(const DevNet& g, int n0, int nn) {
    WarpGeom w;
    w.lane = threadIdx.x & 31;
    w.pin0 = g.net_ptr[n0];
    w.h = (w.lane <= nn) ? g.net_ptr[n0 + w.lane] - w.pin0 : 0;
    w.npins = __shfl_sync(kFull, w.h, nn);
    w.heads = __reduce_or_sync(kFull, (w.lane < nn) ? (1u << w.h) : 0u);
    const unsigned upto = w.heads & lanes_upto(w.lane);
    w.hd = 31 - __clz(upto);
    w.j = __popc(upto) - 1;
    const unsigned after = w.heads & ~lanes_upto(w.lane);
    w.last = (after ? __ffs(after) - 1 : w.npins) - 1;
    w.valid = w.lane < w.npins;
    return w;
}

// fixed-order block reductions (256 threads)
template <typename Op>
__device__ __forceinline__ float block_reduce(float v, float* sh, Op op) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = op(v, __shfl_xor_sync(kFull, v, off));
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    float r = sh[0];
#pragma unroll
    for (int k = 1; k < kWarpsPerBlock; ++k) r = op(r, sh[k]);
    return r;
}

struct OpSum { __device__ float operator()(float a, float b) const { return a + b; } };
struct OpMax { __device__ float operator()(float a, float b) const { return fmaxf(a, b); } };
struct OpMin { __device__ float operator()(float a, float b) const { return fminf(a, b); } };

__device__ __forceinline__ float rc_sink(const DevNet& g, const DevState& s, int p, float2 xy, float2 xyd, float cap) {
    const float dist = fabsf(xy.x - xyd.x) + fabsf(xy.y - xyd.y);
    const float R = g.r * dist;
    const float C = fmaf(0.5f * g.c, dist, cap);
    const float D = R * C * kKrc;
    const float m = 2.f * R * C * D * kKrc - D * D;
    s.wdi[p] = make_float2(D, sqrtf(fmaxf(m, 0.f)));
    return fmaf(g.c, dist, cap);
}

// RC of one chunk of a large net's sinks (one 256-thread block): every sink's
// (delay, impulse) and the chunk's share of the load, reduced in a fixed order.
// A net's only chunk writes its load; otherwise the chunk stores its partial and
// the last chunk of the net to finish (a device-scope counter, reset by that
// chunk for the next launch) adds the partials in chunk order, so the load does
// not depend on which block finishes last.
__device__ __forceinline__ void rc_chunk(const DevNet& g, const DevState& s, int4 ck, int2 cn) {
    __shared__ float sh[kWarpsPerBlock];
    __shared__ int last;
    const int n = ck.x, d = g.net_ptr[n];
    const float2 xyd = s.xy[d];
    const int e = ck.y + ck.z;
    float acc = 0.f;
#pragma unroll 4
    for (int p = ck.y + threadIdx.x; p < e; p += kBlock) acc += rc_sink(g, s, p, s.xy[p], xyd, g.pin_cap[p]);
    acc = block_reduce(acc, sh, OpSum());
    if (ck.w < 0) {
        if (threadIdx.x == 0) s.load[n] = g.pin_cap[d] + acc;
        return;
    }
    if (threadIdx.x == 0) {
        s.rc_part[ck.w] = acc;
        __threadfence();
        last = atomicAdd(s.rc_count + cn.x, 1) == cn.y - 1;
    }
    __syncthreads();
    if (last && threadIdx.x == 0) {
        __threadfence();
        float sum = 0.f;
        for (int k = 0; k < cn.y; ++k) sum += __ldcg(s.rc_part + cn.x + k);
        s.load[n] = g.pin_cap[d] + sum;
        s.rc_count[cn.x] = 0;
    }
}

__device__ __forceinline__ void store_sink(const DevState& s, int p, const float* A, const float* S, float z0,
                                           float z1, bool lse) {
    const float2 w = s.wdi[p];
    const float i2 = w.y * w.y;
    reinterpret_cast<float4*>(s.at)[p] = make_float4(A[0] + w.x, A[1] + w.x, A[2] + w.x, A[3] + w.x);
    reinterpret_cast<float4*>(s.slew)[p] =
        make_float4(sqrtf(fmaf(S[0], S[0], i2)), sqrtf(fmaf(S[1], S[1], i2)), sqrtf(fmaf(S[2], S[2], i2)),
                    sqrtf(fmaf(S[3], S[3], i2)));
    if (lse) reinterpret_cast<float2*>(s.ats)[p] = make_float2(z0 + w.x, z1 + w.x);
}

struct SinkBwd {
    float r[4];      // RAT_s - Delay_s
    float ga[2];     // g_ats of the sink
    float gs[2];     // g_slew_s * slew_d / slew_s
    float gwire;     // d loss / d Delay_s + d loss / d Impulse_s
};

__device__ __forceinline__ SinkBwd sink_bwd(const DevState& s, int p, float2 sld, int mode) {
    SinkBwd b;
    const float2 w = s.wdi[p];
    if (mode & 1) {
        const float4 rr = reinterpret_cast<const float4*>(s.rat)[p];
        b.r[0] = rr.x - w.x;
        b.r[1] = rr.y - w.x;
        b.r[2] = rr.z - w.x;
        b.r[3] = rr.w - w.x;
    } else {
        b.r[0] = b.r[1] = -kInf;
        b.r[2] = b.r[3] = kInf;
    }
    b.ga[0] = b.ga[1] = b.gs[0] = b.gs[1] = b.gwire = 0.f;
    if (mode & 2) {
        const float2 ga = reinterpret_cast<const float2*>(s.g_ats)[p];
        const float2 gs = reinterpret_cast<const float2*>(s.g_slew)[p];
        const float2 sl = reinterpret_cast<const float2*>(s.slew)[2 * p + 1];
        const float q0 = sl.x > 0.f ? gs.x / sl.x : 0.f;
        const float q1 = sl.y > 0.f ? gs.y / sl.y : 0.f;
        b.ga[0] = ga.x;
        b.ga[1] = ga.y;
        b.gs[0] = q0 * sld.x;
        b.gs[1] = q1 * sld.y;
        b.gwire = ga.x + ga.y + (q0 + q1) * w.y;
    }
    return b;
}

// d loss / d (x, y) of sink p given d loss / d Load of its net (star RC).
__device__ __forceinline__ float2 sink_grad(const DevNet& g, const DevState& s, int p, float2 xy, float2 xyd, float gwire,
                                            float gload) {
    const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
    const float dist = fabsf(dx) + fabsf(dy);
    const float cap = g.pin_cap[p];
    // dDelay/dd = k r (cap + c d); on a star Eq. 3 gives Impulse = Delay, same slope
    const float gd = fmaf(gload, g.c, gwire * kKrc * g.r * fmaf(g.c, dist, cap));
    const float sx = (dx > 0.f) - (dx < 0.f), sy = (dy > 0.f) - (dy < 0.f);
    return make_float2(gd * sx, gd * sy);
}

// softmin_gamma(a, b, 0) = m - gamma log(sum exp(-(x - m) / gamma)), m = min
__device__ __forceinline__ float softmin3(float a, float b, float gamma) {
    const float m = fminf(fminf(a, b), 0.f);
    return m - gamma * logf(expf(-(a - m) / gamma) + expf(-(b - m) / gamma) + expf(m / gamma));
}


}  // namespace
}  // namespace sta
