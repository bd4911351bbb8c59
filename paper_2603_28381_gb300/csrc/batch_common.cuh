// batch_common.cuh -- device helpers shared by the batched sweeps of
// batch.cu (a lane per placement and timing condition) and batch_wide.cu (a
// lane per placement, all four conditions), so that both compute every value
// with the same operations in the same order.
#pragma once

#include "dataflow_sync.cuh"
#include "device_common.cuh"

namespace sta {
namespace {

// per-placement state is pin-major, placement-minor: value[row * Bp + b]
__device__ __forceinline__ size_t ix(int row, int Bp, int b) { return (size_t)row * Bp + b; }

// Strong relaxed load / store of a polled word without a compiler memory
// barrier.  A batched task takes each polled value from the poll itself and
// never reads data that another word's store publishes (the one such hand-off,
// a large net's d loss / d load, goes through wait_ready's acquire), so the
// compiler may issue the task's independent plain loads and arithmetic across
// these; the accesses themselves stay in program order (volatile).
__device__ __forceinline__ float ld_poll(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p));
    return v;
}

__device__ __forceinline__ void st_poll(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v));
}

// the first of n consecutive queue entries for the warp
__device__ __forceinline__ int grab_n(int32_t* head, int n) {
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(head, n);
    return __shfl_sync(0xffffffffu, t, 0);
}

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

// slew segment and fraction from registers (same result as axis_seg)
__device__ __forceinline__ void seg_reg(const float* sidx, const float* sinv, float v, int& is, float& ts) {
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

// the smoothed loss's endpoint seed terms of one placement
struct BSeed {
    float W, wt, ww;  // WNS_gamma of this placement, w_tns, w_wns
};

// d loss / d (x, y) of a sink from its wire adjoint and the net's d loss / d load
__device__ __forceinline__ float2 bsink_grad(const DevNet& g, float2 xy, float2 xyd, float cap, float gwire,
                                             float gload) {
    const float dx = xy.x - xyd.x, dy = xy.y - xyd.y;
    const float gd = fmaf(gload, g.c, gwire * kKrc * g.r * fmaf(g.c, fabsf(dx) + fabsf(dy), cap));
    return make_float2(gd * ((dx > 0.f) - (dx < 0.f)), gd * ((dy > 0.f) - (dy < 0.f)));
}

}  // namespace
}  // namespace sta
