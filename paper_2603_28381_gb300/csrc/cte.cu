// cte.cu -- net RC (Eqs. 1-3) in the CTE scheme of Algorithm 2, kept as an
// ablation of the pin-based warp tasks.
//
// Collaborative task engagement: each thread of a block takes one net, the
// block turns the nets' workloads (one task per sink) into a shared task pool
// with a work-efficient (Blelloch) exclusive scan, and the threads then stride
// over the pool, each finding the net of its task by a binary search of the
// scan (lower bound) before doing the per-sink work.  The per-net load sums
// the sink terms of a warp's run of tasks with a shuffle scan and adds the run
// with one shared-memory atomic, so its rounding order is not fixed (the
// pin-based kernels sum in a fixed order).
#include "device_common.cuh"

namespace sta {
namespace {

constexpr int kCteNets = 256;  // nets per block (one per thread)

__global__ void __launch_bounds__(kCteNets) k_rc_cte(DevNet g, DevState s, int n0, int n1) {
    __shared__ int scan[kCteNets];
    __shared__ float load[kCteNets];
    __shared__ int first_pin[kCteNets];
    const int tid = threadIdx.x;
    const int base = n0 + blockIdx.x * kCteNets;
    const int n = base + tid;
    const bool has = n < n1;
    const int dp = has ? g.net_ptr[n] : 0;
    const int work = has ? g.net_ptr[n + 1] - dp - 1 : 0;  // one task per sink
    scan[tid] = work;
    load[tid] = 0.f;
    first_pin[tid] = dp;
    __syncthreads();
    // Blelloch scan: up-sweep ...
    for (int off = 1; off < kCteNets; off <<= 1) {
        const int i = (tid + 1) * off * 2 - 1;
        if (i < kCteNets) scan[i] += scan[i - off];
        __syncthreads();
    }
    const int total = scan[kCteNets - 1];
    __syncthreads();
    if (tid == 0) scan[kCteNets - 1] = 0;
    __syncthreads();
    // ... and down-sweep: scan[k] = tasks before net k
    for (int off = kCteNets / 2; off >= 1; off >>= 1) {
        const int i = (tid + 1) * off * 2 - 1;
        if (i < kCteNets) {
            const int t = scan[i - off];
            scan[i - off] = scan[i];
            scan[i] += t;
        }
        __syncthreads();
    }
    // threads stride over the pool; a warp iterates while any of its lanes has a task
    const int lane = tid & 31;
    for (int k0 = tid - lane; k0 < total; k0 += kCteNets) {
        const int task = k0 + lane;
        const bool ok = task < total;
        int lo = 0;
        float v = 0.f;
        if (ok) {
            // lower bound: the last net whose first task is <= task
            int hi = kCteNets - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (scan[mid] <= task) lo = mid;
                else hi = mid - 1;
            }
            const int d = first_pin[lo];
            const int p = d + 1 + (task - scan[lo]);
            v = rc_sink(g, s, p, s.xy[p], s.xy[d], g.pin_cap[p]);
        }
        // tasks of a warp are consecutive, so lanes of one net form runs: sum each
        // run with a segmented shuffle scan and add it with one atomic
        const int key = ok ? lo : -1 - lane;
        const int prev = __shfl_up_sync(kFull, key, 1);
        const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != key);
        const int hd = 31 - __clz(heads & (kFull >> (31 - lane)));
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const float u = __shfl_up_sync(kFull, v, off);
            if (lane - off >= hd) v += u;
        }
        const int next = __shfl_down_sync(kFull, key, 1);
        if (ok && (lane == 31 || next != key)) atomicAdd(&load[lo], v);
    }
    __syncthreads();
    if (has) s.load[n] = g.pin_cap[dp] + load[tid];
}

}  // namespace

void launch_rc_cte(const DevNet& g, const DevState& s, int n0, int n1, cudaStream_t st) {
    if (n1 <= n0) return;
    const int blocks = (n1 - n0 + kCteNets - 1) / kCteNets;
    k_rc_cte<<<blocks, kCteNets, 0, st>>>(g, s, n0, n1);
}

}  // namespace sta
