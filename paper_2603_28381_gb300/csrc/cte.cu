// cte.cu -- net RC (Eqs. 1-3) in the CTE scheme of Algorithm 2, kept as an
// ablation of the pin-based warp tasks.
//
// Collaborative task engagement: each thread of a block takes one net, the
// block turns the nets' workloads (one task per sink) into a shared task pool
// with a work-efficient (Blelloch) exclusive scan, and the threads then stride
// over the pool, each finding the net of its task by a binary search of the
// scan (lower bound) before doing the per-sink work.  The per-net load sums
// the sink terms with shared-memory atomics, so its rounding order is not
// fixed (the pin-based kernels sum in a fixed order).
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
    for (int task = tid; task < total; task += kCteNets) {
        // lower bound: the last net whose first task is <= task
        int lo = 0, hi = kCteNets - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (scan[mid] <= task) lo = mid;
            else hi = mid - 1;
        }
        const int d = first_pin[lo];
        const int p = d + 1 + (task - scan[lo]);
        const float2 xy = s.xy[p], xyd = s.xy[d];
        const float cap = g.pin_cap[p];
        const float v = rc_sink(g, s, p, xy, xyd, cap);
        atomicAdd(&load[lo], v);
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
