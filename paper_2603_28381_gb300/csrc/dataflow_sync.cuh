// dataflow_sync.cuh -- task queue, waits on data words, dependency counters
// and their bounds, for the persistent dataflow kernels (single-placement and
// batched schedules).
//
// A sweep's tasks are listed in a topological order and taken from a queue
// head (atomicAdd).  A task waits for the data it reads: words reset to
// kUnwritten before the sweep and written once (poll_words), or, for the
// gradient chunks of a large net, a counter its driver step increments with a
// release (wait_ready / signal_consumers).  A waiting warp only waits for tasks
// with smaller queue indices, which running warps hold, so a sweep always
// progresses; every wait is still bounded in time.
#pragma once

#include <cstdint>

#include <cuda_runtime.h>

#include "sta_internal.h"

namespace sta {
namespace {

constexpr unsigned long long kWaitBudgetNs = 1000000000ull;  // 1 s per wait

// pause between two polls of a wait (ns; a scheduling hint to the SM)
#ifndef STA_POLL_NS
#define STA_POLL_NS 128
#endif

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed(const int32_t* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Wait until cnt[t] reaches need (its producer count).  The whole warp polls
// the one counter together (the lanes read the same address, one transaction)
// with relaxed loads and acquires it once the count is reached; every branch
// is decided by a warp vote, so the warp never splits into a polling lane and
// waiting lanes (a split warp would run the rest of the task as separate
// groups).  Bounded: after kWaitBudgetNs, or once any wait of the launch has
// expired, it sets the abort word and returns (the host then reports
// STA_ERR_TIMEOUT).
__device__ __forceinline__ void wait_ready(const int32_t* cnt, int t, int need, int32_t* abort_word) {
    if (need <= 0) return;
    if (__all_sync(0xffffffffu, ld_acquire(cnt + t) >= need)) return;
    unsigned long long t0 = 0;
    for (unsigned it = 1;; ++it) {
        __nanosleep(STA_POLL_NS);
        if (__all_sync(0xffffffffu, ld_relaxed(cnt + t) >= need)) {
            (void)ld_acquire(cnt + t);
            return;
        }
        if ((it & 63) == 0) {
            if (__any_sync(0xffffffffu, ld_relaxed(abort_word) != 0)) return;
            const unsigned long long now = __shfl_sync(0xffffffffu, global_ns(), 0);
            if (t0 == 0) {
                t0 = now;
            } else if (now - t0 > kWaitBudgetNs) {
                if ((threadIdx.x & 31) == 0) {
                    atomicExch(abort_word, 1);      // ends the other waits of this launch
                    atomicExch(abort_word + 1, 1);  // sticky until the host reports it
                }
                __syncwarp();
                return;
            }
        }
    }
}


// ---- waiting on data words -------------------------------------------------
// A word that a sweep's tasks poll is set to kUnwritten (a NaN) before the
// sweep and written exactly once during it with a strong relaxed store; a
// waiting task loads it with strong relaxed loads until it holds a value.  A
// word carries its own value, so no fence or counter is needed, and by
// per-location coherence a word once seen written stays written for the thread.
__device__ __forceinline__ float ld_relaxed_f(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_f(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

__device__ __forceinline__ bool written(float v) { return __float_as_uint(v) != kUnwritten; }

// Poll until ready() holds on every lane of the warp (ready() reloads the
// lane's words each call).  Bounded like wait_ready: after kWaitBudgetNs, or
// once any wait of the launch has expired, it sets the abort words and returns.
template <typename F>
__device__ __forceinline__ void poll_words(F&& ready, int32_t* abort_word) {
    unsigned long long t0 = 0;
    for (unsigned it = 0;; ++it) {
        if (__all_sync(0xffffffffu, ready())) return;
        __nanosleep(STA_POLL_NS);
        if ((it & 63) == 63) {
            if (__any_sync(0xffffffffu, ld_relaxed(abort_word) != 0)) return;
            const unsigned long long now = __shfl_sync(0xffffffffu, global_ns(), 0);
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

__device__ __forceinline__ int grab(int32_t* head) {
    int t = 0;
    if ((threadIdx.x & 31) == 0) t = atomicAdd(head, 1);
    return __shfl_sync(0xffffffffu, t, 0);
}

__device__ __forceinline__ void red_release_add(int32_t* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Signal the task's consumers: one release increment per consumer, after a
// warp barrier, so every lane's stores happen before each increment (the
// barrier orders the lanes, the release makes their writes visible at GPU
// scope to whoever acquires the counter).
__device__ __forceinline__ void signal_consumers(int32_t* cnt, const int32_t* out_ptr, const int32_t* out, int t) {
    __syncwarp();
    const int k1 = out_ptr[t + 1];
    for (int k = out_ptr[t] + (int)(threadIdx.x & 31); k < k1; k += 32) red_release_add(cnt + out[k], 1);
}

// cooperative launch: every block of the grid is resident at once (the waits
// rely on it); `grid` must not exceed the kernel's co-resident block count.  A
// refused launch returns its error, which also stays the thread's last runtime
// error for the caller's check after the launch.
template <typename K, typename... Args>
cudaError_t launch_coop(K kernel, int grid, int block, size_t smem, cudaStream_t st, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}


}  // namespace
}  // namespace sta
