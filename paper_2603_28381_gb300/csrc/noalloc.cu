// noalloc.cu -- allocation-free endpoint summary.
//
// Some callers cannot call cudaMalloc: code that runs while a stream is being
// captured into a CUDA graph (allocation is not a capturable operation), and
// processes whose device memory is fully reserved by another framework's pool
// allocator, where a driver allocation would fail or stall the pool.  This
// entry point serves them: it computes the same endpoint slacks, WNS, TNS and
// smoothed TNS/WNS as the reduction inside sta_forward, from per-pin arrays the
// caller already holds, and it allocates nothing.  Its only scratch is the
// file-scope device array below (per-block partials of the reduction).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "sta.h"

namespace sta {
void set_last_error_text(const std::string& msg);  // capi.cu: text for sta_last_error()
}

namespace {

constexpr int kNaBlock = 256;
constexpr int kNaMaxParts = STA_NOALLOC_MAX_ENDPOINTS / kNaBlock;

struct NaAcc {
    double tns_e, tns_l, tns_g, count;  // sums in double, fixed order
    float wns_e, wns_l, wmin, wsum;     // wsum = sum exp(-(s - wmin) / gamma)
    double viol, pad;
};

// The scratch: one partial per block of 256 endpoints.  Every GPU that loads
// libsta holds it (about 1 MiB) until the process exits.  Host code must not
// pass this name to a kernel (on the host it is only a stand-in); the device
// address comes from cudaGetSymbolAddress in na_scratch().
static __device__ __align__(256) NaAcc g_na_partials[kNaMaxParts];

__device__ __forceinline__ NaAcc na_identity() {
    NaAcc a;
    a.tns_e = a.tns_l = a.tns_g = a.count = a.viol = a.pad = 0.0;
    a.wns_e = a.wns_l = a.wmin = __builtin_huge_valf();
    a.wsum = 0.f;
    return a;
}

__device__ __forceinline__ void na_merge(NaAcc& a, const NaAcc& b, float gamma) {
    a.tns_e += b.tns_e;
    a.tns_l += b.tns_l;
    a.tns_g += b.tns_g;
    a.count += b.count;
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

__device__ void na_block_reduce(NaAcc& acc, float gamma) {
    __shared__ NaAcc sh[kNaBlock];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int stride = kNaBlock / 2; stride > 0; stride >>= 1) {
        if ((int)threadIdx.x < stride) na_merge(sh[threadIdx.x], sh[threadIdx.x + stride], gamma);
        __syncthreads();
    }
    acc = sh[0];
}

// One block per 256 endpoints: slacks and the block's partial.  An endpoint
// whose pin index (or capturing clock pin) is outside [0, num_pins) gets NaN
// slacks and is left out.  With a capturing clock pin k the hold bound adds k's
// late rising arrival and the setup bound its early rising arrival (the latest
// and the earliest capture edge), as in sta_forward.
__global__ void __launch_bounds__(kNaBlock) k_na_part(const float4* __restrict__ at, const float2* __restrict__ ats,
                                                      int num_pins, const int32_t* __restrict__ end_pins,
                                                      const float4* __restrict__ end_rat,
                                                      const int32_t* __restrict__ end_clk, int num_end, float gamma,
                                                      float2* __restrict__ ep_slack, NaAcc* __restrict__ parts) {
    NaAcc acc = na_identity();
    const int e = blockIdx.x * kNaBlock + threadIdx.x;
    if (e < num_end) {
        const int p = end_pins[e];
        const int k = end_clk ? end_clk[e] : -1;
        if (p >= 0 && p < num_pins && k < num_pins) {
            float4 con = end_rat[e];
            if (k >= 0) {
                const float4 ck = at[k];
                con.x += ck.z;
                con.y += ck.z;
                con.z += ck.x;
                con.w += ck.x;
            }
            const float4 a = at[p];
            const float se = fminf(a.x - con.x, a.y - con.y);
            const float sl = fminf(con.z - a.z, con.w - a.w);
            ep_slack[e] = make_float2(se, sl);
            acc.count = 1.0;
            acc.wns_e = se;
            acc.wns_l = sl;
            acc.tns_e = fminf(se, 0.f);
            acc.tns_l = fminf(sl, 0.f);
            acc.viol = sl < 0.f ? 1.0 : 0.0;
            if (ats) {
                const float2 z = ats[p];
                const float sr = con.z - z.x, sf = con.w - z.y;
                const float m = fminf(fminf(sr, sf), 0.f);
                acc.tns_g = m - gamma * logf(expf(-(sr - m) / gamma) + expf(-(sf - m) / gamma) + expf(m / gamma));
                acc.wmin = fminf(sr, sf);
                acc.wsum = expf(-(sr - acc.wmin) / gamma) + expf(-(sf - acc.wmin) / gamma);
            }
        } else {
            ep_slack[e] = make_float2(__int_as_float(0x7fc00000), __int_as_float(0x7fc00000));
        }
    }
    na_block_reduce(acc, gamma);
    if (threadIdx.x == 0) parts[blockIdx.x] = acc;
}

// One block combines the partials this call wrote, in a fixed order.
__global__ void __launch_bounds__(kNaBlock) k_na_final(const NaAcc* __restrict__ parts, int nparts, float gamma,
                                                       int lse, double* __restrict__ summary) {
    NaAcc acc = na_identity();
    for (int i = threadIdx.x; i < nparts; i += kNaBlock) na_merge(acc, parts[i], gamma);
    na_block_reduce(acc, gamma);
    if (threadIdx.x == 0) {
        summary[STA_SUM_WNS_EARLY] = acc.wns_e;
        summary[STA_SUM_TNS_EARLY] = acc.tns_e;
        summary[STA_SUM_WNS_LATE] = acc.wns_l;
        summary[STA_SUM_TNS_LATE] = acc.tns_l;
        summary[STA_SUM_TNS_GAMMA] = lse ? acc.tns_g : 0.0;
        summary[STA_SUM_WNS_GAMMA] = (lse && acc.wsum > 0.f) ? (double)acc.wmin - (double)gamma * log((double)acc.wsum)
                                                             : (double)__builtin_huge_valf();
        summary[STA_SUM_LATE_VIOLATIONS] = acc.viol;
        summary[STA_SUM_NUM_ENDPOINTS] = acc.count;
    }
}

StaStatus na_fail(StaStatus st, const std::string& msg) {
    sta::set_last_error_text(msg);
    return st;
}

// Device address of the scratch for the current device.  Looked up on every
// call (a host query once the module is loaded), so a device reset or a new
// primary context between calls never leaves a stale address behind.
StaStatus na_scratch(NaAcc** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_na_partials);
    if (e != cudaSuccess || !p)
        return na_fail(STA_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    *out = static_cast<NaAcc*>(p);
    return STA_OK;
}

bool na_aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

extern "C" {

StaStatus sta_endpoint_summary_noalloc(const float* at, const float* ats, int32_t num_pins, const int32_t* end_pins,
                                       const float* end_rat, const int32_t* end_clk, int32_t num_end, float gamma,
                                       float* ep_slack, double* summary, void* stream) {
    if (num_pins < 0 || num_end < 0) return na_fail(STA_ERR_INVALID_ARG, "negative size");
    if (num_end > STA_NOALLOC_MAX_ENDPOINTS)
        return na_fail(STA_ERR_INVALID_ARG, "num_end " + std::to_string(num_end) + " exceeds STA_NOALLOC_MAX_ENDPOINTS (" +
                                                std::to_string(STA_NOALLOC_MAX_ENDPOINTS) + ")");
    if (!summary || (num_end > 0 && (!at || !end_pins || !end_rat || !ep_slack)))
        return na_fail(STA_ERR_INVALID_ARG, "null argument");
    // the kernels read at / end_rat as float4, ats as float2 and write ep_slack
    // as float2: a misaligned view (a sliced tensor) would fault on the device
    if (!na_aligned(at, 16) || !na_aligned(end_rat, 16) || !na_aligned(ats, 8) || !na_aligned(ep_slack, 8) ||
        !na_aligned(summary, 8) || !na_aligned(end_pins, 4) || !na_aligned(end_clk, 4))
        return na_fail(STA_ERR_INVALID_ARG,
                       "misaligned pointer: at and end_rat need 16 bytes, ats, ep_slack and summary 8, "
                       "end_pins and end_clk 4");
    if (ats && !(std::isfinite(gamma) && gamma > 0.f)) return na_fail(STA_ERR_INVALID_ARG, "gamma must be > 0");
    if (!ats) gamma = 1.f;
    NaAcc* parts = nullptr;
    StaStatus st = na_scratch(&parts);
    if (st != STA_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nparts = (num_end + kNaBlock - 1) / kNaBlock;
    if (nparts > 0)
        k_na_part<<<nparts, kNaBlock, 0, s>>>(reinterpret_cast<const float4*>(at), reinterpret_cast<const float2*>(ats),
                                              num_pins, end_pins, reinterpret_cast<const float4*>(end_rat), end_clk,
                                              num_end, gamma, reinterpret_cast<float2*>(ep_slack), parts);
    k_na_final<<<1, kNaBlock, 0, s>>>(parts, nparts, gamma, ats ? 1 : 0, summary);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return na_fail(STA_ERR_CUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return STA_OK;
}

}  // extern "C"
