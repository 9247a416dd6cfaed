// kernels_probe.cu -- throughput probe of the FP32 pipe.  Not part of the method: it gives
// the measured FP32 peak that the window reuse kernel (K^2 pair densities, bound by FP32
// arithmetic) is rated against.
//
// Every thread runs kChains independent fused multiply-add chains, so each scheduler always
// has ready FMAs (the FMA latency is covered by the chains of one warp and by the warps of
// the SM); a loop trip issues kChains FMAs against three loop-control instructions.  The
// paired variant issues fma.rn.f32x2 (two lanes' worth of FMAs per instruction, Blackwell),
// which shows whether the pipe or the instruction issue limits scalar FP32 code.
#include <cuda_runtime.h>

#include <cstdint>

#include "occ_kernels.h"
#include "occ_path.cuh"

namespace occ {
namespace {

constexpr int kChains = 16;
constexpr int kProbeThreads = 256;

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float2 unpack2(unsigned long long v) {
    float a, b;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
    return make_float2(a, b);
}

template <bool PAIRED>
__global__ void __launch_bounds__(kProbeThreads) k_fp32_peak(int iters, float* sink) {
    // multiplier just below 1 and a tiny addend: the chains stay finite and normal
    const float m = 0.99999988f, c = 1.0e-7f;
    const float seed = (float)(threadIdx.x + 1) * 1.0e-3f;
    float acc = 0.0f;
    if (PAIRED) {
        unsigned long long a[kChains];
        const unsigned long long mm = pack2(m, m), cc = pack2(c, c);
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = pack2(seed + (float)i, seed - (float)i);
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(a[i]) : "l"(mm), "l"(cc));
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) {
            const float2 v = unpack2(a[i]);
            acc += v.x + v.y;
        }
    } else {
        float a[kChains];
#pragma unroll
        for (int i = 0; i < kChains; ++i) a[i] = seed + (float)i;
        for (int it = 0; it < iters; ++it) {
#pragma unroll
            for (int i = 0; i < kChains; ++i)
                asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(a[i]) : "f"(m), "f"(c));
        }
#pragma unroll
        for (int i = 0; i < kChains; ++i) acc += a[i];
    }
    sink[(size_t)blockIdx.x * kProbeThreads + threadIdx.x] = acc;
}

// Streaming ceiling of the group reuse kernel's memory pattern (4 x 2 groups, FP32): the
// same CTA shape (4 warps side by side, each warp 16 x 2 pixels), the same loads (G-buffer
// position and normal and record plane 0 for every pixel, record plane 1 for pixels whose
// ray hit) and the same 4-byte store per pixel, with no arithmetic beyond a sum that keeps
// the loads alive.  Its time is what the group kernel's bytes cost on their own.
__global__ void __launch_bounds__(128) k_stream_ceiling(GBufView gb, RecView rec, float* out) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 3, m = lane & 7;
    const int x = (blockIdx.x * 4 + warp) * 16 + g * 4 + (m & 3);
    const int y = blockIdx.y * 2 + (m >> 2);
    if (x >= gb.W || y >= gb.H) return;
    const int i = y * gb.W + x, gi = gb_index(gb, x, y);
    const float4 P = __ldg(gb.pos + gi), N = __ldg(gb.nrm + gi), R0 = __ldg(rec.r0 + i);
    float4 R1 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (P.w != 0.0f && __float_as_int(R0.w) >= 0) R1 = __ldg(rec.r1 + i);
    out[i] = P.x + N.y + R0.z + R1.x;
}

}  // namespace

cudaError_t launch_stream_ceiling(const GBufView& gb, const RecView& rec, float* out,
                                  cudaStream_t s) {
    if (gb.W <= 0 || gb.H <= 0) return cudaSuccess;
    const dim3 grid((unsigned)((gb.W + 63) / 64), (unsigned)((gb.H + 1) / 2));
    k_stream_ceiling<<<grid, 128, 0, s>>>(gb, rec, out);
    return cudaGetLastError();
}

cudaError_t launch_fp32_peak(int paired, int iters, int blocks, float* sink, double* flop,
                             cudaStream_t s) {
    *flop = 2.0 * (paired ? 2.0 : 1.0) * kChains * (double)iters * kProbeThreads * blocks;
    if (paired)
        k_fp32_peak<true><<<blocks, kProbeThreads, 0, s>>>(iters, sink);
    else
        k_fp32_peak<false><<<blocks, kProbeThreads, 0, s>>>(iters, sink);
    return cudaGetLastError();
}

}  // namespace occ
