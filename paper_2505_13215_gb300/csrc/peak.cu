// peak.cu -- throughput probes of the SM pipes the compositing kernels use.
//
// The compositing kernels are bound by FP32 arithmetic and the multi-function
// unit (base-2 exponential, reciprocal), not by memory.  Their roofline needs
// the ceiling of those pipes on the GPU at hand, measured rather than derived
// from unit counts: these kernels run long chains of one instruction each,
// with enough independent chains per thread that the pipe, not the latency
// of a chain, limits them.  splat_peak_probe launches one of them; the caller
// times it with CUDA events and divides the operation count by the time.
#include "splat_internal.cuh"

namespace splat {

constexpr int kProbeChains = 8;  // independent chains per thread

// fma.rn.f32 chains: x = x a + b converges to b / (1 - a), so no value overflows
// or becomes subnormal.  Counted as 2 FP32 operations per FMA.
__global__ void __launch_bounds__(256) k_probe_ffma(int iters, float a, float b, float* out)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.f) out[threadIdx.x] = s;  // keeps the chains alive; never true in practice
}

// fma.rn.f32x2 chains (two FP32 lanes per instruction), the packed form the
// compositing kernels use for pixel pairs.  4 FP32 operations per instruction.
__global__ void __launch_bounds__(256) k_probe_ffma2(int iters, float a, float b, float* out)
{
    float2 x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)(c - (int)threadIdx.x));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c].x + x[c].y;
    if (s == 12345.f) out[threadIdx.x] = s;
}

// ex2.approx.ftz.f32 chains: x = 2^-|x| (the sign bit set by a logic
// operation on the ALU pipe), which stays in (0, 1].
__global__ void __launch_bounds__(256) k_probe_ex2(int iters, float* out)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 0.1f * (float)c + 1e-3f * (float)(threadIdx.x & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            const float nx = __uint_as_float(__float_as_uint(x[c]) | 0x80000000u);
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(nx));
        }
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            const float nx = __uint_as_float(__float_as_uint(x[c]) | 0x80000000u);
            asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(nx));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.f) out[threadIdx.x] = s;
}

// rcp.approx.ftz.f32 chains: x = 1 / x', x' = x with its lowest mantissa bit
// flipped by a logic operation (two reciprocals in a row could otherwise be
// simplified away); x stays near x0 and 1 / x0.
__global__ void __launch_bounds__(256) k_probe_rcp(int iters, float* out)
{
    float x[kProbeChains];
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) x[c] = 1.5f + 0.1f * (float)c + 1e-3f * (float)(threadIdx.x & 31);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            const float nx = __uint_as_float(__float_as_uint(x[c]) ^ 1u);
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(nx));
        }
#pragma unroll
        for (int c = 0; c < kProbeChains; ++c) {
            const float nx = __uint_as_float(__float_as_uint(x[c]) ^ 1u);
            asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(x[c]) : "f"(nx));
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kProbeChains; ++c) s += x[c];
    if (s == 12345.f) out[threadIdx.x] = s;
}

}  // namespace splat

using namespace splat;

extern "C" double splat_peak_probe(int kind, int blocks, int iters, float* out, void* stream)
{
    if (blocks < 1 || iters < 1 || !out || kind < 0 || kind > 3) return -1.0;
    const cudaStream_t st = (cudaStream_t)stream;
    const double threads = (double)blocks * 256.0;
    double ops = 0.0;
    count_launch();
    switch (kind) {
    case SPLAT_PROBE_FFMA:
        k_probe_ffma<<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-3f, out);
        ops = threads * kProbeChains * iters * 2.0;
        break;
    case SPLAT_PROBE_FFMA2:
        k_probe_ffma2<<<blocks, 256, 0, st>>>(iters, 0.999f, 1e-3f, out);
        ops = threads * kProbeChains * iters * 4.0;
        break;
    case SPLAT_PROBE_EX2:
        k_probe_ex2<<<blocks, 256, 0, st>>>(iters, out);
        ops = threads * kProbeChains * iters * 2.0;
        break;
    default:
        k_probe_rcp<<<blocks, 256, 0, st>>>(iters, out);
        ops = threads * kProbeChains * iters * 2.0;
        break;
    }
    return cudaGetLastError() == cudaSuccess ? ops : -1.0;
}
