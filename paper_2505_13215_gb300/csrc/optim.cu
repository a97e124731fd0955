// optim.cu -- the parameter update of a training step: one Adam step over
// every field of both parameter sets in a single launch, and the storage cast
// (FP32 master values -> the dtype the rasterizer reads).
//
// Layout: a "segment" is one field of one set, n rows x width floats, dense.
// The grid is (blocks, segments); each thread walks its segment four floats at
// a time (float4 loads where the segment allows it).  Every float is read and
// written once: gradient, master value, m, v in (16 B), master, m, v and the
// storage copy out (12 B + the storage element size), so the kernel is
// HBM-bound.
#include <cmath>

#include "splat_internal.cuh"

namespace splat {

constexpr int kMaxSegs = 11;
constexpr int kOptThreads = 256;

struct OptSeg {
    float* p;         // FP32 master values
    float* m;         // first moments
    float* v;         // second moments
    const float* g;   // gradient
    void* st;         // storage copy (dtype), may equal p for FP32 storage
    int64_t n;        // floats in the segment
    float lr;         // step size of the segment's floats
    float lr_rest;    // SH segments: step size of the coefficients of degree >= 1
    int sh;           // SH fields: floats per row (the first 3 of a row are the degree-0, time-constant
                      // coefficients, which take lr); 0 for the other fields
};

struct OptArgs {
    OptSeg seg[kMaxSegs];
    int nseg;
    int dtype;        // storage dtype of every segment
    float b1, b2, eps;
    float c1, c2;     // 1 / (1 - b1^t), 1 / (1 - b2^t)
    int32_t* status;
};

template <int DT>
__device__ __forceinline__ void store_one(void* st, int64_t i, float x)
{
    using S = Storage<DT>;
    ((typename S::T*)st)[i] = S::from(x);
}

// Kingma and Ba (2015), Algorithm 1, one element
__device__ __forceinline__ float adam_one(const OptArgs& a, float lr, float g, float& m, float& v, float p)
{
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * (g * g);
    const float mh = m * a.c1, vh = v * a.c2;
    return p - lr * mh / (sqrtf(vh) + a.eps);
}

template <int DT>
__global__ void __launch_bounds__(kOptThreads) k_adam(OptArgs a)
{
    if (status_failed(a.status)) return;
    const OptSeg s = a.seg[blockIdx.y];
    const int64_t n4 = s.n / 4;
    const bool vec = ((uintptr_t)s.p | (uintptr_t)s.m | (uintptr_t)s.v | (uintptr_t)s.g) % 16 == 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < (vec ? n4 : 0); q += stride) {
        const float4 g = ((const float4*)s.g)[q];
        float4 m = ((float4*)s.m)[q], v = ((float4*)s.v)[q];
        float4 p = ((float4*)s.p)[q];
        float lr[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) lr[k] = (s.sh && (4 * q + k) % s.sh >= 3) ? s.lr_rest : s.lr;
        p.x = adam_one(a, lr[0], g.x, m.x, v.x, p.x);
        p.y = adam_one(a, lr[1], g.y, m.y, v.y, p.y);
        p.z = adam_one(a, lr[2], g.z, m.z, v.z, p.z);
        p.w = adam_one(a, lr[3], g.w, m.w, v.w, p.w);
        ((float4*)s.m)[q] = m;
        ((float4*)s.v)[q] = v;
        ((float4*)s.p)[q] = p;
        if (s.st != (void*)s.p) {
            store_one<DT>(s.st, 4 * q + 0, p.x);
            store_one<DT>(s.st, 4 * q + 1, p.y);
            store_one<DT>(s.st, 4 * q + 2, p.z);
            store_one<DT>(s.st, 4 * q + 3, p.w);
        }
    }
    // the floats a float4 walk does not cover (all of them when unaligned)
    for (int64_t i = (vec ? 4 * n4 : 0) + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n; i += stride) {
        const float lr = (s.sh && i % s.sh >= 3) ? s.lr_rest : s.lr;
        float m = s.m[i], v = s.v[i];
        const float p = adam_one(a, lr, s.g[i], m, v, s.p[i]);
        s.m[i] = m;
        s.v[i] = v;
        s.p[i] = p;
        if (s.st != (void*)s.p) store_one<DT>(s.st, i, p);
    }
}

template <int DT>
__global__ void __launch_bounds__(kOptThreads) k_cast(OptArgs a)
{
    const OptSeg s = a.seg[blockIdx.y];
    if (s.st == (void*)s.p) return;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < s.n; i += (int64_t)gridDim.x * blockDim.x)
        store_one<DT>(s.st, i, s.p[i]);
}

static int opt_blocks(const OptArgs& a, const LaunchCtx& ctx)
{
    int64_t mx = 1;
    for (int k = 0; k < a.nseg; ++k) mx = a.seg[k].n > mx ? a.seg[k].n : mx;
    const int64_t want = (mx / 4 + kOptThreads - 1) / kOptThreads;
    const int64_t cap = (int64_t)ctx.num_sms * 4;
    return (int)(want < 1 ? 1 : (want > cap ? cap : want));
}

cudaError_t launch_adam(const OptArgs& a, const LaunchCtx& ctx)
{
    if (a.nseg == 0) return cudaSuccess;
    const dim3 grid(opt_blocks(a, ctx), a.nseg);
    count_launch();
    switch (a.dtype) {
    case SPLAT_F32: k_adam<SPLAT_F32><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    case SPLAT_BF16: k_adam<SPLAT_BF16><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    default: k_adam<SPLAT_F16><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_cast(const OptArgs& a, const LaunchCtx& ctx)
{
    if (a.nseg == 0) return cudaSuccess;
    const dim3 grid(opt_blocks(a, ctx), a.nseg);
    count_launch();
    switch (a.dtype) {
    case SPLAT_F32: k_cast<SPLAT_F32><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    case SPLAT_BF16: k_cast<SPLAT_BF16><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    default: k_cast<SPLAT_F16><<<grid, kOptThreads, 0, ctx.stream>>>(a); break;
    }
    return cudaGetLastError();
}

}  // namespace splat
