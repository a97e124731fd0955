// convert.cu -- Sec. 4.1 static/dynamic identification and Sec. 4.2 4D -> 3D
// conversion.
//
// A 4D Gaussian is static when exp(s_t) > tau.  Its spatial part
// (mu_x, q_3D, s_x, s_y, s_z, opacity, SH) is appended to the 3D set, where
// q_3D is the quaternion of the top-left 3x3 block of R_4D (Eq. 4) by Eq. 9;
// mu_t and s_t are dropped.  The remaining 4D Gaussians are compacted,
// order preserved.  Three passes: per-block counts, one-block scan of the
// counts (+ capacity check), scatter into the 3D tail and a workspace copy of
// the kept 4D rows, then a copy back.
#include <algorithm>

#include "splat_internal.cuh"

namespace splat {

constexpr int kConvThreads = 256;
constexpr int kConvItems = 4;
constexpr int kConvBlock = kConvThreads * kConvItems;

template <int DT>
__device__ __forceinline__ bool is_static(const splat_g4& g4, int64_t i, float tau)
{
    using S = Storage<DT>;
    const float st = S::ld((const typename S::T*)g4.log_scale + i * 4 + 3);
    return expf(st) > tau;
}

template <int DT>
__global__ void __launch_bounds__(kConvThreads) k_conv_count(splat_g4 g4, float tau, uint32_t* block_counts)
{
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kConvBlock;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < kConvItems; ++k) {
        const int64_t i = base + k * kConvThreads + threadIdx.x;
        if (i < g4.n && is_static<DT>(g4, i, tau)) ++c;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(&s_cnt, c);
    __syncthreads();
    if (threadIdx.x == 0) block_counts[blockIdx.x] = s_cnt;
}

// One block: exclusive scan of the block counts in place, total -> n_moved.
__global__ void __launch_bounds__(1024) k_conv_scan(uint32_t* block_counts, int64_t nb, int64_t n3, int64_t cap3,
                                                   int64_t* n_moved, int32_t* status)
{
    __shared__ unsigned long long s_carry;
    __shared__ unsigned long long s_warp[32];
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t i = b0 + threadIdx.x;
        const unsigned long long v = i < nb ? block_counts[i] : 0ull;
        unsigned long long x = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[warp] = x;
        __syncthreads();
        unsigned long long wbase = 0, tot = 0;
        for (int w = 0; w < 32; ++w) {
            if (w < warp) wbase += s_warp[w];
            tot += s_warp[w];
        }
        const unsigned long long carry = s_carry;
        if (i < nb) block_counts[i] = (uint32_t)(carry + wbase + x - v);
        __syncthreads();
        if (threadIdx.x == 0) s_carry = carry + tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int64_t moved = (int64_t)s_carry;
        *n_moved = moved;
        if (n3 + moved > cap3) set_status(status, SPLAT_ERR_CAPACITY, SPLAT_STAGE_CONVERT, n3 + moved);
    }
}

// Eq. 9 on a (not necessarily orthonormal) 3x3 block, 1-based R(i,j); the
// largest-diagonal branch of Shepperd's method when 1 + tr(R) <= 1e-2.
__device__ __forceinline__ void matrix_to_quat(const float R[9], float q[4])
{
#define RR(i, j) R[((i) - 1) * 3 + ((j) - 1)]
    const float tr = RR(1, 1) + RR(2, 2) + RR(3, 3);
    float w, x, y, z;
    if (1.f + tr > 1e-2f) {
        w = 0.5f * sqrtf(1.f + tr);
        const float i4w = 1.f / (4.f * w);
        x = (RR(3, 2) - RR(2, 3)) * i4w;
        y = (RR(1, 3) - RR(3, 1)) * i4w;
        z = (RR(2, 1) - RR(1, 2)) * i4w;
    } else if (RR(1, 1) >= RR(2, 2) && RR(1, 1) >= RR(3, 3)) {
        x = 0.5f * sqrtf(fmaxf(0.f, 1.f + RR(1, 1) - RR(2, 2) - RR(3, 3)));
        const float i4 = 1.f / (4.f * x);
        w = (RR(3, 2) - RR(2, 3)) * i4;
        y = (RR(1, 2) + RR(2, 1)) * i4;
        z = (RR(1, 3) + RR(3, 1)) * i4;
    } else if (RR(2, 2) >= RR(3, 3)) {
        y = 0.5f * sqrtf(fmaxf(0.f, 1.f - RR(1, 1) + RR(2, 2) - RR(3, 3)));
        const float i4 = 1.f / (4.f * y);
        w = (RR(1, 3) - RR(3, 1)) * i4;
        x = (RR(1, 2) + RR(2, 1)) * i4;
        z = (RR(2, 3) + RR(3, 2)) * i4;
    } else {
        z = 0.5f * sqrtf(fmaxf(0.f, 1.f - RR(1, 1) - RR(2, 2) + RR(3, 3)));
        const float i4 = 1.f / (4.f * z);
        w = (RR(2, 1) - RR(1, 2)) * i4;
        x = (RR(1, 3) + RR(3, 1)) * i4;
        y = (RR(2, 3) + RR(3, 2)) * i4;
    }
#undef RR
    const float in = rsqrtf(w * w + x * x + y * y + z * z) * (w < 0.f ? -1.f : 1.f);
    q[0] = w * in; q[1] = x * in; q[2] = y * in; q[3] = z * in;
}

struct ConvTmp {  // workspace copy of the kept 4D rows (storage dtype)
    void *mean, *log_scale, *ql, *qr, *opacity, *sh;
};

template <int DT>
__global__ void __launch_bounds__(kConvThreads) k_conv_scatter(splat_g4 g4, splat_g3 g3, float tau,
                                                               const uint32_t* block_offsets, ConvTmp tmp,
                                                               int32_t* status)
{
    using S = Storage<DT>;
    using T = typename S::T;
    __shared__ uint32_t s_tmp[8];
    if (status_failed(status)) return;
    const int64_t base = (int64_t)blockIdx.x * kConvBlock;
    uint32_t carry = block_offsets[blockIdx.x];  // moved rows before this block
    for (int k = 0; k < kConvItems; ++k) {
        const int64_t i = base + k * kConvThreads + threadIdx.x;
        const bool st = i < g4.n && is_static<DT>(g4, i, tau);
        // block exclusive scan of st
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned bal = __ballot_sync(0xffffffffu, st);
        if (lane == 0) s_tmp[warp] = __popc(bal);
        __syncthreads();
        uint32_t wbase = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            if (w < warp) wbase += s_tmp[w];
            tot += s_tmp[w];
        }
        __syncthreads();
        const uint32_t before = carry + wbase + __popc(bal & lanemask_lt());
        carry += tot;
        if (i >= g4.n) continue;
        const T* m = (const T*)g4.mean + i * 4;
        const T* ls = (const T*)g4.log_scale + i * 4;
        const int wsh = 48 * (g4.sh_time + 1);  // SH floats per 4D row
        const T* sh = (const T*)g4.sh + i * wsh;
        if (st) {
            const int64_t d = g3.n + before;
            float ql[4], qr[4];
            load4<DT>(g4.ql, i, ql);
            load4<DT>(g4.qr, i, qr);
            const float il = inv_norm4(ql), ir = inv_norm4(qr);
#pragma unroll
            for (int c = 0; c < 4; ++c) { ql[c] *= il; qr[c] *= ir; }
            float R4[16];
            rot4(ql, qr, R4);
            const float R3[9] = {R4[0], R4[1], R4[2], R4[4], R4[5], R4[6], R4[8], R4[9], R4[10]};
            float q[4];
            matrix_to_quat(R3, q);
            T* dm = (T*)g3.mean + d * 3;
            T* dl = (T*)g3.log_scale + d * 3;
            T* dq = (T*)g3.quat + d * 4;
            for (int c = 0; c < 3; ++c) { dm[c] = m[c]; dl[c] = ls[c]; }
            for (int c = 0; c < 4; ++c) dq[c] = S::from(q[c]);
            ((T*)g3.opacity)[d] = ((const T*)g4.opacity)[i];
            T* dsh = (T*)g3.sh + d * 48;
            for (int c = 0; c < 48; ++c) dsh[c] = sh[c];  // the time-constant block
        } else {
            const int64_t d = i - before;  // rows kept before i
            for (int c = 0; c < 4; ++c) {
                ((T*)tmp.mean)[d * 4 + c] = m[c];
                ((T*)tmp.log_scale)[d * 4 + c] = ls[c];
                ((T*)tmp.ql)[d * 4 + c] = ((const T*)g4.ql)[i * 4 + c];
                ((T*)tmp.qr)[d * 4 + c] = ((const T*)g4.qr)[i * 4 + c];
            }
            ((T*)tmp.opacity)[d] = ((const T*)g4.opacity)[i];
            for (int c = 0; c < wsh; ++c) ((T*)tmp.sh)[d * wsh + c] = sh[c];
        }
    }
}

template <int DT>
__global__ void __launch_bounds__(kConvThreads) k_conv_copyback(splat_g4 g4, ConvTmp tmp, const int64_t* n_moved,
                                                                int32_t* status)
{
    using T = typename Storage<DT>::T;
    if (status_failed(status)) return;
    const int64_t kept = g4.n - *n_moved;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kept; i += (int64_t)gridDim.x * blockDim.x) {
        for (int c = 0; c < 4; ++c) {
            ((T*)g4.mean)[i * 4 + c] = ((const T*)tmp.mean)[i * 4 + c];
            ((T*)g4.log_scale)[i * 4 + c] = ((const T*)tmp.log_scale)[i * 4 + c];
            ((T*)g4.ql)[i * 4 + c] = ((const T*)tmp.ql)[i * 4 + c];
            ((T*)g4.qr)[i * 4 + c] = ((const T*)tmp.qr)[i * 4 + c];
        }
        ((T*)g4.opacity)[i] = ((const T*)tmp.opacity)[i];
        const int wsh = 48 * (g4.sh_time + 1);
        for (int c = 0; c < wsh; ++c) ((T*)g4.sh)[i * wsh + c] = ((const T*)tmp.sh)[i * wsh + c];
    }
}

// Optimizer state of the conversion: the moments of the kept 4D rows follow
// their parameters (same stable compaction), the 3D rows the moved Gaussians
// land in get zero moments.  The decision reads the parameter set g4, which
// must still hold the values before the conversion.
__host__ __device__ constexpr int width3(int f) { return f < 2 ? 3 : (f == 2 ? 4 : (f == 3 ? 1 : 48)); }
// floats per 4D row of field f; sh holds a block of 48 per time frequency
__host__ __device__ constexpr int width4(int f, int sh_time) { return f < 4 ? 4 : (f == 4 ? 1 : 48 * (sh_time + 1)); }

struct StateTmp {  // workspace copy of the kept 4D rows' moments
    float* m[6];
    float* v[6];
};

template <int DT>
__global__ void __launch_bounds__(kConvThreads) k_state_scatter(splat_g4 g4, float tau, int64_t n3,
                                                                const uint32_t* block_offsets, splat_adam_set s4,
                                                                splat_adam_set s3, StateTmp tmp, int32_t* status)
{
    const int T = g4.sh_time;
    __shared__ uint32_t s_tmp[8];
    if (status_failed(status)) return;
    const int64_t base = (int64_t)blockIdx.x * kConvBlock;
    uint32_t carry = block_offsets[blockIdx.x];
    for (int k = 0; k < kConvItems; ++k) {
        const int64_t i = base + k * kConvThreads + threadIdx.x;
        const bool st = i < g4.n && is_static<DT>(g4, i, tau);
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
        const unsigned bal = __ballot_sync(0xffffffffu, st);
        if (lane == 0) s_tmp[warp] = __popc(bal);
        __syncthreads();
        uint32_t wbase = 0, tot = 0;
#pragma unroll
        for (int w = 0; w < 8; ++w) {
            if (w < warp) wbase += s_tmp[w];
            tot += s_tmp[w];
        }
        __syncthreads();
        const uint32_t before = carry + wbase + __popc(bal & lanemask_lt());
        carry += tot;
        if (i >= g4.n) continue;
        if (st) {
            const int64_t d = n3 + before;
#pragma unroll
            for (int f = 0; f < 5; ++f)
                for (int c = 0; c < width3(f); ++c) {
                    s3.m[f][d * width3(f) + c] = 0.f;
                    s3.v[f][d * width3(f) + c] = 0.f;
                }
        } else {
            const int64_t d = i - before;
#pragma unroll
            for (int f = 0; f < 6; ++f)
                for (int c = 0; c < width4(f, T); ++c) {
                    tmp.m[f][d * width4(f, T) + c] = s4.m[f][i * width4(f, T) + c];
                    tmp.v[f][d * width4(f, T) + c] = s4.v[f][i * width4(f, T) + c];
                }
        }
    }
}

__global__ void __launch_bounds__(256) k_state_copyback(int64_t n4, int T, splat_adam_set s4, StateTmp tmp,
                                                        const int64_t* n_moved, int32_t* status)
{
    if (status_failed(status)) return;
    const int64_t kept = n4 - *n_moved;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < kept; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < 6; ++f)
            for (int c = 0; c < width4(f, T); ++c) {
                s4.m[f][i * width4(f, T) + c] = tmp.m[f][i * width4(f, T) + c];
                s4.v[f][i * width4(f, T) + c] = tmp.v[f][i * width4(f, T) + c];
            }
    }
}

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t convert_state_workspace(int64_t n4, int T)
{
    const int64_t nb = (n4 + kConvBlock - 1) / kConvBlock;
    size_t o = a256(4 * (size_t)(nb + 1)) + a256(8);
    for (int f = 0; f < 6; ++f) o += 2 * a256(4 * (size_t)n4 * width4(f, T));
    return o;
}

template <int DT>
static cudaError_t convert_state_impl(const splat_g4& g4, const splat_g3& g3, float tau, const splat_adam_set& s4,
                                      const splat_adam_set& s3, int32_t* status, void* ws, const LaunchCtx& ctx)
{
    const int64_t n4 = g4.n;
    const int T = g4.sh_time;
    if (n4 == 0) return cudaSuccess;
    const int64_t nb = (n4 + kConvBlock - 1) / kConvBlock;
    char* w = (char*)ws;
    uint32_t* counts = (uint32_t*)w;
    size_t o = a256(4 * (size_t)(nb + 1));
    int64_t* n_moved = (int64_t*)(w + o);
    o += a256(8);
    StateTmp tmp;
    for (int f = 0; f < 6; ++f) {
        tmp.m[f] = (float*)(w + o);
        o += a256(4 * (size_t)n4 * width4(f, T));
        tmp.v[f] = (float*)(w + o);
        o += a256(4 * (size_t)n4 * width4(f, T));
    }
    cudaStream_t s = ctx.stream;
    count_launch(4);
    k_conv_count<DT><<<(int)nb, kConvThreads, 0, s>>>(g4, tau, counts);
    k_conv_scan<<<1, 1024, 0, s>>>(counts, nb, g3.n, g3.capacity, n_moved, status);
    k_state_scatter<DT><<<(int)nb, kConvThreads, 0, s>>>(g4, tau, g3.n, counts, s4, s3, tmp, status);
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, (int64_t)ctx.num_sms * 8);
    k_state_copyback<<<blocks, 256, 0, s>>>(n4, T, s4, tmp, n_moved, status);
    return cudaGetLastError();
}

cudaError_t launch_convert_state(const splat_g4& g4, const splat_g3& g3, float tau, const splat_adam_set& s4,
                                 const splat_adam_set& s3, int32_t* status, void* ws, const LaunchCtx& ctx)
{
    switch (g4.dtype) {
    case SPLAT_F32: return convert_state_impl<SPLAT_F32>(g4, g3, tau, s4, s3, status, ws, ctx);
    case SPLAT_BF16: return convert_state_impl<SPLAT_BF16>(g4, g3, tau, s4, s3, status, ws, ctx);
    default: return convert_state_impl<SPLAT_F16>(g4, g3, tau, s4, s3, status, ws, ctx);
    }
}

size_t convert_workspace(int64_t n4, int dtype_bytes, int sh_time)
{
    const int64_t nb = (n4 + kConvBlock - 1) / kConvBlock;
    return a256(4 * (size_t)(nb + 1)) + a256((size_t)dtype_bytes * n4 * 4) * 4 + a256((size_t)dtype_bytes * n4) +
           a256((size_t)dtype_bytes * n4 * 48 * (sh_time + 1));
}

template <int DT>
static cudaError_t convert_impl(const splat_g4& g4, const splat_g3& g3, float tau, int64_t* n_moved, int32_t* status,
                                void* ws, const LaunchCtx& ctx)
{
    using T = typename Storage<DT>::T;
    const int64_t n4 = g4.n;
    const int64_t nb = (n4 + kConvBlock - 1) / kConvBlock;
    char* w = (char*)ws;
    uint32_t* counts = (uint32_t*)w;
    size_t o = a256(4 * (size_t)(nb + 1));
    ConvTmp tmp;
    tmp.mean = w + o; o += a256(sizeof(T) * n4 * 4);
    tmp.log_scale = w + o; o += a256(sizeof(T) * n4 * 4);
    tmp.ql = w + o; o += a256(sizeof(T) * n4 * 4);
    tmp.qr = w + o; o += a256(sizeof(T) * n4 * 4);
    tmp.opacity = w + o; o += a256(sizeof(T) * n4);
    tmp.sh = w + o;
    cudaStream_t s = ctx.stream;
    if (n4 == 0) return cudaMemsetAsync(n_moved, 0, sizeof(int64_t), s);
    count_launch(4);
    k_conv_count<DT><<<(int)nb, kConvThreads, 0, s>>>(g4, tau, counts);
    k_conv_scan<<<1, 1024, 0, s>>>(counts, nb, g3.n, g3.capacity, n_moved, status);
    k_conv_scatter<DT><<<(int)nb, kConvThreads, 0, s>>>(g4, g3, tau, counts, tmp, status);
    const int blocks = (int)std::min<int64_t>((n4 + 255) / 256, (int64_t)ctx.num_sms * 8);
    k_conv_copyback<DT><<<blocks, 256, 0, s>>>(g4, tmp, n_moved, status);
    return cudaGetLastError();
}

cudaError_t launch_convert(const splat_g4& g4, const splat_g3& g3, float tau, int64_t* n_moved, int32_t* status,
                           void* ws, const LaunchCtx& ctx)
{
    switch (g4.dtype) {
    case SPLAT_F32: return convert_impl<SPLAT_F32>(g4, g3, tau, n_moved, status, ws, ctx);
    case SPLAT_BF16: return convert_impl<SPLAT_BF16>(g4, g3, tau, n_moved, status, ws, ctx);
    default: return convert_impl<SPLAT_F16>(g4, g3, tau, n_moved, status, ws, ctx);
    }
}

}  // namespace splat
