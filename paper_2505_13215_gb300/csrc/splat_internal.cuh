// splat_internal.cuh -- device-side helpers shared by the libsplat kernels.
//
// Everything here is internal to the CUDA library (sm_103a).  The public
// contract is include/splat.h.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "splat.h"

namespace splat {

constexpr int kTile = SPLAT_TILE;
constexpr int kRadix = 256;
constexpr float kAlphaMin = 1.0f / 255.0f;  // Alg. 1 BlendInOrder: negligible alpha
constexpr float kAlphaClamp = 0.99f;        // opacity clamp (3DGS convention)
constexpr float kTMin = 1e-4f;              // transmittance stop
constexpr float kDilation = 0.3f;           // px^2 added to the 2D covariance diagonal
constexpr float kFovClamp = 1.3f;           // Jacobian evaluated at x/z clamped to 1.3 tan(fov/2)

// Per-view camera data passed by value to kernels (constant bank).
struct ViewParams {
    float R[9];
    float T[3];
    float cam[3];    // camera centre -R^T T
    float fx, fy, cx, cy;
    float limx, limy;  // 1.3 * tan(fov/2) per axis
    float t, z_near;
    float bg[3];
    int W, H, TX, TY;
    int tile_base;   // first global tile index of this view
    int64_t pix_base;  // first pixel of this view in the image buffers
};

struct ViewBatch {
    ViewParams v[SPLAT_MAX_VIEWS];
    int V;
    int total_tiles;
};

// ---------------------------------------------------------------------------
// Device status word (status[4], see splat.h)
// ---------------------------------------------------------------------------

__device__ __forceinline__ void set_status(int32_t* status, int code, int stage, int64_t aux = 0)
{
    if (atomicCAS(status, 0, code) == 0) {
        status[1] = stage;
        status[2] = (int32_t)(aux & 0xffffffffll);
        status[3] = (int32_t)(aux >> 32);
    }
}

__device__ __forceinline__ bool status_failed(const int32_t* status)
{
    return *((volatile const int32_t*)status) != 0;
}

// ---------------------------------------------------------------------------
// Relaxed / acquire / release global accesses for the decoupled look-backs
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p)
{
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v)
{
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// ---------------------------------------------------------------------------
// Storage dtype loads / stores (FP32 arithmetic everywhere)
// ---------------------------------------------------------------------------

template <int DT> struct Storage;
template <> struct Storage<SPLAT_F32> {
    using T = float;
    __device__ __forceinline__ static float ld(const T* p) { return __ldg(p); }
    __device__ __forceinline__ static T from(float x) { return x; }
};
template <> struct Storage<SPLAT_BF16> {
    using T = __nv_bfloat16;
    __device__ __forceinline__ static float ld(const T* p) { return __bfloat162float(__ldg(p)); }
    __device__ __forceinline__ static T from(float x) { return __float2bfloat16_rn(x); }
};
template <> struct Storage<SPLAT_F16> {
    using T = __half;
    __device__ __forceinline__ static float ld(const T* p) { return __half2float(__ldg(p)); }
    __device__ __forceinline__ static T from(float x) { return __float2half_rn(x); }
};

// Vector loads of 3/4 consecutive elements of one Gaussian (rows are not
// necessarily 16-byte aligned for 3-wide fields).
template <int DT>
__device__ __forceinline__ void load4(const void* base, int64_t row, float out[4])
{
    using S = Storage<DT>;
    const typename S::T* p = (const typename S::T*)base + row * 4;
    if constexpr (DT == SPLAT_F32) {
        float4 v = __ldg((const float4*)p);
        out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
    } else {
        uint2 v = __ldg((const uint2*)p);  // 4 x 16-bit
        const typename S::T* h = (const typename S::T*)&v;
        for (int k = 0; k < 4; ++k) out[k] = (DT == SPLAT_BF16) ? __bfloat162float(((const __nv_bfloat16*)h)[k])
                                                                : __half2float(((const __half*)h)[k]);
    }
}

// The 48 coefficients (16 x 3) of one SH block with 16-byte loads: 12 of them for
// FP32, 6 for 16-bit storage.  Blocks are 192 / 96 bytes, so a block starts
// 16-byte aligned whenever the array does.
template <int DT>
__device__ __forceinline__ void load_sh48(const typename Storage<DT>::T* p, float c[48])
{
    if constexpr (DT == SPLAT_F32) {
        const float4* p4 = (const float4*)p;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            const float4 v = __ldg(p4 + q);
            c[4 * q + 0] = v.x; c[4 * q + 1] = v.y; c[4 * q + 2] = v.z; c[4 * q + 3] = v.w;
        }
    } else {
        const uint4* p4 = (const uint4*)p;
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            const uint4 v = __ldg(p4 + q);
            const typename Storage<DT>::T* h = (const typename Storage<DT>::T*)&v;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                c[8 * q + e] = (DT == SPLAT_BF16) ? __bfloat162float(((const __nv_bfloat16*)h)[e])
                                                  : __half2float(((const __half*)h)[e]);
        }
    }
}

template <int DT>
__device__ __forceinline__ void load3(const void* base, int64_t row, float out[3])
{
    using S = Storage<DT>;
    const typename S::T* p = (const typename S::T*)base + row * 3;
    for (int k = 0; k < 3; ++k) out[k] = S::ld(p + k);
}

template <int DT>
__device__ __forceinline__ float load1(const void* base, int64_t row)
{
    using S = Storage<DT>;
    return S::ld((const typename S::T*)base + row);
}

// ---------------------------------------------------------------------------
// Real spherical harmonics, degree 3, Condon-Shortley phase, k = l*l + l + m.
// Constants are the closed-form normalisations
//   K_l^m = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
// times sqrt(2) for m != 0 and the factors of the associated Legendre
// polynomials, e.g. Y_1^0 = sqrt(3/(4 pi)) z,
// Y_3^{+-3} = -sqrt(35/(32 pi)) Re/Im (x+iy)^3.
// ---------------------------------------------------------------------------

constexpr float kSH0 = 0.28209479177387814f;   // 1/(2 sqrt(pi))
constexpr float kSH1 = 0.48860251190291992f;   // sqrt(3/(4 pi))
constexpr float kSH2a = 1.0925484305920792f;   // sqrt(15/(4 pi))
constexpr float kSH2b = 0.31539156525252005f;  // sqrt(5/(16 pi))
constexpr float kSH2c = 0.54627421529603959f;  // sqrt(15/(16 pi))
constexpr float kSH3a = -0.59004358992664352f; // -sqrt(35/(32 pi))
constexpr float kSH3b = 2.8906114426405538f;   // sqrt(105/(4 pi))
constexpr float kSH3c = -0.45704579946446572f; // -sqrt(21/(32 pi))
constexpr float kSH3d = 0.37317633259011540f;  // sqrt(7/(16 pi))
constexpr float kSH3e = 1.4453057213202769f;   // sqrt(105/(16 pi))

__device__ __forceinline__ void sh_basis(float x, float y, float z, float Y[16])
{
    float xx = x * x, yy = y * y, zz = z * z;
    Y[0] = kSH0;
    Y[1] = -kSH1 * y;
    Y[2] = kSH1 * z;
    Y[3] = -kSH1 * x;
    Y[4] = kSH2a * x * y;
    Y[5] = -kSH2a * y * z;
    Y[6] = kSH2b * (3.f * zz - 1.f);
    Y[7] = -kSH2a * x * z;
    Y[8] = kSH2c * (xx - yy);
    Y[9] = kSH3a * y * (3.f * xx - yy);
    Y[10] = kSH3b * x * y * z;
    Y[11] = kSH3c * y * (5.f * zz - 1.f);
    Y[12] = kSH3d * z * (5.f * zz - 3.f);
    Y[13] = kSH3c * x * (5.f * zz - 1.f);
    Y[14] = kSH3e * z * (xx - yy);
    Y[15] = kSH3a * x * (xx - 3.f * yy);
}

// Gradient of sum_k w_k Y_k (polynomial extension above) w.r.t. (x, y, z).
__device__ __forceinline__ void sh_basis_grad(float x, float y, float z, const float w[16], float g[3])
{
    float xx = x * x, yy = y * y, zz = z * z;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gy += -kSH1 * w[1];
    gz += kSH1 * w[2];
    gx += -kSH1 * w[3];
    gx += kSH2a * y * w[4];            gy += kSH2a * x * w[4];
    gy += -kSH2a * z * w[5];           gz += -kSH2a * y * w[5];
    gz += 6.f * kSH2b * z * w[6];
    gx += -kSH2a * z * w[7];           gz += -kSH2a * x * w[7];
    gx += 2.f * kSH2c * x * w[8];      gy += -2.f * kSH2c * y * w[8];
    gx += 6.f * kSH3a * x * y * w[9];  gy += 3.f * kSH3a * (xx - yy) * w[9];
    gx += kSH3b * y * z * w[10];       gy += kSH3b * x * z * w[10];      gz += kSH3b * x * y * w[10];
    gy += kSH3c * (5.f * zz - 1.f) * w[11];                              gz += 10.f * kSH3c * y * z * w[11];
    gz += kSH3d * (15.f * zz - 3.f) * w[12];
    gx += kSH3c * (5.f * zz - 1.f) * w[13];                              gz += 10.f * kSH3c * x * z * w[13];
    gx += 2.f * kSH3e * x * z * w[14]; gy += -2.f * kSH3e * y * z * w[14]; gz += kSH3e * (xx - yy) * w[14];
    gx += 3.f * kSH3a * (xx - yy) * w[15]; gy += -6.f * kSH3a * x * y * w[15];
    g[0] = gx; g[1] = gy; g[2] = gz;
}

__device__ __forceinline__ float sigmoidf_(float x) { return 1.f / (1.f + expf(-x)); }

// Quaternion (w,x,y,z), unit, -> 3x3 rotation, row major (v -> q v q*).
__device__ __forceinline__ void quat_to_rot(float w, float x, float y, float z, float R[9])
{
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z);       R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z);       R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y);       R[7] = 2.f * (y * z + w * x);       R[8] = 1.f - 2.f * (x * x + y * y);
}

// Eq. 4: R = L(a,b,c,d) Rr(p,q,r,s), 4x4 row major.
__device__ __forceinline__ void rot4(const float l[4], const float r[4], float R[16])
{
    const float a = l[0], b = l[1], c = l[2], d = l[3];
    const float p = r[0], q = r[1], s_ = r[2], u = r[3];
    const float L[16] = {a, -b, -c, -d, b, a, -d, c, c, d, a, -b, d, -c, b, a};
    const float Q[16] = {p, -q, -s_, -u, q, p, u, -s_, s_, -u, p, q, u, s_, -q, p};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
            R[i * 4 + j] = L[i * 4 + 0] * Q[0 * 4 + j] + L[i * 4 + 1] * Q[1 * 4 + j] + L[i * 4 + 2] * Q[2 * 4 + j] +
                           L[i * 4 + 3] * Q[3 * 4 + j];
}

__device__ __forceinline__ float inv_norm4(const float q[4])
{
    return rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
}

}  // namespace splat

// Host-side launch helpers shared by the .cu files (defined in api.cu).
#include <atomic>
#include <cmath>
namespace splat {
extern std::atomic<int64_t> g_launches;  // kernels launched or captured (diagnostic)
inline void count_launch(int n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }
// L1 loss fused into the forward compositing (all null when not fused):
// *loss += sum |rgb - target|, dL = scale * sign(rgb - target), per pixel as
// its colour is written.
struct L1Fuse {
    const float* target;
    float scale;
    float* dL;
    float* loss;
};

// Per-call launch context: the stream, the device's SM count and the tuning
// of this call (the library-wide splat_set_* settings, or a caller's
// splat_options).
struct LaunchCtx {
    cudaStream_t stream;
    int num_sms;
    int64_t spin_limit;
    int tile_sort;   // 0 automatic, 1 radix passes, 2 binned partition
    int tile_cull;   // binned path: footprint culling and the saturation cut
    int ppl_fwd, ppl_bwd;
    unsigned long long* stats;
};
LaunchCtx launch_ctx(void* stream, const splat_options* opt = nullptr);

// Host-side argument checks shared by the entry points that take the same
// arguments (splat_bin_sort and its allocation-free variant reject the same
// calls).
inline bool host_aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

inline bool host_valid_views(const splat_view* views, int V)
{
    if (!views || V < 1 || V > SPLAT_MAX_VIEWS) return false;
    for (int v = 0; v < V; ++v) {
        const splat_view& s = views[v];
        if (s.W < 1 || s.H < 1 || s.W > 16384 || s.H > 16384) return false;
        if (!(s.fx > 0.f) || !(s.fy > 0.f) || !std::isfinite(s.cx) || !std::isfinite(s.cy)) return false;
        if (!(s.z_near > 0.f) || !std::isfinite(s.t)) return false;
    }
    return true;
}

inline bool host_valid_proj(const splat_proj* p, int V)
{
    return p && p->views == V && p->n >= 0 &&
           (p->n == 0 || (p->xy && p->conic_opacity && p->rgb_depth && p->rect && p->radius && p->n_tiles)) &&
           (int64_t)V * p->n < (1ll << 32);
}

// splat_bins as splat_bin_sort reads and writes it
inline bool host_valid_bins(const splat_bins* b)
{
    if (!b || b->capacity < 0 || b->capacity > SPLAT_MAX_INSTANCES || !b->ranges || !b->n_instances) return false;
    if (b->capacity > 0 && !b->vals) return false;
    return host_aligned(b->ranges, 8) && host_aligned(b->n_instances, 8);
}
}  // namespace splat
