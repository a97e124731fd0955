// densify.cu -- adaptive densification and pruning of the two parameter sets
// (Sec. 4.3: the 3D and the 4D Gaussians are densified and pruned separately,
// every 100 iterations, with the clone / split rules of 3DGS densification and
// no opacity reset).
//
// Statistics: per Gaussian, the norm of the loss gradient with respect to its
// projected mean in normalised device coordinates, |(dL/dpx W/2, dL/dpy H/2)|,
// summed over the views that see it, and the count of those views.
//
// Densification of one set, rows i < n, on FP32 master values (with Adam's
// moments): sigmoid(o) < min_opacity -> pruned; otherwise, with the mean
// statistic accum / count >= grad_threshold, a Gaussian whose largest spatial
// scale exp(s) is <= dense_scale is cloned (a copy is appended) and a larger
// one is split: it is replaced by two Gaussians at mean + M z (z from the
// caller's N(0, 1) draws, M = R diag(exp(s)): the 3x3 rotation of the
// quaternion for a 3D Gaussian, the 4x4 R of Eq. 4 for a 4D one, which offsets
// (x, y, z, t)), with every log-scale lowered by split_shrink.  Output rows:
// the kept Gaussians in order, then the clones in order, then the split
// children two by two in order.  New rows start with zero moments.
#include <algorithm>

#include "splat_internal.cuh"

namespace splat {

constexpr int kDensThreads = 256;
constexpr int kDensItems = 4;
constexpr int kDensBlock = kDensThreads * kDensItems;

enum : int { kPrune = 0, kKeep = 1, kClone = 2, kSplit = 3 };

// ---------------------------------------------------------------------------
// statistics
// ---------------------------------------------------------------------------

struct StatArgs {
    const float* dproj;        // [V * N][12]
    const uint32_t* n_tiles;   // [V * N]
    int64_t N;
    int V;
    float half_w[SPLAT_MAX_VIEWS], half_h[SPLAT_MAX_VIEWS];
    float* accum;
    float* count;
};

__global__ void __launch_bounds__(256) k_dens_stats(StatArgs a)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < a.N; i += (int64_t)gridDim.x * blockDim.x) {
        float acc = 0.f, cnt = 0.f;
        for (int v = 0; v < a.V; ++v) {
            const int64_t row = v * a.N + i;
            if (a.n_tiles[row] == 0) continue;
            const float2 g = *(const float2*)(a.dproj + row * 12);
            const float gx = g.x * a.half_w[v], gy = g.y * a.half_h[v];
            acc += sqrtf(gx * gx + gy * gy);
            cnt += 1.f;
        }
        if (cnt > 0.f) {
            a.accum[i] += acc;
            a.count[i] += cnt;
        }
    }
}

cudaError_t launch_dens_stats(const StatArgs& a, const LaunchCtx& ctx)
{
    if (a.N == 0) return cudaSuccess;
    const int blocks = (int)std::min<int64_t>((a.N + 255) / 256, (int64_t)ctx.num_sms * 8);
    count_launch();
    k_dens_stats<<<blocks, 256, 0, ctx.stream>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// densification of one set; D = 3 (3D set) or 4 (4D set)
// ---------------------------------------------------------------------------

template <int D>
struct SetLayout;
template <>
struct SetLayout<3> {  // mean, log_scale, quat, opacity, sh
    static constexpr int F = 5;
    // floats per row of field f; wsh: of the SH field
    __host__ __device__ static constexpr int width(int f, int wsh) { return f < 2 ? 3 : (f == 2 ? 4 : (f == 3 ? 1 : wsh)); }
    static constexpr int kOpacity = 3;
};
template <>
struct SetLayout<4> {  // mean, log_scale, ql, qr, opacity, sh (a block of 48 per time frequency)
    static constexpr int F = 6;
    __host__ __device__ static constexpr int width(int f, int wsh) { return f < 4 ? 4 : (f == 4 ? 1 : wsh); }
    static constexpr int kOpacity = 4;
};

struct DensSet {
    int64_t n, capacity;
    float* p[6];
    float* m[6];
    float* v[6];
    const float* accum;
    const float* count;
    const float* noise;  // [n][2][D]
    float* tp[6];        // workspace copies, capacity rows
    float* tm[6];
    float* tv[6];
    uint32_t* blocks;    // per-block counts, then offsets: [nb][3]
    int64_t* n_out;      // new row count
    int wsh;             // floats per row of the SH field
};

struct DensRule {
    float grad_threshold, dense_scale, min_opacity, split_shrink;
};

template <int D>
__device__ __forceinline__ int dens_class(const DensSet& s, const DensRule& r, int64_t i)
{
    const float o = s.p[SetLayout<D>::kOpacity][i];
    if (!(1.f / (1.f + expf(-o)) >= r.min_opacity)) return kPrune;
    const float c = s.count[i];
    const float avg = c > 0.f ? s.accum[i] / c : 0.f;
    if (!(avg >= r.grad_threshold)) return kKeep;
    const float* ls = s.p[1] + i * D;
    const float mx = expf(fmaxf(ls[0], fmaxf(ls[1], ls[2])));
    return mx <= r.dense_scale ? kClone : kSplit;
}

// per block: rows kept (KEEP or CLONE), clones, splits
template <int D>
__global__ void __launch_bounds__(kDensThreads) k_dens_count(DensSet s, DensRule r, int32_t* status)
{
    __shared__ uint32_t s_c[3];
    if (status_failed(status)) return;
    if (threadIdx.x < 3) s_c[threadIdx.x] = 0;
    __syncthreads();
    uint32_t c[3] = {0, 0, 0};
    for (int k = 0; k < kDensItems; ++k) {
        const int64_t i = (int64_t)blockIdx.x * kDensBlock + k * kDensThreads + threadIdx.x;
        if (i >= s.n) continue;
        const int cl = dens_class<D>(s, r, i);
        c[0] += cl == kKeep || cl == kClone;
        c[1] += cl == kClone;
        c[2] += cl == kSplit;
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint32_t x = __reduce_add_sync(0xffffffffu, c[q]);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&s_c[q], x);
    }
    __syncthreads();
    if (threadIdx.x < 3) s.blocks[blockIdx.x * 3 + threadIdx.x] = s_c[threadIdx.x];
}

// one block: exclusive scans of the three per-block counts; the new row count
// and the capacity check
__global__ void __launch_bounds__(1024) k_dens_scan(DensSet s, int64_t nb, int32_t* status)
{
    __shared__ unsigned long long s_warp[32][3];
    __shared__ unsigned long long s_carry[3];
    if (status_failed(status)) return;
    if (threadIdx.x < 3) s_carry[threadIdx.x] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
        const int64_t b = b0 + threadIdx.x;
        unsigned long long x[3], v[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            v[q] = b < nb ? s.blocks[b * 3 + q] : 0ull;
            x[q] = v[q];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, x[q], o);
                if (lane >= o) x[q] += y;
            }
            if (lane == 31) s_warp[warp][q] = x[q];
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            unsigned long long wb = 0, tot = 0;
            for (int w = 0; w < 32; ++w) {
                if (w < warp) wb += s_warp[w][q];
                tot += s_warp[w][q];
            }
            if (b < nb) s.blocks[b * 3 + q] = (uint32_t)(s_carry[q] + wb + x[q] - v[q]);
            __syncthreads();
            if (threadIdx.x == 0) s_carry[q] += tot;
            __syncthreads();
        }
    }
    if (threadIdx.x == 0) {
        const int64_t kept = (int64_t)s_carry[0], clones = (int64_t)s_carry[1], splits = (int64_t)s_carry[2];
        const int64_t n_new = kept + clones + 2 * splits;
        *s.n_out = n_new;
        if (n_new > s.capacity) set_status(status, SPLAT_ERR_CAPACITY, SPLAT_STAGE_DENSIFY, n_new);
        // the clones' and children's sections start after the kept rows
        s_carry[0] = (unsigned long long)kept;
        s_carry[1] = (unsigned long long)(kept + clones);
    }
    __syncthreads();
    // turn the clone and split offsets into absolute first rows of their sections
    for (int64_t b = threadIdx.x; b < nb; b += 1024) {
        s.blocks[b * 3 + 1] += (uint32_t)s_carry[0];
        s.blocks[b * 3 + 2] = (uint32_t)(s_carry[1] + 2ull * s.blocks[b * 3 + 2]);
    }
}

template <int D>
__device__ __forceinline__ void copy_row(const DensSet& s, int64_t src, int64_t dst, bool moments)
{
#pragma unroll
    for (int f = 0; f < SetLayout<D>::F; ++f) {
        const int w = SetLayout<D>::width(f, s.wsh);
        for (int c = 0; c < w; ++c) {
            s.tp[f][dst * w + c] = s.p[f][src * w + c];
            s.tm[f][dst * w + c] = moments ? s.m[f][src * w + c] : 0.f;
            s.tv[f][dst * w + c] = moments ? s.v[f][src * w + c] : 0.f;
        }
    }
}

// M = R diag(exp(s)) of Gaussian i
template <int D>
__device__ __forceinline__ void dens_frame(const DensSet& s, int64_t i, float M[D * D]);

template <>
__device__ __forceinline__ void dens_frame<3>(const DensSet& s, int64_t i, float M[9])
{
    const float* q = s.p[2] + i * 4;
    const float* ls = s.p[1] + i * 3;
    const float iq = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    float R[9];
    quat_to_rot(q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq, R);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int k = 0; k < 3; ++k) M[r * 3 + k] = R[r * 3 + k] * expf(ls[k]);
}

template <>
__device__ __forceinline__ void dens_frame<4>(const DensSet& s, int64_t i, float M[16])
{
    float ql[4], qr[4];
    for (int k = 0; k < 4; ++k) {
        ql[k] = s.p[2][i * 4 + k];
        qr[k] = s.p[3][i * 4 + k];
    }
    const float il = inv_norm4(ql), ir = inv_norm4(qr);
    for (int k = 0; k < 4; ++k) {
        ql[k] *= il;
        qr[k] *= ir;
    }
    float R[16];
    rot4(ql, qr, R);
    const float* ls = s.p[1] + i * 4;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int k = 0; k < 4; ++k) M[r * 4 + k] = R[r * 4 + k] * expf(ls[k]);
}

template <int D>
__global__ void __launch_bounds__(kDensThreads) k_dens_scatter(DensSet s, DensRule r, int32_t* status)
{
    __shared__ uint32_t s_tmp[3][8];
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t base[3] = {s.blocks[blockIdx.x * 3 + 0], s.blocks[blockIdx.x * 3 + 1], s.blocks[blockIdx.x * 3 + 2]};
    for (int k = 0; k < kDensItems; ++k) {
        const int64_t i = (int64_t)blockIdx.x * kDensBlock + k * kDensThreads + threadIdx.x;
        const int cl = i < s.n ? dens_class<D>(s, r, i) : kPrune;
        const bool f[3] = {cl == kKeep || cl == kClone, cl == kClone, cl == kSplit};
        uint32_t rank[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const unsigned bal = __ballot_sync(0xffffffffu, f[q]);
            if (lane == 0) s_tmp[q][warp] = __popc(bal);
            rank[q] = __popc(bal & lanemask_lt());
        }
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            uint32_t wb = 0, tot = 0;
            for (int w = 0; w < 8; ++w) {
                if (w < warp) wb += s_tmp[q][w];
                tot += s_tmp[q][w];
            }
            const uint32_t per = q == 2 ? 2u : 1u;  // rows each member of the class writes
            rank[q] = base[q] + per * (wb + rank[q]);
            base[q] += per * tot;
        }
        __syncthreads();
        if (i >= s.n) continue;
        if (f[0]) copy_row<D>(s, i, rank[0], true);
        if (f[1]) copy_row<D>(s, i, rank[1], false);
        if (f[2]) {
            const int64_t dd[2] = {rank[2], (int64_t)rank[2] + 1};  // the two children
            float M[D * D];
            dens_frame<D>(s, i, M);
            for (int h = 0; h < 2; ++h) {
                copy_row<D>(s, i, dd[h], false);
                const float* z = s.noise + (i * 2 + h) * D;
                for (int rr = 0; rr < D; ++rr) {
                    float off = 0.f;
                    for (int c = 0; c < D; ++c) off += M[rr * D + c] * z[c];
                    s.tp[0][dd[h] * D + rr] = s.p[0][i * D + rr] + off;
                    s.tp[1][dd[h] * D + rr] = s.p[1][i * D + rr] - r.split_shrink;
                }
            }
        }
    }
}

template <int D>
__global__ void __launch_bounds__(256) k_dens_copyback(DensSet s, int32_t* status)
{
    if (status_failed(status)) return;
    const int64_t n = *s.n_out;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int f = 0; f < SetLayout<D>::F; ++f) {
            const int w = SetLayout<D>::width(f, s.wsh);
            for (int c = 0; c < w; ++c) {
                s.p[f][i * w + c] = s.tp[f][i * w + c];
                s.m[f][i * w + c] = s.tm[f][i * w + c];
                s.v[f][i * w + c] = s.tv[f][i * w + c];
            }
        }
    }
}

static size_t a256d(size_t x) { return (x + 255) & ~(size_t)255; }

template <int D>
size_t dens_set_workspace(int64_t n, int64_t capacity, int wsh)
{
    const int64_t nb = (n + kDensBlock - 1) / kDensBlock + 1;
    size_t o = a256d(12 * (size_t)nb);
    for (int f = 0; f < SetLayout<D>::F; ++f) o += 3 * a256d(4 * (size_t)capacity * SetLayout<D>::width(f, wsh));
    return o;
}

size_t densify_workspace(int64_t n3, int64_t cap3, int64_t n4, int64_t cap4, int sh_time4)
{
    return dens_set_workspace<3>(n3, cap3, 48) + dens_set_workspace<4>(n4, cap4, 48 * (sh_time4 + 1));
}

template <int D>
static DensSet carve_set(DensSet s, char* ws)
{
    const int64_t nb = (s.n + kDensBlock - 1) / kDensBlock;
    size_t o = 0;
    s.blocks = (uint32_t*)(ws + o);
    o += a256d(12 * (size_t)(nb + 1));
    for (int f = 0; f < SetLayout<D>::F; ++f) {
        const size_t b = a256d(4 * (size_t)s.capacity * SetLayout<D>::width(f, s.wsh));
        s.tp[f] = (float*)(ws + o);
        s.tm[f] = (float*)(ws + o + b);
        s.tv[f] = (float*)(ws + o + 2 * b);
        o += 3 * b;
    }
    return s;
}

// counts and capacity checks of both sets first, so that an overflow in
// either set leaves both unchanged; then the scatters and copies
cudaError_t launch_densify(const DensSet& s3in, const DensSet& s4in, const DensRule& r, void* ws, int32_t* status,
                           const LaunchCtx& ctx)
{
    char* w = (char*)ws;
    const DensSet s3 = carve_set<3>(s3in, w);
    const DensSet s4 = carve_set<4>(s4in, w + dens_set_workspace<3>(s3in.n, s3in.capacity, s3in.wsh));
    const int64_t nb3 = (s3.n + kDensBlock - 1) / kDensBlock, nb4 = (s4.n + kDensBlock - 1) / kDensBlock;
    cudaStream_t st = ctx.stream;
    cudaError_t e;
    if (s3.n == 0 && (e = cudaMemsetAsync(s3.n_out, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
    if (s4.n == 0 && (e = cudaMemsetAsync(s4.n_out, 0, sizeof(int64_t), st)) != cudaSuccess) return e;
    if (s3.n > 0) {
        count_launch(2);
        k_dens_count<3><<<(int)nb3, kDensThreads, 0, st>>>(s3, r, status);
        k_dens_scan<<<1, 1024, 0, st>>>(s3, nb3, status);
    }
    if (s4.n > 0) {
        count_launch(2);
        k_dens_count<4><<<(int)nb4, kDensThreads, 0, st>>>(s4, r, status);
        k_dens_scan<<<1, 1024, 0, st>>>(s4, nb4, status);
    }
    if (s3.n > 0) {
        count_launch(2);
        k_dens_scatter<3><<<(int)nb3, kDensThreads, 0, st>>>(s3, r, status);
        const int blocks = (int)std::min<int64_t>((s3.capacity + 255) / 256, (int64_t)ctx.num_sms * 8);
        k_dens_copyback<3><<<blocks, 256, 0, st>>>(s3, status);
    }
    if (s4.n > 0) {
        count_launch(2);
        k_dens_scatter<4><<<(int)nb4, kDensThreads, 0, st>>>(s4, r, status);
        const int blocks = (int)std::min<int64_t>((s4.capacity + 255) / 256, (int64_t)ctx.num_sms * 8);
        k_dens_copyback<4><<<blocks, 256, 0, st>>>(s4, status);
    }
    return cudaGetLastError();
}

}  // namespace splat
