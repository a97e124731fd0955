// composite.cu -- Alg. 1 BlendInOrder (Eq. 3) and its adjoint.
//
// Work decomposition: a "unit" is one tile (or a horizontal band of it, see
// PPL) handled by ONE warp, independently of every other warp: no block
// barriers.  Lane l owns pixel column l % 16 and rows (l / 16) + 2k, k < PPL,
// of the band, so a warp covers 32 * PPL pixels (PPL = 8: the whole 16x16
// tile).  The warp walks the tile's sorted list in batches of 32 Gaussians:
// each lane gathers one Gaussian's projected features into the warp's
// shared-memory slot, then every lane evaluates all its pixels against the
// 32 staged Gaussians (broadcast reads).  The warp leaves the list as soon as
// a vote shows every one of its pixels has saturated (T would drop below
// 1e-4).
//
// The adjoint walks the same list back to front from each pixel's stored last
// contributor, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final
// transmittance.  Per Gaussian each lane keeps 9 sums over its pixels; batches
// of kRedBatch Gaussians are summed over the warp through shared memory and
// added to the 2D gradients with one vector atomic per 4 components.
#include "splat_internal.cuh"

namespace splat {

constexpr int kCompWarps = 4;  // warps (units) per CTA
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2x2 = 1.3862943611198906f;  // 2 ln 2: converts the staged log2-scaled conic back

// 2^x by the PTX approximate base-2 exponential (relative error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Projected features of one Gaussian as staged in shared memory.  The conic is
// staged scaled by -log2(e)/2 (a2, c2) and -log2(e) (b2), so that
// p2 = a2 dx^2 + b2 dx dy + c2 dy^2 is the power in base 2 and
// alpha = alpha_max 2^p2 needs no extra multiply; pcut2 = log2(1/(255 alpha_max))
// turns the alpha < 1/255 skip into a test on p2.  Forward and backward take
// every decision (p2 > 0, p2 < pcut2, the clamp, the stop) on the same values.
struct Feat {
    float px, py, a2, b2, c2, op, r, g, bl, pcut2;
};

__device__ __forceinline__ void load_feat(const float4* s, Feat& f)
{
    const float4 f0 = s[0], f1 = s[1], f2 = s[2];
    f.px = f0.x; f.py = f0.y; f.a2 = f0.z; f.b2 = f0.w;
    f.c2 = f1.x; f.op = f1.y; f.r = f1.z; f.g = f1.w;
    f.bl = f2.x; f.pcut2 = f2.y;
}

__device__ __forceinline__ void stage_feat(const splat_proj& proj, uint32_t row, float4* s)
{
    const float2 xy = ((const float2*)proj.xy)[row];
    const float4 co = ((const float4*)proj.conic_opacity)[row];
    const float4 rd = ((const float4*)proj.rgb_depth)[row];
    const float pcut2 = __log2f(kAlphaMin / co.w);
    s[0] = make_float4(xy.x, xy.y, -0.5f * kLog2e * co.x, -kLog2e * co.y);
    s[1] = make_float4(-0.5f * kLog2e * co.z, co.w, rd.x, rd.y);
    s[2] = make_float4(rd.z, pcut2, 0.f, 0.f);
}

__device__ __forceinline__ int find_view(const ViewBatch& vb, int tile)
{
    int v = 0;
    for (int w = 1; w < vb.V; ++w)
        if (tile >= vb.v[w].tile_base) v = w;
    return v;
}

// STATS: also count, per warp, the pixel-Gaussian pairs evaluated (power
// computed) and blended, into stats[0..1] (diagnostic instantiation only).
template <int PPL, bool STATS>
__global__ void __launch_bounds__(kCompWarps * 32) k_composite_fwd(splat_proj proj, const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges, ViewBatch vb,
                                                                   splat_image img, int32_t* status,
                                                                   unsigned long long* stats)
{
    constexpr int BANDS = 8 / PPL;
    __shared__ float4 s_feat[kCompWarps][32][3];
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t unit = (int64_t)blockIdx.x * kCompWarps + warp;
    if (unit >= (int64_t)vb.total_tiles * BANDS) return;
    const int tile = (int)(unit / BANDS), band = (int)(unit % BANDS);
    const int v = find_view(vb, tile);
    const ViewParams& vp = vb.v[v];
    const int local = tile - vp.tile_base;
    const int ty = local / vp.TX, tx = local - ty * vp.TX;
    const int u = tx * kTile + (lane & 15);
    const int y0 = ty * kTile + band * (2 * PPL) + (lane >> 4);
    const float uf = (float)u;
    // yk[k]: row of pixel k, +inf once the pixel is done (outside the image or
    // saturated): dy = -inf then makes p2 = -inf, which the skip test rejects
    float T[PPL], C[PPL][3], yk[PPL];
    int last[PPL];
    unsigned done = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        T[k] = 1.f;
        C[k][0] = C[k][1] = C[k][2] = 0.f;
        last[k] = 0;
        yk[k] = (float)(y0 + 2 * k);
        if (u >= vp.W || y0 + 2 * k >= vp.H) {
            done |= 1u << k;
            yk[k] = __int_as_float(0x7f800000);
        }
    }
    const uint2 rg = ranges[tile];
    const unsigned all_done = (1u << PPL) - 1;
    float4* sf = &s_feat[warp][0][0];
    unsigned n_eval = 0, n_blend = 0;
    for (uint32_t b = rg.x; b < rg.y; b += 32) {
        if (__all_sync(0xffffffffu, done == all_done)) break;
        const uint32_t idx = b + lane;
        if (idx < rg.y) stage_feat(proj, vals[idx], sf + lane * 3);
        __syncwarp();
        const int n = (int)min(32u, rg.y - b);
        if (done != all_done) {
            const int pos0 = (int)(b - rg.x) + 1;
            for (int j = 0; j < n; ++j) {
                Feat f;
                load_feat(sf + j * 3, f);
                const float dx = f.px - uf;
                const float A2 = f.a2 * dx * dx, Bx2 = f.b2 * dx;
#pragma unroll
                for (int k = 0; k < PPL; ++k) {
                    const float dy = f.py - yk[k];
                    const float p2 = A2 + dy * (Bx2 + f.c2 * dy);
                    if (STATS) n_eval += (done >> k & 1u) ^ 1u;
                    // skip power > 0 and alpha < 1/255 (as p2 < pcut2); NaN and -inf skip too
                    if (!(p2 <= 0.f && p2 >= f.pcut2)) continue;
                    const float alpha = fminf(kAlphaClamp, f.op * ex2_approx(p2));
                    const float w = alpha * T[k];
                    const float tT = T[k] - w;  // T (1 - alpha)
                    if (tT < kTMin) {
                        done |= 1u << k;
                        yk[k] = __int_as_float(0x7f800000);
                        continue;
                    }
                    if (STATS) ++n_blend;
                    C[k][0] += f.r * w;
                    C[k][1] += f.g * w;
                    C[k][2] += f.bl * w;
                    T[k] = tT;
                    last[k] = pos0 + j;
                }
                if (done == all_done) break;
            }
        }
        __syncwarp();
    }
    if (STATS) {
        const unsigned e = __reduce_add_sync(0xffffffffu, n_eval), bl = __reduce_add_sync(0xffffffffu, n_blend);
        if (lane == 0) {
            atomicAdd(stats + 0, (unsigned long long)e);
            atomicAdd(stats + 1, (unsigned long long)bl);
        }
    }
    const int64_t HW = (int64_t)vp.W * vp.H;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        if (u >= vp.W || y >= vp.H) continue;
        const int64_t p = (int64_t)y * vp.W + u;
        float* rgb = img.rgb + 3 * vp.pix_base;
        rgb[p] = C[k][0] + T[k] * vp.bg[0];
        rgb[HW + p] = C[k][1] + T[k] * vp.bg[1];
        rgb[2 * HW + p] = C[k][2] + T[k] * vp.bg[2];
        img.final_T[vp.pix_base + p] = T[k];
        img.last[vp.pix_base + p] = last[k];
    }
}

// Gradient sums of a batch of kRedBatch Gaussians over the warp's 32 lanes.
// Each lane leaves 12 floats per Gaussian in shared memory, as three float4
// groups:
//   g0 = (S dx W0, W1, S dx^2 W0, S dx W1)   g1 = (W2, W0, dr, dg)   g2 = (db, 0, 0, 0)
// (W0, W1, W2: the lane's moments of dL/dpower, 1, dy, dy^2, over its pixels;
// dx is the lane's own).  Lane 6 jj + 2 g + h sums group g of Gaussian jj over
// source lanes 16 h .. 16 h + 15, the lane pair adds up, and the h = 0 lane
// turns the sums into the Gaussian's dproj components (4 g .. 4 g + 3) and adds
// them with one vector atomic.
#ifndef SPLAT_RED_BATCH
#define SPLAT_RED_BATCH 4
#endif
// resident CTAs per SM the backward is compiled for: 7 caps PPL <= 4 at 72
// registers, without spills; PPL = 8 needs about 125
template <int PPL>
struct BwdOccupancy {
    static constexpr int kMinBlocks = PPL >= 8 ? 4 : 7;
};
constexpr int kRedBatch = SPLAT_RED_BATCH;
static_assert(kRedBatch >= 1 && kRedBatch <= 5, "the flush maps 6 lanes to each batched Gaussian");

__device__ __forceinline__ void flush_reduction(const float4* red, int nq, uint32_t pend_row, int pend_j,
                                                const float4* sf, float* dproj, int lane)
{
    __syncwarp();
    const int jj = lane / 6, rem = lane - 6 * jj, g = rem >> 1, h = rem & 1;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (jj < nq) {
        // source lane 16 h + (i ^ x): the quarter-warp's loads fall in distinct banks
        const float4* col = red + (jj * 3 + g) * 32 + 16 * h;
        const int x = lane & 7;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float4 t = col[i ^ x];
            acc.x += t.x;
            acc.y += t.y;
            acc.z += t.z;
            acc.w += t.w;
        }
    }
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, 1);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, 1);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, 1);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, 1);
    const int src = jj < kRedBatch ? jj : 0;
    const uint32_t row = __shfl_sync(0xffffffffu, pend_row, src);
    const int jv = __shfl_sync(0xffffffffu, pend_j, src);
    if (jj < nq && h == 0) {
        float4 out;
        if (g == 2) {
            out = make_float4(acc.x, 0.f, 0.f, 0.f);  // db (colour); the row's padding stays zero
        } else {
            const float4 f0 = sf[jv * 3], f1 = sf[jv * 3 + 1];
            if (g == 0) {  // dpx, dpy, da, db with the natural-unit conic (a, b, c)
                const float ca = -kLn2x2 * f0.z, cb = -0.5f * kLn2x2 * f0.w, cc = -kLn2x2 * f1.x;
                out = make_float4(-(ca * acc.x + cb * acc.y), -(cc * acc.y + cb * acc.x), -0.5f * acc.z, -acc.w);
            } else {  // dc, dalpha_max = W0 / alpha_max (unclamped pairs only), dr, dg
                out = make_float4(-0.5f * acc.x, acc.y / f1.y, acc.z, acc.w);
            }
        }
        atomicAdd((float4*)(dproj + (int64_t)row * 12) + g, out);
    }
    __syncwarp();
}

// STATS: also count the pairs evaluated and blended into stats[2..3].
template <int PPL, bool STATS>
__global__ void __launch_bounds__(kCompWarps * 32, BwdOccupancy<PPL>::kMinBlocks) k_composite_bwd(splat_proj proj, const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges, ViewBatch vb,
                                                                   splat_image img, const float* __restrict__ dL,
                                                                   float* dproj, int32_t* status,
                                                                   unsigned long long* stats)
{
    constexpr int BANDS = 8 / PPL;
    __shared__ float4 s_feat[kCompWarps][32][3];
    __shared__ uint32_t s_row[kCompWarps][32];
    __shared__ float4 s_red[kCompWarps][kRedBatch * 3][32];
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t unit = (int64_t)blockIdx.x * kCompWarps + warp;
    if (unit >= (int64_t)vb.total_tiles * BANDS) return;
    const int tile = (int)(unit / BANDS), band = (int)(unit % BANDS);
    const int v = find_view(vb, tile);
    const ViewParams& vp = vb.v[v];
    const int local = tile - vp.tile_base;
    const int ty = local / vp.TX, tx = local - ty * vp.TX;
    const int u = tx * kTile + (lane & 15);
    const int y0 = ty * kTile + band * (2 * PPL) + (lane >> 4);
    const float uf = (float)u;
    const int64_t HW = (int64_t)vp.W * vp.H;
    // Per pixel: T = T_{j+1} (replayed transmittance behind the current Gaussian j),
    // G = dL/dC, and Q = <G, S_j> / T_{j+1} with S_j = sum_{i>j} c_i alpha_i T_i + T_final bg
    // the colour accumulated behind j.  Then dL/dalpha_j = T_j (<G, c_j> - Q) and
    // Q_{j-1} = Q + alpha_j (<G, c_j> - Q): S itself is never needed per channel, and
    // Q starts at <G, bg>.
    float T[PPL], Q[PPL], G[PPL][3];
    int last[PPL];
    int maxlast = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        last[k] = 0;
        T[k] = 1.f;
        Q[k] = 0.f;
        G[k][0] = G[k][1] = G[k][2] = 0.f;
        if (u < vp.W && y < vp.H) {
            const int64_t p = (int64_t)y * vp.W + u;
            const float* g = dL + 3 * vp.pix_base;
            G[k][0] = g[p];
            G[k][1] = g[HW + p];
            G[k][2] = g[2 * HW + p];
            T[k] = img.final_T[vp.pix_base + p];
            last[k] = img.last[vp.pix_base + p];
            Q[k] = G[k][0] * vp.bg[0] + G[k][1] * vp.bg[1] + G[k][2] * vp.bg[2];
            maxlast = max(maxlast, last[k]);
        }
    }
    const float y0f = (float)y0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) maxlast = max(maxlast, __shfl_xor_sync(0xffffffffu, maxlast, o));
    if (maxlast == 0) return;
    const uint2 rg = ranges[tile];
    float4* sf = &s_feat[warp][0][0];
    float4* red = &s_red[warp][0][0];
    const int nb = (maxlast + 31) / 32;
    unsigned n_eval = 0, n_blend = 0;
    for (int bi = nb - 1; bi >= 0; --bi) {
        const uint32_t b = rg.x + 32u * bi;
        const uint32_t end = min(rg.x + (uint32_t)maxlast, rg.y);
        const uint32_t idx = b + lane;
        if (idx < end) {
            const uint32_t row = vals[idx];
            s_row[warp][lane] = row;
            stage_feat(proj, row, sf + lane * 3);
        }
        __syncwarp();
        const int n = (int)min(32u, end - b);
        int nq = 0;            // Gaussians waiting in the reduction buffer
        uint32_t pend_row = 0; // lane q: row of waiting Gaussian q
        int pend_j = 0;        // lane q: its slot in the staged batch
        for (int j = n - 1; j >= 0; --j) {
            Feat f;
            load_feat(sf + j * 3, f);
            const int li = 32 * bi + j;  // position in the tile list
            const float dx = f.px - uf;
            const float A2 = f.a2 * dx * dx, Bx2 = f.b2 * dx;
            const float pyr = f.py - y0f;  // dy of pixel k is pyr - 2 k (up to rounding)
            // per lane, over its pixels: dL/drgb and the moments of dL/dpower
            // W0 = sum dpow, V1 = sum k dpow, V2 = sum k^2 dpow
            float W0 = 0.f, V1 = 0.f, V2 = 0.f, cr = 0.f, cg = 0.f, cb = 0.f;
            bool any = false;
#pragma unroll
            for (int k = 0; k < PPL; ++k) {
                // the forward's dy: py minus the row, an exact integer in FP32
                const float dy = f.py - (y0f + (float)(2 * k));
                const float p2 = A2 + dy * (Bx2 + f.c2 * dy);
                if (STATS) n_eval += li < last[k];
                // the forward's skip, bit for bit, on the pixels that reached this Gaussian
                if (!(li < last[k] && p2 <= 0.f && p2 >= f.pcut2)) continue;
                const float raw = f.op * ex2_approx(p2);
                const float alpha = fminf(kAlphaClamp, raw);
                if (STATS) ++n_blend;
                any = true;
                const float Tj = T[k] * __fdividef(1.f, 1.f - alpha);  // 1 - alpha >= 0.01
                const float w = alpha * Tj;
                cr += w * G[k][0];
                cg += w * G[k][1];
                cb += w * G[k][2];
                const float d = G[k][0] * f.r + G[k][1] * f.g + G[k][2] * f.bl - Q[k];
                Q[k] += alpha * d;
                T[k] = Tj;
                // dL/dpower = dL/dalpha * alpha = w d where alpha is not clamped
                const float dpow = raw < kAlphaClamp ? w * d : 0.f;
                W0 += dpow;
                if (k > 0) {
                    V1 += (float)k * dpow;
                    V2 += (float)(k * k) * dpow;
                }
            }
            const float W1 = pyr * W0 - 2.f * V1;                             // sum dpow dy
            const float W2 = pyr * (pyr * W0 - 4.f * V1) + 4.f * V2;          // sum dpow dy^2
            if (!__any_sync(0xffffffffu, any)) continue;
            float4* slot = red + nq * 3 * 32 + lane;
            const float dxW0 = dx * W0;
            slot[0] = make_float4(dxW0, W1, dx * dxW0, dx * W1);
            slot[32] = make_float4(W2, W0, cr, cg);
            slot[64] = make_float4(cb, 0.f, 0.f, 0.f);
            if (lane == nq) {
                pend_row = s_row[warp][j];
                pend_j = j;
            }
            if (++nq == kRedBatch) {
                flush_reduction(red, nq, pend_row, pend_j, sf, dproj, lane);
                nq = 0;
            }
        }
        if (nq) flush_reduction(red, nq, pend_row, pend_j, sf, dproj, lane);
        __syncwarp();
    }
    if (STATS) {
        const unsigned e = __reduce_add_sync(0xffffffffu, n_eval), bl = __reduce_add_sync(0xffffffffu, n_blend);
        if (lane == 0) {
            atomicAdd(stats + 2, (unsigned long long)e);
            atomicAdd(stats + 3, (unsigned long long)bl);
        }
    }
}

// L1 photometric loss of the rendered images against a target (the loss of
// the paper's training step): loss += sum |img - target|, dL/dimg =
// sign(img - target) * scale.
__global__ void __launch_bounds__(256) k_l1_loss(const float* __restrict__ img, const float* __restrict__ target,
                                                 int64_t n, float scale, float* __restrict__ dL, float* loss)
{
    float acc = 0.f;
    const int64_t n4 = n / 4;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = ((const float4*)img)[i], b = ((const float4*)target)[i];
        const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
        acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
        auto sg = [](float d) { return d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f); };
        ((float4*)dL)[i] = make_float4(sg(d0) * scale, sg(d1) * scale, sg(d2) * scale, sg(d3) * scale);
    }
    for (int64_t i = 4 * n4 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float d = img[i] - target[i];
        acc += fabsf(d);
        dL[i] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * scale;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    __shared__ float s_acc[8];
    if ((threadIdx.x & 31) == 0) s_acc[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int w = 0; w < 8; ++w) t += s_acc[w];
        atomicAdd(loss, t);
    }
}

cudaError_t launch_l1_loss(const float* img, const float* target, int64_t n, float scale, float* dL, float* loss,
                           const LaunchCtx& ctx)
{
    cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), ctx.stream);
    if (e != cudaSuccess || n == 0) return e;
    const int64_t want = (n / 4 + 255) / 256 + 1;
    const int blocks = (int)(want < (int64_t)ctx.num_sms * 8 ? want : (int64_t)ctx.num_sms * 8);
    count_launch();
    k_l1_loss<<<blocks, 256, 0, ctx.stream>>>(img, target, n, scale, dL, loss);
    return cudaGetLastError();
}

template <bool ST>
static void fwd_launch(int ppl, int blocks, cudaStream_t st, const splat_proj& proj, const splat_bins& bins,
                       const ViewBatch& vb, const splat_image& img, int32_t* status, unsigned long long* stats)
{
    const uint2* rg = (const uint2*)bins.ranges;
    switch (ppl) {
    case 8: k_composite_fwd<8, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, status, stats); break;
    case 4: k_composite_fwd<4, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, status, stats); break;
    case 2: k_composite_fwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, status, stats); break;
    default: k_composite_fwd<1, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, status, stats); break;
    }
}

template <bool ST>
static void bwd_launch(int ppl, int blocks, cudaStream_t st, const splat_proj& proj, const splat_bins& bins,
                       const ViewBatch& vb, const splat_image& img, const float* dL, float* dproj, int32_t* status,
                       unsigned long long* stats)
{
    const uint2* rg = (const uint2*)bins.ranges;
    switch (ppl) {
    case 8: k_composite_bwd<8, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, dL, dproj, status, stats); break;
    case 4: k_composite_bwd<4, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, dL, dproj, status, stats); break;
    case 2: k_composite_bwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, dL, dproj, status, stats); break;
    default: k_composite_bwd<1, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, dL, dproj, status, stats); break;
    }
}

cudaError_t launch_composite_fwd(const splat_proj& proj, const splat_bins& bins, const ViewBatch& vb,
                                 const splat_image& img, int32_t* status, int ppl, unsigned long long* stats,
                                 const LaunchCtx& ctx)
{
    if (vb.total_tiles == 0) return cudaSuccess;
    const int bands = 8 / ppl;
    const int64_t units = (int64_t)vb.total_tiles * bands;
    const int blocks = (int)((units + kCompWarps - 1) / kCompWarps);
    count_launch();
    if (stats) fwd_launch<true>(ppl, blocks, ctx.stream, proj, bins, vb, img, status, stats);
    else fwd_launch<false>(ppl, blocks, ctx.stream, proj, bins, vb, img, status, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_composite_bwd(const splat_proj& proj, const splat_bins& bins, const ViewBatch& vb,
                                 const splat_image& img, const float* dL, float* dproj, int32_t* status, int ppl,
                                 unsigned long long* stats, const LaunchCtx& ctx)
{
    if (vb.total_tiles == 0) return cudaSuccess;
    const int bands = 8 / ppl;
    const int64_t units = (int64_t)vb.total_tiles * bands;
    const int blocks = (int)((units + kCompWarps - 1) / kCompWarps);
    count_launch();
    if (stats) bwd_launch<true>(ppl, blocks, ctx.stream, proj, bins, vb, img, dL, dproj, status, stats);
    else bwd_launch<false>(ppl, blocks, ctx.stream, proj, bins, vb, img, dL, dproj, status, nullptr);
    return cudaGetLastError();
}

}  // namespace splat
