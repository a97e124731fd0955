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

// Packed FP32 pairs: a lane evaluates its pixels two at a time with the
// sm_100-family f32x2 instructions (each component rounds like the scalar
// operation).
__device__ __forceinline__ float2 dup2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One Gaussian seen from one lane's pixel column: the x-only terms of the
// power, duplicated for the pixel pairs.  Forward and backward build them
// with the same operations, so both evaluate bit-identical powers.
struct ColTerms {
    float2 A2, Bx2, c2, py;
};

__device__ __forceinline__ ColTerms col_terms(const Feat& f, float uf)
{
    const float dx = f.px - uf;
    ColTerms c;
    c.A2 = dup2(f.a2 * dx * dx);
    c.Bx2 = dup2(f.b2 * dx);
    c.c2 = dup2(f.c2);
    c.py = dup2(f.py);
    return c;
}

// base-2 power at a pixel pair whose rows are -nrow: A2 + dy (Bx2 + c2 dy),
// dy = py - row.  A row of -inf (a finished pixel) gives dy = -inf and
// p2 = -inf (c2 < 0), which the skip test rejects.
__device__ __forceinline__ float2 pair_power(const ColTerms& c, float2 nrow)
{
    const float2 dy = add2(c.py, nrow);
    return fma2(dy, fma2(c.c2, dy, c.Bx2), c.A2);
}

// A Gaussian with alpha_max below this never reaches the 0.99 clamp (p2 <= 0
// makes 2^p2 <= 1, and ex2.approx overshoots 1 by far less than the margin),
// so the clamp and its zero derivative are evaluated only above it.
constexpr float kClampFree = 0.989f;

// STATS: also count, per warp, the pixel-Gaussian pairs evaluated (power
// computed) and blended, into stats[0..1] (diagnostic instantiation only).
template <int PPL, bool STATS>
__global__ void __launch_bounds__(kCompWarps * 32) k_composite_fwd(splat_proj proj, const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges, ViewBatch vb,
                                                                   splat_image img, int32_t* status,
                                                                   unsigned long long* stats)
{
    static_assert(PPL == 2 || PPL == 4 || PPL == 8, "pixels per lane come in pairs");
    constexpr int BANDS = 8 / PPL, NP = PPL / 2;
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
    // pair p holds pixels k = 2p, 2p + 1 (rows y0 + 4p, y0 + 4p + 2).  nrow:
    // minus the row, -inf once the pixel is done (outside the image or
    // saturated).  nC: minus the accumulated colour.
    float2 T[NP], nC[NP][3], nrow[NP];
    int last[PPL];
    unsigned done = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = make_float2(1.f, 1.f);
        nC[p][0] = nC[p][1] = nC[p][2] = make_float2(0.f, 0.f);
        nrow[p] = make_float2(-(float)(y0 + 4 * p), -(float)(y0 + 4 * p + 2));
        last[2 * p] = last[2 * p + 1] = 0;
        if (u >= vp.W || y0 + 4 * p >= vp.H) {
            done |= 1u << (2 * p);
            nrow[p].x = __int_as_float(0xff800000);
        }
        if (u >= vp.W || y0 + 4 * p + 2 >= vp.H) {
            done |= 2u << (2 * p);
            nrow[p].y = __int_as_float(0xff800000);
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
                const ColTerms ct = col_terms(f, uf);
                const float2 nop = dup2(-f.op), cr = dup2(f.r), cg = dup2(f.g), cb = dup2(f.bl);
                const bool clamp = f.op >= kClampFree;  // same Gaussian on every lane
#pragma unroll
                for (int p = 0; p < NP; ++p) {
                    const float2 p2 = pair_power(ct, nrow[p]);
                    if (STATS) n_eval += ((done >> (2 * p)) & 1u ^ 1u) + ((done >> (2 * p + 1)) & 1u ^ 1u);
                    // skip power > 0 and alpha < 1/255 (as p2 < pcut2); NaN and -inf skip too
                    const bool ox = p2.x <= 0.f && p2.x >= f.pcut2, oy = p2.y <= 0.f && p2.y >= f.pcut2;
                    if (!(ox || oy)) continue;
                    // na = -alpha (0 for a skipped pixel of the pair)
                    float2 na = mul2(nop, make_float2(ex2_approx(p2.x), ex2_approx(p2.y)));
                    if (clamp) {
                        na.x = fmaxf(na.x, -kAlphaClamp);
                        na.y = fmaxf(na.y, -kAlphaClamp);
                    }
                    na.x = ox ? na.x : 0.f;
                    na.y = oy ? na.y : 0.f;
                    float2 nw = mul2(na, T[p]);  // -alpha T
                    float2 tT = add2(T[p], nw);  // T (1 - alpha)
                    const bool sx = ox && tT.x < kTMin, sy = oy && tT.y < kTMin;
                    if (sx || sy) {  // the pixel saturates: this Gaussian does not contribute
                        if (sx) {
                            done |= 1u << (2 * p);
                            nrow[p].x = __int_as_float(0xff800000);
                            nw.x = 0.f;
                            tT.x = T[p].x;
                        }
                        if (sy) {
                            done |= 2u << (2 * p);
                            nrow[p].y = __int_as_float(0xff800000);
                            nw.y = 0.f;
                            tT.y = T[p].y;
                        }
                    }
                    if (STATS) n_blend += (ox && !sx) + (oy && !sy);
                    nC[p][0] = fma2(cr, nw, nC[p][0]);
                    nC[p][1] = fma2(cg, nw, nC[p][1]);
                    nC[p][2] = fma2(cb, nw, nC[p][2]);
                    T[p] = tT;
                    if (ox && !sx) last[2 * p] = pos0 + j;
                    if (oy && !sy) last[2 * p + 1] = pos0 + j;
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
    float* rgb = img.rgb + 3 * vp.pix_base;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        if (u >= vp.W || y >= vp.H) continue;
        const int64_t p = (int64_t)y * vp.W + u;
        const float Tk = (k & 1) ? T[k >> 1].y : T[k >> 1].x;
        const float c0 = (k & 1) ? nC[k >> 1][0].y : nC[k >> 1][0].x;
        const float c1 = (k & 1) ? nC[k >> 1][1].y : nC[k >> 1][1].x;
        const float c2 = (k & 1) ? nC[k >> 1][2].y : nC[k >> 1][2].x;
        rgb[p] = Tk * vp.bg[0] - c0;
        rgb[HW + p] = Tk * vp.bg[1] - c1;
        rgb[2 * HW + p] = Tk * vp.bg[2] - c2;
        img.final_T[vp.pix_base + p] = Tk;
        img.last[vp.pix_base + p] = last[k];
    }
}

// Gradient sums over the warp's 32 lanes of a batch of up to kRedBatch = 7
// Gaussians.  Each lane leaves its sums (negated: the walk accumulates minus
// each quantity) in shared memory as 16 float4 groups of 32 lanes:
//   group 2 q     = (S dx W0, W1, S dx^2 W0, S dx W1)   of Gaussian q
//   group 2 q + 1 = (W2, W0, dr, dg)                    of Gaussian q
//   groups 14, 15 = the blue-channel sums db of Gaussians 0-3 and 4-6
// (W0, W1, W2: the lane's moments of dL/dpower, 1, dy, dy^2, over its pixels;
// dx is the lane's own).  Lane 2 gi + h sums group gi over source lanes
// 16 h .. 16 h + 15 and the lane pair adds up; the h = 0 lane of group 2 q + g
// turns the sums into Gaussian q's dproj components 4 g .. 4 g + 3 and adds
// them with one vector atomic, and the h = 1 lane of group q adds Gaussian q's
// blue-channel gradient (component 8).
constexpr int kRedBatch = 7;
constexpr int kRedGroups = 16;
// resident CTAs per SM the backward is compiled for (registers; shared memory
// holds 5 CTAs): PPL = 8 needs about 125 registers
template <int PPL>
struct BwdOccupancy {
    static constexpr int kMinBlocks = PPL >= 8 ? 4 : 5;
};

__device__ __forceinline__ void flush_reduction(const float4* red, int nq, uint32_t pend_row, int pend_j,
                                                const float4* sf, float* dproj, int lane)
{
    __syncwarp();
    const int gi = lane >> 1, h = lane & 1;
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
    if (gi < 2 * nq || gi == 14 || (gi == 15 && nq > 4)) {
        // source lane 16 h + (i ^ x): the quarter-warp's loads fall in distinct banks
        const float4* col = red + gi * 32 + 16 * h;
        const int x = lane & 7;
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const float4 t = col[i ^ x];
            s0 = add2(s0, make_float2(t.x, t.y));
            s1 = add2(s1, make_float2(t.z, t.w));
        }
    }
    s0.x += __shfl_xor_sync(0xffffffffu, s0.x, 1);
    s0.y += __shfl_xor_sync(0xffffffffu, s0.y, 1);
    s1.x += __shfl_xor_sync(0xffffffffu, s1.x, 1);
    s1.y += __shfl_xor_sync(0xffffffffu, s1.y, 1);
    // Gaussian of this lane: gi / 2 for the h = 0 (group) lanes, gi for the
    // h = 1 (blue-channel) lanes
    const int q = h ? gi : gi >> 1;
    const int src = q < kRedBatch ? q : 0;
    const uint32_t row = __shfl_sync(0xffffffffu, pend_row, src);
    const int jv = __shfl_sync(0xffffffffu, pend_j, src);
    const int bl = 28 + 2 * (q >> 2);  // a lane holding the blue sums of Gaussians 4 (q / 4) ..
    const float b0 = __shfl_sync(0xffffffffu, s0.x, bl & 31), b1 = __shfl_sync(0xffffffffu, s0.y, bl & 31);
    const float b2 = __shfl_sync(0xffffffffu, s1.x, bl & 31), b3 = __shfl_sync(0xffffffffu, s1.y, bl & 31);
    if (q < nq) {
        if (h == 0) {
            const float4 f0 = sf[jv * 3], f1 = sf[jv * 3 + 1];
            float4 out;
            if ((gi & 1) == 0) {  // dpx, dpy, da, db with the natural-unit conic (a, b, c)
                const float ca = -kLn2x2 * f0.z, cb = -0.5f * kLn2x2 * f0.w, cc = -kLn2x2 * f1.x;
                out = make_float4(ca * s0.x + cb * s0.y, cc * s0.y + cb * s0.x, 0.5f * s1.x, s1.y);
            } else {  // dc, dalpha_max = W0 / alpha_max (unclamped pairs only), dr, dg
                out = make_float4(0.5f * s0.x, -s0.y / f1.y, -s1.x, -s1.y);
            }
            atomicAdd((float4*)(dproj + (int64_t)row * 12) + (gi & 1), out);
        } else {
            const int c = q & 3;
            const float nb = c == 0 ? b0 : (c == 1 ? b1 : (c == 2 ? b2 : b3));
            atomicAdd(dproj + (int64_t)row * 12 + 8, -nb);
        }
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
    static_assert(PPL == 2 || PPL == 4 || PPL == 8, "pixels per lane come in pairs");
    constexpr int BANDS = 8 / PPL, NP = PPL / 2;
    __shared__ float4 s_feat[kCompWarps][32][3];
    __shared__ uint32_t s_row[kCompWarps][32];
    __shared__ float4 s_red[kCompWarps][kRedGroups][32];
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
    // Q starts at <G, bg>.  Pixels in pairs as in the forward; nQ = -Q.
    float2 T[NP], nQ[NP], G[NP][3], nrow[NP];
    int last[PPL];
    int maxlast = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        float t = 1.f, q = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        last[k] = 0;
        if (u < vp.W && y < vp.H) {
            const int64_t p = (int64_t)y * vp.W + u;
            const float* g = dL + 3 * vp.pix_base;
            g0 = g[p];
            g1 = g[HW + p];
            g2 = g[2 * HW + p];
            t = img.final_T[vp.pix_base + p];
            last[k] = img.last[vp.pix_base + p];
            q = -(g0 * vp.bg[0] + g1 * vp.bg[1] + g2 * vp.bg[2]);
            maxlast = max(maxlast, last[k]);
        }
        if (k & 1) {
            T[k >> 1].y = t; nQ[k >> 1].y = q; G[k >> 1][0].y = g0; G[k >> 1][1].y = g1; G[k >> 1][2].y = g2;
            nrow[k >> 1].y = -(float)y;
        } else {
            T[k >> 1].x = t; nQ[k >> 1].x = q; G[k >> 1][0].x = g0; G[k >> 1][1].x = g1; G[k >> 1][2].x = g2;
            nrow[k >> 1].x = -(float)y;
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
    const float2 one = make_float2(1.f, 1.f);
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
            const ColTerms ct = col_terms(f, uf);
            const float2 nop = dup2(-f.op), cr = dup2(f.r), cg = dup2(f.g), cb = dup2(f.bl);
            const bool clamp = f.op >= kClampFree;  // same Gaussian on every lane
            const float dx = f.px - uf;
            const float pyr = f.py - y0f;  // dy of pixel k is pyr - 2 k (up to rounding)
            // per lane, over its pixels, negated: dL/drgb and the moments of
            // dL/dpower W0 = sum dpow, V1 = sum k dpow, V2 = sum k^2 dpow
            float2 sW0 = make_float2(0.f, 0.f), sV1 = sW0, sV2 = sW0, sr = sW0, sg = sW0, sb = sW0;
            bool any = false;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                const float2 p2 = pair_power(ct, nrow[p]);
                const bool ax = li < last[2 * p], ay = li < last[2 * p + 1];
                if (STATS) n_eval += ax + ay;
                // the forward's skip, bit for bit, on the pixels that reached this Gaussian
                const bool ox = ax && p2.x <= 0.f && p2.x >= f.pcut2, oy = ay && p2.y <= 0.f && p2.y >= f.pcut2;
                if (!(ox || oy)) continue;
                if (STATS) n_blend += ox + oy;
                any = true;
                const float2 nraw = mul2(nop, make_float2(ex2_approx(p2.x), ex2_approx(p2.y)));
                float2 na = nraw;  // -alpha, 0 for a skipped pixel of the pair
                if (clamp) {
                    na.x = fmaxf(na.x, -kAlphaClamp);
                    na.y = fmaxf(na.y, -kAlphaClamp);
                }
                na.x = ox ? na.x : 0.f;
                na.y = oy ? na.y : 0.f;
                const float2 om = add2(one, na);  // 1 - alpha >= 0.01
                const float2 rc = make_float2(ox ? rcp_approx(om.x) : 1.f, oy ? rcp_approx(om.y) : 1.f);
                const float2 Tj = mul2(T[p], rc);
                const float2 nw = mul2(na, Tj);  // -alpha T_j
                sr = fma2(nw, G[p][0], sr);
                sg = fma2(nw, G[p][1], sg);
                sb = fma2(nw, G[p][2], sb);
                float2 d = fma2(G[p][0], cr, nQ[p]);  // <G, c_j> - Q
                d = fma2(G[p][1], cg, d);
                d = fma2(G[p][2], cb, d);
                nQ[p] = fma2(na, d, nQ[p]);
                T[p] = Tj;
                // dL/dpower = dL/dalpha * alpha = w d where alpha is not clamped
                float2 dp = mul2(nw, d);
                if (clamp) {
                    dp.x = nraw.x > -kAlphaClamp ? dp.x : 0.f;
                    dp.y = nraw.y > -kAlphaClamp ? dp.y : 0.f;
                }
                sW0 = add2(sW0, dp);
                sV1 = fma2(make_float2((float)(2 * p), (float)(2 * p + 1)), dp, sV1);
                sV2 = fma2(make_float2((float)(4 * p * p), (float)((2 * p + 1) * (2 * p + 1))), dp, sV2);
            }
            if (!__any_sync(0xffffffffu, any)) continue;
            const float W0 = sW0.x + sW0.y, V1 = sV1.x + sV1.y, V2 = sV2.x + sV2.y;
            const float W1 = pyr * W0 - 2.f * V1;                     // sum dpow dy
            const float W2 = pyr * (pyr * W0 - 4.f * V1) + 4.f * V2;  // sum dpow dy^2
            float4* slot = red + 2 * nq * 32 + lane;
            const float dxW0 = dx * W0;
            slot[0] = make_float4(dxW0, W1, dx * dxW0, dx * W1);
            slot[32] = make_float4(W2, W0, sr.x + sr.y, sg.x + sg.y);
            ((float*)(red + (14 + (nq >> 2)) * 32 + lane))[nq & 3] = sb.x + sb.y;
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
    default: k_composite_fwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, status, stats); break;
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
    default: k_composite_bwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, vb, img, dL, dproj, status, stats); break;
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
