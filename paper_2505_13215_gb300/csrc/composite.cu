// composite.cu -- Alg. 1 BlendInOrder (Eq. 3) and its adjoint.
//
// Work decomposition: a "unit" is one tile (or a horizontal band of it, see
// PPL) handled by ONE warp, independently of every other warp: no block
// barriers, one warp per CTA (a CTA never waits for a slower tile), tiles
// taken in the order splat_bin_sort wrote (longest list first) when it wrote
// one.  Lane l owns pixel column l % 16 and rows (l / 16) + 2k, k < PPL, of
// the band, so a warp covers 32 * PPL pixels (PPL = 8: the whole 16x16 tile);
// it evaluates them in pairs with packed FP32x2 arithmetic.  The warp walks
// the tile's sorted list in batches of 32 Gaussians: each lane gathers one
// Gaussian's projected rows into shared memory with cp.async one batch ahead
// (they land while the previous batch is composited) and turns them into the
// staged features, then every lane evaluates all its pixels against the 32
// staged Gaussians (broadcast reads).  The warp leaves the list as soon as a
// vote shows every one of its pixels has saturated (T would drop below 1e-4).
//
// The adjoint walks the same list back to front from where each pixel's walk
// ended, recovering T_i = T_{i+1} / (1 - alpha_i) from the stored final
// transmittance.  Per Gaussian each lane keeps 9 sums over its pixels; batches
// of kRedBatch Gaussians are summed over the warp through shared memory and
// added to the 2D gradients with vector atomics.  Whether the 0.99 opacity
// clamp needs evaluating is decided once per staged batch (one vote over its
// 32 Gaussians), so the walk runs one of two straight-line loop bodies.
#include <type_traits>

#include "splat_internal.cuh"

namespace splat {

constexpr int kCompWarps = 1;  // warps (units) per CTA
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2x2 = 1.3862943611198906f;  // 2 ln 2: converts the staged log2-scaled conic back

// 2^x by the PTX approximate base-2 exponential (relative error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Projected features of one Gaussian as staged in shared memory (four float4),
// the values the pixel pairs use duplicated for the packed arithmetic, the
// column terms' inputs once:
//   (py, py, nc2, nc2) (r, r, g, g) (b, b, px, op) (na2, nb2, ml, 0)
// The conic is staged scaled by log2(e)/2 (na2, nc2) and log2(e) (nb2), and
// ml = -log2(alpha_max) >= 0 joins the x-only term, so that
// np2 = ml + na2 dx^2 + nb2 dx dy + nc2 dy^2 is minus the base-2 logarithm of
// alpha = alpha_max exp(power): alpha = 2^-np2, one exponential and no
// multiply.  The skip test alpha < 1/255 becomes np2 > log2(255), evaluated as
// one unsigned compare of the bits of np2 with the bits of log2(255)
// (non-negative floats order like their bit patterns; a NaN or a negative np2,
// which needs power > -ml, i.e. alpha above alpha_max, is above the limit).
// Forward and backward take every decision (the skip, the clamp, the stop) on
// the same values.
constexpr int kFeat = 4;  // float4 per staged Gaussian
constexpr uint32_t kLimBits = 0x40ffd1beu;  // bits of log2(255) rounded to FP32 (7.9943533)
struct Feat {
    float2 py, nc2, r, g, bl;
    float px, op, na2, nb2, ml;
};

__device__ __forceinline__ void load_feat(const float4* s, Feat& f)
{
    const float4 f0 = s[0], f1 = s[1], f2 = s[2], f3 = s[3];
    f.py = make_float2(f0.x, f0.y); f.nc2 = make_float2(f0.z, f0.w);
    f.r = make_float2(f1.x, f1.y); f.g = make_float2(f1.z, f1.w);
    f.bl = make_float2(f2.x, f2.y);
    f.px = f2.z; f.op = f2.w;
    f.na2 = f3.x; f.nb2 = f3.y; f.ml = f3.z;
}

// The projected rows of the next batch are gathered while the current batch
// is composited: each lane copies its entry's three rows (xy, conic/opacity,
// rgb/depth; 40 bytes) into its own slot of a per-warp buffer with cp.async,
// and turns them into staged features when the walk reaches that batch.  The
// slot is private to the lane, so only the features need a warp barrier.
struct RawRows {
    float4 co[32];
    float4 rd[32];
    float2 xy[32];
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem)
{
    const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(s), "l"(gmem) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// all but the most recently committed group have landed
__device__ __forceinline__ void cp_async_wait_one() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

__device__ __forceinline__ void gather_rows(const splat_proj& proj, uint32_t row, RawRows& raw, int lane)
{
    cp_async16(&raw.co[lane], (const float4*)proj.conic_opacity + row);
    cp_async16(&raw.rd[lane], (const float4*)proj.rgb_depth + row);
    cp_async8(&raw.xy[lane], (const float2*)proj.xy + row);
}

// The staged features (Feat) of the lane's gathered rows, after its copies
// have landed.
__device__ __forceinline__ void stage_feat(const RawRows& raw, int lane, float4* s)
{
    const float2 xy = raw.xy[lane];
    const float4 co = raw.co[lane];
    const float4 rd = raw.rd[lane];
    // alpha_max <= 1 (a sigmoid times a temporal factor), so ml >= 0; a
    // Gaussian with alpha_max < 1/255 (none is listed) has ml > log2(255) and
    // fails every skip test
    const float ml = 0.f - __log2f(co.w);
    const float na2 = 0.5f * kLog2e * co.x, nb2 = kLog2e * co.y, nc2 = 0.5f * kLog2e * co.z;
    s[0] = make_float4(xy.y, xy.y, nc2, nc2);
    s[1] = make_float4(rd.x, rd.x, rd.y, rd.y);
    s[2] = make_float4(rd.z, rd.z, xy.x, co.w);
    s[3] = make_float4(na2, nb2, ml, 0.f);
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
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ float rcp_approx(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One Gaussian seen from one lane's pixel column (-u in nu): the x-only terms
// of np2 (with ml) for the pixel pairs.  Forward and backward build them with
// the same operations, so both evaluate bit-identical values.
struct ColTerms {
    float2 nA2, nBx2;
    float dx;
};

// Both halves of a pair share the column, so the terms are computed once in
// scalar arithmetic (a packed operation on equal halves costs the FMA pipe
// twice as much) and then duplicated.
__device__ __forceinline__ ColTerms col_terms(const Feat& f, float2 nu)
{
    ColTerms c;
    c.dx = f.px + nu.x;
    const float a = fmaf(f.na2 * c.dx, c.dx, f.ml), b = f.nb2 * c.dx;
    c.nA2 = make_float2(a, a);
    c.nBx2 = make_float2(b, b);
    return c;
}

// Row of a pixel that is done (forward) or not yet reached (backward): dy is
// then about -1e30 and np2 about nc2 1e60, +inf or far above any lim, so the
// skip test rejects the pixel; dy stays finite, so the backward's moment sums
// (dL/dpower = 0 times dy) stay 0.
constexpr float kOffRow = 1e30f;

// np2 = -log2(alpha) at a pixel pair whose rows are -nrow:
// nA2 + dy (nBx2 + nc2 dy), dy = py - row.
__device__ __forceinline__ float2 pair_npower(const Feat& f, const ColTerms& c, float2 dy)
{
    return fma2(dy, fma2(f.nc2, dy, c.nBx2), c.nA2);
}

__device__ __forceinline__ float2 pair_alpha(float2 np2)
{
    return make_float2(ex2_approx(-np2.x), ex2_approx(-np2.y));  // alpha = 2^-np2
}

// A Gaussian with alpha_max below this never reaches the 0.99 clamp (np2 >= ml
// up to rounding, so 2^-np2 <= alpha_max, and the logarithm, the rounding and
// ex2.approx move that by far less than the margin), so the clamp and its zero
// derivative are evaluated only above it.
constexpr float kClampFree = 0.989f;

// The forward's work for one staged Gaussian (list position pos, 1-based) on
// all pixel pairs of the lane; returns true once every pixel of the warp is
// done.  A pixel's walk ends at the entry that would bring T below 1e-4: its
// `last` becomes that entry's 0-based index (pos - 1), the number of entries
// the backward walks for it (the entries after its last contributor are
// skipped for it there as here).  Every pair is blended in straight-line code,
// a skipped pixel with alpha = 0 (no effect): few listed Gaussians reach no
// pixel of the band, and a block of independent pairs keeps the pipes fed.
// The saturation stop is rare and handled behind a vote.  No test result
// is kept across the pairs (the skip test is one compare, redone where
// needed), which keeps the predicate registers free.
template <int NP, bool CLAMP, bool STATS>
__device__ __forceinline__ bool fwd_gaussian(const Feat& f, const ColTerms& ct, float2 (&T)[NP],
                                             float2 (&nC)[NP][3], float2 (&nrow)[NP], int (&last)[2 * NP],
                                             unsigned& done, int pos, unsigned& n_eval, unsigned& n_blend)
{
    float2 np2[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        np2[p] = pair_npower(f, ct, add2(f.py, nrow[p]));
        if (STATS) n_eval += ((done >> (2 * p)) & 1u ^ 1u) + ((done >> (2 * p + 1)) & 1u ^ 1u);
    }
    float2 nw[NP], tT[NP];
    bool stop = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        float2 a = pair_alpha(np2[p]);  // alpha, 0 for a skipped pixel
        if (CLAMP) {
            a.x = fminf(a.x, kAlphaClamp);
            a.y = fminf(a.y, kAlphaClamp);
        }
        a.x = __float_as_uint(np2[p].x) <= kLimBits ? a.x : 0.f;
        a.y = __float_as_uint(np2[p].y) <= kLimBits ? a.y : 0.f;
        nw[p] = mul2(make_float2(-a.x, -a.y), T[p]);  // -alpha T: nonzero exactly for the blended pixels
        tT[p] = add2(T[p], nw[p]);  // T (1 - alpha); T itself for a skipped pixel (T >= 1e-4)
        stop |= (tT[p].x < kTMin) | (tT[p].y < kTMin);
    }
    bool finished = false;
    if (__any_sync(0xffffffffu, stop)) {
        // a pixel saturates: this Gaussian does not contribute to it
#pragma unroll
        for (int p = 0; p < NP; ++p) {
            if (tT[p].x < kTMin) {
                done |= 1u << (2 * p);
                nrow[p].x = -kOffRow;
                nw[p].x = 0.f;
                tT[p].x = T[p].x;
                last[2 * p] = pos - 1;
            }
            if (tT[p].y < kTMin) {
                done |= 2u << (2 * p);
                nrow[p].y = -kOffRow;
                nw[p].y = 0.f;
                tT[p].y = T[p].y;
                last[2 * p + 1] = pos - 1;
            }
        }
        finished = __all_sync(0xffffffffu, done == (1u << (2 * NP)) - 1);
    }
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        if (STATS) n_blend += (nw[p].x != 0.f) + (nw[p].y != 0.f);
        nC[p][0] = fma2(f.r, nw[p], nC[p][0]);
        nC[p][1] = fma2(f.g, nw[p], nC[p][1]);
        nC[p][2] = fma2(f.bl, nw[p], nC[p][2]);
        T[p] = tT[p];
    }
    return finished;
}

// Resident one-warp CTAs per SM the forward is compiled for.  The register
// file is split among the four schedulers, so occupancy moves in steps of four
// warps: PPL = 8 at 24 (80 registers, 8 bytes spilled) measured 0.329 ->
// 0.317 ms per 4-view step against 20 at 92 registers (28 at 72 registers:
// 0.321, 32 at 64: 0.337); the smaller variants fit 32 in 64 registers.
template <int PPL>
struct FwdOccupancy {
    static constexpr int kMinBlocks = PPL >= 8 ? 24 : 32;
};

// STATS: also count, per warp, the pixel-Gaussian pairs evaluated (power
// computed) and blended, into stats[0..1] (diagnostic instantiation only).
template <int PPL, bool STATS>
__global__ void __launch_bounds__(kCompWarps * 32, FwdOccupancy<PPL>::kMinBlocks) k_composite_fwd(splat_proj proj, const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ order, ViewBatch vb,
                                                                   splat_image img, L1Fuse l1, int32_t* status,
                                                                   unsigned long long* stats)
{
    static_assert(PPL == 2 || PPL == 4 || PPL == 8, "pixels per lane come in pairs");
    constexpr int BANDS = 8 / PPL, NP = PPL / 2;
    __shared__ float4 s_feat[kCompWarps][32][kFeat];
    __shared__ RawRows s_raw[kCompWarps];
    __shared__ float s_target[kCompWarps][3 * PPL][32];  // the fused loss's target at the lane's pixels
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t unit = (int64_t)blockIdx.x * kCompWarps + warp;
    if (unit >= (int64_t)vb.total_tiles * BANDS) return;
    // tiles in the bin sort's order (longest list first) when it wrote one
    const int slot = (int)(unit / BANDS), band = (int)(unit % BANDS);
    const int tile = order ? (int)__ldg(order + slot) : slot;
    const int v = find_view(vb, tile);
    const ViewParams& vp = vb.v[v];
    const int local = tile - vp.tile_base;
    const int ty = local / vp.TX, tx = local - ty * vp.TX;
    const int u = tx * kTile + (lane & 15);
    const int y0 = ty * kTile + band * (2 * PPL) + (lane >> 4);
    const float2 nu = make_float2(-(float)u, -(float)u);
    const int64_t HW = (int64_t)vp.W * vp.H;
    // pair p holds pixels k = 2p, 2p + 1 (rows y0 + 4p, y0 + 4p + 2).  nrow:
    // minus the row, -kOffRow once the pixel is done (outside the image or
    // saturated).  nC: minus the accumulated colour.
    const uint2 rg = ranges[tile];
    float2 T[NP], nC[NP][3], nrow[NP];
    int last[PPL];  // end of the walk: the list length unless the pixel saturates
    unsigned done = 0;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        T[p] = make_float2(1.f, 1.f);
        nC[p][0] = nC[p][1] = nC[p][2] = make_float2(0.f, 0.f);
        nrow[p] = make_float2(-(float)(y0 + 4 * p), -(float)(y0 + 4 * p + 2));
        last[2 * p] = last[2 * p + 1] = (int)(rg.y - rg.x);
        if (u >= vp.W || y0 + 4 * p >= vp.H) {
            done |= 1u << (2 * p);
            nrow[p].x = -kOffRow;
            last[2 * p] = 0;
        }
        if (u >= vp.W || y0 + 4 * p + 2 >= vp.H) {
            done |= 2u << (2 * p);
            nrow[p].y = -kOffRow;
            last[2 * p + 1] = 0;
        }
    }
    const unsigned all_done = (1u << PPL) - 1;
    float4* sf = &s_feat[warp][0][0];
    RawRows& raw = s_raw[warp];
    unsigned n_eval = 0, n_blend = 0;
    // the rows of batch 0 in flight, the list entries of batch 1 in a register;
    // then the fused loss's target at the lane's pixels, which lands in shared
    // memory during the walk (a group of its own, committed after batch 0's:
    // groups complete in order, so batch 0 need not wait for it)
    if (rg.x + lane < rg.y) gather_rows(proj, vals[rg.x + lane], raw, lane);
    cp_async_commit();
    if (l1.target) {  // same for every lane
#pragma unroll
        for (int k = 0; k < PPL; ++k) {
            const int y = y0 + 2 * k;
            if (u < vp.W && y < vp.H) {
                const int64_t q = 3 * vp.pix_base + (int64_t)y * vp.W + u;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) cp_async4(&s_target[warp][3 * k + ch][lane], l1.target + q + ch * HW);
            }
        }
    }
    cp_async_commit();
    uint32_t next_row = rg.x + 32 + lane < rg.y ? vals[rg.x + 32 + lane] : 0u;
    for (uint32_t b = rg.x; b < rg.y; b += 32) {
        if (__all_sync(0xffffffffu, done == all_done)) break;
        const uint32_t idx = b + lane;
        if (b == rg.x) cp_async_wait_one();  // batch 0's rows (the target may still be in flight)
        else cp_async_wait_all();
        if (idx < rg.y) stage_feat(raw, lane, sf + lane * kFeat);
        __syncwarp();
        // the next batch's rows land while this one is composited
        if (idx + 32 < rg.y) gather_rows(proj, next_row, raw, lane);
        cp_async_commit();
        next_row = idx + 64 < rg.y ? vals[idx + 64] : 0u;
        const int n = (int)min(32u, rg.y - b);
        const int pos0 = (int)(b - rg.x) + 1;
        // every lane walks the batch (finished pixels fail every test) so that
        // the votes inside see the whole warp
        for (int j = 0; j < n; ++j) {
            Feat f;
            load_feat(sf + j * kFeat, f);
            const ColTerms ct = col_terms(f, nu);
            const bool finished =
                f.op < kClampFree  // same Gaussian on every lane
                    ? fwd_gaussian<NP, false, STATS>(f, ct, T, nC, nrow, last, done, pos0 + j, n_eval, n_blend)
                    : fwd_gaussian<NP, true, STATS>(f, ct, T, nC, nrow, last, done, pos0 + j, n_eval, n_blend);
            if (finished) break;  // warp-uniform
        }
        __syncwarp();
    }
    cp_async_wait_all();  // no copy may land in shared memory after the CTA has left
    if (STATS) {
        const unsigned e = __reduce_add_sync(0xffffffffu, n_eval), bl = __reduce_add_sync(0xffffffffu, n_blend);
        if (lane == 0) {
            atomicAdd(stats + 0, (unsigned long long)e);
            atomicAdd(stats + 1, (unsigned long long)bl);
        }
    }
    float* rgb = img.rgb + 3 * vp.pix_base;
    float l1sum = 0.f;  // the lane's share of the fused L1 loss
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        if (u >= vp.W || y >= vp.H) continue;
        const int64_t p = (int64_t)y * vp.W + u;
        const float Tk = (k & 1) ? T[k >> 1].y : T[k >> 1].x;
        const float c0 = (k & 1) ? nC[k >> 1][0].y : nC[k >> 1][0].x;
        const float c1 = (k & 1) ? nC[k >> 1][1].y : nC[k >> 1][1].x;
        const float c2 = (k & 1) ? nC[k >> 1][2].y : nC[k >> 1][2].x;
        const float out[3] = {Tk * vp.bg[0] - c0, Tk * vp.bg[1] - c1, Tk * vp.bg[2] - c2};
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) rgb[ch * HW + p] = out[ch];
        img.final_T[vp.pix_base + p] = Tk;
        img.last[vp.pix_base + p] = last[k];
        if (l1.target) {  // same for every lane
            const int64_t q = 3 * vp.pix_base + p;
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) {
                const float d = out[ch] - s_target[warp][3 * k + ch][lane];
                l1sum += fabsf(d);
                l1.dL[q + ch * HW] = (d > 0.f ? 1.f : (d < 0.f ? -1.f : 0.f)) * l1.scale;
            }
        }
    }
    if (l1.target) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l1sum += __shfl_xor_sync(0xffffffffu, l1sum, o);
        if (lane == 0) atomicAdd(l1.loss, l1sum);
    }
}

// Gradient sums over the warp's 32 lanes of a group of up to kRedBatch = 7
// consecutive Gaussians of the walk (Gaussian q of the group in slot q, a
// compile-time index of the unrolled group).  Each lane leaves its sums (negated: the walk accumulates minus
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
// resident one-warp CTAs per SM the backward is compiled for: 16 leave
// PPL = 8 its 128 registers (20, at 96 registers, spill in the loop and
// measured slower: 0.615 -> 0.641 ms per 4-view step), 20 give the smaller
// variants 96
template <int PPL>
struct BwdOccupancy {
    static constexpr int kMinBlocks = PPL >= 8 ? 16 : 20;
};

// Reduction of a group of consecutive staged Gaussians j0, j0 - 1, ..,
// j0 - nq + 1 held in slots 0 .. nq - 1; slot q is added to dproj when bit q of
// `used` is set.
__device__ __forceinline__ void flush_group(const float4* red, int nq, unsigned used, int j0, const float4* sf,
                                            const uint32_t* srow, float* dproj, int lane)
{
    __syncwarp();
    const int gi = lane >> 1, h = lane & 1;
    float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
    if (gi < 2 * nq || gi == 14 || (gi == 15 && nq > 4)) {
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
    const int q = h ? gi : gi >> 1;
    const int bl = 28 + 2 * (q >> 2);
    const float b0 = __shfl_sync(0xffffffffu, s0.x, bl & 31), b1 = __shfl_sync(0xffffffffu, s0.y, bl & 31);
    const float b2 = __shfl_sync(0xffffffffu, s1.x, bl & 31), b3 = __shfl_sync(0xffffffffu, s1.y, bl & 31);
    if (q < nq && ((used >> q) & 1u)) {
        const int jv = j0 - q;
        const uint32_t row = srow[jv];
        if (h == 0) {
            const float4 f3 = sf[jv * kFeat + 3];
            const float nc2 = sf[jv * kFeat].z, nop = -sf[jv * kFeat + 2].w;
            float4 out;
            if ((gi & 1) == 0) {
                const float ca = kLn2x2 * f3.x, cb = 0.5f * kLn2x2 * f3.y, cc = kLn2x2 * nc2;
                out = make_float4(ca * s0.x + cb * s0.y, cc * s0.y + cb * s0.x, 0.5f * s1.x, s1.y);
            } else {
                out = make_float4(0.5f * s0.x, s0.y / nop, -s1.x, -s1.y);
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

// Per-lane sums of one Gaussian over the lane's pixels, negated (the walk
// accumulates minus each quantity): the moments of dL/dpower, 1, dy, dy^2
// (W0, W1, W2) and dL/drgb, each as a pair of partial sums.
struct BwdSums {
    float2 W0, W1, W2, r, g, b;
};

// The backward's work for one staged Gaussian on all pixel pairs of the lane,
// in straight-line code (a skipped pixel with alpha = 0, no effect).  Returns
// whether the Gaussian's sums are to be added to dproj: with STATS, whether
// any lane of the warp blended it (one vote); otherwise always, as the sums of
// a Gaussian no pixel blended are exactly zero, and few listed Gaussians reach
// no pixel, so a vote per Gaussian costs more than the atomics it saves.
template <int NP, bool CLAMP, bool STATS>
__device__ __forceinline__ bool bwd_gaussian(const Feat& f, const ColTerms& ct, float2 (&T)[NP], float2 (&nQ)[NP],
                                             const float2 (&G)[NP][3], const float2 (&nrow)[NP], BwdSums& S,
                                             unsigned& n_blend)
{
    const float2 one = make_float2(1.f, 1.f);
    bool anyv = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 dy = add2(f.py, nrow[p]);
        const float2 np2 = pair_npower(f, ct, dy);
        // the forward's skip, bit for bit, on the pixels that reached this Gaussian
        const bool ox = __float_as_uint(np2.x) <= kLimBits, oy = __float_as_uint(np2.y) <= kLimBits;
        if (STATS) {
            anyv |= ox | oy;
            n_blend += ox + oy;
        }
        const float2 araw = pair_alpha(np2);
        float2 a = araw;  // alpha, 0 for a skipped pixel of the pair
        if (CLAMP) {
            a.x = fminf(a.x, kAlphaClamp);
            a.y = fminf(a.y, kAlphaClamp);
        }
        a.x = ox ? a.x : 0.f;
        a.y = oy ? a.y : 0.f;
        const float2 na = make_float2(-a.x, -a.y);  // -alpha
        const float2 om = add2(one, na);  // 1 - alpha >= 0.01
        // T_j = T / (1 - alpha), one reciprocal and one multiply (a skipped
        // pixel multiplies T by the reciprocal of exactly 1)
        const float2 Tj = mul2(T[p], make_float2(rcp_approx(om.x), rcp_approx(om.y)));
        const float2 nw = mul2(na, Tj);  // -alpha T_j
        // the sums start at the first pair's terms
        S.r = p ? fma2(nw, G[p][0], S.r) : mul2(nw, G[p][0]);
        S.g = p ? fma2(nw, G[p][1], S.g) : mul2(nw, G[p][1]);
        S.b = p ? fma2(nw, G[p][2], S.b) : mul2(nw, G[p][2]);
        float2 d = fma2(G[p][0], f.r, nQ[p]);  // <G, c_j> - Q
        d = fma2(G[p][1], f.g, d);
        d = fma2(G[p][2], f.bl, d);
        nQ[p] = fma2(na, d, nQ[p]);
        T[p] = Tj;
        // dL/dpower = dL/dalpha * alpha = w d where alpha is not clamped
        float2 dp = mul2(nw, d);
        if (CLAMP) {
            dp.x = araw.x < kAlphaClamp ? dp.x : 0.f;
            dp.y = araw.y < kAlphaClamp ? dp.y : 0.f;
        }
        const float2 dpy = mul2(dp, dy);
        S.W0 = p ? add2(S.W0, dp) : dp;
        S.W1 = p ? add2(S.W1, dpy) : dpy;
        S.W2 = p ? fma2(dpy, dy, S.W2) : mul2(dpy, dy);
    }
    return STATS ? __any_sync(0xffffffffu, anyv) : true;
}

// STATS: also count the pairs evaluated and blended into stats[2..3].
template <int PPL, bool STATS>
__global__ void __launch_bounds__(kCompWarps * 32, BwdOccupancy<PPL>::kMinBlocks) k_composite_bwd(splat_proj proj, const uint32_t* __restrict__ vals,
                                                                   const uint2* __restrict__ ranges,
                                                                   const uint32_t* __restrict__ order, ViewBatch vb,
                                                                   splat_image img, const float* __restrict__ dL,
                                                                   float* dproj, int32_t* status,
                                                                   unsigned long long* stats)
{
    static_assert(PPL == 2 || PPL == 4 || PPL == 8, "pixels per lane come in pairs");
    constexpr int BANDS = 8 / PPL, NP = PPL / 2;
    __shared__ float4 s_feat[kCompWarps][32][kFeat];
    __shared__ uint32_t s_row[kCompWarps][32];
    __shared__ float4 s_red[kCompWarps][kRedGroups][32];
    __shared__ RawRows s_raw[kCompWarps];
    if (status_failed(status)) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t unit = (int64_t)blockIdx.x * kCompWarps + warp;
    if (unit >= (int64_t)vb.total_tiles * BANDS) return;
    // tiles in the bin sort's order (longest list first) when it wrote one
    const int slot = (int)(unit / BANDS), band = (int)(unit % BANDS);
    const int tile = order ? (int)__ldg(order + slot) : slot;
    const int v = find_view(vb, tile);
    const ViewParams& vp = vb.v[v];
    const int local = tile - vp.tile_base;
    const int ty = local / vp.TX, tx = local - ty * vp.TX;
    const int u = tx * kTile + (lane & 15);
    const int y0 = ty * kTile + band * (2 * PPL) + (lane >> 4);
    const float2 nu = make_float2(-(float)u, -(float)u);
    const int64_t HW = (int64_t)vp.W * vp.H;
    // Per pixel: T = T_{j+1} (replayed transmittance behind the current Gaussian j),
    // G = dL/dC, and Q = <G, S_j> / T_{j+1} with S_j = sum_{i>j} c_i alpha_i T_i + T_final bg
    // the colour accumulated behind j.  Then dL/dalpha_j = T_j (<G, c_j> - Q) and
    // Q_{j-1} = Q + alpha_j (<G, c_j> - Q): S itself is never needed per channel, and
    // Q starts at <G, bg>.  Pixels in pairs as in the forward; nQ = -Q.  A pixel's
    // row enters nrow (as minus the row) only once the walk reaches its last
    // contributor; before that nrow is -kOffRow and every test fails.
    const uint2 rg = ranges[tile];  // loaded with the pixels' state, not after it
    float2 T[NP], nQ[NP], G[NP][3], nrow[NP];
    int last[PPL];
    int maxlast = 0;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
        const int y = y0 + 2 * k;
        float t = 1.f, q = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f;
        int lk = 0;
        if (u < vp.W && y < vp.H) {
            const int64_t p = (int64_t)y * vp.W + u;
            const float* g = dL + 3 * vp.pix_base;
            g0 = g[p];
            g1 = g[HW + p];
            g2 = g[2 * HW + p];
            t = img.final_T[vp.pix_base + p];
            lk = img.last[vp.pix_base + p];
            q = -(g0 * vp.bg[0] + g1 * vp.bg[1] + g2 * vp.bg[2]);
            maxlast = max(maxlast, lk);
        }
        last[k] = lk;
        if (k & 1) {
            T[k >> 1].y = t; nQ[k >> 1].y = q; G[k >> 1][0].y = g0; G[k >> 1][1].y = g1; G[k >> 1][2].y = g2;
            nrow[k >> 1].y = -kOffRow;
        } else {
            T[k >> 1].x = t; nQ[k >> 1].x = q; G[k >> 1][0].x = g0; G[k >> 1][1].x = g1; G[k >> 1][2].x = g2;
            nrow[k >> 1].x = -kOffRow;
        }
    }
    const float y0f = (float)y0;
    maxlast = __reduce_max_sync(0xffffffffu, maxlast);
    if (maxlast == 0) return;
    // act: the list position (0-based) at or below which one of the warp's
    // pixels still has to switch on (its last contributor), -1 when none is left
    int act = maxlast - 1;
    float4* sf = &s_feat[warp][0][0];
    float4* red = &s_red[warp][0][0];
    // entries walked: [rg.x, end); batches 0 .. nb - 2 are full
    const uint32_t end = min(rg.x + (uint32_t)maxlast, rg.y);
    if (end <= rg.x) return;
    const int nb = (int)((end - rg.x + 31) / 32);
    RawRows& raw = s_raw[warp];
    unsigned n_eval = 0, n_blend = 0;
    // the walk goes back to front: the last (possibly partial) batch's rows in
    // flight first, the list entries of the one before it in a register; every
    // earlier batch is full
    uint32_t cur_row = 0, next_row = 0;
    {
        const uint32_t idx = rg.x + 32u * (nb - 1) + lane;
        if (idx < end) {
            cur_row = vals[idx];
            gather_rows(proj, cur_row, raw, lane);
        }
        cp_async_commit();
        if (nb >= 2) next_row = vals[rg.x + 32u * (nb - 2) + lane];
    }
    for (int bi = nb - 1; bi >= 0; --bi) {
        const uint32_t b = rg.x + 32u * bi;
        const uint32_t idx = b + lane;
        cp_async_wait_all();
        if (idx < end) {
            s_row[warp][lane] = cur_row;
            stage_feat(raw, lane, sf + lane * kFeat);
        }
        __syncwarp();
        // the previous batch's rows land while this one is walked
        if (bi >= 1) gather_rows(proj, next_row, raw, lane);
        cp_async_commit();
        cur_row = next_row;
        if (bi >= 2) next_row = vals[b - 64u + lane];
        const int n = (int)min(32u, end - b);
        // one vote per batch: does any staged Gaussian reach the 0.99 clamp
        const bool clamp_batch = __any_sync(0xffffffffu, lane < n && sf[lane * kFeat + 2].w >= kClampFree);
        auto walk = [&](auto clamp_tag) {
            constexpr bool CL = decltype(clamp_tag)::value;
            // groups of kRedBatch consecutive Gaussians, back to front; Gaussian
            // j0 - q of a group sums into reduction slot q
            for (int j0 = n - 1; j0 >= 0; j0 -= kRedBatch) {
                unsigned used = 0;
#pragma unroll
                for (int q = 0; q < kRedBatch; ++q) {
                    const int j = j0 - q;
                    if (j < 0) break;  // warp-uniform: the last group of a batch may be short
                    const int li = 32 * bi + j;  // position in the tile list
                    if (li <= act) {  // (warp-uniform) pixels whose last contributor is at li or later switch on
                        int nxt = -1;
#pragma unroll
                        for (int k = 0; k < PPL; ++k) {
                            const float nr = -(y0f + (float)(2 * k));
                            const int lk = last[k];
                            if (li < lk) {
                                if (k & 1) nrow[k >> 1].y = nr;
                                else nrow[k >> 1].x = nr;
                            } else {
                                nxt = max(nxt, lk - 1);
                            }
                        }
                        act = __reduce_max_sync(0xffffffffu, nxt);
                    }
                    if (STATS) {
#pragma unroll
                        for (int k = 0; k < PPL; ++k) n_eval += li < last[k];
                    }
                    Feat f;
                    load_feat(sf + j * kFeat, f);
                    const ColTerms ct = col_terms(f, nu);
                    BwdSums S;
                    const bool any = bwd_gaussian<NP, CL, STATS>(f, ct, T, nQ, G, nrow, S, n_blend);
                    used |= (unsigned)any << q;
                    const float W0 = S.W0.x + S.W0.y, W1 = S.W1.x + S.W1.y;
                    float4* slot = red + 2 * q * 32 + lane;
                    const float dx = ct.dx, dxW0 = dx * W0;
                    slot[0] = make_float4(dxW0, W1, dx * dxW0, dx * W1);
                    slot[32] = make_float4(S.W2.x + S.W2.y, W0, S.r.x + S.r.y, S.g.x + S.g.y);
                    ((float*)(red + (14 + (q >> 2)) * 32 + lane))[q & 3] = S.b.x + S.b.y;
                }
                if (used) flush_group(red, min(kRedBatch, j0 + 1), used, j0, sf, s_row[warp], dproj, lane);
            }
        };
        if (clamp_batch) walk(std::integral_constant<bool, true>());
        else walk(std::integral_constant<bool, false>());
        __syncwarp();
    }
    cp_async_wait_all();  // no copy may land in shared memory after the CTA has left
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
                       const ViewBatch& vb, const splat_image& img, const L1Fuse& l1, int32_t* status,
                       unsigned long long* stats)
{
    const uint2* rg = (const uint2*)bins.ranges;
    switch (ppl) {
    case 8: k_composite_fwd<8, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, l1, status, stats); break;
    case 4: k_composite_fwd<4, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, l1, status, stats); break;
    default: k_composite_fwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, l1, status, stats); break;
    }
}

template <bool ST>
static void bwd_launch(int ppl, int blocks, cudaStream_t st, const splat_proj& proj, const splat_bins& bins,
                       const ViewBatch& vb, const splat_image& img, const float* dL, float* dproj, int32_t* status,
                       unsigned long long* stats)
{
    const uint2* rg = (const uint2*)bins.ranges;
    switch (ppl) {
    case 8: k_composite_bwd<8, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, dL, dproj, status, stats); break;
    case 4: k_composite_bwd<4, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, dL, dproj, status, stats); break;
    default: k_composite_bwd<2, ST><<<blocks, kCompWarps * 32, 0, st>>>(proj, bins.vals, rg, bins.tile_order, vb, img, dL, dproj, status, stats); break;
    }
}

cudaError_t launch_composite_fwd(const splat_proj& proj, const splat_bins& bins, const ViewBatch& vb,
                                 const splat_image& img, const L1Fuse* l1p, int32_t* status, int ppl,
                                 unsigned long long* stats, const LaunchCtx& ctx)
{
    const L1Fuse l1 = l1p ? *l1p : L1Fuse{nullptr, 0.f, nullptr, nullptr};
    if (l1.loss) {
        const cudaError_t e = cudaMemsetAsync(l1.loss, 0, sizeof(float), ctx.stream);
        if (e != cudaSuccess) return e;
    }
    if (vb.total_tiles == 0) return cudaSuccess;
    const int bands = 8 / ppl;
    const int64_t units = (int64_t)vb.total_tiles * bands;
    const int blocks = (int)((units + kCompWarps - 1) / kCompWarps);
    count_launch();
    if (stats) fwd_launch<true>(ppl, blocks, ctx.stream, proj, bins, vb, img, l1, status, stats);
    else fwd_launch<false>(ppl, blocks, ctx.stream, proj, bins, vb, img, l1, status, nullptr);
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
