// project.cu -- slice + cull + EWA projection + SH colour (forward, one thread
// per Gaussian, all views) and its adjoint (a group of lanes per Gaussian, one
// per view, summed over views without atomics).
//
// Forward follows Alg. 1 CullGaussian / ProjGaussian4D / ProjGaussian3D:
//   4D: R = R_l R_r (Eq. 4), M = R diag(exp s), Sigma_4D = M M^T.  With m_t the
//       time row of M and M_x its three spatial rows,
//         Sigma_{1:3,4} = M_x m_t^T, Sigma_44 = |m_t|^2,
//         mu_{xyz|t} = mu_{1:3} + Sigma_{1:3,4} (t - mu_t) / Sigma_44      (Eq. 5)
//         Sigma_{xyz|t} = M_x (I - u u^T) M_x^T, u = m_t / |m_t|           (Eq. 6)
//       The projector form is algebraically Eq. 6 and stays positive
//       semi-definite in FP32 (no cancellation of two nearly equal terms).
//       Peak opacity sigmoid(o) exp(-(t - mu_t)^2 / (2 Sigma_44)).
//   3D: Sigma = R S S^T R^T (Eq. 2), peak opacity sigmoid(o).
//   EWA: Jacobian of the pinhole map at the clamped mean, 0.3 px^2 dilation,
//   radius ceil(3 sqrt(lambda_max)), tile rectangle, degree-3 SH colour.
#include "splat_internal.cuh"

namespace splat {

struct Sym3 {
    float xx, xy, xz, yy, yz, zz;
};

__device__ __forceinline__ void mat3_vec(const Sym3& S, const float v[3], float o[3])
{
    o[0] = S.xx * v[0] + S.xy * v[1] + S.xz * v[2];
    o[1] = S.xy * v[0] + S.yy * v[1] + S.yz * v[2];
    o[2] = S.xz * v[0] + S.yz * v[1] + S.zz * v[2];
}

// Camera-space EWA state shared by the forward and the adjoint.
struct Ewa {
    float xc[3];
    float z;
    float ux, uy;
    bool clx, cly;
    float J00, J02, J11, J12;
    float t0[3], t1[3];  // rows of T = J R
    float s00, s01, s11; // 2D covariance incl. dilation
    float det;
};

// r . m + t in FP32 with compensated products and sums (the Dot2 scheme of
// Ogita, Rump and Oishi, 2005): the result is the FP32 rounding of the exact
// value unless that value lies within ~1e-13 x (|r0 m0| + |r1 m1| + |r2 m2| + |t|)
// of a rounding boundary.  Used for the
// camera depth, whose float bits are the sort key: Gaussians whose exact depths
// round to the same FP32 number then tie exactly and keep their merged-index
// order, whatever the evaluation order.
__device__ __forceinline__ float dot3_exact_rounded(const float r[3], const float m[3], float t)
{
    float s = t, c = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = __fmul_rn(r[k], m[k]);
        const float pe = __fmaf_rn(r[k], m[k], -p);  // product error, exact
        const float s2 = __fadd_rn(s, p);
        const float bv = __fsub_rn(s2, s);
        const float se = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, bv)), __fsub_rn(p, bv));  // sum error, exact
        s = s2;
        c = __fadd_rn(c, __fadd_rn(pe, se));
    }
    return __fadd_rn(s, c);
}

__device__ __forceinline__ void ewa_setup(const ViewParams& vp, const float mu[3], const Sym3& S, Ewa& e)
{
#pragma unroll
    for (int r = 0; r < 2; ++r)
        e.xc[r] = vp.R[r * 3 + 0] * mu[0] + vp.R[r * 3 + 1] * mu[1] + vp.R[r * 3 + 2] * mu[2] + vp.T[r];
    e.xc[2] = dot3_exact_rounded(&vp.R[6], mu, vp.T[2]);
    e.z = e.xc[2];
    const float iz = 1.f / e.z;
    e.ux = e.xc[0] * iz;
    e.uy = e.xc[1] * iz;
    e.clx = (e.ux < -vp.limx) || (e.ux > vp.limx);
    e.cly = (e.uy < -vp.limy) || (e.uy > vp.limy);
    const float txc = e.z * fminf(vp.limx, fmaxf(-vp.limx, e.ux));
    const float tyc = e.z * fminf(vp.limy, fmaxf(-vp.limy, e.uy));
    e.J00 = vp.fx * iz;
    e.J11 = vp.fy * iz;
    e.J02 = -vp.fx * txc * iz * iz;
    e.J12 = -vp.fy * tyc * iz * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        e.t0[k] = e.J00 * vp.R[0 * 3 + k] + e.J02 * vp.R[2 * 3 + k];
        e.t1[k] = e.J11 * vp.R[1 * 3 + k] + e.J12 * vp.R[2 * 3 + k];
    }
    float St0[3], St1[3];
    mat3_vec(S, e.t0, St0);
    mat3_vec(S, e.t1, St1);
    e.s00 = e.t0[0] * St0[0] + e.t0[1] * St0[1] + e.t0[2] * St0[2] + kDilation;
    e.s01 = e.t0[0] * St1[0] + e.t0[1] * St1[1] + e.t0[2] * St1[2];
    e.s11 = e.t1[0] * St1[0] + e.t1[1] * St1[1] + e.t1[2] * St1[2] + kDilation;
    e.det = e.s00 * e.s11 - e.s01 * e.s01;
}

// weight of time frequency n at t: cos(2 pi n t), t in units of the sequence length
__device__ __forceinline__ float time_weight(int n, float t) { return cospif(2.f * (float)n * t); }

// rgb += w sum_k c_k Y_k for one block of coefficients c (16 x 3, k*3 + channel)
__device__ __forceinline__ void sh_accumulate(const float c[48], float w, const float Y[16], float& r, float& g,
                                              float& b)
{
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        r += w * c[3 * k + 0] * Y[k];
        g += w * c[3 * k + 1] * Y[k];
        b += w * c[3 * k + 2] * Y[k];
    }
}

// rgb = 0.5 + sum_{n=0..T} cos(2 pi n t) sum_k c_nk Y_k(d) (unclamped); T = 0: plain SH.
// Y receives the SH basis at d, c0 the coefficients of block 0.
template <int DT>
__device__ __forceinline__ void sh_rgb(const void* sh_base, int64_t row, int T, float t, const float dir[3],
                                       float rgb[3], float Y[16], float c0[48])
{
    using S = Storage<DT>;
    sh_basis(dir[0], dir[1], dir[2], Y);
    const typename S::T* p = (const typename S::T*)sh_base + row * 48 * (T + 1);
    load_sh48<DT>(p, c0);
    float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
    for (int k = 0; k < 16; ++k) {  // block 0 (weight 1): exactly the plain SH sum
        r += c0[3 * k + 0] * Y[k];
        g += c0[3 * k + 1] * Y[k];
        b += c0[3 * k + 2] * Y[k];
    }
    for (int n = 1; n <= T; ++n) {
        float cn[48];
        load_sh48<DT>(p + 48 * n, cn);
        sh_accumulate(cn, time_weight(n, t), Y, r, g, b);
    }
    rgb[0] = r; rgb[1] = g; rgb[2] = b;
}

// w[k] += tw sum_c gc[c] c_kc for one block of coefficients (16 x 3, k*3 + c),
// streamed from storage 16 bytes at a time (never all 48 in registers).
template <int DT>
__device__ __forceinline__ void sh_weights(const typename Storage<DT>::T* p, const float gc[3], float tw, float w[16])
{
    const float g0 = tw * gc[0], g1 = tw * gc[1], g2 = tw * gc[2];
    auto add = [&](int e, float c) { w[e / 3] += (e % 3 == 0 ? g0 : (e % 3 == 1 ? g1 : g2)) * c; };
    if constexpr (DT == SPLAT_F32) {
        const float4* p4 = (const float4*)p;
#pragma unroll
        for (int qq = 0; qq < 12; ++qq) {
            const float4 v = __ldg(p4 + qq);
            add(4 * qq, v.x); add(4 * qq + 1, v.y); add(4 * qq + 2, v.z); add(4 * qq + 3, v.w);
        }
    } else {
        const uint4* p4 = (const uint4*)p;
#pragma unroll
        for (int qq = 0; qq < 6; ++qq) {
            const uint4 v = __ldg(p4 + qq);
            const typename Storage<DT>::T* h = (const typename Storage<DT>::T*)&v;
#pragma unroll
            for (int e = 0; e < 8; ++e)
                add(8 * qq + e, DT == SPLAT_BF16 ? __bfloat162float(((const __nv_bfloat16*)h)[e])
                                                 : __half2float(((const __half*)h)[e]));
        }
    }
}

// View-independent geometry of one merged Gaussian.
struct Geo {
    float mu[3];   // world mean (3D) or mu_x (4D)
    Sym3 S;        // covariance (sliced for 4D)
    float op;      // sigmoid(o)
    // 4D only
    float mu_t, inv_n2;
    float b[3];    // Sigma_{1:3,4}
};

template <int DT>
__device__ __forceinline__ void load_geo(const splat_g3& g3, const splat_g4& g4, int64_t i, bool is4, Geo& G)
{
    if (is4) {
        float m[4], ls[4], ql[4], qr[4];
        load4<DT>(g4.mean, i, m);
        load4<DT>(g4.log_scale, i, ls);
        load4<DT>(g4.ql, i, ql);
        load4<DT>(g4.qr, i, qr);
        const float o = load1<DT>(g4.opacity, i);
        const float il = inv_norm4(ql), ir = inv_norm4(qr);
#pragma unroll
        for (int k = 0; k < 4; ++k) { ql[k] *= il; qr[k] *= ir; }
        float R[16];
        rot4(ql, qr, R);
        float s[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] = expf(ls[k]);
        float M[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) M[r * 4 + k] = R[r * 4 + k] * s[k];
        const float* mt = &M[12];
        const float n2 = mt[0] * mt[0] + mt[1] * mt[1] + mt[2] * mt[2] + mt[3] * mt[3];
        const float in = rsqrtf(n2);
        const float u[4] = {mt[0] * in, mt[1] * in, mt[2] * in, mt[3] * in};
        float B[12];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            const float vr = M[r * 4 + 0] * u[0] + M[r * 4 + 1] * u[1] + M[r * 4 + 2] * u[2] + M[r * 4 + 3] * u[3];
            G.b[r] = M[r * 4 + 0] * mt[0] + M[r * 4 + 1] * mt[1] + M[r * 4 + 2] * mt[2] + M[r * 4 + 3] * mt[3];
#pragma unroll
            for (int k = 0; k < 4; ++k) B[r * 4 + k] = M[r * 4 + k] - vr * u[k];
        }
        auto dot4 = [&](int a, int c) {
            return B[a * 4 + 0] * B[c * 4 + 0] + B[a * 4 + 1] * B[c * 4 + 1] + B[a * 4 + 2] * B[c * 4 + 2] +
                   B[a * 4 + 3] * B[c * 4 + 3];
        };
        G.S = {dot4(0, 0), dot4(0, 1), dot4(0, 2), dot4(1, 1), dot4(1, 2), dot4(2, 2)};
        G.mu[0] = m[0]; G.mu[1] = m[1]; G.mu[2] = m[2];
        G.mu_t = m[3];
        G.inv_n2 = 1.f / n2;
        G.op = sigmoidf_(o);
    } else {
        const int64_t j = i - g4.n;
        float q[4], ls[3];
        load3<DT>(g3.mean, j, G.mu);
        load3<DT>(g3.log_scale, j, ls);
        load4<DT>(g3.quat, j, q);
        const float o = load1<DT>(g3.opacity, j);
        const float iq = inv_norm4(q);
        float R[9];
        quat_to_rot(q[0] * iq, q[1] * iq, q[2] * iq, q[3] * iq, R);
        float M[9];
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int k = 0; k < 3; ++k) M[r * 3 + k] = R[r * 3 + k] * expf(ls[k]);
        auto dot3 = [&](int a, int c) {
            return M[a * 3 + 0] * M[c * 3 + 0] + M[a * 3 + 1] * M[c * 3 + 1] + M[a * 3 + 2] * M[c * 3 + 2];
        };
        G.S = {dot3(0, 0), dot3(0, 1), dot3(0, 2), dot3(1, 1), dot3(1, 2), dot3(2, 2)};
        G.op = sigmoidf_(o);
        G.mu_t = 0.f;
        G.inv_n2 = 0.f;
        G.b[0] = G.b[1] = G.b[2] = 0.f;
    }
}

// World mean and peak opacity of Gaussian G at time t (Eq. 5 and the temporal factor).
__device__ __forceinline__ void at_time(const Geo& G, bool is4, float t, float mu[3], float& alpha, float& p_t,
                                        float& dt)
{
    if (is4) {
        dt = t - G.mu_t;
        const float f = dt * G.inv_n2;
#pragma unroll
        for (int k = 0; k < 3; ++k) mu[k] = G.mu[k] + G.b[k] * f;
        p_t = expf(-0.5f * dt * dt * G.inv_n2);
        alpha = G.op * p_t;
    } else {
        mu[0] = G.mu[0]; mu[1] = G.mu[1]; mu[2] = G.mu[2];
        p_t = 1.f;
        dt = 0.f;
        alpha = G.op;
    }
}

template <int DT>
__global__ void __launch_bounds__(128, 7) k_slice_project(splat_g3 g3, splat_g4 g4, ViewBatch vb, splat_proj out,
                                                       int32_t* status)
{
    const int64_t N = out.n;
    const int64_t n4 = g4.n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
        const bool is4 = i < n4;
        Geo G;
        load_geo<DT>(g3, g4, i, is4, G);
        const void* sh_base = is4 ? g4.sh : g3.sh;
        const int64_t sh_row = is4 ? i : i - n4;
        // non-finite parameters: reported (row of the first view) and the Gaussian culled
        const float gsum = G.mu[0] + G.mu[1] + G.mu[2] + G.S.xx + G.S.xy + G.S.xz + G.S.yy + G.S.yz + G.S.zz + G.op +
                           (is4 ? G.mu_t + G.inv_n2 : 0.f);
        const bool bad = !isfinite(gsum);
        if (bad) set_status(status, SPLAT_ERR_NONFINITE, SPLAT_STAGE_SLICE_PROJECT, i);
        for (int v = 0; v < vb.V; ++v) {
            const ViewParams& vp = vb.v[v];
            const int64_t row = v * N + i;
            if (bad) {
                ((float2*)out.xy)[row] = make_float2(0.f, 0.f);
                ((float4*)out.conic_opacity)[row] = make_float4(0.f, 0.f, 0.f, 0.f);
                ((float4*)out.rgb_depth)[row] = make_float4(0.f, 0.f, 0.f, 0.f);
                ((int4*)out.rect)[row] = make_int4(0, 0, 0, 0);
                out.radius[row] = 0;
                out.n_tiles[row] = 0;
                continue;
            }
            float mu[3], alpha, p_t, dt;
            at_time(G, is4, vp.t, mu, alpha, p_t, dt);
            Ewa e;
            ewa_setup(vp, mu, G.S, e);
            bool culled = !(e.z > vp.z_near) || !(alpha >= kAlphaMin) || !(e.det > 0.f);
            float4 co = make_float4(0.f, 0.f, 0.f, 0.f), rd = make_float4(0.f, 0.f, 0.f, 0.f);
            float2 xy = make_float2(0.f, 0.f);
            int4 rect = make_int4(0, 0, 0, 0);
            int radius = 0;
            unsigned n_tiles = 0;
            if (!culled) {
                const float idet = 1.f / e.det;
                co = make_float4(e.s11 * idet, -e.s01 * idet, e.s00 * idet, alpha);
                // lambda_max = mid + sqrt(max(0.1, mid^2 - det)); mid^2 - det is evaluated as
                // ((s00 - s11)/2)^2 + s01^2, the same number without the FP32 cancellation
                const float mid = 0.5f * (e.s00 + e.s11);
                const float hd = 0.5f * (e.s00 - e.s11);
                const float lam = mid + sqrtf(fmaxf(0.1f, hd * hd + e.s01 * e.s01));
                const float rf = ceilf(3.f * sqrtf(lam));
                const float px = vp.fx * e.ux + vp.cx, py = vp.fy * e.uy + vp.cy;
                xy = make_float2(px, py);
                if (!isfinite(px) || !isfinite(py) || !isfinite(rf) || !isfinite(co.x) || !isfinite(co.y) ||
                    !isfinite(co.z) || !isfinite(alpha)) {
                    set_status(status, SPLAT_ERR_NONFINITE, SPLAT_STAGE_SLICE_PROJECT, row);
                    culled = true;
                } else {
                    const float inv = 1.f / kTile;
                    const int x0 = min(max((int)floorf((px - rf) * inv), 0), vp.TX);
                    const int x1 = min(max((int)ceilf((px + rf) * inv), 0), vp.TX);
                    const int y0 = min(max((int)floorf((py - rf) * inv), 0), vp.TY);
                    const int y1 = min(max((int)ceilf((py + rf) * inv), 0), vp.TY);
                    n_tiles = (unsigned)((x1 - x0) * (y1 - y0));
                    if (n_tiles == 0) {
                        culled = true;
                    } else {
                        rect = make_int4(x0, y0, x1, y1);
                        radius = (int)rf;
                        float d[3] = {mu[0] - vp.cam[0], mu[1] - vp.cam[1], mu[2] - vp.cam[2]};
                        const float id = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                        d[0] *= id; d[1] *= id; d[2] *= id;
                        float rgb[3], Y[16], c0[48];
                        sh_rgb<DT>(sh_base, sh_row, is4 ? g4.sh_time : 0, vp.t, d, rgb, Y, c0);
                        rd = make_float4(fmaxf(rgb[0], 0.f), fmaxf(rgb[1], 0.f), fmaxf(rgb[2], 0.f), e.z);
                        if (!isfinite(rgb[0] + rgb[1] + rgb[2])) {  // non-finite colour coefficients
                            set_status(status, SPLAT_ERR_NONFINITE, SPLAT_STAGE_SLICE_PROJECT, row);
                            culled = true;
                        }
                    }
                }
            }
            if (culled) {
                co = make_float4(0.f, 0.f, 0.f, 0.f);
                rd = make_float4(0.f, 0.f, 0.f, 0.f);
                xy = make_float2(0.f, 0.f);
                rect = make_int4(0, 0, 0, 0);
                radius = 0;
                n_tiles = 0;
            }
            ((float2*)out.xy)[row] = xy;
            ((float4*)out.conic_opacity)[row] = co;
            ((float4*)out.rgb_depth)[row] = rd;
            ((int4*)out.rect)[row] = rect;
            out.radius[row] = radius;
            out.n_tiles[row] = n_tiles;
        }
    }
}

// ---------------------------------------------------------------------------
// Adjoint (A11): dproj rows -> parameter gradients, summed over views.
// ---------------------------------------------------------------------------

struct SymG {  // symmetric gradient, dL = sum_ij G_ij dS_ij
    float xx, xy, xz, yy, yz, zz;
};

// Reverse of ewa_setup + px/py + conic for one view.  Adds dL/dmu (world) and
// the symmetric dL/dSigma.
__device__ __forceinline__ void ewa_backward(const ViewParams& vp, const Ewa& e, const Sym3& S, const float dp[5],
                                             float gmu[3], SymG& GS)
{
    // conic Q = Sigma2^-1, G2 = -Q G_Q Q with G_Q = [[da, db/2], [db/2, dc]]
    const float idet = 1.f / e.det;
    const float q00 = e.s11 * idet, q01 = -e.s01 * idet, q11 = e.s00 * idet;
    const float ga = dp[2], gb = 0.5f * dp[3], gc = dp[4];
    // A = Q G_Q
    const float a00 = q00 * ga + q01 * gb, a01 = q00 * gb + q01 * gc;
    const float a10 = q01 * ga + q11 * gb, a11 = q01 * gb + q11 * gc;
    const float g00 = -(a00 * q00 + a01 * q01);
    const float g01 = -(a00 * q01 + a01 * q11);
    const float g11 = -(a10 * q01 + a11 * q11);
    // Sigma2 = T Sigma T^T:  G_Sigma += T^T G2 T,  G_T = 2 G2 T Sigma
    const float* t0 = e.t0;
    const float* t1 = e.t1;
    GS.xx += g00 * t0[0] * t0[0] + 2.f * g01 * t0[0] * t1[0] + g11 * t1[0] * t1[0];
    GS.yy += g00 * t0[1] * t0[1] + 2.f * g01 * t0[1] * t1[1] + g11 * t1[1] * t1[1];
    GS.zz += g00 * t0[2] * t0[2] + 2.f * g01 * t0[2] * t1[2] + g11 * t1[2] * t1[2];
    GS.xy += g00 * t0[0] * t0[1] + g01 * (t0[0] * t1[1] + t1[0] * t0[1]) + g11 * t1[0] * t1[1];
    GS.xz += g00 * t0[0] * t0[2] + g01 * (t0[0] * t1[2] + t1[0] * t0[2]) + g11 * t1[0] * t1[2];
    GS.yz += g00 * t0[1] * t0[2] + g01 * (t0[1] * t1[2] + t1[1] * t0[2]) + g11 * t1[1] * t1[2];
    float St0[3], St1[3];
    mat3_vec(S, t0, St0);
    mat3_vec(S, t1, St1);
    float gt0[3], gt1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        gt0[k] = 2.f * (g00 * St0[k] + g01 * St1[k]);
        gt1[k] = 2.f * (g01 * St0[k] + g11 * St1[k]);
    }
    // T rows: t0 = J00 R0 + J02 R2, t1 = J11 R1 + J12 R2
    const float* R = vp.R;
    const float gJ00 = gt0[0] * R[0] + gt0[1] * R[1] + gt0[2] * R[2];
    const float gJ02 = gt0[0] * R[6] + gt0[1] * R[7] + gt0[2] * R[8];
    const float gJ11 = gt1[0] * R[3] + gt1[1] * R[4] + gt1[2] * R[5];
    const float gJ12 = gt1[0] * R[6] + gt1[1] * R[7] + gt1[2] * R[8];
    const float z = e.z, iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
    const float fx = vp.fx, fy = vp.fy;
    float gx = 0.f, gy = 0.f, gz = 0.f;
    gz += -fx * iz2 * gJ00 - fy * iz2 * gJ11;
    if (!e.clx) {
        gx += -fx * iz2 * gJ02;
        gz += 2.f * fx * e.xc[0] * iz3 * gJ02;
    } else {
        const float c = e.ux > 0.f ? vp.limx : -vp.limx;
        gz += fx * c * iz2 * gJ02;
    }
    if (!e.cly) {
        gy += -fy * iz2 * gJ12;
        gz += 2.f * fy * e.xc[1] * iz3 * gJ12;
    } else {
        const float c = e.uy > 0.f ? vp.limy : -vp.limy;
        gz += fy * c * iz2 * gJ12;
    }
    // px = fx x / z + cx, py = fy y / z + cy
    gx += dp[0] * fx * iz;
    gz += -dp[0] * fx * e.xc[0] * iz2;
    gy += dp[1] * fy * iz;
    gz += -dp[1] * fy * e.xc[1] * iz2;
    // xc = R mu + T
#pragma unroll
    for (int k = 0; k < 3; ++k) gmu[k] += R[0 * 3 + k] * gx + R[1 * 3 + k] * gy + R[2 * 3 + k] * gz;
}

__device__ __forceinline__ void normalise_backward(const float q[4], const float g[4], float out[4])
{
    const float in = inv_norm4(q);
    const float qn[4] = {q[0] * in, q[1] * in, q[2] * in, q[3] * in};
    const float dot = qn[0] * g[0] + qn[1] * g[1] + qn[2] * g[2] + qn[3] * g[3];
#pragma unroll
    for (int k = 0; k < 4; ++k) out[k] = (g[k] - qn[k] * dot) * in;
}

constexpr int kAdjThreads = 128;  // threads per block of the adjoint

// One lane's share of the colour gradient, staged for its group: the view's
// dL/drgb where the colour is not clamped (gc), the view's timestamp, and the
// SH basis at the view direction.  The group sums dsh_n[k][c] = sum_v
// cos(2 pi n t_v) gc_v[c] Y_v[k] from these.
struct ShPart {
    float4 gct;   // (gc_r, gc_g, gc_b, t_v); zero when the lane's view does not see the Gaussian
    float4 Y[4];  // Y_0 .. Y_15
};

// View-parallel adjoint.  A warp takes 32 consecutive Gaussians at a time.
// Each lane computes one Gaussian's view-independent geometry (Eq. 2 / Eq. 4
// and the projector form of Eq. 6) into shared memory.  Then, in L sub-batches
// of 32 / L Gaussians, a group of L lanes (L: the
// view count rounded up to a power of two) per Gaussian, lane q chaining view
// q's 2D gradients through the colour and the EWA projection; the group sums
// its views -- the 15 view-summed quantities by shuffles, the SH gradient from
// the staged ShPart (each lane writes 16 / L of the 16 SH functions, all time
// blocks) -- and parks the 15 sums in shared memory.  Then every lane chains
// one Gaussian's sums through the slicing / covariance and writes its other
// gradients.  No atomics; the views' memory requests are independent of one
// another, and the heavy view-independent chain runs on full warps.
template <int DT, int L>
__global__ void __launch_bounds__(kAdjThreads, 6) k_adjoint(splat_g3 g3, splat_g4 g4, ViewBatch vb, splat_proj proj,
                                                 const float* __restrict__ dproj, splat_grads3 dg3,
                                                 splat_grads4 dg4, int32_t* status)
{
    static_assert(L == 1 || L == 2 || L == 4 || L == 8 || L == 16, "lanes per Gaussian");
    constexpr int KPL = 16 / L;  // SH functions whose gradient a lane writes
    constexpr int GPS = 32 / L;  // Gaussians per sub-batch of a warp
    __shared__ ShPart s_part[kAdjThreads];
    __shared__ float s_sum[kAdjThreads / 32][15][32];  // per warp: the 15 view sums of its 32 Gaussians
    __shared__ float s_geo[kAdjThreads / 32][15][32];  // per warp: the view-independent geometry (Geo)
    __shared__ ViewParams s_view[SPLAT_MAX_VIEWS];  // lanes of one warp read different views
    if (status_failed(status)) return;
    for (int v = threadIdx.x; v < vb.V; v += blockDim.x) s_view[v] = vb.v[v];
    __syncthreads();
    const int64_t N = proj.n;
    const int64_t n4 = g4.n;
    const int lane = threadIdx.x & 31, q = threadIdx.x % L, warp = threadIdx.x >> 5;
    const int gbase = threadIdx.x - q;  // first lane of the group
    float (*sums)[32] = s_sum[warp];
    float (*geo)[32] = s_geo[warp];
    // every lane of a warp takes the same number of trips (the group sums are warp collectives)
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t c0 = (int64_t)blockIdx.x * blockDim.x + warp * 32; c0 < N; c0 += stride) {
      {
        // the geometry of Gaussian c0 + lane, once (the view lanes below share it)
        const int64_t i = c0 + lane;
        if (i < N) {
            Geo G;
            load_geo<DT>(g3, g4, i, i < n4, G);
            const float g15[15] = {G.mu[0], G.mu[1], G.mu[2], G.S.xx, G.S.xy, G.S.xz, G.S.yy, G.S.yz, G.S.zz,
                                   G.op, G.mu_t, G.inv_n2, G.b[0], G.b[1], G.b[2]};
#pragma unroll
            for (int e = 0; e < 15; ++e) geo[e][lane] = g15[e];
        }
        __syncwarp();
      }
      for (int sb = 0; sb < L; ++sb) {
        const int slot = sb * GPS + lane / L;  // the Gaussian's lane in the chain phase
        const int64_t i = c0 + slot;
        const bool valid = i < N;
        const bool is4 = i < n4;
        const int Tn = is4 ? g4.sh_time : 0;  // time frequencies of the colour
        SymG GS = {0, 0, 0, 0, 0, 0};
        float gmu_sum[3] = {0, 0, 0};   // sum_v dL/dmu_v
        float gmu_dt[3] = {0, 0, 0};    // sum_v dL/dmu_v (t_v - mu_t)       (4D)
        float gal = 0.f;                // sum_v dL/dalpha_v p_v            (opacity)
        float gp_dt = 0.f, gp_dt2 = 0.f;// sum_v g_p p dt, sum_v g_p p dt^2/2 (4D)
        ShPart part;
        part.gct = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < 4; ++k) part.Y[k] = make_float4(0.f, 0.f, 0.f, 0.f);
        Geo G;
        const int v = q;
        const int64_t row = (int64_t)v * N + i;
        if (valid && v < vb.V && proj.radius[row] != 0) {
            G.mu[0] = geo[0][slot]; G.mu[1] = geo[1][slot]; G.mu[2] = geo[2][slot];
            G.S = {geo[3][slot], geo[4][slot], geo[5][slot], geo[6][slot], geo[7][slot], geo[8][slot]};
            G.op = geo[9][slot]; G.mu_t = geo[10][slot]; G.inv_n2 = geo[11][slot];
            G.b[0] = geo[12][slot]; G.b[1] = geo[13][slot]; G.b[2] = geo[14][slot];
            const typename Storage<DT>::T* shp =
                (const typename Storage<DT>::T*)(is4 ? g4.sh : g3.sh) + (is4 ? i : i - n4) * 48 * (Tn + 1);
            const ViewParams& vp = s_view[v];
            const float4* dq = (const float4*)(dproj + row * 12);
            const float4 d0 = dq[0], d1 = dq[1], d2 = dq[2];
            const float dp[9] = {d0.x, d0.y, d0.z, d0.w, d1.x, d1.y, d1.z, d1.w, d2.x};
            float mu[3], alpha, p_t, dt;
            at_time(G, is4, vp.t, mu, alpha, p_t, dt);
            Ewa e;
            ewa_setup(vp, mu, G.S, e);
            float gmu[3] = {0.f, 0.f, 0.f};
            ewa_backward(vp, e, G.S, dp, gmu, GS);
            // colour: rgb = max(0, 0.5 + sum_k sh_k Y_k(d)), d = (mu - cam)/|mu - cam|.  The
            // forward stored max(0, rgb) from the same evaluation, so a channel is clamped
            // exactly where its stored value is 0
            float d[3] = {mu[0] - vp.cam[0], mu[1] - vp.cam[1], mu[2] - vp.cam[2]};
            const float id = rsqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            d[0] *= id; d[1] *= id; d[2] *= id;
            const float4 rd = ((const float4*)proj.rgb_depth)[row];
            const float gc[3] = {rd.x > 0.f ? dp[6] : 0.f, rd.y > 0.f ? dp[7] : 0.f, rd.z > 0.f ? dp[8] : 0.f};
            float w[16];  // <dL/drgb, effective coefficients of Y_k at t>
#pragma unroll
            for (int k = 0; k < 16; ++k) w[k] = 0.f;
            sh_weights<DT>(shp, gc, 1.f, w);
            for (int n = 1; n <= Tn; ++n) sh_weights<DT>(shp + 48 * n, gc, time_weight(n, vp.t), w);
            float Y[16];
            sh_basis(d[0], d[1], d[2], Y);
            part.gct = make_float4(gc[0], gc[1], gc[2], vp.t);
#pragma unroll
            for (int k = 0; k < 4; ++k) part.Y[k] = make_float4(Y[4 * k], Y[4 * k + 1], Y[4 * k + 2], Y[4 * k + 3]);
            float gdir[3];
            sh_basis_grad(d[0], d[1], d[2], w, gdir);
            const float dd = d[0] * gdir[0] + d[1] * gdir[1] + d[2] * gdir[2];
#pragma unroll
            for (int k = 0; k < 3; ++k) gmu[k] += (gdir[k] - d[k] * dd) * id;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                gmu_sum[k] = gmu[k];
                gmu_dt[k] = gmu[k] * dt;
            }
            gal = dp[5] * p_t;
            const float gp = dp[5] * G.op * p_t;  // dL/dp times p
            gp_dt = gp * dt;
            gp_dt2 = gp * 0.5f * dt * dt;
        }
        // sums over the group's views
        if (L > 1) {
#pragma unroll
            for (int o = 1; o < L; o <<= 1) {
                auto add = [&](float& x) { x += __shfl_xor_sync(0xffffffffu, x, o); };
                add(GS.xx); add(GS.xy); add(GS.xz); add(GS.yy); add(GS.yz); add(GS.zz);
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    add(gmu_sum[k]);
                    add(gmu_dt[k]);
                }
                add(gal); add(gp_dt); add(gp_dt2);
            }
        }
        s_part[threadIdx.x] = part;
        __syncwarp();
        if (valid) {
            // SH gradient of functions k0 .. k0 + KPL - 1, every time block
            const int k0 = q * KPL;
            float* shrow = (is4 ? dg4.sh + i * (Tn + 1) * 48 : dg3.sh + (i - n4) * 48) + 3 * k0;
            for (int n = 0; n <= Tn; ++n) {
                float acc[3 * KPL];
#pragma unroll
                for (int e = 0; e < 3 * KPL; ++e) acc[e] = 0.f;
#pragma unroll
                for (int j = 0; j < L; ++j) {
                    const ShPart& pj = s_part[gbase + j];
                    const float4 g = pj.gct;
                    const float tw = n == 0 ? 1.f : time_weight(n, g.w);
                    const float gr = tw * g.x, gg = tw * g.y, gb = tw * g.z;
#pragma unroll
                    for (int kk = 0; kk < KPL; ++kk) {
                        const float4 y4 = pj.Y[(k0 + kk) >> 2];
                        const int c = (k0 + kk) & 3;
                        const float y = c == 0 ? y4.x : (c == 1 ? y4.y : (c == 2 ? y4.z : y4.w));
                        acc[3 * kk + 0] += gr * y;
                        acc[3 * kk + 1] += gg * y;
                        acc[3 * kk + 2] += gb * y;
                    }
                }
                float* out = shrow + n * 48;
                if constexpr ((3 * KPL) % 4 == 0) {
#pragma unroll
                    for (int e = 0; e < 3 * KPL; e += 4)
                        *(float4*)(out + e) = make_float4(acc[e], acc[e + 1], acc[e + 2], acc[e + 3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 3 * KPL; ++e) out[e] = acc[e];
                }
            }
        }
        if (q == 0) {
            const float v15[15] = {GS.xx, GS.xy, GS.xz, GS.yy, GS.yz, GS.zz, gmu_sum[0], gmu_sum[1], gmu_sum[2],
                                   gmu_dt[0], gmu_dt[1], gmu_dt[2], gal, gp_dt, gp_dt2};
#pragma unroll
            for (int e = 0; e < 15; ++e) sums[e][slot] = v15[e];
        }
        __syncwarp();  // s_part is rewritten in the next sub-batch, sums are read below
      }
        // every lane: the view-independent chain of one Gaussian's summed gradients
        const int64_t i = c0 + lane;
        if (i < N) {
        const bool is4 = i < n4;
        const SymG GS = {sums[0][lane], sums[1][lane], sums[2][lane], sums[3][lane], sums[4][lane], sums[5][lane]};
        const float gmu_sum[3] = {sums[6][lane], sums[7][lane], sums[8][lane]};
        const float gmu_dt[3] = {sums[9][lane], sums[10][lane], sums[11][lane]};
        const float gal = sums[12][lane], gp_dt = sums[13][lane], gp_dt2 = sums[14][lane];
        if (is4) {
                // Rebuild the 4D factors (view independent).
                float m[4], ls[4], ql[4], qr[4];
                load4<DT>(g4.mean, i, m);
                load4<DT>(g4.log_scale, i, ls);
                load4<DT>(g4.ql, i, ql);
                load4<DT>(g4.qr, i, qr);
                const float o = load1<DT>(g4.opacity, i);
                float qln[4], qrn[4];
                const float il = inv_norm4(ql), ir = inv_norm4(qr);
    #pragma unroll
                for (int k = 0; k < 4; ++k) { qln[k] = ql[k] * il; qrn[k] = qr[k] * ir; }
                float R[16], s[4], M[16];
                rot4(qln, qrn, R);
    #pragma unroll
                for (int k = 0; k < 4; ++k) s[k] = expf(ls[k]);
    #pragma unroll
                for (int r = 0; r < 4; ++r)
    #pragma unroll
                    for (int k = 0; k < 4; ++k) M[r * 4 + k] = R[r * 4 + k] * s[k];
                const float* mt = &M[12];
                const float n2 = mt[0] * mt[0] + mt[1] * mt[1] + mt[2] * mt[2] + mt[3] * mt[3];
                const float in = rsqrtf(n2), in2 = 1.f / n2;
                const float u[4] = {mt[0] * in, mt[1] * in, mt[2] * in, mt[3] * in};
                float vx[3], B[12], b[3];
    #pragma unroll
                for (int r = 0; r < 3; ++r) {
                    vx[r] = M[r * 4 + 0] * u[0] + M[r * 4 + 1] * u[1] + M[r * 4 + 2] * u[2] + M[r * 4 + 3] * u[3];
                    b[r] = M[r * 4 + 0] * mt[0] + M[r * 4 + 1] * mt[1] + M[r * 4 + 2] * mt[2] + M[r * 4 + 3] * mt[3];
    #pragma unroll
                    for (int k = 0; k < 4; ++k) B[r * 4 + k] = M[r * 4 + k] - vx[r] * u[k];
                }
                // Sigma3 = B B^T: G_B = 2 G_S B
                const float Gs[9] = {GS.xx, GS.xy, GS.xz, GS.xy, GS.yy, GS.yz, GS.xz, GS.yz, GS.zz};
                float GB[12];
    #pragma unroll
                for (int r = 0; r < 3; ++r)
    #pragma unroll
                    for (int k = 0; k < 4; ++k)
                        GB[r * 4 + k] = 2.f * (Gs[r * 3 + 0] * B[0 * 4 + k] + Gs[r * 3 + 1] * B[1 * 4 + k] +
                                               Gs[r * 3 + 2] * B[2 * 4 + k]);
                // B = M_x - (M_x u) u^T
                float GBu[3];
    #pragma unroll
                for (int r = 0; r < 3; ++r) GBu[r] = GB[r * 4 + 0] * u[0] + GB[r * 4 + 1] * u[1] + GB[r * 4 + 2] * u[2] + GB[r * 4 + 3] * u[3];
                float GM[16];
    #pragma unroll
                for (int r = 0; r < 3; ++r)
    #pragma unroll
                    for (int k = 0; k < 4; ++k) GM[r * 4 + k] = GB[r * 4 + k] - GBu[r] * u[k];
                float gu[4];
    #pragma unroll
                for (int k = 0; k < 4; ++k)
                    gu[k] = -(M[0 * 4 + k] * GBu[0] + M[1 * 4 + k] * GBu[1] + M[2 * 4 + k] * GBu[2]) -
                            (GB[0 * 4 + k] * vx[0] + GB[1 * 4 + k] * vx[1] + GB[2 * 4 + k] * vx[2]);
                // mu3 = mu_x + M_x m_t dt / n2 (summed over views through gmu_dt)
                const float a_b = gmu_dt[0] * b[0] + gmu_dt[1] * b[1] + gmu_dt[2] * b[2];
                float gmt[4];
    #pragma unroll
                for (int k = 0; k < 4; ++k) {
    #pragma unroll
                    for (int r = 0; r < 3; ++r) GM[r * 4 + k] += gmu_dt[r] * mt[k] * in2;
                    gmt[k] = (M[0 * 4 + k] * gmu_dt[0] + M[1 * 4 + k] * gmu_dt[1] + M[2 * 4 + k] * gmu_dt[2]) * in2;
                }
                float gn2 = -a_b * in2 * in2 + gp_dt2 * in2 * in2;
                const float gmu_t = -(gmu_sum[0] * b[0] + gmu_sum[1] * b[1] + gmu_sum[2] * b[2]) * in2 + gp_dt * in2;
                // u = m_t / |m_t|
                const float ugu = u[0] * gu[0] + u[1] * gu[1] + u[2] * gu[2] + u[3] * gu[3];
    #pragma unroll
                for (int k = 0; k < 4; ++k) gmt[k] += (gu[k] - u[k] * ugu) * in + 2.f * mt[k] * gn2;
    #pragma unroll
                for (int k = 0; k < 4; ++k) GM[12 + k] = gmt[k];
                // M = R diag(s)
                float GR[16], gls[4];
    #pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float acc = 0.f;
    #pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        GR[r * 4 + k] = GM[r * 4 + k] * s[k];
                        acc += GM[r * 4 + k] * R[r * 4 + k];
                    }
                    gls[k] = acc * s[k];
                }
                // R = L Rr:  G_L = G_R Rr^T,  G_Rr = L^T G_R
                const float a = qln[0], bb = qln[1], c = qln[2], dd = qln[3];
                const float p = qrn[0], q = qrn[1], rr = qrn[2], ss = qrn[3];
                const float Lm[16] = {a, -bb, -c, -dd, bb, a, -dd, c, c, dd, a, -bb, dd, -c, bb, a};
                const float Q[16] = {p, -q, -rr, -ss, q, p, ss, -rr, rr, -ss, p, q, ss, rr, -q, p};
                float GL[16], GQ[16];
    #pragma unroll
                for (int r = 0; r < 4; ++r)
    #pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        GL[r * 4 + k] = GR[r * 4 + 0] * Q[k * 4 + 0] + GR[r * 4 + 1] * Q[k * 4 + 1] +
                                        GR[r * 4 + 2] * Q[k * 4 + 2] + GR[r * 4 + 3] * Q[k * 4 + 3];
                        GQ[r * 4 + k] = Lm[0 * 4 + r] * GR[0 * 4 + k] + Lm[1 * 4 + r] * GR[1 * 4 + k] +
                                        Lm[2 * 4 + r] * GR[2 * 4 + k] + Lm[3 * 4 + r] * GR[3 * 4 + k];
                    }
                const float gan[4] = {GL[0] + GL[5] + GL[10] + GL[15], -GL[1] + GL[4] - GL[11] + GL[14],
                                      -GL[2] + GL[7] + GL[8] - GL[13], -GL[3] - GL[6] + GL[9] + GL[12]};
                const float gbn[4] = {GQ[0] + GQ[5] + GQ[10] + GQ[15], -GQ[1] + GQ[4] + GQ[11] - GQ[14],
                                      -GQ[2] - GQ[7] + GQ[8] + GQ[13], -GQ[3] + GQ[6] - GQ[9] + GQ[12]};
                float gql[4], gqr[4];
                normalise_backward(ql, gan, gql);
                normalise_backward(qr, gbn, gqr);
                const float sg = sigmoidf_(o);
                ((float4*)dg4.mean)[i] = make_float4(gmu_sum[0], gmu_sum[1], gmu_sum[2], gmu_t);
                ((float4*)dg4.log_scale)[i] = make_float4(gls[0], gls[1], gls[2], gls[3]);
                ((float4*)dg4.ql)[i] = make_float4(gql[0], gql[1], gql[2], gql[3]);
                ((float4*)dg4.qr)[i] = make_float4(gqr[0], gqr[1], gqr[2], gqr[3]);
                dg4.opacity[i] = gal * sg * (1.f - sg);
        } else {
                const int64_t j = i - n4;
                float q[4], ls[3];
                load4<DT>(g3.quat, j, q);
                load3<DT>(g3.log_scale, j, ls);
                const float o = load1<DT>(g3.opacity, j);
                const float iq = inv_norm4(q);
                const float w = q[0] * iq, x = q[1] * iq, y = q[2] * iq, z = q[3] * iq;
                float R[9], s[3], M[9];
                quat_to_rot(w, x, y, z, R);
    #pragma unroll
                for (int k = 0; k < 3; ++k) s[k] = expf(ls[k]);
    #pragma unroll
                for (int r = 0; r < 3; ++r)
    #pragma unroll
                    for (int k = 0; k < 3; ++k) M[r * 3 + k] = R[r * 3 + k] * s[k];
                const float Gs[9] = {GS.xx, GS.xy, GS.xz, GS.xy, GS.yy, GS.yz, GS.xz, GS.yz, GS.zz};
                float GR[9], gls[3];
    #pragma unroll
                for (int k = 0; k < 3; ++k) {
                    float acc = 0.f;
    #pragma unroll
                    for (int r = 0; r < 3; ++r) {
                        const float gm = 2.f * (Gs[r * 3 + 0] * M[0 * 3 + k] + Gs[r * 3 + 1] * M[1 * 3 + k] +
                                                Gs[r * 3 + 2] * M[2 * 3 + k]);
                        GR[r * 3 + k] = gm * s[k];
                        acc += gm * R[r * 3 + k];
                    }
                    gls[k] = acc * s[k];
                }
                float g4v[4];
                g4v[0] = GR[1] * (-2.f * z) + GR[2] * (2.f * y) + GR[3] * (2.f * z) + GR[5] * (-2.f * x) + GR[6] * (-2.f * y) + GR[7] * (2.f * x);
                g4v[1] = GR[1] * (2.f * y) + GR[2] * (2.f * z) + GR[3] * (2.f * y) + GR[4] * (-4.f * x) + GR[5] * (-2.f * w) + GR[6] * (2.f * z) + GR[7] * (2.f * w) + GR[8] * (-4.f * x);
                g4v[2] = GR[0] * (-4.f * y) + GR[1] * (2.f * x) + GR[2] * (2.f * w) + GR[3] * (2.f * x) + GR[5] * (2.f * z) + GR[6] * (-2.f * w) + GR[7] * (2.f * z) + GR[8] * (-4.f * y);
                g4v[3] = GR[0] * (-4.f * z) + GR[1] * (-2.f * w) + GR[2] * (2.f * x) + GR[3] * (2.f * w) + GR[4] * (-4.f * z) + GR[5] * (2.f * y) + GR[6] * (2.f * x) + GR[7] * (2.f * y);
                float gq[4];
                normalise_backward(q, g4v, gq);
                const float sg = sigmoidf_(o);
                float* dm = dg3.mean + j * 3;
                dm[0] = gmu_sum[0]; dm[1] = gmu_sum[1]; dm[2] = gmu_sum[2];
                float* dl = dg3.log_scale + j * 3;
                dl[0] = gls[0]; dl[1] = gls[1]; dl[2] = gls[2];
                ((float4*)dg3.quat)[j] = make_float4(gq[0], gq[1], gq[2], gq[3]);
                dg3.opacity[j] = gal * sg * (1.f - sg);
        }
        }
        __syncwarp();  // sums and geometry are rewritten by the next chunk
    }
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------

cudaError_t launch_slice_project(const splat_g3& g3, const splat_g4& g4, const ViewBatch& vb, const splat_proj& out,
                                 int32_t* status, int dtype, const LaunchCtx& ctx)
{
    const int64_t N = out.n;
    if (N == 0) return cudaSuccess;
    const int threads = 128;
    const int64_t want = (N + threads - 1) / threads;
    const int blocks = (int)(want < (int64_t)ctx.num_sms * 64 ? want : (int64_t)ctx.num_sms * 64);
    count_launch();
    switch (dtype) {
    case SPLAT_F32: k_slice_project<SPLAT_F32><<<blocks, threads, 0, ctx.stream>>>(g3, g4, vb, out, status); break;
    case SPLAT_BF16: k_slice_project<SPLAT_BF16><<<blocks, threads, 0, ctx.stream>>>(g3, g4, vb, out, status); break;
    default: k_slice_project<SPLAT_F16><<<blocks, threads, 0, ctx.stream>>>(g3, g4, vb, out, status); break;
    }
    return cudaGetLastError();
}

template <int DT, int L>
static void adjoint_launch(int blocks, cudaStream_t st, const splat_g3& g3, const splat_g4& g4, const ViewBatch& vb,
                           const splat_proj& proj, const float* dproj, const splat_grads3& dg3,
                           const splat_grads4& dg4, int32_t* status)
{
    k_adjoint<DT, L><<<blocks, kAdjThreads, 0, st>>>(g3, g4, vb, proj, dproj, dg3, dg4, status);
}

template <int DT>
static void adjoint_lanes(int V, int64_t N, int num_sms, cudaStream_t st, const splat_g3& g3, const splat_g4& g4,
                          const ViewBatch& vb, const splat_proj& proj, const float* dproj, const splat_grads3& dg3,
                          const splat_grads4& dg4, int32_t* status)
{
    // lanes per Gaussian: the view count rounded up to a power of two
    const int L = V <= 1 ? 1 : V <= 2 ? 2 : V <= 4 ? 4 : V <= 8 ? 8 : 16;
    const int64_t want = (N + kAdjThreads - 1) / kAdjThreads;
    const int blocks = (int)(want < (int64_t)num_sms * 64 ? want : (int64_t)num_sms * 64);
    switch (L) {
    case 1: adjoint_launch<DT, 1>(blocks, st, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    case 2: adjoint_launch<DT, 2>(blocks, st, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    case 4: adjoint_launch<DT, 4>(blocks, st, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    case 8: adjoint_launch<DT, 8>(blocks, st, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    default: adjoint_launch<DT, 16>(blocks, st, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    }
}

cudaError_t launch_adjoint(const splat_g3& g3, const splat_g4& g4, const ViewBatch& vb, const splat_proj& proj,
                           const float* dproj, const splat_grads3& dg3, const splat_grads4& dg4, int32_t* status,
                           int dtype, const LaunchCtx& ctx)
{
    const int64_t N = proj.n;
    if (N == 0) return cudaSuccess;
    count_launch();
    switch (dtype) {
    case SPLAT_F32: adjoint_lanes<SPLAT_F32>(vb.V, N, ctx.num_sms, ctx.stream, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    case SPLAT_BF16: adjoint_lanes<SPLAT_BF16>(vb.V, N, ctx.num_sms, ctx.stream, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    default: adjoint_lanes<SPLAT_F16>(vb.V, N, ctx.num_sms, ctx.stream, g3, g4, vb, proj, dproj, dg3, dg4, status); break;
    }
    return cudaGetLastError();
}

}  // namespace splat
