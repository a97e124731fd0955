/*
 * oracle.c -- plain FP64 CPU oracle for the hybrid 3D-4D Gaussian rasterizer.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file:
 * only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load it.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * What it computes (paper: "Hybrid 3D-4D Gaussian Splatting for Fast Dynamic
 * Scene Representation"):
 *   - 3D covariance from quaternion and log-scale                (Eq. 2)
 *   - 4D rotation R = R_l R_r from two quaternions               (Eq. 4)
 *   - temporal slicing of a 4D Gaussian at time t, conditional
 *     mean and Schur-complement covariance, written literally     (Eq. 5, Eq. 6)
 *   - temporal opacity factor p(t) (inherited from 4DGS, Sec. 3.2 defers
 *     to it; reading D1: unnormalised marginal exp(-(t-mu_t)^2 / 2 S_tt))
 *   - cull, EWA projection, degree-3 SH colour, tile rectangle    (Alg. 1, lines "CullGaussian",
 *     "ProjGaussian4D", "ProjGaussian3D"; 3DGS conventions, readings D5, D8)
 *   - the rendered pixel as the PLAIN DEFINITION of alpha compositing (Eq. 3):
 *     every visible Gaussian whose tile rectangle holds the pixel's tile,
 *     ordered by (depth rounded to FP32, merged index), blended front to back
 *     (Alg. 1 "CreateTiles" .. "BlendInOrder", readings D4, D6, D7)
 *   - the reverse-mode gradient of all of the above, hand written
 *   - the 4D -> 3D conversion of Sec. 4.1-4.2 with the quaternion of Eq. 9
 *   - a stable sort of 64-bit keys (Alg. 1 "SortByKeys")
 *
 * Merged index convention (Alg. 1 fills M' with the 4D Gaussians first and
 * appends the 3D ones): i in [0, N4) are 4D Gaussians, i in [N4, N4+N3) are 3D.
 *
 * Every floating-point decision (cull, radius ceil, tile-rectangle floor/ceil,
 * alpha skip, transmittance stop, clamps) also reports a relative "margin":
 * the distance of the decided quantity to its threshold.  Tests use these to
 * tell apart results that an FP32 implementation may legitimately decide the
 * other way.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Data types                                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    const double *mean;      /* [n][3] world position                        */
    const double *log_scale; /* [n][3] s, scale = exp(s)                     */
    const double *quat;      /* [n][4] (w,x,y,z), not normalised             */
    const double *opacity;   /* [n]    logit, opacity = sigmoid(o)           */
    const double *sh;        /* [n][16][3] SH coefficients, degree 3          */
} og3;

typedef struct {
    int64_t n;
    const double *mean;      /* [n][4] (x,y,z,t)                             */
    const double *log_scale; /* [n][4] (s_x,s_y,s_z,s_t)                     */
    const double *ql;        /* [n][4] left quaternion (a,b,c,d)             */
    const double *qr;        /* [n][4] right quaternion (p,q,r,s)            */
    const double *opacity;   /* [n]                                          */
    const double *sh;        /* [n][T+1][16][3]: coefficient block per time frequency */
    int64_t n_time;          /* T: time frequencies of the colour, 0 = plain SH      */
} og4;

typedef struct {
    double R[9];     /* world -> camera rotation, row major                  */
    double T[3];     /* world -> camera translation: x_c = R x_w + T         */
    double fx, fy, cx, cy;
    int32_t W, H;
    int32_t pad0, pad1;
    double time;     /* the timestamp t the 4D Gaussians are sliced at       */
    double z_near;
    double bg[3];
} oview;

typedef struct {
    double px, py, depth;
    double conic[3];     /* (a, b, c) of the inverse 2D covariance            */
    double alpha;        /* alpha_max: sigmoid(o) (times p(t) for 4D)        */
    double rgb[3];
    double margin_fwd;   /* min relative margin of cull/radius/rect decisions */
    double margin_grad;  /* min relative margin of clamp decisions           */
    int32_t radius;      /* 0 when culled                                    */
    int32_t rect[4];     /* tile rectangle x0,y0,x1,y1, half open            */
    int32_t visible;     /* not culled and the rectangle is not empty        */
    int32_t n_tiles;
    int32_t pad;
    double r3;           /* 3 sqrt(lambda_max) before the ceil               */
    double margin_cull;  /* min relative margin of the near-plane and alpha cull */
} oproj;

/* reading D5: thresholds inherited from the 3DGS rasterizer */
#define TILE 16
#define ALPHA_MIN (1.0 / 255.0)
#define ALPHA_MAX_CLAMP 0.99
#define T_MIN 1e-4
#define DILATION 0.3
#define FOV_CLAMP 1.3

static double sigmoid(double x) { return 1.0 / (1.0 + exp(-x)); }

/* distance of q to the nearest integer, relative to max(1,|q|) */
static double int_margin(double q)
{
    double d = fabs(q - nearbyint(q));
    double s = fabs(q) > 1.0 ? fabs(q) : 1.0;
    return d / s;
}

static double dmin(double a, double b) { return a < b ? a : b; }

/* ------------------------------------------------------------------------ */
/* Small dense linear algebra, row major                                     */
/* ------------------------------------------------------------------------ */

static void matmul(const double *A, const double *B, double *C, int n, int k, int m)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) {
            double s = 0.0;
            for (int l = 0; l < k; ++l) s += A[i * k + l] * B[l * m + j];
            C[i * m + j] = s;
        }
}

static void transpose(const double *A, double *At, int n, int m)
{
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < m; ++j) At[j * n + i] = A[i * m + j];
}

/* ------------------------------------------------------------------------ */
/* Rotations                                                                 */
/* ------------------------------------------------------------------------ */

/* Unit quaternion (w,x,y,z) -> 3x3 rotation (Hamilton convention, v -> q v q*).
 * This is the matrix that Eq. 9 inverts.  Input need not be normalised. */
void oracle_quat_to_R3(const double q_in[4], double R[9])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

/* Eq. 4: left isoclinic matrix of (a,b,c,d). */
static void left_matrix(const double q[4], double L[16])
{
    double a = q[0], b = q[1], c = q[2], d = q[3];
    double M[16] = { a, -b, -c, -d,
                     b,  a, -d,  c,
                     c,  d,  a, -b,
                     d, -c,  b,  a };
    memcpy(L, M, sizeof M);
}

/* Eq. 4: right isoclinic matrix of (p,q,r,s). */
static void right_matrix(const double q[4], double Rr[16])
{
    double p = q[0], qq = q[1], r = q[2], s = q[3];
    double M[16] = { p, -qq, -r, -s,
                     qq,  p,  s, -r,
                     r,  -s,  p, qq,
                     s,   r, -qq, p };
    memcpy(Rr, M, sizeof M);
}

static void normalise4(const double q[4], double out[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    for (int i = 0; i < 4; ++i) out[i] = q[i] / n;
}

/* Eq. 4: R = R_l R_r from normalised (a,b,c,d) and (p,q,r,s) (reading D3). */
void oracle_rot4(const double ql[4], const double qr[4], double R[16])
{
    double a[4], b[4], L[16], Rr[16];
    normalise4(ql, a);
    normalise4(qr, b);
    left_matrix(a, L);
    right_matrix(b, Rr);
    matmul(L, Rr, R, 4, 4, 4);
}

/* Eq. 2: Sigma = R S S^T R^T with S = diag(exp(s)). */
void oracle_cov3(const double quat[4], const double log_scale[3], double S[9])
{
    double R[9], M[9], Mt[9];
    oracle_quat_to_R3(quat, R);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[i * 3 + k] = R[i * 3 + k] * exp(log_scale[k]);
    transpose(M, Mt, 3, 3);
    matmul(M, Mt, S, 3, 3, 3);
}

/* 4D covariance Sigma_4D = R S S^T R^T, R from Eq. 4, S = diag(exp(s)) (reading D2). */
void oracle_cov4(const double ql[4], const double qr[4], const double log_scale[4], double S[16])
{
    double R[16], M[16], Mt[16];
    oracle_rot4(ql, qr, R);
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) M[i * 4 + k] = R[i * 4 + k] * exp(log_scale[k]);
    transpose(M, Mt, 4, 4);
    matmul(M, Mt, S, 4, 4, 4);
}

/* Eq. 5 and Eq. 6 exactly as written, plus the temporal factor of reading D1.
 * Sigma4 is the full 4x4 covariance, coordinates (x,y,z,t). */
void oracle_slice(const double mean4[4], const double Sigma4[16], double t,
                  double mu3[3], double cov3[9], double *p_t)
{
    double s44 = Sigma4[15];
    double s14[3] = { Sigma4[3], Sigma4[7], Sigma4[11] };
    double dt = t - mean4[3];
    for (int i = 0; i < 3; ++i) mu3[i] = mean4[i] + s14[i] / s44 * dt;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) cov3[i * 3 + j] = Sigma4[i * 4 + j] - s14[i] * s14[j] / s44;
    *p_t = exp(-0.5 * dt * dt / s44);
}

/* ------------------------------------------------------------------------ */
/* Real spherical harmonics, degree <= 3 (reading D8)                        */
/* ------------------------------------------------------------------------ */
/*
 * Y_l^m with the Condon-Shortley phase, ordered k = l*l + l + m, m = -l..l.
 * Built from the closed forms, not from a constant table:
 *   K_l^m = sqrt((2l+1)/(4 pi) * (l-|m|)! / (l+|m|)!)
 *   P_l^m(z) = (-1)^m (1-z^2)^(m/2) d^m/dz^m P_l(z)
 *   (1-z^2)^(m/2) cos(m phi) = Re (x+iy)^m,  ... sin(m phi) = Im (x+iy)^m
 * so on the unit sphere
 *   Y_l^0  = K_l^0 P_l(z)
 *   Y_l^m  = sqrt2 K_l^m (-1)^m P_l^(m)(z) Re(x+iy)^m      (m > 0)
 *   Y_l^-m = sqrt2 K_l^m (-1)^m P_l^(m)(z) Im(x+iy)^m      (m > 0)
 * which is a polynomial in (x,y,z), so its gradient is available exactly.
 * The Legendre polynomial coefficients come from Bonnet's recurrence.
 */

static double factorial(int n)
{
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= i;
    return f;
}

/* coefficients of P_l(z), c[j] multiplies z^j, l <= 4 */
static void legendre_coeffs(int l, double c[8])
{
    double p0[8] = { 1 }, p1[8] = { 0, 1 }, pn[8];
    if (l == 0) { memcpy(c, p0, sizeof p0); return; }
    for (int n = 1; n < l; ++n) {
        /* (n+1) P_{n+1} = (2n+1) z P_n - n P_{n-1} */
        memset(pn, 0, sizeof pn);
        for (int j = 0; j < 7; ++j) pn[j + 1] += (2 * n + 1) * p1[j];
        for (int j = 0; j < 8; ++j) pn[j] -= n * p0[j];
        for (int j = 0; j < 8; ++j) pn[j] /= (n + 1);
        memcpy(p0, p1, sizeof p1);
        memcpy(p1, pn, sizeof pn);
    }
    memcpy(c, p1, sizeof p1);
}

/* d^m/dz^m of the polynomial c, evaluated at z */
static double poly_deriv_eval(const double c[8], int m, double z)
{
    double s = 0.0, zp = 1.0;
    for (int j = m; j < 8; ++j) {
        double coef = c[j];
        for (int k = 0; k < m; ++k) coef *= (j - k);
        s += coef * zp;
        zp *= z;
    }
    return s;
}

/* Re and Im of (x+iy)^m */
static void cpow(double x, double y, int m, double *re, double *im)
{
    double a = 1.0, b = 0.0;
    for (int k = 0; k < m; ++k) {
        double na = a * x - b * y, nb = a * y + b * x;
        a = na;
        b = nb;
    }
    *re = a;
    *im = b;
}

/* Y[16] at dir; if dY != NULL, also dY[16][3] = d Y / d(x,y,z) of the polynomial extension */
void oracle_sh_basis(const double dir[3], double Y[16], double *dY)
{
    double x = dir[0], y = dir[1], z = dir[2];
    for (int l = 0; l <= 3; ++l) {
        double c[8];
        legendre_coeffs(l, c);
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            int k = l * l + l + m;
            double K = sqrt((2 * l + 1) / (4 * M_PI) * factorial(l - am) / factorial(l + am));
            double D = poly_deriv_eval(c, am, z);
            double Dz = poly_deriv_eval(c, am + 1, z);
            if (m == 0) {
                Y[k] = K * D;
                if (dY) { dY[k * 3 + 0] = 0; dY[k * 3 + 1] = 0; dY[k * 3 + 2] = K * Dz; }
                continue;
            }
            double N = sqrt(2.0) * K * ((am & 1) ? -1.0 : 1.0);
            double re, im, re1, im1;
            cpow(x, y, am, &re, &im);
            cpow(x, y, am - 1, &re1, &im1);
            /* d/dx (x+iy)^m = m (x+iy)^(m-1); d/dy = i m (x+iy)^(m-1) */
            double A, Ax, Ay;
            if (m > 0) { A = re; Ax = am * re1; Ay = -am * im1; }
            else       { A = im; Ax = am * im1; Ay = am * re1; }
            Y[k] = N * D * A;
            if (dY) {
                dY[k * 3 + 0] = N * D * Ax;
                dY[k * 3 + 1] = N * D * Ay;
                dY[k * 3 + 2] = N * Dz * A;
            }
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Per-Gaussian forward: cull, EWA projection, SH colour, tile rectangle      */
/* ------------------------------------------------------------------------ */

static int grid_tiles(int n) { return (n + TILE - 1) / TILE; }

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* floor / ceil to int, saturating far outside the image */
static int ifloor(double q) { return (int)floor(fmax(-1e9, fmin(1e9, q))); }
static int iceil(double q) { return (int)ceil(fmax(-1e9, fmin(1e9, q))); }

/* The 4D colour model with T > 0 time frequencies (4D spherindrical harmonics
 * of 4DGS, which Sec. 3.2 defers to; reading N3): colour(d, t) = max(0, 0.5 +
 * sum_n cos(2 pi n t) sum_k c_nk Y_k(d)), t in units of the sequence length.
 * These are the effective degree-3 coefficients at t: sum_n cos(2 pi n t) c_n. */
static void sh_at_time(const og4 *g4, int64_t i, double t, double out[48])
{
    const int64_t T = g4->n_time;
    const double *c = g4->sh + 48 * (T + 1) * i;
    for (int k = 0; k < 48; ++k) out[k] = 0.0;
    for (int64_t n = 0; n <= T; ++n) {
        const double w = cos(2.0 * M_PI * (double)n * t);
        for (int k = 0; k < 48; ++k) out[k] += w * c[48 * n + k];
    }
}

/* world mean/covariance of merged Gaussian i at the view's time (Eq. 2 or Eq. 5/6);
 * sh points into the scene or, for a time-dependent 4D colour, to sh_buf */
static void gaussian_world(const og3 *g3, const og4 *g4, int64_t i, double t,
                           double mu[3], double cov[9], double *alpha_max, const double **sh, double sh_buf[48])
{
    int64_t n4 = g4 ? g4->n : 0;
    if (i < n4) {
        double S4[16], p;
        oracle_cov4(g4->ql + 4 * i, g4->qr + 4 * i, g4->log_scale + 4 * i, S4);
        oracle_slice(g4->mean + 4 * i, S4, t, mu, cov, &p);
        *alpha_max = sigmoid(g4->opacity[i]) * p;
        if (g4->n_time > 0) {
            sh_at_time(g4, i, t, sh_buf);
            *sh = sh_buf;
        } else {
            *sh = g4->sh + 48 * i;
        }
    } else {
        int64_t j = i - n4;
        oracle_cov3(g3->quat + 4 * j, g3->log_scale + 3 * j, cov);
        for (int k = 0; k < 3; ++k) mu[k] = g3->mean[3 * j + k];
        *alpha_max = sigmoid(g3->opacity[j]);
        *sh = g3->sh + 48 * j;
    }
}

static void camera_centre(const oview *v, double c[3])
{
    /* x_c = R x_w + T = 0  =>  x_w = -R^T T */
    for (int k = 0; k < 3; ++k)
        c[k] = -(v->R[0 * 3 + k] * v->T[0] + v->R[1 * 3 + k] * v->T[1] + v->R[2 * 3 + k] * v->T[2]);
}

static void project_one(const double mu[3], const double cov[9], double alpha_max, const double *sh,
                        const oview *v, oproj *o)
{
    memset(o, 0, sizeof *o);
    int TX = grid_tiles(v->W), TY = grid_tiles(v->H);
    double xc[3];
    for (int r = 0; r < 3; ++r)
        xc[r] = v->R[r * 3 + 0] * mu[0] + v->R[r * 3 + 1] * mu[1] + v->R[r * 3 + 2] * mu[2] + v->T[r];
    double z = xc[2];
    o->depth = z;
    double m_fwd = INFINITY, m_grad = INFINITY;
    o->margin_cull = dmin(fabs(z - v->z_near) / v->z_near, fabs(alpha_max - ALPHA_MIN) / ALPHA_MIN);
    m_fwd = dmin(m_fwd, o->margin_cull);
    o->alpha = alpha_max;
    int culled = (z <= v->z_near) || (alpha_max < ALPHA_MIN);
    if (z <= 0.0) {  /* no projection exists behind the camera */
        o->margin_fwd = m_fwd;
        o->margin_grad = m_grad;
        return;
    }
    /* EWA (reading D5): Jacobian of the perspective map at the clamped mean */
    double limx = FOV_CLAMP * (0.5 * v->W / v->fx), limy = FOV_CLAMP * (0.5 * v->H / v->fy);
    double ux = xc[0] / z, uy = xc[1] / z;
    m_grad = dmin(m_grad, fabs(fabs(ux) - limx) / limx);
    m_grad = dmin(m_grad, fabs(fabs(uy) - limy) / limy);
    double tx = z * fmin(limx, fmax(-limx, ux)), ty = z * fmin(limy, fmax(-limy, uy));
    double J[6] = { v->fx / z, 0.0, -v->fx * tx / (z * z),
                    0.0, v->fy / z, -v->fy * ty / (z * z) };
    double Tm[6], TS[6], Tt[6], S2[4];
    matmul(J, v->R, Tm, 2, 3, 3);
    matmul(Tm, cov, TS, 2, 3, 3);
    transpose(Tm, Tt, 2, 3);
    matmul(TS, Tt, S2, 2, 3, 2);
    S2[0] += DILATION;
    S2[3] += DILATION;
    double det = S2[0] * S2[3] - S2[1] * S2[2];
    if (det <= 0.0) culled = 1;
    double a = S2[3] / det, b = -S2[1] / det, c = S2[0] / det;
    o->conic[0] = a; o->conic[1] = b; o->conic[2] = c;
    double mid = 0.5 * (S2[0] + S2[3]);
    double lam = mid + sqrt(fmax(0.1, mid * mid - det));
    double r3 = 3.0 * sqrt(lam);
    o->r3 = r3;
    m_fwd = dmin(m_fwd, int_margin(r3));
    int radius = (int)ceil(r3);
    double px = v->fx * xc[0] / z + v->cx, py = v->fy * xc[1] / z + v->cy;
    o->px = px;
    o->py = py;
    double qx0 = (px - radius) / TILE, qx1 = (px + radius) / TILE;
    double qy0 = (py - radius) / TILE, qy1 = (py + radius) / TILE;
    int x0 = clampi(ifloor(qx0), 0, TX), x1 = clampi(iceil(qx1), 0, TX);
    int y0 = clampi(ifloor(qy0), 0, TY), y1 = clampi(iceil(qy1), 0, TY);
    double m_rect = dmin(dmin(int_margin(qx0), int_margin(qx1)), dmin(int_margin(qy0), int_margin(qy1)));
    m_fwd = dmin(m_fwd, m_rect);
    /* colour: degree-3 SH at the viewing direction (reading D8) */
    double cc[3], d[3], Y[16];
    camera_centre(v, cc);
    double nrm = 0.0;
    for (int k = 0; k < 3; ++k) { d[k] = mu[k] - cc[k]; nrm += d[k] * d[k]; }
    nrm = sqrt(nrm);
    for (int k = 0; k < 3; ++k) d[k] /= nrm;
    oracle_sh_basis(d, Y, NULL);
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5, mag = 0.5;
        for (int k = 0; k < 16; ++k) { s += sh[k * 3 + ch] * Y[k]; mag += fabs(sh[k * 3 + ch] * Y[k]); }
        m_grad = dmin(m_grad, fabs(s) / mag);
        o->rgb[ch] = s > 0.0 ? s : 0.0;
    }
    int n_tiles = (x1 - x0) * (y1 - y0);
    if (!culled && n_tiles > 0) {
        o->visible = 1;
        o->radius = radius;
        o->rect[0] = x0; o->rect[1] = y0; o->rect[2] = x1; o->rect[3] = y1;
        o->n_tiles = n_tiles;
    }
    o->margin_fwd = m_fwd;
    o->margin_grad = m_grad;
}

/* Project every merged Gaussian for one view.  out has n4 + n3 entries. */
void oracle_project(const og3 *g3, const og4 *g4, const oview *v, oproj *out)
{
    int64_t n4 = g4 ? g4->n : 0, n3 = g3 ? g3->n : 0;
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t i = 0; i < n4 + n3; ++i) {
        double mu[3], cov[9], am;
        const double *sh;
        double sh_buf[48];
        gaussian_world(g3, g4, i, v->time, mu, cov, &am, &sh, sh_buf);
        project_one(mu, cov, am, sh, v, &out[i]);
    }
}

/* ------------------------------------------------------------------------ */
/* Per-pixel compositing: the plain definition of Eq. 3                      */
/* ------------------------------------------------------------------------ */

/* Sort key of one Gaussian in a tile list (reading D6): the depth as an FP32
 * number, the precision of the key that Alg. 1's SortByKeys orders (tile id in
 * the high bits, the depth's float bits in the low 32), then the merged index. */
typedef struct { float key; int64_t idx; } dkey;

static int cmp_dkey(const void *pa, const void *pb)
{
    const dkey *a = pa, *b = pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* relative distance of d > 0 to the nearest rounding boundary (midpoint between
 * two neighbouring FP32 numbers): how far d is from rounding differently */
static double fp32_midpoint_margin(double d)
{
    float f = (float)d;
    double lo = 0.5 * ((double)f + (double)nextafterf(f, 0.0f));
    double hi = 0.5 * ((double)f + (double)nextafterf(f, INFINITY));
    return fmin(fabs(d - lo), fabs(hi - d)) / d;
}

/* the pixel's ordered list: visible Gaussians whose rectangle holds tile (tx,ty) */
static int64_t pixel_list(const oproj *P, int64_t n, int tx, int ty, dkey *buf)
{
    int64_t m = 0;
    for (int64_t i = 0; i < n; ++i) {
        const oproj *o = &P[i];
        if (!o->visible) continue;
        if (tx < o->rect[0] || tx >= o->rect[2] || ty < o->rect[1] || ty >= o->rect[3]) continue;
        buf[m].key = (float)o->depth;
        buf[m].idx = i;
        ++m;
    }
    qsort(buf, (size_t)m, sizeof(dkey), cmp_dkey);
    return m;
}

/* one entry of the front-to-back walk, kept for the reverse pass */
typedef struct {
    int64_t idx;
    double G, alpha, T_before, dx, dy;
    int clamped;
} tape_ent;

/* Walks the list front to back for pixel (u,v); returns the number of tape
 * entries (contributing Gaussians).  Reading D5 for the skip / stop rules. */
/* margins of one pixel, each the min over its walk of |quantity - threshold| / scale */
enum { MG_POWER = 0, MG_ALPHA = 1, MG_STOP = 2, MG_TIE = 3, MG_CLAMP = 4, MG_TIE3 = 5, MG_COUNT = 6 };

/* A forward decision's margin is recorded only when flipping it could change
 * the pixel by at least this much (0: record every decision).  Bounds used:
 * alpha skip 2 T c_max / 255; power sign 2 T alpha_max c_max; order of two
 * touching Gaussians T alpha_1 alpha_2 |c_1 - c_2|; the stop is always kept. */
static double g_margin_impact = 0.0;
static double g_cmax = 1.0;  /* largest colour channel of the current render */

void oracle_set_margin_impact(double impact) { g_margin_impact = impact > 0.0 ? impact : 0.0; }

static int64_t blend_pixel(const oproj *P, int64_t n4, const dkey *list, int64_t m, int u, int vpix,
                           const double bg[3], double rgb[3], double *T_out, int32_t *last_out,
                           double mg_out[MG_COUNT], tape_ent *tape)
{
    double T = 1.0, C[3] = { 0, 0, 0 };
    double mgn[MG_COUNT] = { INFINITY, INFINITY, INFINITY, INFINITY, INFINITY, INFINITY };
    int32_t last = (int32_t)m;  /* end of the walk: the list length unless T saturates */
    int64_t nt = 0;
    double prev_depth = -1.0;  /* depth, T, alpha, colour of the previous Gaussian that touched the pixel */
    int prev_3d = 0;
    double prev_T = 0.0, prev_alpha = 0.0;
    const double *prev_rgb = NULL;
    const double imp = g_margin_impact;
    for (int64_t j = 0; j < m; ++j) {
        const oproj *o = &P[list[j].idx];
        double dx = o->px - u, dy = o->py - vpix;
        double a = o->conic[0], b = o->conic[1], c = o->conic[2];
        double power = -0.5 * (a * dx * dx + c * dy * dy) - b * dx * dy;
        double pmag = 0.5 * fabs(a) * dx * dx + 0.5 * fabs(c) * dy * dy + fabs(b * dx * dy);
        if (pmag > 0.0 && 2.0 * T * o->alpha * g_cmax >= imp)
            mgn[MG_POWER] = dmin(mgn[MG_POWER], fabs(power) / pmag);
        if (power > 0.0) continue;
        double G = exp(power);
        double raw = o->alpha * G;
        if (2.0 * T * g_cmax * ALPHA_MIN >= imp)
            mgn[MG_ALPHA] = dmin(mgn[MG_ALPHA], fabs(raw - ALPHA_MIN) / ALPHA_MIN);
        mgn[MG_CLAMP] = dmin(mgn[MG_CLAMP], fabs(raw - ALPHA_MAX_CLAMP) / ALPHA_MAX_CLAMP);
        if (raw >= ALPHA_MIN) {
            /* two touching Gaussians at nearly equal depth: their order is a decision too.
             * Keys are FP32 depths.  A 3D Gaussian's depth is a dot product of FP32
             * inputs, which a compensated evaluation rounds exactly; two of them swap
             * only if one depth sits at an FP32 rounding boundary while their keys are
             * at most one step apart (MG_TIE3).  A sliced 4D Gaussian's depth carries
             * the FP32 rounding of the slice: any FP64 gap below a few FP32 steps is a
             * decision (MG_TIE); an exact FP64 tie comes only from equal inputs and is
             * resolved by the merged index on both sides. */
            double a_cur = raw < ALPHA_MAX_CLAMP ? raw : ALPHA_MAX_CLAMP;
            const int cur_3d = list[j].idx >= n4;
            if (prev_depth > 0.0) {
                double dc = 0.0;
                for (int ch = 0; ch < 3; ++ch) dc = fmax(dc, fabs(o->rgb[ch] - prev_rgb[ch]));
                if (prev_T * prev_alpha * a_cur * dc >= imp) {
                    if (cur_3d && prev_3d) {
                        float kp = (float)prev_depth, kc = (float)o->depth;
                        if (kc <= nextafterf(kp, INFINITY))
                            mgn[MG_TIE3] = dmin(mgn[MG_TIE3], fmin(fp32_midpoint_margin(prev_depth),
                                                                   fp32_midpoint_margin(o->depth)));
                    } else if (o->depth != prev_depth) {
                        mgn[MG_TIE] = dmin(mgn[MG_TIE], fabs(o->depth - prev_depth) / o->depth);
                    }
                }
            }
            prev_3d = cur_3d;
            prev_depth = o->depth;
            prev_T = T;
            prev_alpha = a_cur;
            prev_rgb = o->rgb;
        }
        double alpha = raw < ALPHA_MAX_CLAMP ? raw : ALPHA_MAX_CLAMP;
        if (alpha < ALPHA_MIN) continue;
        double test_T = T * (1.0 - alpha);
        mgn[MG_STOP] = dmin(mgn[MG_STOP], fabs(test_T - T_MIN) / T_MIN);
        if (test_T < T_MIN) {  /* this Gaussian does not contribute; the walk ends here */
            last = (int32_t)j;
            break;
        }
        if (tape) {
            tape[nt].idx = list[j].idx;
            tape[nt].G = G;
            tape[nt].alpha = alpha;
            tape[nt].T_before = T;
            tape[nt].dx = dx;
            tape[nt].dy = dy;
            tape[nt].clamped = raw >= ALPHA_MAX_CLAMP;
        }
        ++nt;
        for (int ch = 0; ch < 3; ++ch) C[ch] += o->rgb[ch] * alpha * T;
        T = test_T;
    }
    for (int ch = 0; ch < 3; ++ch) rgb[ch] = C[ch] + T * bg[ch];
    *T_out = T;
    *last_out = last;
    if (mg_out)
        for (int k = 0; k < MG_COUNT; ++k) mg_out[k] = mgn[k];
    return nt;
}

/* Render the given pixels (flat indices v*W+u; NULL = the whole image).
 * rgb is [3][npix] planar, T and last are [npix]; margins (may be NULL) is
 * [6][npix]: power sign, alpha skip, transmittance stop, depth order of two
 * touching Gaussians (one of them 4D), alpha clamp (only matters to gradients),
 * depth order of two touching 3D Gaussians (FP32 rounding boundary). */
void oracle_render(const og3 *g3, const og4 *g4, const oview *v, const int64_t *pix, int64_t npix,
                   double *rgb, double *T, int32_t *last, double *margins)
{
    int64_t n = (g4 ? g4->n : 0) + (g3 ? g3->n : 0);
    oproj *P = malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    oracle_project(g3, g4, v, P);
    if (!pix) npix = (int64_t)v->W * v->H;
    g_cmax = fmax(fmax(v->bg[0], v->bg[1]), v->bg[2]);
    for (int64_t i = 0; i < n; ++i)
        if (P[i].visible)
            for (int ch = 0; ch < 3; ++ch) g_cmax = fmax(g_cmax, P[i].rgb[ch]);
#pragma omp parallel
    {
        dkey *buf = malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < npix; ++q) {
            int64_t p = pix ? pix[q] : q;
            int u = (int)(p % v->W), vv = (int)(p / v->W);
            int64_t m = pixel_list(P, n, u / TILE, vv / TILE, buf);
            double c3[3], mg[MG_COUNT];
            blend_pixel(P, g4 ? g4->n : 0, buf, m, u, vv, v->bg, c3, &T[q], &last[q], mg, NULL);
            for (int ch = 0; ch < 3; ++ch) rgb[ch * npix + q] = c3[ch];
            if (margins)
                for (int k = 0; k < MG_COUNT; ++k) margins[k * npix + q] = mg[k];
        }
        free(buf);
    }
    free(P);
}

/* The per-tile ordered list of Gaussian ids the method's sort produces, i.e. the
 * pixel list of any pixel of that tile.  ids must hold n entries; returns length. */
int64_t oracle_tile_list(const og3 *g3, const og4 *g4, const oview *v, int tx, int ty, int64_t *ids)
{
    int64_t n = (g4 ? g4->n : 0) + (g3 ? g3->n : 0);
    oproj *P = malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    dkey *buf = malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
    oracle_project(g3, g4, v, P);
    int64_t m = pixel_list(P, n, tx, ty, buf);
    for (int64_t j = 0; j < m; ++j) ids[j] = buf[j].idx;
    free(buf);
    free(P);
    return m;
}

/* ------------------------------------------------------------------------ */
/* Reverse mode                                                              */
/* ------------------------------------------------------------------------ */
/*
 * d_proj layout per merged Gaussian (9 doubles):
 *   [0] dL/dpx  [1] dL/dpy  [2] dL/da  [3] dL/db  [4] dL/dc
 *   [5] dL/dalpha_max  [6..8] dL/drgb
 * with (a, b, c) the conic and power = -(a dx^2 + c dy^2)/2 - b dx dy,
 * dx = px - u, dy = py - v.
 */

/* Reverse of blend_pixel for one pixel, given dL/dC of the pixel. */
static void blend_pixel_bwd(const oproj *P, const tape_ent *tape, int64_t nt, double T_final,
                            const double bg[3], const double dLdC[3], double *dproj)
{
    /* suffix[j] = sum_{i>j} c_i alpha_i T_i + T_final bg   (per channel) */
    double suffix[3] = { T_final * bg[0], T_final * bg[1], T_final * bg[2] };
    for (int64_t j = nt - 1; j >= 0; --j) {
        const tape_ent *e = &tape[j];
        const oproj *o = &P[e->idx];
        double *g = dproj + 9 * e->idx;
        /* C = sum_i c_i alpha_i T_i + T_final bg, T_i = prod_{k<i} (1 - alpha_k) */
        double dL_dalpha = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            double dc = e->alpha * e->T_before * dLdC[ch];
#pragma omp atomic
            g[6 + ch] += dc;
            dL_dalpha += dLdC[ch] * (o->rgb[ch] * e->T_before - suffix[ch] / (1.0 - e->alpha));
        }
        for (int ch = 0; ch < 3; ++ch) suffix[ch] += o->rgb[ch] * e->alpha * e->T_before;
        if (e->clamped) continue;  /* alpha = 0.99: no dependence on the inputs */
        /* alpha = alpha_max * G, G = exp(power) */
        double dL_dam = dL_dalpha * e->G;
        double dL_dpower = dL_dalpha * o->alpha * e->G;
        double a = o->conic[0], b = o->conic[1], c = o->conic[2];
        double dx = e->dx, dy = e->dy;
        double dpx = dL_dpower * (-(a * dx + b * dy));
        double dpy = dL_dpower * (-(c * dy + b * dx));
        double da = dL_dpower * (-0.5 * dx * dx);
        double db = dL_dpower * (-dx * dy);
        double dcc = dL_dpower * (-0.5 * dy * dy);
#pragma omp atomic
        g[0] += dpx;
#pragma omp atomic
        g[1] += dpy;
#pragma omp atomic
        g[2] += da;
#pragma omp atomic
        g[3] += db;
#pragma omp atomic
        g[4] += dcc;
#pragma omp atomic
        g[5] += dL_dam;
    }
}

/* Reverse of project_one.  Returns dL/dmu (world), the symmetric dL/dSigma
 * (dL = sum_ij G_ij dSigma_ij for symmetric dSigma), dL/dalpha_max, dL/dsh. */
static void project_one_bwd(const double mu[3], const double cov[9], const double *sh, const oview *v,
                            const double *dp, double dmu[3], double dcov[9], double *dalpha, double dsh[48])
{
    double xc[3];
    for (int r = 0; r < 3; ++r)
        xc[r] = v->R[r * 3 + 0] * mu[0] + v->R[r * 3 + 1] * mu[1] + v->R[r * 3 + 2] * mu[2] + v->T[r];
    double z = xc[2];
    double limx = FOV_CLAMP * (0.5 * v->W / v->fx), limy = FOV_CLAMP * (0.5 * v->H / v->fy);
    double ux = xc[0] / z, uy = xc[1] / z;
    int clx = (ux < -limx) || (ux > limx), cly = (uy < -limy) || (uy > limy);
    double tx = z * fmin(limx, fmax(-limx, ux)), ty = z * fmin(limy, fmax(-limy, uy));
    double J[6] = { v->fx / z, 0.0, -v->fx * tx / (z * z),
                    0.0, v->fy / z, -v->fy * ty / (z * z) };
    double Tm[6], TS[6], Tt[6], S2[4];
    matmul(J, v->R, Tm, 2, 3, 3);
    matmul(Tm, cov, TS, 2, 3, 3);
    transpose(Tm, Tt, 2, 3);
    matmul(TS, Tt, S2, 2, 3, 2);
    S2[0] += DILATION;
    S2[3] += DILATION;
    double det = S2[0] * S2[3] - S2[1] * S2[2];
    double Q[4] = { S2[3] / det, -S2[1] / det, -S2[2] / det, S2[0] / det };

    /* conic -> Sigma2: G_Sigma2 = -Q G_Q Q with G_Q = [[da, db/2],[db/2, dc]] */
    double GQ[4] = { dp[2], 0.5 * dp[3], 0.5 * dp[3], dp[4] }, tmp[4], GS2[4];
    matmul(Q, GQ, tmp, 2, 2, 2);
    matmul(tmp, Q, GS2, 2, 2, 2);
    for (int k = 0; k < 4; ++k) GS2[k] = -GS2[k];
    /* Sigma2 = Tm cov Tm^T + 0.3 I */
    double GT[6], GSig[9], tmp23[6], tmp32[6];
    matmul(GS2, Tm, tmp23, 2, 2, 3);          /* G2 T      */
    matmul(Tt, tmp23, GSig, 3, 2, 3);         /* T^T G2 T  */
    matmul(tmp23, cov, GT, 2, 3, 3);          /* G2 T cov  */
    for (int k = 0; k < 6; ++k) GT[k] *= 2.0;
    (void)tmp32;
    memcpy(dcov, GSig, sizeof GSig);
    /* Tm = J R  =>  G_J = G_T R^T */
    double Rt[9], GJ[6];
    transpose(v->R, Rt, 3, 3);
    matmul(GT, Rt, GJ, 2, 3, 3);
    /* J entries as functions of the camera-space mean */
    double gxc[3] = { 0, 0, 0 };
    double fx = v->fx, fy = v->fy;
    gxc[2] += GJ[0] * (-fx / (z * z));
    gxc[2] += GJ[4] * (-fy / (z * z));
    if (!clx) {  /* J02 = -fx x / z^2 */
        gxc[0] += GJ[2] * (-fx / (z * z));
        gxc[2] += GJ[2] * (2.0 * fx * xc[0] / (z * z * z));
    } else {     /* J02 = -fx c / z, c = +-limx */
        double cst = ux > 0 ? limx : -limx;
        gxc[2] += GJ[2] * (fx * cst / (z * z));
    }
    if (!cly) {
        gxc[1] += GJ[5] * (-fy / (z * z));
        gxc[2] += GJ[5] * (2.0 * fy * xc[1] / (z * z * z));
    } else {
        double cst = uy > 0 ? limy : -limy;
        gxc[2] += GJ[5] * (fy * cst / (z * z));
    }
    /* px = fx x / z + cx, py = fy y / z + cy */
    gxc[0] += dp[0] * fx / z;
    gxc[2] += dp[0] * (-fx * xc[0] / (z * z));
    gxc[1] += dp[1] * fy / z;
    gxc[2] += dp[1] * (-fy * xc[1] / (z * z));
    /* xc = R mu + T */
    for (int k = 0; k < 3; ++k)
        dmu[k] = v->R[0 * 3 + k] * gxc[0] + v->R[1 * 3 + k] * gxc[1] + v->R[2 * 3 + k] * gxc[2];
    *dalpha = dp[5];
    /* SH colour */
    double cc[3], d[3], Y[16], dY[48];
    camera_centre(v, cc);
    double nrm = 0.0;
    for (int k = 0; k < 3; ++k) { d[k] = mu[k] - cc[k]; nrm += d[k] * d[k]; }
    nrm = sqrt(nrm);
    for (int k = 0; k < 3; ++k) d[k] /= nrm;
    oracle_sh_basis(d, Y, dY);
    double gdir[3] = { 0, 0, 0 };
    for (int ch = 0; ch < 3; ++ch) {
        double s = 0.5;
        for (int k = 0; k < 16; ++k) s += sh[k * 3 + ch] * Y[k];
        double g = s > 0.0 ? dp[6 + ch] : 0.0;
        for (int k = 0; k < 16; ++k) {
            dsh[k * 3 + ch] = g * Y[k];
            for (int e = 0; e < 3; ++e) gdir[e] += g * sh[k * 3 + ch] * dY[k * 3 + e];
        }
    }
    /* d = (mu - cc)/|mu - cc|: dL/dmu += (I - d d^T) gdir / |mu - cc| */
    double dd = d[0] * gdir[0] + d[1] * gdir[1] + d[2] * gdir[2];
    for (int k = 0; k < 3; ++k) dmu[k] += (gdir[k] - d[k] * dd) / nrm;
}

/* reverse of normalisation q / |q| */
static void normalise_bwd(const double q[4], const double gqn[4], double gq[4])
{
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    double qn[4] = { q[0] / n, q[1] / n, q[2] / n, q[3] / n };
    double dot = qn[0] * gqn[0] + qn[1] * gqn[1] + qn[2] * gqn[2] + qn[3] * gqn[3];
    for (int k = 0; k < 4; ++k) gq[k] = (gqn[k] - qn[k] * dot) / n;
}

/* reverse of Eq. 2 */
static void cov3_bwd(const double quat[4], const double log_scale[3], const double G[9],
                     double gquat[4], double glog[3])
{
    double R[9], M[9], s[3];
    oracle_quat_to_R3(quat, R);
    for (int k = 0; k < 3; ++k) s[k] = exp(log_scale[k]);
    for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) M[i * 3 + k] = R[i * 3 + k] * s[k];
    double GM[9];
    matmul(G, M, GM, 3, 3, 3);
    for (int k = 0; k < 9; ++k) GM[k] *= 2.0;  /* Sigma = M M^T */
    double GR[9];
    for (int k = 0; k < 3; ++k) {
        double gs = 0.0;
        for (int i = 0; i < 3; ++i) { GR[i * 3 + k] = GM[i * 3 + k] * s[k]; gs += GM[i * 3 + k] * R[i * 3 + k]; }
        glog[k] = gs * s[k];
    }
    double n = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
    double w = quat[0] / n, x = quat[1] / n, y = quat[2] / n, z = quat[3] / n;
    /* partial derivatives of the 9 entries of oracle_quat_to_R3 */
    double gw = 0, gx = 0, gy = 0, gz = 0;
    gw += GR[1] * (-2 * z) + GR[2] * (2 * y) + GR[3] * (2 * z) + GR[5] * (-2 * x) + GR[6] * (-2 * y) + GR[7] * (2 * x);
    gx += GR[1] * (2 * y) + GR[2] * (2 * z) + GR[3] * (2 * y) + GR[4] * (-4 * x) + GR[5] * (-2 * w) + GR[6] * (2 * z) + GR[7] * (2 * w) + GR[8] * (-4 * x);
    gy += GR[0] * (-4 * y) + GR[1] * (2 * x) + GR[2] * (2 * w) + GR[3] * (2 * x) + GR[5] * (2 * z) + GR[6] * (-2 * w) + GR[7] * (2 * z) + GR[8] * (-4 * y);
    gz += GR[0] * (-4 * z) + GR[1] * (-2 * w) + GR[2] * (2 * x) + GR[3] * (2 * w) + GR[4] * (-4 * z) + GR[5] * (2 * y) + GR[6] * (2 * x) + GR[7] * (2 * y);
    double gqn[4] = { gw, gx, gy, gz };
    normalise_bwd(quat, gqn, gquat);
}

/* reverse of Eq. 5/6 + reading D1 + the 4D covariance of Eq. 4 */
static void slice_bwd(const double *mean4, const double *ql, const double *qr, const double *log_scale,
                      double t, const double gmu3[3], const double Gcov3[9], double g_p,
                      double gmean4[4], double gql[4], double gqr[4], double glog[4])
{
    double S4[16];
    oracle_cov4(ql, qr, log_scale, S4);
    double c = S4[15];
    double b[3] = { S4[3], S4[7], S4[11] };
    double dt = t - mean4[3];
    double p = exp(-0.5 * dt * dt / c);
    /* symmetric gradient of Sigma4 */
    double G4[16] = { 0 };
    double Gb_b[3];
    for (int i = 0; i < 3; ++i) {
        Gb_b[i] = 0.0;
        for (int j = 0; j < 3; ++j) Gb_b[i] += Gcov3[i * 3 + j] * b[j];
    }
    double bGb = b[0] * Gb_b[0] + b[1] * Gb_b[1] + b[2] * Gb_b[2];
    double gmu_b = gmu3[0] * b[0] + gmu3[1] * b[1] + gmu3[2] * b[2];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) G4[i * 4 + j] = Gcov3[i * 3 + j];
    for (int i = 0; i < 3; ++i) {
        /* Sigma3 = A - b b^T / c contributes -2 (G b)/c to d/db; mu3 = mu_x + b dt / c contributes gmu dt / c.
           b sits in two symmetric entries, each carrying half. */
        double gb = -2.0 * Gb_b[i] / c + gmu3[i] * dt / c;
        G4[i * 4 + 3] = 0.5 * gb;
        G4[3 * 4 + i] = 0.5 * gb;
    }
    G4[15] = bGb / (c * c) - gmu_b * dt / (c * c) + g_p * p * 0.5 * dt * dt / (c * c);
    for (int k = 0; k < 3; ++k) gmean4[k] = gmu3[k];
    gmean4[3] = -gmu_b / c + g_p * p * dt / c;
    /* Sigma4 = M M^T, M = R diag(exp(s)) */
    double R[16], M[16], s[4];
    oracle_rot4(ql, qr, R);
    for (int k = 0; k < 4; ++k) s[k] = exp(log_scale[k]);
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 4; ++k) M[i * 4 + k] = R[i * 4 + k] * s[k];
    double GM[16];
    matmul(G4, M, GM, 4, 4, 4);
    for (int k = 0; k < 16; ++k) GM[k] *= 2.0;
    double GR[16];
    for (int k = 0; k < 4; ++k) {
        double gs = 0.0;
        for (int i = 0; i < 4; ++i) { GR[i * 4 + k] = GM[i * 4 + k] * s[k]; gs += GM[i * 4 + k] * R[i * 4 + k]; }
        glog[k] = gs * s[k];
    }
    /* R = L Rr */
    double a[4], bq[4], L[16], Rr[16], Lt[16], Rrt[16], GL[16], GRr[16];
    normalise4(ql, a);
    normalise4(qr, bq);
    left_matrix(a, L);
    right_matrix(bq, Rr);
    transpose(L, Lt, 4, 4);
    transpose(Rr, Rrt, 4, 4);
    matmul(GR, Rrt, GL, 4, 4, 4);
    matmul(Lt, GR, GRr, 4, 4, 4);
    /* entries of the Eq. 4 matrices are +-1 times one quaternion component */
    double gan[4], gbn[4];
    gan[0] = GL[0] + GL[5] + GL[10] + GL[15];
    gan[1] = -GL[1] + GL[4] - GL[11] + GL[14];
    gan[2] = -GL[2] + GL[7] + GL[8] - GL[13];
    gan[3] = -GL[3] - GL[6] + GL[9] + GL[12];
    gbn[0] = GRr[0] + GRr[5] + GRr[10] + GRr[15];
    gbn[1] = -GRr[1] + GRr[4] + GRr[11] - GRr[14];
    gbn[2] = -GRr[2] - GRr[7] + GRr[8] + GRr[13];
    gbn[3] = -GRr[3] + GRr[6] - GRr[9] + GRr[12];
    normalise_bwd(ql, gan, gql);
    normalise_bwd(qr, gbn, gqr);
}

/*
 * Full reverse pass for one view.
 * dLdC: [3][H][W] planar.  Gradients are ADDED into the outputs (so views can
 * be summed by calling once per view); dproj_out ([n][9], may be NULL) is
 * overwritten with the 2D gradients of this view.
 * 3D outputs: dmean3[n3][3], dlog3[n3][3], dquat3[n3][4], dop3[n3], dsh3[n3][48]
 * 4D outputs: dmean4[n4][4], dlog4[n4][4], dql[n4][4], dqr[n4][4], dop4[n4], dsh4[n4][T+1][48]
 */
void oracle_render_bwd(const og3 *g3, const og4 *g4, const oview *v, const double *dLdC,
                       double *dmean3, double *dlog3, double *dquat3, double *dop3, double *dsh3,
                       double *dmean4, double *dlog4, double *dql, double *dqr, double *dop4, double *dsh4,
                       double *dproj_out)
{
    int64_t n4 = g4 ? g4->n : 0, n3 = g3 ? g3->n : 0, n = n4 + n3;
    int64_t npix = (int64_t)v->W * v->H;
    oproj *P = malloc(sizeof(oproj) * (size_t)(n > 0 ? n : 1));
    double *dproj = calloc((size_t)(n > 0 ? n : 1) * 9, sizeof(double));
    oracle_project(g3, g4, v, P);
#pragma omp parallel
    {
        dkey *buf = malloc(sizeof(dkey) * (size_t)(n > 0 ? n : 1));
        tape_ent *tape = malloc(sizeof(tape_ent) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t p = 0; p < npix; ++p) {
            double g[3] = { dLdC[p], dLdC[npix + p], dLdC[2 * npix + p] };
            if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0) continue;
            int u = (int)(p % v->W), vv = (int)(p / v->W);
            int64_t m = pixel_list(P, n, u / TILE, vv / TILE, buf);
            double c3[3], T;
            int32_t last;
            int64_t nt = blend_pixel(P, g4 ? g4->n : 0, buf, m, u, vv, v->bg, c3, &T, &last, NULL, tape);
            blend_pixel_bwd(P, tape, nt, T, v->bg, g, dproj);
        }
        free(tape);
        free(buf);
    }
    if (dproj_out) memcpy(dproj_out, dproj, sizeof(double) * 9 * (size_t)n);
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n; ++i) {
        if (!P[i].visible) continue;
        const double *dp = dproj + 9 * i;
        double mu[3], cov[9], am, dmu[3], dcov[9], dam, dsh[48], sh_buf[48];
        const double *sh;
        gaussian_world(g3, g4, i, v->time, mu, cov, &am, &sh, sh_buf);
        project_one_bwd(mu, cov, sh, v, dp, dmu, dcov, &dam, dsh);
        if (i < n4) {
            double S4[16], p_t, mu3[3], cov3[9];
            oracle_cov4(g4->ql + 4 * i, g4->qr + 4 * i, g4->log_scale + 4 * i, S4);
            oracle_slice(g4->mean + 4 * i, S4, v->time, mu3, cov3, &p_t);
            double sg = sigmoid(g4->opacity[i]);
            /* alpha_max = sigmoid(o) p(t) */
            double g_p = dam * sg;
            dop4[i] += dam * p_t * sg * (1.0 - sg);
            double gm4[4], gl[4], gr[4], gs[4];
            slice_bwd(g4->mean + 4 * i, g4->ql + 4 * i, g4->qr + 4 * i, g4->log_scale + 4 * i, v->time,
                      dmu, dcov, g_p, gm4, gl, gr, gs);
            for (int k = 0; k < 4; ++k) {
                dmean4[4 * i + k] += gm4[k];
                dql[4 * i + k] += gl[k];
                dqr[4 * i + k] += gr[k];
                dlog4[4 * i + k] += gs[k];
            }
            /* colour = sum_n cos(2 pi n t) (block n): block n gets cos(2 pi n t) dL/dsh_eff */
            const int64_t T = g4->n_time;
            for (int64_t n = 0; n <= T; ++n) {
                const double w = cos(2.0 * M_PI * (double)n * v->time);
                for (int k = 0; k < 48; ++k) dsh4[48 * ((T + 1) * i + n) + k] += w * dsh[k];
            }
        } else {
            int64_t j = i - n4;
            double sg = sigmoid(g3->opacity[j]);
            dop3[j] += dam * sg * (1.0 - sg);
            double gq[4], gs[3];
            cov3_bwd(g3->quat + 4 * j, g3->log_scale + 3 * j, dcov, gq, gs);
            for (int k = 0; k < 3; ++k) { dmean3[3 * j + k] += dmu[k]; dlog3[3 * j + k] += gs[k]; }
            for (int k = 0; k < 4; ++k) dquat3[4 * j + k] += gq[k];
            for (int k = 0; k < 48; ++k) dsh3[48 * j + k] += dsh[k];
        }
    }
    free(dproj);
    free(P);
}

/* ------------------------------------------------------------------------ */
/* 4D -> 3D conversion (Sec. 4.1 identification, Sec. 4.2 conversion, Eq. 9) */
/* ------------------------------------------------------------------------ */

/* Eq. 9 with 1-based R(i,j) (reading D10).  When 1 + tr(R) is too small for
 * the printed formula (reading D9) the largest-diagonal branch of Shepperd's
 * method is used.  The result is normalised with w >= 0. */
void oracle_matrix_to_quat(const double R[9], double q[4])
{
#define RR(i, j) R[((i) - 1) * 3 + ((j) - 1)]
    double tr = RR(1, 1) + RR(2, 2) + RR(3, 3);
    double w, x, y, z;
    if (1.0 + tr > 1e-2) {
        w = 0.5 * sqrt(1.0 + tr);
        x = (RR(3, 2) - RR(2, 3)) / (4.0 * w);
        y = (RR(1, 3) - RR(3, 1)) / (4.0 * w);
        z = (RR(2, 1) - RR(1, 2)) / (4.0 * w);
    } else if (RR(1, 1) >= RR(2, 2) && RR(1, 1) >= RR(3, 3)) {
        x = 0.5 * sqrt(fmax(0.0, 1.0 + RR(1, 1) - RR(2, 2) - RR(3, 3)));
        w = (RR(3, 2) - RR(2, 3)) / (4.0 * x);
        y = (RR(1, 2) + RR(2, 1)) / (4.0 * x);
        z = (RR(1, 3) + RR(3, 1)) / (4.0 * x);
    } else if (RR(2, 2) >= RR(3, 3)) {
        y = 0.5 * sqrt(fmax(0.0, 1.0 - RR(1, 1) + RR(2, 2) - RR(3, 3)));
        w = (RR(1, 3) - RR(3, 1)) / (4.0 * y);
        x = (RR(1, 2) + RR(2, 1)) / (4.0 * y);
        z = (RR(2, 3) + RR(3, 2)) / (4.0 * y);
    } else {
        z = 0.5 * sqrt(fmax(0.0, 1.0 - RR(1, 1) - RR(2, 2) + RR(3, 3)));
        w = (RR(2, 1) - RR(1, 2)) / (4.0 * z);
        x = (RR(1, 3) + RR(3, 1)) / (4.0 * z);
        y = (RR(2, 3) + RR(3, 2)) / (4.0 * z);
    }
#undef RR
    double n = sqrt(w * w + x * x + y * y + z * z);
    double sgn = w < 0.0 ? -1.0 : 1.0;
    q[0] = sgn * w / n; q[1] = sgn * x / n; q[2] = sgn * y / n; q[3] = sgn * z / n;
}

/*
 * Sec. 4.1: Gaussian i is static iff exp(s_t,i) > tau.  Sec. 4.2: a static
 * Gaussian becomes (mu_x, q_3D, s_x, s_y, s_z, sigma, SH), q_3D from the
 * top-left 3x3 of R_4D by Eq. 9; mu_t and s_t are dropped.
 * Outputs: moved[n4] (0/1); for each moved Gaussian in increasing 4D index
 * order, one appended 3D record (mean3, log3, quat3, op3, sh3).  The 4D set
 * keeps the rest in order (keep_idx lists their original indices).
 * Returns the number moved.
 */
int64_t oracle_convert(const og4 *g4, double tau, int32_t *moved,
                       double *mean3, double *log3, double *quat3, double *op3, double *sh3,
                       int64_t *keep_idx)
{
    int64_t nm = 0, nk = 0;
    for (int64_t i = 0; i < g4->n; ++i) {
        int is_static = exp(g4->log_scale[4 * i + 3]) > tau;
        moved[i] = is_static;
        if (!is_static) { keep_idx[nk++] = i; continue; }
        double R4[16], R3[9];
        oracle_rot4(g4->ql + 4 * i, g4->qr + 4 * i, R4);
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) R3[r * 3 + c] = R4[r * 4 + c];
        oracle_matrix_to_quat(R3, quat3 + 4 * nm);
        for (int k = 0; k < 3; ++k) {
            mean3[3 * nm + k] = g4->mean[4 * i + k];
            log3[3 * nm + k] = g4->log_scale[4 * i + k];
        }
        op3[nm] = g4->opacity[i];
        /* the colour keeps its time-constant block (the average over the sequence) */
        for (int k = 0; k < 48; ++k) sh3[48 * nm + k] = g4->sh[48 * (g4->n_time + 1) * i + k];
        ++nm;
    }
    return nm;
}

/* ------------------------------------------------------------------------ */
/* Stable sort of 64-bit keys (Alg. 1 "SortByKeys"): perm = argsort, ties by  */
/* position                                                                  */
/* ------------------------------------------------------------------------ */

typedef struct { uint64_t key; int64_t pos; } kp;

static int cmp_kp(const void *pa, const void *pb)
{
    const kp *a = pa, *b = pb;
    if (a->key != b->key) return a->key < b->key ? -1 : 1;
    return (a->pos > b->pos) - (a->pos < b->pos);
}

void oracle_stable_sort_u64(const uint64_t *keys, int64_t n, int64_t *perm)
{
    kp *a = malloc(sizeof(kp) * (size_t)(n > 0 ? n : 1));
    for (int64_t i = 0; i < n; ++i) { a[i].key = keys[i]; a[i].pos = i; }
    qsort(a, (size_t)n, sizeof(kp), cmp_kp);
    for (int64_t i = 0; i < n; ++i) perm[i] = a[i].pos;
    free(a);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
