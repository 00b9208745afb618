/*
 * qb_oracle.c -- plain, slow FP64 CPU oracle for the QuadBox tile rasteriser.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this file:
 * only the tests, the smoke check and the CPU-baseline leg of the benchmark
 * do.  It shares no code, header, table or helper with the CUDA library.
 *
 * It follows "QuadBox: Accelerating 3D Gaussian Splatting with Geometry-Aware
 * Boxes" (arXiv 2605.04844):
 *   - Gaussian primitive, Eq. 1 (Sec. 2); EWA projection to 2D (Sec. 2, the
 *     paper cites Zwicker et al. and the 3DGS code base for the details);
 *   - front-to-back compositing, Eq. 2 (Sec. 2);
 *   - opacity-aware confidence ellipse, Eq. 3 and Eq. 4 (Sec. 3.1.1), read on
 *     the kept side  d^T Lambda d <= gamma,  gamma = 2 ln(o / alpha_min);
 *   - extents via the support function, Eqs. support / extents-inv (Sec. 3.1.2);
 *   - the stretching factor f, Eq. f-closed (Sec. 3.1.2);
 *   - DualBox / QuadBox sub-boxes (Sec. 3.1.2);
 *   - QPass scan-line traversal (Sec. 3.2) and the naive nested-loop traversal
 *     the paper compares it with (Sec. 3.2, Table 3 "QuadBox-dagger").
 *
 * Everything is double precision except the tile-rectangle replay
 * (orc_rects_f32), which deliberately repeats the float32 rounding rule of
 * the tile mapping so that it can be fed float32 box parameters and produce
 * the same integers (see the comment there).
 *
 * Parity status: every function here is pinned by a CPU test against closed
 * forms, brute force or a library routine (tests/test_oracle_pins.py).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_TILE 16
#define ORC_NF 32   /* doubles per Gaussian in the projection record */

/* projection record fields */
enum {
    F_VALID = 0, F_X = 1, F_Y = 2, F_DEPTH = 3,
    F_S11 = 4, F_S12 = 5, F_S22 = 6,          /* 2D covariance Sigma^2D      */
    F_A = 7, F_B = 8, F_C = 9,                 /* conic Lambda = [a b; b c]   */
    F_O = 10,                                   /* opacity o                   */
    F_R = 11, F_G = 12, F_BL = 13,              /* colour after clamp          */
    F_CLAMP = 14,                               /* bit c set: channel c < 0    */
    F_GAMMA = 15, F_GAMMAB = 16,                /* gamma and box threshold     */
    F_XMAX = 17, F_YMAX = 18,                   /* AdR extents (Eq. extents)   */
    F_XMIN = 19, F_YMIN = 20,                   /* f*x_max, f*y_max            */
    F_F = 21, F_R3 = 22, F_ORIENT = 23,
    F_TXCLAMP = 24, F_TYCLAMP = 25              /* Jacobian clamp active       */
};

/* camera: viewmat[16] row-major world->view, fx, fy, cx, cy, tan_fovx,
 * tan_fovy, campos[3], znear */
enum { CAM_FX = 16, CAM_FY = 17, CAM_CX = 18, CAM_CY = 19, CAM_TANX = 20,
       CAM_TANY = 21, CAM_POS = 22, CAM_ZNEAR = 25 };

/* binning modes (the same numbering the library uses in its public header) */
enum { M_AABB3S = 0, M_QUADBOX = 1, M_ADR = 2, M_QUADBOX_NAIVE = 3, M_DUALBOX = 4 };

static const double ALPHA_MIN = 1.0 / 255.0;

/* ------------------------------------------------------------------------ */
/* Spherical harmonics from their definition.                                */
/* ------------------------------------------------------------------------ */

static double factorial(int k)
{
    double r = 1.0;
    for (int i = 2; i <= k; ++i) r *= (double)i;
    return r;
}

/* Associated Legendre function P_l^m(x), m >= 0, including the
 * Condon-Shortley phase (-1)^m; textbook three-term recurrence in l. */
static double assoc_legendre(int l, int m, double x)
{
    double s = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;
    for (int i = 1; i <= m; ++i) pmm *= -(2.0 * i - 1.0) * s;
    if (l == m) return pmm;
    double pm1 = x * (2.0 * m + 1.0) * pmm;
    if (l == m + 1) return pm1;
    double pll = 0.0;
    for (int ll = m + 2; ll <= l; ++ll) {
        pll = ((2.0 * ll - 1.0) * x * pm1 - (ll + m - 1.0) * pmm) / (double)(ll - m);
        pmm = pm1;
        pm1 = pll;
    }
    return pll;
}

/* Real spherical harmonics built from the complex ones Y_l^m (with the
 * Condon-Shortley phase):  m<0: sqrt2 Im Y_l^|m|,  m=0: Y_l^0,
 * m>0: sqrt2 Re Y_l^m.  Coefficient index k = l*l + l + m.  d is a unit
 * vector; the angles are taken from it directly. */
/* Threads of the OpenMP loops (timing only; results do not depend on it). */
void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int orc_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_sh_basis(int deg, const double *d, double *Y)
{
    double z = fmax(-1.0, fmin(1.0, d[2]));
    double phi = atan2(d[1], d[0]);
    for (int l = 0; l <= deg; ++l) {
        for (int m = -l; m <= l; ++m) {
            int am = m < 0 ? -m : m;
            double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * factorial(l - am) / factorial(l + am));
            double P = assoc_legendre(l, am, z);
            double v;
            if (m == 0) v = K * P;
            else if (m > 0) v = sqrt(2.0) * K * P * cos(m * phi);
            else v = sqrt(2.0) * K * P * sin(am * phi);
            Y[l * l + l + m] = v;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Projection (Sec. 2): one Gaussian -> projection record.                   */
/* ------------------------------------------------------------------------ */

/* Rotation matrix of the unit quaternion (w, x, y, z). */
void orc_quat_to_rot(const double *q_in, double R[9])
{
    double n = sqrt(q_in[0] * q_in[0] + q_in[1] * q_in[1] + q_in[2] * q_in[2] + q_in[3] * q_in[3]);
    double w = q_in[0] / n, x = q_in[1] / n, y = q_in[2] / n, z = q_in[3] / n;
    R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z);       R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (x * y + w * z);       R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (x * z - w * y);       R[7] = 2.0 * (y * z + w * x);       R[8] = 1.0 - 2.0 * (x * x + y * y);
}

static void project_one(const double *mean, const double *scale, const double *quat, double opac_in,
                        const double *sh, int deg, int raw, const double *cam, double *out)
{
    memset(out, 0, ORC_NF * sizeof(double));
    const double *V = cam;
    double t[3];
    for (int i = 0; i < 3; ++i)
        t[i] = V[4 * i] * mean[0] + V[4 * i + 1] * mean[1] + V[4 * i + 2] * mean[2] + V[4 * i + 3];
    /* near-plane cull (3DGS convention; the paper is silent) */
    if (!(t[2] > cam[CAM_ZNEAR])) return;

    double s[3];
    for (int i = 0; i < 3; ++i) s[i] = raw ? exp(scale[i]) : scale[i];
    double R[9];
    orc_quat_to_rot(quat, R);
    /* Sigma_3D = R diag(s^2) R^T */
    double S3[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * s[k] * s[k] * R[3 * j + k];
            S3[3 * i + j] = acc;
        }

    double fx = cam[CAM_FX], fy = cam[CAM_FY];
    double limx = 1.3 * cam[CAM_TANX], limy = 1.3 * cam[CAM_TANY];
    double txtz = t[0] / t[2], tytz = t[1] / t[2];
    double cxtz = fmin(limx, fmax(-limx, txtz));
    double cytz = fmin(limy, fmax(-limy, tytz));
    double txc = cxtz * t[2], tyc = cytz * t[2];
    /* local affine approximation J of the perspective map (EWA) */
    double J[6] = { fx / t[2], 0.0, -fx * txc / (t[2] * t[2]),
                    0.0, fy / t[2], -fy * tyc / (t[2] * t[2]) };
    double M[6];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += J[3 * i + k] * V[4 * k + j];
            M[3 * i + j] = acc;
        }
    double S2[4];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 2; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                for (int l = 0; l < 3; ++l) acc += M[3 * i + k] * S3[3 * k + l] * M[3 * j + l];
            S2[2 * i + j] = acc;
        }
    S2[0] += 0.3; /* low-pass dilation of the 3DGS code base */
    S2[3] += 0.3;
    double s11 = S2[0], s12 = 0.5 * (S2[1] + S2[2]), s22 = S2[3];
    double det = s11 * s22 - s12 * s12;
    if (!(det > 0.0)) return;
    double a = s22 / det, b = -s12 / det, c = s11 / det; /* Lambda = Sigma2D^-1 */

    double o = raw ? 1.0 / (1.0 + exp(-opac_in)) : opac_in;
    if (!(o >= ALPHA_MIN)) return; /* no pixel can reach alpha_min */

    /* Eq. 3 on its kept side: alpha >= alpha_min  <=>  d^T Lambda d <= gamma */
    double gamma = 2.0 * log(o / ALPHA_MIN);
    /* Eq. f-closed */
    double f = sqrt(1.0 - b * b / (a * c));
    /* box threshold: gamma plus a margin that covers float32 evaluation of
     * the ellipse test by the renderer (relative 2^-18 / f^2, absolute 1e-3) */
    double gamma_b = gamma * (1.0 + ldexp(1.0, -18) / (f * f)) + 1e-3;
    /* Eq. extents-inv: x_max = sqrt(gamma (Lambda^-1)_11), (Lambda^-1) = Sigma2D */
    double xmax = sqrt(gamma_b * s11), ymax = sqrt(gamma_b * s22);

    /* 3-sigma radius of the vanilla rasteriser (Sec. 2): side 6 sqrt(lambda_max) */
    double mid = 0.5 * (s11 + s22);
    double lmax = mid + sqrt(fmax(0.1, mid * mid - det));
    double r3 = ceil(3.0 * sqrt(lmax));

    /* colour from SH (Sec. 2, "spherical harmonic coefficients") */
    double v[3] = { mean[0] - cam[CAM_POS], mean[1] - cam[CAM_POS + 1], mean[2] - cam[CAM_POS + 2] };
    double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double d[3] = { v[0] / vn, v[1] / vn, v[2] / vn };
    double Y[16];
    orc_sh_basis(deg, d, Y);
    int K = (deg + 1) * (deg + 1);
    int clampmask = 0;
    double rgb[3];
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += sh[3 * k + ch] * Y[k];
        acc += 0.5;
        if (acc < 0.0) { clampmask |= 1 << ch; acc = 0.0; }
        rgb[ch] = acc;
    }

    out[F_X] = fx * t[0] / t[2] + cam[CAM_CX];
    out[F_Y] = fy * t[1] / t[2] + cam[CAM_CY];
    out[F_DEPTH] = t[2];
    out[F_S11] = s11; out[F_S12] = s12; out[F_S22] = s22;
    out[F_A] = a; out[F_B] = b; out[F_C] = c;
    out[F_O] = o;
    out[F_R] = rgb[0]; out[F_G] = rgb[1]; out[F_BL] = rgb[2];
    out[F_CLAMP] = clampmask;
    out[F_GAMMA] = gamma; out[F_GAMMAB] = gamma_b;
    out[F_XMAX] = xmax; out[F_YMAX] = ymax;
    out[F_XMIN] = f * xmax; out[F_YMIN] = f * ymax;
    out[F_F] = f; out[F_R3] = r3;
    out[F_ORIENT] = (s12 >= 0.0) ? 1.0 : 0.0;
    out[F_TXCLAMP] = (txtz != cxtz) ? 1.0 : 0.0;
    out[F_TYCLAMP] = (tytz != cytz) ? 1.0 : 0.0;
    int finite = 1;
    for (int i = 1; i <= F_R3; ++i) finite &= isfinite(out[i]) ? 1 : 0;
    out[F_VALID] = finite ? 1.0 : 0.0;
}

void orc_project(int n, const double *means, const double *scales, const double *quats,
                 const double *opac, const double *sh, int deg, int raw, const double *cam,
                 double *out)
{
    int K = (deg + 1) * (deg + 1);
#pragma omp parallel for schedule(static)
    for (int i = 0; i < n; ++i)
        project_one(means + 3 * (size_t)i, scales + 3 * (size_t)i, quats + 4 * (size_t)i, opac[i],
                    sh + (size_t)K * 3 * i, deg, raw, cam, out + (size_t)ORC_NF * i);
}

/* ------------------------------------------------------------------------ */
/* Tile rectangles.                                                          */
/*                                                                           */
/* A closed pixel interval [lo, hi] (pixel centres at integer coordinates)   */
/* covers the centres ceil(lo) .. floor(hi), clipped to the image; tile t    */
/* holds the centres 16t .. 16t+15.  Each sub-box is a closed rectangle with */
/* one corner at mu^2D.  The 3-sigma rectangle is                             */
/* [ceil(mu) - r3, floor(mu) + r3] per axis, and in the clamped (default)    */
/* configuration every sub-box is intersected with it.                       */
/* ------------------------------------------------------------------------ */

typedef struct { int x0, y0, x1, y1; } orc_rect; /* inclusive, empty if x0>x1 || y0>y1 */

static const orc_rect EMPTY_RECT = { 1, 1, 0, 0 };

static int rect_empty(orc_rect r) { return r.x0 > r.x1 || r.y0 > r.y1; }

/* float32 replay: every operation below is one IEEE single-precision
 * operation, so float32 inputs give exactly the integers the renderer
 * computes from the same inputs. */
static int tiles_f(float lo, float hi, int npx, int *t0, int *t1)
{
    float p0 = ceilf(lo), p1 = floorf(hi);
    p0 = fmaxf(p0, 0.0f);
    p1 = fminf(p1, (float)(npx - 1));
    if (!(p0 <= p1)) return 0;
    *t0 = (int)p0 / ORC_TILE;
    *t1 = (int)p1 / ORC_TILE;
    return 1;
}

static int tiles_d(double lo, double hi, int npx, int *t0, int *t1)
{
    double p0 = ceil(lo), p1 = floor(hi);
    p0 = fmax(p0, 0.0);
    p1 = fmin(p1, (double)(npx - 1));
    if (!(p0 <= p1)) return 0;
    *t0 = (int)p0 / ORC_TILE;
    *t1 = (int)p1 / ORC_TILE;
    return 1;
}

static orc_rect intersect(orc_rect a, orc_rect b)
{
    orc_rect r = { a.x0 > b.x0 ? a.x0 : b.x0, a.y0 > b.y0 ? a.y0 : b.y0,
                   a.x1 < b.x1 ? a.x1 : b.x1, a.y1 < b.y1 ? a.y1 : b.y1 };
    return rect_empty(r) ? EMPTY_RECT : r;
}

/* Quadrant order: I (+x,+y), II (-x,+y), III (-x,-y), IV (+x,-y).
 * orient = 1: Sigma12 >= 0, the major axis runs through quadrants I and III. */
static int quadrant_is_major(int q, int orient)
{
    int same_sign = (q == 0 || q == 2);
    return orient ? same_sign : !same_sign;
}

static void build_rects(int mode, int clamp3s, int have, orc_rect r3s,
                        orc_rect quad[4], orc_rect adr, orc_rect *out4)
{
    for (int q = 0; q < 4; ++q) out4[q] = EMPTY_RECT;
    if (!have) return;
    switch (mode) {
    case M_AABB3S: out4[0] = r3s; break;
    case M_ADR: out4[0] = clamp3s ? intersect(adr, r3s) : adr; break;
    case M_QUADBOX:
    case M_QUADBOX_NAIVE:
        for (int q = 0; q < 4; ++q) out4[q] = clamp3s ? intersect(quad[q], r3s) : quad[q];
        break;
    case M_DUALBOX:
        for (int q = 0; q < 4; ++q) out4[q] = clamp3s ? intersect(quad[q], r3s) : quad[q];
        break;
    default: break;
    }
    for (int q = 0; q < 4; ++q)
        if (rect_empty(out4[q])) out4[q] = EMPTY_RECT;
}

#define DEFINE_RECTS(NAME, T, TILES, CEIL, FLOOR)                                              \
static void NAME(T mx, T my, T ex, T ey, T exm, T eym, T r3, int orient, int mode,           \
                 int clamp3s, int W, int H, orc_rect *out4)                                    \
{                                                                                              \
    orc_rect r3s = EMPTY_RECT;                                                                 \
    int ok = TILES((T)(CEIL(mx) - r3), (T)(FLOOR(mx) + r3), W, &r3s.x0, &r3s.x1)              \
           & TILES((T)(CEIL(my) - r3), (T)(FLOOR(my) + r3), H, &r3s.y0, &r3s.y1);             \
    if (!ok) r3s = EMPTY_RECT;                                                                 \
    orc_rect quad[4], adr = EMPTY_RECT;                                                        \
    for (int q = 0; q < 4; ++q) {                                                              \
        int major = quadrant_is_major(q, orient);                                              \
        if (mode == M_DUALBOX && !major) { quad[q] = EMPTY_RECT; continue; }                   \
        T exq = major ? ex : exm, eyq = major ? ey : eym;                                      \
        int sx = (q == 0 || q == 3) ? 1 : -1, sy = (q == 0 || q == 1) ? 1 : -1;                \
        T xlo = sx > 0 ? mx : (T)(mx - exq), xhi = sx > 0 ? (T)(mx + exq) : mx;                \
        T ylo = sy > 0 ? my : (T)(my - eyq), yhi = sy > 0 ? (T)(my + eyq) : my;                \
        orc_rect r;                                                                            \
        int okq = TILES(xlo, xhi, W, &r.x0, &r.x1) & TILES(ylo, yhi, H, &r.y0, &r.y1);         \
        quad[q] = okq ? r : EMPTY_RECT;                                                        \
    }                                                                                          \
    {                                                                                          \
        orc_rect r;                                                                            \
        int oka = TILES((T)(mx - ex), (T)(mx + ex), W, &r.x0, &r.x1)                           \
                & TILES((T)(my - ey), (T)(my + ey), H, &r.y0, &r.y1);                          \
        adr = oka ? r : EMPTY_RECT;                                                            \
    }                                                                                          \
    int have = (mode == M_AABB3S) ? !rect_empty(r3s) : 1;                                      \
    if (clamp3s && rect_empty(r3s)) have = 0;                                                  \
    build_rects(mode, clamp3s, have, r3s, quad, adr, out4);                                    \
}

DEFINE_RECTS(rects_one_f, float, tiles_f, ceilf, floorf)
DEFINE_RECTS(rects_one_d, double, tiles_d, ceil, floor)

/* Tile rectangles from float32 box parameters (the GPU's record):
 * xy[n][2], ext[n][4] = (x_max, y_max, f x_max, f y_max), r3[n], orient[n],
 * valid[n].  rects[n][4][4] = (x0, y0, x1, y1) per sub-box. */
void orc_rects_f32(int n, const float *xy, const float *ext, const float *r3, const int32_t *orient,
                   const int32_t *valid, int mode, int clamp3s, int W, int H, int32_t *rects)
{
    for (int i = 0; i < n; ++i) {
        orc_rect out4[4];
        if (valid[i])
            rects_one_f(xy[2 * i], xy[2 * i + 1], ext[4 * i], ext[4 * i + 1], ext[4 * i + 2], ext[4 * i + 3],
                        r3[i], orient[i], mode, clamp3s, W, H, out4);
        else
            for (int q = 0; q < 4; ++q) out4[q] = EMPTY_RECT;
        for (int q = 0; q < 4; ++q) {
            int32_t *o = rects + 16 * (size_t)i + 4 * q;
            o[0] = out4[q].x0; o[1] = out4[q].y0; o[2] = out4[q].x1; o[3] = out4[q].y1;
        }
    }
}

/* Tile rectangles from the oracle's own FP64 projection records. */
void orc_rects_f64(int n, const double *proj, int mode, int clamp3s, int W, int H, int32_t *rects)
{
    for (int i = 0; i < n; ++i) {
        const double *p = proj + (size_t)ORC_NF * i;
        orc_rect out4[4];
        if (p[F_VALID] != 0.0)
            rects_one_d(p[F_X], p[F_Y], p[F_XMAX], p[F_YMAX], p[F_XMIN], p[F_YMIN], p[F_R3],
                        (int)p[F_ORIENT], mode, clamp3s, W, H, out4);
        else
            for (int q = 0; q < 4; ++q) out4[q] = EMPTY_RECT;
        for (int q = 0; q < 4; ++q) {
            int32_t *o = rects + 16 * (size_t)i + 4 * q;
            o[0] = out4[q].x0; o[1] = out4[q].y0; o[2] = out4[q].x1; o[3] = out4[q].y1;
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Tile enumeration.                                                          */
/* ------------------------------------------------------------------------ */

static orc_rect get_rect(const int32_t *rects, int i, int q)
{
    const int32_t *o = rects + 16 * (size_t)i + 4 * q;
    orc_rect r = { o[0], o[1], o[2], o[3] };
    return r;
}

/* QPass (Sec. 3.2): (1) tile bounds per sub-box, aggregated into the global
 * range; (2) scan lines along the shorter axis of that range; (3) on each
 * line, the sub-boxes whose range overlaps the line contribute their extent
 * on the other axis, merged by min/max.  If tiles is NULL only counts. */
static int64_t qpass_one(const int32_t *rects, int i, int tiles_x, uint32_t *tiles)
{
    orc_rect b[4];
    int gx0 = 1 << 30, gy0 = 1 << 30, gx1 = -1, gy1 = -1, any = 0;
    for (int q = 0; q < 4; ++q) {
        b[q] = get_rect(rects, i, q);
        if (rect_empty(b[q])) continue;
        any = 1;
        if (b[q].x0 < gx0) gx0 = b[q].x0;
        if (b[q].y0 < gy0) gy0 = b[q].y0;
        if (b[q].x1 > gx1) gx1 = b[q].x1;
        if (b[q].y1 > gy1) gy1 = b[q].y1;
    }
    if (!any) return 0;
    int columns = (gx1 - gx0) <= (gy1 - gy0); /* scan the shorter axis */
    int64_t cnt = 0;
    int s0 = columns ? gx0 : gy0, s1 = columns ? gx1 : gy1;
    for (int s = s0; s <= s1; ++s) {
        int lo = 1 << 30, hi = -1;
        for (int q = 0; q < 4; ++q) {
            if (rect_empty(b[q])) continue;
            int a0 = columns ? b[q].x0 : b[q].y0, a1 = columns ? b[q].x1 : b[q].y1;
            if (s < a0 || s > a1) continue; /* interval overlap test */
            int o0 = columns ? b[q].y0 : b[q].x0, o1 = columns ? b[q].y1 : b[q].x1;
            if (o0 < lo) lo = o0;
            if (o1 > hi) hi = o1;
        }
        for (int u = lo; u <= hi; ++u) {
            if (tiles) {
                int tx = columns ? s : u, ty = columns ? u : s;
                tiles[cnt] = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx;
            }
            ++cnt;
        }
    }
    return cnt;
}

/* Naive traversal (QuadBox-dagger): nested loops over each sub-box's tile
 * rectangle, skipping a tile already covered by an earlier sub-box. */
static int64_t naive_one(const int32_t *rects, int i, int tiles_x, uint32_t *tiles)
{
    int64_t cnt = 0;
    for (int q = 0; q < 4; ++q) {
        orc_rect r = get_rect(rects, i, q);
        if (rect_empty(r)) continue;
        for (int ty = r.y0; ty <= r.y1; ++ty)
            for (int tx = r.x0; tx <= r.x1; ++tx) {
                int seen = 0;
                for (int p = 0; p < q; ++p) {
                    orc_rect e = get_rect(rects, i, p);
                    if (!rect_empty(e) && tx >= e.x0 && tx <= e.x1 && ty >= e.y0 && ty <= e.y1) seen = 1;
                }
                if (seen) continue;
                if (tiles) tiles[cnt] = (uint32_t)ty * (uint32_t)tiles_x + (uint32_t)tx;
                ++cnt;
            }
    }
    return cnt;
}

void orc_count(int n, const int32_t *rects, int use_qpass, int64_t *counts)
{
    for (int i = 0; i < n; ++i)
        counts[i] = use_qpass ? qpass_one(rects, i, 0, NULL) : naive_one(rects, i, 0, NULL);
}

/* Writes each Gaussian's tiles at offsets[i] (exclusive prefix of counts). */
void orc_emit(int n, const int32_t *rects, int use_qpass, int tiles_x, const int64_t *offsets,
              uint32_t *tiles_out, uint32_t *gid_out)
{
    for (int i = 0; i < n; ++i) {
        uint32_t *dst = tiles_out + offsets[i];
        int64_t c = use_qpass ? qpass_one(rects, i, tiles_x, dst) : naive_one(rects, i, tiles_x, dst);
        for (int64_t k = 0; k < c; ++k) gid_out[offsets[i] + k] = (uint32_t)i;
    }
}

/* ------------------------------------------------------------------------ */
/* Compositing (Eq. 2), per pixel over the depth-sorted tile list.           */
/*                                                                           */
/* Per entry: q = d^T Lambda d, skip if -q/2 > 0; alpha = min(0.99, o e^{-q/2});*/
/* skip if alpha < 1/255; T' = T (1 - alpha); stop (without adding) once      */
/* T' < 1e-4; else C += alpha T c, T = T'.  out = C + T bg.  (The 0.99 cap, */
/* the 1/255 skip and the 1e-4 stop are 3DGS conventions.)                   */
/*                                                                           */
/* amb[p] flags pixels whose discrete decisions are within a float32        */
/* evaluation's error of their thresholds: alpha vs 1/255 and o G vs the     */
/* 0.99 cap within 1e-3 relative (a float32 alpha carries |power| times the */
/* conic's relative error, up to ~1e-4 for ill-conditioned projections),    */
/* T' vs 1e-4 within 1e-3, and two consecutive contributors of nearly equal */
/* depth.                                                                    */
/* ------------------------------------------------------------------------ */

static void composite_pixel(int px, int py, const int32_t *ids, int64_t cnt, const double *proj,
                            const double *bg, double *C3, double *Tfin, int32_t *last, int32_t *amb)
{
    double T = 1.0, C[3] = { 0.0, 0.0, 0.0 };
    int32_t lastc = 0;
    int a = 0;
    double prev_depth = -1.0;
    for (int64_t k = 0; k < cnt; ++k) {
        const double *p = proj + (size_t)ORC_NF * ids[k];
        double dx = p[F_X] - px, dy = p[F_Y] - py;
        double q = p[F_A] * dx * dx + 2.0 * p[F_B] * dx * dy + p[F_C] * dy * dy;
        double power = -0.5 * q;
        if (power > 0.0) continue;
        double oG = p[F_O] * exp(power);
        double alpha = fmin(0.99, oG);
        if (fabs(alpha / ALPHA_MIN - 1.0) < 1e-3) a = 1;
        if (alpha < ALPHA_MIN) continue;
        if (fabs(oG / 0.99 - 1.0) < 1e-3) a = 1;
        double testT = T * (1.0 - alpha);
        if (fabs(testT / 1e-4 - 1.0) < 1e-3) a = 1;
        if (prev_depth >= 0.0 && fabs(p[F_DEPTH] - prev_depth) <= 1e-6 * p[F_DEPTH]) a = 1;
        if (testT < 1e-4) break;
        for (int ch = 0; ch < 3; ++ch) C[ch] += alpha * T * p[F_R + ch];
        T = testT;
        lastc = (int32_t)(k + 1);
        prev_depth = p[F_DEPTH];
    }
    for (int ch = 0; ch < 3; ++ch) C3[ch] = C[ch] + T * bg[ch];
    *Tfin = T;
    *last = lastc;
    *amb = a;
}

/* ranges[t] = [start, end) into vals for tile t (row-major tile id). */
void orc_render(int W, int H, const int64_t *ranges, const int32_t *vals, const double *proj,
                const double *bg, double *img, double *Tfin, int32_t *ncontrib, int32_t *amb)
{
    int tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
#pragma omp parallel for schedule(dynamic, 4)
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int t = (py / ORC_TILE) * tiles_x + px / ORC_TILE;
            int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
            double C3[3];
            size_t pix = (size_t)py * W + px;
            composite_pixel(px, py, vals + s, e - s, proj, bg, C3, &Tfin[pix], &ncontrib[pix], &amb[pix]);
            for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + pix] = C3[ch];
        }
}

/* Same compositing for a list of sampled pixels (px[k], py[k]). */
void orc_render_pixels(int W, int H, int npix, const int32_t *pxs, const int32_t *pys,
                       const int64_t *ranges, const int32_t *vals, const double *proj,
                       const double *bg, double *rgb_out, double *Tfin, int32_t *ncontrib,
                       int32_t *amb)
{
    int tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
    (void)H;
#pragma omp parallel for schedule(dynamic, 4)
    for (int k = 0; k < npix; ++k) {
        int px = pxs[k], py = pys[k];
        int t = (py / ORC_TILE) * tiles_x + px / ORC_TILE;
        int64_t s = ranges[2 * t], e = ranges[2 * t + 1];
        composite_pixel(px, py, vals + s, e - s, proj, bg, rgb_out + 3 * (size_t)k, &Tfin[k],
                        &ncontrib[k], &amb[k]);
    }
}

typedef struct { double depth; int32_t id; } depth_id;

static int cmp_depth_id(const void *pa, const void *pb)
{
    const depth_id *a = (const depth_id *)pa, *b = (const depth_id *)pb;
    if (a->depth < b->depth) return -1;
    if (a->depth > b->depth) return 1;
    return (a->id > b->id) - (a->id < b->id);
}

/* Tile-free brute force: every pixel composites all Gaussians whose tile
 * set (given as rectangles) contains the pixel's tile, sorted by
 * (depth, index).  No key, no sort of pairs, no ranges. */
void orc_render_brute(int W, int H, int n, const int32_t *rects, const double *proj, const double *bg,
                      double *img, double *Tfin, int32_t *ncontrib, int32_t *amb)
{
#pragma omp parallel
    {
        depth_id *buf = (depth_id *)malloc(sizeof(depth_id) * (size_t)(n > 0 ? n : 1));
        int32_t *ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
#pragma omp for schedule(dynamic, 1)
        for (int py = 0; py < H; ++py)
            for (int px = 0; px < W; ++px) {
                int tx = px / ORC_TILE, ty = py / ORC_TILE;
                int m = 0;
                for (int i = 0; i < n; ++i) {
                    if (proj[(size_t)ORC_NF * i + F_VALID] == 0.0) continue;
                    int in = 0;
                    for (int q = 0; q < 4; ++q) {
                        orc_rect r = get_rect(rects, i, q);
                        if (!rect_empty(r) && tx >= r.x0 && tx <= r.x1 && ty >= r.y0 && ty <= r.y1) in = 1;
                    }
                    if (in) { buf[m].depth = proj[(size_t)ORC_NF * i + F_DEPTH]; buf[m].id = i; ++m; }
                }
                qsort(buf, (size_t)m, sizeof(depth_id), cmp_depth_id);
                for (int k = 0; k < m; ++k) ids[k] = buf[k].id;
                size_t pix = (size_t)py * W + px;
                double C3[3];
                composite_pixel(px, py, ids, m, proj, bg, C3, &Tfin[pix], &ncontrib[pix], &amb[pix]);
                for (int ch = 0; ch < 3; ++ch) img[(size_t)ch * W * H + pix] = C3[ch];
            }
        free(buf);
        free(ids);
    }
}

/* ------------------------------------------------------------------------ */
/* Backward of Eq. 2 per pixel (plain differentiation, no reverse trick).    */
/*                                                                           */
/* C = sum_i T_i alpha_i c_i + T_N bg  over the accepted entries i.          */
/*   dC/dc_k     = T_k alpha_k                                               */
/*   dC/dalpha_k = T_k c_k - (sum_{i>k} T_i alpha_i c_i + T_N bg)/(1-alpha_k)  */
/* then alpha = min(0.99, o G), G = exp(-q/2), q = a dx^2 + 2b dx dy + c dy^2 */
/* (zero derivative where the 0.99 cap is active).  dL/dconic is w.r.t. the */
/* three numbers (a, b, c) as they appear in q.                              */
/* ------------------------------------------------------------------------ */
/* One pixel's share of the backward: the forward walk over its tile list
 * (recording every counted entry), then, per counted entry k, the colour
 * behind it S_k = sum_{i>k} T_i alpha_i c_i + T_final bg and the gradient
 * of sum_ch g_ch C_ch through alpha_k (Eq. 2 differentiated), chained to o,
 * the conic and mu^2D.  acc_* are caller-provided buffers of the tile list's
 * length. */
typedef struct {
    int32_t *id;
    double *T, *a, *G, *dx, *dy;
    int *cap;
} orc_bwd_scratch;

/* With a_xy etc. non-NULL, every accumulated term's absolute value is
 * summed there too (the magnitude sum_p |term_p| of each gradient entry,
 * the scale of its rounding error when the terms are computed in float32). */
static void backward_pixel(int px, int py, const int32_t *ids, int64_t cnt, const double *proj,
                           const double *bg, const double g[3], orc_bwd_scratch *w, double *g_xy,
                           double *g_conic, double *g_o, double *g_rgb, double *a_xy, double *a_conic,
                           double *a_o, double *a_rgb)
{
    double T = 1.0;
    int m = 0;
    for (int64_t k = 0; k < cnt; ++k) {
        const double *p = proj + (size_t)ORC_NF * ids[k];
        double dx = p[F_X] - px, dy = p[F_Y] - py;
        double q = p[F_A] * dx * dx + 2.0 * p[F_B] * dx * dy + p[F_C] * dy * dy;
        double power = -0.5 * q;
        if (power > 0.0) continue;
        double G = exp(power);
        double alpha = fmin(0.99, p[F_O] * G);
        if (alpha < ALPHA_MIN) continue;
        double testT = T * (1.0 - alpha);
        if (testT < 1e-4) break;
        w->id[m] = ids[k]; w->T[m] = T; w->a[m] = alpha; w->G[m] = G;
        w->dx[m] = dx; w->dy[m] = dy; w->cap[m] = (p[F_O] * G >= 0.99);
        ++m;
        T = testT;
    }
    for (int k = 0; k < m; ++k) {
        const double *p = proj + (size_t)ORC_NF * w->id[k];
        double behind[3];
        for (int ch = 0; ch < 3; ++ch) {
            double sacc = T * bg[ch];
            for (int i = k + 1; i < m; ++i) {
                const double *pi = proj + (size_t)ORC_NF * w->id[i];
                sacc += w->T[i] * w->a[i] * pi[F_R + ch];
            }
            behind[ch] = sacc;
        }
        double dL_dalpha = 0.0, dL_dalpha_abs = 0.0;
        for (int ch = 0; ch < 3; ++ch) {
            g_rgb[3 * (size_t)w->id[k] + ch] += w->T[k] * w->a[k] * g[ch];
            dL_dalpha += g[ch] * (w->T[k] * p[F_R + ch] - behind[ch] / (1.0 - w->a[k]));
            dL_dalpha_abs += fabs(g[ch]) * (w->T[k] * p[F_R + ch] + behind[ch] / (1.0 - w->a[k]));
            if (a_rgb) a_rgb[3 * (size_t)w->id[k] + ch] += fabs(w->T[k] * w->a[k] * g[ch]);
        }
        if (w->cap[k]) continue;
        double G = w->G[k], o = p[F_O];
        g_o[w->id[k]] += G * dL_dalpha;
        double dL_dq = dL_dalpha * o * G * (-0.5);
        double dx = w->dx[k], dy = w->dy[k];
        g_conic[3 * (size_t)w->id[k] + 0] += dL_dq * dx * dx;
        g_conic[3 * (size_t)w->id[k] + 1] += dL_dq * 2.0 * dx * dy;
        g_conic[3 * (size_t)w->id[k] + 2] += dL_dq * dy * dy;
        g_xy[2 * (size_t)w->id[k] + 0] += dL_dq * 2.0 * (p[F_A] * dx + p[F_B] * dy);
        g_xy[2 * (size_t)w->id[k] + 1] += dL_dq * 2.0 * (p[F_B] * dx + p[F_C] * dy);
        if (a_o) {
            double q_abs = dL_dalpha_abs * o * G * 0.5;
            a_o[w->id[k]] += G * dL_dalpha_abs;
            a_conic[3 * (size_t)w->id[k] + 0] += q_abs * dx * dx;
            a_conic[3 * (size_t)w->id[k] + 1] += q_abs * 2.0 * fabs(dx * dy);
            a_conic[3 * (size_t)w->id[k] + 2] += q_abs * dy * dy;
            a_xy[2 * (size_t)w->id[k] + 0] += q_abs * 2.0 * (fabs(p[F_A] * dx) + fabs(p[F_B] * dy));
            a_xy[2 * (size_t)w->id[k] + 1] += q_abs * 2.0 * (fabs(p[F_B] * dx) + fabs(p[F_C] * dy));
        }
    }
}

static int bwd_scratch_alloc(orc_bwd_scratch *w, int64_t maxlen)
{
    size_t n = (size_t)(maxlen + 1);
    w->id = (int32_t *)malloc(sizeof(int32_t) * n);
    w->T = (double *)malloc(sizeof(double) * n);
    w->a = (double *)malloc(sizeof(double) * n);
    w->G = (double *)malloc(sizeof(double) * n);
    w->dx = (double *)malloc(sizeof(double) * n);
    w->dy = (double *)malloc(sizeof(double) * n);
    w->cap = (int *)malloc(sizeof(int) * n);
    return w->id && w->T && w->a && w->G && w->dx && w->dy && w->cap;
}

static void bwd_scratch_free(orc_bwd_scratch *w)
{
    free(w->id); free(w->T); free(w->a); free(w->G); free(w->dx); free(w->dy); free(w->cap);
}

static int64_t longest_list(int W, int H, const int64_t *ranges)
{
    int ntiles = ((W + ORC_TILE - 1) / ORC_TILE) * ((H + ORC_TILE - 1) / ORC_TILE);
    int64_t maxlen = 0;
    for (int t = 0; t < ntiles; ++t)
        if (ranges[2 * t + 1] - ranges[2 * t] > maxlen) maxlen = ranges[2 * t + 1] - ranges[2 * t];
    return maxlen;
}

/* Gradients of sum(dL_dimg * image) w.r.t. mu^2D, the conic, o and the
 * colour, accumulated over every pixel (dL_dimg planar [3][H][W]). */
void orc_render_backward(int W, int H, const int64_t *ranges, const int32_t *vals, const double *proj,
                         const double *bg, const double *dL_dimg, double *g_xy, double *g_conic,
                         double *g_o, double *g_rgb)
{
    int tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
    orc_bwd_scratch w;
    if (!bwd_scratch_alloc(&w, longest_list(W, H, ranges))) { bwd_scratch_free(&w); return; }
    for (int py = 0; py < H; ++py)
        for (int px = 0; px < W; ++px) {
            int t = (py / ORC_TILE) * tiles_x + px / ORC_TILE;
            size_t pix = (size_t)py * W + px;
            double g[3] = { dL_dimg[pix], dL_dimg[(size_t)W * H + pix], dL_dimg[2 * (size_t)W * H + pix] };
            backward_pixel(px, py, vals + ranges[2 * t], ranges[2 * t + 1] - ranges[2 * t], proj, bg, g, &w,
                           g_xy, g_conic, g_o, g_rgb, NULL, NULL, NULL, NULL);
        }
    bwd_scratch_free(&w);
}

/* The same sums over the m listed pixels (pxs[k], pys[k]) only, with their
 * loss gradients dL[k][3]; equal to orc_render_backward with dL_dimg zero
 * at every other pixel.  a_xy, a_conic, a_o, a_rgb (all NULL, or all
 * non-NULL and zeroed) receive the sums of the terms' absolute values. */
void orc_render_backward_pixels(int W, int H, int m, const int32_t *pxs, const int32_t *pys,
                                const int64_t *ranges, const int32_t *vals, const double *proj,
                                const double *bg, const double *dL, double *g_xy, double *g_conic,
                                double *g_o, double *g_rgb, double *a_xy, double *a_conic, double *a_o,
                                double *a_rgb)
{
    int tiles_x = (W + ORC_TILE - 1) / ORC_TILE;
    orc_bwd_scratch w;
    if (!bwd_scratch_alloc(&w, longest_list(W, H, ranges))) { bwd_scratch_free(&w); return; }
    for (int k = 0; k < m; ++k) {
        int px = pxs[k], py = pys[k];
        int t = (py / ORC_TILE) * tiles_x + px / ORC_TILE;
        backward_pixel(px, py, vals + ranges[2 * t], ranges[2 * t + 1] - ranges[2 * t], proj, bg, dL + 3 * (size_t)k,
                       &w, g_xy, g_conic, g_o, g_rgb, a_xy, a_conic, a_o, a_rgb);
    }
    bwd_scratch_free(&w);
}

/* ------------------------------------------------------------------------ */
/* Backward of the projection (chain rule through Sec. 2's EWA projection).  */
/* Inputs are the loss gradients w.r.t. mu^2D, (a, b, c), o and the clamped */
/* colour.  Outputs are gradients w.r.t. the raw parameters: means, scales  */
/* (log-scales when raw), quaternions (w,x,y,z, before normalisation),       */
/* opacities (logits when raw) and SH coefficients.                          */
/* ------------------------------------------------------------------------ */
void orc_project_backward(int n, const double *means, const double *scales, const double *quats,
                          const double *opac, const double *sh, int deg, int raw, const double *cam,
                          const double *g_xy, const double *g_conic, const double *g_o,
                          const double *g_rgb, double *gm, double *gs, double *gq, double *go,
                          double *gsh)
{
    int K = (deg + 1) * (deg + 1);
    const double *V = cam;
    for (int i = 0; i < n; ++i) {
        double rec[ORC_NF];
        const double *mean = means + 3 * (size_t)i, *scale = scales + 3 * (size_t)i;
        const double *quat = quats + 4 * (size_t)i, *shi = sh + (size_t)K * 3 * i;
        project_one(mean, scale, quat, opac[i], shi, deg, raw, cam, rec);
        if (rec[F_VALID] == 0.0) continue;

        /* --- recompute forward intermediates --- */
        double t[3];
        for (int r = 0; r < 3; ++r)
            t[r] = V[4 * r] * mean[0] + V[4 * r + 1] * mean[1] + V[4 * r + 2] * mean[2] + V[4 * r + 3];
        double s[3];
        for (int r = 0; r < 3; ++r) s[r] = raw ? exp(scale[r]) : scale[r];
        double qn = sqrt(quat[0] * quat[0] + quat[1] * quat[1] + quat[2] * quat[2] + quat[3] * quat[3]);
        double w = quat[0] / qn, x = quat[1] / qn, y = quat[2] / qn, z = quat[3] / qn;
        double R[9];
        orc_quat_to_rot(quat, R);
        double S3[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[3 * a + k] * s[k] * s[k] * R[3 * b + k];
                S3[3 * a + b] = acc;
            }
        double fx = cam[CAM_FX], fy = cam[CAM_FY];
        int clx = rec[F_TXCLAMP] != 0.0, cly = rec[F_TYCLAMP] != 0.0;
        double limx = 1.3 * cam[CAM_TANX], limy = 1.3 * cam[CAM_TANY];
        double txc = clx ? (t[0] > 0 ? limx : -limx) * t[2] : t[0];
        double tyc = cly ? (t[1] > 0 ? limy : -limy) * t[2] : t[1];
        double tz = t[2];
        double J[6] = { fx / tz, 0.0, -fx * txc / (tz * tz), 0.0, fy / tz, -fy * tyc / (tz * tz) };
        double M[6];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += J[3 * a + k] * V[4 * k + b];
                M[3 * a + b] = acc;
            }
        double La = rec[F_A], Lb = rec[F_B], Lc = rec[F_C];
        double Lam[4] = { La, Lb, Lb, Lc };

        /* --- conic -> Sigma2D:  H = -Lambda Ghat Lambda,  Ghat symmetric --- */
        double Gh[4] = { g_conic[3 * i], 0.5 * g_conic[3 * i + 1], 0.5 * g_conic[3 * i + 1], g_conic[3 * i + 2] };
        double tmp[4], Hs[4];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) tmp[2 * a + b] = Lam[2 * a] * Gh[b] + Lam[2 * a + 1] * Gh[2 + b];
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 2; ++b) Hs[2 * a + b] = -(tmp[2 * a] * Lam[b] + tmp[2 * a + 1] * Lam[2 + b]);

        /* --- Sigma2D = M S3 M^T + 0.3 I --- */
        double G3[9]; /* dL/dS3 = M^T H M */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 2; ++l) acc += M[3 * k + a] * Hs[2 * k + l] * M[3 * l + b];
                G3[3 * a + b] = acc;
            }
        double GM[6]; /* dL/dM = (H + H^T) M S3 */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 2; ++k)
                    for (int l = 0; l < 3; ++l)
                        acc += (Hs[2 * a + k] + Hs[2 * k + a]) * M[3 * k + l] * S3[3 * l + b];
                GM[3 * a + b] = acc;
            }
        double GJ[6]; /* dL/dJ = dL/dM W^T */
        for (int a = 0; a < 2; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += GM[3 * a + k] * V[4 * b + k];
                GJ[3 * a + b] = acc;
            }
        /* --- J(t) and mu2D(t) -> t --- */
        double gt[3] = { 0.0, 0.0, 0.0 };
        gt[0] += g_xy[2 * i] * fx / tz;
        gt[1] += g_xy[2 * i + 1] * fy / tz;
        gt[2] += -g_xy[2 * i] * fx * t[0] / (tz * tz) - g_xy[2 * i + 1] * fy * t[1] / (tz * tz);
        gt[2] += GJ[0] * (-fx / (tz * tz)) + GJ[4] * (-fy / (tz * tz));
        if (clx) gt[2] += GJ[2] * (fx * txc / tz) / (tz * tz);         /* J02 = -fx L / tz */
        else { gt[0] += GJ[2] * (-fx / (tz * tz)); gt[2] += GJ[2] * (2.0 * fx * t[0] / (tz * tz * tz)); }
        if (cly) gt[2] += GJ[5] * (fy * tyc / tz) / (tz * tz);
        else { gt[1] += GJ[5] * (-fy / (tz * tz)); gt[2] += GJ[5] * (2.0 * fy * t[1] / (tz * tz * tz)); }
        for (int b = 0; b < 3; ++b) gm[3 * (size_t)i + b] += V[b] * gt[0] + V[4 + b] * gt[1] + V[8 + b] * gt[2];

        /* --- S3 = R diag(s^2) R^T --- */
        double RtGR[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k)
                    for (int l = 0; l < 3; ++l) acc += R[3 * k + a] * G3[3 * k + l] * R[3 * l + b];
                RtGR[3 * a + b] = acc;
            }
        for (int a = 0; a < 3; ++a) {
            double g_s = 2.0 * s[a] * RtGR[4 * a];
            gs[3 * (size_t)i + a] += raw ? g_s * s[a] : g_s;
        }
        double GR[9]; /* dL/dR = (G3 + G3^T) R D */
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += (G3[3 * a + k] + G3[3 * k + a]) * R[3 * k + b];
                GR[3 * a + b] = acc * s[b] * s[b];
            }
        /* partial derivatives of R entries w.r.t. (w, x, y, z) */
        double dR[9][4] = {
            { 0, 0, -4 * y, -4 * z },  { -2 * z, 2 * y, 2 * x, -2 * w }, { 2 * y, 2 * z, 2 * w, 2 * x },
            { 2 * z, 2 * y, 2 * x, 2 * w }, { 0, -4 * x, 0, -4 * z },   { -2 * x, -2 * w, 2 * z, 2 * y },
            { -2 * y, 2 * z, -2 * w, 2 * x }, { 2 * x, 2 * w, 2 * z, 2 * y }, { 0, -4 * x, -4 * y, 0 } };
        double gqn[4] = { 0, 0, 0, 0 };
        for (int e = 0; e < 9; ++e)
            for (int k = 0; k < 4; ++k) gqn[k] += GR[e] * dR[e][k];
        double qh[4] = { w, x, y, z };
        double dot = gqn[0] * qh[0] + gqn[1] * qh[1] + gqn[2] * qh[2] + gqn[3] * qh[3];
        for (int k = 0; k < 4; ++k) gq[4 * (size_t)i + k] += (gqn[k] - qh[k] * dot) / qn;

        /* --- opacity --- */
        double o = rec[F_O];
        go[i] += raw ? g_o[i] * o * (1.0 - o) : g_o[i];

        /* --- colour from SH --- */
        double v[3] = { mean[0] - cam[CAM_POS], mean[1] - cam[CAM_POS + 1], mean[2] - cam[CAM_POS + 2] };
        double vn = sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
        double d[3] = { v[0] / vn, v[1] / vn, v[2] / vn };
        double Y[16];
        orc_sh_basis(deg, d, Y);
        int cm = (int)rec[F_CLAMP];
        double gc[3];
        for (int ch = 0; ch < 3; ++ch) gc[ch] = (cm & (1 << ch)) ? 0.0 : g_rgb[3 * (size_t)i + ch];
        for (int k = 0; k < K; ++k)
            for (int ch = 0; ch < 3; ++ch) gsh[(size_t)K * 3 * i + 3 * k + ch] += Y[k] * gc[ch];
        if (deg > 0) {
            /* gradient of Y_k(u/|u|) at u = d by central differences (the basis
             * is evaluated in spherical form, so it is differentiated numerically) */
            double gd[3] = { 0, 0, 0 };
            const double h = 1e-6;
            for (int j = 0; j < 3; ++j) {
                double up[3] = { d[0], d[1], d[2] }, dn[3] = { d[0], d[1], d[2] };
                up[j] += h; dn[j] -= h;
                double nu = sqrt(up[0] * up[0] + up[1] * up[1] + up[2] * up[2]);
                double nd = sqrt(dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2]);
                for (int c = 0; c < 3; ++c) { up[c] /= nu; dn[c] /= nd; }
                double Yu[16], Yd[16];
                orc_sh_basis(deg, up, Yu);
                orc_sh_basis(deg, dn, Yd);
                double acc = 0.0;
                for (int k = 1; k < K; ++k)
                    for (int ch = 0; ch < 3; ++ch)
                        acc += shi[3 * k + ch] * gc[ch] * (Yu[k] - Yd[k]) / (2.0 * h);
                gd[j] = acc;
            }
            for (int j = 0; j < 3; ++j) gm[3 * (size_t)i + j] += gd[j] / vn;
        }
    }
}
