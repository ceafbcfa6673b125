/* stp_oracle.c -- FP64 CPU oracle of StopThePop's sorted splatting renderer.
 *
 * TEST INFRASTRUCTURE ONLY (see stp_oracle.h). Plain, slow, double-precision code that
 * follows the paper's definitions and algorithm steps in order, so that a reader can hold
 * it against the paper:
 *   Radl, Steiner et al., StopThePop, TOG 43(4) 2024, arXiv 2402.00525.
 * It is compiled by oracle/build.py and shares nothing with the CUDA library.
 *
 * Section map:
 *   Sec. 2.1 (3DGS preliminaries)       : Gaussian, covariance, EWA splat, alpha blending
 *   Eq. "dopt" and Appendix A           : per-ray depth t_opt and Sigma^-1 = R S^-2 R^T
 *   Sec. 3.2                            : S^-1 bounded by 1e3; full per-ray sort (FULL mode)
 *   Sec. 3.3                            : per-ray resort window (WINDOW mode); sort error delta
 *   Sec. 3.4 "Tile-based culling"       : exact culling with Algorithm 1 (appendix B.1)
 *   Sec. 3.4 "Tile-depth adjustment"    : key depth is t_opt on the ray through x_hat
 *   Appendix B.2                        : opacity-aware bound t_O = sqrt(2 ln(alpha/eps_O))
 *   Sec. 3.4 "Hierarchically sorted rendering": tail / mid / head queues (HIER mode)
 *   Sec. 3.5                            : backward pass front to back with C - C_i, T_N / T_i
 *   Sec. 4.1 "Depth Evaluation"           : volumetric depth with phi = t_opt
 *
 * Readings where the paper is silent or ambiguous are listed in the repository's design
 * notes; the ones that shape code here are restated at the place they apply.
 */
#include "stp_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define HEADMAX 256
#define TAILMAX 1024
#define MIDMAX 256

/* counters (index meaning mirrored in oracle.py) */
enum {
    CNT_VISIBLE = 0, CNT_ENTRIES, CNT_EVAL_S, CNT_SURV_S, CNT_EVAL_Q, CNT_SURV_Q,
    CNT_EVAL_P, CNT_HEAD_INS, CNT_BLENDS, CNT_CANDIDATES, CNT_DONE_PIX, CNT_N
};

/* ------------------------------------------------------------------ small helpers */
static double clampd(double x, double lo, double hi) { return x < lo ? lo : (x > hi ? hi : x); }
static double relgap(double a, double b)
{
    double m = fmax(fmax(fabs(a), fabs(b)), 1e-30);
    return fabs(a - b) / m;
}
static void transpose3(const double* A, double* T)
{
    double r[9];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) r[3 * j + i] = A[3 * i + j];
    memcpy(T, r, sizeof r);
}
static void matvec3(const double* A, const double* x, double* y)
{
    double r[3];
    for (int i = 0; i < 3; i++) r[i] = A[3 * i] * x[0] + A[3 * i + 1] * x[1] + A[3 * i + 2] * x[2];
    memcpy(y, r, sizeof r);
}

/* rotation of the normalised quaternion q = (w, x, y, z) */
static void quat_to_rot(const double q[4], double R[9])
{
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}
static void normalise_quat(const double qin[4], double q[4], double* len)
{
    double l = sqrt(qin[0] * qin[0] + qin[1] * qin[1] + qin[2] * qin[2] + qin[3] * qin[3]);
    *len = l;
    for (int i = 0; i < 4; i++) q[i] = qin[i] / l;
}

/* ------------------------------------------------------------------ Gaussian covariance
 * Sec. 2.1: Sigma = R S S^T R^T with S = diag(s), s = exp(log_scale).                     */
void orc_sigma(const double quat[4], const double log_scale[3], double sigma[9])
{
    double q[4], l, R[9];
    normalise_quat(quat, q, &l);
    quat_to_rot(q, R);
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += R[3 * i + k] * exp(2 * log_scale[k]) * R[3 * j + k];
            sigma[3 * i + j] = s;
        }
}

/* Appendix A: Sigma^-1 = R S^-1 S^-1 R^T; Sec. 3.2: entries of S^-1 bounded by 1e3.      */
void orc_sigma_inv(const double quat[4], const double log_scale[3], double inv_scale_max,
                   double sinv[9])
{
    double q[4], l, R[9], w[3];
    normalise_quat(quat, q, &l);
    quat_to_rot(q, R);
    for (int k = 0; k < 3; k++) {
        double si = fmin(exp(-log_scale[k]), inv_scale_max);
        w[k] = si * si;
    }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += R[3 * i + k] * w[k] * R[3 * j + k];
            sinv[3 * i + j] = s;
        }
}

/* ------------------------------------------------------------------ per-ray depth
 * Eq. "dopt": t_opt = d^T Sigma^-1 (mu - o) / (d^T Sigma^-1 d), the maximiser of the 3D
 * Gaussian along r(t) = o + t d.                                                           */
double orc_t_opt(const double d[3], const double o[3], const double mu[3], const double sinv[9])
{
    double m[3] = {mu[0] - o[0], mu[1] - o[1], mu[2] - o[2]};
    double sm[3], sd[3];
    matvec3(sinv, m, sm);
    matvec3(sinv, d, sd);
    double num = d[0] * sm[0] + d[1] * sm[1] + d[2] * sm[2];
    double den = d[0] * sd[0] + d[1] * sd[1] + d[2] * sd[2];
    return num / den;
}

/* ------------------------------------------------------------------ Algorithm 1
 * Maximum of a 2D Gaussian (mean mu2, inverse covariance conic = (A00, A01, A11)) inside
 * the axis-aligned box [x0, x1] x [y0, y1] (box = {x0, x1, y0, y1}).                      */
void orc_alg1(const double mu2[2], const double conic[3], const double box[4], double xhat[2])
{
    const double x0 = box[0], x1 = box[1], y0 = box[2], y1 = box[3];
    if (mu2[0] >= x0 && mu2[0] <= x1 && mu2[1] >= y0 && mu2[1] <= y1) {
        xhat[0] = mu2[0];
        xhat[1] = mu2[1];
        return;
    }
    /* corner closest to mu2 (per axis; on a tie within the range the lower bound)       */
    double px = mu2[0] < x0 ? x0 : (mu2[0] > x1 ? x1 : (mu2[0] - x0 <= x1 - mu2[0] ? x0 : x1));
    double py = mu2[1] < y0 ? y0 : (mu2[1] > y1 ? y1 : (mu2[1] - y0 <= y1 - mu2[1] ? y0 : y1));
    /* vectors to the next corners in x and y direction                                   */
    double dxv[2] = {(px == x0 ? x1 : x0) - px, 0.0};
    double dyv[2] = {0.0, (py == y0 ? y1 : y0) - py};
    double diff[2] = {mu2[0] - px, mu2[1] - py};
    double tx = 0.0, ty = 0.0;
    /* Sigma2^-1 times a vector                                                          */
#define AV(v, out) do { out[0] = conic[0] * v[0] + conic[1] * v[1]; \
                        out[1] = conic[1] * v[0] + conic[2] * v[1]; } while (0)
    if (mu2[0] < x0 || mu2[0] > x1) {
        double ad[2], ay[2];
        AV(diff, ad);
        AV(dyv, ay);
        double num = dyv[0] * ad[0] + dyv[1] * ad[1];
        double den = dyv[0] * ay[0] + dyv[1] * ay[1];
        ty = den > 0 ? clampd(num / den, 0.0, 1.0) : 0.0;
    }
    if (mu2[1] < y0 || mu2[1] > y1) {
        double ad[2], ax[2];
        AV(diff, ad);
        AV(dxv, ax);
        double num = dxv[0] * ad[0] + dxv[1] * ad[1];
        double den = dxv[0] * ax[0] + dxv[1] * ax[1];
        tx = den > 0 ? clampd(num / den, 0.0, 1.0) : 0.0;
    }
#undef AV
    xhat[0] = px + tx * dxv[0] + ty * dyv[0];
    xhat[1] = py + tx * dxv[1] + ty * dyv[1];
}

/* Appendix B.2: t_O = sqrt(2 log(alpha / eps_O)).                                          */
double orc_t_o(double opacity, double eps_o) { return sqrt(2.0 * log(opacity / eps_o)); }

/* ------------------------------------------------------------------ real SH basis
 * Real spherical harmonics up to degree 3 (Condon-Shortley phase), as polynomials of the
 * unit direction (x, y, z). Order: l = 0; l = 1: m = -1, 0, 1; ...; l = 3: m = -3..3.
 * Constants are the closed-form normalisations sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) (x sqrt 2
 * for m != 0), written out per polynomial. grad (optional, 16x3) is the gradient of each
 * polynomial with respect to (x, y, z).                                                    */
static void sh_basis_grad(const double dir[3], double y[16], double* grad)
{
    const double PI = 3.14159265358979323846;
    const double k0 = 0.5 * sqrt(1.0 / PI);
    const double k1 = sqrt(3.0 / (4.0 * PI));
    const double k2a = sqrt(15.0 / (4.0 * PI)), k2b = sqrt(5.0 / (16.0 * PI)),
                 k2c = sqrt(15.0 / (16.0 * PI));
    const double k3a = sqrt(35.0 / (32.0 * PI)), k3b = sqrt(105.0 / (4.0 * PI)),
                 k3c = sqrt(21.0 / (32.0 * PI)), k3d = sqrt(7.0 / (16.0 * PI)),
                 k3e = sqrt(105.0 / (16.0 * PI));
    double x = dir[0], Y = dir[1], z = dir[2];
    double g[16][3];
    memset(g, 0, sizeof g);
    y[0] = k0;
    y[1] = -k1 * Y;                 g[1][1] = -k1;
    y[2] = k1 * z;                  g[2][2] = k1;
    y[3] = -k1 * x;                 g[3][0] = -k1;
    y[4] = k2a * x * Y;             g[4][0] = k2a * Y;  g[4][1] = k2a * x;
    y[5] = -k2a * Y * z;            g[5][1] = -k2a * z; g[5][2] = -k2a * Y;
    y[6] = k2b * (2 * z * z - x * x - Y * Y);
    g[6][0] = -2 * k2b * x; g[6][1] = -2 * k2b * Y; g[6][2] = 4 * k2b * z;
    y[7] = -k2a * x * z;            g[7][0] = -k2a * z; g[7][2] = -k2a * x;
    y[8] = k2c * (x * x - Y * Y);   g[8][0] = 2 * k2c * x; g[8][1] = -2 * k2c * Y;
    y[9] = -k3a * Y * (3 * x * x - Y * Y);
    g[9][0] = -k3a * 6 * x * Y; g[9][1] = -k3a * (3 * x * x - 3 * Y * Y);
    y[10] = k3b * x * Y * z;
    g[10][0] = k3b * Y * z; g[10][1] = k3b * x * z; g[10][2] = k3b * x * Y;
    y[11] = -k3c * Y * (4 * z * z - x * x - Y * Y);
    g[11][0] = -k3c * Y * (-2 * x); g[11][1] = -k3c * (4 * z * z - x * x - 3 * Y * Y);
    g[11][2] = -k3c * Y * 8 * z;
    y[12] = k3d * z * (2 * z * z - 3 * x * x - 3 * Y * Y);
    g[12][0] = k3d * z * (-6 * x); g[12][1] = k3d * z * (-6 * Y);
    g[12][2] = k3d * (6 * z * z - 3 * x * x - 3 * Y * Y);
    y[13] = -k3c * x * (4 * z * z - x * x - Y * Y);
    g[13][0] = -k3c * (4 * z * z - 3 * x * x - Y * Y); g[13][1] = -k3c * x * (-2 * Y);
    g[13][2] = -k3c * x * 8 * z;
    y[14] = k3e * z * (x * x - Y * Y);
    g[14][0] = k3e * z * 2 * x; g[14][1] = -k3e * z * 2 * Y; g[14][2] = k3e * (x * x - Y * Y);
    y[15] = -k3a * x * (x * x - 3 * Y * Y);
    g[15][0] = -k3a * (3 * x * x - 3 * Y * Y); g[15][1] = -k3a * x * (-6 * Y);
    if (grad) memcpy(grad, g, sizeof g);
}
void orc_sh_basis(const double dir[3], double y[16]) { sh_basis_grad(dir, y, NULL); }

/* ------------------------------------------------------------------ EWA projection
 * Sec. 2.1 (kept untouched from 3DGS, Sec. 3.4): the first-order (Jacobian) approximation
 * of the perspective projection at the camera-space mean, with the 3DGS frustum clamp of
 * the Jacobian and the 3DGS low-pass dilation (readings: both kept, both parameters).    */
typedef struct {
    int visible;
    double mu[3], p[3];
    double qn[4], qlen, Rq[9], s[3];
    double sigma[9];
    double J[6], Tm[6];          /* J (2x3), Tm = J R_c (2x3)                              */
    int clampx, clampy;
    double cov2[3], det;
    double mean2[2], conic[3];
    double opacity;
    double u[3], ulen, dir[3];   /* mu - o and its direction (SH view direction)          */
    double raw[3], color[3];
    double w[3];                 /* clamped S^-2 entries                                   */
    double sinv[9], v[3];
    double radius;
    int rect[4];                 /* tiles [x0, x1] x [y0, y1] inclusive; x1 < x0 if empty  */
    int ntiles;
    double margin;               /* min relative margin of this Gaussian's own decisions  */
    int invalid;                 /* inputs outside the method's domain: dropped, counted  */
} grec;

static void project_core(const orc_camera* cam, const orc_params* prm, const double p[3],
                         const double sigma[9], double mean2[2], double cov2[3], double J[6],
                         double Tm[6], int* clx, int* cly)
{
    double limx = prm->frustum_clamp * 0.5 * cam->width / cam->fx;
    double limy = prm->frustum_clamp * 0.5 * cam->height / cam->fy;
    double ux = p[0] / p[2], uy = p[1] / p[2];
    double cx = clampd(ux, -limx, limx), cy = clampd(uy, -limy, limy);
    if (clx) *clx = (cx != ux);
    if (cly) *cly = (cy != uy);
    J[0] = cam->fx / p[2]; J[1] = 0.0;            J[2] = -cam->fx * cx / p[2];
    J[3] = 0.0;            J[4] = cam->fy / p[2]; J[5] = -cam->fy * cy / p[2];
    /* Tm = J R_c */
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += J[3 * r + k] * cam->R[3 * k + c];
            Tm[3 * r + c] = s;
        }
    /* Sigma2 = Tm Sigma Tm^T + dilation I */
    double M[6];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 3; c++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += Tm[3 * r + k] * sigma[3 * k + c];
            M[3 * r + c] = s;
        }
    double S2[4];
    for (int r = 0; r < 2; r++)
        for (int c = 0; c < 2; c++) {
            double s = 0;
            for (int k = 0; k < 3; k++) s += M[3 * r + k] * Tm[3 * c + k];
            S2[2 * r + c] = s;
        }
    cov2[0] = S2[0] + prm->dilation;
    cov2[1] = 0.5 * (S2[1] + S2[2]);
    cov2[2] = S2[3] + prm->dilation;
    mean2[0] = cam->fx * ux + cam->cx;
    mean2[1] = cam->fy * uy + cam->cy;
}

void orc_project(const orc_camera* cam, const orc_params* prm, const double mu[3],
                 const double sigma[9], double mean2[2], double cov2[3], double jac[6])
{
    double p[3], Tm[6];
    matvec3(cam->R, mu, p);
    for (int i = 0; i < 3; i++) p[i] += cam->t[i];
    project_core(cam, prm, p, sigma, mean2, cov2, jac, Tm, NULL, NULL);
}

/* ------------------------------------------------------------------ context */
typedef struct { double t; int id; } entry;
typedef struct { double t; int id; double m; } near_entry;
typedef struct {
    int selected;
    entry* e; int n, cap;
    near_entry* nr; int nn, ncap;
    double pre_margin;          /* whole-tile margin from Gaussian-level decisions       */
    double *bm_d, *bm_c;        /* per-batch margins, nb + 1 entries                       */
} tlist;

typedef struct { int id; double a, t, T; } brec;
typedef struct { brec* r; int n, cap; } blist;

typedef struct {
    const orc_params* prm;
    orc_camera cam;
    orc_params P;
    double o[3], Rt[9];
    int64_t n;
    grec* g;
    int txn, tyn, ntiles;
    tlist* tl;
    int32_t* sel; int nsel;
    const double* syn_t; double syn_alpha; const int32_t* syn_keep;
    /* outputs of the last render */
    double *C, *Z, *T;          /* per pixel (FP64 copies kept for the adjoint)           */
    blist* bl;                  /* per pixel blend records                                 */
} ctx;

typedef struct { double t; int id; double a; } hent;
typedef struct {
    int pix, done;
    double x, y;                /* pixel centre                                            */
    double T, C[3], Z;
    double dmin, cmin;
    int nb; uint64_t h;
    int has_last; double last_t, delta;
    hent head[HEADMAX + 1]; int nh;
    int batch, sat_batch;       /* HIER batch being processed (-1: drain or flat order) and
                                   the one during which the ray terminated (-2: never)    */
} pstate;

typedef struct {                /* per-render output sinks                                */
    double *rgb, *depth, *tfinal, *dmargin, *cmargin, *delta;
    int32_t* nblend; uint64_t* hash; int32_t* seq; int max_seq;
    int32_t* satb;              /* per pixel: pstate.sat_batch                             */
} sinks;

static void cam_ray(const ctx* c, double x, double y, double d[3])
{
    double dc[3] = {(x - c->cam.cx) / c->cam.fx, (y - c->cam.cy) / c->cam.fy, 1.0};
    matvec3(c->Rt, dc, d);
    double l = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    d[0] /= l; d[1] /= l; d[2] /= l;
}

static double gauss2(const grec* g, double x, double y)
{
    double dx = x - g->mean2[0], dy = y - g->mean2[1];
    double q = g->conic[0] * dx * dx + 2.0 * g->conic[1] * dx * dy + g->conic[2] * dy * dy;
    return exp(-0.5 * q);
}

/* box of the pixel centres of the s x s block at pixel origin (ox, oy), clipped to the
 * image; returns 0 if the block has no pixel inside the image.                            */
static int make_box(const ctx* c, int ox, int oy, int s, double box[4])
{
    if (ox >= c->cam.width || oy >= c->cam.height) return 0;
    int xe = ox + s - 1, ye = oy + s - 1;
    if (xe > c->cam.width - 1) xe = c->cam.width - 1;
    if (ye > c->cam.height - 1) ye = c->cam.height - 1;
    box[0] = ox + 0.5; box[1] = xe + 0.5; box[2] = oy + 0.5; box[3] = ye + 0.5;
    return 1;
}

/* ------------------------------------------------------------------ preprocess */
/* The method is defined for finite parameters and a rotation quaternion of non-zero length.
 * A Gaussian with a non-finite mean, log-scale, quaternion component, opacity logit or SH
 * coefficient, or with a quaternion whose squared length is below 1e-20, is invalid: it is
 * dropped before any other step (it covers no pixel) and counted (reading: the paper does
 * not discuss such inputs).                                                               */
static int gaussian_valid(const orc_scene* sc, int64_t i, int sh_degree)
{
    double q2 = 0.0;
    for (int k = 0; k < 3; k++)
        if (!isfinite(sc->means[3 * i + k]) || !isfinite(sc->log_scales[3 * i + k])) return 0;
    for (int k = 0; k < 4; k++) {
        double q = sc->quats[4 * i + k];
        if (!isfinite(q)) return 0;
        q2 += q * q;
    }
    if (!(q2 >= 1e-20) || !isfinite(sc->logits[i])) return 0;
    int K = (sh_degree + 1) * (sh_degree + 1);
    for (int j = 0; j < 3 * K; j++)
        if (!isfinite(sc->sh[i * 3 * K + j])) return 0;
    return 1;
}

static void preprocess_one(ctx* c, const orc_scene* sc, int64_t i)
{
    grec* g = &c->g[i];
    const orc_params* P = &c->P;
    memset(g, 0, sizeof *g);
    g->margin = INFINITY;
    if (!gaussian_valid(sc, i, P->sh_degree)) {
        g->invalid = 1;
        g->rect[2] = -1; g->rect[3] = -1;
        return;
    }
    for (int k = 0; k < 3; k++) g->mu[k] = sc->means[3 * i + k];
    matvec3(c->cam.R, g->mu, g->p);
    for (int k = 0; k < 3; k++) g->p[k] += c->cam.t[k];
    g->rect[0] = 0; g->rect[2] = -1; g->rect[1] = 0; g->rect[3] = -1;
    /* near plane (3DGS convention, parameter znear)                                      */
    g->margin = fmin(g->margin, relgap(g->p[2], P->znear));
    if (!(g->p[2] > 0.25 * P->znear)) return;      /* far behind the near plane: nothing */
    double qin[4], ls[3];
    for (int k = 0; k < 4; k++) qin[k] = sc->quats[4 * i + k];
    for (int k = 0; k < 3; k++) ls[k] = sc->log_scales[3 * i + k];
    normalise_quat(qin, g->qn, &g->qlen);
    quat_to_rot(g->qn, g->Rq);
    for (int k = 0; k < 3; k++) g->s[k] = exp(ls[k]);
    orc_sigma(qin, ls, g->sigma);
    project_core(&c->cam, P, g->p, g->sigma, g->mean2, g->cov2, g->J, g->Tm, &g->clampx, &g->clampy);
    g->det = g->cov2[0] * g->cov2[2] - g->cov2[1] * g->cov2[1];
    if (!(g->det > 0)) return;
    g->conic[0] = g->cov2[2] / g->det;
    g->conic[1] = -g->cov2[1] / g->det;
    g->conic[2] = g->cov2[0] / g->det;
    g->opacity = 1.0 / (1.0 + exp(-sc->logits[i]));
    g->margin = fmin(g->margin, fabs(g->opacity / P->eps_o - 1.0));
    /* colour from SH with the direction camera -> mean (Appendix B.4)                   */
    for (int k = 0; k < 3; k++) g->u[k] = g->mu[k] - c->o[k];
    g->ulen = sqrt(g->u[0] * g->u[0] + g->u[1] * g->u[1] + g->u[2] * g->u[2]);
    for (int k = 0; k < 3; k++) g->dir[k] = g->u[k] / g->ulen;
    double Y[16];
    orc_sh_basis(g->dir, Y);
    int K = (P->sh_degree + 1) * (P->sh_degree + 1);
    for (int ch = 0; ch < 3; ch++) {
        double s = 0.5;
        for (int j = 0; j < K; j++) s += Y[j] * sc->sh[(i * K + j) * 3 + ch];
        g->raw[ch] = s;
        g->color[ch] = s > 0 ? s : 0.0;
    }
    /* Sigma^-1 with the S^-1 clamp (Sec. 3.2), v = Sigma^-1 (mu - o) (Appendix B.4)       */
    for (int k = 0; k < 3; k++) {
        double si = fmin(exp(-ls[k]), P->inv_scale_max);
        g->w[k] = si * si;
    }
    orc_sigma_inv(qin, ls, P->inv_scale_max, g->sinv);
    matvec3(g->sinv, g->u, g->v);
    /* opacity-aware radius (Appendix B.2): t_O sqrt(lambda_max), then the tile rectangle of
     * every tile that holds a pixel centre within [mean2 - r, mean2 + r], r = ceil(.)    */
    double tO = g->opacity > P->eps_o ? orc_t_o(g->opacity, P->eps_o) : 0.0;
    double mid = 0.5 * (g->cov2[0] + g->cov2[2]);
    double lam = mid + sqrt(fmax(0.0, mid * mid - g->det));
    g->radius = tO * sqrt(lam);
    double r = ceil(g->radius);
    int tx0 = (int)ceil((g->mean2[0] - r - 15.5) / 16.0), tx1 = (int)floor((g->mean2[0] + r - 0.5) / 16.0);
    int ty0 = (int)ceil((g->mean2[1] - r - 15.5) / 16.0), ty1 = (int)floor((g->mean2[1] + r - 0.5) / 16.0);
    if (tx0 < 0) tx0 = 0;
    if (ty0 < 0) ty0 = 0;
    if (tx1 > c->txn - 1) tx1 = c->txn - 1;
    if (ty1 > c->tyn - 1) ty1 = c->tyn - 1;
    g->rect[0] = tx0; g->rect[1] = ty0; g->rect[2] = tx1; g->rect[3] = ty1;
    g->visible = (g->p[2] > P->znear) && (g->opacity >= P->eps_o);
}

static void tl_push(tlist* L, double t, int id)
{
    if (L->n == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 16;
        L->e = (entry*)realloc(L->e, (size_t)L->cap * sizeof(entry));
    }
    L->e[L->n].t = t;
    L->e[L->n].id = id;
    L->n++;
}
static void tl_push_near(tlist* L, double t, int id, double m)
{
    if (L->nn == L->ncap) {
        L->ncap = L->ncap ? 2 * L->ncap : 8;
        L->nr = (near_entry*)realloc(L->nr, (size_t)L->ncap * sizeof(near_entry));
    }
    L->nr[L->nn].t = t; L->nr[L->nn].id = id; L->nr[L->nn].m = m;
    L->nn++;
}
static int cmp_entry(const void* a, const void* b)
{
    const entry *x = (const entry*)a, *y = (const entry*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->id > y->id) - (x->id < y->id);
}

/* depth of Gaussian g on the ray through the pixel-space point (x, y)                    */
static double depth_at(const ctx* c, const grec* g, double x, double y)
{
    double d[3];
    cam_ray(c, x, y, d);
    return orc_t_opt(d, c->o, g->mu, g->sinv);
}

/* Per-batch decision margins of a sorted list of L->n entries (allocated here): bm_d[b] is
 * the depth gap at the boundary after batch b (which 32 entries load together, Sec. 3.4),
 * bm_c[b] the smallest cull margin of a near-threshold entry whose key falls into batch b
 * (b = nb: after the list). Only near entries with key t < key_cut belong to the list.     */
static void batch_margins(tlist* L, double key_cut)
{
    int nb = (L->n + 31) / 32;
    L->bm_d = (double*)malloc((size_t)(nb + 1) * sizeof(double));
    L->bm_c = (double*)malloc((size_t)(nb + 1) * sizeof(double));
    for (int b = 0; b <= nb; b++) {
        L->bm_d[b] = INFINITY;
        L->bm_c[b] = INFINITY;
    }
    for (int b = 0; b + 1 < nb; b++) L->bm_d[b] = relgap(L->e[32 * b + 31].t, L->e[32 * b + 32].t);
    for (int k = 0; k < L->nn; k++) {
        if (!(L->nr[k].t < key_cut)) continue;
        int lo = 0, hi = L->n;
        entry key = {L->nr[k].t, L->nr[k].id};
        while (lo < hi) {
            int md = (lo + hi) / 2;
            if (cmp_entry(&L->e[md], &key) < 0) lo = md + 1; else hi = md;
        }
        int b = lo / 32;
        if (b > nb) b = nb;
        L->bm_c[b] = fmin(L->bm_c[b], L->nr[k].m);
    }
}

/* Duplicate (Sec. 3.4 "Tile-based culling", "Tile-depth adjustment"): for every visible
 * Gaussian (ascending id) and every tile of its rectangle (row major), x_hat by Algorithm 1
 * on the tile's pixel-centre box; keep iff opacity * G2(x_hat) >= eps_O; key depth is
 * t_opt on the ray through x_hat. The tile's list is then sorted by (depth, id), which is
 * what a stable global sort of (tile, depth) keys generated in id order produces.        */
static void build_lists(ctx* c)
{
    const orc_params* P = &c->P;
    for (int64_t i = 0; i < c->n; i++) {
        grec* g = &c->g[i];
        if (!(g->det > 0) || g->rect[2] < g->rect[0] || g->rect[3] < g->rect[1]) continue;
        int near_decision = g->margin < P->cull_thr;
        if (!g->visible && !near_decision) continue;
        /* expanded rectangle: tiles just outside are evaluated for their margin only    */
        for (int ty = g->rect[1] - 1; ty <= g->rect[3] + 1; ty++) {
            if (ty < 0 || ty >= c->tyn) continue;
            for (int tx = g->rect[0] - 1; tx <= g->rect[2] + 1; tx++) {
                if (tx < 0 || tx >= c->txn) continue;
                int tile = ty * c->txn + tx;
                tlist* L = &c->tl[tile];
                int in_rect = tx >= g->rect[0] && tx <= g->rect[2] && ty >= g->rect[1] && ty <= g->rect[3];
                double box[4];
                if (!make_box(c, tx * 16, ty * 16, 16, box)) continue;
                double xh[2];
                orc_alg1(g->mean2, g->conic, box, xh);
                double val = g->opacity * gauss2(g, xh[0], xh[1]);
                double m = fabs(val / P->eps_o - 1.0);
                int keep = val >= P->eps_o;
                /* flag 512: no tile-based culling (ablation D of Tab. performance_ablation):
                 * every tile of the rectangle is kept; the key depth still goes through x_hat */
                if (P->flags & 512) {
                    keep = 1;
                    m = INFINITY;
                }
                if (in_rect && g->visible && keep) g->ntiles++;
                if (!L->selected) continue;
                /* key depth: t_opt through x_hat (default); flag 4: through the tile centre
                 * (the naive per-tile depth of Sec. 3.3); flag 8: the mean's view-space depth
                 * (3DGS global depth, ablation B of Tab. performance_ablation)               */
                double t;
                if (P->flags & 8) t = g->p[2];
                else if (P->flags & 4) t = depth_at(c, g, 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3]));
                else t = depth_at(c, g, xh[0], xh[1]);
                if (near_decision && in_rect) L->pre_margin = fmin(L->pre_margin, g->margin);
                if (in_rect && g->visible && keep) tl_push(L, t, (int)i);
                if (m < P->cull_thr) tl_push_near(L, t, (int)i, m);
            }
        }
    }
    for (int tile = 0; tile < c->ntiles; tile++) {
        tlist* L = &c->tl[tile];
        if (!L->selected) continue;
        if (L->n > 1) qsort(L->e, (size_t)L->n, sizeof(entry), cmp_entry);
        batch_margins(L, INFINITY);
    }
}

/* ------------------------------------------------------------------ blending */
static const uint64_t HASH_MUL = 1099511628211ULL, HASH_INIT = 1469598103934665603ULL;

static void bl_push(blist* B, int id, double a, double t, double T)
{
    if (B->n == B->cap) {
        B->cap = B->cap ? 2 * B->cap : 16;
        B->r = (brec*)realloc(B->r, (size_t)B->cap * sizeof(brec));
    }
    B->r[B->n].id = id; B->r[B->n].a = a; B->r[B->n].t = t; B->r[B->n].T = T;
    B->n++;
}

/* Eq. "volume_desc" front to back, with the 3DGS early-out: a Gaussian that would take the
 * transmittance below t_min is not blended and the ray stops (reading). Depth accumulates
 * the volumetric depth with phi = t_opt (Sec. 4.1 "Depth Evaluation"), unnormalised.        */
static void blend(ctx* c, pstate* ps, const sinks* sk, double t, int id, double a, int64_t* cnt)
{
    if (ps->done) return;
    double Tn = ps->T * (1.0 - a);
    ps->cmin = fmin(ps->cmin, fabs(Tn / c->P.t_min - 1.0));
    if (Tn < c->P.t_min) {
        ps->done = 1;
        ps->sat_batch = ps->batch;
        cnt[CNT_DONE_PIX]++;
        return;
    }
    double col[3];
    if (c->syn_t) { col[0] = col[1] = col[2] = 0.5; }
    else for (int k = 0; k < 3; k++) col[k] = c->g[id].color[k];
    for (int k = 0; k < 3; k++) ps->C[k] += col[k] * a * ps->T;
    ps->Z += t * a * ps->T;
    if (ps->has_last && ps->last_t > t) ps->delta += ps->last_t - t;
    ps->has_last = 1;
    ps->last_t = t;
    if (c->bl && ps->pix >= 0) bl_push(&c->bl[ps->pix], id, a, t, ps->T);
    if (sk && sk->seq && ps->nb < sk->max_seq) sk->seq[(int64_t)ps->pix * sk->max_seq + ps->nb] = id;
    ps->h = ps->h * HASH_MUL + (uint64_t)(id + 1);
    ps->nb++;
    ps->T = Tn;
    cnt[CNT_BLENDS]++;
}

static void pixel_init(const ctx* c, pstate* ps, int X, int Y)
{
    memset(ps, 0, sizeof *ps);
    ps->pix = (X < c->cam.width && Y < c->cam.height) ? Y * c->cam.width + X : -1;
    ps->done = ps->pix < 0;
    ps->x = X + 0.5;
    ps->y = Y + 0.5;
    ps->T = 1.0;
    ps->dmin = INFINITY;
    ps->cmin = INFINITY;
    ps->h = HASH_INIT;
    ps->batch = -1;
    ps->sat_batch = -2;
}

static void pixel_out(const ctx* c, const pstate* ps, const sinks* sk)
{
    if (ps->pix < 0) return;
    int64_t p = ps->pix;
    if (sk->rgb) for (int k = 0; k < 3; k++) sk->rgb[3 * p + k] = ps->C[k] + ps->T * c->P.bg[k];
    if (sk->depth) sk->depth[p] = ps->Z;
    if (sk->tfinal) sk->tfinal[p] = ps->T;
    if (sk->nblend) sk->nblend[p] = ps->nb;
    if (sk->hash) sk->hash[p] = ps->h;
    if (sk->dmargin) sk->dmargin[p] = ps->dmin;
    if (sk->cmargin) sk->cmargin[p] = ps->cmin;
    if (sk->delta) sk->delta[p] = ps->delta;
    if (sk->satb) sk->satb[p] = ps->sat_batch;
    if (c->C) {
        for (int k = 0; k < 3; k++) c->C[3 * p + k] = ps->C[k];
        c->Z[p] = ps->Z;
        c->T[p] = ps->T;
    }
}

/* per-pixel alpha (Eq. "volume_desc": alpha = opacity * G2, clamped at alpha_max)        */
static double pixel_alpha(const ctx* c, int id, const pstate* ps)
{
    if (c->syn_t) return c->syn_alpha;
    const grec* g = &c->g[id];
    return fmin(c->P.alpha_max, g->opacity * gauss2(g, ps->x, ps->y));
}
static double pixel_depth(const ctx* c, int id, const pstate* ps)
{
    if (c->syn_t) return c->syn_t[id];
    return depth_at(c, &c->g[id], ps->x, ps->y);
}

/* evaluation of Gaussian `id` for a 4x4 or 2x2 box: Algorithm 1 maximum, cull against
 * eps_O, depth on the ray through x_hat (reading: the level's own x_hat, as for tiles;
 * flag 2 selects the level's centre ray instead).                                        */
static int eval_box(const ctx* c, int id, const double box[4], double* t, double* margin)
{
    if (c->syn_t) {
        *t = c->syn_t[id];
        *margin = INFINITY;
        return c->syn_keep ? c->syn_keep[id] != 0 : 1;
    }
    const grec* g = &c->g[id];
    double xh[2];
    orc_alg1(g->mean2, g->conic, box, xh);
    double val = g->opacity * gauss2(g, xh[0], xh[1]);
    *margin = fabs(val / c->P.eps_o - 1.0);
    /* flag 1024: no hierarchical culling inside Render (ablation E): every entry passes the
     * 4x4 and 2x2 levels; only the per-pixel alpha test drops Gaussians                   */
    if (c->P.flags & 1024) *margin = INFINITY;
    else if (val < c->P.eps_o) return 0;
    if (c->P.flags & 2) *t = depth_at(c, g, 0.5 * (box[0] + box[1]), 0.5 * (box[2] + box[3]));
    else *t = depth_at(c, g, xh[0], xh[1]);
    return 1;
}

/* head (per-pixel) queue: insertion after equal keys; when more than `head` entries are
 * held, the smallest is blended (Sec. 3.3: a full resorting window gives up its nearest
 * entry; reading: insert then evict; flag 1 evicts before inserting).                    */
static void head_push(ctx* c, pstate* ps, const sinks* sk, int hsize, hent e, int64_t* cnt)
{
    if (ps->done) return;
    cnt[CNT_HEAD_INS]++;
    if ((c->P.flags & 1) && ps->nh == hsize) {
        if (ps->nh >= 2) ps->dmin = fmin(ps->dmin, relgap(ps->head[0].t, ps->head[1].t));
        hent f = ps->head[0];
        memmove(&ps->head[0], &ps->head[1], (size_t)(ps->nh - 1) * sizeof(hent));
        ps->nh--;
        blend(c, ps, sk, f.t, f.id, f.a, cnt);
        if (ps->done) return;
    }
    int pos = 0;
    while (pos < ps->nh && ps->head[pos].t <= e.t) pos++;
    memmove(&ps->head[pos + 1], &ps->head[pos], (size_t)(ps->nh - pos) * sizeof(hent));
    ps->head[pos] = e;
    ps->nh++;
    if (ps->nh > hsize) {
        ps->dmin = fmin(ps->dmin, relgap(ps->head[0].t, ps->head[1].t));
        hent f = ps->head[0];
        memmove(&ps->head[0], &ps->head[1], (size_t)(ps->nh - 1) * sizeof(hent));
        ps->nh--;
        blend(c, ps, sk, f.t, f.id, f.a, cnt);
    }
}
static void head_flush(ctx* c, pstate* ps, const sinks* sk, int64_t* cnt)
{
    for (int k = 0; k < ps->nh; k++) {
        if (ps->done) break;
        if (k + 1 < ps->nh) ps->dmin = fmin(ps->dmin, relgap(ps->head[k].t, ps->head[k + 1].t));
        blend(c, ps, sk, ps->head[k].t, ps->head[k].id, ps->head[k].a, cnt);
    }
    ps->nh = 0;
}

/* ------------------------------------------------------------------ HIER schedule
 * Sec. 3.4 "Hierarchically sorted rendering", one 4x4 subtile S of a 16x16 tile (the
 * subtiles are independent). Reading of the push discipline (queue sizes TAIL=32n+32,
 * MID=4m+4, HEAD):
 *   - the tile list is consumed in batches of 32 entries; each batch is culled against S's
 *     box (Algorithm 1), gets t_opt on the ray through S's x_hat, is stably sorted and
 *     merged into the tail queue (existing entries first on equal depth); culled entries
 *     are discarded;
 *   - while the tail holds more than TAIL-32 entries, its 16 front entries are pushed to
 *     the mid level; at the end the tail is drained in chunks of at most 16;
 *   - a chunk is processed in consecutive sub-batches of 4; each 2x2 quad Q culls the
 *     sub-batch against Q's box, computes t_opt through Q's x_hat, sorts the survivors and
 *     merges them into its mid queue (existing first); when the mid queue then holds more
 *     than MID-4 entries its 4 front entries go to Q's pixels; at the end the mid queues
 *     are flushed in groups of at most 4;
 *   - each pixel evaluates alpha at its centre, drops alpha < eps_O, computes t_opt on its
 *     own ray and inserts into its head queue; overflow blends the smallest; at the end the
 *     head is blended in order.
 * Margins: every comparison whose outcome a small perturbation could flip is recorded
 * (relative depth gap at batch / pop / sub-batch boundaries and at every head eviction;
 * relative distance of each cull or alpha test to eps_O and of T to t_min), for the pixels
 * still running when it is taken.                                                          */
typedef struct {
    ctx* c;
    const sinks* sk;
    int64_t* cnt;
    pstate px[16];              /* index q*4 + p                                           */
    int qvalid[4];
    double boxS[4], boxQ[4][4];
    entry tail[TAILMAX]; int nt;
    entry mid[4][MIDMAX]; int nm[4];
} sub_state;

static void margin_S(sub_state* s, double d, double m)
{
    for (int k = 0; k < 16; k++)
        if (!s->px[k].done) {
            s->px[k].dmin = fmin(s->px[k].dmin, d);
            s->px[k].cmin = fmin(s->px[k].cmin, m);
        }
}
static void margin_Q(sub_state* s, int q, double d, double m)
{
    for (int k = 0; k < 4; k++) {
        pstate* ps = &s->px[q * 4 + k];
        if (!ps->done) {
            ps->dmin = fmin(ps->dmin, d);
            ps->cmin = fmin(ps->cmin, m);
        }
    }
}

static void stable_sort_entries(entry* a, int n)   /* insertion sort: stable            */
{
    for (int i = 1; i < n; i++) {
        entry x = a[i];
        int j = i - 1;
        while (j >= 0 && a[j].t > x.t) { a[j + 1] = a[j]; j--; }
        a[j + 1] = x;
    }
}
static void merge_into(entry* q, int* nq, const entry* nw, int nn)   /* existing first */
{
    entry out[TAILMAX];
    int i = 0, j = 0, k = 0;
    while (i < *nq && j < nn) out[k++] = (q[i].t <= nw[j].t) ? q[i++] : nw[j++];
    while (i < *nq) out[k++] = q[i++];
    while (j < nn) out[k++] = nw[j++];
    memcpy(q, out, (size_t)k * sizeof(entry));
    *nq = k;
}

static void headstage(sub_state* s, int q, const entry* el, int cnt)
{
    ctx* c = s->c;
    for (int p = 0; p < 4; p++) {
        pstate* ps = &s->px[q * 4 + p];
        for (int e = 0; e < cnt; e++) {
            if (ps->done) break;
            s->cnt[CNT_EVAL_P]++;
            double a = pixel_alpha(c, el[e].id, ps);
            if (!c->syn_t) ps->cmin = fmin(ps->cmin, fabs(a / c->P.eps_o - 1.0));
            if (a < c->P.eps_o) continue;
            hent h = {pixel_depth(c, el[e].id, ps), el[e].id, a};
            head_push(c, ps, s->sk, c->P.head, h, s->cnt);
        }
    }
}

static int pop_mid(sub_state* s, int q, int cnt, entry* out)
{
    entry* m = s->mid[q];
    for (int k = 1; k < cnt; k++) margin_Q(s, q, relgap(m[k - 1].t, m[k].t), INFINITY);
    if (cnt < s->nm[q]) margin_Q(s, q, relgap(m[cnt - 1].t, m[cnt].t), INFINITY);
    memcpy(out, m, (size_t)cnt * sizeof(entry));
    memmove(m, m + cnt, (size_t)(s->nm[q] - cnt) * sizeof(entry));
    s->nm[q] -= cnt;
    return cnt;
}

static void midstage(sub_state* s, const entry* chunk, int cn)
{
    ctx* c = s->c;
    for (int j0 = 0; j0 < cn; j0 += 4) {
        int m = cn - j0 < 4 ? cn - j0 : 4;
        for (int q = 0; q < 4; q++) {
            if (!s->qvalid[q]) continue;
            entry nw[4];
            int nn = 0;
            for (int e = 0; e < m; e++) {
                int id = chunk[j0 + e].id;
                double t, mg;
                s->cnt[CNT_EVAL_Q]++;
                int keep = eval_box(c, id, s->boxQ[q], &t, &mg);
                margin_Q(s, q, INFINITY, mg);
                if (!keep) continue;
                s->cnt[CNT_SURV_Q]++;
                nw[nn].t = t;
                nw[nn].id = id;
                nn++;
            }
            stable_sort_entries(nw, nn);
            merge_into(s->mid[q], &s->nm[q], nw, nn);
            if (s->nm[q] > c->P.mid - 4) {
                entry out[4];
                int k = pop_mid(s, q, 4, out);
                headstage(s, q, out, k);
            }
        }
    }
}

static int pop_tail(sub_state* s, int cnt, entry* out)
{
    for (int k = 4; k < cnt; k += 4) margin_S(s, relgap(s->tail[k - 1].t, s->tail[k].t), INFINITY);
    if (cnt < s->nt) margin_S(s, relgap(s->tail[cnt - 1].t, s->tail[cnt].t), INFINITY);
    memcpy(out, s->tail, (size_t)cnt * sizeof(entry));
    memmove(s->tail, s->tail + cnt, (size_t)(s->nt - cnt) * sizeof(entry));
    s->nt -= cnt;
    return cnt;
}

static void hier_subtile(ctx* c, const sinks* sk, int tile, int S, int64_t* cnt)
{
    const orc_params* P = &c->P;
    int tx = tile % c->txn, ty = tile / c->txn;
    int ox = tx * 16 + (S % 4) * 4, oy = ty * 16 + (S / 4) * 4;
    sub_state* s = (sub_state*)calloc(1, sizeof(sub_state));
    s->c = c; s->sk = sk; s->cnt = cnt;
    if (!make_box(c, ox, oy, 4, s->boxS)) { free(s); return; }
    for (int q = 0; q < 4; q++) {
        int qx = ox + (q % 2) * 2, qy = oy + (q / 2) * 2;
        s->qvalid[q] = make_box(c, qx, qy, 2, s->boxQ[q]);
        for (int p = 0; p < 4; p++) pixel_init(c, &s->px[q * 4 + p], qx + p % 2, qy + p / 2);
    }
    tlist* L = &c->tl[tile];
    margin_S(s, INFINITY, L->pre_margin);
    int nb = (L->n + 31) / 32;
    for (int b = 0; b < nb; b++) {
        for (int k = 0; k < 16; k++) s->px[k].batch = b;
        margin_S(s, L->bm_d[b], L->bm_c[b]);
        entry nw[32];
        int nn = 0;
        int end = L->n < 32 * b + 32 ? L->n : 32 * b + 32;
        for (int j = 32 * b; j < end; j++) {
            int id = L->e[j].id;
            double t, mg;
            cnt[CNT_EVAL_S]++;
            int keep = eval_box(c, id, s->boxS, &t, &mg);
            margin_S(s, INFINITY, mg);
            if (!keep) continue;
            cnt[CNT_SURV_S]++;
            nw[nn].t = t;
            nw[nn].id = id;
            nn++;
        }
        stable_sort_entries(nw, nn);
        merge_into(s->tail, &s->nt, nw, nn);
        while (s->nt > P->tail - 32) {
            entry ch[16];
            int k = pop_tail(s, 16, ch);
            midstage(s, ch, k);
        }
    }
    for (int k = 0; k < 16; k++) s->px[k].batch = -1;        /* the drain */
    margin_S(s, INFINITY, L->bm_c[nb]);
    while (s->nt > 0) {
        entry ch[16];
        int k = pop_tail(s, s->nt < 16 ? s->nt : 16, ch);
        midstage(s, ch, k);
    }
    for (int q = 0; q < 4; q++) {
        if (!s->qvalid[q]) continue;
        while (s->nm[q] > 0) {
            entry out[4];
            int k = pop_mid(s, q, s->nm[q] < 4 ? s->nm[q] : 4, out);
            headstage(s, q, out, k);
        }
    }
    for (int k = 0; k < 16; k++) {
        head_flush(c, &s->px[k], sk, cnt);
        pixel_out(c, &s->px[k], sk);
    }
    free(s);
}

/* ------------------------------------------------------------------ other orderings  */
typedef struct { double t; int pos, id; double a; } fent;
static int cmp_fent(const void* a, const void* b)
{
    const fent *x = (const fent*)a, *y = (const fent*)b;
    if (x->t < y->t) return -1;
    if (x->t > y->t) return 1;
    return (x->pos > y->pos) - (x->pos < y->pos);
}

/* FULL (Sec. 3.2): every list entry with alpha >= eps_O, stably sorted by the pixel's own
 * t_opt. GLOBAL: blended in tile-list order. WINDOW (Sec. 3.3): k-buffer of window_k over
 * the tile list.                                                                          */
static void flat_tile(ctx* c, const sinks* sk, int tile, int64_t* cnt)
{
    const orc_params* P = &c->P;
    int tx = tile % c->txn, ty = tile / c->txn;
    tlist* L = &c->tl[tile];
    double allc = L->pre_margin;
    int nb = (L->n + 31) / 32;
    for (int b = 0; b <= nb; b++) allc = fmin(allc, L->bm_c[b]);
    fent* buf = (fent*)malloc((size_t)(L->n + 1) * sizeof(fent));
    pstate* ps = (pstate*)malloc(sizeof(pstate));
    for (int yy = 0; yy < 16; yy++)
        for (int xx = 0; xx < 16; xx++) {
            int X = tx * 16 + xx, Y = ty * 16 + yy;
            if (X >= c->cam.width || Y >= c->cam.height) continue;
            pixel_init(c, ps, X, Y);
            ps->cmin = fmin(ps->cmin, allc);
            if (P->mode == 1) {
                int k = 0;
                for (int j = 0; j < L->n; j++) {
                    cnt[CNT_EVAL_P]++;
                    double a = pixel_alpha(c, L->e[j].id, ps);
                    ps->cmin = fmin(ps->cmin, fabs(a / P->eps_o - 1.0));
                    if (a < P->eps_o) continue;
                    buf[k].t = pixel_depth(c, L->e[j].id, ps);
                    buf[k].pos = j; buf[k].id = L->e[j].id; buf[k].a = a;
                    k++;
                }
                qsort(buf, (size_t)k, sizeof(fent), cmp_fent);
                for (int j = 0; j < k && !ps->done; j++) {
                    if (j + 1 < k) ps->dmin = fmin(ps->dmin, relgap(buf[j].t, buf[j + 1].t));
                    blend(c, ps, sk, buf[j].t, buf[j].id, buf[j].a, cnt);
                }
            } else {
                int have_prev = 0;
                double prev_key = 0;
                for (int j = 0; j < L->n; j++) {
                    cnt[CNT_EVAL_P]++;
                    double a = pixel_alpha(c, L->e[j].id, ps);
                    ps->cmin = fmin(ps->cmin, fabs(a / P->eps_o - 1.0));
                    if (a < P->eps_o) continue;
                    if (have_prev) ps->dmin = fmin(ps->dmin, relgap(prev_key, L->e[j].t));
                    /* once the ray has terminated, the list order of the entry that ended it
                     * and the next contributing entry is the last decision that matters: had
                     * they been swapped, the other one would have been taken first           */
                    if (ps->done) break;
                    have_prev = 1;
                    prev_key = L->e[j].t;
                    double t = pixel_depth(c, L->e[j].id, ps);
                    if (P->mode == 2) blend(c, ps, sk, t, L->e[j].id, a, cnt);
                    else {
                        hent h = {t, L->e[j].id, a};
                        head_push(c, ps, sk, P->window_k, h, cnt);
                    }
                }
                if (P->mode == 3) head_flush(c, ps, sk, cnt);
            }
            pixel_out(c, ps, sk);
        }
    free(ps);
    free(buf);
}

/* ------------------------------------------------------------------ API */
static void free_lists(ctx* c)
{
    if (!c->tl) return;
    for (int t = 0; t < c->ntiles; t++) {
        free(c->tl[t].e); free(c->tl[t].nr); free(c->tl[t].bm_d); free(c->tl[t].bm_c);
    }
    free(c->tl);
    c->tl = NULL;
}
static void free_records(ctx* c)
{
    if (c->bl) {
        int64_t np = (int64_t)c->cam.width * c->cam.height;
        for (int64_t p = 0; p < np; p++) free(c->bl[p].r);
        free(c->bl);
        c->bl = NULL;
    }
    free(c->C); free(c->Z); free(c->T);
    c->C = c->Z = c->T = NULL;
}

static ctx* ctx_new(const orc_camera* cam, const orc_params* prm, int64_t n)
{
    ctx* c = (ctx*)calloc(1, sizeof(ctx));
    c->cam = *cam;
    c->P = *prm;
    c->prm = &c->P;
    transpose3(cam->R, c->Rt);
    matvec3(c->Rt, cam->t, c->o);
    for (int k = 0; k < 3; k++) c->o[k] = -c->o[k];          /* o = -R^T t             */
    c->n = n;
    c->txn = (cam->width + 15) / 16;
    c->tyn = (cam->height + 15) / 16;
    c->ntiles = c->txn * c->tyn;
    c->tl = (tlist*)calloc((size_t)c->ntiles, sizeof(tlist));
    for (int t = 0; t < c->ntiles; t++) c->tl[t].pre_margin = INFINITY;
    return c;
}

void* orc_create(const orc_scene* sc, const orc_camera* cam, const orc_params* prm,
                 const int32_t* tile_sel, int32_t nsel)
{
    ctx* c = ctx_new(cam, prm, sc->n);
    c->g = (grec*)calloc((size_t)(sc->n > 0 ? sc->n : 1), sizeof(grec));
    if (tile_sel) {
        c->sel = (int32_t*)malloc((size_t)(nsel > 0 ? nsel : 1) * sizeof(int32_t));
        c->nsel = 0;
        for (int k = 0; k < nsel; k++)
            if (tile_sel[k] >= 0 && tile_sel[k] < c->ntiles && !c->tl[tile_sel[k]].selected) {
                c->tl[tile_sel[k]].selected = 1;
                c->sel[c->nsel++] = tile_sel[k];
            }
    } else {
        c->sel = (int32_t*)malloc((size_t)c->ntiles * sizeof(int32_t));
        c->nsel = c->ntiles;
        for (int t = 0; t < c->ntiles; t++) { c->tl[t].selected = 1; c->sel[t] = t; }
    }
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < sc->n; i++) preprocess_one(c, sc, i);
    build_lists(c);
    return c;
}

void orc_destroy(void* h)
{
    ctx* c = (ctx*)h;
    if (!c) return;
    free_lists(c);
    free_records(c);
    free(c->g);
    free(c->sel);
    free(c);
}

int64_t orc_num_invalid(void* h)
{
    ctx* c = (ctx*)h;
    int64_t k = 0;
    for (int64_t i = 0; i < c->n; i++) k += c->g[i].invalid;
    return k;
}

int64_t orc_num_entries(void* h)
{
    ctx* c = (ctx*)h;
    int64_t e = 0;
    for (int t = 0; t < c->ntiles; t++) e += c->tl[t].n;
    return e;
}

void orc_get_preprocess(void* h, int32_t* visible, double* mean2, double* conic, double* opacity,
                        double* color, double* sinv6, double* v3, double* pcam, int32_t* rect,
                        int32_t* ntiles, double* margin)
{
    ctx* c = (ctx*)h;
    for (int64_t i = 0; i < c->n; i++) {
        const grec* g = &c->g[i];
        if (visible) visible[i] = g->visible;
        if (mean2) { mean2[2 * i] = g->mean2[0]; mean2[2 * i + 1] = g->mean2[1]; }
        if (conic) for (int k = 0; k < 3; k++) conic[3 * i + k] = g->conic[k];
        if (opacity) opacity[i] = g->opacity;
        if (color) for (int k = 0; k < 3; k++) color[3 * i + k] = g->color[k];
        if (sinv6) {
            sinv6[6 * i + 0] = g->sinv[0]; sinv6[6 * i + 1] = g->sinv[1]; sinv6[6 * i + 2] = g->sinv[2];
            sinv6[6 * i + 3] = g->sinv[4]; sinv6[6 * i + 4] = g->sinv[5]; sinv6[6 * i + 5] = g->sinv[8];
        }
        if (v3) for (int k = 0; k < 3; k++) v3[3 * i + k] = g->v[k];
        if (pcam) for (int k = 0; k < 3; k++) pcam[3 * i + k] = g->p[k];
        if (rect) for (int k = 0; k < 4; k++) rect[4 * i + k] = g->rect[k];
        if (ntiles) ntiles[i] = g->visible ? g->ntiles : 0;
        if (margin) margin[i] = g->margin;
    }
}

void orc_get_tile_lists(void* h, int64_t* start, int32_t* ids, double* ts)
{
    ctx* c = (ctx*)h;
    int64_t o = 0;
    for (int t = 0; t < c->ntiles; t++) {
        if (start) start[t] = o;
        for (int k = 0; k < c->tl[t].n; k++) {
            if (ids) ids[o + k] = c->tl[t].e[k].id;
            if (ts) ts[o + k] = c->tl[t].e[k].t;
        }
        o += c->tl[t].n;
    }
    if (start) start[c->ntiles] = o;
}

static void render_impl(ctx* c, const sinks* skp, int64_t* counters, double key_cut)
{
    sinks sk = *skp;
    free_records(c);
    int64_t np = (int64_t)c->cam.width * c->cam.height;
    if (c->P.record_blends) {
        c->bl = (blist*)calloc((size_t)np, sizeof(blist));
        c->C = (double*)calloc((size_t)np * 3, sizeof(double));
        c->Z = (double*)calloc((size_t)np, sizeof(double));
        c->T = (double*)calloc((size_t)np, sizeof(double));
    }
    int64_t tot[CNT_N];
    memset(tot, 0, sizeof tot);
    for (int64_t i = 0; i < c->n; i++)
        if (c->g[i].visible) {
            tot[CNT_VISIBLE]++;
            int w = c->g[i].rect[2] - c->g[i].rect[0] + 1, hh = c->g[i].rect[3] - c->g[i].rect[1] + 1;
            if (w > 0 && hh > 0) tot[CNT_CANDIDATES] += (int64_t)w * hh;
        }
    tot[CNT_ENTRIES] = orc_num_entries(c);
    /* a key cut renders each tile's list truncated to its entries with t < key_cut (a
     * prefix: the lists are sorted by (t, id)) with the decision margins of that prefix;
     * the full lengths and margins are restored after                                    */
    int* full_n = NULL;
    double **full_bd = NULL, **full_bc = NULL;
    if (key_cut < INFINITY) {
        full_n = (int*)malloc((size_t)c->nsel * sizeof(int));
        full_bd = (double**)malloc((size_t)c->nsel * sizeof(double*));
        full_bc = (double**)malloc((size_t)c->nsel * sizeof(double*));
        for (int k = 0; k < c->nsel; k++) {
            tlist* L = &c->tl[c->sel[k]];
            full_n[k] = L->n;
            full_bd[k] = L->bm_d;
            full_bc[k] = L->bm_c;
            int m = 0;
            while (m < L->n && L->e[m].t < key_cut) m++;
            L->n = m;
            batch_margins(L, key_cut);
        }
    }
#pragma omp parallel
    {
        int64_t cnt[CNT_N];
        memset(cnt, 0, sizeof cnt);
#pragma omp for schedule(dynamic, 1)
        for (int k = 0; k < c->nsel; k++) {
            int tile = c->sel[k];
            if (c->P.mode == 0)
                for (int S = 0; S < 16; S++) hier_subtile(c, &sk, tile, S, cnt);
            else
                flat_tile(c, &sk, tile, cnt);
        }
#pragma omp critical
        for (int k = 0; k < CNT_N; k++)
            if (k != CNT_VISIBLE && k != CNT_ENTRIES && k != CNT_CANDIDATES) tot[k] += cnt[k];
    }
    if (full_n) {
        for (int k = 0; k < c->nsel; k++) {
            tlist* L = &c->tl[c->sel[k]];
            free(L->bm_d);
            free(L->bm_c);
            L->n = full_n[k];
            L->bm_d = full_bd[k];
            L->bm_c = full_bc[k];
        }
        free(full_n);
        free(full_bd);
        free(full_bc);
    }
    if (counters) memcpy(counters, tot, sizeof tot);
}

void orc_render(void* h, double* rgb, double* depth, double* tfinal, int32_t* nblend,
                uint64_t* hash, double* dmargin, double* cmargin, double* delta,
                int32_t* seq, int32_t max_seq, int64_t* counters)
{
    sinks sk = {rgb, depth, tfinal, dmargin, cmargin, delta, nblend, hash, seq, max_seq, NULL};
    render_impl((ctx*)h, &sk, counters, INFINITY);
}

void orc_render_ex(void* h, double* rgb, double* depth, double* tfinal, int32_t* nblend,
                   uint64_t* hash, double* dmargin, double* cmargin, double* delta,
                   int32_t* seq, int32_t max_seq, int64_t* counters, int32_t* sat_batch, double key_cut)
{
    sinks sk = {rgb, depth, tfinal, dmargin, cmargin, delta, nblend, hash, seq, max_seq, sat_batch};
    render_impl((ctx*)h, &sk, counters, key_cut);
}

int32_t orc_schedule_synthetic(int32_t n, const double* t, const int32_t* keep, double alpha,
                               int32_t mode, int32_t tail, int32_t mid, int32_t head,
                               int32_t flags, int32_t* order)
{
    orc_camera cam;
    memset(&cam, 0, sizeof cam);
    cam.R[0] = cam.R[4] = cam.R[8] = 1.0;
    cam.fx = cam.fy = 16.0; cam.cx = cam.cy = 8.0;
    cam.width = 16; cam.height = 16;
    orc_params P;
    memset(&P, 0, sizeof P);
    P.tail = tail; P.mid = mid; P.head = head; P.flags = flags;
    P.mode = mode; P.window_k = head;
    P.eps_o = 1.0 / 255.0; P.t_min = 1e-300; P.alpha_max = 0.99;
    ctx* c = ctx_new(&cam, &P, n);
    c->syn_t = t;
    c->syn_alpha = alpha;
    c->syn_keep = keep;
    tlist* L = &c->tl[0];
    L->selected = 1;
    L->pre_margin = INFINITY;
    for (int k = 0; k < n; k++) tl_push(L, t[k], k);     /* list order as given        */
    int nb = (n + 31) / 32;
    L->bm_d = (double*)malloc((size_t)(nb + 1) * sizeof(double));
    L->bm_c = (double*)malloc((size_t)(nb + 1) * sizeof(double));
    for (int b = 0; b <= nb; b++) L->bm_d[b] = L->bm_c[b] = INFINITY;
    int32_t* seq = (int32_t*)malloc((size_t)256 * (n + 1) * sizeof(int32_t));
    sinks sk;
    memset(&sk, 0, sizeof sk);
    int32_t* nbl = (int32_t*)calloc(256, sizeof(int32_t));
    sk.seq = seq; sk.max_seq = n + 1; sk.nblend = nbl;
    int64_t cnt[CNT_N];
    memset(cnt, 0, sizeof cnt);
    if (mode == 0) hier_subtile(c, &sk, 0, 0, cnt);
    else flat_tile(c, &sk, 0, cnt);
    int32_t m = nbl[0];
    for (int k = 0; k < m; k++) order[k] = seq[k];
    free(seq);
    free(nbl);
    orc_destroy(c);
    return m;
}

/* ------------------------------------------------------------------ adjoint
 * Sec. 3.5: gradients in front-to-back blend order with the suffix colour C - C_i and the
 * suffix transmittance T_N / T_i; then the chain rule through the preprocess (3DGS
 * structure: conic -> Sigma2 -> Sigma -> scale, rotation; mean2 and J -> mean; colour ->
 * SH and direction -> mean; opacity -> logit), and through t_opt for the depth output.  */
void orc_backward(void* h, const orc_scene* sc, const double* dl_drgb, const double* dl_ddepth,
                  double* d_means, double* d_log_scales, double* d_quats, double* d_logits,
                  double* d_sh, double* d_mean2, double* d_conic, double* d_opacity,
                  double* d_color)
{
    ctx* c = (ctx*)h;
    const orc_params* P = &c->P;
    int64_t n = c->n;
    if (!c->bl) return;
    double* gm2 = (double*)calloc((size_t)n * 2, sizeof(double));
    double* gcon = (double*)calloc((size_t)n * 3, sizeof(double));
    double* gop = (double*)calloc((size_t)n, sizeof(double));
    double* gcol = (double*)calloc((size_t)n * 3, sizeof(double));
    double* gmu = (double*)calloc((size_t)n * 3, sizeof(double));
    double* gsinv = (double*)calloc((size_t)n * 9, sizeof(double));
    int64_t np = (int64_t)c->cam.width * c->cam.height;
    double bgdot_w[3] = {P->bg[0], P->bg[1], P->bg[2]};
    for (int64_t p = 0; p < np; p++) {
        blist* B = &c->bl[p];
        if (B->n == 0) continue;
        double x = (double)(p % c->cam.width) + 0.5, y = (double)(p / c->cam.width) + 0.5;
        const double* g = &dl_drgb[3 * p];
        double gz = dl_ddepth ? dl_ddepth[p] : 0.0;
        double Cf[3] = {c->C[3 * p], c->C[3 * p + 1], c->C[3 * p + 2]};
        double Zf = c->Z[p], Tf = c->T[p];
        double gbg = g[0] * bgdot_w[0] + g[1] * bgdot_w[1] + g[2] * bgdot_w[2];
        double Ca[3] = {0, 0, 0}, Za = 0;
        double d[3];
        cam_ray(c, x, y, d);
        for (int k = 0; k < B->n; k++) {
            int id = B->r[k].id;
            const grec* G = &c->g[id];
            double a = B->r[k].a, t = B->r[k].t, T = B->r[k].T;
            for (int ch = 0; ch < 3; ch++) Ca[ch] += G->color[ch] * a * T;
            Za += t * a * T;
            for (int ch = 0; ch < 3; ch++) gcol[3 * id + ch] += g[ch] * a * T;
            double da = 0;
            for (int ch = 0; ch < 3; ch++) da += g[ch] * (G->color[ch] * T - (Cf[ch] - Ca[ch]) / (1.0 - a));
            da -= gbg * Tf / (1.0 - a);
            da += gz * (t * T - (Zf - Za) / (1.0 - a));
            double dt = gz * a * T;
            /* alpha = min(alpha_max, opacity * G2)                                       */
            double G2 = gauss2(G, x, y);
            if (G->opacity * G2 < P->alpha_max) {
                gop[id] += da * G2;
                double dG = da * G->opacity;
                double dx = x - G->mean2[0], dy = y - G->mean2[1];
                gcon[3 * id + 0] += dG * G2 * (-0.5 * dx * dx);
                gcon[3 * id + 1] += dG * G2 * (-dx * dy);
                gcon[3 * id + 2] += dG * G2 * (-0.5 * dy * dy);
                gm2[2 * id + 0] += dG * G2 * (G->conic[0] * dx + G->conic[1] * dy);
                gm2[2 * id + 1] += dG * G2 * (G->conic[1] * dx + G->conic[2] * dy);
            }
            /* t = d^T Sinv (mu - o) / (d^T Sinv d)                                       */
            if (dt != 0.0) {
                double m[3] = {G->mu[0] - c->o[0], G->mu[1] - c->o[1], G->mu[2] - c->o[2]};
                double sd[3], sm[3];
                matvec3(G->sinv, d, sd);
                matvec3(G->sinv, m, sm);
                double num = d[0] * sm[0] + d[1] * sm[1] + d[2] * sm[2];
                double den = d[0] * sd[0] + d[1] * sd[1] + d[2] * sd[2];
                for (int r = 0; r < 3; r++) gmu[3 * id + r] += dt * sd[r] / den;
                for (int r = 0; r < 3; r++)
                    for (int cc = 0; cc < 3; cc++)
                        gsinv[9 * id + 3 * r + cc] += dt * (d[r] * m[cc] / den - num / (den * den) * d[r] * d[cc]);
            }
        }
    }
    int K = (P->sh_degree + 1) * (P->sh_degree + 1);
    for (int64_t i = 0; i < n; i++) {
        const grec* G = &c->g[i];
        if (d_mean2) { d_mean2[2 * i] = gm2[2 * i]; d_mean2[2 * i + 1] = gm2[2 * i + 1]; }
        if (d_conic) for (int k = 0; k < 3; k++) d_conic[3 * i + k] = gcon[3 * i + k];
        if (d_opacity) d_opacity[i] = gop[i];
        if (d_color) for (int k = 0; k < 3; k++) d_color[3 * i + k] = gcol[3 * i + k];
        double dmu[3] = {gmu[3 * i], gmu[3 * i + 1], gmu[3 * i + 2]};
        double dls[3] = {0, 0, 0}, dq[4] = {0, 0, 0, 0};
        double dlogit = 0;
        double dsh[16 * 3];
        memset(dsh, 0, sizeof dsh);
        if (G->visible) {
            /* colour -> SH; colour -> view direction -> mean                               */
            double Y[16], dY[48];
            sh_basis_grad(G->dir, Y, dY);
            double ddir[3] = {0, 0, 0};
            for (int ch = 0; ch < 3; ch++) {
                double draw = G->raw[ch] > 0 ? gcol[3 * i + ch] : 0.0;
                for (int j = 0; j < K; j++) {
                    double coef = sc->sh[(i * K + j) * 3 + ch];
                    dsh[3 * j + ch] = draw * Y[j];
                    for (int r = 0; r < 3; r++) ddir[r] += draw * coef * dY[3 * j + r];
                }
            }
            /* dir = u / |u|, u = mu - o: d dir / d u = (I - dir dir^T) / |u|                */
            double dd = ddir[0] * G->dir[0] + ddir[1] * G->dir[1] + ddir[2] * G->dir[2];
            for (int r = 0; r < 3; r++) dmu[r] += (ddir[r] - dd * G->dir[r]) / G->ulen;
            /* opacity -> logit                                                            */
            dlogit = gop[i] * G->opacity * (1.0 - G->opacity);
            /* conic -> Sigma2: dSigma2 = -A dA A with dA the symmetric matrix gradient     */
            double A[4] = {G->conic[0], G->conic[1], G->conic[1], G->conic[2]};
            double Ab[4] = {gcon[3 * i], 0.5 * gcon[3 * i + 1], 0.5 * gcon[3 * i + 1], gcon[3 * i + 2]};
            double tmp[4], S2b[4];
            for (int r = 0; r < 2; r++)
                for (int cc = 0; cc < 2; cc++) tmp[2 * r + cc] = A[2 * r] * Ab[cc] + A[2 * r + 1] * Ab[2 + cc];
            for (int r = 0; r < 2; r++)
                for (int cc = 0; cc < 2; cc++) S2b[2 * r + cc] = -(tmp[2 * r] * A[cc] + tmp[2 * r + 1] * A[2 + cc]);
            /* Sigma2 = Tm Sigma Tm^T + dil I                                              */
            double Sb[9], Tmb[6];
            for (int r = 0; r < 3; r++)
                for (int cc = 0; cc < 3; cc++) {
                    double s = 0;
                    for (int a2 = 0; a2 < 2; a2++)
                        for (int b2 = 0; b2 < 2; b2++) s += G->Tm[3 * a2 + r] * S2b[2 * a2 + b2] * G->Tm[3 * b2 + cc];
                    Sb[3 * r + cc] = s;
                }
            for (int r = 0; r < 2; r++)
                for (int cc = 0; cc < 3; cc++) {
                    double s = 0;
                    for (int b2 = 0; b2 < 2; b2++)
                        for (int k = 0; k < 3; k++) s += S2b[2 * r + b2] * G->Tm[3 * b2 + k] * G->sigma[3 * k + cc];
                    Tmb[3 * r + cc] = 2.0 * s;
                }
            /* Tm = J R_c -> J bar = Tm bar R_c^T                                          */
            double Jb[6];
            for (int r = 0; r < 2; r++)
                for (int cc = 0; cc < 3; cc++) {
                    double s = 0;
                    for (int k = 0; k < 3; k++) s += Tmb[3 * r + k] * c->cam.R[3 * cc + k];
                    Jb[3 * r + cc] = s;
                }
            double px = G->p[0], py = G->p[1], pz = G->p[2];
            double fx = c->cam.fx, fy = c->cam.fy;
            double dp[3] = {0, 0, 0};
            dp[2] += Jb[0] * (-fx / (pz * pz)) + Jb[4] * (-fy / (pz * pz));
            if (!G->clampx) { dp[0] += Jb[2] * (-fx / (pz * pz)); dp[2] += Jb[2] * (2.0 * fx * px / (pz * pz * pz)); }
            else { double cx = G->J[2] * pz / (-fx); dp[2] += Jb[2] * (fx * cx / (pz * pz)); }
            if (!G->clampy) { dp[1] += Jb[5] * (-fy / (pz * pz)); dp[2] += Jb[5] * (2.0 * fy * py / (pz * pz * pz)); }
            else { double cy = G->J[5] * pz / (-fy); dp[2] += Jb[5] * (fy * cy / (pz * pz)); }
            /* mean2 = (fx px / pz + cx, fy py / pz + cy)                                  */
            dp[0] += gm2[2 * i] * fx / pz;
            dp[1] += gm2[2 * i + 1] * fy / pz;
            dp[2] += -gm2[2 * i] * fx * px / (pz * pz) - gm2[2 * i + 1] * fy * py / (pz * pz);
            /* p = R_c mu + t_c                                                            */
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) dmu[r] += c->cam.R[3 * k + r] * dp[k];
            /* Sigma = M M^T, M = Rq diag(s): M bar = 2 Sigma bar M (Sigma bar symmetric)   */
            double Rqb[9];
            memset(Rqb, 0, sizeof Rqb);
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) {
                    double mb = 0;
                    for (int j = 0; j < 3; j++) mb += 2.0 * Sb[3 * r + j] * G->Rq[3 * j + k] * G->s[k];
                    dls[k] += mb * G->Rq[3 * r + k] * G->s[k];     /* d/dlog s = s d/ds      */
                    Rqb[3 * r + k] += mb * G->s[k];
                }
            /* Sigma^-1 = Rq diag(w) Rq^T (depth path)                                      */
            const double* Gi = &gsinv[9 * i];
            double Gs[9];
            for (int r = 0; r < 3; r++)
                for (int cc = 0; cc < 3; cc++) Gs[3 * r + cc] = Gi[3 * r + cc] + Gi[3 * cc + r];
            for (int r = 0; r < 3; r++)
                for (int k = 0; k < 3; k++) {
                    double s = 0;
                    for (int j = 0; j < 3; j++) s += Gs[3 * r + j] * G->Rq[3 * j + k];
                    Rqb[3 * r + k] += s * G->w[k];
                }
            for (int k = 0; k < 3; k++) {
                double dw = 0;
                for (int r = 0; r < 3; r++)
                    for (int j = 0; j < 3; j++) dw += G->Rq[3 * r + k] * Gi[3 * r + j] * G->Rq[3 * j + k];
                if (1.0 / G->s[k] < P->inv_scale_max) dls[k] += dw * (-2.0 * G->w[k]);
            }
            /* rotation -> normalised quaternion -> raw quaternion                          */
            double w = G->qn[0], x = G->qn[1], yq = G->qn[2], z = G->qn[3];
            const double* R = Rqb;
            double gq[4];
            gq[0] = 2 * (-z * R[1] + yq * R[2] + z * R[3] - x * R[5] - yq * R[6] + x * R[7]);
            gq[1] = 2 * (yq * R[1] + z * R[2] + yq * R[3] - 2 * x * R[4] - w * R[5] + z * R[6] + w * R[7] - 2 * x * R[8]);
            gq[2] = 2 * (-2 * yq * R[0] + x * R[1] + w * R[2] + x * R[3] + z * R[5] - w * R[6] + z * R[7] - 2 * yq * R[8]);
            gq[3] = 2 * (-2 * z * R[0] - w * R[1] + x * R[2] + w * R[3] - 2 * z * R[4] + yq * R[5] + x * R[6] + yq * R[7]);
            double dotq = gq[0] * w + gq[1] * x + gq[2] * yq + gq[3] * z;
            for (int k = 0; k < 4; k++) dq[k] = (gq[k] - dotq * G->qn[k]) / G->qlen;
        }
        if (d_means) for (int k = 0; k < 3; k++) d_means[3 * i + k] = dmu[k];
        if (d_log_scales) for (int k = 0; k < 3; k++) d_log_scales[3 * i + k] = dls[k];
        if (d_quats) for (int k = 0; k < 4; k++) d_quats[4 * i + k] = dq[k];
        if (d_logits) d_logits[i] = dlogit;
        if (d_sh) for (int k = 0; k < K * 3; k++) d_sh[(int64_t)i * K * 3 + k] = dsh[k];
    }
    free(gm2); free(gcon); free(gop); free(gcol); free(gmu); free(gsinv);
}
