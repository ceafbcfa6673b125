/* stp_oracle.h -- FP64 CPU oracle of StopThePop's sorted splatting renderer.
 *
 * TEST INFRASTRUCTURE ONLY. This library is the slow, plain restatement of the paper's
 * method that the CUDA path is checked against. Only the tests, the package's smoke check
 * and the CPU-baseline leg of the bench may load it; the product path never does.
 * It shares no code, header, table or constant with the CUDA library.
 *
 * Paper: Radl, Steiner et al., "StopThePop: Sorted Gaussian Splatting for View-Consistent
 * Real-time Rendering", TOG 43(4) 2024 (arXiv 2402.00525).
 */
#ifndef STP_ORACLE_H
#define STP_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    double R[9];          /* world -> camera rotation, row major: p = R x + t          */
    double t[3];
    double fx, fy, cx, cy;
    int32_t width, height;
} orc_camera;

typedef struct {
    int32_t tail, mid, head;   /* queue sizes (Sec. 3.4): 32n+32, 4m+4, any             */
    int32_t mode;              /* 0 HIER, 1 FULL, 2 GLOBAL, 3 WINDOW                    */
    int32_t window_k;          /* WINDOW mode k-buffer size (Sec. 3.3)                 */
    int32_t flags;             /* 1: head evict-before-insert; 2: level-centre rays;
                                  4: tile-centre key; 8: view-space-depth key;
                                  512: no tile-based culling; 1024: no culling at the
                                  4x4 / 2x2 levels of Render (ablations D, E)           */
    int32_t sh_degree;
    int32_t record_blends;     /* keep per-pixel blend lists (needed by the adjoint)   */
    double eps_o, t_min, alpha_max, inv_scale_max, dilation, frustum_clamp, znear;
    double bg[3];
    double gap_thr;            /* relative depth gap below which an order is undecided  */
    double cull_thr;           /* relative distance to eps_O / t_min that is undecided  */
} orc_params;

typedef struct {               /* caller's SoA inputs, FP64                              */
    int64_t n;
    const double *means, *log_scales, *quats, *logits, *sh;
} orc_scene;

/* ---- building blocks (pinned one by one in the tests) ---- */
double orc_t_opt(const double d[3], const double o[3], const double mu[3], const double sinv[9]);
void   orc_alg1(const double mu2[2], const double conic[3], const double box[4], double xhat[2]);
void   orc_sigma_inv(const double quat[4], const double log_scale[3], double inv_scale_max,
                     double sinv[9]);
void   orc_sigma(const double quat[4], const double log_scale[3], double sigma[9]);
void   orc_sh_basis(const double dir[3], double y[16]);
double orc_t_o(double opacity, double eps_o);
void   orc_project(const orc_camera* cam, const orc_params* prm, const double mu[3],
                   const double sigma[9], double mean2[2], double cov2[3], double jac[6]);

/* ---- whole pipeline ---- */
/* tile_sel: tiles to build and render (NULL = all). Returns an opaque handle.           */
void*   orc_create(const orc_scene* sc, const orc_camera* cam, const orc_params* prm,
                   const int32_t* tile_sel, int32_t nsel);
void    orc_destroy(void* h);
int64_t orc_num_entries(void* h);
/* Gaussians dropped as invalid: a non-finite mean, log-scale, quaternion, logit or SH
 * coefficient, or a quaternion of squared length below 1e-20.                            */
int64_t orc_num_invalid(void* h);
/* per-Gaussian preprocess results (any pointer may be NULL)                              */
void    orc_get_preprocess(void* h, int32_t* visible, double* mean2, double* conic,
                           double* opacity, double* color, double* sinv6, double* v3,
                           double* pcam, int32_t* rect, int32_t* ntiles, double* margin);
/* tile lists: start[T+1] offsets, ids[E], depth keys ts[E] (sorted by (t, id) per tile)  */
void    orc_get_tile_lists(void* h, int64_t* start, int32_t* ids, double* ts);
/* render the selected tiles. Every output may be NULL. counters[16] (see oracle.py).     */
void    orc_render(void* h, double* rgb, double* depth, double* tfinal, int32_t* nblend,
                   uint64_t* hash, double* dmargin, double* cmargin, double* delta,
                   int32_t* seq, int32_t max_seq, int64_t* counters);
/* orc_render with two additions: sat_batch[pixel] (may be NULL) receives the HIER batch
 * during whose processing the pixel's ray terminated (-1: during the final drain or in a
 * flat order, -2: never), and key_cut < INFINITY renders every tile list truncated to its
 * entries with key t < key_cut (a prefix of the sorted list).                            */
void    orc_render_ex(void* h, double* rgb, double* depth, double* tfinal, int32_t* nblend,
                      uint64_t* hash, double* dmargin, double* cmargin, double* delta,
                      int32_t* seq, int32_t max_seq, int64_t* counters, int32_t* sat_batch,
                      double key_cut);
/* adjoint of the last orc_render (record_blends must have been set); sc is the scene the
 * handle was created from.                                                               */
void    orc_backward(void* h, const orc_scene* sc, const double* dl_drgb, const double* dl_ddepth,
                     double* d_means, double* d_log_scales, double* d_quats, double* d_logits,
                     double* d_sh, double* d_mean2, double* d_conic, double* d_opacity,
                     double* d_color);
/* Schedule on a synthetic tile list (list order as given) whose depth is t[k] at every
 * level and whose alpha is `alpha` everywhere; keep[k] = 0 culls entry k at the 4x4 level
 * (keep may be NULL). mode 0 = HIER (tail/mid/head sizes), 3 = WINDOW (k = head). Writes
 * the blend order of one pixel and returns its length.                                   */
int32_t orc_schedule_synthetic(int32_t n, const double* t, const int32_t* keep, double alpha,
                               int32_t mode, int32_t tail, int32_t mid, int32_t head,
                               int32_t flags, int32_t* order);

#ifdef __cplusplus
}
#endif
#endif
