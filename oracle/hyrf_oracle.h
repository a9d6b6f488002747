/*
 * HyRF oracle: a plain, slow, single-threaded FP64 CPU implementation of the
 * HyRF render-and-train path (arXiv 2509.17083, Sec. 3 and App. A).
 *
 * TEST INFRASTRUCTURE ONLY. It exists to check the CUDA path. Only the tests,
 * the smoke check and the CPU-baseline leg of the benchmark may load it. The
 * product path never links, imports or calls it. It shares no code, header,
 * table or constant with the CUDA library.
 *
 * Conventions (all arrays row-major, contiguous, caller-owned):
 *   - floating point is double unless stated; integer decisions that the GPU
 *     takes in FP32 (visibility, tile rectangles, sort keys, the near-singular
 *     flag) are replayed here in float with the same operation order
 *     ("FP32 replay"), so that they can be compared bit for bit;
 *   - every *_backward function ACCUMULATES into its gradient outputs;
 *   - functions return 0 on success and a negative number on invalid input.
 *
 * Parity pins (tests/test_oracle_*.py; each pins against something other
 * than the oracle itself):
 *   contraction      closed-form values, range (0,1), C1 at |x| = 1, FD Jacobian
 *   hash encoding    linear functions reproduced on a dense level, partition
 *                    of unity, level resolutions, Instant-NGP hash definition
 *   MLP / PE         numpy matmul reference; closed-form sin/cos values
 *   query + bwd      reduction to the biases; central finite differences;
 *                    outputs unchanged under a camera roll about its centre
 *                    (world-space view direction), geometry independent of
 *                    the camera
 *   pre-cull         hand cases; FP64 agreement away from the thresholds
 *   projection       on-axis closed form; scipy rotation + FD Jacobian
 *                    reference; FD backward; FP32 rect vs FP64 definition
 *   binning          brute-force tile coverage; tiled == untiled compositing
 *   footprint        threshold against numpy's logarithm; brute force over
 *                    every pixel centre (no tile that Eq. 1 can show the
 *                    Gaussian in is dropped); packed row spans decode to the
 *                    instance lists; footprint lists composite exactly like
 *                    the rectangles
 *   compositing      single-Gaussian closed form; two overlapping Gaussians
 *                    in either depth order (front-to-back closed form);
 *                    weights sum to 1 - T_final; FD backward
 *   background       |o + t d| = r with t > 0; constant field; FD backward;
 *                    a camera rolled by 180 degrees sees the same colour
 *                    along the same world ray (pixel (W-1-i, H-1-j)).
 *                    The equirect "background map" layout is a reading of
 *                    the paper's one-line mention: parity unpinned against
 *                    the paper for map mode (pinned by FD, the
 *                    constant-field case and, from the centre of a cubic
 *                    box, O(h^2) convergence of the map colour to the exact
 *                    mode's colour of each ray).
 *   loss             scipy-correlate SSIM reference, SSIM(x,x) = 1, L1 closed
 *                    form, FD gradient
 *   whole path       reduction to isotropic 3DGS (Tab. 5 "w/o Neural"); FD of
 *                    the loss w.r.t. every parameter class
 *   Adam             first-step closed form p - lr g / (|g| + eps); constant
 *                    gradient over t steps; zero gradient decays the moments
 *   8-bit codec      codes of an affine ramp; min/max map to 0/255;
 *                    round trip within step / 2
 *   density control  hand-built keep / prune / clone / split cases; counts
 *                    and offsets by brute force; split halves at p + s * z
 *                    for the identity rotation, mirrored for q and -q
 */
#ifndef HYRF_ORACLE_H
#define HYRF_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Pinhole camera, world -> camera: x_c = R x_w + t (Sec. 3.3, Eq. 8).
 * Pixel (i, j) samples the image plane at (i + 0.5, j + 0.5). */
typedef struct {
  double R[9];
  double t[3];
  double fx, fy, cx, cy;
  int32_t width, height;
  double z_near;   /* "too close" threshold of the pre-cull (Sec. 3.3) */
  double cull_tol; /* tolerance band "tol" of Eq. 9 */
} orc_camera;

/* Scene box B0 used for normalisation (App. A.1). */
typedef struct {
  double lo[3], hi[3];
} orc_aabb;

/* Multi-resolution hash grid (Eq. 3, Instant-NGP encoding).
 * table: [n_levels][2^log2_T][n_feat] */
typedef struct {
  int32_t n_levels, log2_T, n_feat, base_res;
  double growth;
  const double* table;
} orc_grid;

/* Decoder MLP (Eqs. 4 and 6): n_hidden ReLU layers of `width`, linear output.
 * W[0]: [width][n_in], W[l]: [width][width], W[n_hidden]: [n_out][width].
 * relu_replay selects the precision in which each hidden unit's ReLU branch
 * (active or not) is decided; the values themselves are always FP64:
 *   0: from the FP64 pre-activation;
 *   1: from a replay of the layers as a BF16-operand kernel evaluates them:
 *      every layer input rounded to bfloat16 (through float, ties to even),
 *      products summed exactly, the ReLU output rounded to bfloat16 before
 *      the next layer. A kernel that accumulates in FP32 then takes the same
 *      branches except where a pre-activation lies within FP32 rounding of
 *      zero, so the FP64 values differ from it by rounding, not by a flipped
 *      branch. */
typedef struct {
  int32_t n_in, width, n_hidden, n_out;
  const double* W[3];
  const double* b[3];
  int32_t relu_replay;
} orc_mlp;

typedef struct {
  double* W[3];
  double* b[3];
} orc_mlp_grad;

/* ---------------- building blocks (exposed for the pins) ---------------- */

/* App. A.1 normalisation followed by Eq. 2 contraction (+0.5 reading).
 * y[3] receives contract(normalize(p)); J[9] (may be NULL) receives dy/dp. */
void orc_contract(const orc_aabb* box, const double p[3], double y[3], double J[9]);

/* Hash encoding of one point y in (0,1)^3: f[n_levels * n_feat], level-major. */
void orc_hash_encode(const orc_grid* g, const double y[3], double* f);

/* Resolution of level l: floor(base_res * growth^l). */
int32_t orc_level_res(const orc_grid* g, int32_t l);

/* Index of grid vertex (ix, iy, iz) at level l (dense or hashed). */
uint32_t orc_level_index(const orc_grid* g, int32_t l, uint32_t ix, uint32_t iy, uint32_t iz);

/* MLP forward on one input vector. */
void orc_mlp_forward(const orc_mlp* m, const double* x, double* y);

/* NeRF positional encoding of a unit direction (Eq. 5): 3 + 6 * n_freq values. */
void orc_pos_enc(const double d[3], int32_t n_freq, double* out);

/* ---------------- stage 1: pre-cull (Eqs. 8-9), FP32 replay ------------- */
/* pos: [n][3] float. vis: [n] (1 = kept). Returns the number kept. */
int32_t orc_precull_f32(int32_t n, const float* pos, const orc_camera* cam, uint8_t* vis);

/* ---------------- stage 2: field query + aggregation (Eqs. 2-7) --------- */
typedef struct {
  orc_aabb box;
  orc_grid geo, rad;
  orc_mlp geo_mlp, col_mlp;
  int32_t pe_freq;  /* number of PE frequencies */
  int32_t pe_pad;   /* PE block width in the colour-MLP input (>= 3 + 6 pe_freq) */
} orc_fields;

/* For each of the n (already visible) Gaussians: alpha[n], scale[n][3],
 * quat[n][4] (w,x,y,z), color[n][3]. */
int32_t orc_query_fields(int32_t n, const double* pos, const double* alpha_e,
                         const double* scale_e, const double* color_e,
                         const orc_camera* cam, const orc_fields* fl,
                         double* alpha, double* scale, double* quat, double* color);

int32_t orc_query_fields_backward(int32_t n, const double* pos, const double* alpha_e,
                                  const double* scale_e, const double* color_e,
                                  const orc_camera* cam, const orc_fields* fl,
                                  const double* d_alpha, const double* d_scale,
                                  const double* d_quat, const double* d_color,
                                  double* d_pos, double* d_alpha_e, double* d_scale_e,
                                  double* d_color_e, double* d_geo_table, double* d_rad_table,
                                  const orc_mlp_grad* d_geo_mlp, const orc_mlp_grad* d_col_mlp);

/* Smallest relative ReLU margin of each point's decoders: over every hidden
 * unit, min |z| / (sum_i |W_i a_i| + |b|), where z is the pre-activation the
 * unit's branch is decided on and a the layer input (FP64, or the replay's
 * values when relu_replay is set): a diagnostic used to find points whose
 * ReLU branches another evaluation could take differently.
 * margin_geo[n], margin_col[n]. */
int32_t orc_decoder_margins(int32_t n, const double* pos, const orc_camera* cam,
                            const orc_fields* fl, double* margin_geo, double* margin_col);

/* Running sum, over every decoder evaluation since the last reset, of a
 * 64-bit mix of that evaluation's hidden ReLU branch pattern (a diagnostic
 * for finite-difference drivers: a step that changes any branch anywhere
 * changes the sum). */
void orc_branch_sum_reset(void);
uint64_t orc_branch_sum(void);

/* ---------------- stage 3: projection (EWA, 3DGS conventions) ----------- */
/* FP64: mean2d[n][2], conic[n][3] (a, b, c of the inverse 2D covariance),
 * depth[n]. */
int32_t orc_project(int32_t n, const double* pos, const double* scale, const double* quat,
                    const orc_camera* cam, double* mean2d, double* conic, double* depth);

/* FP32 replay of the integer outputs: rect[n][4] = (x0, y0, x1, y1) tiles,
 * half-open; ntiles[n]; depth bits (float) in depth[n]; near-singular flag. */
int32_t orc_project_f32(int32_t n, const float* pos, const float* scale, const float* quat,
                        const orc_camera* cam, int32_t tile, int32_t* rect, int32_t* ntiles,
                        float* depth, uint8_t* flag);

/* As orc_project_f32, with the binning's opacity-aware footprint: with foot
 * given, ntiles counts only the tiles of the rectangle whose pixel centres
 * meet the ellipse q <= t (q = d^T Sigma'^-1 d, t = 1.02 x 2 ln(255 o) +
 * 0.05, o = alpha[i] or 1 when alpha is NULL; no footprint when o < 1/255;
 * near-singular Gaussians keep their rectangle, t = +inf), and foot[n][12]
 * receives (Sigma'_xx, Sigma'_xy, Sigma'_yy, t) in FP32 followed by eight
 * words of row spans: when the rectangle has at most 16 rows and 255
 * columns, row j's 16-bit field (word j / 2, bits from 16 (j % 2)) holds its
 * first tile column minus x0 and, in the high byte, its length; otherwise
 * zeros. mean2d[n][2] (may be NULL) receives the FP32 pixel position. */
int32_t orc_project_f32_fp(int32_t n, const float* pos, const float* scale, const float* quat,
                           const float* alpha, const orc_camera* cam, int32_t tile, int32_t* rect,
                           int32_t* ntiles, float* depth, uint8_t* flag, float* mean2d, float* foot);

int32_t orc_project_backward(int32_t n, const double* pos, const double* scale,
                             const double* quat, const orc_camera* cam,
                             const double* d_mean2d, const double* d_conic,
                             double* d_pos, double* d_scale, double* d_quat);

/* ---------------- stage 4: binning and depth sort ----------------------- */
/* Instances in (Gaussian, tile row-major) order, keyed (tile << 32) | bits(depth),
 * stable-sorted. keys/vals capacity `cap`; ranges[tiles][2] (start, end).
 * Returns K (number of instances) or -1 if K > cap. */
int64_t orc_bin_sort(int32_t n, const int32_t* rect, const float* depth, int32_t tiles_x,
                     int32_t tiles_y, int64_t cap, uint64_t* keys, int32_t* vals,
                     int32_t* ranges);

/* As orc_bin_sort, with the instances of each rectangle row limited to the
 * footprint's tile columns (mean2d and foot from orc_project_f32_fp; NULL
 * foot: whole rectangles). */
int64_t orc_bin_sort_fp(int32_t n, const int32_t* rect, const float* depth, const float* mean2d,
                        const float* foot, int32_t tile, int32_t tiles_x, int32_t tiles_y, int64_t cap,
                        uint64_t* keys, int32_t* vals, int32_t* ranges);

/* ---------------- stage 5: front-to-back compositing (Eq. 1) ------------ */
/* C_fg[H][W][3], T_final[H][W], n_contrib[H][W] (list position of the last
 * contributor + 1), margin[H][W] = smallest relative distance of any
 * threshold test of the pixel from its threshold (diagnostic; may be NULL). */
int32_t orc_rasterize(int32_t width, int32_t height, int32_t tile, const int32_t* ranges,
                      const int32_t* vals, const double* mean2d, const double* conic,
                      const double* opacity, const double* color, double* C_fg,
                      double* T_final, int32_t* n_contrib, double* margin);

int32_t orc_rasterize_backward(int32_t width, int32_t height, int32_t tile,
                               const int32_t* ranges, const int32_t* vals,
                               const double* mean2d, const double* conic,
                               const double* opacity, const double* color,
                               const double* d_C_fg, const double* d_T_final,
                               double* d_mean2d, double* d_conic, double* d_opacity,
                               double* d_color);

/* Untiled brute force of Eq. 1: every pixel composites, in (depth, index)
 * order, every Gaussian whose tile rectangle contains the pixel's tile. */
int32_t orc_rasterize_untiled(int32_t width, int32_t height, int32_t tile, int32_t n,
                              const int32_t* rect, const float* depth,
                              const double* mean2d, const double* conic,
                              const double* opacity, const double* color, double* C_fg,
                              double* T_final);

/* ---------------- stage 6: neural background (Eqs. 10-11, App. A.2) ----- */
typedef struct {
  int32_t mode; /* 0 = exact per-pixel query, 1 = equirect map */
  int32_t map_h, map_w;
  double radius;
} orc_bg;

/* Ray/sphere hit in normalised space for pixel (i, j): p_s[3] and t. */
void orc_ray_sphere(const orc_camera* cam, const orc_aabb* box, double radius, int32_t i,
                    int32_t j, double p_s[3], double* t_hit, double o_n[3], double d_n[3]);

int32_t orc_background(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg,
                       const double* C_fg, const double* T_final, double* C, double* c_s);

int32_t orc_background_backward(const orc_camera* cam, const orc_fields* fl,
                                const orc_bg* bg, const double* T_final, const double* d_C,
                                double* d_C_fg, double* d_T_final, double* d_rad_table,
                                const orc_mlp_grad* d_col_mlp);

/* Smallest relative ReLU margin of the colour decoder evaluated for each
 * pixel's background (exact mode: at its sphere hit; map mode: the four
 * texels it samples). margin[H][W]. Diagnostic, like orc_decoder_margins. */
int32_t orc_bg_margins(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg,
                       double* margin);

/* ---------------- stage 7: loss (Eq. 12) -------------------------------- */
/* L = (1 - lambda) * mean|C - target| + lambda * (1 - SSIM(C, target)).
 * d_C receives dL/dC (overwritten, not accumulated). */
double orc_loss(int32_t width, int32_t height, const double* C, const double* target,
                double lambda, double* d_C);

/* SSIM alone (11x11 Gaussian window, sigma 1.5, zero padding), mean over
 * pixels and channels. */
double orc_ssim(int32_t width, int32_t height, const double* x, const double* y);

/* ---------------- 8-bit min-max codec of a grid (Sec. 4.4) -------------- */
/* Per level of per_level values: lo = min, step = (max - lo) / 255 (float),
 * code = rint((x - lo) / step) in [0, 255] (0 if step = 0); FP32 replay.
 * qparams [n_levels][2] = (lo, step); decoded (optional) = lo + step code
 * in FP64. */
int32_t orc_quantize_grid(int32_t n_levels, int64_t per_level, const float* table, uint8_t* codes,
                          float* qparams, double* decoded);

/* ---------------- training: Adam (Kingma & Ba, Algorithm 1) ------------- */
/* One Adam step of n parameters in place (3DGS and Instant-NGP train with
 * it; the paper keeps 3DGS's other hyper-parameters, Sec. 4.1). With
 * g = grad_scale * grad: m <- b1 m + (1 - b1) g; v <- b2 v + (1 - b2) g^2;
 * p <- p - lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps). */
int32_t orc_adam_step(int64_t n, double* p, const double* grad, double* m, double* v, double lr,
                      double b1, double b2, double eps, int32_t t, double grad_scale);

/* ---------------- training: adaptive density control (3DGS rules) ------ */
/* Statistics of one view, FP32 replay: for visible row i with ntiles > 0,
 * g = vis_ids[i]: accum[g] += sqrt((dm_x W/2)^2 + (dm_y H/2)^2) (each
 * product and sum rounded to float), count[g] += 1. */
int32_t orc_densify_stats(int32_t n, int32_t n_vis, const int32_t* vis_ids, const float* d_mean2d,
                          const int32_t* ntiles, int32_t width, int32_t height, float* accum,
                          int32_t* count);
/* Decision per Gaussian (0 keep, 1 prune, 2 clone, 3 split), FP32 replay of
 * the comparisons; row [n] (visible row or -1), offset [n + 1]. Returns the
 * new count. */
int64_t orc_densify_plan(int32_t n, int32_t n_vis, const int32_t* vis_ids, const float* alpha,
                         const float* scale, const float* accum, const int32_t* count, float grad_threshold,
                         float dense_scale, float min_opacity, uint8_t* action, int32_t* row,
                         int64_t* offset);
/* New arrays per the plan (FP64 positions of the split halves
 * p + R(q) (s * z_k)); kinds: 0 parameter, 1 optimiser state, 2 position,
 * 3 explicit scale logit. */
int32_t orc_densify_apply(int32_t n, const uint8_t* action, const int32_t* row, const int64_t* offset,
                          const double* scale, const double* quat, const double* noise,
                          double split_log_scale, int32_t width, int32_t kind, const double* src,
                          double* dst);

#ifdef __cplusplus
}
#endif
#endif
