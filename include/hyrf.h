/*
 * libhyrf: the HyRF render-and-train hot path (arXiv 2509.17083) as
 * hand-written sm_103a CUDA kernels behind a C ABI.
 *
 * One view is rendered and differentiated by five stages, each a forward call
 * and a backward call:
 *
 *   hyrf_query_fields          pre-cull + field query + aggregation  (Sec. 3.2-3.3, Eqs. 2-9)
 *   hyrf_project               EWA projection to screen space         (Sec. 3.2: "3DGS rasterizer")
 *   hyrf_bin_sort              tile binning + depth sort              (Sec. 3.1: Gaussians "ordered by depth")
 *   hyrf_rasterize             front-to-back alpha compositing        (Sec. 3.1, Eq. 1)
 *   hyrf_composite_background  neural background blend               (Sec. 3.3, Eqs. 10-11, App. A.2)
 *
 * plus the training loss of Sec. 3.4 (Eq. 12), hyrf_loss.
 *
 * Conventions shared by every call
 *   - Every pointer argument is a DEVICE pointer unless its comment says
 *     "host". The caller owns all memory; the library never allocates,
 *     frees or synchronises (except hyrf_read_status, which synchronises
 *     the given stream). Temporary storage is the caller's `workspace`
 *     (device, 256-byte aligned), at least hyrf_X_workspace_size(args)
 *     bytes; workspace contents need not be preserved between calls.
 *   - Arrays are contiguous and row-major. float32 unless stated.
 *   - All launches go to `stream` (a cudaStream_t, passed as void*), in
 *     order; no stage call reads device memory on the host, so the stage
 *     calls may be captured in a CUDA graph (this statement does not cover
 *     hyrf_bin_sort_noalloc).
 *   - Return value: HYRF_OK, or HYRF_ERR_INVALID_ARG / HYRF_ERR_UNSUPPORTED
 *     for arguments rejected on the host (nothing is launched), or
 *     HYRF_ERR_CUDA if a launch failed. Errors found on the device
 *     (capacity overflow, out-of-range input) are OR-ed into the optional
 *     `status` word (device int32, caller-zeroed) as HYRF_ERR_* bit flags
 *     and read back with hyrf_read_status. No call traps or prints.
 *   - Outputs marked "accumulate" are added to (caller zeroes them);
 *     all other outputs are overwritten.
 *   - Index spaces: N = number of Gaussians (full arrays), V = the visible
 *     subset produced by hyrf_query_fields (compacted arrays of capacity N,
 *     valid entries [0, *n_vis)), K = tile instances (capacity `capacity`).
 */
#ifndef HYRF_H
#define HYRF_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  HYRF_OK = 0,
  HYRF_ERR_INVALID_ARG = 1,
  HYRF_ERR_UNSUPPORTED = 2,
  HYRF_ERR_CUDA = 4,
  HYRF_ERR_OVERFLOW = 8,  /* device: more tile instances than `capacity` */
  HYRF_ERR_BOUNDS = 16,   /* device: an index read from memory was out of range */
  HYRF_ERR_TIMEOUT = 32,  /* device: a bounded wait on a tensor-core completion gave up */
} hyrf_status;

/* HYRF_F16 (grids and decoder weights; render only, the real-time path of
 * the paper's speed claims): IEEE half instead of bfloat16 operands. */
typedef enum { HYRF_F32 = 0, HYRF_BF16 = 1, HYRF_U8 = 2, HYRF_F16 = 3 } hyrf_dtype;

/* Pinhole camera, world to camera x_c = R x_w + t (Eq. 8). Pixel (i, j)
 * samples the image plane at (i + 0.5, j + 0.5); u = fx x_c/z_c + cx.
 * z_near: Gaussians with z_c <= z_near are culled ("too close", Sec. 3.3).
 * cull_tol: the tolerance band "tol" of Eq. 9, applied to normalised device
 * coordinates 2u/W - 1 and 2v/H - 1. Passed by value (host struct). */
typedef struct {
  float R[9];
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float z_near, cull_tol;
} hyrf_camera;

/* Multi-resolution hash grid (Eq. 3): table [n_levels][2^log2_T][n_feat] of
 * `dtype`. Level l has resolution floor(base_res * growth^l) and is stored
 * densely when its (res+1)^3 vertices fit in 2^log2_T entries, else
 * spatially hashed. n_feat must be 2. HYRF_U8 (render only; the 8-bit
 * min-max codec of the compressed model, Sec. 4.4): uint8 codes, value =
 * qparams[2 l] + qparams[2 l + 1] * code (see hyrf_quantize_grid). */
typedef struct {
  const void* table;
  int32_t n_levels, log2_T, n_feat, base_res;
  float growth;
  int32_t dtype;
  const float* qparams;      /* HYRF_U8: [n_levels][2] (lo, step) device; else NULL */
} hyrf_grid;

/* Decoder MLP (Eqs. 4, 6; Sec. 4.1): n_hidden ReLU layers of `width`, then a
 * linear output layer. W[0] [width][n_in], W[1] [width][width] (if
 * n_hidden = 2), W[n_hidden] [n_out][width], all of `dtype`; biases b[l]
 * float32. Supported: (n_hidden, width) in {(1, 32), (2, 64)}. */
typedef struct {
  const void* W[3];
  const float* b[3];
  int32_t n_in, width, n_hidden, n_out;
  int32_t dtype;
} hyrf_mlp;

/* The two decoupled fields of Sec. 3.2 with their decoders. box: the scene
 * box B0 mapped onto [-1,1]^3 before the contraction (App. A.1). The colour
 * decoder's input is [f_rad (n_levels*2), PE(dir) (3 + 6 pe_freq), zero
 * padding up to pe_pad]. geo_mlp.n_out = 8: (alpha_n, s_n[3], r_n[4]);
 * col_mlp.n_out = 3. */
typedef struct {
  float box_lo[3], box_hi[3];
  hyrf_grid geo, rad;
  hyrf_mlp geo_mlp, col_mlp;
  int32_t pe_freq, pe_pad;
} hyrf_fields;

/* float32 gradient buffers matching hyrf_fields (accumulate). Any pointer
 * may be NULL to skip that gradient. Tables [n_levels][2^log2_T][2]. */
typedef struct {
  float* geo_table;
  float* rad_table;
  float* geo_W[3];
  float* geo_b[3];
  float* col_W[3];
  float* col_b[3];
} hyrf_field_grads;

/* ------------------------------------------------------------------------
 * hyrf_query_fields: visibility pre-culling (Eqs. 8-9) of all N Gaussians,
 * ascending compaction of the kept ones (a negative cam.z_near keeps
 * Gaussians behind the camera too: the "w/o Pre-culling" ablation sets
 * z_near = -1e30 and a huge cull_tol to query every Gaussian), then for each
 * kept Gaussian the
 * contraction (Eq. 2), both hash encodings (Eq. 3), both decoders
 * (Eqs. 4-6) and the aggregation with the explicit parameters (Eq. 7).
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;                 /* N */
  const float* pos;          /* [N][3] p_e */
  const float* alpha_e;      /* [N] explicit opacity logit */
  const float* scale_e;      /* [N] explicit isotropic scale logit */
  const float* color_e;      /* [N][3] explicit colour logits */
  hyrf_camera cam;
  hyrf_fields fields;
  int32_t* vis_ids;          /* out [N]: ids of visible Gaussians, ascending, first *n_vis valid */
  int32_t* n_vis;            /* out [1] */
  float* alpha;              /* out [V] sigma(alpha_n + alpha_e) */
  float* scale;              /* out [V][3] sigma(s_n + s_e) */
  float* quat;               /* out [V][4] r_n / |r_n|, (w, x, y, z) */
  float* color;              /* out [V][3] sigma(c_n + c_e) */
  int32_t* status;           /* optional device status word */
  /* Optional out, BF16 fields only (must be NULL for float32 fields):
   * [2][N][32] bf16, 16-byte aligned, caller-owned. Row i of block 0 / 1
   * receives the geometry / radiance hash features (Eq. 3) of visible
   * Gaussian i. Passing the buffer on to hyrf_query_fields_backward saves
   * that call the gather (memory for time; NULL: the backward gathers). */
  void* features;
  /* Ablations of Tab. 5 ("w/o Neural", "w/o Explicit"): explicit_only = 1
   * skips the fields (alpha = sigma(alpha_e), scale = sigma(s_e) on all
   * three axes, rotation (1, 0, 0, 0), colour = sigma(c_e): isotropic,
   * diffuse 3DGS; `fields` is not read). NULL alpha_e / scale_e / color_e
   * mean zero explicit parts (neural only). 0 and non-NULL: HyRF. */
  int32_t explicit_only;
  /* 1: vis_ids / n_vis already hold this call's pre-culled set (from
   * hyrf_precull with the same n, pos and cam): the pre-cull is skipped. */
  int32_t vis_ready;
} hyrf_query_fields_args;

/* hyrf_precull: the pre-culling and ascending compaction of
 * hyrf_query_fields (Eqs. 8-9) as a call of its own, for callers that start
 * depth ordering (hyrf_depth_order) beside the field query, which then
 * takes vis_ready = 1. */
typedef struct {
  int32_t n;                 /* N */
  const float* pos;          /* [N][3] */
  hyrf_camera cam;
  int32_t* vis_ids;          /* out [N] */
  int32_t* n_vis;            /* out [1] */
} hyrf_precull_args;

size_t hyrf_precull_workspace_size(const hyrf_precull_args* a);
hyrf_status hyrf_precull(const hyrf_precull_args* a, void* workspace, size_t ws_bytes, void* stream);

size_t hyrf_query_fields_workspace_size(const hyrf_query_fields_args* a);
hyrf_status hyrf_query_fields(const hyrf_query_fields_args* a, void* workspace, size_t ws_bytes,
                              void* stream);

/* Reverse of hyrf_query_fields. Takes dL/d(alpha, scale, quat, color) of
 * the visible set and adds dL/d(pos, alpha_e, scale_e, color_e) at the
 * Gaussians' full indices and the field gradients (tables, weights,
 * biases). Decoder activations are recomputed, not stored. loss_scale
 * multiplies the upstream gradient inside the BF16 decoders and is divided
 * out again before anything is written (use 1 for the FP32 path). */
typedef struct {
  int32_t n;
  const float* pos;
  const float* alpha_e;
  const float* scale_e;
  const float* color_e;
  hyrf_camera cam;
  hyrf_fields fields;
  const int32_t* vis_ids;    /* [N] from the forward */
  const int32_t* n_vis;      /* [1] */
  const float* d_alpha;      /* [V] */
  const float* d_scale;      /* [V][3] */
  const float* d_quat;       /* [V][4] */
  const float* d_color;      /* [V][3] */
  float* d_pos;              /* accumulate [N][3] */
  float* d_alpha_e;          /* accumulate [N] */
  float* d_scale_e;          /* accumulate [N] */
  float* d_color_e;          /* accumulate [N][3] */
  hyrf_field_grads grads;    /* accumulate */
  float loss_scale;
  int32_t* status;
  /* Optional, BF16 fields only: the `features` buffer filled by the forward
   * call of the same view, with the tables unchanged since; NULL: the hash
   * features are gathered again. */
  const void* features;
  /* As in the forward. NULL d_alpha_e / d_scale_e / d_color_e (or explicit
   * inputs) skip those gradients. */
  int32_t explicit_only;
} hyrf_query_fields_backward_args;

size_t hyrf_query_fields_backward_workspace_size(const hyrf_query_fields_backward_args* a);
hyrf_status hyrf_query_fields_backward(const hyrf_query_fields_backward_args* a, void* workspace,
                                       size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_project: EWA splatting of the visible Gaussians (the 3DGS rasterizer
 * the paper builds on): Sigma = R_q diag(s)^2 R_q^T, J the perspective
 * Jacobian with the tangent clamped at 1.3 x the half field of view,
 * Sigma' = J R Sigma R^T J^T + 0.3 I, conic = Sigma'^-1, radius
 * ceil(3 sqrt(lambda_max)), and the half-open tile rectangle
 * [floor((u - r)/tile), floor((u + r)/tile) + 1) clamped to the grid.
 * Integer outputs follow a fixed FP32 operation order (no contraction), so
 * they are reproducible bit for bit; when |det Sigma'| < 1e-2 a c the conic
 * is recomputed in FP64 (fp64_flag = 1).
 * With `footprint` given, the binning is culled to the Gaussian's
 * opacity-aware footprint (Eq. 1 skips a pixel where o exp(-q/2) < 1/255,
 * q = d^T conic d): per tile row of the rectangle, only the tile columns
 * whose pixel centres meet the ellipse q <= t, t = 1.02 x 2 ln(255 o) +
 * 0.05 (o = alpha[i], or 1 when alpha is NULL; no tile when o < 1/255;
 * near-singular Gaussians keep their rectangle), and ntiles counts those.
 * Every dropped tile has alpha < 1/255 at each of its pixels, so the image
 * is unchanged. hyrf_bin_sort must then be given mean2d and footprint.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;                 /* N (capacity of the V arrays) */
  const float* pos;          /* [N][3] */
  const int32_t* vis_ids;    /* [N] */
  const int32_t* n_vis;      /* [1] */
  const float* scale;        /* [V][3] */
  const float* quat;         /* [V][4] */
  hyrf_camera cam;
  int32_t tile;              /* tile edge in pixels; must be 16 */
  float* mean2d;             /* out [V][2] */
  float* conic;              /* out [V][3] (a, b, c) of Sigma'^-1 */
  float* depth;              /* out [V] camera-space z */
  int32_t* rect;             /* out [V][4] (x0, y0, x1, y1) in tiles, half-open */
  int32_t* ntiles;           /* out [V] (x1-x0)(y1-y0), 0 if empty; the footprint's tile count with `footprint` */
  uint8_t* fp64_flag;        /* out [V], may be NULL */
  int32_t* status;
  const float* alpha;        /* [V] opacity for the footprint; may be NULL (o = 1) */
  float* footprint;          /* out [V][12], 16-byte aligned; NULL: no culling. Per row:
                              * (Sigma'_xx, Sigma'_xy, Sigma'_yy, t), then eight 32-bit words
                              * of row spans when the rectangle has at most 16 rows and 255
                              * columns (row j: word j/2, bits 16 (j%2) on; low byte = first
                              * tile column - x0, high byte = length), zeros otherwise */
} hyrf_project_args;

size_t hyrf_project_workspace_size(const hyrf_project_args* a);
hyrf_status hyrf_project(const hyrf_project_args* a, void* workspace, size_t ws_bytes,
                         void* stream);

/* Reverse of hyrf_project: dL/d(mean2d, conic) -> dL/dpos (accumulate at
 * full index), dL/dscale and dL/dquat (overwrite, [V]). */
typedef struct {
  int32_t n;
  const float* pos;
  const int32_t* vis_ids;
  const int32_t* n_vis;
  const float* scale;
  const float* quat;
  hyrf_camera cam;
  const float* d_mean2d;     /* [V][2] */
  const float* d_conic;      /* [V][3] */
  float* d_pos;              /* accumulate [N][3] */
  float* d_scale;            /* out [V][3] */
  float* d_quat;             /* out [V][4] */
  int32_t* status;
} hyrf_project_backward_args;

size_t hyrf_project_backward_workspace_size(const hyrf_project_backward_args* a);
hyrf_status hyrf_project_backward(const hyrf_project_backward_args* a, void* workspace,
                                  size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_bin_sort: tile instances of every visible Gaussian (one per tile of
 * its rectangle, or of its footprint when mean2d and footprint are given
 * (see hyrf_project), emitted in (Gaussian, tile row-major) order), ordered by
 * the 64-bit key (tile << 32) | float_bits(depth) with a stable LSD radix
 * sort, and the per-tile [start, end) ranges. The 32 depth bits are sorted
 * on the V Gaussians before the instances are emitted (identical result to
 * sorting the instances on them: a Gaussian's instances share its depth and
 * are contiguous), the tile bits on the K instances.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;                 /* N (capacity of the V arrays) */
  const int32_t* n_vis;      /* [1] */
  const int32_t* rect;       /* [V][4] */
  const int32_t* ntiles;     /* [V] */
  const float* depth;        /* [V] (> 0) */
  int32_t tiles_x, tiles_y;
  int64_t capacity;          /* capacity of keys / vals */
  uint64_t* keys;            /* out [capacity] sort keys, may be NULL */
  int32_t* vals;             /* out [capacity] visible index per instance */
  int32_t* ranges;           /* out [tiles_y*tiles_x][2] */
  int32_t* n_instances;      /* out [1] K (clamped to capacity; HYRF_ERR_OVERFLOW if above) */
  int32_t* status;
  /* Optional [V]: the visible rows in depth order from hyrf_depth_order
   * (same camera and visible set); the call then skips its own depth sort
   * (the result is identical). NULL: sorted here. */
  const int32_t* depth_order;
  /* Optional, together: mean2d [V][2] and footprint [V][12] from
   * hyrf_project (with ntiles counted on the footprint); each rectangle row
   * then yields only its footprint's tile columns. NULL: whole rectangles. */
  const float* mean2d;
  const float* footprint;
} hyrf_bin_sort_args;

/* hyrf_depth_order: the visible rows ordered by camera-space depth exactly
 * as hyrf_bin_sort orders them (keys: the FP32 depth z of hyrf_project,
 * computed with the same operations from the positions; stable, ties by
 * visible index). It needs only the positions, so it can run beside the
 * field query (which the projection's rectangles need); hyrf_bin_sort then
 * takes the result in depth_order. order[V] out. */
typedef struct {
  int32_t n;                 /* N (capacity) */
  const float* pos;          /* [N][3] */
  const int32_t* vis_ids;    /* [N] */
  const int32_t* n_vis;      /* [1] */
  hyrf_camera cam;
  int32_t* order;            /* out [N]: first *n_vis valid */
  int32_t* status;
} hyrf_depth_order_args;

size_t hyrf_depth_order_workspace_size(const hyrf_depth_order_args* a);
hyrf_status hyrf_depth_order(const hyrf_depth_order_args* a, void* workspace, size_t ws_bytes, void* stream);

size_t hyrf_bin_sort_workspace_size(const hyrf_bin_sort_args* a);
hyrf_status hyrf_bin_sort(const hyrf_bin_sort_args* a, void* workspace, size_t ws_bytes,
                          void* stream);
/* Binning is discrete: its reverse only validates the arguments. */
hyrf_status hyrf_bin_sort_backward(const hyrf_bin_sort_args* a, void* workspace, size_t ws_bytes,
                                   void* stream);

/* hyrf_bin_sort without a caller workspace. The paper has no counterpart:
 * this entry point exists for callers that cannot allocate device memory
 * themselves, such as a host program that links this library through its C
 * interface without any device allocator of its own, or one that must not
 * call cudaMalloc while it runs (the call can synchronise the device and can
 * fail under a memory budget fixed up front). It computes exactly what
 * hyrf_bin_sort computes, with the same arguments and outputs (all still
 * caller-provided), but takes its temporary storage from one fixed array of
 * HYRF_NOALLOC_SCRATCH_BYTES in device memory that the library declares;
 * every GPU that loads the library holds that array until the process exits.
 * It never calls cudaMalloc, cudaFree or any other allocating routine.
 *   - Limits: a->n <= HYRF_NOALLOC_MAX_GAUSSIANS and a->capacity <=
 *     HYRF_NOALLOC_MAX_INSTANCES; larger requests return
 *     HYRF_ERR_INVALID_ARG and launch nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current).
 *   - All calls share the one array, which keeps whatever the last call left
 *     in it (no part of it is read before a call writes it). Calls whose
 *     work overlaps on the GPU (other streams, other host threads) race on
 *     it: order them, e.g. on one stream. */
#define HYRF_NOALLOC_MAX_GAUSSIANS 65536
#define HYRF_NOALLOC_MAX_INSTANCES 262144
#define HYRF_NOALLOC_SCRATCH_BYTES 4718592
hyrf_status hyrf_bin_sort_noalloc(const hyrf_bin_sort_args* a, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_rasterize: per 16x16 tile, front-to-back compositing of Eq. 1:
 * alpha_i = min(0.99, o_i exp(-1/2 d^T conic d)), skipped if < 1/255;
 * a pixel stops before T (1 - alpha) < 1e-4.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;                 /* N (capacity of the V arrays) */
  const int32_t* n_vis;
  const int32_t* ranges;     /* [tiles][2] */
  const int32_t* vals;       /* [K] */
  const float* mean2d;       /* [V][2] */
  const float* conic;        /* [V][3] */
  const float* alpha;        /* [V] opacity */
  const float* color;        /* [V][3] */
  int32_t width, height, tile;
  float* C_fg;               /* out [H][W][3] */
  float* T_final;            /* out [H][W] */
  int32_t* n_contrib;        /* out [H][W] list position of the last contributor + 1 */
  int32_t* status;
  /* Optional [tiles] permutation of the tile indices: the order in which
   * the CTAs take the tiles (the result does not depend on it). NULL:
   * index order in the forward; the reverse then orders the tiles itself
   * (longest pixel list first, from n_contrib). A forward given the order
   * that hyrf_tile_order computed from a previous frame's n_contrib runs
   * its long tiles first; the reverse given the order of this frame's
   * n_contrib skips computing it. Entries outside [0, tiles) set
   * HYRF_ERR_BOUNDS and are skipped. */
  const int32_t* tile_order;
  /* Optional [N][12] float, 16-byte aligned: the per-Gaussian records the
   * compositing reads (mean2d, conic, opacity, colour and the exponent
   * bound of the opacity test). NULL: each call packs them into its
   * workspace. Given, the forward packs them here and the reverse given
   * the same pointer reads them instead of packing again: between the two
   * calls mean2d, conic, alpha and color must not change. */
  float* records;
} hyrf_rasterize_args;

size_t hyrf_rasterize_workspace_size(const hyrf_rasterize_args* a);
hyrf_status hyrf_rasterize(const hyrf_rasterize_args* a, void* workspace, size_t ws_bytes,
                           void* stream);

/* Tile order for hyrf_rasterize(_backward): the tiles by decreasing bit
 * length of their longest pixel list (n_contrib of a forward); order[tiles]
 * out, a permutation (order inside a class of equal length unspecified). */
typedef struct {
  int32_t width, height, tile;
  const int32_t* n_contrib;  /* [H][W] */
  int32_t* order;            /* out [tiles] */
} hyrf_tile_order_args;

size_t hyrf_tile_order_workspace_size(const hyrf_tile_order_args* a);
hyrf_status hyrf_tile_order(const hyrf_tile_order_args* a, void* workspace, size_t ws_bytes, void* stream);

/* Reverse of hyrf_rasterize, back to front, recovering T from T_final:
 * dL/d(C_fg, T_final) -> dL/d(mean2d, conic, alpha, color) (accumulate). */
typedef struct {
  hyrf_rasterize_args fwd;   /* the forward's arguments; its outputs are inputs here */
  const float* d_C_fg;       /* [H][W][3] */
  const float* d_T_final;    /* [H][W], or NULL with C below */
  float* d_mean2d;           /* accumulate [V][2] */
  float* d_conic;            /* accumulate [V][3] */
  float* d_alpha;            /* accumulate [V] */
  float* d_color;            /* accumulate [V][3] */
  /* Optional (used when d_T_final is NULL): the composited image C of
   * hyrf_composite_background, [H][W][3]. Eq. 11 gives C - C_fg =
   * T_final c_s, so dL/dT_final T_final = dL/dC . (C - C_fg) per pixel
   * (d_C_fg = dL/dC) and this call need not wait for the background's
   * reverse, which may then run on another stream with its d_T_final
   * NULL. The product is formed from the rounded C (absolute error of a
   * few ulp of C). */
  const float* C;
} hyrf_rasterize_backward_args;

size_t hyrf_rasterize_backward_workspace_size(const hyrf_rasterize_backward_args* a);
hyrf_status hyrf_rasterize_backward(const hyrf_rasterize_backward_args* a, void* workspace,
                                    size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_composite_background: for each pixel, the ray o + t d hits the
 * sphere |x| = radius (centred at the origin of the normalised box space,
 * App. A.2; positive root); the colour c_s = sigma(dec(enc(contract(p_s);
 * Theta_rad) (+) PE(d); Phi_c)) and C = C_fg + T_final c_s (Eqs. 10-11).
 * mode 0 queries the field per pixel; mode 1 evaluates it on a map_h x
 * map_w equirectangular map of directions and samples it bilinearly.
 * ---------------------------------------------------------------------- */
/* mode 2: no background (Tab. 5 "w/o Background"): C = C_fg, and the
 * reverse gives dL/dC_fg = dL/dC, dL/dT_final = 0, no field gradients.
 * tau_T > 0 (mode 0, BF16 fields, forward only): the paper's render-time
 * rule (Sec. 3.4, tau_T = 0.2 in its experiments) queries the background
 * only at pixels with T_final >= tau_T; elsewhere C = C_fg. A reverse call
 * with tau_T > 0 is rejected (training composites the background
 * everywhere). */
typedef struct {
  int32_t mode, map_h, map_w;
  float radius;
  float tau_T;
} hyrf_background;

typedef struct {
  hyrf_camera cam;
  hyrf_fields fields;        /* rad grid and col_mlp are used */
  hyrf_background bg;
  const float* C_fg;         /* [H][W][3] */
  const float* T_final;      /* [H][W] */
  float* C;                  /* out [H][W][3] */
  int32_t* status;
  /* Optional, mode 0 with BF16 fields only (NULL otherwise): [H*W][32]
   * bf16, 16-byte aligned, caller-owned. The forward writes the radiance
   * hash features of every pixel's sphere hit; the backward, which gets
   * these arguments as `fwd`, reads them instead of gathering again (the
   * buffer must still hold the forward's values). A forward with
   * bg.tau_T > 0 does not write it. */
  void* features;
  /* 1: `features` already holds this view's features (filled by
   * hyrf_gather_background, e.g. on another stream while the foreground is
   * rendered): the forward skips its gather. */
  int32_t features_ready;
} hyrf_composite_background_args;

size_t hyrf_composite_background_workspace_size(const hyrf_composite_background_args* a);
/* The radiance hash features of every pixel's sphere hit into a->features
 * (mode 0, BF16 fields, tau_T = 0): the gather of hyrf_composite_background,
 * callable ahead of it (it reads neither C_fg nor T_final). */
hyrf_status hyrf_gather_background(const hyrf_composite_background_args* a, void* stream);
hyrf_status hyrf_composite_background(const hyrf_composite_background_args* a, void* workspace,
                                      size_t ws_bytes, void* stream);

/* Reverse: dL/dC -> dL/dT_final (out; may be NULL when the compositing
 * reverse takes the composited image instead, see
 * hyrf_rasterize_backward_args.C), dL/dC_fg (out, = dL/dC; may be NULL
 * when the caller passes dL/dC on as dL/dC_fg) and the radiance-field and
 * colour-decoder gradients (accumulate, into grads.rad_table / col_*;
 * decoder gradients are added atomically, so another call accumulating
 * into the same buffers may run concurrently on another stream). */
typedef struct {
  hyrf_composite_background_args fwd;
  const float* d_C;          /* [H][W][3] */
  float* d_C_fg;             /* out [H][W][3], may be NULL */
  float* d_T_final;          /* out [H][W], may be NULL */
  hyrf_field_grads grads;    /* accumulate */
  float loss_scale;
  /* Optional (BF16 exact mode): a second stream for the radiance-table
   * gradient scatter, which then runs after this call's decoder work (an
   * event orders it) and concurrently with whatever the caller issues next
   * on `stream`. The caller must order its use of grads.rad_table after
   * scatter_stream (e.g. make `stream` wait on it). */
  void* scatter_stream;
} hyrf_composite_background_backward_args;

size_t hyrf_composite_background_backward_workspace_size(
    const hyrf_composite_background_backward_args* a);
hyrf_status hyrf_composite_background_backward(const hyrf_composite_background_backward_args* a,
                                               void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_loss: Eq. 12, L = (1 - lambda) mean|C - target| + lambda (1 - SSIM)
 * with an 11x11 Gaussian window (sigma 1.5, zero padding), means over all
 * pixels and channels. Writes L to *loss and, if d_C is not NULL,
 * grad_scale * dL/dC to d_C.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t width, height;
  const float* C;            /* [H][W][3] */
  const float* target;       /* [H][W][3] */
  float lambda;
  float grad_scale;
  float* loss;               /* out [1] */
  float* d_C;                /* out [H][W][3], may be NULL */
} hyrf_loss_args;

size_t hyrf_loss_workspace_size(const hyrf_loss_args* a);
hyrf_status hyrf_loss(const hyrf_loss_args* a, void* workspace, size_t ws_bytes, void* stream);

/* ------------------------------------------------------------------------
 * hyrf_adam_step: one Adam update (Kingma & Ba) of a list of float32
 * parameter tensors, the optimiser the paper inherits from 3DGS for the
 * explicit parameters and from Instant-NGP for the fields (Sec. 4.1: "other
 * hyperparameters as 3DGS"). Per element, with g = grad_scale * grad:
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   p -= lr * lr_scale * (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps),
 * then, if `shadow` is set, shadow = bf16(p) (round to nearest even): the
 * working copy of a BF16 table or weight matrix whose float32 master is p.
 * All tensors are updated by one launch (at most HYRF_ADAM_MAX_TENSORS per
 * call). Pointers are device pointers to n contiguous elements, 16-byte
 * aligned; m and v are caller-owned state (zero before the first step).
 * Errors: HYRF_ERR_INVALID_ARG for a bad count, hyper-parameter or pointer.
 * ---------------------------------------------------------------------- */
/* ------------------------------------------------------------------------
 * Adaptive density control. The paper keeps 3DGS's schedule (Sec. 3.3 end:
 * periodic reset of the explicit opacity, pruning of low-opacity Gaussians;
 * densification "as the original 3DGS", Sec. 2 and Sec. 4.1). Three calls:
 *
 * hyrf_densify_stats, after a view's reverse pass: for every visible
 * Gaussian with at least one tile, accum[g] += |dL/d mean2d| measured in
 * NDC units (the pixel-space gradient times (W/2, H/2)) and count[g] += 1.
 *
 * hyrf_densify_plan: one action per Gaussian g (the visible rows of the last
 * hyrf_query_fields give its opacity and scale; other Gaussians are kept):
 *   prune  (HYRF_DENSIFY_PRUNE) if opacity < min_opacity, else if
 *   count > 0 and accum / count >= grad_threshold:
 *     split (HYRF_DENSIFY_SPLIT) if max(scale) > dense_scale, else
 *     clone (HYRF_DENSIFY_CLONE); otherwise keep.
 * It writes action [N], row [N] (the visible row of g, or -1), offset
 * [N + 1] (exclusive scan of the output multiplicity 1 / 0 / 2 / 2) and
 * *n_out = offset[N] (device). The caller reads n_out to size the new arrays.
 *
 * hyrf_densify_apply: writes the new per-Gaussian arrays. Gaussian g's
 * outputs start at offset[g], in the old order: kept -> 1 copy; clone -> the
 * original then an identical copy; split -> two Gaussians at
 * p + R(q) (s * z_k) (z_k = noise[g][k][0..3), k = 0, 1, the visible row's
 * scale s and rotation q) whose explicit scale logit is lowered by
 * split_log_scale (ln 1.6 shrinks small scales by 1.6, as 3DGS's 1 / (0.8 x 2)).
 * Optimiser state arrays (kind HYRF_REMAP_STATE) start at zero for every new
 * Gaussian (clone copies, both split halves) and keep their values for kept
 * Gaussians and clone originals.
 * ---------------------------------------------------------------------- */
#define HYRF_DENSIFY_KEEP 0
#define HYRF_DENSIFY_PRUNE 1
#define HYRF_DENSIFY_CLONE 2
#define HYRF_DENSIFY_SPLIT 3
#define HYRF_REMAP_MAX 24
#define HYRF_REMAP_PARAM 0      /* copied (clone: both) */
#define HYRF_REMAP_STATE 1      /* copied for kept / clone originals, zero for new Gaussians */
#define HYRF_REMAP_POSITION 2   /* width 3; split halves are sampled */
#define HYRF_REMAP_SCALE_LOGIT 3 /* width 1; split halves lowered by split_log_scale */

typedef struct {
  int32_t n;
  const int32_t* vis_ids;    /* [N] */
  const int32_t* n_vis;      /* [1] */
  const float* d_mean2d;     /* [V][2] pixel units, from hyrf_rasterize_backward */
  const int32_t* ntiles;     /* [V] from hyrf_project */
  int32_t width, height;
  float* accum;              /* [N] accumulate */
  int32_t* count;            /* [N] accumulate */
} hyrf_densify_stats_args;

hyrf_status hyrf_densify_stats(const hyrf_densify_stats_args* a, void* stream);

typedef struct {
  int32_t n;
  const int32_t* vis_ids;    /* [N] */
  const int32_t* n_vis;      /* [1] */
  const float* alpha;        /* [V] opacity of the visible rows */
  const float* scale;        /* [V][3] */
  const float* accum;        /* [N] */
  const int32_t* count;      /* [N] */
  float grad_threshold, dense_scale, min_opacity;
  uint8_t* action;           /* out [N] */
  int32_t* row;              /* out [N] */
  int64_t* offset;           /* out [N + 1] */
  int64_t* n_out;            /* out [1] */
} hyrf_densify_plan_args;

size_t hyrf_densify_plan_workspace_size(const hyrf_densify_plan_args* a);
hyrf_status hyrf_densify_plan(const hyrf_densify_plan_args* a, void* workspace, size_t ws_bytes,
                              void* stream);

typedef struct {
  const float* src;          /* [N][width] */
  float* dst;                /* [n_out][width] */
  int32_t width;             /* 1..4 */
  int32_t kind;              /* HYRF_REMAP_* */
} hyrf_remap_array;

typedef struct {
  int32_t n;
  const uint8_t* action;     /* [N] from the plan */
  const int32_t* row;        /* [N] */
  const int64_t* offset;     /* [N + 1] */
  const float* scale;        /* [V][3] of the visible rows */
  const float* quat;         /* [V][4] */
  const float* noise;        /* [N][2][3] standard normal draws (caller-drawn) */
  float split_log_scale;
  int32_t n_arrays;
  hyrf_remap_array arrays[HYRF_REMAP_MAX];
} hyrf_densify_apply_args;

hyrf_status hyrf_densify_apply(const hyrf_densify_apply_args* a, void* stream);

/* hyrf_reset_opacity: the periodic reset of the explicit opacity (Sec. 3.3
 * end): alpha_e[g] = min(alpha_e[g], max_logit) for all n Gaussians (3DGS
 * resets to opacity 0.01, max_logit = logit(0.01)); the Adam moments of
 * alpha_e (m, v; may be NULL) restart from zero. */
hyrf_status hyrf_reset_opacity(float* alpha_e, int64_t n, float max_logit, float* m, float* v,
                               void* stream);

/* hyrf_quantize_grid: the 8-bit min-max codec of a hash table (Sec. 4.4's
 * compressed model quantises the grids). Per level l over its T x 2 values:
 * lo = min, hi = max, step = (hi - lo) / 255 (float), code = rint((x - lo)
 * / step) clamped to [0, 255] (0 when step = 0). table: [n_levels][T][2]
 * float32, bf16 or f16 (dtype); codes [n_levels][T][2]
 * uint8 out; qparams [n_levels][2] float32 out. */
hyrf_status hyrf_quantize_grid(const void* table, int32_t dtype, int32_t n_levels, int32_t log2_T,
                               uint8_t* codes, float* qparams, void* stream);

/* ------------------------------------------------------------------------
 * Storage order (no counterpart in the paper; a data-layout step of this
 * library). hyrf_spatial_order: perm[k] = the Gaussian that comes k-th in
 * the Morton (Z-curve) order of its contracted position (App. A.1, Eq. 2)
 * quantised to 10 bits per axis; ties keep the input order. Storing the
 * Gaussians in this order puts neighbours next to each other, so the hash
 * gathers and scatters of consecutive rows share cache lines.
 * hyrf_permute_rows: dst[k] = src[perm[k]] for every array (width floats
 * per row; kind ignored), count <= HYRF_REMAP_MAX.
 * ---------------------------------------------------------------------- */
typedef struct {
  int32_t n;
  const float* pos;          /* [N][3] */
  float box_lo[3], box_hi[3];
  int32_t* perm;             /* out [N] */
} hyrf_spatial_order_args;

size_t hyrf_spatial_order_workspace_size(const hyrf_spatial_order_args* a);
hyrf_status hyrf_spatial_order(const hyrf_spatial_order_args* a, void* workspace, size_t ws_bytes,
                               void* stream);
hyrf_status hyrf_permute_rows(const int32_t* perm, int32_t n, const hyrf_remap_array* arrays, int32_t count,
                              void* stream);

#define HYRF_ADAM_MAX_TENSORS 32
typedef struct {
  float* param;              /* [n] float32 master values, updated in place */
  const float* grad;         /* [n] float32 */
  float* m;                  /* [n] float32 first moment */
  float* v;                  /* [n] float32 second moment */
  void* shadow;              /* optional [n] bf16 working copy, or NULL */
  int64_t n;
  float lr_scale;            /* multiplies lr for this tensor */
} hyrf_adam_tensor;

typedef struct {
  float lr, beta1, beta2, eps;
  int32_t step;              /* t >= 1, for the bias corrections */
  float grad_scale;
} hyrf_adam_hparams;

hyrf_status hyrf_adam_step(const hyrf_adam_tensor* tensors, int32_t count,
                           const hyrf_adam_hparams* hp, void* stream);

/* ------------------------------------------------------------------------ */
/* Synchronises `stream`, copies the device status word to *host_out (host
 * pointer) and returns it as hyrf_status bits (HYRF_ERR_CUDA if the copy
 * failed). */
hyrf_status hyrf_read_status(const int32_t* status, void* stream, int32_t* host_out);
const char* hyrf_error_string(int32_t status);
/* Check of the library's bounded waits: one CTA waits on an mbarrier that
 * nothing completes, polling it `polls` times as the tensor-core kernels
 * poll their completion barriers (there 2^24 times), then gives up the
 * way they do: HYRF_ERR_TIMEOUT is OR-ed into *status (device word) and the
 * kernel returns, leaving the context usable. polls in [1, 2^24]. */
hyrf_status hyrf_check_bounded_wait(int32_t* status, uint32_t polls, void* stream);
/* Number of kernel launches issued by this library since load (host
 * counter; for launch accounting in benchmarks). */
uint64_t hyrf_launch_count(void);

/* Kernel timer (measurement support; the paper has no counterpart). While
 * enabled, every kernel launch of this library records a pair of CUDA events
 * on its own launching stream around the launch; launches issued while that
 * stream is being captured into a CUDA graph are not timed. The events are
 * library-owned and reused. hyrf_timer_read waits for every recorded pair,
 * writes at most `max_entries` per-kernel totals to `out` (host array owned
 * by the caller; `name` points to a static string of the library), clears
 * the totals and returns the number of distinct kernels seen (which may
 * exceed max_entries). Timing adds two event records per launch. Not
 * thread-safe against concurrent launches from other host threads while
 * enabled or read. */
typedef struct {
  const char* name;
  uint64_t launches;
  double total_ms;
} hyrf_kernel_time;
void hyrf_timer_enable(int on);
int hyrf_timer_read(hyrf_kernel_time* out, int max_entries);

#ifdef __cplusplus
}
#endif
#endif
