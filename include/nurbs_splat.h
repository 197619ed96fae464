/*
 * nurbs_splat.h -- C ABI of the NURBS Splatting hot path (sm_103a).
 *
 * The path turns planar NURBS curves into isotropic Gaussians and splats them,
 * forward and backward:
 *
 *   nurbs_sample    curves -> Gaussians: contour samples along open and closed
 *                   strokes (§3.2, Eq. 1-5) and SDF-modulated fill inside
 *                   closed filled curves (§3.3, Eq. 6-7, Eq. S1-S3)
 *   splat_forward   Gaussians -> image: tile binning, a sort by (tile, layer,
 *                   sample) and per-tile front-to-back compositing (§3.4, Eq. 8-9)
 *   splat_backward  dL/dimage -> gradients of control points, rational weights,
 *                   knot intervals, widths, colours and opacities (§3.5)
 *
 * Conventions shared by every entry point
 *   - Pointers named in a struct or argument as "device" point to GPU memory
 *     the caller owns; the library never allocates, frees or keeps them.
 *   - `stream` is a cudaStream_t passed as void*.  Every call only enqueues
 *     work on it and returns without synchronising, except ns_poll_status.
 *   - Scalar arguments are checked on the host: a bad one returns
 *     NS_ERR_INVALID_ARG before anything is enqueued, and ns_last_error()
 *     says which.  Per-curve data lives on the device and is checked there:
 *     a bad curve emits no Gaussians and raises a device status that
 *     ns_poll_status reports.  Nothing aborts, traps or waits without bound.
 *   - Sizes that depend on the data (Gaussians, boundary points, tile pairs)
 *     are bounded by the capacities in ns_capacity.  Work beyond a capacity
 *     is dropped (never written out of bounds) and NS_ERR_CAPACITY is raised
 *     with the size that would have been needed.
 *   - Coordinates are pixels; pixel (x, y) is sampled at (x + 1/2, y + 1/2);
 *     y grows downwards.  Images are float32 [n_scenes, height, width, channels].
 *   - The library's kernels are launched with programmatic stream
 *     serialization (programmatic dependent launch): each begins by waiting
 *     for the kernel before it in the stream, so results and the order of
 *     memory effects are those of a plain stream.  Setting the environment
 *     variable NS_PDL=0 before the first call launches them without it.
 */
#ifndef NURBS_SPLAT_H
#define NURBS_SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  NS_OK = 0,
  NS_ERR_INVALID_ARG = 1,   /* host-side argument check failed */
  NS_ERR_CAPACITY = 2,      /* a data-dependent size exceeded its capacity */
  NS_ERR_INVALID_CURVE = 3, /* a curve's degree, key count or interval count is inconsistent */
  NS_ERR_CUDA = 4           /* a CUDA launch or copy failed */
} ns_status;

#define NS_CLOSED 1 /* curve flag: closed (periodic) curve */
#define NS_FILLED 2 /* curve flag: closed curve whose interior is filled */
#define NS_MAX_DEGREE 5

/*
 * A batch of scenes and their curves (§3.1).  All scenes share one image size.
 * Curves are grouped by scene and listed back to front inside a scene
 * (painter's order: the last curve of a scene is in front).
 *
 * Key points are the learnable parameters (§3.1): an open curve of degree p
 * with n_k key points uses them as its n_k control points and stores n_k - p
 * knot intervals; a closed curve wraps the last ceil(p/2) and first floor(p/2)
 * key points into n_k + p control points and stores n_k core knot intervals.
 * The width s is the control points' third coordinate (§3.1, last paragraph).
 */
typedef struct {
  int32_t n_scenes, n_curves, n_keys, n_taus;
  int32_t height, width, channels;     /* channels: 1 or 3 (first colour components) */
  const int32_t* scene_curve_offset;   /* device [n_scenes+1]; NULL: one scene holds all curves */
  const int32_t* degree;               /* device [n_curves], 1..NS_MAX_DEGREE */
  const int32_t* flags;                /* device [n_curves], NS_CLOSED | NS_FILLED */
  const int32_t* key_offset;           /* device [n_curves+1], CSR into key */
  const int32_t* tau_offset;           /* device [n_curves+1], CSR into tau */
  const float* key;                    /* device [n_keys*4]: {x, y, s, w} per key point */
  const float* tau;                    /* device [n_taus]: knot intervals, >= 0 */
  const float* color;                  /* device [n_curves*4]: {r, g, b, opacity} */
  /* Host-side hint, optional: 0 = not given.  Otherwise bit 0 is set and bit p
   * (1..NS_MAX_DEGREE) is set for every degree p among the curves that are not
   * filled (strokes).  splat_backward then launches the contour-chain kernels
   * of those degrees only (one per degree; none for a batch of fills), and
   * nurbs_sample no stroke sampling kernel for a batch of fills.  A
   * stroke whose degree's bit is clear while bit 0 is set is reported by
   * nurbs_sample as an invalid curve (NS_ERR_INVALID_CURVE, bad_curve). */
  int32_t stroke_degrees;
} ns_curves;

/* Sampling settings (§3.2, §3.3; defaults of Table S1 from ns_default_sample_params). */
typedef struct {
  float delta_c;    /* contour density: M = ceil(delta_c L) samples (§3.2) */
  float rho;        /* sigma = s / rho for contours, eta h / rho for fills (Eq. 5, 6) */
  float delta_b;    /* boundary density: ceil(delta_b L) polyline points (§3.3) */
  float h;          /* fill grid step in pixels (Eq. 6) */
  float eta;        /* fill coverage factor (Eq. 6) */
  float gamma;      /* sigmoid sharpness of the fill opacity (Eq. 7) */
  float pad_frac;   /* padding of the boundary's box, fraction of its extent */
  int32_t kappa;    /* endpoint replicas of open curves (§3.2, last paragraph) */
  int32_t nl_mult;  /* N_L = nl_mult * max(width, height) arc-length nodes (Eq. 3) */
  int32_t fill_rule;/* 0: inside iff winding number > 0.5 (Eq. S3); 1: nonzero */
  float fill_cull;  /* > 0: fill points provably outside with opacity below this
                       value (pass the rasterizer's alpha_min) get opacity 0 without
                       an exact distance; they bin to no tile either way.  0: off */
  int32_t contour_mode; /* 0: isotropic contour Gaussians (Eq. 5, the paper's method);
                       1: tangent-aligned (the paper's anisotropic prototype): each
                       contour Gaussian is stretched along the unit tangent
                       C'_xy/|C'_xy| (Eq. 2) with sigma_t = |C'_xy| du / rho, du the
                       parameter step between samples, and keeps sigma_n = s / rho
                       across; the Gaussian set then needs `shape` */
  int32_t fill_tile;  /* fill Gaussians per sampling block: the signed distance and the
                       fill chain run one block per fill_tile x fill_tile tile of a
                       curve's grid, 8 or 16 (64 or 256 Gaussians); 0 = 16.  Changes
                       no result, only the work decomposition */
} ns_sample_params;

/* Blend decomposition flag for ns_raster_params.ppt_fwd / ppt_bwd: with it,
 * each warp's 8-column sub-block is split into four groups of eight lanes, two
 * pixel columns each, and every group walks only the Gaussians that can reach
 * its own pixels (pixels per thread 1 or 2).  Pays off for Gaussians much
 * smaller than the sub-block, such as fill Gaussians at grid step 1 px. */
#define NS_BLEND_LANE_GROUPS 16

/* Rasterizer settings (§3.4). */
typedef struct {
  int32_t tile;     /* tile edge in pixels: 8, 16 or 32 */
  float k_sigma;    /* a Gaussian is binned to the tiles of mu +- k_sigma sigma */
  float alpha_min;  /* a Gaussian with alpha < alpha_min at a pixel is skipped there */
  float alpha_max;  /* alpha is capped at alpha_max (keeps 1 - alpha > 0) */
  float t_min;      /* compositing stops before transmittance would drop below t_min */
  float bg[3];      /* background colour behind the residual transmittance (§3.4) */
  int32_t ppt_fwd;  /* decomposition of the forward blend: pixels per thread 1, 2 or 4 (4 needs
                       tile >= 16), or 1 or 2 plus NS_BLEND_LANE_GROUPS; 0 = default */
  int32_t ppt_bwd;  /* the same for the backward blend; neither changes any result */
  int32_t fill_layers; /* 1: the Gaussians of a filled curve, which lie on its grid (§3.3), are
                          binned as one tile pair per tile their bin rectangles cover, and the blend
                          kernels find the grid points that can reach a pixel by index arithmetic.
                          Every pixel composites the same Gaussians in the same order as with 0
                          (one pair per Gaussian and tile), so images are identical; gradients
                          differ only in the order of float additions.  Needs a Gaussian set
                          written by nurbs_sample into the same workspace, and tile 8 or 16 (or
                          tile 32 with 4 pixels per thread); the decomposition falls back to one
                          of those when needed.  0: one pair per Gaussian and tile. */
} ns_raster_params;

/* Capacities that bound the data-dependent sizes. */
typedef struct {
  int64_t gaussians;  /* Gaussian records */
  int64_t pairs;      /* (tile, Gaussian) pairs */
  int64_t boundary;   /* boundary polyline points of filled curves */
} ns_capacity;

/*
 * A Gaussian set, caller-owned device memory of `capacity` records.  Records
 * are stored front to back inside each scene: scene ascending, then curve
 * from the last (front) to the first, then sample index ascending.
 */
typedef struct {
  int64_t capacity;
  float* rec;       /* device [capacity*4]: {mu_x, mu_y, sigma, opacity} */
  int32_t* curve;   /* device [capacity]: owning curve (selects colour and scene) */
  int32_t* aux;     /* device [capacity]: fills: nearest boundary segment i*, as
                       i* (inside) or ~i* (outside), or 0x7fffffff for a point so
                       deep inside that its sigmoid (Eq. 7) is exactly 1 in FP32,
                       or 0x80000000 for a point culled by fill_cull (no segment
                       needed for either); contours: -1 */
  int32_t* count;   /* device scalar: records in use */
  float* shape;     /* device [capacity*4] or NULL.  Non-NULL marks a tangent-
                       aligned set: {sigma_t, cos, sin, 0} per record, whose
                       rec.sigma is the deviation across the tangent; isotropic
                       records in it (fills) hold {sigma, 1, 0, 0}.  Written by
                       nurbs_sample with contour_mode 1; the splat calls then use
                       the exponent -(along^2/sigma_t^2 + across^2/sigma^2)/2 */
} ns_gaussians;

/* Parameters held fixed (the paper's "w/o weights", "w/o knots" and "w/o
 * w & k" variants, Table 1): their gradients are not formed. */
#define NS_FROZEN_WEIGHTS 1  /* rational weights: nothing is added to dkey's w column */
#define NS_FROZEN_KNOTS 2    /* knot intervals: dtau may be NULL and is not touched;
                                the reverse sweeps that only feed knot gradients are skipped */

/* Gradient outputs, caller-owned device memory, accumulated into (the caller
 * zeroes them, or passes zero_outputs = 1 to splat_backward). */
typedef struct {
  float* dkey;      /* device [n_keys*4]: dL/d{x, y, s, w} */
  float* dtau;      /* device [n_taus]; may be NULL with NS_FROZEN_KNOTS */
  float* dcolor;    /* device [n_curves*4]: dL/d{r, g, b, opacity} */
  int32_t frozen;   /* NS_FROZEN_WEIGHTS | NS_FROZEN_KNOTS, or 0 */
} ns_curve_grads;

/* What ns_poll_status reads back. */
typedef struct {
  int32_t status;        /* ns_status raised on the device (first one wins) */
  int32_t bad_curve;     /* first curve that failed validation, or -1 */
  int64_t gaussians;     /* Gaussians the last nurbs_sample needed */
  int64_t pairs;         /* tile pairs the last splat_forward needed */
  int64_t boundary;      /* boundary points the last nurbs_sample needed */
  int64_t fill_culled;   /* fill Gaussians with opacity below alpha_min (bin no tile) */
  int64_t blend_evals;   /* (pixel, Gaussian) alpha evaluations of the last splat_forward */
  int64_t blend_bwd_evals; /* the same for the last splat_backward */
  int64_t blend_contribs;  /* (pixel, Gaussian) pairs composited by the last splat_forward */
  int64_t blend_visits;    /* (pixel, list entry) pairs the last splat_forward walked: per pixel, its
                              tile list up to and including the entry that ended it (Eq. 8-9's loop
                              with early termination), whether or not the entry was evaluated; 0 with
                              fill layers, whose lists hold one entry per layer, not per Gaussian */
  int64_t blend_bwd_visits; /* the same for the last splat_backward: per pixel, the entries in front
                               of its last composited one, inclusive (0 with fill layers) */
} ns_report;

/* Kernel ids for ns_profile_next_launch. */
enum {
  NS_KERNEL_PLAN = 1, NS_KERNEL_BOUNDARY = 2, NS_KERNEL_EMIT = 3, NS_KERNEL_BIN_COUNT = 4,
  NS_KERNEL_BIN_EMIT = 5, NS_KERNEL_RADIX_HIST = 6, NS_KERNEL_RADIX_SCATTER = 7, NS_KERNEL_RANGES = 8,
  NS_KERNEL_BLEND_FWD = 9, NS_KERNEL_BLEND_BWD = 10, NS_KERNEL_CHAIN = 11, NS_KERNEL_CHAIN_BOUNDARY = 12,
  NS_KERNEL_KNOT_GRADS = 13, NS_KERNEL_MSE = 14, NS_KERNEL_ADAM = 15, NS_KERNEL_SCAN = 16,
  NS_KERNEL_OTHER = 17, NS_KERNEL_CHAIN_CONTOUR = 18, NS_KERNEL_DERIV_LOSS = 19, NS_KERNEL_BBOX_LOSS = 20,
  NS_KERNEL_FILL_SDF = 21
};

ns_sample_params ns_default_sample_params(void);
ns_raster_params ns_default_raster_params(void);

/*
 * Bytes of device workspace for a batch with these sizes.  The same workspace
 * must be passed to nurbs_sample, splat_forward and splat_backward of one
 * step: it carries the per-curve plan (knot vectors, counts, offsets, boundary
 * polylines), the sorted tile lists and the per-pixel state that the backward
 * pass reuses.  The caller allocates it (256-byte aligned); its contents need
 * no initialisation.  The part nurbs_sample uses comes first and does not
 * depend on the raster settings, so size the workspace with the raster
 * settings of the splat calls.  Returns 0 for invalid sizes (see ns_last_error).
 */
size_t ns_workspace_size(const ns_curves* curves, const ns_capacity* cap,
                         const ns_raster_params* raster);

/*
 * Curves -> Gaussians (§3.1-§3.3).  Per curve: knot vector from the intervals
 * (§3.1), arc length by N_L-node midpoint quadrature of |C'| (Eq. 2-3), then
 *   open or closed stroke: M = ceil(delta_c L) samples uniform in the domain
 *     [u_p, u_{m-p}] (open: both ends included, plus kappa copies of the first
 *     and last centre; closed: the start is not repeated); centre C_xy(u_j)
 *     evaluated span-locally (Eq. 4), sigma = C_s(u_j) / rho, opacity o (Eq. 5);
 *   filled closed curve: ceil(delta_b L) boundary points, their box padded by
 *     pad_frac of its extent and clipped to the canvas, a grid of step h with
 *     points at origin + (i + 1/2) h; per point sigma = eta h / rho and opacity
 *     o * sigmoid(gamma / h * sdf), sdf = sign(winding) * distance to the
 *     closed polyline (Eq. 6-7, S1-S3).
 * Writes out->rec/curve/aux/count (count = Gaussians emitted, at most
 * out->capacity; see ns_report.gaussians for the size needed).
 */
ns_status nurbs_sample(const ns_curves* curves, const ns_sample_params* sp,
                       const ns_capacity* cap, const ns_gaussians* out,
                       void* workspace, size_t workspace_bytes, void* stream);

/*
 * Gaussians -> image (§3.4, Eq. 8-9).  Bins each Gaussian to the tiles
 * overlapped by mu +- k_sigma sigma (float32 rule: floor((mu -+ k_sigma*sigma)
 * * (1/tile)), each operation rounded to nearest), sorts the (tile, Gaussian)
 * pairs by (tile, layer, sample), and composites each pixel front to back:
 *   alpha = min(alpha_max, o exp(-|x - mu|^2 / (2 sigma^2))),
 *   skipped where alpha < alpha_min, stopping before T would drop below t_min,
 *   image = sum c alpha T + T_final bg.
 * `g` is usually nurbs_sample's output but may be any set in the documented
 * order.  image: device [n_scenes*height*width*channels], overwritten.
 */
ns_status splat_forward(const ns_curves* curves, const ns_gaussians* g,
                        const ns_raster_params* rp, const ns_capacity* cap,
                        float* image, void* workspace, size_t workspace_bytes,
                        void* stream);

/*
 * dL/dimage -> gradients (§3.5).  Walks each tile's list back to front from
 * the last Gaussian each pixel composited, recovering the transmittance by
 * division rather than storing it, and accumulates per-Gaussian gradients of
 * (mu, sigma, opacity, colour).  If `out` is non-NULL these are chained
 * through the sampling of nurbs_sample (same workspace, same settings) into
 * the key points, knot intervals, colours and opacities; counts, spans, grid
 * placement, nearest segments and winding signs are held fixed.
 *   rp: the raster settings of the splat_forward this call follows (the
 *     lists and per-pixel state it left in the workspace).  With other
 *     settings the gradients are wrong (a per-Gaussian adjoint skips the
 *     entries of fill layers), though nothing is read out of bounds.
 *   dL_dimage: device, same layout as the image.
 *   dgauss: device [g->capacity*8] or NULL: {dmu_x, dmu_y, dsigma, 0,
 *     dopacity, dr, dg, db} per Gaussian, zeroed and written by this call.
 *     For a tangent-aligned set (g->shape non-NULL) rows are 12 floats,
 *     {dmu_x, dmu_y, dA, dB2, dopacity, dr, dg, db, dC, 0, 0, 0}, the
 *     gradients of the exponent A dx^2 + B2 dx dy + C dy^2's coefficients.
 *     When dgauss is NULL and `out` is given, the workspace holds them and the
 *     centre and sigma gradients of fill Gaussians, which the chain does not
 *     use (their grid is fixed), are not computed; with fill layers the fill
 *     Gaussians' opacity gradients are then kept as one float per Gaussian
 *     and only the contour Gaussians' rows are cleared and written.
 *   zero_outputs: 1 zeroes *out before accumulating, 0 adds to it.
 */
ns_status splat_backward(const ns_curves* curves, const ns_gaussians* g,
                         const ns_sample_params* sp, const ns_raster_params* rp,
                         const ns_capacity* cap, const float* dL_dimage,
                         float* dgauss, const ns_curve_grads* out, int32_t zero_outputs,
                         void* workspace, size_t workspace_bytes, void* stream);

/*
 * Grid-step annealing (Eq. 14): the fill grid step for iteration t of T,
 * h_max until t/T reaches t_b, then a cosine ramp to h_min reached at t_e,
 * h_min afterwards:  h = h_max + (h_min - h_max) (1 + cos(pi (1 - phi))) / 2,
 * phi = (t/T - t_b) / (t_e - t_b).  Host function; pass the result as
 * ns_sample_params.h.
 */
float ns_grid_step(int32_t t, int32_t T, float h_max, float h_min, float t_b, float t_e);

/*
 * L2 image loss (Eq. 10 with an L2 image term): loss = mean((image - target)^2)
 * over n values; dL_dimage = 2 (image - target) / n.  loss: device scalar,
 * overwritten.  dL_dimage may be NULL.
 */
ns_status ns_mse_loss(const float* image, const float* target, int64_t n,
                      float* dL_dimage, float* loss, void* stream);

/*
 * One Adam step on n parameters in place, then a clamp: element i is clamped
 * to [lo[i % group], hi[i % group]] (group 1..4; lo, hi are host arrays of
 * `group` floats, use +-INFINITY for no bound).  The paper clamps weights to
 * [0.01, 10] and knot intervals to [0, 2] (Table S1): for key points {x, y, s,
 * w} use group 4 with lo = {-inf, -inf, 0, 0.01}, hi = {inf, inf, inf, 10}.
 * Element i uses the learning rate lr * lr_scale[i % group] (lr_scale: host
 * array of `group` floats, or NULL for lr everywhere; the layer-wise loop of
 * §5 uses 2.0 for positions and 0.01 for the rest).
 * m, v: device moment buffers of n floats.  step >= 1.
 */
ns_status ns_adam_step(float* param, const float* grad, float* m, float* v, int64_t n,
                       float lr, float beta1, float beta2, float eps, int32_t step,
                       const float* lo, const float* hi, int32_t group,
                       const float* lr_scale, void* stream);

/* Penalties of the bounding-box loss (Eq. 12). */
#define NS_PENALTY_RELU 0      /* phi(x) = max(x, 0), derivative 0 at 0 */
#define NS_PENALTY_SOFTPLUS 1  /* phi(x) = log(1 + e^x), x in pixels */

/* Weights and settings of the geometric regularisers (§3.6, Eq. 10-12). */
typedef struct {
  float lambda_deriv;  /* weight of the derivative loss (Eq. 11); 0 skips it */
  int32_t order;       /* derivative order r, 1..4 (the paper uses 3) */
  int32_t nodes;       /* midpoint nodes per curve; 0: N_L = nl_mult * max(width, height) */
  float lambda_bbox;   /* weight of the bounding-box loss (Eq. 12); 0 skips it */
  int32_t penalty;     /* NS_PENALTY_RELU or NS_PENALTY_SOFTPLUS */
  float box[4];        /* x_min, y_min, x_max, y_max in pixels; an empty box
                          (x_max <= x_min or y_max <= y_min) means the canvas
                          [0, width] x [0, height] */
} ns_geometry_params;

/* Table S1's calligraphy weights lambda_deriv = 1, lambda_bbox = 5; order 3,
 * N_L nodes, ReLU, the canvas. */
ns_geometry_params ns_default_geometry_params(void);

/*
 * Geometric regularisers of the total loss (§3.6, Eq. 10-12) and their
 * gradients, on the plan, knot vectors, boundary polylines and Gaussian set
 * `g` that nurbs_sample left in `workspace` and wrote to `g` (same curves and
 * sample parameters; call it after nurbs_sample, before or after the splat
 * calls of the same step).
 *   Derivative loss (Eq. 11): per curve, (1/(b - a)) int_a^b |C^(r)_xy(u)|^2 du
 *     over its domain [a, b] = [u_p, u_{m-p}], by the `nodes`-node midpoint
 *     rule of Eq. 3, with C^(r) the exact r-th derivative of the rational
 *     curve (Eq. 1-2 differentiated r times); averaged over all curves.
 *   Bounding-box loss (Eq. 12): sum over the sampled curve points -- the M
 *     contour centres of every stroke (not the endpoint copies) and the
 *     boundary points of every filled curve -- of phi(b_min - P) + phi(P -
 *     b_max), per axis.  g->rec, g->curve and g->count are read for it.
 *   loss: device float[2], overwritten with {lambda_deriv * L_deriv,
 *     lambda_bbox * L_bbox}.
 *   out: NULL for the values only; otherwise the gradients with respect to
 *     the key points {x, y, w} and knot intervals are ADDED to out->dkey and
 *     out->dtau (out->dcolor is not touched), except those out->frozen names.  Knot spans of the nodes and the
 *     sample counts are held fixed, as in splat_backward.
 * Uses the workspace's knot-gradient scratch, so it must not run concurrently
 * with splat_backward on the same workspace (the same stream orders them).
 */
ns_status ns_geometry_loss(const ns_curves* curves, const ns_gaussians* g,
                           const ns_sample_params* sp, const ns_raster_params* rp,
                           const ns_geometry_params* gp,
                           const ns_capacity* cap, float* loss, const ns_curve_grads* out,
                           void* workspace, size_t workspace_bytes, void* stream);

/*
 * Layer-wise vectorisation (§4.2, the LIVE adaptation): the image term of its
 * loss (Eq. 15), L_img, a distance-weighted mean square error.  For every
 * scene s, new_curve[s] names the filled path the scene received this round
 * (or -1).  Per pixel centre, d is the distance to that path's closed
 * boundary polyline (§3.3, the points nurbs_sample left in `workspace`) and
 * w = max(0, tau - d); the scene's loss is sum w sum_c (I - I*)^2 / (C sum w).
 * A scene without a new path, or with no pixel within tau, takes the plain
 * mean square error.  loss = mean over scenes; the weights are constants.
 *   new_curve: device int32 [n_scenes]; an index that is not a filled curve
 *     counts as -1.
 *   image, target: device, image layout; dL_dimage: device, overwritten (or NULL).
 *   loss: device scalar, overwritten.
 * Uses the same workspace as the splat calls of the step (after nurbs_sample).
 */
ns_status ns_udf_mse_loss(const ns_curves* curves, const ns_sample_params* sp,
                          const ns_raster_params* rp, const ns_capacity* cap,
                          const int32_t* new_curve, float tau, const float* image,
                          const float* target, float* dL_dimage, float* loss,
                          void* workspace, size_t workspace_bytes, void* stream);

/*
 * Self-crossing penalty L_xing of the same loss (Eq. 15): for every curve, the
 * legs a_i = K_{i+1} - K_i of its key-point polygon (cyclic for closed curves),
 * the sine of each turn sin_i = (a_i x a_{i+1}) / (|a_i| |a_{i+1}|) and the
 * curve's winding sign sigma = sign(sum_i a_i x a_{i+1}) (held fixed):
 *   loss = lambda * sum over curves and turns of max(0, -sigma sin_i).
 * loss: device scalar, overwritten.  dkey: device [n_keys*4] or NULL; the
 * gradient with respect to x and y is ADDED to it.
 */
ns_status ns_xing_loss(const ns_curves* curves, float lambda, float* loss, float* dkey, void* stream);

/* Bytes of scratch ns_seed_windows needs (0 for invalid sizes). */
size_t ns_seed_scratch_size(int32_t n_scenes, int32_t height, int32_t width);

/*
 * Where the layer-wise loop starts a new path (§4.2: at the region of highest
 * reconstruction error): per scene, the pixel whose (2 radius + 1)^2 window
 * (clipped to the image) holds the largest sum of the squared error
 * sum_c (I - I*)^2, the first in row-major order on ties.
 *   image, target: device [n_scenes, height, width, channels] float32.
 *   scratch: device, ns_seed_scratch_size bytes, 256-byte aligned.
 *   seed_xy: device int32 [n_scenes*2] (x, y); seed_value: device float
 *   [n_scenes] (the window sum) or NULL.
 */
ns_status ns_seed_windows(const float* image, const float* target, int32_t n_scenes,
                          int32_t height, int32_t width, int32_t channels, int32_t radius,
                          void* scratch, size_t scratch_bytes, int32_t* seed_xy,
                          float* seed_value, void* stream);

/* Synchronises `stream`, reads the device status and counters. */
ns_status ns_poll_status(void* workspace, ns_report* report, void* stream);

/* Clears the device status word (enqueued on `stream`). */
ns_status ns_clear_status(void* workspace, void* stream);

/*
 * Internal arrays of a workspace, for tests and tools: copies `bytes` bytes of
 * array `which` to device memory `dst` (enqueued on `stream`).
 *   0 sorted pair tile ids (uint32), 1 sorted pair Gaussian ids (uint32),
 *   2 tile ranges (int32 [n_tiles*2], [start, end) per tile),
 *   3 per-curve plan records, 64 bytes each: float32 {L, a, b, x0, y0} (arc
 *     length, parameter domain, fill grid origin) then int32 {kind (0 invalid,
 *     1 open, 2 closed stroke, 3 filled), M (contour samples, or boundary
 *     points of a fill), Gaussians, nx, ny, first Gaussian, first boundary
 *     point, first task among the curves of its kind (fill or contour), scene,
 *     tasks of the other kind before it, 0},
 *   4 boundary points (float32 pairs), 5 per-pixel final transmittance,
 *   6 per-pixel composited-list length (int32)
 */
ns_status ns_workspace_copy(void* workspace, const ns_curves* curves, const ns_capacity* cap,
                            const ns_raster_params* rp, int32_t which, void* dst,
                            size_t bytes, void* stream);

/*
 * Chooses the blend decomposition for this batch by timing: every valid
 * pixels-per-thread setting of the forward and backward blend kernels is run
 * `repeats` times on the workspace of a completed splat_forward (and, if
 * dL_dimage is non-NULL, the backward with that upstream gradient), with and
 * without NS_BLEND_LANE_GROUPS, and the fastest is written to rp->ppt_fwd /
 * rp->ppt_bwd.  The choice changes no
 * result: every setting composites each pixel over the same list in the same
 * order.  `image` is rewritten with identical values.  Synchronises the
 * stream; call it before capturing a graph.  The tile size is fixed by the
 * workspace layout; to choose it, size one workspace per candidate tile.
 */
ns_status ns_autotune_blend(const ns_curves* curves, const ns_gaussians* g, ns_raster_params* rp,
                            const ns_capacity* cap, float* image, const float* dL_dimage,
                            void* workspace, size_t workspace_bytes, int32_t repeats, void* stream);

/*
 * Profiling aid.  The next launch of kernel `kernel_id` issued by the calling
 * thread records the cudaEvent_t `start` just before it and `stop` just after
 * it on the launch stream; while that stream is being captured into a CUDA
 * graph the two records are captured as external event-record nodes, so they
 * fire on every replay.  Up to 32 launches can be armed at once (each call
 * arms one; each armed entry fires once).  kernel_id 0 disarms all.
 */
ns_status ns_profile_next_launch(int32_t kernel_id, void* start, void* stop);

/* Number of kernels the calling thread has launched (or captured) through the library. */
uint64_t ns_launch_count(void);

/*
 * splat_forward for callers that cannot allocate device memory where they
 * render: an engine or server that owns and pre-plans all device memory, a
 * plugin limited to the buffers it is handed, or a loop that must not trigger
 * the device-wide synchronisation an allocation can cause.  The paper has no
 * counterpart; it is a packaging of splat_forward.
 *
 * Same inputs and output as splat_forward, but no workspace: the scratch
 * (tile pairs, sort buffers, ranges, per-pixel state, status) is a fixed
 * 16 MiB device array inside this library, held by every GPU that loads it
 * until the process exits.  Limits: g->capacity <= 65536 Gaussians, at most
 * 262144 (tile, Gaussian) pairs, and the batch's workspace (ns_workspace_size
 * with those capacities and no boundary points) must fit the 16 MiB; a larger
 * request returns NS_ERR_INVALID_ARG with a message saying which limit.  More
 * pairs than the limit is only known on the device: that work is dropped (the
 * image stays finite but misses those pairs) and the status reads
 * NS_ERR_CAPACITY -- visible only through a non-NULL report, since the array
 * is private to the library and the next call clears it.
 *   report: host pointer or NULL.  When non-NULL the call synchronises the
 *   stream and fills it: status, pairs (needed), fill_culled and the blend
 *   counters as ns_poll_status would, and gaussians = the set's count.  With
 *   NULL the call only enqueues work and returns.
 * Each call that is not being captured into a CUDA graph looks up the array's
 * device address (cudaGetSymbolAddress), so a device reset is picked up; a
 * call made during stream capture reuses the address found by the last
 * uncaptured call on that device, so make one call before any capture.  All
 * calls on one device share the array: calls that overlap on the GPU (other
 * streams or threads) race and must be serialised by the caller.  Each call
 * clears the status it inherits from the previous one.  It calls no
 * allocator.  It always bins one pair per Gaussian and tile (rp->fill_layers
 * is ignored: fill layers need the sampling plans of a workspace, which it
 * has none of).
 */
ns_status splat_forward_noalloc(const ns_curves* curves, const ns_gaussians* g,
                                const ns_raster_params* rp, float* image, ns_report* report,
                                void* stream);

/* Message of the last error on the calling thread ("" if none). */
const char* ns_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NURBS_SPLAT_H */
