/*
 * cc.h -- C ABI of libccgpu: microlensing critical curves, caustics, caustic-crossing
 * maps and distance-to-caustic maps on one NVIDIA GB300 (sm_103a).
 *
 * Method: Weisenbach (2025), "A GPU Code for Finding Microlensing Critical Curves and
 * Caustics".  Units: theta_* = 1 (Einstein radius of a unit mass).  Lens model: N point
 * masses (x_i, y_i, m_i), smooth convergence kappa_s and external shear gamma, with the
 * compensating mass sheet extended to infinity (Appendix A), so
 *     w(z)     = (1 - kappa_s) z + gamma conj(z) - sum_i m_i / conj(z - z_i)     (Sec. 3.1)
 *     F(z,phi) = gamma + sum_i m_i / (z - z_i)^2 - (1 - kappa_s) e^{-i phi}      (Sec. 3.1)
 * and for every phase phi the n_r = 2N critical points are the roots of F(., phi)
 * (Sec. 3.1, rationalised polynomial P = F prod (z - z_i)^2).
 *
 * Conventions for every call
 *   - Return value: a cc_status (CC_OK = 0).  On error, cc_last_error() gives a message
 *     (thread-local, valid until the next call on the same thread).
 *   - Complex arrays are interleaved (re, im) pairs of IEEE doubles (complex128).
 *   - Device buffers are allocated and owned by the caller; the library never frees
 *     them.  Unless stated otherwise, pointers are device pointers on the field's device.
 *   - Calls taking a stream enqueue work on it and return without waiting; results are
 *     valid once the stream has reached that point.  A NULL stream is the legacy default
 *     stream.  cc_stream_t is binary-compatible with cudaStream_t.
 *   - Device memory the library allocates itself: one block per field in cc_field_create
 *     (its star layouts, report and far-field tables: O(N) plus a cell grid) from a
 *     library-owned stream-ordered pool, returned to the pool by cc_field_destroy (the pool
 *     keeps freed blocks for reuse), and the fixed static scratch of
 *     cc_distance_map_static.  cc_field_create and cc_batch_create also create CUDA events.
 *     Everything of size O(m N) or O(W H) (rows, tracer state, polish tables, batch tables,
 *     map scratch) is caller memory: the workspaces whose sizes the *_workspace_bytes calls
 *     return.
 *   - No kernel spins on a flag or a lock, so no call waits on the device for anything but
 *     its own work to finish.
 */
#ifndef CC_H_
#define CC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* cc_stream_t;
typedef struct cc_field cc_field;

typedef enum cc_status {
    CC_OK = 0,
    CC_EINVAL = 1,       /* bad argument (NULL pointer, odd m, size out of range, ...) */
    CC_ENOMEM = 2,       /* device allocation failed (cc_field_create) or workspace too small */
    CC_ENOCONV = 3,      /* reported by cc_field_report: some roots did not converge */
    CC_EDEGENERATE = 4,  /* |1 - kappa_s - gamma| < 1e-12: a root runs to infinity at phi = 0 */
    CC_ECUDA = 5         /* a CUDA runtime call failed (message has the CUDA error string) */
} cc_status;

/* Arithmetic of the root tracer (Sec. 3.2 iteration, Sec. 4.4 runtime). */
typedef enum cc_precision {
    /* Aberth-Ehrlich in FP32 (plain FP32 star and root sums: the FP32 grid of positions,
     * not the summation, sets the tracer's resolution), then a Newton polish on F with
     * double-float or FP64 star sums (hp_arith), fused with the caustic mapping, that
     * certifies every point to tol_cert (1e-10). */
    CC_MIXED = 0,
    /* Aberth-Ehrlich entirely in FP64 with the |dz| < tol_abs stop rule, as in the
     * paper's double-precision code; caustics by a separate FP64 lens-map pass. */
    CC_FP64 = 1
} cc_precision;

/* Arithmetic of the polish / caustic-mapping star sums. */
typedef enum cc_hp_arith {
    CC_HP_DFLOAT = 0, /* double-float (pairs of FP32, ~48-bit significand) on the FP32 pipes */
    CC_HP_FP64 = 1    /* native FP64 */
} cc_hp_arith;

/* Shape of the microlens field (Sec. 4.2, Appendices A and B).
 *   CC_FIELD_DISC  circular field; its smooth sheet is extended to infinity (Appendix A):
 *                  alpha_s = -kappa_* z, n_r = 2N roots per phi.
 *   CC_FIELD_RECT  rectangular field |Re z| <= c1, |Im z| <= c2 (the stars should lie in it)
 *                  with the logarithms of alpha_s replaced by their series truncated at the
 *                  odd order t and the sheet extended to infinity (Appendix B): F gains
 *                  -conj(dalpha_s/dconj z), a polynomial of degree t - 1 in z, and the
 *                  lens map gains the matching odd polynomial in conj(z); n_r = 2N + t - 1. */
typedef enum cc_field_shape { CC_FIELD_DISC = 0, CC_FIELD_RECT = 1 } cc_field_shape;
#define CC_RECT_MAX_T 129

typedef struct cc_options {
    double tol_abs;      /* freeze a root when |z^{a+1} - z^a| < tol_abs (Sec. 3.2 footnote: 1e-9) */
    double mu_max;       /* also freeze when |mu| > mu_max (Sec. 3.2 footnote: 1e9); 0 = off.
                            Used by CC_FP64 only; the mixed form never freezes on |mu|. */
    double tol_cert;     /* polish stops when the estimated Newton error < tol_cert (1e-10) */
    int32_t max_iter_cold; /* Aberth iteration cap at a subchain's centre row (500) */
    int32_t max_iter_warm; /* cap for warm-started rows (200) */
    int32_t max_polish;    /* polish passes per point (8); rows that still hold an uncertified
                              point are re-solved by FP64 Aberth warm-started from the polish */
    int32_t precision;     /* cc_precision */
    int32_t hp_arith;      /* cc_hp_arith (polish and cc_map_caustics) */
    int32_t subchains;     /* phi sub-ranges grown in parallel (Sec. 4.3); 0 = automatic */
    int32_t predictor;     /* warm start of a row (Sec. 3.2 last paragraph) from the rows before it
                              on its chain: 0 copies the previous row, 1 extrapolates linearly
                              through the last two, 2 quadratically through the last three */
    int32_t block_threads; /* threads per tracing CTA (0 = automatic) */
    int32_t far_field;     /* 1: polish stars beyond a 5x5 block of cells through local expansions
                              (Sec. 4.1, fast multipole method; used when N >= 128 and hp_arith is
                              CC_HP_DFLOAT); 0: every star summed directly */
    /* Shape of the microlens field and its smooth sheet (Sec. 4.2, Appendices A and B). */
    int32_t field_shape;   /* cc_field_shape: CC_FIELD_DISC (default) or CC_FIELD_RECT */
    int32_t rect_t;        /* CC_FIELD_RECT: odd truncation order t >= 3 of the logarithm series of
                              alpha_s, at most CC_RECT_MAX_T; 0 = the Appendix B rule (the smallest
                              odd t whose error bound is <= rect_eps for |z| rect_s < |c|, then
                              t + 2 while (t - 1) Arg(c) lies within 0.1 pi of a multiple of pi) */
    double kappa_star;     /* CC_FIELD_RECT: convergence of the stars' smooth sheet, kappa_* > 0 */
    double rect_c1, rect_c2; /* CC_FIELD_RECT: corner c = c1 + i c2 of the field (half-width,
                              half-height, both > 0) */
    double rect_eps, rect_s; /* CC_FIELD_RECT, rect_t == 0: error target (1e-9) and ratio s > 1 (2) */
    int32_t row_ctas;      /* CTAs (one thread-block cluster) that share each phi sub-range of the
                              tracer (either precision), each updating a slice of the roots:
                              0 = automatic (1 when n_r < 4096, or when m >= 8 x the SM count and
                              the form is CC_FP64 or root_refresh >= 2; else 8), 1 = one CTA per
                              sub-range, 2..16 = that many */
    int32_t root_refresh;  /* Aberth root sum of the FP32 tracer (one CTA or a cluster per
                              sub-range): 0 or 1 = exact in every sweep (Sec. 3.2); K >= 2 = exact
                              every K-th row of a chain (and whenever an iterate moves beyond a
                              quarter cell from its refresh position), where each root's sum is
                              split into the roots of the 3 x 3 cells around it (summed exactly in
                              every sweep) and the rest (kept from the refresh).  Cold rows split
                              too, from cells at the guesses.  The roots found are the same zeros
                              of F; only the Aberth iteration path changes.  At most 4096; default
                              64.  The FP64 forms always sum exactly. */
} cc_options;

/* Solve statistics of the last cc_critical_curves on a field (host copy). */
typedef struct cc_report {
    int64_t rows;              /* m + 1 */
    int64_t n_roots;           /* n_r = 2N (disc) or 2N + t - 1 (rectangle) */
    int64_t subchains;         /* sub-ranges used */
    int64_t root_iterations;   /* Aberth updates executed (all rows, all roots) */
    int64_t cold_root_iterations; /* of which at the subchain centre rows */
    int64_t unconverged;       /* root-rows that hit the Aberth cap */
    int64_t polish_passes;     /* star-sum passes of the polish (all points) */
    int64_t uncertified;       /* points whose final error estimate exceeds tol_cert */
    int64_t seam_ambiguous;    /* sub-range joins that were not a clean 1:1 match */
    int32_t max_iter_row;      /* largest per-root iteration count in any row */
    double max_err_est;        /* largest error estimate of a certified point (theta_*) */
    /* Device time of each stage of the last solve (CUDA events on the caller's stream):
     * tracing (Aberth), joining sub-ranges, polish + caustics (mixed form) or
     * reordering + caustics (FP64 form). */
    float trace_ms, join_ms, polish_ms;
    int64_t rescued_points;    /* uncertified points re-solved by FP64 Aberth (root alone, the
                                  rest of its row fixed) and now converged */
    int64_t jumped;            /* points the polish moved > 1e-3 (1 + |z|) from the tracer's
                                  root (a sign of a root swap; diagnostic) */
    int64_t star_terms;        /* tracer: star terms summed directly (all roots, iterations) */
    int64_t far_evals;         /* tracer: root updates that used a cell's local expansions */
    int64_t root_terms;        /* tracer: root-root terms summed (all roots, iterations) */
    int64_t split_redone_rows; /* root_refresh >= 2: rows solved again with the exact root sum
                                  because an iterate moved beyond its displacement limit */
} cc_report;

/* Fill *opt with the defaults listed above. */
int cc_options_default(cc_options* opt);

/* Create a field on the current CUDA device.
 *   x, y, mass: n star positions and masses, FP64, host OR device pointers (copied in).
 *   kappa_s: smooth convergence (Sec. 2.1 with Appendix A: 1 - kappa - dalpha_s/dz
 *            = 1 - kappa_s); gamma >= 0: shear (Sec. 2.1).
 *   opt: NULL for defaults.
 * Errors: CC_EINVAL (n < 1, NULL pointer, non-finite value, mass <= 0),
 *         CC_EDEGENERATE (|1 - kappa_s - gamma| < 1e-12), CC_ENOMEM, CC_ECUDA.
 * Blocks until the stars are on the device. */
int cc_field_create(const double* x, const double* y, const double* mass, int64_t n,
                    double kappa_s, double gamma, const cc_options* opt, cc_field** out);

/* Free the field's device arrays.  NULL is accepted. */
int cc_field_destroy(cc_field* field);

/* Number of stars and roots (n_r = 2N, Sec. 3.1) of a field. */
int cc_field_size(const cc_field* field, int64_t* n_stars, int64_t* n_roots);

/* Device scratch bytes that cc_critical_curves needs for m phi steps. */
int cc_critical_curves_workspace_bytes(const cc_field* field, int64_t m, size_t* bytes);

/* Critical curves on the phi grid phi_j = 2 pi j / m, j = 0..m (Sec. 3.1, chain matrix of
 * Sec. 4.3; m even, >= 2).  Roots are found by simultaneous Aberth-Ehrlich iteration
 * (Sec. 3.2) at the centre row of each phi sub-range, then grown row by row toward both
 * ends of the sub-range, each row warm-started from its neighbour (Secs. 3.2, 4.3).
 * Sub-ranges are joined so that column k of every row follows one chain.
 * Initial guesses at a centre row (the paper uses z_i +- 1): roots 2i and 2i+1 start at the
 * two critical points of star i alone in the field of the others, z_i +- sqrt(-m_i / c_i)
 * with c_i = gamma - (1 - kappa_s) e^{-i phi} + sum_{j != i} m_j / (z_i - z_j)^2 (the sum
 * direct over a star tile, or through the FP32 far-field tables), scaled by
 * 1 + (i mod 64) 2^-12 so that coincident stars keep distinct guesses; z_i +- (1 + 1i/64)
 * for a rectangular field, a star outside the far-field grid, a field too large for one
 * star tile without that grid, or c_i ~ 0.  Guesses do not change the roots found.
 *   z_out:     (m+1) x n_r complex128, row j holds the roots at phi_j (device).
 *   w_out:     optional (NULL to skip), same layout: the caustic point w(z) of each root
 *              (Sec. 5.1), computed in the same pass as the polish.
 *   iters_out: optional (NULL to skip), (m+1) x n_r int32: Aberth iterations per root.
 *   workspace: device scratch of at least cc_critical_curves_workspace_bytes bytes,
 *              256-byte aligned; its contents on entry do not matter.
 * Errors: CC_EINVAL (odd/small m, NULL z_out or workspace, misaligned or too small
 *         workspace), CC_ECUDA.  Convergence problems are not errors of this call: see
 *         cc_field_report. */
int cc_critical_curves(cc_field* field, int64_t m, double* z_out, double* w_out,
                       int32_t* iters_out, void* workspace, size_t workspace_bytes,
                       cc_stream_t stream);

/* Wait for the field's last cc_critical_curves and copy its statistics.  Returns CC_OK,
 * or CC_ENOCONV if any root-row hit the iteration cap or any point is uncertified. */
int cc_field_report(cc_field* field, cc_report* out);

/* Caustic points (Sec. 3.1 lens equation, Sec. 5.1): w_out[p] = w(z[p]) for count points.
 * z, w_out: count complex128 (device).  Arithmetic follows the field's hp_arith option.
 * Errors: CC_EINVAL, CC_ECUDA. */
int cc_map_caustics(cc_field* field, const double* z, int64_t count, double* w_out,
                    cc_stream_t stream);

/* Number of caustic crossings N_cc on a W x H source-plane grid (Sec. 5.1): minus the
 * winding number (Sunday's crossing rule, exact orientation predicate) of the caustic
 * polygons, which are the columns of the rows x n_r vertex matrix w (segment
 * (w[j][k], w[j+1][k]) for j = 0..rows-2).  Pixel centres are
 *   x_i = x0 + (i + 0.5) * ((x1 - x0) / W),  y_r = y0 + (r + 0.5) * ((y1 - y0) / H)
 * in IEEE FP64 without fused multiply-add.  A segment counts for pixel centres with
 * min(a.y, b.y) <= y < max(a.y, b.y) lying strictly left (upward) / right (downward).
 *   w: rows x n_r complex128 (device).  ncc_out: H x W int32, row 0 at y0 (device).
 * Errors: CC_EINVAL (W, H < 1, x1 <= x0, y1 <= y0, rows < 1, NULL), CC_ECUDA. */
int cc_crossing_map(const double* w, int64_t rows, int64_t n_r, double x0, double x1, double y0,
                    double y1, int32_t W, int32_t H, int32_t* ncc_out, cc_stream_t stream);

/* Device scratch bytes that cc_distance_map needs for a W x H map. */
int cc_distance_map_workspace_bytes(int32_t W, int32_t H, size_t* bytes);

/* Distance from each pixel to the nearest caustic for an expanding source (Sec. 5.2):
 * the exact Euclidean distance transform of the N_cc map.  A caustic (feature) pixel
 * has a 4-neighbour inside the map with a different N_cc; the map border is not a
 * caustic.  d_out[p] = pixel * sqrt(squared index distance to the nearest feature);
 * +inf if the map has no feature.
 *   ncc: H x W int32 (device).  d_out: H x W double (device).
 *   workspace: >= cc_distance_map_workspace_bytes, 256-byte aligned (device).
 * Errors: CC_EINVAL, CC_ECUDA. */
int cc_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, double* d_out,
                    void* workspace, size_t workspace_bytes, cc_stream_t stream);

/* Distance to the nearest caustic for a source moving in direction angle (radians from
 * the +x axis, i.e. the source-plane y1 axis) (Sec. 5.2, the moving-source map): from each
 * pixel centre the ray is followed through the pixel grid (cell traversal in pixel units,
 * IEEE single precision in a fixed order: after k steps the next vertical / horizontal grid
 * line lies at (0.5 + k) / |cos| and (0.5 + k) / |sin|, the horizontal one on ties) to the
 * first caustic pixel (same feature rule as cc_distance_map).  d_out = pixel * ray
 * parameter at entry into that pixel; 0 on a caustic pixel; +inf when the ray leaves the
 * map first (the border is not a caustic; Sec. 5.2 figure caption).
 *   ncc: H x W int32 (device).  d_out: H x W double (device).  No scratch.
 * Errors: CC_EINVAL, CC_ECUDA. */
int cc_moving_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, double angle,
                           double* d_out, cc_stream_t stream);

/* ---------------------------------------------------------------------------------
 * Batched critical curves: many fields of uneven N in one persistent launch (each field
 * as cc_critical_curves computes it; the paper solves one field at a time, Sec. 4.4).
 * Work items are (field, phi sub-range) pairs sized in proportion to each field's work
 * and handed out most expensive first to the resident CTAs of one launch; the chain
 * joining and the polish then run once over all fields.
 * --------------------------------------------------------------------------------- */
typedef struct cc_batch cc_batch;

/* Plan a batch of count fields (all CC_MIXED, one device) with m[f] phi steps each.
 * The fields must outlive the batch.  Tolerances and caps come from fields[0]'s options.
 * Tile shape: block_threads (tracing CTA size, multiple of 32 in [32, 512]; 0 = the
 * field's option or 512) and items_per_cta (work items per resident CTA the fields are cut
 * into, 0 = 4); an autotuner may pick both.  Errors: CC_EINVAL, CC_ECUDA. */
int cc_batch_create(cc_field* const* fields, int32_t count, const int64_t* m, int32_t block_threads,
                    int32_t items_per_cta, cc_batch** out);

/* Device scratch bytes the batch needs (tables, tracer rows, joins, per-field reports). */
int cc_batch_workspace_bytes(const cc_batch* batch, size_t* bytes);

/* Bind outputs and workspace: z_out[f] / w_out[f] are device pointers to (m[f]+1) x n_r[f]
 * complex128 (w_out may be NULL, or hold NULL entries); workspace >= the size above,
 * 256-byte aligned.  Uploads the batch's device tables (blocking).  Errors: CC_EINVAL,
 * CC_ENOMEM, CC_ECUDA. */
int cc_batch_bind(cc_batch* batch, double* const* z_out, double* const* w_out, void* workspace,
                  size_t workspace_bytes);

/* Enqueue the whole batch on stream.  use_graph != 0: the launch sequence is captured
 * once into a CUDA graph (per stream; needs a non-default stream) and replayed on later
 * calls; rebinding discards the graph.  Errors: CC_EINVAL, CC_ECUDA. */
int cc_batch_launch(cc_batch* batch, int32_t use_graph, cc_stream_t stream);

/* Wait for the last launch; per_field (count entries) and total may be NULL.  Stage times
 * are in total.  Returns CC_OK or CC_ENOCONV like cc_field_report. */
int cc_batch_report(cc_batch* batch, cc_report* per_field, cc_report* total);

/* Work items, persistent grid size and block size of the batch. */
int cc_batch_info(const cc_batch* batch, int32_t* items, int32_t* grid, int32_t* threads);

/* Free the batch (not the fields, outputs or workspace). */
int cc_batch_destroy(cc_batch* batch);

/* Largest map (W * H pixels) that cc_distance_map_static accepts. */
#define CC_DISTANCE_MAP_STATIC_MAX_PIXELS 1048576

/* The distance map of cc_distance_map, for callers that cannot allocate device memory
 * when they call it (a plugin whose host application owns all device memory through its
 * own allocator, a process whose device-memory budget is fully reserved, a loop that must
 * never enter the allocator).  The paper has no counterpart: this is an interface of this
 * library only.  The call allocates nothing: its scratch is a fixed array of
 * CC_DISTANCE_MAP_STATIC_MAX_PIXELS * 8 + 512 bytes in this library's device memory,
 * held by every GPU that loads the library until the process exits.
 *   ncc, d_out, W, H, pixel: as for cc_distance_map (caller-allocated device buffers).
 * The array is used on the current device, so stream must belong to that device.  The
 * first call in each CUDA context looks up the array's device address (with that device
 * current) and keeps it for that context; make that first call before any stream capture
 * on the device.  After a reset of the device's primary context the next call looks the
 * address up again.  All calls share the one array and it keeps the last call's contents
 * (nothing needs clearing: every scratch entry is written before it is read); calls that
 * overlap on the GPU race on it, so order them on one stream or serialise them.
 * Errors: CC_EINVAL (W * H > CC_DISTANCE_MAP_STATIC_MAX_PIXELS, NULL, bad size or
 *         pixel, a stream of another device), CC_ECUDA. */
int cc_distance_map_static(const int32_t* ncc, int32_t W, int32_t H, double pixel, double* d_out,
                           cc_stream_t stream);

/* Last error message of this thread ("" if none). */
const char* cc_last_error(void);

/* Library version string. */
const char* cc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CC_H_ */
