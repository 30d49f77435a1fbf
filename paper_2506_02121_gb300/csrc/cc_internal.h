// Internal interfaces between the translation units of libccgpu (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "../../include/cc.h"
#include "cc_common.cuh"

namespace ccg {

// FP64 star record for the plain-FP64 tracer (32 bytes, two 16-byte loads).
struct __align__(32) StarD {
    double x, y, z, w;  // position (x, y), mass z, padding w
};

// Tracer far-field tables of a field (built once in cc_field_create): a grid of cells
// over the stars (plus a margin); per cell the stars of its 5x5 block ("near") and FP32
// local expansions of the other stars' sums sum 1/(z - z_i) and sum m_i/(z - z_i).
constexpr int TFMM_P = 14;        // expansion terms (rho <= 0.29: rho^14 ~ 3e-8)
constexpr int TFMM_NEAR_MAX = 48;  // near stars stored per cell (more: the cell sums directly)
struct TfmmParams {
    float x0, y0, b, inv_b;
    int nbx, nby;
    int ok;
};
struct TCell {
    float cx, cy;     // centre
    int near_cnt;     // -1: sum every star directly
    float far_m_d2;   // sum_far m/|z_i - c|^2 (scale of the far-field rounding noise)
};

// Smooth-sheet polynomial of a rectangular field (Appendix B): F gains -Q(z),
//   Q(z) = conj(dalpha_s/dconj z) = sum_{k=0}^{K} q_k z^{2k}  (real q_k, K = (t - 1)/2),
//   q_0 = kappa_* (1 - 4 Arg(c)/pi),  q_k = -(4 kappa_*/pi) sin(2k Arg c) / (2k |c|^{2k}),
// and the lens map gains V(conj z) = -sum_k q_k conj(z)^{2k+1} / (2k + 1) (its conj(z)
// derivative is -conj(Q)); the constant of V is 0.  Both are evaluated in zeta = z / |c|
// with the O(1) coefficients qn_k = q_k |c|^{2k} (q_k alone underflows FP32 for large |c|):
//   Q = sum qn_k zeta^{2k},  V = -|c| conj(zeta) sum vn_k conj(zeta)^{2k},  vn_k = qn_k/(2k+1).
// Device memory, one per field.
constexpr int POLY_MAX_K = (CC_RECT_MAX_T - 1) / 2;
struct SmoothPoly {
    int K;
    double ac, inv_ac;             // |c| and 1/|c|
    float acf, inv_acf;
    float2 inv_acdf;               // 1/|c| as double-float
    double rg;                     // radius of the extra roots' initial guesses (|c|)
    float qf[POLY_MAX_K + 1];      // qn_k in FP32 (tracer)
    double q[POLY_MAX_K + 1];      // qn_k in FP64
    float2 qdf[POLY_MAX_K + 1];    // qn_k as double-float
    float2 vdf[POLY_MAX_K + 1];    // vn_k as double-float
    double v[POLY_MAX_K + 1];      // vn_k in FP64
};

// Q(z), dQ/dz and d2Q/dz2 by Horner in u = zeta^2 (T = float or double), with
// qa = sum |qn_k| |zeta|^{2k}, the scale of the rounding error of Q.
template <typename T>
__device__ __forceinline__ void poly_eval(const SmoothPoly* P, T zx, T zy, T& Qx, T& Qy, T& Q1x, T& Q1y, T& Q2x,
                                          T& Q2y, T& qa) {
    const T* q;
    T ic;
    if constexpr (sizeof(T) == 4) {
        q = (const T*)P->qf;
        ic = (T)P->inv_acf;
    } else {
        q = (const T*)P->q;
        ic = (T)P->inv_ac;
    }
    const T sx = zx * ic, sy = zy * ic;
    const T ux = sx * sx - sy * sy, uy = (T)2 * sx * sy, au = sx * sx + sy * sy;
    T px = q[P->K], py = 0, dx = 0, dy = 0, ex = 0, ey = 0;
    T pa = q[P->K] < (T)0 ? -q[P->K] : q[P->K];
    for (int k = P->K - 1; k >= 0; k--) {
        const T nex = ex * ux - ey * uy + dx, ney = ex * uy + ey * ux + dy;
        const T ndx = dx * ux - dy * uy + px, ndy = dx * uy + dy * ux + py;
        const T npx = px * ux - py * uy + q[k], npy = px * uy + py * ux;
        ex = nex;
        ey = ney;
        dx = ndx;
        dy = ndy;
        px = npx;
        py = npy;
        pa = pa * au + (q[k] < (T)0 ? -q[k] : q[k]);
    }
    Qx = px;
    Qy = py;
    // dQ/dzeta = 2 zeta p'(u);  d2Q/dzeta2 = 2 p'(u) + 4 u p''(u), p''(u) = 2 e;  d/dz = ic d/dzeta
    Q1x = (T)2 * (sx * dx - sy * dy) * ic;
    Q1y = (T)2 * (sx * dy + sy * dx) * ic;
    Q2x = ((T)2 * dx + (T)8 * (ux * ex - uy * ey)) * ic * ic;
    Q2y = ((T)2 * dy + (T)8 * (ux * ey + uy * ex)) * ic * ic;
    qa = pa;
}

// FP32 form for iterates anywhere in the plane: Q and dQ/dz times a common complex scale
// sc, with |Q sc| = O(1) also where zeta^{2K} would overflow FP32 (an Aberth cold start
// can fling an iterate far out).  For |u| <= 1 (u = zeta^2) sc = 1; otherwise, with
// w = 1/u and the reversed polynomial pr(w) = sum_k qn_k w^{K-k} = w^K p(u),
//   sc = w^K,  sc Q = pr(w),  sc dp/du = w (K pr(w) - w pr'(w)),  sc dQ/dz = 2 zeta ic sc dp/du.
// qa_sc = |sc| sum |qn_k| |u|^k.  The Aberth step needs only F'/F, and the stop rule
// compares scaled noise with a scaled |F'|, so the common scale drops out.
__device__ __forceinline__ void poly_eval_scaled(const SmoothPoly* P, float zx, float zy, float& Qx, float& Qy,
                                                 float& Q1x, float& Q1y, float& scx, float& scy, float& qa) {
    const float* q = P->qf;
    const float ic = P->inv_acf;
    const float sx = zx * ic, sy = zy * ic;
    const float ux = sx * sx - sy * sy, uy = 2.f * sx * sy, au = sx * sx + sy * sy;
    const int K = P->K;
    float dx, dy;
    if (au <= 1.f) {
        float px = q[K], py = 0.f, pa = fabsf(q[K]);
        dx = 0.f;
        dy = 0.f;
        for (int k = K - 1; k >= 0; k--) {
            const float ndx = dx * ux - dy * uy + px, ndy = dx * uy + dy * ux + py;
            const float npx = px * ux - py * uy + q[k], npy = px * uy + py * ux;
            dx = ndx;
            dy = ndy;
            px = npx;
            py = npy;
            pa = pa * au + fabsf(q[k]);
        }
        Qx = px;
        Qy = py;
        scx = 1.f;
        scy = 0.f;
        qa = pa;
    } else {
        const float r = 1.f / (au * au);  // 1/|u|^2
        const float wx = ux * r, wy = -uy * r, aw = 1.f / au;
        float px = q[0], py = 0.f, ex = 0.f, ey = 0.f, pa = fabsf(q[0]), cx = 1.f, cy = 0.f;
        for (int k = 1; k <= K; k++) {
            const float nex = ex * wx - ey * wy + px, ney = ex * wy + ey * wx + py;
            const float npx = px * wx - py * wy + q[k], npy = px * wy + py * wx;
            const float ncx = cx * wx - cy * wy, ncy = cx * wy + cy * wx;
            ex = nex;
            ey = ney;
            px = npx;
            py = npy;
            cx = ncx;
            cy = ncy;
            pa = pa * aw + fabsf(q[k]);
        }
        Qx = px;  // sc Q
        Qy = py;
        // sc dp/du = w (K pr - w pr')
        const float tx = (float)K * px - (wx * ex - wy * ey), ty = (float)K * py - (wx * ey + wy * ex);
        dx = wx * tx - wy * ty;
        dy = wx * ty + wy * tx;
        scx = cx;
        scy = cy;
        qa = pa;
    }
    Q1x = 2.f * (sx * dx - sy * dy) * ic;
    Q1y = 2.f * (sx * dy + sy * dx) * ic;
}

// V(conj z) = -|c| conj(zeta) sum vn_k conj(zeta)^{2k} in FP64.
__device__ __forceinline__ double2 poly_V(const SmoothPoly* P, double zx, double zy) {
    const double sx = zx * P->inv_ac, sy = -zy * P->inv_ac;  // conj(zeta)
    const double ux = sx * sx - sy * sy, uy = 2.0 * sx * sy;
    double px = P->v[P->K], py = 0.0;
    for (int k = P->K - 1; k >= 0; k--) {
        const double npx = px * ux - py * uy + P->v[k], npy = px * uy + py * ux;
        px = npx;
        py = npy;
    }
    return make_double2(-P->ac * (sx * px - sy * py), -P->ac * (sx * py + sy * px));
}

// Device-side copy of a field's stars in the layouts the kernels read.
struct FieldDev {
    cudaEvent_t ready;        // recorded after the field's uploads and tables (stream 0)
    int64_t n;
    int64_t nr;               // roots per row: 2n (disc) or 2n + t - 1 (rectangle)
    const SmoothPoly* poly;   // rectangle polynomial (device), nullptr for the disc
    int poly_K;               // host copy of poly->K (0 for the disc)
    double kappa_s, gamma;
    bool unit_mass;
    float fmm_cell;   // far-field cell size aimed at ~6 stars in a 5x5 block of cells
    float4* star32;   // (x, y, m, 0) rounded to FP32
    StarD* star64;    // FP64
    float4* star_dfp; // (x_hi, x_lo, y_hi, y_lo) double-float positions
    float2* star_dfm; // (m_hi, m_lo)
    float2* star_tf;  // (x_l, y_l): third float of the positions (x = x_hi + x_lo + x_l)
    // tracer far field (tfmm.ok == 0: none)
    TfmmParams tfmm;
    TCell* tcells;    // nbx * nby
    int* tnear;       // nbx * nby * TFMM_NEAR_MAX star indices
    float4* tcoeff;   // nbx * nby * TFMM_P: (U_k re, S1'_k re, U_k im, S1'_k im), S1'_k = (k + 1) L_(k+1)
};
cudaError_t launch_tracer_far_field(const float4* s32, int n, const TfmmParams& P, TCell* cells, int* near,
                                    float4* coeff, cudaStream_t st);

// Tracing (Aberth) launch arguments shared by the FP32 and FP64 tracers.
struct TraceArgs {
    const FieldDev* f;     // host pointer to the field description (values copied into kernel args)
    int64_t m;             // phi steps
    int S;                 // subchains
    const double2* phase;  // (m+1) x (cos phi_j, sin phi_j)
    void* zrows;           // (m+1) x nr complex (T): each row in its subchain's column order
    void* seam;            // S x nr complex (T): up-end row of subchain s, s < S-1
    int32_t* iters;        // (m+1) x nr
    void* work;            // per-CTA scratch
    size_t work_stride;    // bytes per CTA (multiple of 256)
    DevReport* rep;
    double tol_abs, mu_max;
    int max_iter_cold, max_iter_warm, predictor;
    int root_refresh;      // FP32 warm rows: exact far part of the root sum every root_refresh rows
    int threads;
    int cluster;           // CTAs per sub-range (> 1: one thread-block cluster per sub-range)
    float4* ext;           // FP32 form, may be null: per CTA the extent (min x, min y, max x, max y) of
                           // the points it wrote to zrows, x = NaN if one was not finite
};

// One field of a batched launch (device table entry).
struct TraceTask {
    const void* stars;     // FP32 star records
    const SmoothPoly* poly;
    TfmmParams tfmm;
    const TCell* tcells;
    const int* tnear;
    const float4* tcoeff;
    int n, nr;
    double kappa_s, gamma;
    int64_t m;
    int S;
    const double2* phase;
    void* zrows;
    void* seam;
    int32_t* iters;
    int32_t *match, *hits, *perm;
    DevReport* rep;
};

struct BatchTraceArgs {
    const TraceTask* tasks;
    const int2* items;      // (field, sub-range), most expensive first
    int nitems;
    unsigned int* queue;    // work counter, zero before the launch
    void* work;
    size_t work_stride;
    double tol_abs;
    int max_iter_cold, max_iter_warm, predictor;
    int root_refresh;
    int near_cap;           // shared-memory rows of the split (0: none)
    int near_ext;           // tracer_near_ext(CT<float>::TS stars, near_cap)
};

// One field's points for the FP64 rescue of uncertified points.
struct RescueTask {
    const StarD* stars;
    const SmoothPoly* poly;
    int n, nr;
    double kappa_s, gamma;
    int64_t m;
    const double2* phase;
    double2* z;
    double2* w;
    DevReport* rep;
};
constexpr int RESCUE_MAX_POINTS = 65536;
// list entries: (field, row, column, 0); *nlist counts entries (may exceed max_list)
cudaError_t launch_rescue(const RescueTask* host_task, const RescueTask* dev_tasks, const int4* list, const int* nlist,
                          int max_list, double tol_abs, int max_iter, cudaStream_t st);

int tracer_batch_blocks_per_sm(int threads, int near_cap);
cudaError_t launch_phase_batch(const TraceTask* tasks, int count, int64_t max_m, cudaStream_t st);
cudaError_t launch_trace_batch(const BatchTraceArgs& b, int grid, int threads, cudaStream_t st);
cudaError_t launch_seam_join_batch(const TraceTask* tasks, int count, const int2* seams, int nseams, int max_nr,
                                   cudaStream_t st);

// Workspace layout of cc_critical_curves (byte offsets from the workspace base).
struct CurveLayout {
    int S;
    int threads;
    int G;                 // CTAs per sub-range (cluster size; 1 = one CTA)
    size_t elem;           // bytes per tracer complex (8 FP32, 16 FP64)
    size_t off_phase, off_zrows, off_seam, off_iters, off_match, off_hits, off_perm, off_work,
        off_report, off_list, off_nlist, off_fmm, total;
    size_t off_ext;        // per tracing CTA: extent of the points it wrote (FP32 form)
    bool fmm;
    size_t work_stride;
};

// Cells per direction available to the near/far split of the tracer's root sum.
__host__ __device__ inline int near_cells_max(int nr) { return nr / 4 + 64; }
// Rows of up to this many roots keep the split's ordered positions in shared memory.
constexpr int NEAR_SMEM_NR = 4096;
size_t tracer_work_stride(int64_t nr, size_t elem);
size_t tracer_smem_bytes(bool fp64, int64_t n, int near_cap = 0);
bool tracer_near_ext(int64_t n, int near_cap);
int tracer_blocks_per_sm(bool fp64, int threads, int64_t n);
int subchain_count(int64_t m, int64_t nr, const cc_options& o, int sms, int blocks_per_sm);
constexpr int WIDE_MIN_NR = 4096;   // automatic cluster tracing from this many roots per row
int tracer_cluster_size(const cc_options& o, int64_t nr, bool fp64, int64_t m, int sms);
int tracer_max_clusters(int G, int threads, bool fp64);  // co-resident clusters of G tracing CTAs

cudaError_t launch_phase_table(double2* phase, int64_t m, cudaStream_t st);
cudaError_t launch_trace(const TraceArgs& a, bool fp64, cudaStream_t st);
// work, work_stride: the sub-ranges' tracer work areas (scratch of the FP32 form's grid join;
// nullptr: the full scan)
cudaError_t launch_seam_join(const void* zrows, const void* seam, int64_t m, int S, int64_t nr,
                             bool fp64, int32_t* match, int32_t* hits, int32_t* perm,
                             DevReport* rep, cudaStream_t st, void* work = nullptr, size_t work_stride = 0);
size_t seam_grid_bytes(int64_t nr);

// Polish + caustic (mixed form) and the FP64 finalisation.
struct PolishArgs {
    const FieldDev* f;
    int64_t m;
    int S;
    int64_t nr;
    const double2* phase;
    const float2* zrows;    // tracer output (FP32)
    const int32_t* perm;    // S x nr
    const int32_t* iters_in;
    double2* z_out;
    double2* w_out;         // may be null
    int32_t* iters_out;     // may be null
    DevReport* rep;
    double tol_cert;
    int max_polish;
    int hp_fp64;            // 1: native FP64 star sums, 0: double-float
    int4* rescue_list;      // uncertified points go here (field_id, row, column, 0)
    int* rescue_count;
    int field_id;
    const int* skip_if;     // direct polish does nothing when *skip_if != 0 (may be null)
    const float4* ext;      // far-field polish: ext_n partial extents of zrows from the tracer (null: the
    int ext_n;              // polish measures them itself)
};
constexpr int FMM_MIN_STARS = 128;
cudaError_t launch_polish(const PolishArgs& a, cudaStream_t st);
// Far-field (local-expansion) polish: scratch of fmm_workspace_bytes(points) bytes; falls back
// to the direct polish on the device when its tables do not fit.
size_t fmm_workspace_bytes(int64_t points);
cudaError_t launch_polish_fmm(const PolishArgs& a, void* ws, cudaStream_t st);
// Batched polish: a device table of per-field task records (polish_task_bytes() each,
// filled on the host by polish_task_fill), blocks of all fields in one launch.
int64_t polish_blocks(int64_t points);
size_t polish_task_bytes();
void polish_task_fill(const PolishArgs& a, int64_t first_block, void* out);
cudaError_t launch_polish_batch(const void* tasks, int count, int64_t total_blocks, cudaStream_t st);

struct FinalizeArgs {
    int64_t m;
    int S;
    int64_t nr;
    const double2* zrows;
    const int32_t* perm;
    const int32_t* iters_in;
    double2* z_out;
    int32_t* iters_out;
};
cudaError_t launch_finalize_fp64(const FinalizeArgs& a, cudaStream_t st);

cudaError_t launch_map_caustics(const FieldDev& f, const double2* z, int64_t count, double2* w,
                                int hp_fp64, cudaStream_t st);

// Rasterisation.
cudaError_t launch_crossing_map(const double2* w, int64_t rows, int64_t nr, double x0, double x1,
                                double y0, double y1, int32_t W, int32_t H, int32_t* ncc,
                                cudaStream_t st);
size_t distance_workspace_bytes(int32_t W, int32_t H);
cudaError_t launch_moving_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, float c, float s,
                                       double* d_out, cudaStream_t st);
cudaError_t launch_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                                double* d_out, void* ws, cudaStream_t st);

// Device description, device index and options of a field (cc_field is opaque elsewhere).
const FieldDev* field_dev(const cc_field* f, int* device, cc_options* opt);

// Set the thread's last-error message (as the C ABI functions do) and return code.
int api_error(int code, const char* msg);

// Subchain of a row: rows [b_s, b_{s+1}) belong to s, row m to S-1; b_s = floor(s m / S).
__host__ __device__ __forceinline__ int64_t subchain_begin(int64_t s, int64_t m, int64_t S) {
    return (s * m) / S;
}
__host__ __device__ __forceinline__ int subchain_of_row(int64_t j, int64_t m, int64_t S) {
    if (j >= m) return (int)(S - 1);
    int64_t s = (j * S) / m;
    while (s + 1 < S && subchain_begin(s + 1, m, S) <= j) s++;
    while (s > 0 && subchain_begin(s, m, S) > j) s--;
    return (int)s;
}
// The same in 32-bit unsigned arithmetic where (m + 1) S < 2^32 (then every product below
// fits), else the 64-bit form: equal results, a fraction of the instructions.
__device__ __forceinline__ int subchain_of_row_fast(int64_t j, int64_t m, int64_t S) {
    if ((m + 1) * S >= (int64_t)1 << 32) return subchain_of_row(j, m, S);
    const unsigned jj = (unsigned)j, mm = (unsigned)m, SS = (unsigned)S;
    if (jj >= mm) return (int)(SS - 1);
    unsigned q = jj * SS / mm;
    while (q + 1 < SS && (q + 1) * mm / SS <= jj) q++;
    while (q > 0 && q * mm / SS > jj) q--;
    return (int)q;
}

}  // namespace ccg
