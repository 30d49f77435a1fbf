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

// Device-side copy of a field's stars in the layouts the kernels read.
struct FieldDev {
    int64_t n;
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
    float4* tcoeff;   // nbx * nby * TFMM_P: (U_k re, U_k im, L_k re, L_k im)
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
    int threads;
};

// One field of a batched launch (device table entry).
struct TraceTask {
    const void* stars;     // FP32 star records
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
};

// One field's points for the FP64 rescue of uncertified points.
struct RescueTask {
    const StarD* stars;
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

int tracer_batch_blocks_per_sm(int threads);
cudaError_t launch_phase_batch(const TraceTask* tasks, int count, int64_t max_m, cudaStream_t st);
cudaError_t launch_trace_batch(const BatchTraceArgs& b, int grid, int threads, cudaStream_t st);
cudaError_t launch_seam_join_batch(const TraceTask* tasks, int count, const int2* seams, int nseams, int max_nr,
                                   cudaStream_t st);

// Workspace layout of cc_critical_curves (byte offsets from the workspace base).
struct CurveLayout {
    int S;
    int threads;
    size_t elem;           // bytes per tracer complex (8 FP32, 16 FP64)
    size_t off_phase, off_zrows, off_seam, off_iters, off_match, off_hits, off_perm, off_work,
        off_report, off_list, off_nlist, off_fmm, total;
    bool fmm;
    size_t work_stride;
};

size_t tracer_work_stride(int64_t nr, size_t elem);
size_t tracer_smem_bytes(bool fp64);
int tracer_blocks_per_sm(bool fp64, int threads);
int subchain_count(int64_t m, int64_t nr, const cc_options& o, int sms, int blocks_per_sm);

cudaError_t launch_phase_table(double2* phase, int64_t m, cudaStream_t st);
cudaError_t launch_trace(const TraceArgs& a, bool fp64, cudaStream_t st);
cudaError_t launch_seam_join(const void* zrows, const void* seam, int64_t m, int S, int64_t nr,
                             bool fp64, int32_t* match, int32_t* hits, int32_t* perm,
                             DevReport* rep, cudaStream_t st);

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

}  // namespace ccg
