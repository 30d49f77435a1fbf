// Shared device helpers of libccgpu: FP32/FP64 complex arithmetic and double-float
// ("df": an unevaluated sum hi + lo of two FP32 numbers, ~48-bit significand) built from
// error-free transformations.  Used only by the CUDA library.
//
// Error-free transformations (all with IEEE round-to-nearest intrinsics that the compiler
// never contracts or reassociates):
//   two_sum      Knuth (TAOCP vol. 2, 4.2.2): s + e == a + b exactly.
//   fast_two_sum Dekker (1971), requires |a| >= |b| (or a == 0).
//   two_prod     with one FMA: p + e == a * b exactly.
// Reciprocal: one Newton-Raphson step y' = y + y (1 - a y) on the hardware FP32
// reciprocal approximation, with the residual 1 - a y formed from an exact product.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace ccg {

// ----------------------------------------------------------------------------------
// FP32
// ----------------------------------------------------------------------------------
__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// ----------------------------------------------------------------------------------
// Small integers <-> float
// ----------------------------------------------------------------------------------
// Integer <-> float without conversion instructions (which share the FP64 pipe's low rate on
// this part): adding an integer to the bits of 1.5 * 2^23 steps its value by exactly one per
// unit, so for |x| < 2^22 the value is 1.5 * 2^23 + x, and an FP32 sum with 1.5 * 2^23
// rounds to the nearest integer.
constexpr float MAGIC_F = 12582912.0f;  // 1.5 * 2^23
constexpr int MAGIC_I = 0x4B400000;     // its bits
__device__ __forceinline__ float i2f_small(int x) { return __int_as_float(MAGIC_I + x) - MAGIC_F; }  // |x| < 2^22
__device__ __forceinline__ int ceil_small(float x) {  // |x| < 2^21
    const float t = x + MAGIC_F;
    const int n = __float_as_int(t) - MAGIC_I;
    return (t - MAGIC_F) < x ? n + 1 : n;
}
__device__ __forceinline__ int floor_small(float x) {  // |x| < 2^21
    const float t = x + MAGIC_F;
    const int n = __float_as_int(t) - MAGIC_I;
    return (t - MAGIC_F) > x ? n - 1 : n;
}

// ----------------------------------------------------------------------------------
// double-float
// ----------------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h) { return df{h, 0.0f}; }

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df{s, e};
}

__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float e = __fsub_rn(b, __fsub_rn(s, a));
    return df{s, e};
}

__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    float e = __fmaf_rn(a, b, -p);
    return df{p, e};
}

__device__ __forceinline__ df df_neg(df a) { return df{-a.hi, -a.lo}; }

// a + b; absolute error O(2^-48 (|a| + |b|)), enough here because every sum either has
// operands of one sign or is a difference whose result is used in absolute terms.
__device__ __forceinline__ df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, df_neg(b)); }

// a (double-float) minus b (plain float), e.g. a root coordinate minus nothing.
__device__ __forceinline__ df df_sub_f(df a, float b) {
    df s = two_sum(a.hi, -b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.lo, p.lo);
    e = __fmaf_rn(a.lo, b.hi, e);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_mul_f(df a, float b) {
    df p = two_prod(a.hi, b);
    float e = __fmaf_rn(a.lo, b, p.lo);
    return fast_two_sum(p.hi, e);
}

__device__ __forceinline__ df df_sqr(df a) {
    df p = two_prod(a.hi, a.hi);
    float e = __fmaf_rn(__fadd_rn(a.hi, a.hi), a.lo, p.lo);
    return fast_two_sum(p.hi, e);
}

// 1 / a for a > 0 (a.hi normal): relative error ~2^-46.
__device__ __forceinline__ df df_rcp(df a) {
    float y = rcp_approx(a.hi);
    df p = two_prod(a.hi, y);                // a.hi * y exactly
    float t = __fsub_rn(1.0f, p.hi);          // exact: p.hi is within 2^-22 of 1
    t = __fsub_rn(t, p.lo);
    t = __fmaf_rn(-a.lo, y, t);               // t = 1 - a * y (to ~2^-47 relative)
    return fast_two_sum(y, __fmul_rn(y, t));
}

__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// A coordinate as three floats h + m + l (~72-bit significand) and the difference of two
// such coordinates as a double-float: the pieces are subtracted with error-free sums, so
// the difference of two close points keeps its full relative precision (the caustic
// point of a root next to a star depends on that difference at 1 / |d|^2).
struct tf {
    float h, m, l;
};

__device__ __forceinline__ tf tf_from_double(double x) {
    const float h = __double2float_rn(x);
    const double r = x - (double)h;
    const float m = __double2float_rn(r);
    const float l = __double2float_rn(r - (double)m);
    return tf{h, m, l};
}

__device__ __forceinline__ df tf_sub(const tf& a, float bh, float bm, float bl) {
    const df s = two_sum(a.h, -bh);
    const df t = two_sum(a.m, -bm);
    const df u = two_sum(s.hi, t.hi);
    const float lo = __fadd_rn(__fadd_rn(s.lo, t.lo), __fadd_rn(u.lo, __fsub_rn(a.l, bl)));
    return fast_two_sum(u.hi, lo);
}

// a + b for a triple-float a and a float b: error-free sums throughout, the rounding of
// the two smallest pieces aside (~2^-70 relative).
__device__ __forceinline__ tf tf_add_f(const tf& a, float b) {
    const df s = two_sum(a.h, b);
    const df t = two_sum(a.m, s.lo);
    const df u = two_sum(s.hi, t.hi);
    const df v = two_sum(u.lo, __fadd_rn(t.lo, a.l));
    return tf{u.hi, v.hi, v.lo};
}

__device__ __forceinline__ double tf_to_double(const tf& a) {
    return ((double)a.h + (double)a.m) + (double)a.l;
}

__device__ __forceinline__ df df_from_double(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df{h, l};
}

// ----------------------------------------------------------------------------------
// Status words shared by the kernels (device-side report, reduced by atomics)
// ----------------------------------------------------------------------------------
struct DevReport {
    unsigned long long root_iterations;
    unsigned long long cold_root_iterations;
    unsigned long long unconverged;
    unsigned long long polish_passes;
    unsigned long long uncertified;
    unsigned long long seam_ambiguous;
    unsigned long long jumped;   // polish moved a root further than the tracer's scale
    unsigned long long rescued_points;  // uncertified points re-solved in FP64 (converged)
    unsigned long long star_terms;      // tracer: star terms summed directly
    unsigned long long far_evals;       // tracer: root updates that used a cell expansion
    unsigned long long root_terms;      // tracer: root-root terms summed
    unsigned long long split_redone_rows;  // tracer: rows solved again with the exact root sum
    int max_iter_row;
    double max_err_est;          // stored as the bit pattern of a non-negative double
};

__device__ __forceinline__ void atomic_max_double_nonneg(double* addr, double v) {
    // non-negative doubles order like their bit patterns as signed 64-bit integers
    atomicMax((long long*)addr, __double_as_longlong(v));
}

}  // namespace ccg
