// High-precision polish of the FP32 critical points, fused with the caustic mapping.
//
// For every traced point z0 (all rows, all roots; fully parallel) one pass over the stars
// gives, at z,
//   S1 = sum m_i/(z - z_i),  S2 = sum m_i/(z - z_i)^2            (high precision)
//   S3 = sum m_i/(z - z_i)^3, S4 = sum m_i/(z - z_i)^4            (FP32)
// so that F = gamma + S2 - (1 - kappa_s) e^{-i phi} (Sec. 3.1), F' = -2 S3, and the Newton
// step delta = -F/F' lands within |F''/(2F')| |delta|^2 = 1.5 |S4/S3| |delta|^2 of the root
// (plus the FP32 error of F').  Passes repeat until that estimate is below tol_cert.  The
// caustic point (Sec. 3.1 lens equation, Sec. 5.1) of the final z = z_p + delta follows
// from the same sums by Taylor expansion of S1 about z_p:
//   S1(z_p + delta) = S1 - S2 delta + S3 delta^2 - S4 delta^3 + O(delta^4 sum m/d^5),
//   w = (1 - kappa_s) z + gamma conj(z) - conj(S1(z)).
// High precision is either double-float (FP32 pairs on the FP32 pipes; GB300 runs FP64
// at ~1/70 of the FP32 rate) or native FP64.
#include <float.h>
#include <string.h>

#include "cc_internal.h"

namespace ccg {

constexpr int PB_THREADS = 256;
constexpr int TSB = 2048;  // stars per shared-memory tile

struct PolishK {
    const SmoothPoly* poly;  // rectangular field: smooth-sheet polynomial; nullptr for the disc
    const float4* dfp;
    const float2* dfm;
    const float2* dtf;
    const StarD* s64;
    int n;
    int64_t nr, m, points;
    int S;
    double kappa_s, gamma;
    double wgx, wgy;      // 1 - kappa_s + gamma, 1 - kappa_s - gamma (the lens map's linear terms)
    const double2* phase;
    const float2* zrows;
    const int32_t* perm;
    const int32_t* iters_in;
    double2* z_out;
    double2* w_out;
    int32_t* iters_out;
    DevReport* rep;
    double tol_cert;
    int max_polish;
    int unit_mass;        // batched launches: all masses equal to 1
    int64_t first_block;  // batched launches: first block of this field
    int4* rescue_list;    // uncertified points, for the FP64 rescue
    int* rescue_count;
    int field_id;
    const int* skip_if;   // direct polish: return at once when *skip_if != 0 (far-field path took over)
};

struct Sums {
    df S1x, S1y, S2x, S2y;
    float s3x, s3y, s4x, s4y, a3;
};

// One star in double-float.  d = z - z_i; r2 = |d|^2; inv = 1/r2; q = m inv;
// m/d = q conj(d); m/d^2 = q inv conj(d)^2 with conj(d)^2 = (dx^2 - dy^2, -2 dx dy).
template <bool UNIT>
__device__ __forceinline__ void star_df(const tf& zx, const tf& zy, const float4 p, const float2 p3, const float2 mm,
                                        Sums& s) {
    const df dx = tf_sub(zx, p.x, p.y, p3.x);
    const df dy = tf_sub(zy, p.z, p.w, p3.y);
    const df dx2 = df_sqr(dx), dy2 = df_sqr(dy);
    const df r2 = df_add(dx2, dy2);
    const df inv = df_rcp(r2);
    const df q = UNIT ? inv : df_mul(df{mm.x, mm.y}, inv);
    // S1 += m/d = q (dx, -dy)
    s.S1x = df_add(s.S1x, df_mul(q, dx));
    s.S1y = df_sub(s.S1y, df_mul(q, dy));
    // S2 += m/d^2 = q inv (dx^2 - dy^2, -2 dx dy)
    const df qi = df_mul(q, inv);
    const df a = df_sub(dx2, dy2);
    const df b = df_mul(dx, dy);
    const df t2x = df_mul(qi, a);
    const df t2b = df_mul(qi, b);
    const df t2y = df{-2.0f * t2b.hi, -2.0f * t2b.lo};
    s.S2x = df_add(s.S2x, t2x);
    s.S2y = df_add(s.S2y, t2y);
    // FP32: u = 1/d, S3 += (m/d^2) u, S4 += (m/d^3) u
    const float ux = dx.hi * inv.hi, uy = -dy.hi * inv.hi;
    const float t3x = fmaf(t2x.hi, ux, -t2y.hi * uy);
    const float t3y = fmaf(t2x.hi, uy, t2y.hi * ux);
    s.s3x += t3x;
    s.s3y += t3y;
    s.a3 += fabsf(t3x) + fabsf(t3y);
    s.s4x += fmaf(t3x, ux, -t3y * uy);
    s.s4y += fmaf(t3x, uy, t3y * ux);
}

struct SumsD {
    double S1x, S1y, S2x, S2y;
    float s3x, s3y, s4x, s4y, a3;
};

__device__ __forceinline__ void star_fp64(double zx, double zy, const StarD& st, SumsD& s) {
    const double dx = zx - st.x, dy = zy - st.y;
    const double dx2 = dx * dx, dy2 = dy * dy;
    const double r2 = dx2 + dy2;
    const double inv = 1.0 / r2;
    const double q = st.z * inv;
    s.S1x = fma(q, dx, s.S1x);
    s.S1y = fma(-q, dy, s.S1y);
    const double qi = q * inv;
    const double t2x = qi * (dx2 - dy2);
    const double t2y = -2.0 * qi * (dx * dy);
    s.S2x += t2x;
    s.S2y += t2y;
    const float ux = (float)(dx * inv), uy = (float)(-dy * inv);
    const float fx = (float)t2x, fy = (float)t2y;
    const float t3x = fmaf(fx, ux, -fy * uy);
    const float t3y = fmaf(fx, uy, fy * ux);
    s.s3x += t3x;
    s.s3y += t3y;
    s.a3 += fabsf(t3x) + fabsf(t3y);
    s.s4x += fmaf(t3x, ux, -t3y * uy);
    s.s4y += fmaf(t3x, uy, t3y * ux);
}

// Newton step, certification and (when done) output.  All in FP64: a few dozen operations
// per point and pass against thousands in the star loop.  Returns true when finished.
__device__ __forceinline__ bool polish_epilogue(const PolishK& K, int64_t point, int64_t row,
                                                double S1x, double S1y, double S2x, double S2y,
                                                float s3x, float s3y, float s4x, float s4y, float a3,
                                                double& zx, double& zy, float z0x, float z0y,
                                                int pass, int32_t it_in, double& est_out, double s2_err = 0.0) {
    const double oms = 1.0 - K.kappa_s;
    const double2 ph = K.phase[row];
    double Fx = K.gamma + S2x - oms * ph.x;
    double Fy = S2y + oms * ph.y;
    const float s3sx = s3x, s3sy = s3y, s4sx = s4x, s4sy = s4y;  // star sums, for the Taylor of S1
    if (K.poly) {
        // rectangular field: F -= Q, F' = -2 (S3 + Q'/2), F'' = 6 (S4 - Q''/6)
        double Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa;
        poly_eval<double>(K.poly, zx, zy, Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa);
        Fx -= Qx;
        Fy -= Qy;
        s3x += (float)(0.5 * Q1x);
        s3y += (float)(0.5 * Q1y);
        s4x -= (float)(Q2x / 6.0);
        s4y -= (float)(Q2y / 6.0);
        a3 += (float)(0.5 * (fabs(Q1x) + fabs(Q1y)));
    }
    // delta = -F / F' = F / (2 S3)
    const double tx = 2.0 * (double)s3x, ty = 2.0 * (double)s3y;
    const double den = tx * tx + ty * ty;
    double dx = 0.0, dy = 0.0;
    if (den > 0.0) {
        dx = (Fx * tx + Fy * ty) / den;
        dy = (Fy * tx - Fx * ty) / den;
    }
    const double ad = sqrt(dx * dx + dy * dy);
    const double s3a = sqrt(den) * 0.5;
    const double s4a = sqrt((double)s4x * s4x + (double)s4y * s4y);
    double est;
    if (s3a > 0.0)
        est = 1.5 * ad * ad * s4a / s3a + ad * 4.0 * (double)FLT_EPSILON * (double)a3 / s3a + 0.5 * s2_err / s3a;
    else
        est = (ad == 0.0) ? 0.0 : DBL_MAX;
    const double nzx = zx + dx, nzy = zy + dy;
    const bool done = est < K.tol_cert || pass + 1 >= K.max_polish;
    if (!done) {
        zx = nzx;
        zy = nzy;
        return false;
    }
    // S1 at the final point by Taylor expansion about the evaluation point.
    const double d2x = dx * dx - dy * dy, d2y = 2.0 * dx * dy;       // delta^2
    const double d3x = d2x * dx - d2y * dy, d3y = d2x * dy + d2y * dx; // delta^3
    const double S1nx = S1x - (S2x * dx - S2y * dy) + ((double)s3sx * d2x - (double)s3sy * d2y) -
                        ((double)s4sx * d3x - (double)s4sy * d3y);
    const double S1ny = S1y - (S2x * dy + S2y * dx) + ((double)s3sx * d2y + (double)s3sy * d2x) -
                        ((double)s4sx * d3y + (double)s4sy * d3x);
    K.z_out[point] = make_double2(nzx, nzy);
    if (K.w_out) {
        double wx = oms * nzx + K.gamma * nzx - S1nx;
        double wy = oms * nzy - K.gamma * nzy + S1ny;
        if (K.poly) {
            const double2 V = poly_V(K.poly, nzx, nzy);
            wx += V.x;
            wy += V.y;
        }
        K.w_out[point] = make_double2(wx, wy);
    }
    if (K.iters_out) K.iters_out[point] = it_in;
    if (est >= K.tol_cert) {
        atomicAdd(&K.rep->uncertified, 1ull);
        if (K.rescue_list) {
            const int idx = atomicAdd(K.rescue_count, 1);
            if (idx < RESCUE_MAX_POINTS)
                K.rescue_list[idx] = make_int4(K.field_id, (int)row, (int)(point - row * K.nr), 0);
        }
    }
    const double jx = nzx - (double)z0x, jy = nzy - (double)z0y;
    const double zs = 1.0 + sqrt(nzx * nzx + nzy * nzy);
    if (jx * jx + jy * jy > 1e-6 * zs * zs) atomicAdd(&K.rep->jumped, 1ull);
    est_out = est < K.tol_cert ? est : 0.0;  // certified points only; the caller reduces
    return true;
}

// Complex double-float and the rectangle's Q(z) in double-float (Horner in u = zeta^2,
// zeta = z/|c|): the residual F nearly cancels at a critical point, so Q enters it with
// the precision of the star sums.
struct dfc {
    df x, y;
};

// a1 b1 + a2 b2 in double-float with one normalisation: both high products and their sum
// exact (two_prod, two_sum), the error terms and the four low-part cross products gathered by
// FP32 adds and FMAs: 20 FP32 operations against 27 for two df_mul and a df_add, with the same
// ~2^-46 relative rounding (the final fast two-sum assumes, as df_add does, that the sum does
// not cancel below its accumulated error).
__device__ __forceinline__ df df_dot2(df a1, df b1, df a2, df b2) {
    const df p1 = two_prod(a1.hi, b1.hi), p2 = two_prod(a2.hi, b2.hi);
    const df s1 = two_sum(p1.hi, p2.hi);
    float e = __fadd_rn(__fadd_rn(p1.lo, p2.lo), s1.lo);
    e = __fmaf_rn(a1.hi, b1.lo, e);
    e = __fmaf_rn(a1.lo, b1.hi, e);
    e = __fmaf_rn(a2.hi, b2.lo, e);
    e = __fmaf_rn(a2.lo, b2.hi, e);
    return fast_two_sum(s1.hi, e);
}

__device__ __forceinline__ dfc dfc_mul(const dfc& a, const dfc& b) {
    return dfc{df_dot2(a.x, b.x, df_neg(a.y), b.y), df_dot2(a.x, b.y, a.y, b.x)};
}

__device__ __forceinline__ dfc poly_Q_df(const SmoothPoly* P, df zx, df zy) {
    const df ic = df{P->inv_acdf.x, P->inv_acdf.y};
    const df sx = df_mul(zx, ic), sy = df_mul(zy, ic);
    const dfc u = dfc{df_sub(df_sqr(sx), df_sqr(sy)), df_mul_f(df_mul(sx, sy), 2.f)};
    dfc p = dfc{df{P->qdf[P->K].x, P->qdf[P->K].y}, df{0.f, 0.f}};
    for (int k = P->K - 1; k >= 0; k--) {
        p = dfc_mul(p, u);
        p.x = df_add(p.x, df{P->qdf[k].x, P->qdf[k].y});
    }
    return p;
}

// Newton step delta = F / (2 S3) (F' = -2 S3, Eq. 7), certificate and, when done, the
// outputs, from double-float sums and a triple-float z.  The residual F = S2 + c with
// c = gamma - (1 - kappa_s) e^{-i phi} is a double-float sum: S2 nearly cancels c at a
// critical point, and the sum keeps the residual's full relative precision.  What only
// needs the relative precision of the FP32 sums S3 and S4 is FP32: the step, its length,
// the certificate (which charges the FP32 rounding of the step) and the delta^2, delta^3
// terms of the Taylor correction of S1.  FP64 is used for the outputs alone.
__device__ __forceinline__ bool polish_epilogue_df(const PolishK& K, int64_t point, int64_t row, const Sums& s,
                                                   const df& cx, const df& cy, tf& zx, tf& zy, float z0x, float z0y,
                                                   int pass, int32_t it_in, double& est_out, float s2_err = 0.f,
                                                   float s3_err = 0.f) {
    df Fx = df_add(s.S2x, cx), Fy = df_add(s.S2y, cy);
    float s3x = s.s3x, s3y = s.s3y, s4x = s.s4x, s4y = s.s4y, a3 = s.a3;
    if (K.poly) {
        // rectangular field: F -= Q (double-float), F' = -2 (S3 + Q'/2), F'' = 6 (S4 - Q''/6)
        const dfc Q = poly_Q_df(K.poly, df{zx.h, zx.m}, df{zy.h, zy.m});
        Fx = df_sub(Fx, Q.x);
        Fy = df_sub(Fy, Q.y);
        float Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa;
        poly_eval<float>(K.poly, zx.h, zy.h, Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa);
        s3x += 0.5f * Q1x;
        s3y += 0.5f * Q1y;
        s4x -= Q2x * (1.f / 6.f);
        s4y -= Q2y * (1.f / 6.f);
        a3 += 0.5f * (fabsf(Q1x) + fabsf(Q1y)) + qa * (float)K.poly->K * K.poly->inv_acf;
    }
    const float fx = __fadd_rn(Fx.hi, Fx.lo), fy = __fadd_rn(Fy.hi, Fy.lo);
    const float tx = 2.f * s3x, ty = 2.f * s3y;
    const float den = fmaf(tx, tx, ty * ty);
    float dx = 0.f, dy = 0.f, est;
    if (den > 0.f && den < FLT_MAX) {
        const float rd = __frcp_rn(den);
        dx = fmaf(fx, tx, fy * ty) * rd;
        dy = fmaf(fy, tx, -fx * ty) * rd;
        const float ad = sqrtf(fmaf(dx, dx, dy * dy));
        const float s3a = 0.5f * sqrtf(den);
        const float s4a = sqrtf(fmaf(s4x, s4x, s4y * s4y));
        const float r3 = __frcp_rn(s3a);
        est = 1.5f * ad * ad * s4a * r3 + ad * ((4.f * FLT_EPSILON * a3 + s3_err) * r3 + 8.f * FLT_EPSILON) +
              0.5f * s2_err * r3;
    } else {
        // F' vanishes (or the sums overflowed): no step, certified only at an exact zero of F
        est = (fx == 0.f && fy == 0.f) ? 0.f : FLT_MAX;
    }
    const tf nzx = tf_add_f(zx, dx), nzy = tf_add_f(zy, dy);
    const bool done = est < (float)K.tol_cert || pass + 1 >= K.max_polish;
    if (!done) {
        zx = nzx;
        zy = nzy;
        return false;
    }
    // S1 at the final point by Taylor expansion about the evaluation point:
    // S1 - S2 delta + S3 delta^2 - S4 delta^3
    const float d2x = fmaf(dx, dx, -dy * dy), d2y = 2.f * dx * dy;
    const float d3x = fmaf(d2x, dx, -d2y * dy), d3y = fmaf(d2x, dy, d2y * dx);
    const float hx = fmaf(s.s3x, d2x, -s.s3y * d2y) - fmaf(s.s4x, d3x, -s.s4y * d3y);
    const float hy = fmaf(s.s3x, d2y, s.s3y * d2x) - fmaf(s.s4x, d3y, s.s4y * d3x);
    const df S1nx = df_add(df_sub(s.S1x, df_sub(df_mul_f(s.S2x, dx), df_mul_f(s.S2y, dy))), df{hx, 0.f});
    const df S1ny = df_add(df_sub(s.S1y, df_add(df_mul_f(s.S2x, dy), df_mul_f(s.S2y, dx))), df{hy, 0.f});
    const double ozx = tf_to_double(nzx), ozy = tf_to_double(nzy);
    K.z_out[point] = make_double2(ozx, ozy);
    if (K.w_out) {
        double wx = fma(K.wgx, ozx, -df_to_double(S1nx));
        double wy = fma(K.wgy, ozy, df_to_double(S1ny));
        if (K.poly) {
            const double2 V = poly_V(K.poly, ozx, ozy);
            wx += V.x;
            wy += V.y;
        }
        K.w_out[point] = make_double2(wx, wy);
    }
    if (K.iters_out) K.iters_out[point] = it_in;
    if (!(est < (float)K.tol_cert)) {
        atomicAdd(&K.rep->uncertified, 1ull);
        if (K.rescue_list) {
            const int idx = atomicAdd(K.rescue_count, 1);
            if (idx < RESCUE_MAX_POINTS)
                K.rescue_list[idx] = make_int4(K.field_id, (int)row, (int)(point - row * K.nr), 0);
        }
    }
    const float jx = nzx.h - z0x, jy = nzy.h - z0y;
    const float zs = 1.f + sqrtf(fmaf(nzx.h, nzx.h, nzy.h * nzy.h));
    if (fmaf(jx, jx, jy * jy) > 1e-6f * zs * zs) atomicAdd(&K.rep->jumped, 1ull);
    est_out = est < (float)K.tol_cert ? (double)est : 0.0;  // certified points only; the caller reduces
    return true;
}

// c = gamma - (1 - kappa_s) e^{-i phi} of a row as double-float (F = S2 + c)
__device__ __forceinline__ void row_constant(const PolishK& K, int64_t row, df& cx, df& cy) {
    const double oms = 1.0 - K.kappa_s;
    const double2 ph = K.phase[row];
    cx = df_from_double(fma(-oms, ph.x, K.gamma));
    cy = df_from_double(oms * ph.y);
}

template <bool UNIT, bool FP64>
__device__ __forceinline__ void polish_body(const PolishK& K, const int64_t blk, unsigned char* smem,
                                            unsigned long long* s_passes_p) {
    float4* sp = (float4*)smem;
    float2* sm = (float2*)(smem + TSB * sizeof(float4));
    float2* st3 = (float2*)(smem + TSB * (sizeof(float4) + sizeof(float2)));
    StarD* sd = (StarD*)smem;
    unsigned long long& s_passes = *s_passes_p;
    const int tid = threadIdx.x;
    if (K.skip_if && *K.skip_if) return;  // uniform across the grid
    const int64_t point = blk * (int64_t)PB_THREADS + tid;
    const bool valid = point < K.points;
    int64_t row = 0;
    float z0x = 0.f, z0y = 0.f;
    int32_t it_in = 0;
    if (valid) {
        row = point / K.nr;
        const int64_t g = point - row * K.nr;
        const int s = subchain_of_row_fast(row, K.m, K.S);
        const int32_t k = K.perm[(size_t)s * K.nr + g];
        const float2 z0 = K.zrows[(size_t)row * K.nr + k];
        z0x = z0.x;
        z0y = z0.y;
        if (K.iters_out) it_in = K.iters_in[(size_t)row * K.nr + k];
    }
    double zx = z0x, zy = z0y;
    tf zxt = tf{z0x, 0.f, 0.f}, zyt = tf{z0y, 0.f, 0.f};
    df cx = df{0.f, 0.f}, cy = df{0.f, 0.f};
    if (!FP64 && valid) row_constant(K, row, cx, cy);
    bool need = valid;
    double est_max = 0.0;
    if (tid == 0) s_passes = 0;
    const bool resident = K.n <= TSB;
    if (resident) {
        if (FP64) {
            for (int j = tid; j < K.n; j += PB_THREADS) sd[j] = K.s64[j];
        } else {
            for (int j = tid; j < K.n; j += PB_THREADS) {
                sp[j] = K.dfp[j];
                sm[j] = K.dfm[j];
                st3[j] = K.dtf[j];
            }
        }
    }
    for (int pass = 0; pass < K.max_polish; pass++) {
        if (!__syncthreads_or(need)) break;
        if (need) atomicAdd(&s_passes, 1ull);
        if (FP64) {
            SumsD s = {0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f};
            for (int t0 = 0; t0 < K.n; t0 += TSB) {
                const int tn = min(TSB, K.n - t0);
                if (!resident) {
                    __syncthreads();
                    for (int j = tid; j < tn; j += PB_THREADS) sd[j] = K.s64[t0 + j];
                    __syncthreads();
                }
                if (need)
                    for (int j = 0; j < tn; j++) star_fp64(zx, zy, sd[j], s);
            }
            double est = 0.0;
            if (need && polish_epilogue(K, point, row, s.S1x, s.S1y, s.S2x, s.S2y, s.s3x, s.s3y, s.s4x,
                                        s.s4y, s.a3, zx, zy, z0x, z0y, pass, it_in, est)) {
                need = false;
                est_max = fmax(est_max, est);
            }
        } else {
            Sums s;
            s.S1x = s.S1y = s.S2x = s.S2y = df{0.f, 0.f};
            s.s3x = s.s3y = s.s4x = s.s4y = s.a3 = 0.f;
            for (int t0 = 0; t0 < K.n; t0 += TSB) {
                const int tn = min(TSB, K.n - t0);
                if (!resident) {
                    __syncthreads();
                    for (int j = tid; j < tn; j += PB_THREADS) {
                        sp[j] = K.dfp[t0 + j];
                        sm[j] = K.dfm[t0 + j];
                        st3[j] = K.dtf[t0 + j];
                    }
                    __syncthreads();
                }
                if (need) {
#pragma unroll 2
                    for (int j = 0; j < tn; j++) star_df<UNIT>(zxt, zyt, sp[j], st3[j], sm[j], s);
                }
            }
            double est = 0.0;
            if (need && polish_epilogue_df(K, point, row, s, cx, cy, zxt, zyt, z0x, z0y, pass, it_in, est)) {
                need = false;
                est_max = fmax(est_max, est);
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) est_max = fmax(est_max, __shfl_xor_sync(0xffffffffu, est_max, off));
    if ((tid & 31) == 0 && est_max > 0.0) atomic_max_double_nonneg(&K.rep->max_err_est, est_max);
    __syncthreads();
    if (tid == 0 && s_passes) atomicAdd(&K.rep->polish_passes, s_passes);
}

template <bool UNIT, bool FP64>
__global__ void __launch_bounds__(PB_THREADS) polish_kernel(PolishK K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_passes;
    polish_body<UNIT, FP64>(K, blockIdx.x, smem, &s_passes);
}

// The direct polish as the far-field path's fallback: a small grid striding over the blocks,
// so that the usual case (*skip_if set: the far-field path did the job) costs one short launch.
template <bool UNIT, bool FP64>
__global__ void __launch_bounds__(PB_THREADS) polish_fallback_kernel(PolishK K, int64_t nblocks) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_passes;
    if (*K.skip_if) return;  // uniform across the grid (set before this launch)
    for (int64_t blk = blockIdx.x; blk < nblocks; blk += gridDim.x) {
        polish_body<UNIT, FP64>(K, blk, smem, &s_passes);
        __syncthreads();
    }
}

// Batched: the blocks of all fields in one launch; each field's points start on a block
// boundary, so every block polishes points of one field against that field's stars.
__global__ void __launch_bounds__(PB_THREADS) polish_batch_kernel(const PolishK* tasks, int count) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_passes;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tasks[mid].first_block <= (int64_t)blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    const PolishK K = tasks[lo];
    const int64_t blk = (int64_t)blockIdx.x - K.first_block;
    if (K.unit_mass) polish_body<true, false>(K, blk, smem, &s_passes);
    else polish_body<false, false>(K, blk, smem, &s_passes);
}

static PolishK make_polish_k(const PolishArgs& a) {
    PolishK K;
    K.poly = a.f->poly;
    K.dfp = a.f->star_dfp;
    K.dfm = a.f->star_dfm;
    K.dtf = a.f->star_tf;
    K.s64 = a.f->star64;
    K.n = (int)a.f->n;
    K.nr = a.nr;
    K.m = a.m;
    K.points = (a.m + 1) * a.nr;
    K.S = a.S;
    K.kappa_s = a.f->kappa_s;
    K.gamma = a.f->gamma;
    K.wgx = 1.0 - a.f->kappa_s + a.f->gamma;
    K.wgy = 1.0 - a.f->kappa_s - a.f->gamma;
    K.phase = a.phase;
    K.zrows = a.zrows;
    K.perm = a.perm;
    K.iters_in = a.iters_in;
    K.z_out = a.z_out;
    K.w_out = a.w_out;
    K.iters_out = a.iters_out;
    K.rep = a.rep;
    K.tol_cert = a.tol_cert;
    K.max_polish = a.max_polish < 1 ? 1 : a.max_polish;
    K.unit_mass = a.f->unit_mass ? 1 : 0;
    K.first_block = 0;
    K.rescue_list = a.rescue_list;
    K.rescue_count = a.rescue_count;
    K.field_id = a.field_id;
    K.skip_if = a.skip_if;
    return K;
}

int64_t polish_blocks(int64_t points) { return (points + PB_THREADS - 1) / PB_THREADS; }

size_t polish_task_bytes() { return sizeof(PolishK); }

void polish_task_fill(const PolishArgs& a, int64_t first_block, void* out) {
    PolishK K = make_polish_k(a);
    K.first_block = first_block;
    memcpy(out, &K, sizeof K);
}

cudaError_t launch_polish_batch(const void* tasks, int count, int64_t total_blocks, cudaStream_t st) {
    if (total_blocks <= 0) return cudaSuccess;
    const size_t smem = TSB * (sizeof(float4) + 2 * sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(polish_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    polish_batch_kernel<<<(unsigned)total_blocks, PB_THREADS, smem, st>>>((const PolishK*)tasks, count);
    return cudaGetLastError();
}

cudaError_t launch_polish(const PolishArgs& a, cudaStream_t st) {
    PolishK K = make_polish_k(a);
    const unsigned blocks = (unsigned)((K.points + PB_THREADS - 1) / PB_THREADS);
    const size_t smem_df = TSB * (sizeof(float4) + 2 * sizeof(float2));
    const size_t smem_d = TSB * sizeof(StarD);
    int sms = 1, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const unsigned fb_blocks = (unsigned)std::min<int64_t>(blocks, (int64_t)sms * 8);
    cudaError_t e;
#define CC_LAUNCH_POLISH(U, D, SM)                                                                     \
    do {                                                                                               \
        if (K.skip_if) {                                                                               \
            e = cudaFuncSetAttribute(polish_fallback_kernel<U, D>,                                     \
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(SM));          \
            if (e != cudaSuccess) return e;                                                            \
            polish_fallback_kernel<U, D><<<fb_blocks, PB_THREADS, SM, st>>>(K, (int64_t)blocks);       \
        } else {                                                                                       \
            e = cudaFuncSetAttribute(polish_kernel<U, D>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                     (int)(SM));                                                       \
            if (e != cudaSuccess) return e;                                                            \
            polish_kernel<U, D><<<blocks, PB_THREADS, SM, st>>>(K);                                    \
        }                                                                                              \
    } while (0)
    if (a.hp_fp64)
        CC_LAUNCH_POLISH(false, true, smem_d);
    else if (a.f->unit_mass)
        CC_LAUNCH_POLISH(true, false, smem_df);
    else
        CC_LAUNCH_POLISH(false, false, smem_df);
#undef CC_LAUNCH_POLISH
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Far-field polish (the star-sum splitting of Sec. 4.1, fast multipole method): the plane
// of the traced points is cut into square cells of side b.  For a point in cell B the
// stars of the 5x5 block of cells around B are summed directly in double-float, as in the
// direct polish; the other stars ("far": at least 2.5 b from B's centre c, while the point
// is within 0.72 b of c) enter through the local expansion of B,
//   S1_far(z) = sum_far m_i / (z - z_i) = sum_k L_k (z - c)^k,  L_k = -sum_far m_i / (z_i - c)^(k+1),
// truncated at FMM_P terms.  With D1, D2, D3 the first three derivatives of S1_far:
// S2 = -D1, S3 = D2 / 2, S4 = -D3 / 6, all from the same coefficients (Horner with
// derivatives: double-float for S1, S2, FP32 for S3, S4).  The truncation bound (ratio
// rho <= 0.29, rho^31 ~ 1e-17) joins the polish error estimate.  Cells, expansions and
// near lists are built on the device from the traced points, so the whole path stays
// asynchronous.
// ----------------------------------------------------------------------------------
constexpr int FMM_P = 32;
constexpr int FMM_K0 = 20;  // expansion terms k >= FMM_K0 evaluated in FP32 (see fmm_polish_kernel)
constexpr int FMM_K = 2;
constexpr int FMM_G = 2048;

struct FmmParams {
    float x0, y0, b, inv_b;  // cell (0, 0) lower-left corner, cell side and its inverse (FP32)
    int nbx, nby;
    int ok;                   // 1 while every table is complete (else the direct polish runs)
    int nocc;                 // occupied cells
    int ncocc;                // occupied coarse cells (FMM_F x FMM_F cells each)
    int pool_used;            // near-list entries handed out
    int cpool_used;           // coarse star-list entries handed out
    int cap, pool_cap;
    int sub_used;             // sub-cell table entries handed out
};

struct BoxInfo {
    float4 c;        // centre as double-float (x_hi, x_lo, y_hi, y_lo)
    int near_off, near_cnt;
    float s2_err;    // truncation bound of S2_far (theta_*^-2) plus the FP32 rounding of terms >= FMM_K0
    float s2_trunc;  // the truncation part alone
};

// Sub-cells: each occupied cell is cut into FMM_SUB x FMM_SUB sub-cells, and the cell's
// 32-term expansion is re-centred exactly (a Taylor shift) at the centre of every sub-cell
// that holds a traced point (tables handed out from a pool of FMM_SUBPOOL).  A point within FMM_SUBR b of its sub-cell centre sees the far
// stars at a ratio of about 0.1 instead of 0.29, so FMM_PS terms of the re-centred
// polynomial, FMM_KS0 of them in double-float, hold what 32 (20) did; the dropped terms'
// exact bound, from the re-centred coefficients, joins the certificate.
constexpr int FMM_SUB = 4;
constexpr int FMM_SUB2 = FMM_SUB * FMM_SUB;
constexpr int FMM_PS = 16;            // terms kept at a sub-cell centre
constexpr int FMM_KS0 = 9;            // of which terms k >= FMM_KS0 in FP32
constexpr int FMM_OCC_ROWS = 64;     // rows per thread of the occupancy pass
constexpr int FMM_SUBPOOL = 1 << 20;  // sub-cell tables (occupied sub-cells) at most; cells beyond use the cell's
constexpr float FMM_SUBR = 0.185f;    // sub-cell radius / b: 1.05 x the half-diagonal sqrt(2)/8 (so that
                                      // |z - c| <= 0.375 sqrt(2) b + 0.185 b <= 0.72 b, the cell bound's radius)

struct SubInfo {
    float4 c;       // sub-cell centre as double-float
    float s2_err;   // bound on S2's error from the cell's truncation, the dropped terms and the FP32 part
    float s3_err;   // bound on S3's error from the dropped terms
    float r2;       // squared radius within which the bounds hold
    float pad;
};

// Binomial coefficients C(j, k), j, k < 32, as double-float (exact: C(31, 15) < 2^29).
struct BinomTable {
    float hi[32][32], lo[32][32];
};
constexpr BinomTable make_binom_table() {
    BinomTable t{};
    long long c[32][32] = {};
    for (int j = 0; j < 32; j++) {
        c[j][0] = 1;
        for (int k = 1; k <= j; k++) c[j][k] = c[j - 1][k - 1] + (k <= j - 1 ? c[j - 1][k] : 0);
    }
    for (int j = 0; j < 32; j++)
        for (int k = 0; k < 32; k++) {
            const float h = (float)c[j][k];
            t.hi[j][k] = h;
            t.lo[j][k] = (float)(c[j][k] - (long long)h);
        }
    return t;
}
__constant__ BinomTable kBinom = make_binom_table();

__device__ __forceinline__ int fmm_cell(float v, float v0, float inv_b) {
    const float t = floorf(__fmul_rn(__fsub_rn(v, v0), inv_b));
    return (int)fminf(fmaxf(t, -1.0e6f), 1.0e6f);
}

// Sub-cell coordinate (0 .. FMM_SUB - 1) of v inside its cell c (the same arithmetic wherever
// a traced point is placed, so that its sub-cell is one that was marked occupied).
__device__ __forceinline__ int fmm_subcell(float v, float v0, float inv_b, int c) {
    const float u = __fmul_rn(__fsub_rn(v, v0), inv_b) - i2f_small(c);
    return min(max(floor_small(u * (float)FMM_SUB), 0), FMM_SUB - 1);
}

__global__ void fmm_extent_kernel(const float2* z, int64_t npts, float4* part) {
    float mnx = 3.0e38f, mny = 3.0e38f, mxx = -3.0e38f, mxy = -3.0e38f;
    bool bad = false;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npts; p += (int64_t)gridDim.x * blockDim.x) {
        const float2 v = z[p];
        if (!(isfinite(v.x) && isfinite(v.y))) {
            bad = true;
            continue;
        }
        mnx = fminf(mnx, v.x);
        mny = fminf(mny, v.y);
        mxx = fmaxf(mxx, v.x);
        mxy = fmaxf(mxy, v.y);
    }
    for (int off = 16; off > 0; off >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, off));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, off));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, off));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, off));
    }
    __shared__ float4 sh[32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    __syncthreads();
    if (bad) sbad = 1;
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = make_float4(mnx, mny, mxx, mxy);
    __syncthreads();
    if (threadIdx.x == 0) {
        float4 r = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
            r.x = fminf(r.x, sh[w].x);
            r.y = fminf(r.y, sh[w].y);
            r.z = fmaxf(r.z, sh[w].z);
            r.w = fmaxf(r.w, sh[w].w);
        }
        if (sbad) r.x = __int_as_float(0x7fc00000);  // NaN marks a block that saw a bad point
        part[blockIdx.x] = r;
    }
}

__global__ void fmm_setup_kernel(const float4* part, int nparts, float b_target, int cap, int pool_cap,
                                 FmmParams* P) {
    if (blockIdx.x != 0) return;
    // one warp: each lane reduces a share of the partial extents, then a butterfly
    const int lane = threadIdx.x & 31;
    if (threadIdx.x >= 32) return;
    float mnx = 3.0e38f, mny = 3.0e38f, mxx = -3.0e38f, mxy = -3.0e38f;
    bool ok = true;
    for (int i = lane; i < nparts; i += 32) {
        const float4 r = part[i];
        if (r.x != r.x) {
            ok = false;
            continue;
        }
        mnx = fminf(mnx, r.x);
        mny = fminf(mny, r.y);
        mxx = fmaxf(mxx, r.z);
        mxy = fmaxf(mxy, r.w);
    }
    for (int off = 16; off > 0; off >>= 1) {
        mnx = fminf(mnx, __shfl_xor_sync(0xffffffffu, mnx, off));
        mny = fminf(mny, __shfl_xor_sync(0xffffffffu, mny, off));
        mxx = fmaxf(mxx, __shfl_xor_sync(0xffffffffu, mxx, off));
        mxy = fmaxf(mxy, __shfl_xor_sync(0xffffffffu, mxy, off));
    }
    ok = __all_sync(0xffffffffu, ok);
    if (lane != 0) return;
    float b = b_target > 0.f ? b_target : 1.0f;
    const float span = fmaxf(mxx - mnx, mxy - mny);
    const int margin = 2 * (FMM_K + 1) + 2;
    if (span / b + margin > (float)FMM_G) b = span / (float)(FMM_G - margin - 1);
    if (!(b > 0.f) || !isfinite(b) || !(span >= 0.f)) {
        b = 1.0f;
        ok = false;
        mnx = mny = mxx = mxy = 0.f;
    }
    const float inv_b = __fdiv_rn(1.0f, b);
    const float x0 = mnx - (FMM_K + 1) * b, y0 = mny - (FMM_K + 1) * b;
    const int nbx = fmm_cell(mxx, x0, inv_b) + FMM_K + 2;
    const int nby = fmm_cell(mxy, y0, inv_b) + FMM_K + 2;
    if (nbx > FMM_G || nby > FMM_G || nbx < 1 || nby < 1) ok = false;
    P->x0 = x0;
    P->y0 = y0;
    P->b = b;
    P->inv_b = inv_b;
    P->nbx = min(max(nbx, 1), FMM_G);
    P->nby = min(max(nby, 1), FMM_G);
    P->ok = ok ? 1 : 0;
    P->nocc = 0;
    P->ncocc = 0;
    P->pool_used = 0;
    P->cpool_used = 0;
    P->cap = cap;
    P->pool_cap = pool_cap;
    P->sub_used = 0;
}

// Occupied cells and sub-cells (a bit mask per cell).
__global__ void fmm_occupy_kernel(const float2* z, int64_t rows, int64_t nr, FmmParams* P, unsigned* occ) {
    // one thread per (column, run of FMM_OCC_ROWS rows): neighbouring threads read neighbouring
    // columns of a row (coalesced); a chain stays in one cell for many rows, so each thread ORs
    // its sub-cell bits per cell it enters rather than per point
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t col = t % nr, r0 = (t / nr) * FMM_OCC_ROWS;
    if (r0 >= rows || !P->ok) return;
    const int64_t r1 = r0 + FMM_OCC_ROWS < rows ? r0 + FMM_OCC_ROWS : rows;
    int cur = -1;  // < FMM_G^2 = 2^22
    unsigned bits = 0;
    for (int64_t rb = r0; rb < r1; rb += 4) {
        float2 v[4];
#pragma unroll
        for (int u = 0; u < 4; u++)
            if (rb + u < r1) v[u] = z[(rb + u) * nr + col];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (rb + u >= r1) break;
            const int cx = fmm_cell(v[u].x, P->x0, P->inv_b), cy = fmm_cell(v[u].y, P->y0, P->inv_b);
            if (!(cx >= 0 && cx < P->nbx && cy >= 0 && cy < P->nby)) {
                P->ok = 0;
                continue;
            }
            const int cell = cy * P->nbx + cx;
            if (cell != cur) {
                if (cur >= 0 && (occ[cur] & bits) != bits) atomicOr(occ + cur, bits);
                cur = cell;
                bits = 0;
            }
            // occ[cell]: bit s set when sub-cell s holds a traced point
            bits |= 1u << (fmm_subcell(v[u].y, P->y0, P->inv_b, cy) * FMM_SUB + fmm_subcell(v[u].x, P->x0, P->inv_b, cx));
        }
    }
    if (cur >= 0 && (occ[cur] & bits) != bits) atomicOr(occ + cur, bits);
}

__global__ void fmm_slot_kernel(FmmParams* P, const unsigned* occ, int* slot, int2* boxlist) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t ncell = (int64_t)P->nbx * P->nby;
    if (cell >= ncell) return;
    int v = -1;
    if (occ[cell]) {
        const int idx = atomicAdd(&P->nocc, 1);
        if (idx < P->cap) {
            v = idx;
            boxlist[idx] = make_int2((int)(cell % P->nbx), (int)(cell / P->nbx));
        } else {
            P->ok = 0;
        }
    }
    slot[cell] = v;
}

// Local expansions of the occupied cells, two levels (each cell's expansion is the same
// sum as with one level; only the work is organised differently):
//   coarse cells of FMM_F x FMM_F cells; for a coarse cell X with centre C,
//     Lc_k = -sum m_i / (z_i - C)^(k+1) over the stars outside X's 5x5 block of coarse cells
//     (|z_i - C| >= 2.5 FMM_F b), and the stars inside that block are listed in star order;
//   for each occupied cell B inside X, with centre c,
//     L_k(B) = [Lc re-centred at c]_k + -sum m_i / (z_i - c)^(k+1) over the listed stars
//     outside B's 5x5 block; the listed stars inside it form B's near list.
// Re-centring a polynomial is exact (a Taylor shift, O(P^2)), so the far sum's truncation
// error is that of Lc at the points (ratio <= (|c - C| + 0.72 b) / (2.5 FMM_F b) <= 0.28)
// plus that of the direct part (ratio <= 0.72 b / 2.5 b); both enter the bound.  Work per
// coarse cell: one pass over the N stars; per cell: the stars of the coarse block (about
// 25 FMM_F^2 times the stars per cell) instead of all N.
constexpr int FMM_WARPS = 4;
constexpr int FMM_CT = FMM_WARPS * 32;
constexpr int FMM_ACC = FMM_WARPS * FMM_P * 32;  // floats per accumulator component
constexpr int FMM_F = 8;
constexpr int FMM_CLIST = 8192;                  // stars of one coarse 5x5 block (more: direct polish)
constexpr int FMM_COARSE_MAX = (FMM_G / FMM_F) * (FMM_G / FMM_F);
constexpr int FMM_CPOOL = 1 << 23;               // coarse star-list entries (more: direct polish)

__global__ void fmm_coarse_list_kernel(FmmParams* P, const unsigned* occ, int2* clist) {
    const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (!P->ok) return;
    const int nbx = P->nbx, nby = P->nby;
    const int ncx = (nbx + FMM_F - 1) / FMM_F, ncy = (nby + FMM_F - 1) / FMM_F;
    if (c >= (int64_t)ncx * ncy) return;
    const int X = (int)(c % ncx), Y = (int)(c / ncx);
    bool any = false;
    for (int fy = Y * FMM_F; fy < min(nby, (Y + 1) * FMM_F) && !any; fy++)
        for (int fx = X * FMM_F; fx < min(nbx, (X + 1) * FMM_F); fx++) any |= occ[(int64_t)fy * nbx + fx] != 0;
    if (any) {
        const int i = atomicAdd(&P->ncocc, 1);
        if (i < FMM_COARSE_MAX) clist[i] = make_int2(X, Y);
    }
}

// One star's contribution -m (z_i - c)^-(k+1), k < FMM_P, to this lane's accumulators, and
// to the bound's sums.
__device__ __forceinline__ void fmm_acc_star(float* acc, int warp, int lane, const float4 pd, const float2 md,
                                             const df& cx, const df& cy, float& r2, float& dmin) {
    const df dx = df_sub(df{pd.x, pd.y}, cx), dy = df_sub(df{pd.z, pd.w}, cy);
    const df inv = df_rcp(df_add(df_sqr(dx), df_sqr(dy)));
    const df ux = df_mul(dx, inv), uy = df_neg(df_mul(dy, inv));  // u = 1/(z_i - c)
    df wx = df_mul(df{md.x, md.y}, ux), wy = df_mul(df{md.x, md.y}, uy);
    const float dd = sqrtf(dx.hi * dx.hi + dy.hi * dy.hi);
    r2 += md.x / (dd * dd);
    dmin = fminf(dmin, dd);
    for (int k = 0; k < FMM_P; k++) {
        const int a = ((warp * FMM_P + k) << 5) + lane;
        df ax = df{acc[a], acc[a + FMM_ACC]}, ay = df{acc[a + 2 * FMM_ACC], acc[a + 3 * FMM_ACC]};
        ax = df_sub(ax, wx);
        ay = df_sub(ay, wy);
        acc[a] = ax.hi;
        acc[a + FMM_ACC] = ax.lo;
        acc[a + 2 * FMM_ACC] = ay.hi;
        acc[a + 3 * FMM_ACC] = ay.lo;
        const df nx = df_dot2(wx, ux, df_neg(wy), uy);  // w <- w u
        const df ny = df_dot2(wx, uy, wy, ux);
        wx = nx;
        wy = ny;
    }
}

// Sum of each coefficient over the warps and lanes, in a fixed order: warp w takes the
// coefficients k = w, w + FMM_WARPS, ...; each lane adds the warps' partials at its lane, then
// a butterfly adds the lanes. Lane 0 writes out[k] = (x.hi, x.lo, y.hi, y.lo).
__device__ __forceinline__ void fmm_acc_reduce(const float* acc, int warp, int lane, float4* out) {
    for (int k = warp; k < FMM_P; k += FMM_WARPS) {
        df sx = df{0.f, 0.f}, sy = df{0.f, 0.f};
        for (int w = 0; w < FMM_WARPS; w++) {
            const int a = ((w * FMM_P + k) << 5) + lane;
            sx = df_add(sx, df{acc[a], acc[a + FMM_ACC]});
            sy = df_add(sy, df{acc[a + 2 * FMM_ACC], acc[a + 3 * FMM_ACC]});
        }
        for (int off = 16; off > 0; off >>= 1) {
            sx = df_add(sx, df{__shfl_xor_sync(0xffffffffu, sx.hi, off), __shfl_xor_sync(0xffffffffu, sx.lo, off)});
            sy = df_add(sy, df{__shfl_xor_sync(0xffffffffu, sy.hi, off), __shfl_xor_sync(0xffffffffu, sy.lo, off)});
        }
        if (lane == 0) out[k] = make_float4(sx.hi, sx.lo, sy.hi, sy.lo);
    }
}

// Sum of the per-thread bound terms: r2 added, dmin minimised (warp 0, all lanes get it).
__device__ __forceinline__ void fmm_bound_reduce(const float* s_r2, const float* s_dmin, int lane, float& R2,
                                                 float& D) {
    R2 = 0.f;
    D = 3.0e38f;
    for (int t = lane; t < FMM_CT; t += 32) {
        R2 += s_r2[t];
        D = fminf(D, s_dmin[t]);
    }
    for (int off = 16; off > 0; off >>= 1) {
        R2 += __shfl_xor_sync(0xffffffffu, R2, off);
        D = fminf(D, __shfl_xor_sync(0xffffffffu, D, off));
    }
}

__device__ __forceinline__ float fmm_tail(float r2, float rho) {
    // tail of -S1_far' after FMM_P terms: sum m/|d|^2 * P rho^(P-1) / (1 - rho)^2
    if (!(r2 > 0.f)) return 0.f;
    rho = fminf(rho, 0.99f);
    return r2 * (float)FMM_P * powf(rho, (float)(FMM_P - 1)) / ((1.f - rho) * (1.f - rho));
}

// Pass 1: one CTA per occupied coarse cell X: the coarse expansion Lc of the stars outside
// X's 5x5 coarse block, the bound's sums for them, and the block's stars in star order
// (written to cpool; their count and offset to cinfo).
struct CoarseInfo {
    int off, cnt;     // star list in cpool
    float r2, dmin;   // sum m/|z_i - C|^2 and min |z_i - C| over the stars outside the block
};

// Rounding of the FP32 Horner steps (terms k >= FMM_K0) in S2: their sum of magnitudes is
// at most sum m/|d|^2 * K0 rho^(K0-1) / (1 - rho)^2; complex Horner in FP32 over
// FMM_P - FMM_K0 steps errs by at most 4 (FMM_P - FMM_K0) 2^-24 of it.
__device__ __forceinline__ float fmm_fp32_part(float r2, float rho) {
    if (!(r2 > 0.f)) return 0.f;
    rho = fminf(rho, 0.99f);
    const float mag = r2 * (float)FMM_K0 * powf(rho, (float)(FMM_K0 - 1)) / ((1.f - rho) * (1.f - rho));
    return mag * (4.0f * (float)(FMM_P - FMM_K0) * 5.97e-8f);
}

__global__ void __launch_bounds__(FMM_CT) fmm_coarse_kernel(FmmParams* P, const int2* clist, int* cslot,
                                                            const float4* dfp, const float2* dfm, const float4* s32,
                                                            int n, float4* cLc, CoarseInfo* cinfo, int* cpool,
                                                            int cpool_cap) {
    extern __shared__ __align__(16) float acc[];  // [4 components][warp][k][lane], then the star list
    int* s_list = (int*)(acc + 4 * FMM_ACC);
    __shared__ int s_wcnt[FMM_WARPS];
    __shared__ int s_lcnt, s_off;
    __shared__ float s_r2[FMM_CT], s_dmin[FMM_CT];
    __shared__ int s_ok, s_ncocc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_ok = P->ok;
        s_ncocc = min(P->ncocc, FMM_COARSE_MAX);
    }
    __syncthreads();
    if (!s_ok) return;  // block-uniform
    const int ncx = (P->nbx + FMM_F - 1) / FMM_F;
    const double b = (double)P->b;
    for (int ci = blockIdx.x; ci < s_ncocc; ci += gridDim.x) {
        const int2 X = clist[ci];
        const double Cxd = (double)P->x0 + ((double)(X.x * FMM_F) + 0.5 * FMM_F) * b;
        const double Cyd = (double)P->y0 + ((double)(X.y * FMM_F) + 0.5 * FMM_F) * b;
        const df Cx = df_from_double(Cxd), Cy = df_from_double(Cyd);
        for (int q = tid; q < 4 * FMM_ACC; q += FMM_CT) acc[q] = 0.f;
        if (tid == 0) s_lcnt = 0;
        float r2 = 0.f, dmin = 3.0e38f;
        __syncthreads();
        for (int j0 = 0; j0 < n; j0 += FMM_CT) {
            const int j = j0 + tid;
            bool nearc = false;
            if (j < n) {
                const float4 sp = s32[j];
                const int sx = fmm_cell(sp.x, P->x0, P->inv_b) >> 3, sy = fmm_cell(sp.y, P->y0, P->inv_b) >> 3;
                nearc = abs(sx - X.x) <= 2 && abs(sy - X.y) <= 2;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, nearc);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < FMM_WARPS; w++) {
                if (w < warp) before += s_wcnt[w];
                total += s_wcnt[w];
            }
            const int pos = s_lcnt + before + __popc(bal & ((1u << lane) - 1u));
            if (nearc && pos < FMM_CLIST) s_list[pos] = j;
            __syncthreads();
            if (tid == 0) s_lcnt += total;
            if (j < n && !nearc) fmm_acc_star(acc, warp, lane, dfp[j], dfm[j], Cx, Cy, r2, dmin);
        }
        s_r2[tid] = r2;
        s_dmin[tid] = dmin;
        __syncthreads();
        const int lcnt = s_lcnt;
        if (warp == 0) {
            float R2, D;
            fmm_bound_reduce(s_r2, s_dmin, lane, R2, D);
            if (lane == 0) {
                const int off = lcnt <= FMM_CLIST ? atomicAdd(&P->cpool_used, lcnt) : 0;
                if (lcnt > FMM_CLIST || off + lcnt > cpool_cap) P->ok = 0;  // the direct polish takes over
                s_off = off;
                CoarseInfo c;
                c.off = off;
                c.cnt = lcnt;
                c.r2 = R2;
                c.dmin = D;
                cinfo[ci] = c;
                cslot[X.y * ncx + X.x] = ci;
            }
        }
        fmm_acc_reduce(acc, warp, lane, cLc + (size_t)ci * FMM_P);
        __syncthreads();
        if (lcnt <= FMM_CLIST && s_off + lcnt <= cpool_cap)
            for (int i = tid; i < lcnt; i += FMM_CT) cpool[s_off + i] = s_list[i];
        __syncthreads();
    }
}

// Pass 2: one CTA per occupied cell B (parent coarse cell X): near list, direct part of the
// listed stars outside B's block, Lc re-centred at B's centre, bound.
__global__ void __launch_bounds__(FMM_CT) fmm_coeff_kernel(FmmParams* P, const int2* boxlist, const int* cslot,
                                                           const float4* cLc, const CoarseInfo* cinfo,
                                                           const int* cpool, const float4* dfp, const float2* dfm,
                                                           const float4* s32, BoxInfo* info, float4* coeff,
                                                           int* pool) {
    extern __shared__ __align__(16) float acc[];  // [4 components][warp][k][lane]
    __shared__ float2 s_binom[32][32];            // C(j, k) as double-float
    __shared__ float4 s_Ld[FMM_P];                // direct part of each coefficient
    __shared__ int s_wcnt[FMM_WARPS];
    __shared__ int s_off, s_cnt;
    __shared__ float s_r2[FMM_CT], s_dmin[FMM_CT];
    __shared__ int s_ok, s_nocc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) {
        s_ok = P->ok;
        s_nocc = min(P->nocc, P->cap);
    }
    __syncthreads();
    if (!s_ok) return;  // block-uniform
    for (int q = tid; q < 32 * 32; q += FMM_CT) s_binom[q >> 5][q & 31] = make_float2(kBinom.hi[q >> 5][q & 31],
                                                                                   kBinom.lo[q >> 5][q & 31]);
    const int ncx = (P->nbx + FMM_F - 1) / FMM_F;
    const double b = (double)P->b;
    for (int box = blockIdx.x; box < s_nocc; box += gridDim.x) {
        const int2 bc = boxlist[box];
        const int fx = bc.x, fy = bc.y;
        const int ci = cslot[(fy / FMM_F) * ncx + fx / FMM_F];
        const CoarseInfo cI = cinfo[ci];
        const int* list = cpool + cI.off;
        const int lcnt = cI.cnt;
        const double Cxd = (double)P->x0 + ((double)((fx / FMM_F) * FMM_F) + 0.5 * FMM_F) * b;
        const double Cyd = (double)P->y0 + ((double)((fy / FMM_F) * FMM_F) + 0.5 * FMM_F) * b;
        const double cxd = (double)P->x0 + ((double)fx + 0.5) * b;
        const double cyd = (double)P->y0 + ((double)fy + 0.5) * b;
        const df cx = df_from_double(cxd), cy = df_from_double(cyd);
        // near list: count, reserve, ordered write
        int cnt = 0;
        for (int i = tid; i < lcnt; i += FMM_CT) {
            const float4 sp = s32[list[i]];
            const int sx = fmm_cell(sp.x, P->x0, P->inv_b), sy = fmm_cell(sp.y, P->y0, P->inv_b);
            cnt += (abs(sx - fx) <= FMM_K && abs(sy - fy) <= FMM_K);
        }
        for (int off = 16; off > 0; off >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, off);
        if (lane == 0) s_wcnt[warp] = cnt;
        __syncthreads();
        if (tid == 0) {
            int tot = 0;
            for (int w = 0; w < FMM_WARPS; w++) tot += s_wcnt[w];
            const int off = atomicAdd(&P->pool_used, tot);
            if (off + tot > P->pool_cap) P->ok = 0;
            s_off = off;
            s_cnt = tot;
        }
        for (int q = tid; q < 4 * FMM_ACC; q += FMM_CT) acc[q] = 0.f;
        __syncthreads();
        const bool room = s_off + s_cnt <= P->pool_cap;
        int base = 0;
        float r2i = 0.f, dmi = 3.0e38f;
        for (int i0 = 0; i0 < lcnt; i0 += FMM_CT) {
            const int i = i0 + tid;
            bool nr_ = false;
            int j = 0;
            if (i < lcnt) {
                j = list[i];
                const float4 sp = s32[j];
                const int sx = fmm_cell(sp.x, P->x0, P->inv_b), sy = fmm_cell(sp.y, P->y0, P->inv_b);
                nr_ = abs(sx - fx) <= FMM_K && abs(sy - fy) <= FMM_K;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, nr_);
            if (lane == 0) s_wcnt[warp] = __popc(bal);
            __syncthreads();
            int before = 0, total = 0;
            for (int w = 0; w < FMM_WARPS; w++) {
                if (w < warp) before += s_wcnt[w];
                total += s_wcnt[w];
            }
            if (nr_ && room) pool[s_off + base + before + __popc(bal & ((1u << lane) - 1u))] = j;
            base += total;
            __syncthreads();
            if (i < lcnt && !nr_) fmm_acc_star(acc, warp, lane, dfp[j], dfm[j], cx, cy, r2i, dmi);
        }
        s_r2[tid] = r2i;
        s_dmin[tid] = dmi;
        __syncthreads();
        fmm_acc_reduce(acc, warp, lane, s_Ld);  // direct part
        __syncthreads();
        if (tid < FMM_P) {
            // Lc re-centred at c (Taylor shift by t0 = c - C: Horner in t0 with binomial
            // weights C(k, jk)), plus the direct part
            const int jk = tid;
            const float4* Lc = cLc + (size_t)ci * FMM_P;
            const df tx = df_from_double(cxd - Cxd), ty = df_from_double(cyd - Cyd);
            const float4 top = Lc[FMM_P - 1];
            const df b0 = df{s_binom[FMM_P - 1][jk].x, s_binom[FMM_P - 1][jk].y};
            dfc sacc = dfc{df_mul(b0, df{top.x, top.y}), df_mul(b0, df{top.z, top.w})};
            for (int k = FMM_P - 2; k >= jk; k--) {
                const df bk = df{s_binom[k][jk].x, s_binom[k][jk].y};
                const float4 lk = Lc[k];
                sacc = dfc_mul(sacc, dfc{tx, ty});
                sacc.x = df_add(sacc.x, df_mul(bk, df{lk.x, lk.y}));
                sacc.y = df_add(sacc.y, df_mul(bk, df{lk.z, lk.w}));
            }
            const float4 ld = s_Ld[jk];
            const df lx = df_add(sacc.x, df{ld.x, ld.y}), ly = df_add(sacc.y, df{ld.z, ld.w});
            coeff[(size_t)box * FMM_P + jk] = make_float4(lx.hi, lx.lo, ly.hi, ly.lo);
        }
        if (warp == 0) {
            float R2, D;
            fmm_bound_reduce(s_r2, s_dmin, lane, R2, D);
            if (lane == 0) {
                BoxInfo bi;
                bi.c = make_float4(cx.hi, cx.lo, cy.hi, cy.lo);
                bi.near_off = s_off;
                bi.near_cnt = room ? s_cnt : 0;
                // points lie within 0.72 b of c (half-diagonal plus the Newton steps)
                const float tc = (float)sqrt((cxd - Cxd) * (cxd - Cxd) + (cyd - Cyd) * (cyd - Cyd));
                const float rho1 = 0.72f * P->b / D, rho2 = (tc + 0.72f * P->b) / cI.dmin;
                bi.s2_trunc = fmm_tail(R2, rho1) + fmm_tail(cI.r2, rho2);
                bi.s2_err = bi.s2_trunc + fmm_fp32_part(R2, rho1) + fmm_fp32_part(cI.r2, rho2);
                info[box] = bi;
            }
        }
        __syncthreads();
    }
}

// Pass 3: one CTA per occupied cell B: B's 32-term polynomial
// re-centred at the centre c + d of each sub-cell holding a traced point, exactly as an
// algebraic identity, L'_k = sum_{j >= k} C(j, k) L_j d^(j - k) (Horner in d): in
// double-float for the kept terms k < FMM_PS (one thread per (sub-cell, k)), and for the
// dropped ones an FP32 upper bound on |L'_k| by the same sum of magnitudes (rounding covered
// by a 1.001 factor); then each sub-cell's bounds.
constexpr int FMM_ST = FMM_SUB2 * FMM_PS;  // threads of the sub-cell kernel
__global__ void __launch_bounds__(FMM_ST) fmm_subcell_kernel(FmmParams* P, const int2* boxlist,
                                                             const unsigned* occ, const BoxInfo* info,
                                                             const float4* coeff, int* sub_base, float4* scoeff,
                                                             SubInfo* sinfo, int sub_cap) {
    __shared__ float4 s_L[FMM_P];
    __shared__ int s_base;
    __shared__ float2 s_binom[32][32];
    __shared__ float4 s_Ls[FMM_SUB2 * FMM_PS];  // kept terms
    __shared__ float s_tail[FMM_SUB2 * (FMM_P - FMM_PS)];  // bounds on the dropped terms' |L'_k|
    const int tid = threadIdx.x;
    if (!P->ok) return;  // grid-uniform
    const int nocc = min(P->nocc, P->cap);
    for (int q = tid; q < 32 * 32; q += FMM_ST) s_binom[q >> 5][q & 31] = make_float2(kBinom.hi[q >> 5][q & 31],
                                                                                   kBinom.lo[q >> 5][q & 31]);
    const float b = P->b;
    for (int box = blockIdx.x; box < nocc; box += gridDim.x) {
        __syncthreads();
        if (tid < FMM_P) s_L[tid] = coeff[(size_t)box * FMM_P + tid];
        const int2 bc = boxlist[box];
        const unsigned mask = occ[(int64_t)bc.y * P->nbx + bc.x];
        const int nsub = __popc(mask);
        if (tid == 0) {
            // table entries of this cell's occupied sub-cells, in sub-cell order (-1: pool full,
            // its points use the cell's own expansion)
            const int base = atomicAdd(&P->sub_used, nsub);
            s_base = base + nsub <= sub_cap ? base : -1;
            sub_base[box] = s_base;
        }
        __syncthreads();
        const int base = s_base;
        const int r = tid / FMM_PS, k = tid - r * FMM_PS;  // r-th occupied sub-cell, term k (and FMM_PS + k)
        if (base >= 0 && r < nsub) {
            unsigned mm = mask;
            for (int q = 0; q < r; q++) mm &= mm - 1u;
            const int sb = __ffs(mm) - 1;
            const float ox = ((float)(sb % FMM_SUB) + 0.5f) * (1.0f / FMM_SUB) - 0.5f;
            const float oy = ((float)(sb / FMM_SUB) + 0.5f) * (1.0f / FMM_SUB) - 0.5f;
            const dfc d = dfc{two_prod(b, ox), two_prod(b, oy)};
            const float4 top = s_L[FMM_P - 1];
            const df c0 = df{s_binom[FMM_P - 1][k].x, s_binom[FMM_P - 1][k].y};
            dfc a = dfc{df_mul(c0, df{top.x, top.y}), df_mul(c0, df{top.z, top.w})};
            for (int j = FMM_P - 2; j >= k; j--) {
                const float4 lj = s_L[j];
                const df cj = df{s_binom[j][k].x, s_binom[j][k].y};
                a = dfc_mul(a, d);
                a.x = df_add(a.x, df_mul(cj, df{lj.x, lj.y}));
                a.y = df_add(a.y, df_mul(cj, df{lj.z, lj.w}));
            }
            s_Ls[sb * FMM_PS + k] = make_float4(a.x.hi, a.x.lo, a.y.hi, a.y.lo);
            scoeff[((size_t)base + r) * FMM_PS + k] = make_float4(a.x.hi, a.x.lo, a.y.hi, a.y.lo);
            const int kt = FMM_PS + k;  // a dropped term
            if (kt < FMM_P) {
                const float ad = b * sqrtf(fmaf(ox, ox, oy * oy));
                auto mag = [&](int j) {
                    const float4 v = s_L[j];
                    return sqrtf(fmaf(v.x, v.x, v.z * v.z)) * 1.0001f + fabsf(v.y) + fabsf(v.w);
                };
                float m = s_binom[FMM_P - 1][kt].x * mag(FMM_P - 1);
                for (int j = FMM_P - 2; j >= kt; j--) m = fmaf(m, ad, s_binom[j][kt].x * mag(j));
                s_tail[sb * (FMM_P - FMM_PS) + k] = 1.001f * m;
            }
        }
        __syncthreads();
        if (base >= 0 && tid < FMM_SUB2 && ((mask >> tid) & 1u)) {
            // bounds for |z - c_s| <= rp: the dropped terms k >= FMM_PS in S2 = -D1 and S3 = D2/2,
            // and the FP32 rounding of the terms FMM_KS0 <= k < FMM_PS (4 (PS - KS0) 2^-24 of
            // their share of S2), on top of the cell's own truncation bound
            const float rp = FMM_SUBR * b;
            float t2 = 0.f, t3 = 0.f, mg = 0.f, pw = 1.f;  // pw = rp^(k-1)
            for (int kk = 1; kk < FMM_P; kk++) {
                if (kk >= FMM_PS) {
                    const float a = s_tail[tid * (FMM_P - FMM_PS) + kk - FMM_PS];
                    t2 = fmaf((float)kk * a, pw, t2);
                    t3 = fmaf(0.5f * (float)(kk * (kk - 1)) * a, pw / rp, t3);
                } else if (kk >= FMM_KS0) {
                    const float4 v = s_Ls[tid * FMM_PS + kk];
                    const float a = sqrtf(fmaf(v.x, v.x, v.z * v.z)) * 1.0001f + fabsf(v.y) + fabsf(v.w);
                    mg = fmaf((float)kk * a, pw, mg);
                }
                pw *= rp;
            }
            const BoxInfo bi = info[box];
            const float ox = ((float)(tid % FMM_SUB) + 0.5f) * (1.0f / FMM_SUB) - 0.5f;
            const float oy = ((float)(tid / FMM_SUB) + 0.5f) * (1.0f / FMM_SUB) - 0.5f;
            const df csx = df_add(df{bi.c.x, bi.c.y}, two_prod(b, ox)), csy = df_add(df{bi.c.z, bi.c.w}, two_prod(b, oy));
            SubInfo si;
            si.c = make_float4(csx.hi, csx.lo, csy.hi, csy.lo);
            si.s2_err = 1.01f * (bi.s2_trunc + t2 + mg * (4.0f * (float)(FMM_PS - FMM_KS0) * 5.97e-8f));
            si.s3_err = 1.01f * t3;
            si.r2 = 0.999f * rp * rp;
            si.pad = 0.f;
            sinfo[(size_t)base + __popc(mask & ((1u << tid) - 1u))] = si;
        }
    }
}

// Points: warp = one chain (global column g), 32 consecutive rows, so that a warp's
// points sit in one or two neighbouring cells.
// a1 b1 + a2 b2 + c in double-float with one normalisation: the two high products and the
// two sums are formed exactly (two_prod, two_sum), and their error terms, c's low part and
// the four cross products of the low parts are gathered by FP32 adds and FMAs.  26 FP32
// operations against 32 for two df_mul, a df_add and a df_sub, with the same ~2^-46
// relative rounding (the final fast two-sum assumes, as df_add does, that the sum does not
// cancel below its accumulated error).
__device__ __forceinline__ df df_dot2_add(df a1, df b1, df a2, df b2, df c) {
    const df p1 = two_prod(a1.hi, b1.hi), p2 = two_prod(a2.hi, b2.hi);
    const df s1 = two_sum(p1.hi, p2.hi);
    const df s2 = two_sum(s1.hi, c.hi);
    float e = __fadd_rn(__fadd_rn(p1.lo, p2.lo), __fadd_rn(s1.lo, s2.lo));
    e = __fadd_rn(e, c.lo);
    e = __fmaf_rn(a1.hi, b1.lo, e);
    e = __fmaf_rn(a1.lo, b1.hi, e);
    e = __fmaf_rn(a2.hi, b2.lo, e);
    e = __fmaf_rn(a2.lo, b2.hi, e);
    return fast_two_sum(s2.hi, e);
}

// Far-field sums from a local expansion L_0..L_{PN-1} about a centre, at t = z - centre:
// Horner with the first three derivatives, steps PN-2 .. K0N in FP32 (their terms carry so
// little of S1, S2 that their FP32 rounding is negligible and is charged to the bound) and
// the rest in double-float.  S1 += b0, S2 -= b1, S3 += b2, S4 -= b3.
template <int PN, int K0N>
__device__ __forceinline__ void far_horner(const float4* L, const df& tx, const df& ty, Sums& sm) {
    const float tfx = tx.hi, tfy = ty.hi;
    const float4 top = L[PN - 1];
    float h0x = top.x, h0y = top.z, h1x = 0.f, h1y = 0.f;
    float b2x = 0.f, b2y = 0.f, b3x = 0.f, b3y = 0.f;
#pragma unroll
    for (int kk = PN - 2; kk >= K0N; kk--) {
        const float n3x = fmaf(b3x, tfx, fmaf(-b3y, tfy, b2x)), n3y = fmaf(b3x, tfy, fmaf(b3y, tfx, b2y));
        const float n2x = fmaf(b2x, tfx, fmaf(-b2y, tfy, h1x)), n2y = fmaf(b2x, tfy, fmaf(b2y, tfx, h1y));
        const float n1x = fmaf(h1x, tfx, fmaf(-h1y, tfy, h0x)), n1y = fmaf(h1x, tfy, fmaf(h1y, tfx, h0y));
        const float4 Lk = L[kk];
        const float n0x = fmaf(h0x, tfx, fmaf(-h0y, tfy, Lk.x)), n0y = fmaf(h0x, tfy, fmaf(h0y, tfx, Lk.z));
        b3x = n3x;
        b3y = n3y;
        b2x = n2x;
        b2y = n2y;
        h1x = n1x;
        h1y = n1y;
        h0x = n0x;
        h0y = n0y;
    }
    df b0x = df{h0x, 0.f}, b0y = df{h0y, 0.f};
    df b1x = df{h1x, 0.f}, b1y = df{h1y, 0.f};
#pragma unroll 4
    for (int kk = K0N - 1; kk >= 0; kk--) {
        // b3 <- b3 t + b2 ; b2 <- b2 t + b1 ; b1 <- b1 t + b0 ; b0 <- b0 t + L_k
        const float n3x = fmaf(b3x, tfx, fmaf(-b3y, tfy, b2x)), n3y = fmaf(b3x, tfy, fmaf(b3y, tfx, b2y));
        const float n2x = fmaf(b2x, tfx, fmaf(-b2y, tfy, b1x.hi)), n2y = fmaf(b2x, tfy, fmaf(b2y, tfx, b1y.hi));
        b3x = n3x;
        b3y = n3y;
        b2x = n2x;
        b2y = n2y;
        const df m1x = df_dot2_add(b1x, tx, df_neg(b1y), ty, b0x);
        const df m1y = df_dot2_add(b1x, ty, b1y, tx, b0y);
        const float4 Lk = L[kk];
        const df m0x = df_dot2_add(b0x, tx, df_neg(b0y), ty, df{Lk.x, Lk.y});
        const df m0y = df_dot2_add(b0x, ty, b0y, tx, df{Lk.z, Lk.w});
        b1x = m1x;
        b1y = m1y;
        b0x = m0x;
        b0y = m0y;
    }
    sm.S1x = df_add(sm.S1x, b0x);
    sm.S1y = df_add(sm.S1y, b0y);
    sm.S2x = df_sub(sm.S2x, b1x);
    sm.S2y = df_sub(sm.S2y, b1y);
    sm.s3x += b2x;
    sm.s3y += b2y;
    sm.s4x -= b3x;
    sm.s4y -= b3y;
    sm.a3 += 4.0f * (fabsf(b2x) + fabsf(b2y));
}

template <bool UNIT>
__global__ void __launch_bounds__(PB_THREADS, 3) fmm_polish_kernel(PolishK K, const FmmParams* Pm, const int* slot,
                                                                const BoxInfo* info, const float4* coeff,
                                                                const int* pool, const unsigned* occ,
                                                                const int* sub_base, const float4* scoeff,
                                                                const SubInfo* sinfo) {
    if (!Pm->ok) return;  // grid-uniform (set before this launch)
    const int lane = threadIdx.x & 31;
    const int64_t wg = blockIdx.x * (int64_t)(PB_THREADS / 32) + (threadIdx.x >> 5);
    int64_t g, rb;  // column and row block (32-bit division when it fits)
    if (wg < ((int64_t)1 << 32)) {
        const unsigned a = (unsigned)wg, b = (unsigned)K.nr;
        g = a % b;
        rb = a / b;
    } else {
        g = wg % K.nr;
        rb = wg / K.nr;
    }
    const int64_t row0 = rb * 32 + lane;
    const bool valid = wg < K.nr * ((K.m + 32) / 32) && row0 <= K.m;
    int passes = 0;
    float est_max = 0.f;  // certified estimates are FP32 values
    if (valid) {
    const int64_t row = row0;
    const int64_t point = row * K.nr + g;
    const int s = subchain_of_row_fast(row, K.m, K.S);
    const int32_t k = K.perm[(size_t)s * K.nr + g];
    const float2 z0 = K.zrows[(size_t)row * K.nr + k];
    const int32_t it_in = K.iters_out ? K.iters_in[(size_t)row * K.nr + k] : 0;
    const int cx = fmm_cell(z0.x, Pm->x0, Pm->inv_b), cy = fmm_cell(z0.y, Pm->y0, Pm->inv_b);
    const int sl = slot[(int64_t)cy * Pm->nbx + cx];
    const BoxInfo bi = info[sl];
    const float4* L = coeff + (size_t)sl * FMM_P;
    // the point's sub-cell, from its position inside the cell (the radius test in each pass
    // decides whether the sub-cell expansion applies)
    const int sbase = sub_base[sl];
    const bool have_sub = sbase >= 0;
    SubInfo si = {};
    const float4* SL = nullptr;
    if (have_sub) {
        const int sx = fmm_subcell(z0.x, Pm->x0, Pm->inv_b, cx), sy = fmm_subcell(z0.y, Pm->y0, Pm->inv_b, cy);
        const unsigned mask = occ[(int64_t)cy * Pm->nbx + cx];
        const size_t sidx = (size_t)sbase + __popc(mask & ((1u << (sy * FMM_SUB + sx)) - 1u));
        si = sinfo[sidx];
        SL = scoeff + sidx * FMM_PS;
    }
    tf zxt = tf{z0.x, 0.f, 0.f}, zyt = tf{z0.y, 0.f, 0.f};
    df cxr, cyr;
    row_constant(K, row, cxr, cyr);
    for (int pass = 0; pass < K.max_polish; pass++) {
        passes++;
        Sums sm;
        sm.S1x = sm.S1y = sm.S2x = sm.S2y = df{0.f, 0.f};
        sm.s3x = sm.s3y = sm.s4x = sm.s4y = sm.a3 = 0.f;
        for (int q = 0; q < bi.near_cnt; q++) {
            const int j = pool[bi.near_off + q];
            star_df<UNIT>(zxt, zyt, K.dfp[j], K.dtf[j], K.dfm[j], sm);
        }
        // far field: Horner with derivatives, about the sub-cell centre when the point is within
        // the sub-cell's radius (16 terms), else about the cell centre (32 terms)
        float s2e = bi.s2_err, s3e = 0.f;
        bool sub_done = false;
        if (have_sub) {
            const df ux = tf_sub(zxt, si.c.x, si.c.y, 0.f), uy = tf_sub(zyt, si.c.z, si.c.w, 0.f);
            if (fmaf(ux.hi, ux.hi, uy.hi * uy.hi) <= si.r2) {
                far_horner<FMM_PS, FMM_KS0>(SL, ux, uy, sm);
                s2e = si.s2_err;
                s3e = si.s3_err;
                sub_done = true;
            }
        }
        if (!sub_done) {
            const df tx = tf_sub(zxt, bi.c.x, bi.c.y, 0.f), ty = tf_sub(zyt, bi.c.z, bi.c.w, 0.f);
            far_horner<FMM_P, FMM_K0>(L, tx, ty, sm);
        }
        double est = 0.0;
        if (polish_epilogue_df(K, point, row, sm, cxr, cyr, zxt, zyt, z0.x, z0.y, pass, it_in, est, s2e, s3e)) {
            est_max = (float)est;
            break;
        }
    }
    }  // valid
    for (int off = 16; off > 0; off >>= 1) {
        passes += __shfl_xor_sync(0xffffffffu, passes, off);
        est_max = fmaxf(est_max, __shfl_xor_sync(0xffffffffu, est_max, off));
    }
    if (lane == 0) {
        if (passes) atomicAdd(&K.rep->polish_passes, (unsigned long long)passes);
        if (est_max > 0.f) atomic_max_double_nonneg(&K.rep->max_err_est, (double)est_max);
    }
}

size_t fmm_workspace_bytes(int64_t points) {
    const int64_t cap = points < (1 << 18) ? points : (1 << 18);
    const int64_t pool = cap * 64 < (1 << 24) ? cap * 64 : (1 << 24);
    size_t b = 0;
    auto add = [&](size_t x) { b += (x + 255) / 256 * 256; };
    add(sizeof(FmmParams));
    add(sizeof(float4) * 512);
    add(sizeof(unsigned) * (size_t)FMM_G * FMM_G);  // occupancy (sub-cell bits)
    add(sizeof(int) * (size_t)FMM_G * FMM_G);   // slots
    add(sizeof(int2) * cap);
    add(sizeof(BoxInfo) * cap);
    add(sizeof(float4) * FMM_P * cap);
    add(sizeof(int) * pool);
    add(sizeof(int2) * (size_t)FMM_COARSE_MAX);  // occupied coarse cells
    add(sizeof(int) * (size_t)FMM_COARSE_MAX);   // coarse slots
    add(sizeof(float4) * FMM_P * (size_t)FMM_COARSE_MAX);
    add(sizeof(CoarseInfo) * (size_t)FMM_COARSE_MAX);
    add(sizeof(int) * (size_t)FMM_CPOOL);
    const int64_t subs = 4 * cap < FMM_SUBPOOL ? 4 * cap : FMM_SUBPOOL;  // occupied sub-cells (a cell's
                                                                           // curves hold a few of its 16)
    add(sizeof(int) * cap);
    add(sizeof(float4) * FMM_PS * (size_t)subs);
    add(sizeof(SubInfo) * (size_t)subs);
    return b;
}

cudaError_t launch_polish_fmm(const PolishArgs& a, void* ws, cudaStream_t st) {
    const int64_t points = (a.m + 1) * a.nr;
    const int cap = (int)(points < (1 << 18) ? points : (1 << 18));
    const int pool_cap = (int)((int64_t)cap * 64 < (1 << 24) ? (int64_t)cap * 64 : (1 << 24));
    char* p = (char*)ws;
    auto take = [&](size_t x) {
        char* r = p;
        p += (x + 255) / 256 * 256;
        return r;
    };
    FmmParams* P = (FmmParams*)take(sizeof(FmmParams));
    float4* part = (float4*)take(sizeof(float4) * 512);
    unsigned* occ = (unsigned*)take(sizeof(unsigned) * (size_t)FMM_G * FMM_G);
    int* slot = (int*)take(sizeof(int) * (size_t)FMM_G * FMM_G);
    int2* boxlist = (int2*)take(sizeof(int2) * cap);
    BoxInfo* info = (BoxInfo*)take(sizeof(BoxInfo) * cap);
    float4* coeff = (float4*)take(sizeof(float4) * FMM_P * (size_t)cap);
    int* pool = (int*)take(sizeof(int) * (size_t)pool_cap);
    int2* clist = (int2*)take(sizeof(int2) * (size_t)FMM_COARSE_MAX);
    int* cslot = (int*)take(sizeof(int) * (size_t)FMM_COARSE_MAX);
    float4* cLc = (float4*)take(sizeof(float4) * FMM_P * (size_t)FMM_COARSE_MAX);
    CoarseInfo* cinfo = (CoarseInfo*)take(sizeof(CoarseInfo) * (size_t)FMM_COARSE_MAX);
    int* cpool = (int*)take(sizeof(int) * (size_t)FMM_CPOOL);
    const int subs = 4 * (int64_t)cap < FMM_SUBPOOL ? 4 * cap : FMM_SUBPOOL;
    int* sub_base = (int*)take(sizeof(int) * cap);
    float4* scoeff = (float4*)take(sizeof(float4) * FMM_PS * (size_t)subs);
    SubInfo* sinfo = (SubInfo*)take(sizeof(SubInfo) * (size_t)subs);
    cudaError_t e;
    // the points' extent: the tracer's per-CTA extents when it kept them, else one pass here
    if (a.ext && a.ext_n > 0) {
        fmm_setup_kernel<<<1, 32, 0, st>>>(a.ext, a.ext_n, a.f->fmm_cell, cap, pool_cap, P);
    } else {
        fmm_extent_kernel<<<512, 256, 0, st>>>(a.zrows, points, part);
        fmm_setup_kernel<<<1, 32, 0, st>>>(part, 512, a.f->fmm_cell, cap, pool_cap, P);
    }
    if ((e = cudaMemsetAsync(occ, 0, sizeof(unsigned) * (size_t)FMM_G * FMM_G, st)) != cudaSuccess) return e;
    {
        const int64_t threads = ((a.m + 1 + FMM_OCC_ROWS - 1) / FMM_OCC_ROWS) * a.nr;
        fmm_occupy_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(a.zrows, a.m + 1, a.nr, P, occ);
    }
    fmm_slot_kernel<<<(unsigned)(((int64_t)FMM_G * FMM_G + 255) / 256), 256, 0, st>>>(P, occ, slot, boxlist);
    fmm_coarse_list_kernel<<<(unsigned)((FMM_COARSE_MAX + 255) / 256), 256, 0, st>>>(P, occ, clist);
    const size_t csmem1 = sizeof(float) * 4 * FMM_ACC + sizeof(int) * FMM_CLIST;
    const size_t csmem2 = sizeof(float) * 4 * FMM_ACC;
    if ((e = cudaFuncSetAttribute(fmm_coarse_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem1)) !=
            cudaSuccess ||
        (e = cudaFuncSetAttribute(fmm_coeff_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem2)) !=
            cudaSuccess)
        return e;
    fmm_coarse_kernel<<<608, FMM_CT, csmem1, st>>>(P, clist, cslot, a.f->star_dfp, a.f->star_dfm, a.f->star32,
                                                   (int)a.f->n, cLc, cinfo, cpool, FMM_CPOOL);
    fmm_coeff_kernel<<<1216, FMM_CT, csmem2, st>>>(P, boxlist, cslot, cLc, cinfo, cpool, a.f->star_dfp, a.f->star_dfm,
                                                   a.f->star32, info, coeff, pool);
    fmm_subcell_kernel<<<1216, FMM_ST, 0, st>>>(P, boxlist, occ, info, coeff, sub_base, scoeff, sinfo, subs);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    PolishK K = make_polish_k(a);
    const int64_t warps = ((a.m + 1 + 31) / 32) * a.nr;
    const unsigned blocks = (unsigned)((warps + (PB_THREADS / 32) - 1) / (PB_THREADS / 32));
    if (a.f->unit_mass)
        fmm_polish_kernel<true><<<blocks, PB_THREADS, 0, st>>>(K, P, slot, info, coeff, pool, occ, sub_base, scoeff,
                                                              sinfo);
    else
        fmm_polish_kernel<false><<<blocks, PB_THREADS, 0, st>>>(K, P, slot, info, coeff, pool, occ, sub_base, scoeff,
                                                               sinfo);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // the direct polish runs (and does the whole job) only when the tables did not fit
    PolishArgs b = a;
    b.skip_if = &P->ok;
    return launch_polish(b, st);
}

// ----------------------------------------------------------------------------------
// FP64 form: permute the tracer's rows into chain order (no polish).
// ----------------------------------------------------------------------------------
__global__ void finalize_fp64_kernel(FinalizeArgs a) {
    const int64_t point = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (point >= (a.m + 1) * a.nr) return;
    const int64_t row = point / a.nr, g = point - row * a.nr;
    const int s = subchain_of_row(row, a.m, a.S);
    const int32_t k = a.perm[(size_t)s * a.nr + g];
    a.z_out[point] = a.zrows[(size_t)row * a.nr + k];
    if (a.iters_out) a.iters_out[point] = a.iters_in[(size_t)row * a.nr + k];
}

cudaError_t launch_finalize_fp64(const FinalizeArgs& a, cudaStream_t st) {
    const int64_t pts = (a.m + 1) * a.nr;
    finalize_fp64_kernel<<<(unsigned)((pts + 255) / 256), 256, 0, st>>>(a);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Standalone caustic mapping (Sec. 3.1 lens equation): w = (1-kappa_s) z + gamma conj(z)
// - conj(sum m_i/(z - z_i)), star sum in double-float or FP64.
// ----------------------------------------------------------------------------------
struct MapK {
    const SmoothPoly* poly;
    const float4* dfp;
    const float2* dfm;
    const float2* dtf;
    const StarD* s64;
    int n;
    int64_t count;
    double kappa_s, gamma;
    const double2* z;
    double2* w;
};

template <bool UNIT, bool FP64>
__global__ void __launch_bounds__(PB_THREADS) map_kernel(MapK K) {
    extern __shared__ __align__(16) unsigned char smem[];
    float4* sp = (float4*)smem;
    float2* sm = (float2*)(smem + TSB * sizeof(float4));
    float2* st3 = (float2*)(smem + TSB * (sizeof(float4) + sizeof(float2)));
    StarD* sd = (StarD*)smem;
    const int tid = threadIdx.x;
    const int64_t p = blockIdx.x * (int64_t)PB_THREADS + tid;
    const bool valid = p < K.count;
    const double2 z = valid ? K.z[p] : make_double2(0.0, 0.0);
    double S1x = 0.0, S1y = 0.0;
    df ax = df{0.f, 0.f}, ay = df{0.f, 0.f};
    const tf zx = tf_from_double(z.x), zy = tf_from_double(z.y);
    for (int t0 = 0; t0 < K.n; t0 += TSB) {
        const int tn = min(TSB, K.n - t0);
        __syncthreads();
        for (int j = tid; j < tn; j += PB_THREADS) {
            if (FP64) {
                sd[j] = K.s64[t0 + j];
            } else {
                sp[j] = K.dfp[t0 + j];
                sm[j] = K.dfm[t0 + j];
                st3[j] = K.dtf[t0 + j];
            }
        }
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < tn; j++) {
            if (FP64) {
                const StarD st = sd[j];
                const double dx = z.x - st.x, dy = z.y - st.y;
                const double q = st.z / (dx * dx + dy * dy);
                S1x = fma(q, dx, S1x);
                S1y = fma(-q, dy, S1y);
            } else {
                const float4 pp = sp[j];
                const float2 p3 = st3[j];
                const df dx = tf_sub(zx, pp.x, pp.y, p3.x);
                const df dy = tf_sub(zy, pp.z, pp.w, p3.y);
                const df inv = df_rcp(df_add(df_sqr(dx), df_sqr(dy)));
                const df q = UNIT ? inv : df_mul(df{sm[j].x, sm[j].y}, inv);
                ax = df_add(ax, df_mul(q, dx));
                ay = df_sub(ay, df_mul(q, dy));
            }
        }
    }
    if (!valid) return;
    if (!FP64) {
        S1x = df_to_double(ax);
        S1y = df_to_double(ay);
    }
    const double oms = 1.0 - K.kappa_s;
    double2 V = make_double2(0.0, 0.0);
    if (K.poly) V = poly_V(K.poly, z.x, z.y);
    K.w[p] = make_double2(oms * z.x + K.gamma * z.x - S1x + V.x, oms * z.y - K.gamma * z.y + S1y + V.y);
}

cudaError_t launch_map_caustics(const FieldDev& f, const double2* z, int64_t count, double2* w,
                                int hp_fp64, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    MapK K;
    K.poly = f.poly;
    K.dfp = f.star_dfp;
    K.dfm = f.star_dfm;
    K.dtf = f.star_tf;
    K.s64 = f.star64;
    K.n = (int)f.n;
    K.count = count;
    K.kappa_s = f.kappa_s;
    K.gamma = f.gamma;
    K.z = z;
    K.w = w;
    const unsigned blocks = (unsigned)((count + PB_THREADS - 1) / PB_THREADS);
    const size_t smem_df = TSB * (sizeof(float4) + 2 * sizeof(float2));
    const size_t smem_d = TSB * sizeof(StarD);
    cudaError_t e;
#define CC_LAUNCH_MAP(U, D, SM)                                                                       \
    do {                                                                                              \
        e = cudaFuncSetAttribute(map_kernel<U, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                 (int)(SM));                                                          \
        if (e != cudaSuccess) return e;                                                               \
        map_kernel<U, D><<<blocks, PB_THREADS, SM, st>>>(K);                                          \
    } while (0)
    if (hp_fp64)
        CC_LAUNCH_MAP(false, true, smem_d);
    else if (f.unit_mass)
        CC_LAUNCH_MAP(true, false, smem_df);
    else
        CC_LAUNCH_MAP(false, false, smem_df);
#undef CC_LAUNCH_MAP
    return cudaGetLastError();
}

}  // namespace ccg
