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
    const float4* dfp;
    const float2* dfm;
    const StarD* s64;
    int n;
    int64_t nr, m, points;
    int S;
    double kappa_s, gamma;
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
};

struct Sums {
    df S1x, S1y, S2x, S2y;
    float s3x, s3y, s4x, s4y, a3;
};

// One star in double-float.  d = z - z_i; r2 = |d|^2; inv = 1/r2; q = m inv;
// m/d = q conj(d); m/d^2 = q inv conj(d)^2 with conj(d)^2 = (dx^2 - dy^2, -2 dx dy).
template <bool UNIT>
__device__ __forceinline__ void star_df(const df& zx, const df& zy, const float4 p, const float2 mm,
                                        Sums& s) {
    const df dx = df_sub(zx, df{p.x, p.y});
    const df dy = df_sub(zy, df{p.z, p.w});
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
                                                int pass, int32_t it_in) {
    const double oms = 1.0 - K.kappa_s;
    const double2 ph = K.phase[row];
    const double Fx = K.gamma + S2x - oms * ph.x;
    const double Fy = S2y + oms * ph.y;
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
        est = 1.5 * ad * ad * s4a / s3a + ad * 4.0 * (double)FLT_EPSILON * (double)a3 / s3a;
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
    const double S1nx = S1x - (S2x * dx - S2y * dy) + ((double)s3x * d2x - (double)s3y * d2y) -
                        ((double)s4x * d3x - (double)s4y * d3y);
    const double S1ny = S1y - (S2x * dy + S2y * dx) + ((double)s3x * d2y + (double)s3y * d2x) -
                        ((double)s4x * d3y + (double)s4y * d3x);
    K.z_out[point] = make_double2(nzx, nzy);
    if (K.w_out) {
        const double wx = oms * nzx + K.gamma * nzx - S1nx;
        const double wy = oms * nzy - K.gamma * nzy + S1ny;
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
    if (est < K.tol_cert) atomic_max_double_nonneg(&K.rep->max_err_est, est);
    return true;
}

template <bool UNIT, bool FP64>
__device__ __forceinline__ void polish_body(const PolishK& K, const int64_t blk, unsigned char* smem,
                                            unsigned long long* s_passes_p) {
    float4* sp = (float4*)smem;
    float2* sm = (float2*)(smem + TSB * sizeof(float4));
    StarD* sd = (StarD*)smem;
    unsigned long long& s_passes = *s_passes_p;
    const int tid = threadIdx.x;
    const int64_t point = blk * (int64_t)PB_THREADS + tid;
    const bool valid = point < K.points;
    int64_t row = 0;
    float z0x = 0.f, z0y = 0.f;
    int32_t it_in = 0;
    if (valid) {
        row = point / K.nr;
        const int64_t g = point - row * K.nr;
        const int s = subchain_of_row(row, K.m, K.S);
        const int32_t k = K.perm[(size_t)s * K.nr + g];
        const float2 z0 = K.zrows[(size_t)row * K.nr + k];
        z0x = z0.x;
        z0y = z0.y;
        if (K.iters_out) it_in = K.iters_in[(size_t)row * K.nr + k];
    }
    double zx = z0x, zy = z0y;
    bool need = valid;
    if (tid == 0) s_passes = 0;
    const bool resident = K.n <= TSB;
    if (resident) {
        if (FP64) {
            for (int j = tid; j < K.n; j += PB_THREADS) sd[j] = K.s64[j];
        } else {
            for (int j = tid; j < K.n; j += PB_THREADS) {
                sp[j] = K.dfp[j];
                sm[j] = K.dfm[j];
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
            if (need && polish_epilogue(K, point, row, s.S1x, s.S1y, s.S2x, s.S2y, s.s3x, s.s3y, s.s4x,
                                        s.s4y, s.a3, zx, zy, z0x, z0y, pass, it_in))
                need = false;
        } else {
            Sums s;
            s.S1x = s.S1y = s.S2x = s.S2y = df{0.f, 0.f};
            s.s3x = s.s3y = s.s4x = s.s4y = s.a3 = 0.f;
            const df zxd = df_from_double(zx), zyd = df_from_double(zy);
            for (int t0 = 0; t0 < K.n; t0 += TSB) {
                const int tn = min(TSB, K.n - t0);
                if (!resident) {
                    __syncthreads();
                    for (int j = tid; j < tn; j += PB_THREADS) {
                        sp[j] = K.dfp[t0 + j];
                        sm[j] = K.dfm[t0 + j];
                    }
                    __syncthreads();
                }
                if (need) {
#pragma unroll 2
                    for (int j = 0; j < tn; j++) star_df<UNIT>(zxd, zyd, sp[j], sm[j], s);
                }
            }
            if (need && polish_epilogue(K, point, row, df_to_double(s.S1x), df_to_double(s.S1y),
                                        df_to_double(s.S2x), df_to_double(s.S2y), s.s3x, s.s3y, s.s4x,
                                        s.s4y, s.a3, zx, zy, z0x, z0y, pass, it_in))
                need = false;
        }
    }
    __syncthreads();
    if (tid == 0 && s_passes) atomicAdd(&K.rep->polish_passes, s_passes);
}

template <bool UNIT, bool FP64>
__global__ void __launch_bounds__(PB_THREADS) polish_kernel(PolishK K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ unsigned long long s_passes;
    polish_body<UNIT, FP64>(K, blockIdx.x, smem, &s_passes);
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
    K.dfp = a.f->star_dfp;
    K.dfm = a.f->star_dfm;
    K.s64 = a.f->star64;
    K.n = (int)a.f->n;
    K.nr = a.nr;
    K.m = a.m;
    K.points = (a.m + 1) * a.nr;
    K.S = a.S;
    K.kappa_s = a.f->kappa_s;
    K.gamma = a.f->gamma;
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
    const size_t smem = TSB * (sizeof(float4) + sizeof(float2));
    cudaError_t e = cudaFuncSetAttribute(polish_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    polish_batch_kernel<<<(unsigned)total_blocks, PB_THREADS, smem, st>>>((const PolishK*)tasks, count);
    return cudaGetLastError();
}

cudaError_t launch_polish(const PolishArgs& a, cudaStream_t st) {
    PolishK K = make_polish_k(a);
    const unsigned blocks = (unsigned)((K.points + PB_THREADS - 1) / PB_THREADS);
    const size_t smem_df = TSB * (sizeof(float4) + sizeof(float2));
    const size_t smem_d = TSB * sizeof(StarD);
    cudaError_t e;
#define CC_LAUNCH_POLISH(U, D, SM)                                                                     \
    do {                                                                                               \
        e = cudaFuncSetAttribute(polish_kernel<U, D>, cudaFuncAttributeMaxDynamicSharedMemorySize,     \
                                 (int)(SM));                                                           \
        if (e != cudaSuccess) return e;                                                                \
        polish_kernel<U, D><<<blocks, PB_THREADS, SM, st>>>(K);                                        \
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
    const float4* dfp;
    const float2* dfm;
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
    StarD* sd = (StarD*)smem;
    const int tid = threadIdx.x;
    const int64_t p = blockIdx.x * (int64_t)PB_THREADS + tid;
    const bool valid = p < K.count;
    const double2 z = valid ? K.z[p] : make_double2(0.0, 0.0);
    double S1x = 0.0, S1y = 0.0;
    df ax = df{0.f, 0.f}, ay = df{0.f, 0.f};
    const df zx = df_from_double(z.x), zy = df_from_double(z.y);
    for (int t0 = 0; t0 < K.n; t0 += TSB) {
        const int tn = min(TSB, K.n - t0);
        __syncthreads();
        for (int j = tid; j < tn; j += PB_THREADS) {
            if (FP64) {
                sd[j] = K.s64[t0 + j];
            } else {
                sp[j] = K.dfp[t0 + j];
                sm[j] = K.dfm[t0 + j];
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
                const df dx = df_sub(zx, df{pp.x, pp.y});
                const df dy = df_sub(zy, df{pp.z, pp.w});
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
    K.w[p] = make_double2(oms * z.x + K.gamma * z.x - S1x, oms * z.y - K.gamma * z.y + S1y);
}

cudaError_t launch_map_caustics(const FieldDev& f, const double2* z, int64_t count, double2* w,
                                int hp_fp64, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    MapK K;
    K.dfp = f.star_dfp;
    K.dfm = f.star_dfm;
    K.s64 = f.star64;
    K.n = (int)f.n;
    K.count = count;
    K.kappa_s = f.kappa_s;
    K.gamma = f.gamma;
    K.z = z;
    K.w = w;
    const unsigned blocks = (unsigned)((count + PB_THREADS - 1) / PB_THREADS);
    const size_t smem_df = TSB * (sizeof(float4) + sizeof(float2));
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
