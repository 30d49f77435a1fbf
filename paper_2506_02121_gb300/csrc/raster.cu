// Source-plane rasters: caustic-crossing counts (Sec. 5.1) and distance to the nearest
// caustic for an expanding source (Sec. 5.2).
//
// Crossing map.  N_cc = -winding number of the clockwise caustic polygons (Sec. 5.1), by
// Sunday's crossing rule: an upward edge (a.y <= y < b.y) adds +1 to pixel centres strictly
// left of it, a downward edge (b.y <= y < a.y) adds -1 to centres strictly right of it.  For
// both, the affected centres of one pixel row are a prefix 0..c-1 of that row (left of an
// upward edge = right of a downward edge = x below the crossing abscissa), so, as the paper
// does, the kernel loops over segments rather than pixels: each segment adds +-1 at index
// c-1 of a per-row difference array and a suffix scan of every row gives the winding
// number.  c is found from the crossing abscissa and then settled with an exact
// orientation predicate, so the counts equal a per-pixel evaluation bit for bit.
//
// Distance map.  Feature pixels have a 4-neighbour of different N_cc; the map border is not
// a caustic.  Exact squared distances by the separable transform of Felzenszwalb &
// Huttenlocher (2012): a column pass (distance to the nearest feature in the column) and a
// row pass (lower envelope of the parabolas (i - q)^2 + g(q)^2, intersections compared as
// exact integer fractions).
#include <float.h>

#include <algorithm>

#include "cc_internal.h"

namespace ccg {

// ----------------------------------------------------------------------------------
// Exact orientation sign: +1 if c is strictly left of the directed line a->b, -1 if
// strictly right, 0 if on it.  A floating-point filter (Shewchuk 1997, orient2d with the
// error bound (3 + 16 eps) eps |detleft + detright|) settles almost every call; otherwise
// the determinant is summed exactly from error-free pieces.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ void eft_sum(double a, double b, double& s, double& e) {
    s = __dadd_rn(a, b);
    const double bv = __dsub_rn(s, a);
    const double av = __dsub_rn(s, bv);
    e = __dadd_rn(__dsub_rn(a, av), __dsub_rn(b, bv));
}

__device__ __forceinline__ void eft_prod(double a, double b, double& p, double& e) {
    p = __dmul_rn(a, b);
    e = __fma_rn(a, b, -p);
}

__device__ __noinline__ int orient_exact_slow(double ax, double ay, double bx, double by, double cx,
                                              double cy) {
    // The determinant (ax-cx)(by-cy) - (ay-cy)(bx-cx) as an exact sum of 16 doubles.
    double d[8];
    eft_sum(ax, -cx, d[0], d[1]);
    eft_sum(by, -cy, d[2], d[3]);
    eft_sum(ay, -cy, d[4], d[5]);
    eft_sum(bx, -cx, d[6], d[7]);
    double t[16];
    int nt = 0;
    for (int u = 0; u < 2; u++)
        for (int v = 0; v < 2; v++) {
            eft_prod(d[u], d[2 + v], t[nt], t[nt + 1]);
            nt += 2;
            double p, e;
            eft_prod(d[4 + u], d[6 + v], p, e);
            t[nt++] = -p;
            t[nt++] = -e;
        }
    // Fold every term into a non-overlapping expansion (increasing magnitude); each fold is
    // a chain of error-free sums, so the expansion always equals the exact partial sum.
    double h[17];
    int nh = 0;
    for (int i = 0; i < 16; i++) {
        double q = t[i];
        for (int j = 0; j < nh; j++) {
            double s, e;
            eft_sum(q, h[j], s, e);
            h[j] = e;
            q = s;
        }
        h[nh++] = q;
    }
    for (int j = nh - 1; j >= 0; j--) {
        if (h[j] > 0.0) return 1;
        if (h[j] < 0.0) return -1;
    }
    return 0;
}

__device__ __forceinline__ int orient_sign(double ax, double ay, double bx, double by, double cx,
                                           double cy) {
    const double l = __dmul_rn(__dsub_rn(ax, cx), __dsub_rn(by, cy));
    const double r = __dmul_rn(__dsub_rn(ay, cy), __dsub_rn(bx, cx));
    const double det = __dsub_rn(l, r);
    double sum;
    if (l > 0.0) {
        if (r <= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        sum = __dadd_rn(l, r);
    } else if (l < 0.0) {
        if (r >= 0.0) return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
        sum = -__dadd_rn(l, r);
    } else {
        return det > 0.0 ? 1 : (det < 0.0 ? -1 : 0);
    }
    const double eps = 1.1102230246251565e-16;  // 2^-53
    const double bound = __dmul_rn((3.0 + 16.0 * eps) * eps, sum);
    if (det > bound) return 1;
    if (-det > bound) return -1;
    return orient_exact_slow(ax, ay, bx, by, cx, cy);
}

// Pixel centre lo + (i + 0.5) * step in IEEE FP64, no contraction.
__device__ __forceinline__ double pix(double lo, double step, int64_t i) {
    return __dadd_rn(lo, __dmul_rn(__dadd_rn((double)i, 0.5), step));
}

// Maps of up to this many pixels per side take the conversion-free forms above.
constexpr int SMALL_GRID = 1 << 20;

struct CrossK {
    const double2* w;
    int64_t rows, nr;
    double x0, sx, y0, sy;
    int W, H;
    int* D;
    float x0f, inv_sxf, y0f, inv_syf, syf;  // FP32 copies (host round-to-nearest) for the fast path
};

constexpr int XS_THREADS = 256;

// A double as a float by truncating its significand, with integer instructions only (no
// FP64 pipe): |f - v| <= 2^-23 |v|, and 0 for |v| < 2^-100 (|f - v| < 2^-100).  ok turns
// false for a non-finite v or |v| >= 2^100, which the fast path does not take.
__device__ __forceinline__ float f32_trunc(double v, bool& ok) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7FF);
    if (e >= 1023 + 100) {
        ok = false;
        return 0.f;
    }
    if (e < 1023 - 100) return 0.f;
    return __uint_as_float((unsigned)(b >> 63) << 31 | (unsigned)(e - 1023 + 127) << 23 |
                           (unsigned)((b >> 29) & 0x7FFFFFu));
}

// Integer key ordering finite doubles like their values (-0 below +0), so that comparing two
// doubles takes no FP64 instruction.
__device__ __forceinline__ long long dkey(double v) {
    const long long k = __double_as_longlong(v);
    return k ^ ((k >> 63) & 0x7FFFFFFFFFFFFFFFLL);
}

// Segment flags in the scatter kernel's shared memory.
constexpr int XS_FAST = 1;  // coordinates within the fast path's range

// One thread per segment finds the pixel rows its half-open y-range may contain, in FP32
// with a margin (1.5x a rigorous bound on the rounding) that covers the rounding.  The
// (segment, candidate row) pairs of a warp are then laid out by a warp prefix sum and
// processed by all 32 lanes together:
//  - a row more than the margin inside the candidate range is in the segment's half-open
//    y-range for certain; only a row within the margin of either end takes the exact FP64
//    test on its FP64 pixel centre;
//  - the count c of pixel centres left of the crossing abscissa (c = ceil(u) for
//    u = (x_c - x0)/sx - 1/2) comes from an FP32 evaluation of u with a rigorous bound E on
//    its error, propagated term by term from the inputs' truncation (2^-23 relative) and
//    each FP32 rounding (2^-24); when an integer lies within E of u the exact orientation
//    predicate settles c in FP64.
// FP32 carries all but a few pairs per thousand, so the counts equal a per-pixel
// evaluation of Sunday's rule bit for bit while the FP64 pipe (1/64 of the FP32 rate on
// this part) stays off the critical path.
__global__ void __launch_bounds__(XS_THREADS) crossing_scatter_kernel(CrossK K) {
    __shared__ double2 s_a[XS_THREADS], s_b[XS_THREADS];
    __shared__ float4 s_f[XS_THREADS];   // a.x, a.y, b.x, b.y truncated to FP32
    __shared__ float2 s_t[XS_THREADS];   // candidate range ends tl, th (row units, FP32)
    __shared__ float s_eps[XS_THREADS];  // their error margin
    __shared__ int s_r0[XS_THREADS], s_excl[XS_THREADS], s_flag[XS_THREADS];
    const int lane = threadIdx.x & 31;
    const int wbase = threadIdx.x & ~31;
    const int64_t t = blockIdx.x * (int64_t)XS_THREADS + threadIdx.x;
    const int64_t nseg = (K.rows - 1) * K.nr;
    int r0 = 0, cnt = 0, flag = 0;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    float4 fv = make_float4(0.f, 0.f, 0.f, 0.f);
    float tl = 0.f, th = 0.f, eps = 0.f;
    if (t < nseg) {
        a = K.w[t];
        b = K.w[t + K.nr];
        const unsigned long long ya = (unsigned long long)__double_as_longlong(a.y);
        const unsigned long long yb = (unsigned long long)__double_as_longlong(b.y);
        const bool finite = ((((unsigned long long)__double_as_longlong(a.x) >> 52) & 0x7FF) != 0x7FF) &&
                            ((((unsigned long long)__double_as_longlong(b.x) >> 52) & 0x7FF) != 0x7FF) &&
                            (((ya >> 52) & 0x7FF) != 0x7FF) && (((yb >> 52) & 0x7FF) != 0x7FF);
        // a.y == b.y (equal bits, or both zero of either sign): no pixel centre can satisfy
        // a.y <= y < b.y
        const bool same_y = ya == yb || ((ya | yb) << 1) == 0ull;
        if (finite && !same_y) {
            bool ok = true;
            fv.x = f32_trunc(a.x, ok);
            fv.y = f32_trunc(a.y, ok);
            fv.z = f32_trunc(b.x, ok);
            fv.w = f32_trunc(b.y, ok);
            float fr0 = 0.0f, fr1 = 0.0f;
            if (ok) {
                flag = XS_FAST;
                const float lo = fminf(fv.y, fv.w), hi = fmaxf(fv.y, fv.w);
                tl = (lo - K.y0f) * K.inv_syf - 0.5f;
                th = (hi - K.y0f) * K.inv_syf - 0.5f;
                // |tl - exact| <= 2^-23 (|lo| + |y0| + |lo - y0|) / sy + 2^-24 (2 |tl| + 1) (truncation,
                // the host-rounded y0 and 1/sy, each operation rounding once), likewise th; with
                // a 1.5x margin, and 1e-6 row for the FP64 pixel centres' own rounding
                const float ym = fmaxf(fabsf(lo), fabsf(hi)), yd = fmaxf(fabsf(lo - K.y0f), fabsf(hi - K.y0f));
                eps = 1e-6f + 1.8e-7f * ((ym + fabsf(K.y0f) + yd) * fabsf(K.inv_syf) + fabsf(tl) + fabsf(th) + 1.0f);
                if (K.H <= SMALL_GRID) {
                    // (clamped first: the exact range only matters inside [0, H))
                    r0 = max(ceil_small(fminf(fmaxf(tl - eps, -2.0f), (float)SMALL_GRID + 2.0f)), 0);
                    const int r1 = min(floor_small(fminf(fmaxf(th + eps, -2.0f), (float)SMALL_GRID + 2.0f)) + 1, K.H);
                    cnt = max(r1 - r0, 0);
                    if (cnt == 0) r0 = 0;
                    fr0 = fr1 = 0.0f;
                } else {
                    fr0 = fmaxf(ceilf(tl - eps), 0.0f);
                    fr1 = fminf(floorf(th + eps) + 1.0f, (float)K.H);
                }
            } else {
                // coordinates beyond 2^100: candidate rows in FP64 (every row is tested exactly)
                const double lo = fmin(a.y, b.y), hi = fmax(a.y, b.y);
                const double tld = (lo - K.y0) / K.sy - 0.5, thd = (hi - K.y0) / K.sy - 0.5;
                fr0 = (float)fmax(ceil(tld - 1e-3 - 1e-9 * fabs(tld)), 0.0);
                fr1 = (float)fmin(floor(thd + 1e-3 + 1e-9 * fabs(thd)) + 1.0, (double)K.H);
            }
            if (fr1 > fr0) {
                r0 = (int)fr0;
                cnt = (int)fr1 - r0;
            }
        }
    }
    // warp prefix sum of candidate counts
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += y;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    if (total == 0) return;  // whole warp: nothing to do
    s_a[threadIdx.x] = a;
    s_b[threadIdx.x] = b;
    s_f[threadIdx.x] = fv;
    s_t[threadIdx.x] = make_float2(tl, th);
    s_eps[threadIdx.x] = eps;
    s_r0[threadIdx.x] = r0;
    s_excl[threadIdx.x] = incl - cnt;
    s_flag[threadIdx.x] = flag;
    __syncwarp();
    for (int base = 0; base < total; base += 32) {
        const int item = base + lane;
        if (item >= total) break;
        // owning segment: the last lane j with excl[j] <= item
        int lo = 0, hi = 31;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_excl[wbase + mid] <= item) lo = mid;
            else hi = mid - 1;
        }
        const int j = wbase + lo;
        const int r = s_r0[j] + (item - s_excl[j]);
        const bool fast = s_flag[j] & XS_FAST;
        const double2 sa = s_a[j], sb = s_b[j];
        const bool up = dkey(sa.y) < dkey(sb.y);  // exact: a.y != b.y here
        const int sgn = up ? 1 : -1;
        const float rf = K.H <= SMALL_GRID ? i2f_small(r) : (float)r;
        bool sure = false;
        if (fast) {
            const float2 tt = s_t[j];
            const float e = s_eps[j];
            sure = rf > tt.x + e && rf < tt.y - e;
        }
        double py = 0.0;
        if (!sure) {  // exact half-open row test on the FP64 pixel centre
            const bool upx = sa.y < sb.y;
            const double ylo = upx ? sa.y : sb.y, yhi = upx ? sb.y : sa.y;
            py = pix(K.y0, K.sy, r);
            if (!(ylo <= py && py < yhi)) continue;
        }
        int c = -1;
        float u = 0.f;
        bool have_u = false;  // u holds an FP32 estimate of the abscissa
        if (fast) {
            // u = (x_c - x0)/sx - 1/2 in FP32 and a bound E on its error (EPS >= 2^-23 (1 + 2^-23):
            // truncation of the inputs; the host-rounded constants and each operation add
            // 2^-24 relative)
            const float EPS = 1.2e-7f;
            const float4 f = s_f[j];
            const float sxr = f.x - K.x0f, e1 = EPS * (fabsf(f.x) + fabsf(K.x0f) + fabsf(sxr));
            const float exf = f.z - f.x, e2 = EPS * (fabsf(f.x) + fabsf(f.z) + fabsf(exf));
            const float eyf = f.w - f.y, e3 = EPS * (fabsf(f.y) + fabsf(f.w) + fabsf(eyf));
            const float ayr = f.y - K.y0f, e4 = EPS * (fabsf(f.y) + fabsf(K.y0f) + fabsf(ayr));
            const float den = fabsf(eyf) - e3;
            if (den > 0.f) {
                // py - y0 = (r + 1/2) sy: syf and the product each round once; the FP64 pixel
                // centre itself is within 2^-52 (|y0| + |py|) of its real value
                const float pr = (rf + 0.5f) * K.syf;
                const float e5 = 2.0f * EPS * fabsf(pr) + 1e-12f * (fabsf(K.y0f) + fabsf(pr));
                const float ty = pr - ayr, e6 = e5 + e4 + EPS * fabsf(ty);
                const float tf = __fdiv_rn(ty, eyf);
                const float dT = __fdiv_rn(e6 + fabsf(tf) * e3, den) + EPS * fabsf(tf);
                const float p = exf * tf, e7 = fabsf(exf) * dT + (fabsf(tf) + dT) * e2 + EPS * fabsf(p);
                const float sm = sxr + p, e8 = e1 + e7 + EPS * fabsf(sm);
                const float v = sm * K.inv_sxf, e9 = e8 * fabsf(K.inv_sxf) * 1.0001f + 2.0f * EPS * fabsf(v);
                u = v - 0.5f;
                const float E = 1.01f * (e9 + EPS * fabsf(u)) + 1e-6f;
                if (isfinite(u) && isfinite(E)) {
                    have_u = true;
                    if (u - E >= (float)K.W) c = K.W;
                    else if (u + E <= 0.f) c = 0;
                    else if (K.W <= SMALL_GRID) {
                        // u in (-E, W + E): no integer within E of u means c = ceil(u)
                        const float t = u + MAGIC_F, nf = t - MAGIC_F;
                        if (E < 0.5f && fabsf(u - nf) > E) {
                            const int n = __float_as_int(t) - MAGIC_I;
                            c = min(max(nf > u ? n : n + 1, 0), K.W);
                        }
                    } else if (ceilf(u - E) == ceilf(u + E)) {
                        c = (int)fminf(fmaxf(ceilf(u), 0.0f), (float)K.W);
                    }
                }
            }
        }
        if (c < 0) {
            // exact: c = the number of pixel centres i with orient(a, b, P_i) == sgn, which hold
            // for a prefix of the row (left of the crossing).  Test the two centres around an
            // estimate of the crossing first, then bisect what is left: at most about
            // log2(W) + 2 predicate calls however poor the estimate.
            if (sure) py = pix(K.y0, K.sy, r);
            double ue = u;
            if (!have_u) {
                const double ey = sb.y - sa.y;
                ue = ((sa.x - K.x0) + (sb.x - sa.x) * ((py - sa.y) / ey)) / K.sx - 0.5;
            }
            double ce = ceil(ue);
            ce = fmin(fmax(ce, 0.0), (double)K.W);
            if (!(ce == ce)) ce = 0.0;  // NaN guard
            const int ci = (int)ce;
            auto left = [&](int i) { return orient_sign(sa.x, sa.y, sb.x, sb.y, pix(K.x0, K.sx, i), py) == sgn; };
            int lo = 0, hi = K.W;  // c in [lo, hi]
            if (ci > 0) {
                if (left(ci - 1)) lo = ci;
                else hi = ci - 1;
            }
            if (lo <= ci && ci < hi) {
                if (left(ci)) lo = ci + 1;
                else hi = ci;
            }
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (left(mid)) lo = mid + 1;
                else hi = mid;
            }
            c = lo;
        }
        if (c > 0) atomicAdd(&K.D[(int64_t)r * K.W + (c - 1)], sgn);
    }
}

// Per row: ncc[i] = -(sum_{i' >= i} D[i']).  One CTA per row, chunks right to left.
constexpr int SCAN_T = 256, SCAN_ITEMS = 8;
__global__ void __launch_bounds__(SCAN_T) row_suffix_kernel(int* ncc, int W) {
    __shared__ int warp_tot[SCAN_T / 32];
    int* p = ncc + (int64_t)blockIdx.x * W;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int CH = SCAN_T * SCAN_ITEMS;
    int carry = 0;
    for (int end = W; end > 0; end -= CH) {
        const int beg = end - CH;  // may be negative
        int v[SCAN_ITEMS];
        int tsum = 0;
#pragma unroll
        for (int q = 0; q < SCAN_ITEMS; q++) {
            const int idx = beg + tid * SCAN_ITEMS + q;
            v[q] = idx >= 0 ? p[idx] : 0;
            tsum += v[q];
        }
        // inclusive suffix scan of thread sums: reverse thread order within the block
        int x = tsum;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int y = __shfl_down_sync(0xffffffffu, x, off);
            if (lane + off < 32) x += y;
        }
        if (lane == 0) warp_tot[wid] = x;
        __syncthreads();
        int after = 0;  // totals of later warps
        for (int q = wid + 1; q < SCAN_T / 32; q++) after += warp_tot[q];
        int total = 0;
        for (int q = 0; q < SCAN_T / 32; q++) total += warp_tot[q];
        // x = sum of threads tid..end of warp; exclusive suffix of this thread:
        int run = carry + after + (x - tsum);
#pragma unroll
        for (int q = SCAN_ITEMS - 1; q >= 0; q--) {
            run += v[q];
            const int idx = beg + tid * SCAN_ITEMS + q;
            if (idx >= 0) p[idx] = -run;
        }
        carry += total;
        __syncthreads();
    }
}

cudaError_t launch_crossing_map(const double2* w, int64_t rows, int64_t nr, double x0, double x1,
                                double y0, double y1, int32_t W, int32_t H, int32_t* ncc,
                                cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(ncc, 0, sizeof(int32_t) * (size_t)W * H, st);
    if (e != cudaSuccess) return e;
    if (rows >= 2 && nr >= 1) {
        CrossK K;
        K.w = w;
        K.rows = rows;
        K.nr = nr;
        K.x0 = x0;
        K.sx = (x1 - x0) / (double)W;
        K.y0 = y0;
        K.sy = (y1 - y0) / (double)H;
        K.W = W;
        K.H = H;
        K.D = ncc;
        K.x0f = (float)x0;
        K.inv_sxf = (float)(1.0 / K.sx);
        K.y0f = (float)y0;
        K.inv_syf = (float)(1.0 / K.sy);
        K.syf = (float)K.sy;
        const int64_t segs = (rows - 1) * nr;
        crossing_scatter_kernel<<<(unsigned)((segs + XS_THREADS - 1) / XS_THREADS), XS_THREADS, 0, st>>>(K);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    row_suffix_kernel<<<(unsigned)H, SCAN_T, 0, st>>>(ncc, W);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Distance map
// ----------------------------------------------------------------------------------
constexpr int DIST_INF = 1 << 30;

__device__ __forceinline__ bool feature_at(const int32_t* ncc, int W, int H, int r, int i) {
    const int32_t v = ncc[(int64_t)r * W + i];
    if (i > 0 && ncc[(int64_t)r * W + i - 1] != v) return true;
    if (i + 1 < W && ncc[(int64_t)r * W + i + 1] != v) return true;
    if (r > 0 && ncc[(int64_t)(r - 1) * W + i] != v) return true;
    if (r + 1 < H && ncc[(int64_t)(r + 1) * W + i] != v) return true;
    return false;
}

constexpr int EDT_CHUNK = 128;  // rows per column-pass chunk

// Feature flags (1 byte per pixel) into the stack plane, which the row pass reuses later.
__global__ void edt_feature_kernel(const int32_t* ncc, int W, int H, uint8_t* feat) {
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= (int64_t)W * H) return;
    const int r = (int)(p / W), i = (int)(p - (int64_t)r * W);
    feat[p] = feature_at(ncc, W, H, r, i) ? 1 : 0;
}

// First and last feature row of every (chunk, column); -1 when none.
__global__ void edt_chunk_kernel(const uint8_t* feat, int W, int H, int2* summ) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= W) return;
    const int r0 = c * EDT_CHUNK, r1 = min(H, r0 + EDT_CHUNK);
    int first = -1, last = -1;
    for (int r = r0; r < r1; r++)
        if (feat[(int64_t)r * W + i]) {
            if (first < 0) first = r;
            last = r;
        }
    summ[(int64_t)c * W + i] = make_int2(first, last);
}

// g[r][i] = |r - nearest feature row in column i| (DIST_INF if the column has none), one
// thread per (chunk, column) seeded with the nearest features of the other chunks.
__global__ void edt_column_kernel(const uint8_t* feat, const int2* summ, int W, int H, int nchunk,
                                  int32_t* g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= W) return;
    int above = -1, below = -1;
    for (int q = c - 1; q >= 0 && above < 0; q--) above = summ[(int64_t)q * W + i].y;
    for (int q = c + 1; q < nchunk && below < 0; q++) below = summ[(int64_t)q * W + i].x;
    const int r0 = c * EDT_CHUNK, r1 = min(H, r0 + EDT_CHUNK);
    int last = above;
    for (int r = r0; r < r1; r++) {
        if (feat[(int64_t)r * W + i]) last = r;
        g[(int64_t)r * W + i] = last < 0 ? DIST_INF : r - last;
    }
    int next = below;
    for (int r = r1 - 1; r >= r0; r--) {
        const int64_t o = (int64_t)r * W + i;
        if (feat[o]) next = r;
        if (next >= 0 && next - r < g[o]) g[o] = next - r;
    }
}

__device__ __forceinline__ long long edt_key(const int32_t* f, int q) {
    return (long long)f[q] * f[q] + (long long)q * q;
}

// Limits of the banded row pass: g values are 16-bit in shared memory (0xFFFF: no feature in
// the column), hull stacks 8-bit band positions (bands of at most 256 columns).
constexpr int EDT_BAND_MAX_W = 32768;
constexpr int EDT_BAND_MAX_H = 65535;  // g < H fits 16 bits, 0xFFFF marks "no feature"

__device__ __forceinline__ long long edt_lift(int q, int gq) { return (long long)q * q + (long long)gq * gq; }

// Site v (u < v < w in column order) is strictly below the chord u-w of the lifted points,
// i.e. intersection(u, v) < intersection(v, w): its parabola alone is lowest somewhere.
__device__ __forceinline__ bool edt_keep(int u, long long cu, int v, long long cv, int w, long long cw) {
    return (cw - cv) * (long long)(v - u) > (cv - cu) * (long long)(w - v);
}

constexpr int EDT_SQRT_T = 65536;  // entries of the distance table of the banded path

// Row pass for very wide maps: one thread per row, envelope stack in global memory.
__global__ void edt_row_kernel(const int32_t* g, int W, int H, double pixel, int32_t* vstack,
                               double* d_out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int32_t* f = g + (int64_t)r * W;
    int32_t* v = vstack + (int64_t)r * W;
    double* out = d_out + (int64_t)r * W;
    int k = -1;
    for (int q = 0; q < W; q++) {
        if (f[q] >= DIST_INF) continue;
        const long long fq = edt_key(f, q);
        while (k >= 1) {
            const int p = v[k], pp = v[k - 1];
            const long long n1 = fq - edt_key(f, p), d1 = 2LL * (q - p);
            const long long n2 = edt_key(f, p) - edt_key(f, pp), d2 = 2LL * (p - pp);
            if (n1 * d2 <= n2 * d1) k--;
            else break;
        }
        v[++k] = q;
    }
    if (k < 0) {
        for (int i = 0; i < W; i++) out[i] = __longlong_as_double(0x7ff0000000000000LL);
        return;
    }
    int j = 0;
    for (int i = 0; i < W; i++) {
        while (j < k) {
            const int p = v[j], q = v[j + 1];
            const long long n = edt_key(f, q) - edt_key(f, p), d = 2LL * (q - p);
            if (n < (long long)i * d) j++;
            else break;
        }
        const int p = v[j];
        const long long d2 = (long long)(i - p) * (i - p) + (long long)f[p] * f[p];
        out[i] = pixel * sqrt((double)d2);
    }
}

// ----------------------------------------------------------------------------------
// Distance to the nearest caustic for a source moving along a direction (Sec. 5.2): one
// thread per pixel follows the ray from the pixel centre through the pixel grid and stops
// at the first caustic (feature) pixel (0 if it starts on one, +inf if it leaves the map:
// the border is not a caustic).  The traversal uses IEEE single-precision operations in a
// fixed order: after k steps the next vertical (horizontal) grid line is crossed at
// (0.5 + k) * tdx (tdy), tdx = 1/|cos|, tdy = 1/|sin|; the smaller parameter is taken, the
// horizontal line on ties.
// ----------------------------------------------------------------------------------
struct MoveK {
    const int32_t* ncc;
    int W, H;
    double pixel;
    int sx, sy;
    float tdx, tdy;
    double* out;
};

__global__ void moving_distance_kernel(MoveK K) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y;
    if (i >= K.W) return;
    double d;
    if (feature_at(K.ncc, K.W, K.H, r, i)) {
        d = 0.0;
    } else {
        int x = i, y = r;
        long long nx = 0, ny = 0;
        d = __longlong_as_double(0x7ff0000000000000LL);
        for (;;) {
            const float tx = K.sx ? __fmul_rn(__fadd_rn(0.5f, (float)nx), K.tdx) : __int_as_float(0x7f800000);
            const float ty = K.sy ? __fmul_rn(__fadd_rn(0.5f, (float)ny), K.tdy) : __int_as_float(0x7f800000);
            float t;
            if (tx < ty) {
                x += K.sx;
                nx++;
                t = tx;
            } else {
                y += K.sy;
                ny++;
                t = ty;
            }
            if (x < 0 || x >= K.W || y < 0 || y >= K.H) break;
            if (feature_at(K.ncc, K.W, K.H, y, x)) {
                d = __dmul_rn(K.pixel, (double)t);
                break;
            }
        }
    }
    K.out[(int64_t)r * K.W + i] = d;
}

cudaError_t launch_moving_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, float c, float s,
                                       double* d_out, cudaStream_t st) {
    MoveK K;
    K.ncc = ncc;
    K.W = W;
    K.H = H;
    K.pixel = pixel;
    K.sx = c > 0.0f ? 1 : (c < 0.0f ? -1 : 0);
    K.sy = s > 0.0f ? 1 : (s < 0.0f ? -1 : 0);
    volatile float one = 1.0f;  // IEEE divisions on the host, as the kernel's traversal expects
    K.tdx = K.sx ? one / fabsf(c) : 0.0f;
    K.tdy = K.sy ? one / fabsf(s) : 0.0f;
    K.out = d_out;
    dim3 grid((unsigned)((W + 127) / 128), (unsigned)H);
    moving_distance_kernel<<<grid, 128, 0, st>>>(K);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Distance map, banded path (W <= EDT_BAND_MAX_W, H <= EDT_BAND_MAX_H).  The column pass is
// never written out: one read of N_cc gives every pixel's feature bit, packed 64 rows to a
// word per column (W H / 8 bytes), with each 64-row chunk's first and last feature row; a
// scan over the chunks gives, per (chunk, column), the nearest feature row above and below
// the chunk.  The row pass then takes each column distance g from the column's word (the
// nearest set bit on either side of the row, by count-leading/trailing-zeros) or the
// chunk's neighbours, all read from L2, builds the lower envelope, and fills the row.
// ----------------------------------------------------------------------------------
constexpr int EDT_BITS = 64;  // rows per feature word

// Feature word of (chunk c, column i): bit b set when pixel (c * 64 + b, i) is a feature;
// and the chunk's first and last feature row (-1 when none).  One thread per (chunk,
// column); a warp covers 32 adjacent columns and passes the row values to its neighbours
// by shuffles (lanes past the map's edge take part with no loads).
__global__ void __launch_bounds__(128) edt_bits_kernel(const int32_t* ncc, int W, int H, unsigned long long* bits,
                                                         int2* summ) {
    const int lane = threadIdx.x & 31;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    const int r0 = c * EDT_BITS, r1 = min(H, r0 + EDT_BITS);
    const bool in = i < W;
    auto at = [&](int r, int col) -> int32_t { return ncc[(int64_t)r * W + col]; };
    int32_t up = 0, cur = 0, dn = 0;
    const bool has_up = r0 > 0;
    if (in) {
        if (has_up) up = at(r0 - 1, i);
        cur = at(r0, i);
    }
    unsigned long long word = 0ull;
    int first = -1, last = -1;
    for (int r = r0; r < r1; r++) {
        const bool has_dn = r + 1 < H;
        if (in && has_dn) dn = at(r + 1, i);
        int32_t left = __shfl_up_sync(0xffffffffu, cur, 1);
        int32_t right = __shfl_down_sync(0xffffffffu, cur, 1);
        if (in && lane == 0 && i > 0) left = at(r, i - 1);
        if (in && lane == 31 && i + 1 < W) right = at(r, i + 1);
        const bool f = in && ((i > 0 && left != cur) || (i + 1 < W && right != cur) || (r > 0 && up != cur) ||
                              (has_dn && dn != cur));
        if (f) {
            word |= 1ull << (r - r0);
            if (first < 0) first = r;
            last = r;
        }
        up = cur;
        cur = dn;
    }
    if (in) {
        bits[(int64_t)c * W + i] = word;
        summ[(int64_t)c * W + i] = make_int2(first, last);
    }
}

// Per column: nearest feature row above chunk c (in chunks < c) and below it (in chunks > c),
// -1 when none.
__global__ void edt_chunk_scan_kernel(const int2* summ, int W, int nchunk, int2* ab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W) return;
    int above = -1;
    for (int c = 0; c < nchunk; c++) {
        ab[(int64_t)c * W + i].x = above;
        const int l = summ[(int64_t)c * W + i].y;
        if (l >= 0) above = l;
    }
    int below = -1;
    for (int c = nchunk - 1; c >= 0; c--) {
        ab[(int64_t)c * W + i].y = below;
        const int f = summ[(int64_t)c * W + i].x;
        if (f >= 0) below = f;
    }
}

// Distance in rows from row r to the nearest feature of column q (0xFFFF when the column has
// none): the nearest set bit of the column's word on either side of bit b = r mod 64, else
// the nearest feature of the chunks above or below.
__device__ __forceinline__ int edt_col_dist(unsigned long long w, int2 ab, int r, int b) {
    int d = 0xFFFF;
    const unsigned long long lo = b == 63 ? w : (w & ((2ull << b) - 1ull));  // rows <= r in the chunk
    if (lo) d = b - (63 - __clzll(lo));
    else if (ab.x >= 0) d = r - ab.x;
    const unsigned long long hi = w >> b;  // rows >= r in the chunk
    if (hi) d = min(d, __ffsll(hi) - 1);
    else if (ab.y >= 0) d = min(d, ab.y - r);
    return d;
}

// First pixel owned by envelope vertex v = (qv, cv) after its predecessor u = (qu, cu),
// qu < qv: the smallest integer t with (t - qv)^2 + gv^2 <= (t - qu)^2 + gu^2, i.e.
// t (2 (qv - qu)) >= cv - cu (c = q^2 + g^2), clamped to [0, W + 1].  An FP32 quotient lands
// within one of it, and exact int64 products settle it.
__device__ __forceinline__ int edt_start(int qu, long long cu, int qv, long long cv, int W) {
    const long long num = cv - cu;  // |num| < 2^38 (q < 2^15, g < 2^16)
    const int den = 2 * (qv - qu);  // < 2^16
    const float numf = fmaf(i2f_small((int)(num >> 16)), 65536.0f, i2f_small((int)(num & 0xFFFF)));
    const float est = numf / i2f_small(den);
    if (!(est < (float)W + 2.0f)) return W + 1;
    if (est < -2.0f) return 0;
    int t = ceil_small(est);
    while ((long long)(t - 1) * den >= num) t--;
    while ((long long)t * den < num) t++;
    return max(0, min(t, W + 1));
}

// Row pass, one CTA of EDT_NB threads per row.  Thread l owns the band of columns
// [l Bw, (l + 1) Bw), Bw = ceil(W / EDT_NB) <= 256 (band layout: column q = l Bw + k at
// [k EDT_LSB + l], so threads stepping through their bands together touch consecutive
// words).  g of the row comes from the feature words; each thread builds the hull of its
// band; log2(EDT_NB) rounds of bridge merges join neighbouring bands (the hull of two
// column-separated sets keeps a prefix of the left hull and a suffix of the right one,
// found by walking both ends until neither end point can be dropped); then every surviving
// vertex writes its column at the first pixel it owns (own[]; a vertex whose range is empty
// writes nothing), and each warp fills a quarter of the row, 32 pixels at a time, with the
// owner = the running maximum of own[] (envelope columns increase with the pixel), seeded
// with the maximum over the quarters before it.  All comparisons are exact int64.
constexpr int EDT_NB = 128;            // threads (bands) per row
constexpr int EDT_LSB = EDT_NB + 1;    // band-layout stride
constexpr int EDT_NW = EDT_NB / 32;    // warps per row

__device__ __forceinline__ int edt_warp_max_scan(int v, int lane) {
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, off);
        if (lane >= off) v = max(v, y);
    }
    return v;
}

__global__ void __launch_bounds__(EDT_NB) edt_row_env_kernel(const unsigned long long* bits, const int2* ab, int W,
                                                             double pixel, double* d_out, const double* dtab, int T) {
    extern __shared__ uint16_t edt_sh[];
    __shared__ int s_lo[EDT_NB], s_hi[EDT_NB], s_prev[EDT_NB], s_next[EDT_NB];
    __shared__ int s_wred[2][EDT_NW];
    const int r = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int Bw = (W + EDT_NB - 1) / EDT_NB;
    uint16_t* gs = edt_sh;                                   // g by (band position, band)
    uint8_t* st = (uint8_t*)(edt_sh + (size_t)Bw * EDT_LSB);  // hull stacks: band positions
    uint16_t* own = (uint16_t*)((char*)st + (((size_t)Bw * EDT_LSB + 15) & ~(size_t)15));
    const int c = r / EDT_BITS, b = r - c * EDT_BITS;
    {
        const unsigned long long* wr = bits + (int64_t)c * W;
        const int2* abr = ab + (int64_t)c * W;
        int l = tid / Bw, k = tid - l * Bw;  // column q = tid
        for (int q = tid; q < W; q += EDT_NB) {
            gs[k * EDT_LSB + l] = (uint16_t)edt_col_dist(__ldg(wr + q), __ldg(abr + q), r, b);
            k += EDT_NB;
            while (k >= Bw) {
                k -= Bw;
                l++;
            }
        }
        for (int i = tid; i < W; i += EDT_NB) own[i] = 0;
    }
    __syncthreads();
    auto site_g = [&](int l, int k) -> int { return gs[k * EDT_LSB + l]; };
    // 1. hull of the own band
    const int a = tid * Bw;
    const int bl = max(0, min(Bw, W - a));
    int len = 0;
    int ku = 0, kv = 0;
    long long cu = 0, cv = 0;
    for (int k = 0; k < bl; k++) {
        const int gq = site_g(tid, k);
        if (gq == 0xFFFF) continue;
        const long long cq = edt_lift(a + k, gq);
        while (len >= 2 && !edt_keep(ku, cu, kv, cv, k, cq)) {
            len--;
            kv = ku;
            cv = cu;
            if (len >= 2) {
                ku = st[(len - 2) * EDT_LSB + tid];
                cu = edt_lift(a + ku, site_g(tid, ku));
            }
        }
        st[len * EDT_LSB + tid] = (uint8_t)k;
        len++;
        ku = kv;
        cu = cv;
        kv = k;
        cv = cq;
    }
    s_lo[tid] = 0;
    s_hi[tid] = len;
    __syncthreads();
    // 2. bridge merges of the hulls of band groups [b0, b0 + h) and [b0 + h, b0 + 2h)
    for (int h = 1; h < EDT_NB; h <<= 1) {
        if ((tid & (2 * h - 1)) == 0) {
            const int b0 = tid, e = tid + 2 * h;
            int la = b0 + h - 1, lb = b0 + h;
            while (la >= b0 && s_lo[la] == s_hi[la]) la--;
            while (lb < e && s_lo[lb] == s_hi[lb]) lb++;
            if (la >= b0 && lb < e) {
                int pa = s_hi[la] - 1, pb = s_lo[lb];
                int ka = st[pa * EDT_LSB + la], kb = st[pb * EDT_LSB + lb];
                int qa = la * Bw + ka, qb = lb * Bw + kb;
                long long ca = edt_lift(qa, site_g(la, ka)), cb = edt_lift(qb, site_g(lb, kb));
                for (bool changed = true; changed;) {
                    changed = false;
                    for (;;) {  // drop the left end point while it is not below chord(pred, B)
                        int lp = la, pp = pa - 1;
                        if (pp < s_lo[la]) {
                            lp = la - 1;
                            while (lp >= b0 && s_lo[lp] == s_hi[lp]) lp--;
                            if (lp < b0) break;
                            pp = s_hi[lp] - 1;
                        }
                        const int kp = st[pp * EDT_LSB + lp], qp = lp * Bw + kp;
                        const long long cp = edt_lift(qp, site_g(lp, kp));
                        if (edt_keep(qp, cp, qa, ca, qb, cb)) break;
                        s_hi[la] = pa;
                        la = lp;
                        pa = pp;
                        qa = qp;
                        ca = cp;
                        changed = true;
                    }
                    for (;;) {  // drop the right end point while it is not below chord(A, succ)
                        int ln = lb, pn = pb + 1;
                        if (pn >= s_hi[lb]) {
                            ln = lb + 1;
                            while (ln < e && s_lo[ln] == s_hi[ln]) ln++;
                            if (ln >= e) break;
                            pn = s_lo[ln];
                        }
                        const int kn = st[pn * EDT_LSB + ln], qn = ln * Bw + kn;
                        const long long cn = edt_lift(qn, site_g(ln, kn));
                        if (edt_keep(qa, ca, qb, cb, qn, cn)) break;
                        s_lo[lb] = pb + 1;
                        lb = ln;
                        pb = pn;
                        qb = qn;
                        cb = cn;
                        changed = true;
                    }
                }
            }
        }
        __syncthreads();
    }
    // live bands: the nearest non-empty band before (s_prev) and after (s_next) each band
    const bool alive = s_lo[tid] < s_hi[tid];
    {
        const int pv = edt_warp_max_scan(alive ? tid : -1, lane);            // last live <= tid
        int nx = alive ? -tid : -EDT_NB;                                     // first live >= tid,
        for (int off = 1; off < 32; off <<= 1) {                             // as a max of -index
            const int y = __shfl_down_sync(0xffffffffu, nx, off);
            if (lane + off < 32) nx = max(nx, y);
        }
        if (lane == 31) s_wred[0][wid] = pv;
        if (lane == 0) s_wred[1][wid] = nx;
        __syncthreads();
        int before = -1, after = -EDT_NB;
        for (int w2 = 0; w2 < wid; w2++) before = max(before, s_wred[0][w2]);
        for (int w2 = wid + 1; w2 < EDT_NW; w2++) after = max(after, s_wred[1][w2]);
        const int pv_all = max(pv, before), nx_all = max(nx, after);
        // exclusive: the live band strictly before / after tid
        s_prev[tid] = pv_all;
        s_next[tid] = -nx_all;
    }
    __syncthreads();
    double* out = d_out + (int64_t)r * W;
    const int first_live = s_next[0];  // EDT_NB when no band is live
    if (first_live >= EDT_NB) {
        for (int i = tid; i < W; i += EDT_NB) out[i] = __longlong_as_double(0x7ff0000000000000LL);
        return;
    }
    // 3. start pixel of every surviving vertex; a vertex with a non-empty range [s, s_next)
    // inside the row writes its column at own[s]
    if (alive) {
        const int lp = tid > 0 ? s_prev[tid - 1] : -1;
        int qu = -1;
        long long cu2 = 0;
        if (lp >= 0) {
            const int kp = st[(s_hi[lp] - 1) * EDT_LSB + lp];
            qu = lp * Bw + kp;
            cu2 = edt_lift(qu, site_g(lp, kp));
        }
        int qv = tid * Bw + st[s_lo[tid] * EDT_LSB + tid];
        long long cv2 = edt_lift(qv, site_g(tid, qv - tid * Bw));
        int sv = qu < 0 ? 0 : edt_start(qu, cu2, qv, cv2, W);
        const int ln_band = tid + 1 < EDT_NB ? s_next[tid + 1] : EDT_NB;
        for (int p = s_lo[tid]; p < s_hi[tid]; p++) {
            // successor of entry p: the next entry of this band, or the first of the next live band
            int qn = -1;
            long long cn = 0;
            if (p + 1 < s_hi[tid]) {
                const int kn = st[(p + 1) * EDT_LSB + tid];
                qn = tid * Bw + kn;
                cn = edt_lift(qn, site_g(tid, kn));
            } else if (ln_band < EDT_NB) {
                const int kn = st[s_lo[ln_band] * EDT_LSB + ln_band];
                qn = ln_band * Bw + kn;
                cn = edt_lift(qn, site_g(ln_band, kn));
            }
            const int sn = qn < 0 ? W : edt_start(qv, cv2, qn, cn, W);
            if (sv < sn && sv < W) own[sv] = (uint16_t)qv;
            qv = qn;
            cv2 = cn;
            sv = sn;
        }
    }
    __syncthreads();
    // 4. fill: warp w takes the quarter [w Q, (w + 1) Q) of the row (Q a multiple of 32),
    // seeded with the maximum of own[] over the quarters before it
    const int Q = ((W + EDT_NW - 1) / EDT_NW + 31) & ~31;
    const int i0 = wid * Q, i1 = min(W, i0 + Q);
    {
        int mx = 0;
        for (int i = i0 + lane; i < i1; i += 32) mx = max(mx, (int)own[i]);
        for (int off = 16; off > 0; off >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, off));
        if (lane == 0) s_wred[0][wid] = mx;
    }
    __syncthreads();
    int carry = 0;
    for (int w2 = 0; w2 < wid; w2++) carry = max(carry, s_wred[0][w2]);
    // band of column q: floor(q / Bw) = umulhi(q, ceil(2^32 / Bw)) exactly for q < 2^15
    const unsigned bw_mul = Bw > 1 ? 0xFFFFFFFFu / (unsigned)Bw + 1u : 0u;
    for (int t0 = i0; t0 < i1; t0 += 32) {
        const int i = t0 + lane;
        int q = edt_warp_max_scan(i < i1 ? (int)own[i] : 0, lane);
        q = max(q, carry);
        carry = __shfl_sync(0xffffffffu, q, 31);
        if (i < i1) {
            const int l = Bw > 1 ? (int)__umulhi((unsigned)q, bw_mul) : q, k = q - l * Bw;
            const int gq = site_g(l, k);
            const long long d2 = (long long)(i - q) * (i - q) + (long long)gq * gq;
            out[i] = d2 < T ? dtab[d2] : pixel * sqrt((double)d2);
        }
    }
}

size_t edt_env_smem(int W) {
    const size_t Bw = (size_t)((W + EDT_NB - 1) / EDT_NB);
    return sizeof(uint16_t) * Bw * EDT_LSB + ((Bw * EDT_LSB + 15) & ~(size_t)15) +
           sizeof(uint16_t) * (size_t)((W + 31) / 32 * 32);
}

// d = pixel * sqrt(k) for k < T, by the same IEEE FP64 square root and product the row
// pass would take (squared distances are integers), so a table hit returns the same bits.
__global__ void edt_dist_table_kernel(double* tab, int T, double pixel) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < T) tab[k] = pixel * sqrt((double)k);
}

// Workspace of the banded path: feature words, chunk summaries, chunk neighbours, square
// roots.
struct EdtEnvLayout {
    size_t bits, summ, ab, sq, total;
};

EdtEnvLayout edt_env_layout(int32_t W, int32_t H) {
    const size_t nchunk = (size_t)((H + EDT_BITS - 1) / EDT_BITS);
    auto al = [](size_t x) { return (x + 255) / 256 * 256; };
    EdtEnvLayout L;
    L.bits = 0;
    L.summ = L.bits + al(nchunk * W * sizeof(unsigned long long));
    L.ab = L.summ + al(nchunk * W * sizeof(int2));
    L.sq = L.ab + al(nchunk * W * sizeof(int2));
    L.total = L.sq + al(sizeof(double) * EDT_SQRT_T);
    return L;
}

bool edt_banded(int32_t W, int32_t H) { return W <= EDT_BAND_MAX_W && H <= EDT_BAND_MAX_H; }

size_t distance_workspace_bytes(int32_t W, int32_t H) {
    if (edt_banded(W, H)) return edt_env_layout(W, H).total;
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    return 2 * plane;
}

// Scratch of the wide-map path (W > EDT_BAND_MAX_W or H > EDT_BAND_MAX_H): plane 0 = g (int32
// per pixel); plane 1 = feature flags (bytes) during the column pass, then the envelope
// stacks of the global-memory row pass.  The chunk summaries of the column pass live in
// d_out, which the row pass overwrites entirely.
cudaError_t launch_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                                double* d_out, void* ws, cudaStream_t st) {
    cudaError_t e;
    if (edt_banded(W, H)) {
        const EdtEnvLayout L = edt_env_layout(W, H);
        char* base = (char*)ws;
        unsigned long long* bits = (unsigned long long*)(base + L.bits);
        int2* summ = (int2*)(base + L.summ);
        int2* ab = (int2*)(base + L.ab);
        double* sqtab = (double*)(base + L.sq);
        const int nchunk = (H + EDT_BITS - 1) / EDT_BITS;
        edt_bits_kernel<<<dim3((unsigned)((W + 127) / 128), (unsigned)nchunk), 128, 0, st>>>(ncc, W, H, bits, summ);
        edt_chunk_scan_kernel<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(summ, W, nchunk, ab);
        edt_dist_table_kernel<<<(unsigned)((EDT_SQRT_T + 255) / 256), 256, 0, st>>>(sqtab, EDT_SQRT_T, pixel);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const size_t smem = edt_env_smem(W);
        e = cudaFuncSetAttribute(edt_row_env_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        edt_row_env_kernel<<<(unsigned)H, EDT_NB, smem, st>>>(bits, ab, W, pixel, d_out, sqtab, EDT_SQRT_T);
        return cudaGetLastError();
    }
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    int32_t* g = (int32_t*)ws;
    int32_t* v = (int32_t*)((char*)ws + plane);
    uint8_t* feat = (uint8_t*)v;
    int2* summ = (int2*)d_out;  // nchunk * W int2 <= W * H doubles
    const int nchunk = (H + EDT_CHUNK - 1) / EDT_CHUNK;
    const int64_t npx = (int64_t)W * H;
    edt_feature_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(ncc, W, H, feat);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 cg((unsigned)((W + 127) / 128), (unsigned)nchunk);
    edt_chunk_kernel<<<cg, 128, 0, st>>>(feat, W, H, summ);
    edt_column_kernel<<<cg, 128, 0, st>>>(feat, summ, W, H, nchunk, g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    edt_row_kernel<<<(unsigned)((H + 63) / 64), 64, 0, st>>>(g, W, H, pixel, v, d_out);
    return cudaGetLastError();
}

}  // namespace ccg
