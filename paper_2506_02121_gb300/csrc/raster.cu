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

// Smallest r in [0, cnt] with pix(r) >= v (cnt if none); pix is non-decreasing in r.
__device__ __forceinline__ int64_t first_at_or_above(double lo, double step, int64_t cnt, double v) {
    double e = ceil((v - lo) / step - 0.5);
    e = fmin(fmax(e, 0.0), (double)cnt);
    int64_t r = (int64_t)e;
    while (r > 0 && pix(lo, step, r - 1) >= v) r--;
    while (r < cnt && pix(lo, step, r) < v) r++;
    return r;
}

struct CrossK {
    const double2* w;
    int64_t rows, nr;
    double x0, sx, y0, sy;
    int W, H;
    int* D;
};

__global__ void __launch_bounds__(256) crossing_scatter_kernel(CrossK K) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (K.rows - 1) * K.nr) return;
    const double2 a = K.w[t], b = K.w[t + K.nr];
    if (!(isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y))) return;
    if (a.y == b.y) return;
    const bool up = a.y < b.y;
    const double lo = up ? a.y : b.y, hi = up ? b.y : a.y;
    const int64_t r0 = first_at_or_above(K.y0, K.sy, K.H, lo);
    const int64_t r1 = first_at_or_above(K.y0, K.sy, K.H, hi);
    const int sgn = up ? 1 : -1;
    const double ex = b.x - a.x, ey = b.y - a.y;
    for (int64_t r = r0; r < r1; r++) {
        const double py = pix(K.y0, K.sy, r);
        // prefix length c: centres with orient(a, b, P) == sgn
        const double xc = a.x + ex * ((py - a.y) / ey);
        double ce = ceil((xc - K.x0) / K.sx - 0.5);
        ce = fmin(fmax(ce, 0.0), (double)K.W);
        int64_t c = (int64_t)ce;
        while (c > 0 && orient_sign(a.x, a.y, b.x, b.y, pix(K.x0, K.sx, c - 1), py) != sgn) c--;
        while (c < K.W && orient_sign(a.x, a.y, b.x, b.y, pix(K.x0, K.sx, c), py) == sgn) c++;
        if (c > 0) atomicAdd(&K.D[r * K.W + (c - 1)], sgn);
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
        const int64_t segs = (rows - 1) * nr;
        crossing_scatter_kernel<<<(unsigned)((segs + 255) / 256), 256, 0, st>>>(K);
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

// g[r][i] = |r - nearest feature row in column i| (DIST_INF if the column has none).
__global__ void edt_column_kernel(const int32_t* ncc, int W, int H, int32_t* g) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= W) return;
    int last = -1;
    for (int r = 0; r < H; r++) {
        if (feature_at(ncc, W, H, r, i)) last = r;
        g[(int64_t)r * W + i] = last < 0 ? DIST_INF : r - last;
    }
    int next = -1;
    for (int r = H - 1; r >= 0; r--) {
        const int64_t o = (int64_t)r * W + i;
        const int gv = g[o];
        if (gv == 0) next = r;
        if (next >= 0 && next - r < gv) g[o] = next - r;
    }
}

// Row pass: lower envelope of parabolas q -> (i - q)^2 + g[q]^2 over the finite g[q].
__global__ void edt_row_kernel(const int32_t* g, int W, int H, double pixel, int32_t* vstack,
                               double* d_out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= H) return;
    const int32_t* f = g + (int64_t)r * W;
    int32_t* v = vstack + (int64_t)r * W;
    double* out = d_out + (int64_t)r * W;
    // intersection abscissa of parabolas p < q: num / den, den = 2 (q - p) > 0
    auto key = [&](int q) -> long long { return (long long)f[q] * f[q] + (long long)q * q; };
    int k = -1;
    for (int q = 0; q < W; q++) {
        if (f[q] >= DIST_INF) continue;
        const long long fq = key(q);
        while (k >= 1) {
            const int p = v[k], pp = v[k - 1];
            const long long n1 = fq - key(p), d1 = 2LL * (q - p);        // s(p, q)
            const long long n2 = key(p) - key(pp), d2 = 2LL * (p - pp);   // s(pp, p)
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
            const long long n = key(q) - key(p), d = 2LL * (q - p);
            if (n < (long long)i * d) j++;
            else break;
        }
        const int p = v[j];
        const long long d2 = (long long)(i - p) * (i - p) + (long long)f[p] * f[p];
        out[i] = pixel * sqrt((double)d2);
    }
}

size_t distance_workspace_bytes(int32_t W, int32_t H) {
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    return 2 * plane;
}

cudaError_t launch_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                                double* d_out, void* ws, cudaStream_t st) {
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    int32_t* g = (int32_t*)ws;
    int32_t* v = (int32_t*)((char*)ws + plane);
    edt_column_kernel<<<(unsigned)((W + 127) / 128), 128, 0, st>>>(ncc, W, H, g);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    edt_row_kernel<<<(unsigned)((H + 63) / 64), 64, 0, st>>>(g, W, H, pixel, v, d_out);
    return cudaGetLastError();
}

}  // namespace ccg
