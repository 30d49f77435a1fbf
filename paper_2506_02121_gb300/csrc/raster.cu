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

struct CrossK {
    const double2* w;
    int64_t rows, nr;
    double x0, sx, y0, sy;
    int W, H;
    int* D;
    float x0f, inv_sxf, y0f, inv_syf;  // FP32 copies for estimates (exactness comes from FP64 checks)
};

constexpr int XS_THREADS = 256;

// One thread per segment finds, in FP32 with a margin that covers its rounding, the pixel
// rows its half-open y-range may contain.  The (segment, candidate row) pairs of a warp
// are then laid out by a warp prefix sum and processed by all 32 lanes together, so the
// exact FP64 work (row test, prefix length settled by the exact orientation predicate)
// runs without divergence however unevenly crossings are spread over segments.
__global__ void __launch_bounds__(XS_THREADS) crossing_scatter_kernel(CrossK K) {
    __shared__ double2 s_a[XS_THREADS], s_b[XS_THREADS];
    __shared__ int s_r0[XS_THREADS], s_excl[XS_THREADS];
    const int lane = threadIdx.x & 31;
    const int wbase = threadIdx.x & ~31;
    const int64_t t = blockIdx.x * (int64_t)XS_THREADS + threadIdx.x;
    const int64_t nseg = (K.rows - 1) * K.nr;
    int r0 = 0, cnt = 0;
    double2 a = make_double2(0.0, 0.0), b = make_double2(0.0, 0.0);
    if (t < nseg) {
        a = K.w[t];
        b = K.w[t + K.nr];
        if (isfinite(a.x) && isfinite(a.y) && isfinite(b.x) && isfinite(b.y) && a.y != b.y) {
            const float lo = (float)fmin(a.y, b.y), hi = (float)fmax(a.y, b.y);
            const float tl = (lo - K.y0f) * K.inv_syf - 0.5f;
            const float th = (hi - K.y0f) * K.inv_syf - 0.5f;
            const float eps = 1e-3f + 1e-6f * ((fabsf(lo) + fabsf(K.y0f)) * fabsf(K.inv_syf) + fabsf(tl) + fabsf(th));
            const float fr0 = fmaxf(ceilf(tl - eps), 0.0f);
            const float fr1 = fminf(floorf(th + eps) + 1.0f, (float)K.H);  // candidates [fr0, fr1)
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
    s_r0[threadIdx.x] = r0;
    s_excl[threadIdx.x] = incl - cnt;
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
        const double2 sa = s_a[j], sb = s_b[j];
        const int64_t r = s_r0[j] + (item - s_excl[j]);
        const bool up = sa.y < sb.y;
        const double ylo = up ? sa.y : sb.y, yhi = up ? sb.y : sa.y;
        const double py = pix(K.y0, K.sy, r);
        if (!(ylo <= py && py < yhi)) continue;  // exact half-open row test
        const int sgn = up ? 1 : -1;
        // prefix length c: the centres with orient(a, b, P) == sgn are those left of the
        // crossing abscissa xc, i.e. with index i < u = (xc - x0)/sx - 0.5, so c = ceil(u).
        // u in FP32 from FP64 differences; its error is at most
        //   (2.4e-7 |x_a - x0| + 5e-7 |x_b - x_a|) / sx + 6e-8 (|u| + 0.5)
        // (each difference rounded once to FP32, |t| <= 1, IEEE division and products); with
        // no centre index within 4x that bound of u the count is settled, else the exact
        // orientation predicate settles it.
        const float sxr = (float)(sa.x - K.x0);
        const float exf = (float)(sb.x - sa.x), eyf = (float)(sb.y - sa.y);
        const float tf = __fdiv_rn((float)(py - sa.y), eyf);
        const float u = __fsub_rn(__fmul_rn(__fadd_rn(sxr, __fmul_rn(exf, tf)), K.inv_sxf), 0.5f);
        const float err = 4.0f * ((4e-7f * (fabsf(sxr) + fabsf(exf))) * K.inv_sxf + 2.4e-7f * fabsf(u) + 1e-6f);
        int64_t c;
        if (isfinite(u) && isfinite(err) && ceilf(u - err) == ceilf(u + err)) {
            c = (int64_t)fminf(fmaxf(ceilf(u), 0.0f), (float)K.W);
        } else {
            float ce = ceilf(u);
            ce = fminf(fmaxf(ce, 0.0f), (float)K.W);
            if (!(ce == ce)) ce = 0.0f;  // NaN guard
            c = (int64_t)ce;
            while (c > 0 && orient_sign(sa.x, sa.y, sb.x, sb.y, pix(K.x0, K.sx, c - 1), py) != sgn) c--;
            while (c < K.W && orient_sign(sa.x, sa.y, sb.x, sb.y, pix(K.x0, K.sx, c), py) == sgn) c++;
        }
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
        K.x0f = (float)x0;
        K.inv_sxf = (float)(1.0 / K.sx);
        K.y0f = (float)y0;
        K.inv_syf = (float)(1.0 / K.sy);
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

// Row pass, one warp per row, exact integer arithmetic.  D(i) = min_q (i - q)^2 + g[q]^2 is
// the lower envelope of the parabolas of the columns with a feature; its owners are the
// vertices of the lower convex hull of the lifted points (q, q^2 + g[q]^2).  Lane l takes
// the band of columns [l Bw, (l + 1) Bw) and builds the hull of its band with a stack; five
// rounds of bridge merges join neighbouring bands (the hull of two column-separated sets
// keeps a prefix of the left hull and a suffix of the right one, found by walking both
// ends until neither end point can be dropped); then the warp fills the row 32 pixels at
// a time, each lane walking the hull forward from the owner of the tile's first pixel.
// Band position k of lane l is stored at [k * EDT_LS + l] (16-bit g values; 8- or 16-bit
// stack entries), so the lanes of a warp stepping through their bands together never share
// a shared-memory bank word they do not also share an address in.
constexpr int EDT_BAND_MAX_W = 32768;
constexpr int EDT_BAND_MAX_H = 65535;  // g < H fits 16 bits, 0xFFFF marks "no feature"
constexpr int EDT_LS = 33;

// g values (16 bits) and hull stacks of band positions (8 bits while a band holds at most
// 256 columns, i.e. W <= 8192, else 16): the smaller stacks let more rows share an SM.
size_t edt_band_smem(int W) {
    const size_t Bw = (size_t)((W + 31) / 32);
    return (sizeof(uint16_t) + (Bw <= 256 ? sizeof(uint8_t) : sizeof(uint16_t))) * Bw * EDT_LS;
}

__device__ __forceinline__ long long edt_lift(int q, int gq) { return (long long)q * q + (long long)gq * gq; }

// Site v (u < v < w in column order) is strictly below the chord u-w of the lifted points,
// i.e. intersection(u, v) < intersection(v, w): its parabola alone is lowest somewhere.
__device__ __forceinline__ bool edt_keep(int u, long long cu, int v, long long cv, int w, long long cw) {
    return (cw - cv) * (long long)(v - u) > (cv - cu) * (long long)(w - v);
}

// sqrt(k) for k < T by the same IEEE FP64 square root the row pass would take, so that a
// table hit returns the same bits (squared distances are integers).
constexpr int EDT_SQRT_T = 65536;
__global__ void edt_sqrt_table_kernel(double* tab, int T) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < T) tab[k] = sqrt((double)k);
}

template <typename ST>
__global__ void __launch_bounds__(32) edt_row_band_kernel(const int32_t* g, int W, double pixel, double* d_out,
                                                          const double* sqtab, int T) {
    extern __shared__ uint16_t edt_sh[];
    __shared__ int s_lo[32], s_hi[32];
    const int r = blockIdx.x, lane = threadIdx.x;
    const int Bw = (W + 31) / 32;
    uint16_t* gs = edt_sh;                          // g by (band position, lane)
    ST* st = (ST*)(edt_sh + (size_t)Bw * EDT_LS);   // hull stacks: band positions
    const int32_t* gr = g + (int64_t)r * W;
    {
        int l = lane / Bw, k = lane - l * Bw;  // column q = lane
        for (int q = lane; q < W; q += 32) {
            const int32_t v = gr[q];
            gs[k * EDT_LS + l] = v >= 0xFFFF ? (uint16_t)0xFFFF : (uint16_t)v;
            k += 32;
            while (k >= Bw) {
                k -= Bw;
                l++;
            }
        }
    }
    __syncwarp();
    auto site_g = [&](int l, int k) -> int { return gs[k * EDT_LS + l]; };
    // 1. hull of the own band
    const int a = lane * Bw;
    const int bl = max(0, min(Bw, W - a));
    int len = 0;
    int ku = 0, kv = 0;             // band positions of the two top stack entries
    long long cu = 0, cv = 0;       // and their lifted values
    for (int k = 0; k < bl; k++) {
        const int gq = site_g(lane, k);
        if (gq == 0xFFFF) continue;
        const long long cq = edt_lift(a + k, gq);
        while (len >= 2 && !edt_keep(ku, cu, kv, cv, k, cq)) {
            len--;
            kv = ku;
            cv = cu;
            if (len >= 2) {
                ku = st[(len - 2) * EDT_LS + lane];
                cu = edt_lift(a + ku, site_g(lane, ku));
            }
        }
        st[len * EDT_LS + lane] = (ST)k;
        len++;
        ku = kv;
        cu = cv;
        kv = k;
        cv = cq;
    }
    s_lo[lane] = 0;
    s_hi[lane] = len;
    __syncwarp();
    // 2. bridge merges of the hulls of lane groups [b, b + h) and [b + h, b + 2h)
    for (int h = 1; h < 32; h <<= 1) {
        if ((lane & (2 * h - 1)) == 0) {
            const int b = lane, e = lane + 2 * h;
            int la = b + h - 1, lb = b + h;
            while (la >= b && s_lo[la] == s_hi[la]) la--;
            while (lb < e && s_lo[lb] == s_hi[lb]) lb++;
            if (la >= b && lb < e) {
                int pa = s_hi[la] - 1, pb = s_lo[lb];
                int ka = st[pa * EDT_LS + la], kb = st[pb * EDT_LS + lb];
                int qa = la * Bw + ka, qb = lb * Bw + kb;
                long long ca = edt_lift(qa, site_g(la, ka)), cb = edt_lift(qb, site_g(lb, kb));
                for (bool changed = true; changed;) {
                    changed = false;
                    for (;;) {  // drop the left end point while it is not below chord(pred, B)
                        int lp = la, pp = pa - 1;
                        if (pp < s_lo[la]) {
                            lp = la - 1;
                            while (lp >= b && s_lo[lp] == s_hi[lp]) lp--;
                            if (lp < b) break;
                            pp = s_hi[lp] - 1;
                        }
                        const int kp = st[pp * EDT_LS + lp], qp = lp * Bw + kp;
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
                        const int kn = st[pn * EDT_LS + ln], qn = ln * Bw + kn;
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
        __syncwarp();
    }
    // 3. fill, 32 pixels at a time
    double* out = d_out + (int64_t)r * W;
    const unsigned live = __ballot_sync(0xffffffffu, s_lo[lane] < s_hi[lane]);
    if (live == 0) {
        for (int i = lane; i < W; i += 32) out[i] = __longlong_as_double(0x7ff0000000000000LL);
        return;
    }
    int cl = __ffs(live) - 1, cp = s_lo[cl];
    for (int t0 = 0; t0 < W; t0 += 32) {
        const int i = t0 + lane;
        int L = cl, p = cp;
        int k = st[p * EDT_LS + L];
        int q = L * Bw + k, gq = site_g(L, k);
        long long cq = edt_lift(q, gq);
        if (i < W) {
            for (;;) {
                int L2 = L, p2 = p + 1;
                if (p2 >= s_hi[L]) {
                    const unsigned rest = live & ~((2u << L) - 1u);
                    if (rest == 0) break;
                    L2 = __ffs(rest) - 1;
                    p2 = s_lo[L2];
                }
                const int k2 = st[p2 * EDT_LS + L2];
                const int q2 = L2 * Bw + k2, g2 = site_g(L2, k2);
                const long long c2 = edt_lift(q2, g2);
                if (c2 - cq > 2LL * i * (q2 - q)) break;  // the next owner starts right of i
                L = L2;
                p = p2;
                q = q2;
                gq = g2;
                cq = c2;
            }
            const long long d2 = (long long)(i - q) * (i - q) + (long long)gq * gq;
            out[i] = pixel * (d2 < T ? sqtab[d2] : sqrt((double)d2));
        }
        const int last = min(31, W - 1 - t0);
        cl = __shfl_sync(0xffffffffu, L, last);
        cp = __shfl_sync(0xffffffffu, p, last);
    }
}

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

size_t distance_workspace_bytes(int32_t W, int32_t H) {
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    return 2 * plane;
}

// Scratch: plane 0 = g (int32 per pixel); plane 1 = feature flags (bytes) during the
// column pass, then the square-root table of the band row pass (or the envelope stacks of
// the global-memory row pass).  The chunk summaries of the column pass live in d_out, which
// the row pass overwrites entirely.
cudaError_t launch_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel,
                                double* d_out, void* ws, cudaStream_t st) {
    const size_t plane = ((size_t)W * H * sizeof(int32_t) + 255) / 256 * 256;
    int32_t* g = (int32_t*)ws;
    int32_t* v = (int32_t*)((char*)ws + plane);
    uint8_t* feat = (uint8_t*)v;
    int2* summ = (int2*)d_out;  // nchunk * W int2 <= W * H doubles
    const int nchunk = (H + EDT_CHUNK - 1) / EDT_CHUNK;
    const int64_t npx = (int64_t)W * H;
    edt_feature_kernel<<<(unsigned)((npx + 255) / 256), 256, 0, st>>>(ncc, W, H, feat);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 cg((unsigned)((W + 127) / 128), (unsigned)nchunk);
    edt_chunk_kernel<<<cg, 128, 0, st>>>(feat, W, H, summ);
    edt_column_kernel<<<cg, 128, 0, st>>>(feat, summ, W, H, nchunk, g);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (W <= EDT_BAND_MAX_W && H <= EDT_BAND_MAX_H) {
        // square-root table in plane 1 (the row pass needs no stacks there)
        const int T = (int)std::min<size_t>((size_t)EDT_SQRT_T, plane / sizeof(double));
        double* sqtab = (double*)v;
        edt_sqrt_table_kernel<<<(unsigned)((T + 255) / 256), 256, 0, st>>>(sqtab, T);
        const size_t smem = edt_band_smem(W);
        if ((W + 31) / 32 <= 256) {
            e = cudaFuncSetAttribute(edt_row_band_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            edt_row_band_kernel<uint8_t><<<(unsigned)H, 32, smem, st>>>(g, W, pixel, d_out, sqtab, T);
        } else {
            e = cudaFuncSetAttribute(edt_row_band_kernel<uint16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem);
            if (e != cudaSuccess) return e;
            edt_row_band_kernel<uint16_t><<<(unsigned)H, 32, smem, st>>>(g, W, pixel, d_out, sqtab, T);
        }
    } else {
        edt_row_kernel<<<(unsigned)((H + 63) / 64), 64, 0, st>>>(g, W, H, pixel, v, d_out);
    }
    return cudaGetLastError();
}

}  // namespace ccg
