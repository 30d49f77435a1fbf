// Critical-curve tracer: simultaneous Aberth-Ehrlich iteration on the roots of
// P(z) = F(z, phi) prod_i (z - z_i)^2 (Sec. 3.2), grown along the phi grid from the centre
// of each phi sub-range toward both of its ends (Sec. 4.3), each row warm-started from its
// neighbour (Sec. 3.2).
//
// One CTA owns one sub-range ("subchain") for the whole launch: no grid-wide barrier, no
// host round trip per iteration.  Inside the CTA every Aberth iteration is a Jacobi sweep
// over the still-active roots of the (one or two) rows being solved:
//   - active roots are compacted into a list; g lanes (power of two, <= 32) share one root
//     so that a handful of late roots still keep every lane busy; the g partial sums are
//     combined by a butterfly of warp shuffles (fixed order: deterministic results);
//   - star records are staged in shared memory once (resident) or per tile, the current
//     roots of both rows are streamed through shared memory in tiles;
//   - per root the star sums  C = sum 1/d,  A = sum m/d^2,  B = sum m/d^3  and the root
//     sum  D = sum_{r != k} 1/(z_k - z_r)  give  F = gamma + A - (1-kappa_s) e^{-i phi},
//     F' = -2B,  P'/P = F'/F + 2C  and the update  z_k -= 1/(P'/P - D)  (Sec. 3.2).
// Two arithmetics: FP32 (the mixed form; its result is polished afterwards) and FP64 (the
// plain form with the |dz| < tol stop rule of Sec. 3.2).
#include <algorithm>
#include <float.h>
#include <string.h>

#include "cc_internal.h"

namespace ccg {

template <typename T>
struct CT;
template <>
struct CT<float> {
    using C = float2;
    using Star = float4;
    static constexpr int TS = 4096;  // stars per shared-memory tile
};
template <>
struct CT<double> {
    using C = double2;
    using Star = StarD;
    static constexpr int TS = 2048;
};
constexpr int TR = 1024;  // roots per direction per shared-memory tile

template <typename T>
struct Acc {
    T Cx, Cy, Ax, Ay, Bx, By, Dx, Dy;
    T Am;  // sum m/|d|^2 = sum |m/d^2|: scale of the rounding noise of F
};

__device__ __forceinline__ float recip(float x) { return rcp_approx(x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
// Per-update divisions: the FP32 tracer is polished afterwards, so the hardware reciprocal
// (about 1 ulp) is enough there; the FP64 tracer divides exactly.
__device__ __forceinline__ float qdiv(float a, float b) { return a * rcp_approx(b); }
__device__ __forceinline__ float qsqrt(float a) {
    float r;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
__device__ __forceinline__ double qsqrt(double a) { return sqrt(a); }
__device__ __forceinline__ double qdiv(double a, double b) { return a / b; }

// One star: d = z - z_i, u = 1/d = conj(d)/|d|^2; C += u, A += m u^2, B += m u^3.
template <typename T, typename S>
__device__ __forceinline__ void acc_star(T zx, T zy, const S& s, Acc<T>& a) {
    T dx = zx - (T)s.x, dy = zy - (T)s.y;
    T r2 = fma(dx, dx, dy * dy);
    T inv = recip(r2);
    T ux = dx * inv, uy = -dy * inv;
    a.Cx += ux;
    a.Cy += uy;
    T tx = fma(ux, ux, -uy * uy);
    T ty = (ux + ux) * uy;
    T mx = (T)s.z * tx, my = (T)s.z * ty;
    a.Ax += mx;
    a.Ay += my;
    a.Am = fma((T)s.z, inv, a.Am);
    a.Bx = fma(mx, ux, fma(-my, uy, a.Bx));
    a.By = fma(mx, uy, fma(my, ux, a.By));
}

// One other root: D += 1/(z_k - z_r); the root itself (|d| == 0) contributes nothing.
template <typename T, typename C>
__device__ __forceinline__ void acc_root(T zx, T zy, const C& r, Acc<T>& a) {
    T dx = zx - r.x, dy = zy - r.y;
    T r2 = fma(dx, dx, dy * dy);
    T inv = r2 > (T)0 ? recip(r2) : (T)0;
    a.Dx = fma(dx, inv, a.Dx);
    a.Dy = fma(-dy, inv, a.Dy);
}

template <typename T>
__device__ __forceinline__ T shfl_x(T v, int off) {
    return __shfl_xor_sync(0xffffffffu, v, off);
}

struct TK {
    const void* stars;
    const SmoothPoly* poly;  // rectangular field: smooth-sheet polynomial; nullptr for the disc
    int n, nr;
    double kappa_s, gamma;
    int64_t m;
    int S;
    const double2* phase;
    void* zrows;
    void* seam;
    int32_t* iters;
    char* work;
    size_t work_stride;
    DevReport* rep;
    double tol_abs, mu_max;
    int max_iter_cold, max_iter_warm, predictor;
    int root_refresh;  // FP32 warm rows: exact far part of the root sum every root_refresh rows (< 2: every sweep)
    int near_cap;      // rows of up to near_cap roots keep the split's ordered positions in shared memory
    int near_ext;      // ... and also its far parts, refresh positions and cells (the host sized the shared
                       // memory for them)
    // FP32 far-field tables (tfmm.ok == 0: every star summed directly)
    TfmmParams tfmm;
    const TCell* tcells;
    const int* tnear;
    const float4* tcoeff;
    float4* ext;  // FP32 form: this CTA's extent of the points written to zrows (may be null)
};

template <typename T>
struct Ctx {
    using C = typename CT<T>::C;
    using Star = typename CT<T>::Star;
    const TK* k;
    Star* s_star;
    C* s_root;  // [2][TR]
    C *cur, *nxt, *prev, *prev2;  // prev, prev2: the two rows before cur on this direction
    float* dprev;
    int *conv, *it, *act;
    bool resident;
    int lo, hi;       // this CTA's slice [lo, hi) of each direction's roots (all of them unless a
                      // cluster of CTAs shares the sub-range)
    int* s_red;       // cluster reductions: [2][4] shared-memory slots, double-buffered
    int* s_tot;       // [4] reduced totals
    int* red_parity;
    unsigned long long* n_terms;  // this thread's work counters (registers of the caller)
    unsigned long long* n_far;
    unsigned long long* n_root;
    // near/far split of the root sum (per direction d: [d nr, d nr + nr) of each array).  A
    // root's code is d nr + its place in cell order (the refresh's order); arrays indexed by
    // code are read in that order by a light sweep's first pass (neighbouring threads,
    // neighbouring entries)
    float2* nfar;   // [code]: far part of the root's sum, captured at the last refresh row
    float2* npos;   // [code]: current positions
    int* nkey;      // [key]: refresh cell (scratch of the cell building)
    int* ncell;     // [code]: refresh cell as (cy << 16) | cx
    int* nord;      // [code]: key d nr + k (row-major cells, index order within a cell)
    int* ncst;      // [d (ncm + 1) + c]: first entry of cell c in nord
    int* nfill;     // [d ncm + c]: scatter counters
    float2* nref;   // [code]: position at the last refresh
    float2* npred;  // this row's predicted positions
    int* nrank;     // [key]: position of the root within its direction's part of nord
    int* act2;      // second active list (split sweeps alternate between act and act2)
    int ncm;        // cells available per direction
    int* s_ngrid;   // shared: nbx, nby of direction d at [2 d], [2 d + 1]
    float* s_nlim2; // shared: squared displacement limit (h / 4)^2 of direction d
    int* s_nesc;    // shared: an iterate left its limit during this row
};

// One other root in FP32, without a branch: D += 1/(z_k - z_r).  The tiny constant added
// to |d|^2 turns the root's own term into 0 * 1e30 = 0 and leaves every other term as it
// was (two roots that FP32 can tell apart at |z| >= 1e-3 have |d|^2 >= 1e-20).
__device__ __forceinline__ void acc_root_f(float zx, float zy, float rx, float ry, float& Dx, float& Dy) {
    const float dx = zx - rx, dy = zy - ry;
    const float inv = rcp_approx(fmaf(dx, dx, fmaf(dy, dy, 1e-30f)));
    Dx = fmaf(dx, inv, Dx);
    Dy = fmaf(-dy, inv, Dy);
}

// Packed FP32 pairs (two IEEE FP32 operations per instruction, round to nearest).
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2_pack(float a, float b) {
    f2p r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2p v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p f2_sub(f2p a, f2p b) {
    f2p r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2p f2_fma(f2p a, f2p b, f2p c) {
    f2p r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Two other roots at once, (x1, x2), (y1, y2): D += 1/(z - z_1) + 1/(z - z_2), kept as
// packed partial sums Dx2 = (.., ..), Dy2 accumulating +dy/|d|^2 (D_y = -(sum)).
__device__ __forceinline__ void acc_root_f2(f2p zxx, f2p zyy, f2p px, f2p py, f2p& Dx2, f2p& Dy2) {
    const f2p eps = f2_pack(1e-30f, 1e-30f);
    const f2p dx = f2_sub(zxx, px), dy = f2_sub(zyy, py);
    const f2p r2 = f2_fma(dx, dx, f2_fma(dy, dy, eps));
    float ra, rb;
    f2_unpack(r2, ra, rb);
    const f2p inv = f2_pack(rcp_approx(ra), rcp_approx(rb));
    Dx2 = f2_fma(dx, inv, Dx2);
    Dy2 = f2_fma(dy, inv, Dy2);
}

// 16-byte load from shared memory (two FP32 roots); a warp that reads one address gets it
// by broadcast.
__device__ __forceinline__ float4 lds_f4(unsigned addr) {
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "r"(addr)
                 : "memory");
    return v;
}

// The cell's far-field series at t = z - centre, by Horner on packed pairs: the table holds
// per k (U_k re, S1'_k re, U_k im, S1'_k im), U the expansion of sum_far 1/(z - z_i) and S1' =
// sum k L_k t^(k-1) that of the derivative of S1 = sum_far m_i/(z - z_i) (S1'_13 = 0).  One
// chain gives (U, S1') and its derivative chain S1''; out: U, S1' and S1''/2.
__device__ __forceinline__ void far_eval(const float4* L, float tx, float ty, float& Ux, float& Uy, float& Sx,
                                         float& Sy, float& Hx, float& Hy) {
    const f2p TX = f2_pack(tx, tx), TY = f2_pack(ty, ty), NTY = f2_pack(-ty, -ty);
    const float4 top = L[TFMM_P - 1];
    f2p X = f2_pack(top.x, top.y), Y = f2_pack(top.z, top.w);
    f2p DX = f2_pack(0.f, 0.f), DY = DX;
#pragma unroll
    for (int kk = TFMM_P - 2; kk >= 0; kk--) {
        const float4 c4 = L[kk];
        const f2p nDX = f2_fma(DX, TX, f2_fma(DY, NTY, X));
        const f2p nDY = f2_fma(DX, TY, f2_fma(DY, TX, Y));
        const f2p nX = f2_fma(X, TX, f2_fma(Y, NTY, f2_pack(c4.x, c4.y)));
        const f2p nY = f2_fma(X, TY, f2_fma(Y, TX, f2_pack(c4.z, c4.w)));
        DX = nDX;
        DY = nDY;
        X = nX;
        Y = nY;
    }
    float dux, duy;
    f2_unpack(X, Ux, Sx);
    f2_unpack(Y, Uy, Sy);
    f2_unpack(DX, dux, Hx);
    f2_unpack(DY, duy, Hy);
    Hx *= 0.5f;
    Hy *= 0.5f;
}

// Cell of z in the FP32 far-field grid, or -1 when every star is summed directly (FP64
// tracer, no grid, z outside it, or a cell with too many near stars).
template <typename T>
__device__ __forceinline__ int far_cell(const TK& K, T zx, T zy) {
    if (sizeof(T) != 4 || !K.tfmm.ok) return -1;
    const float fx = floorf(((float)zx - K.tfmm.x0) * K.tfmm.inv_b);
    const float fy = floorf(((float)zy - K.tfmm.y0) * K.tfmm.inv_b);
    if (!(fx >= 0.f && fy >= 0.f && fx < (float)K.tfmm.nbx && fy < (float)K.tfmm.nby)) return -1;
    const int c = (int)fy * K.tfmm.nbx + (int)fx;
    return K.tcells[c].near_cnt >= 0 ? c : -1;
}

// Star terms of a root in a far-field cell: its near stars (lanes lane, lane + g, ...) and,
// on lane 0, the cell's local expansions (far_eval): U(t) -> C, A = -S1'(t), B = S1''(t)/2.
template <typename T>
__device__ __forceinline__ void cell_part(const Ctx<T>& x, int cell, T zx, T zy, int lane, int g, Acc<T>& acc) {
    const TK& K = *x.k;
    const TCell tc = K.tcells[cell];
    const int* nl = K.tnear + (size_t)cell * TFMM_NEAR_MAX;
    const typename CT<T>::Star* gs = (const typename CT<T>::Star*)K.stars;
#pragma unroll 4
    for (int q = lane; q < tc.near_cnt; q += g) {
        const int j = nl[q];
        acc_star(zx, zy, x.resident ? x.s_star[j] : gs[j], acc);
    }
    if (lane != 0) return;
    float ux, uy, sx, sy, hx, hy;
    far_eval(K.tcoeff + (size_t)cell * TFMM_P, (float)zx - tc.cx, (float)zy - tc.cy, ux, uy, sx, sy, hx, hy);
    acc.Cx += (T)ux;
    acc.Cy += (T)uy;
    acc.Ax -= (T)sx;
    acc.Ay -= (T)sy;
    acc.Bx += (T)hx;
    acc.By += (T)hy;
    acc.Am += (T)tc.far_m_d2;
}

// Aberth update of one root from its sums (Eq. 9 with F, F' of Eqs. 6-7), and the stop rule.
template <typename T>
__device__ __forceinline__ typename CT<T>::C finish_root(const Ctx<T>& x, int key, typename CT<T>::C z,
                                                         const Acc<T>& acc, T cph, T sph, int* s_maxit) {
    using C = typename CT<T>::C;
    const TK& K = *x.k;
    const T oms = (T)(1.0 - K.kappa_s);
    const T gam = (T)K.gamma;
    // F = gamma + A - Q(z) - (1 - kappa_s) e^{-i phi},  F' = -2 B - Q'(z)  (Q = 0 for the disc)
    T Fx = gam + acc.Ax - oms * cph;
    T Fy = acc.Ay + oms * sph;
    T dFx = (T)-2 * acc.Bx, dFy = (T)-2 * acc.By;
    T qa = 0, sca = 1;  // |common scale| of F, F' (FP32 rectangle far out: see poly_eval_scaled)
    if (K.poly) {
        if constexpr (sizeof(T) == 4) {
            float Qx, Qy, Q1x, Q1y, scx, scy;
            poly_eval_scaled(K.poly, z.x, z.y, Qx, Qy, Q1x, Q1y, scx, scy, qa);
            const T fx = Fx * scx - Fy * scy, fy = Fx * scy + Fy * scx;
            const T gx = dFx * scx - dFy * scy, gy = dFx * scy + dFy * scx;
            Fx = fx - Qx;
            Fy = fy - Qy;
            dFx = gx - Q1x;
            dFy = gy - Q1y;
            sca = sqrtf(scx * scx + scy * scy);
        } else {
            T Qx, Qy, Q1x, Q1y, Q2x, Q2y;
            poly_eval<T>(K.poly, z.x, z.y, Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa);
            Fx -= Qx;
            Fy -= Qy;
            dFx -= Q1x;
            dFy -= Q1y;
        }
    }
    C zn = z;
    T ad = 0;
    T q2 = (T)3.0e38;  // |F'/F|^2: the inverse square of the Newton step (huge at F = 0)
    if (Fx != (T)0 || Fy != (T)0) {
        const T fden = Fx * Fx + Fy * Fy;
        const T qx = qdiv(dFx * Fx + dFy * Fy, fden);
        const T qy = qdiv(dFy * Fx - dFx * Fy, fden);
        q2 = qx * qx + qy * qy;
        const T px = qx + (T)2 * acc.Cx - acc.Dx;
        const T py = qy + (T)2 * acc.Cy - acc.Dy;
        const T pden = px * px + py * py;
        const T delx = qdiv(px, pden), dely = qdiv(-py, pden);
        zn.x = z.x - delx;
        zn.y = z.y - dely;
        ad = qsqrt(delx * delx + dely * dely);
    }
    const int its = x.it[key] + 1;
    x.it[key] = its;
    atomicMax(s_maxit, its);
    bool done;
    if (sizeof(T) == 4) {
        // FP32: freeze at the absolute tolerance or at the rounding floor of this root: a
        // few ulp of |z|, or the FP32 noise of F (~eps sum |m/d^2|) divided by |F'|; or when
        // the corrections stop shrinking within a few times that floor.
        const T sc = (T)1 + qsqrt(z.x * z.x + z.y * z.y);
        const T fpa = qsqrt(dFx * dFx + dFy * dFy);
        const T noise = (T)(4.0 * FLT_EPSILON) * (sca * (acc.Am + fabs(gam) + oms) + qa);
        T tolz = fmax((T)K.tol_abs, (T)(8.0 * FLT_EPSILON) * sc);
        if (fpa > (T)0) tolz = fmax(tolz, (T)4 * noise * qdiv((T)1, fpa));
        // never looser than 64x the ulp floor: an iterate that runs away where F' vanishes
        // must not count as converged
        tolz = fmin(tolz, (T)(512.0 * FLT_EPSILON) * sc);
        // a non-finite step (ad NaN) never freezes a root: it would poison every root sum.
        // The Newton step |F/F'| itself must also be near the floor: a small Aberth step can
        // come from a large root or star sum rather than from F ~ 0 (an iterate stalled
        // beside another root, or a stale far part of the root sum).
        const T nlim = (T)16 * tolz;
        done = (ad < tolz || (its >= 3 && ad > (T)0.25 * (T)x.dprev[key] && ad < (T)4 * tolz)) &&
               q2 * nlim * nlim > (T)1;
        if (!(ad == ad)) zn = z;
    } else {
        done = ad < (T)K.tol_abs;
        if (!(ad == ad)) zn = z;
        if (!done && K.mu_max > 0 && !K.poly) {
            const T gx = gam + acc.Ax, gy = acc.Ay;
            const T detj = oms * oms - (gx * gx + gy * gy);
            done = fabs((double)detj) * K.mu_max < 1.0;
        }
    }
    x.dprev[key] = (float)ad;
    if (done) x.conv[key] = 1;
    x.nxt[key] = zn;
    return zn;
}

// ----------------------------------------------------------------------------------
// Near/far split of the Aberth root sum on warm rows (FP32 tracer).  The Aberth correction
// sum_{r != k} 1/(z_k - z_r) only shapes the iteration, not its fixed points (F(z_k) = 0 is
// decided by F alone, and every point is then polished by Newton on F and certified), and
// on a warm row the predictor already puts each root within a small fraction of the root
// spacing of its zero.  So at a refresh row the exact sum is split into the roots of the
// 3 x 3 cells around root k (its near set) and the rest (its far part, stored); on the
// following rows the near set is summed exactly at the current positions and the stored far
// part is reused.  A perturbation e of the sum moves an Aberth step delta by about
// e delta^2, far below the FP32 stop threshold once delta is small; the near roots, whose
// repulsion keeps two iterates from settling on one zero, are always exact.  Every position
// used is kept within h/4 of its refresh position (h the cell side): a root and any root
// outside its near set, at least h apart at the refresh, then stay h/2 apart, so an iterate
// can neither settle on a far root's zero nor make the stored part stale by more than that
// motion allows.  A prediction beyond the limit makes its row a refresh row; an iterate
// beyond it has its row solved again with the exact sum in every sweep.
// ----------------------------------------------------------------------------------
// Thread-block clusters: several CTAs share one phi sub-range (each updates a slice of the
// roots and reads all of them); hardware cluster barriers order the sweeps, and per-CTA
// counts are summed through distributed shared memory.
__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ unsigned cluster_size() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}

// All threads of all CTAs of the cluster; global and shared writes before it are visible
// to every thread of the cluster after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ int ld_cluster(const int* local, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(local);
    unsigned ra;
    int v;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(ra) : "memory");
    return v;
}

constexpr int NEAR_PER_CELL = 4;  // roots per cell on average over the bounding box

// Loads of the split's arrays.  W: a thread-block cluster shares one sub-range, and the
// arrays (in the sub-range's work area) are written by other SMs of the cluster between
// cluster barriers: read through L2 (ld.cg), never a stale L1 line.  Otherwise a plain load
// (shared or global memory).
template <bool W, typename V>
__device__ __forceinline__ V ldw(const V* p) {
    if constexpr (W) return __ldcg(p);
    else return *p;
}

// sum over the near set of a root of direction d in refresh cell cell (= (cy << 16) | cx) at
// the positions in npos; returns the number of terms.  Its own entry contributes 0 (see
// acc_root_f).
template <bool W = false>
__device__ __forceinline__ int near_sum(const Ctx<float>& x, int d, int cell, float zx, float zy, float& Dx,
                                        float& Dy) {
    const int nr = x.k->nr;
    const int nbx = x.s_ngrid[2 * d], nby = x.s_ngrid[2 * d + 1];
    const int cx = cell & 0xffff, cy = cell >> 16;
    const int* cst = x.ncst + (size_t)d * (x.ncm + 1);
    const float2* p = x.npos + (size_t)d * nr;
    const int xa = max(cx - 1, 0), xb = min(cx + 1, nbx - 1);
    const f2p zxx = f2_pack(zx, zx), zyy = f2_pack(zy, zy);
    f2p Dx2 = f2_pack(0.f, 0.f), Dy2 = Dx2;
    int cnt = 0;
    for (int yy = max(cy - 1, 0); yy <= min(cy + 1, nby - 1); yy++) {
        const int i0 = ldw<W>(cst + yy * nbx + xa), i1 = ldw<W>(cst + yy * nbx + xb + 1);
        cnt += i1 - i0;
        int i = i0;
#pragma unroll 4
        for (; i + 1 < i1; i += 2) {
            const float2 r0 = ldw<W>(p + i), r1 = ldw<W>(p + i + 1);
            acc_root_f2(zxx, zyy, f2_pack(r0.x, r1.x), f2_pack(r0.y, r1.y), Dx2, Dy2);
        }
        if (i < i1) {
            const float2 r = ldw<W>(p + i);
            acc_root_f(zx, zy, r.x, r.y, Dx, Dy);
        }
    }
    float ua, ub, va, vb;
    f2_unpack(Dx2, ua, ub);
    f2_unpack(Dy2, va, vb);
    Dx += ua + ub;
    Dy -= va + vb;
    return cnt;
}

// In-place inclusive prefix sum of a[0, n) by the whole block (blockDim a multiple of 32).
__device__ void block_scan_inclusive(int* a, int n, int* s_scan) {
    const int tid = threadIdx.x, P = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = P >> 5;
    const int ch = (n + P - 1) / P;
    const int i0 = min(n, tid * ch), i1 = min(n, i0 + ch);
    int s = 0;
    for (int i = i0; i < i1; i++) s += a[i];
    int v = s;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) s_scan[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int u = lane < nw ? s_scan[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, u, o);
            if (lane >= o) u += t;
        }
        if (lane < nw) s_scan[lane] = u;
    }
    __syncthreads();
    int off = v - s + (wid > 0 ? s_scan[wid - 1] : 0);
    for (int i = i0; i < i1; i++) {
        off += a[i];
        a[i] = off;
    }
    __syncthreads();
}

// Refresh row, direction d (whole block): cells of side h over the bounding box of the
// current roots with about NEAR_PER_CELL roots per cell (at most ncm cells), every root's
// cell, and the roots listed cell by cell (row-major), each cell in root-index order so that
// the near sums add their terms in a fixed order.
// W (a cluster shares the sub-range): every CTA of the cluster computes the grid (nbx, nby,
// h: the same values from the same positions) into its own shared memory, and only cluster
// rank 0 writes the arrays, which the others read after the caller's cluster barrier.
template <bool W = false>
__device__ void near_build(const Ctx<float>& x, int d) {
    __shared__ float s_box[4][32];
    __shared__ float s_g[3];
    __shared__ int s_scan[32];
    const int nr = x.k->nr, tid = threadIdx.x, P = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = P >> 5;
    const float2* z = x.cur + (size_t)d * nr;
    float b[4] = {FLT_MAX, FLT_MAX, FLT_MAX, FLT_MAX};  // min x, min y, -max x, -max y
    for (int k = tid; k < nr; k += P) {
        const float2 v = ldw<W>(z + k);
        b[0] = fminf(b[0], v.x);
        b[1] = fminf(b[1], v.y);
        b[2] = fminf(b[2], -v.x);
        b[3] = fminf(b[3], -v.y);
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        for (int o = 16; o > 0; o >>= 1) b[q] = fminf(b[q], __shfl_xor_sync(0xffffffffu, b[q], o));
        if (lane == 0) s_box[q][wid] = b[q];
    }
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; w++)
            for (int q = 0; q < 4; q++) b[q] = fminf(b[q], s_box[q][w]);
        const float x0 = b[0], y0 = b[1];
        const float wd = fmaxf(-b[2] - x0, 1e-3f), ht = fmaxf(-b[3] - y0, 1e-3f);
        float h = sqrtf(wd * ht * (float)NEAR_PER_CELL / (float)nr);
        h = fmaxf(h, fmaxf(wd, ht) * (1.f / 1024.f));
        int nbx, nby;
        for (;;) {
            nbx = (int)(wd / h) + 1;
            nby = (int)(ht / h) + 1;
            if (nbx * nby <= x.ncm) break;
            h *= 1.25f;
        }
        x.s_ngrid[2 * d] = nbx;
        x.s_ngrid[2 * d + 1] = nby;
        x.s_nlim2[d] = 0.0625f * h * h;
        s_g[0] = x0;
        s_g[1] = y0;
        s_g[2] = 1.f / h;
    }
    __syncthreads();
    if constexpr (W) {
        if (cluster_rank() != 0) return;  // block-uniform
    }
    const int nbx = x.s_ngrid[2 * d], nby = x.s_ngrid[2 * d + 1], nc = nbx * nby;
    const float x0 = s_g[0], y0 = s_g[1], ih = s_g[2];
    int* key = x.nkey + (size_t)d * nr;
    int* ord = x.nord + (size_t)d * nr;
    int* cst = x.ncst + (size_t)d * (x.ncm + 1);
    int* fill = x.nfill + (size_t)d * x.ncm;
    for (int c = tid; c <= nc; c += P) cst[c] = 0;
    for (int c = tid; c < nc; c += P) fill[c] = 0;
    __syncthreads();
    for (int k = tid; k < nr; k += P) {
        const float2 v = ldw<W>(z + k);
        // clamped in floating point first (a NaN position lands in cell 0)
        const float fx = fminf(fmaxf((v.x - x0) * ih, 0.f), (float)(nbx - 1));
        const float fy = fminf(fmaxf((v.y - y0) * ih, 0.f), (float)(nby - 1));
        const int c = (int)fy * nbx + (int)fx;
        key[k] = c;
        atomicAdd(&cst[c + 1], 1);
    }
    __syncthreads();
    block_scan_inclusive(cst + 1, nc, s_scan);
    for (int k = tid; k < nr; k += P) {
        const int c = key[k];
        ord[cst[c] + atomicAdd(&fill[c], 1)] = d * nr + k;
    }
    __syncthreads();
    for (int c = tid; c < nc; c += P) {
        const int a = cst[c], e = cst[c + 1];
        for (int i = a + 1; i < e; i++) {
            const int v = ord[i];
            int j = i - 1;
            while (j >= a && ord[j] > v) {
                ord[j + 1] = ord[j];
                j--;
            }
            ord[j + 1] = v;
        }
    }
    __syncthreads();
    for (int i = tid; i < nr; i += P) {
        const int kk = ord[i], k = kk - d * nr, c = key[k];
        x.nrank[kk] = i;
        x.nref[d * nr + i] = ldw<W>(z + k);
        x.ncell[d * nr + i] = ((c / nbx) << 16) | (c % nbx);
    }
    __syncthreads();
}

// One sweep over the active FP32 roots with R roots per thread.  Slots [0, A0) hold the
// direction-0 roots, [A0p, A0p + A1) the direction-1 roots, A0p = A0 rounded up to 32 R so
// that a warp never mixes the directions and every root-tile load is a broadcast.  twin: the
// two directions hold the same positions (the first rows either side of a cold row), so
// direction 0's sums serve root k + nr too, which is then updated with direction 1's phase.
template <int R, bool CAPTURE, bool W = false>
__device__ __forceinline__ void sweep_blocked(const Ctx<float>& x, bool a0, bool a1, int A0, int A1, float cph0,
                                              float sph0, float cph1, float sph1, int* s_maxit, bool twin = false) {
    using C = float2;
    constexpr int TS = CT<float>::TS;
    const TK& K = *x.k;
    const int tid = threadIdx.x, P = blockDim.x;
    const int nr = K.nr, n = K.n;
    const int A0p = (A0 + 32 * R - 1) / (32 * R) * (32 * R);
    const int nq = A0p / R + (A1 + R - 1) / R;  // thread items
    for (int qb = 0; qb < nq; qb += P) {
        const int q = qb + tid;
        const int s0 = q * R;
        const int d = s0 >= A0p ? 1 : 0;
        int key[R];
        bool valid[R];
        C z[R];
        int cell[R];
        Acc<float> acc[R];
        bool any = false;
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int s = s0 + r;
            valid[r] = q < nq && (d ? s - A0p < A1 : s < A0);
            key[r] = valid[r] ? (d ? x.act[nr + s - A0p] : x.act[s]) : -1;
            any |= valid[r];
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int kk = valid[r] ? key[r] : (valid[0] ? key[0] : 0);
            z[r] = x.cur[kk];
            acc[r] = Acc<float>{0, 0, 0, 0, 0, 0, 0, 0, 0};
            cell[r] = valid[r] ? far_cell<float>(K, z[r].x, z[r].y) : -1;
            if (valid[r]) {
                *x.n_terms += (unsigned long long)(cell[r] >= 0 ? K.tcells[cell[r]].near_cnt : n);
                *x.n_far += cell[r] >= 0 ? 1ull : 0ull;
                if (cell[r] >= 0) cell_part<float>(x, cell[r], z[r].x, z[r].y, 0, 1, acc[r]);
            }
        }
        for (int t0 = 0; t0 < n; t0 += TS) {
            const int tn = min(TS, n - t0);
            if (!x.resident) {
                __syncthreads();
                const float4* gs = (const float4*)K.stars;
                for (int j = tid; j < tn; j += P) x.s_star[j] = gs[t0 + j];
                __syncthreads();
            }
#pragma unroll
            for (int r = 0; r < R; r++) {
                if (valid[r] && cell[r] < 0) {
#pragma unroll 4
                    for (int j = 0; j < tn; j++) acc_star(z[r].x, z[r].y, x.s_star[j], acc[r]);
                }
            }
        }
        f2p zxx[R], zyy[R], Dx2[R], Dy2[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            zxx[r] = f2_pack(z[r].x, z[r].x);
            zyy[r] = f2_pack(z[r].y, z[r].y);
            Dx2[r] = f2_pack(0.f, 0.f);
            Dy2[r] = f2_pack(0.f, 0.f);
        }
        for (int t0 = 0; t0 < nr; t0 += TR) {
            const int tn = min(TR, nr - t0);
            const int tp = (tn + 1) >> 1;  // root pairs in the tile (an odd tail pairs with a root at 1e30)
            __syncthreads();
            for (int j = tid; j < 2 * tp; j += P) {
                // pair-interleaved tile: pair i = (x_2i, x_2i+1, y_2i, y_2i+1)
                float* s0 = (float*)(x.s_root) + 4 * (j >> 1) + (j & 1);
                float* s1 = (float*)(x.s_root + TR) + 4 * (j >> 1) + (j & 1);
                // L2 loads: in a cluster, other SMs wrote these positions since the last sweep
                C v0 = make_float2(1e30f, 1e30f), v1 = v0;
                if (j < tn) {
                    if (a0) v0 = __ldcg(&x.cur[t0 + j]);
                    if (a1) v1 = __ldcg(&x.cur[nr + t0 + j]);
                }
                if (a0) {
                    s0[0] = v0.x;
                    s0[2] = v0.y;
                }
                if (a1) {
                    s1[0] = v1.x;
                    s1[2] = v1.y;
                }
            }
            __syncthreads();
            if (any) {
                const unsigned base = (unsigned)__cvta_generic_to_shared(x.s_root + d * TR);
#pragma unroll 8
                for (int j2 = 0; j2 < tp; j2++) {
                    const float4 p = lds_f4(base + 16u * (unsigned)j2);
                    const f2p px = f2_pack(p.x, p.y), py = f2_pack(p.z, p.w);
#pragma unroll
                    for (int r = 0; r < R; r++) acc_root_f2(zxx[r], zyy[r], px, py, Dx2[r], Dy2[r]);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; r++) {
            float a, b, c2, d2;
            f2_unpack(Dx2[r], a, b);
            f2_unpack(Dy2[r], c2, d2);
            acc[r].Dx += a + b;
            acc[r].Dy -= c2 + d2;
        }
        if constexpr (CAPTURE) {
#pragma unroll
            for (int r = 0; r < R; r++)
                if (valid[r]) {
                    float nx = 0.f, ny = 0.f;
                    const int code = d * nr + ldw<W>(x.nrank + key[r]);
                    *x.n_root += (unsigned long long)near_sum<W>(x, d, ldw<W>(x.ncell + code), z[r].x, z[r].y, nx, ny);
                    x.nfar[code] = make_float2(acc[r].Dx - nx, acc[r].Dy - ny);
                    if (twin) x.nfar[nr + code] = x.nfar[code];
                }
        }
#pragma unroll
        for (int r = 0; r < R; r++)
            if (valid[r]) {
                finish_root<float>(x, key[r], z[r], acc[r], d ? cph1 : cph0, d ? sph1 : sph0, s_maxit);
                if (twin) finish_root<float>(x, key[r] + nr, z[r], acc[r], cph1, sph1, s_maxit);
            }
    }
}

// Star terms of a root at z for a light sweep: those of cell_part with one thread per root,
// but the cell's header, its first 8 near-star indices and its expansion coefficients are
// requested together (they depend on the cell alone), so that they cost one memory round trip.
__device__ __forceinline__ void star_part_light(const Ctx<float>& x, float zx, float zy, Acc<float>& acc) {
    const TK& K = *x.k;
    const int n = K.n;
    const float4* gs = (const float4*)K.stars;
    int c = -1;
    if (K.tfmm.ok) {
        const float fx = floorf((zx - K.tfmm.x0) * K.tfmm.inv_b);
        const float fy = floorf((zy - K.tfmm.y0) * K.tfmm.inv_b);
        if (fx >= 0.f && fy >= 0.f && fx < (float)K.tfmm.nbx && fy < (float)K.tfmm.nby)
            c = (int)fy * K.tfmm.nbx + (int)fx;
    }
    int cnt = -1;
    float4 hd = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 i0 = make_int4(0, 0, 0, 0), i1 = i0;
    if (c >= 0) {
        hd = *(const float4*)(K.tcells + c);  // cx, cy, near_cnt, far_m_d2
        const int4* nl4 = (const int4*)(K.tnear + (size_t)c * TFMM_NEAR_MAX);
        i0 = nl4[0];
        i1 = nl4[1];
        cnt = __float_as_int(hd.z);
    }
    *x.n_terms += (unsigned long long)(cnt >= 0 ? cnt : n);
    *x.n_far += cnt >= 0 ? 1ull : 0ull;
    if (cnt < 0) {
        if (x.resident) {
#pragma unroll 4
            for (int j = 0; j < n; j++) acc_star(zx, zy, x.s_star[j], acc);
        } else {
#pragma unroll 4
            for (int j = 0; j < n; j++) acc_star(zx, zy, gs[j], acc);
        }
        return;
    }
    const int id[8] = {i0.x, i0.y, i0.z, i0.w, i1.x, i1.y, i1.z, i1.w};
#pragma unroll
    for (int q = 0; q < 8; q++)
        if (q < cnt) acc_star(zx, zy, x.resident ? x.s_star[id[q]] : gs[id[q]], acc);
    const int* nl = K.tnear + (size_t)c * TFMM_NEAR_MAX;
    for (int q = 8; q < cnt; q++) {
        const int j = nl[q];
        acc_star(zx, zy, x.resident ? x.s_star[j] : gs[j], acc);
    }
    float ux, uy, sx, sy, hx, hy;
    far_eval(K.tcoeff + (size_t)c * TFMM_P, zx - hd.x, zy - hd.y, ux, uy, sx, sy, hx, hy);
    acc.Cx += ux;
    acc.Cy += uy;
    acc.Ax -= sx;
    acc.Ay -= sy;
    acc.Bx += hx;
    acc.By += hy;
    acc.Am += hd.w;
}

// One sweep of a row between refreshes: each active root sums its stars as in the full sweep,
// its near roots exactly at their current positions, and adds its stored far part.  One root
// per thread (two interleaved per thread measured 6% slower).  Positions, cells, far parts and
// refresh positions are read by code (in shared memory when they fit).  ordered: the list is
// the refresh's cell order itself (a row's first sweep), so slot s holds code s (direction 0)
// or nr + s - A0 (direction 1) and neighbouring threads read neighbouring entries.
template <bool W = false>
__device__ void sweep_light(const Ctx<float>& x, bool ordered, int A0, int A1, float cph0, float sph0, float cph1,
                            float sph1, int* s_maxit) {
    const TK& K = *x.k;
    const int nr = K.nr, P = blockDim.x, A = A0 + A1;
    // both directions whole: neighbouring lanes take the two directions' roots of one chain
    // (key k and k + nr), which lie close together and mostly share a star cell
    const bool paired = ordered && A0 == nr && A1 == nr;
    for (int slot = threadIdx.x; slot < A; slot += P) {
        int d = slot < A0 ? 0 : 1;
        int key, code;
        if (paired) {
            d = slot & 1;
            key = x.nord[slot >> 1] + d * nr;
            code = d ? nr + x.nrank[key] : slot >> 1;
        } else if (ordered) {
            code = d ? nr + slot - A0 : slot;
            key = x.nord[code];
        } else {
            key = d ? x.act[nr + slot - A0] : x.act[slot];
            code = d * nr + ldw<W>(x.nrank + key);
        }
        const float2 z = ldw<W>(x.npos + code);
        Acc<float> acc = Acc<float>{0, 0, 0, 0, 0, 0, 0, 0, 0};
        star_part_light(x, z.x, z.y, acc);
        float Dx = 0.f, Dy = 0.f;
        *x.n_root += (unsigned long long)near_sum<W>(x, d, ldw<W>(x.ncell + code), z.x, z.y, Dx, Dy);
        const float2 f = x.nfar[code];  // (written by this CTA)
        acc.Dx = Dx + f.x;
        acc.Dy = Dy + f.y;
        const float2 zn = finish_root<float>(x, key, z, acc, d ? cph1 : cph0, d ? sph1 : sph0, s_maxit);
        const float2 zr = ldw<W>(x.nref + code);
        const float ex = zn.x - zr.x, ey = zn.y - zr.y;
        if (!(ex * ex + ey * ey <= x.s_nlim2[d])) *x.s_nesc = 1;
    }
}

// Sum of three CTA-uniform ints over the cluster (called by all threads of every CTA in the
// same order).  Double-buffered slots: a CTA rewrites a slot two reductions later, after
// the barrier of the reduction in between, which every reader of the slot has passed.
template <typename T>
__device__ __forceinline__ void cluster_sum3(const Ctx<T>& x, int& a, int& b, int& c) {
    const int p = *x.red_parity;
    __syncthreads();
    if (threadIdx.x == 0) {
        x.s_red[4 * p] = a;
        x.s_red[4 * p + 1] = b;
        x.s_red[4 * p + 2] = c;
    }
    cluster_sync();
    if (threadIdx.x == 0) {
        const unsigned G = cluster_size();
        int sa = 0, sb = 0, sc = 0;
        for (unsigned r = 0; r < G; r++) {
            sa += ld_cluster(x.s_red + 4 * p, r);
            sb += ld_cluster(x.s_red + 4 * p + 1, r);
            sc += ld_cluster(x.s_red + 4 * p + 2, r);
        }
        x.s_tot[0] = sa;
        x.s_tot[1] = sb;
        x.s_tot[2] = sc;
        *x.red_parity = p ^ 1;
    }
    __syncthreads();
    a = x.s_tot[0];
    b = x.s_tot[1];
    c = x.s_tot[2];
}

// A cluster's split refresh at the current positions: every CTA computes the grid, cluster
// rank 0 writes the cell arrays, each CTA then writes the cell-ordered positions of its own
// roots.  Cluster barriers before (every CTA's positions published), between and after.
// Called by every thread of every CTA of the cluster, with the same a0, a1.
__device__ void wide_refresh(const Ctx<float>& x, bool a0, bool a1) {
    const int nr = x.k->nr, tid = threadIdx.x, P = blockDim.x, W = x.hi - x.lo;
    cluster_sync();
    if (a0) near_build<true>(x, 0);
    if (a1) near_build<true>(x, 1);
    cluster_sync();
    for (int i = tid; i < 2 * W; i += P) {
        const int d = i >= W;
        if (!(d ? a1 : a0)) continue;
        const int key = d * nr + x.lo + (i - d * W);
        x.npos[d * nr + __ldcg(x.nrank + key)] = x.cur[key];
    }
    cluster_sync();
}

// Run Jacobi Aberth sweeps on the active rows (dir 0: row0, dir 1: row1) until every root
// is frozen or max_iter sweeps were made.  Called by all threads of the CTA.  The unfrozen
// roots of direction d are listed in act[d nr, d nr + A_d).  With many of them the FP32
// tracer gives each thread several roots of one direction (sweep_blocked); otherwise g
// lanes share a root and reduce their partial sums with shuffles.
// Root-sum modes of a row's sweeps: every sweep exact; or the first sweep exact with the far
// parts captured and the rest near + far; or every sweep near + far (FP32, one CTA per row).
enum SumMode { SUM_FULL = 0, SUM_CAPTURE = 1, SUM_LIGHT = 2 };

template <typename T, bool WIDE>
__device__ __forceinline__ int solve_rows(const Ctx<T>& x, bool a0, bool a1, int64_t row0, int64_t row1,
                                          int max_iter, bool cold, bool report, int* s_count, int* s_maxit,
                                          int mode = SUM_FULL, bool twin = false) {
    using C = typename CT<T>::C;
    constexpr int TS = CT<T>::TS;
    const TK& K = *x.k;
    const int tid = threadIdx.x, P = blockDim.x;
    const int nr = K.nr, n = K.n;
    T cph0 = 0, sph0 = 0, cph1 = 0, sph1 = 0;
    if (a0) {
        double2 ph = K.phase[row0];
        cph0 = (T)ph.x;
        sph0 = (T)ph.y;
    }
    if (a1) {
        double2 ph = K.phase[row1];
        cph1 = (T)ph.x;
        sph1 = (T)ph.y;
    }
    const int lo = x.lo, W = x.hi - x.lo;
    Ctx<T> xs = x;
    xs.act = x.act + lo;  // this CTA's lists: [lo, lo + A0) and [nr + lo, nr + lo + A1)
    if constexpr (sizeof(T) != 4) mode = SUM_FULL;
    bool split = mode != SUM_FULL;  // (cleared when a sweep's few roots are summed exactly instead)
    if constexpr (sizeof(T) == 4 && !WIDE) {
        if (split) {
            __syncthreads();
            if (tid == 0) *x.s_nesc = 0;
        }
        if (mode == SUM_CAPTURE) {
            __syncthreads();
            if (twin) {
                // both directions at the same positions: direction 0's cells serve both
                near_build(x, 0);
                const int nc1 = x.s_ngrid[0] * x.s_ngrid[1] + 1;
                for (int i = tid; i < nr; i += P) {
                    x.nord[nr + i] = x.nord[i] + nr;
                    x.nrank[nr + i] = x.nrank[i];
                    x.ncell[nr + i] = x.ncell[i];
                    x.nref[nr + i] = x.nref[i];
                }
                for (int c = tid; c < nc1; c += P) x.ncst[(x.ncm + 1) + c] = x.ncst[c];
                if (tid == 0) {
                    x.s_ngrid[2] = x.s_ngrid[0];
                    x.s_ngrid[3] = x.s_ngrid[1];
                    x.s_nlim2[1] = x.s_nlim2[0];
                }
                __syncthreads();
            } else {
                if (a0) near_build(x, 0);
                if (a1) near_build(x, 1);
            }
        }
    }
    if constexpr (sizeof(T) == 4 && WIDE) {
        // (mode is cluster-uniform: the same sequence of cluster barriers in every CTA)
        if (split) {
            __syncthreads();
            if (tid == 0) *x.s_nesc = 0;
        }
        if (mode == SUM_CAPTURE) wide_refresh(x, a0, a1);
    }
    int Ap0 = 0, Ap1 = 0;  // previous sweep's list lengths (split sweeps)
    bool recap = false;    // a cold row's iterate left its limit: new cells and far parts first
    bool esc = false;      // a warm row's iterate left its limit: the caller solves the row again
    int* next = nullptr;   // split sweeps: the next list, already built by the last position update
    int pend = 0;          // cluster: an iterate of this CTA left its limit in the last sweep
    for (int iter = 0;; iter++) {
        __syncthreads();
        if (!next && tid < 2) s_count[tid] = 0;
        __syncthreads();
        bool listed = false;
        if constexpr (sizeof(T) == 4 && !WIDE) {
            if (split) {
                listed = true;
                if (iter == 0) {
                    // every root of the active directions (all unfrozen at a row's start), in
                    // cell order so that a warp's roots are neighbours (near sets of equal
                    // length over the same entries): the cell-ordered list itself.  After a
                    // refresh the positions are gathered in that order; between refreshes the
                    // prediction pass has already stored them.
                    if (mode == SUM_CAPTURE)
                        for (int i = tid; i < nr; i += P) {
                            if (a0) x.npos[i] = x.cur[x.nord[i]];
                            if (a1) x.npos[nr + i] = x.cur[x.nord[nr + i]];
                        }
                    xs.act = x.nord;
                    if (tid == 0) {
                        s_count[0] = a0 ? nr : 0;
                        s_count[1] = a1 ? nr : 0;
                    }
                } else if (next) {
                    xs.act = next;  // (s_count holds its lengths)
                } else {
                    // the previous list's unfrozen roots, into the other list
                    const int* src = xs.act;
                    int* dst = xs.act == x.act ? x.act2 : x.act;  // (after the first sweep src is nord)
                    for (int i = tid; i < Ap0 + Ap1; i += P) {
                        const int key = i < Ap0 ? src[i] : src[nr + i - Ap0];
                        const int d = key >= nr ? 1 : 0;
                        if (!x.conv[key]) dst[d * nr + atomicAdd(&s_count[d], 1)] = key;
                    }
                    xs.act = dst;
                }
            }
        }
        if (!listed) {
            xs.act = x.act + lo;
            for (int i = tid; i < 2 * W; i += P) {
                const int d = i >= W;
                const int key = d * nr + lo + (i - d * W);
                const bool on = d ? a1 : a0;
                if (on && !x.conv[key]) x.act[d * nr + lo + atomicAdd(&s_count[d], 1)] = key;
            }
        }
        __syncthreads();
        const int A0 = s_count[0], A1 = s_count[1];
        Ap0 = A0;
        Ap1 = A1;
        const int A = A0 + A1;
        int At = A;
        if constexpr (WIDE) {
            int u0 = A0, u1 = A1, u2 = pend;
            cluster_sum3(x, u0, u1, u2);  // also publishes the previous sweep's positions
            At = u0 + u1;
            if constexpr (sizeof(T) == 4) {
                // an escape anywhere in the cluster (a cluster-uniform decision): a cold row
                // refreshes the split, a warm row stops and is solved again
                pend = 0;
                if (u2 > 0) {
                    if (cold) {
                        recap = true;
                    } else {
                        esc = true;
                        break;
                    }
                }
            }
        }
        if (At == 0) break;
        if (iter >= max_iter) {
            if (tid == 0 && report) atomicAdd(&K.rep->unconverged, (unsigned long long)A);
            break;
        }
        if (tid == 0) {
            atomicAdd(&K.rep->root_iterations, (unsigned long long)A);
            if (cold) atomicAdd(&K.rep->cold_root_iterations, (unsigned long long)A);
        }
        if constexpr (sizeof(T) == 4) {
            // A light sweep costs about one root update's latency however few roots it
            // holds, an exact sweep of A roots about A nr terms spread over the block: below
            // A nr = 1024 P (over the cluster: its active roots and threads) the rest of the row
            // is summed exactly (always valid; the next row's prediction guard still checks
            // every position against its refresh).  Decided before a CTA without active roots
            // leaves the iteration, from cluster-uniform values.
            int64_t Au = A, Pu = P;
            if constexpr (WIDE) {
                Au = At;
                Pu = (int64_t)P * cluster_size();
            }
            if (split && iter > 0 && mode == SUM_LIGHT && Au * nr <= Pu * 1024) {
                split = false;
                mode = SUM_FULL;
                recap = false;
            }
            if (recap) {  // block- (cluster-) uniform
                // cells at the current positions and an exact sweep capturing the far parts
                // again: from here on the split holds as after any refresh
                if constexpr (WIDE) {
                    wide_refresh(x, a0, a1);
                } else {
                    if (a0) near_build(x, 0);
                    if (a1) near_build(x, 1);
                    for (int i = tid; i < nr; i += P) {
                        if (a0) x.npos[i] = x.cur[x.nord[i]];
                        if (a1) x.npos[nr + i] = x.cur[x.nord[nr + i]];
                    }
                }
                if (tid == 0) *x.s_nesc = 0;
                __syncthreads();
                mode = SUM_CAPTURE;
                recap = false;
            }
        }
        if (A == 0) {
            // (the other CTAs sweep: keep the cluster-uniform state as they will have it)
            if (mode == SUM_CAPTURE) mode = SUM_LIGHT;
            if constexpr (WIDE) cluster_sync();  // the barrier the other CTAs take before their copies
            continue;
        }
        bool blocked = false;
        if constexpr (sizeof(T) == 4) {
            if (mode == SUM_LIGHT) {
                // (a cluster's lists are slices of keys, never the cell order itself)
                sweep_light<WIDE>(xs, !WIDE && iter == 0, A0, A1, cph0, sph0, cph1, sph1, s_maxit);
                blocked = true;
            }
        }
        // twin: direction 0's sweep updates both directions (its first sweep only)
        const bool tw = twin && iter == 0;
        const int SA1 = tw ? 0 : A1;
        if (mode != SUM_LIGHT && tid == 0) *x.n_root += (unsigned long long)(A0 + SA1) * nr;
        if constexpr (sizeof(T) == 4) {
            if (!blocked && A0 + SA1 >= P) {
                const bool cap = mode == SUM_CAPTURE;
                const bool b1 = tw ? false : a1;
                if (A0 + SA1 >= 2 * P) {
                    if (cap) sweep_blocked<4, true, WIDE>(xs, a0, b1, A0, SA1, cph0, sph0, cph1, sph1, s_maxit, tw);
                    else sweep_blocked<4, false, WIDE>(xs, a0, b1, A0, SA1, cph0, sph0, cph1, sph1, s_maxit, tw);
                } else {
                    if (cap) sweep_blocked<2, true, WIDE>(xs, a0, b1, A0, SA1, cph0, sph0, cph1, sph1, s_maxit, tw);
                    else sweep_blocked<2, false, WIDE>(xs, a0, b1, A0, SA1, cph0, sph0, cph1, sph1, s_maxit, tw);
                }
                blocked = true;
            }
        }
        if (!blocked) {
            int g = P / A;
            g = g < 1 ? 1 : (g > 32 ? 32 : g);
            g = 1 << (31 - __clz(g));  // power of two
            const int groups = P / g;
            const int lane = tid & (g - 1);
            const int gid = tid / g;
            for (int base = 0; base < A; base += groups) {
                const int slot = base + gid;
                const bool valid = slot < A;
                const int key = valid ? (slot < A0 ? xs.act[slot] : xs.act[nr + slot - A0]) : lo;
                const int d = key >= nr;
                const C z = x.cur[key];
                Acc<T> acc = {0, 0, 0, 0, 0, 0, 0, 0, 0};
                const int cell = valid ? far_cell<T>(K, z.x, z.y) : -1;
                if (valid && lane == 0) {
                    *x.n_terms += (unsigned long long)(cell >= 0 ? K.tcells[cell].near_cnt : n);
                    *x.n_far += cell >= 0 ? 1ull : 0ull;
                }
                if (cell >= 0) cell_part<T>(x, cell, z.x, z.y, lane, g, acc);
                for (int t0 = 0; t0 < n; t0 += TS) {
                    const int tn = min(TS, n - t0);
                    if (!x.resident) {
                        __syncthreads();
                        const typename CT<T>::Star* gs = (const typename CT<T>::Star*)K.stars;
                        for (int j = tid; j < tn; j += P) x.s_star[j] = gs[t0 + j];
                        __syncthreads();
                    }
                    if (valid && cell < 0) {
#pragma unroll 4
                        for (int j = lane; j < tn; j += g) acc_star(z.x, z.y, x.s_star[j], acc);
                    }
                }
                for (int t0 = 0; t0 < nr; t0 += TR) {
                    const int tn = min(TR, nr - t0);
                    __syncthreads();
                    for (int j = tid; j < tn; j += P) {
                        if (a0) x.s_root[j] = __ldcg(&x.cur[t0 + j]);
                        if (a1) x.s_root[TR + j] = __ldcg(&x.cur[nr + t0 + j]);
                    }
                    __syncthreads();
                    if (valid) {
                        const C* rr = x.s_root + d * TR;
                        if constexpr (sizeof(T) == 4) {
#pragma unroll 4
                            for (int j = lane; j < tn; j += g) acc_root_f(z.x, z.y, rr[j].x, rr[j].y, acc.Dx, acc.Dy);
                        } else {
#pragma unroll 4
                            for (int j = lane; j < tn; j += g) acc_root(z.x, z.y, rr[j], acc);
                        }
                    }
                }
                for (int off = g >> 1; off > 0; off >>= 1) {
                    acc.Cx += shfl_x(acc.Cx, off);
                    acc.Cy += shfl_x(acc.Cy, off);
                    acc.Ax += shfl_x(acc.Ax, off);
                    acc.Ay += shfl_x(acc.Ay, off);
                    acc.Bx += shfl_x(acc.Bx, off);
                    acc.By += shfl_x(acc.By, off);
                    acc.Dx += shfl_x(acc.Dx, off);
                    acc.Dy += shfl_x(acc.Dy, off);
                    acc.Am += shfl_x(acc.Am, off);
                }
                if constexpr (sizeof(T) == 4) {
                    if (mode == SUM_CAPTURE && valid && lane == 0) {
                        float nx = 0.f, ny = 0.f;
                        const int code = d * nr + ldw<WIDE>(x.nrank + key);
                        *x.n_root +=
                            (unsigned long long)near_sum<WIDE>(x, d, ldw<WIDE>(x.ncell + code), z.x, z.y, nx, ny);
                        x.nfar[code] = make_float2(acc.Dx - nx, acc.Dy - ny);
                    }
                }
                if (valid && lane == 0) finish_root<T>(x, key, z, acc, d ? cph1 : cph0, d ? sph1 : sph0, s_maxit);
            }
        }
        if (mode == SUM_CAPTURE) mode = SUM_LIGHT;
        // every CTA of a cluster has finished reading the positions before any is updated
        if constexpr (WIDE) cluster_sync();
        else __syncthreads();
        // an iterate beyond its limit (only light sweeps set the flag): a cold row, with no
        // prediction to fall back on, refreshes the split; a warm row stops here and is solved
        // again from its predictions
        if constexpr (sizeof(T) == 4 && !WIDE) {
            const bool e = split && *x.s_nesc;
            if (cold) recap = e;
            else if (e) {
                esc = true;
                break;
            }
        }
        // a cluster decides at the next reduction, over all its CTAs
        if constexpr (sizeof(T) == 4 && WIDE) pend = (split && *x.s_nesc) ? 1 : 0;
        next = nullptr;
        if constexpr (sizeof(T) == 4 && !WIDE) {
            if (split) {
                // positions, and the unfrozen roots into the next list (the other list; after
                // the first sweep, whose list is the cell order itself, the first one)
                int* dst = xs.act == x.act ? x.act2 : x.act;
                if (tid < 2) s_count[tid] = 0;
                __syncthreads();
                const bool ordered = xs.act == x.nord;
                for (int i = tid; i < A; i += P) {
                    const int d = i < A0 ? 0 : 1;
                    const int key = d ? xs.act[nr + i - A0] : xs.act[i];
                    const int code = ordered ? (d ? nr + i - A0 : i) : d * nr + x.nrank[key];
                    const float2 zn = x.nxt[key];
                    x.cur[key] = zn;
                    x.npos[code] = zn;
                    if (!x.conv[key]) dst[d * nr + atomicAdd(&s_count[d], 1)] = key;
                }
                next = dst;
            }
        }
        if (!next)
            for (int i = tid; i < A; i += P) {
                const int key = i < A0 ? xs.act[i] : xs.act[nr + i - A0];
                x.cur[key] = x.nxt[key];
                if constexpr (sizeof(T) == 4 && WIDE) {
                    // a cluster's own roots into the shared cell-ordered positions (read by the
                    // other CTAs after the next cluster barrier)
                    if (split) x.npos[(key >= nr ? nr : 0) + __ldcg(x.nrank + key)] = x.nxt[key];
                }
            }
    }
    // directions that still hold unfrozen roots
    bool b0 = false, b1 = false;
    for (int i = tid; i < 2 * W; i += P) {
        const int d = i >= W;
        const int key = d * nr + lo + (i - d * W);
        if (x.conv[key]) continue;
        if (d == 0) b0 |= a0;
        else b1 |= a1;
    }
    int m0 = __syncthreads_or(b0), m1 = __syncthreads_or(b1);
    if constexpr (WIDE) {
        int u2 = 0;
        cluster_sum3(x, m0, m1, u2);
    }
    return (m0 ? 1 : 0) | (m1 ? 2 : 0) | (esc ? 4 : 0);
}

// Cold-start guesses for direction d at phase phi (cos, sin).  Near star i alone,
// F = c_i + m_i/(z - z_i)^2 with c_i = gamma - (1 - kappa_s) e^{-i phi} plus the other stars'
// m_j/(z_i - z_j)^2: its two zeros z_i +- sqrt(-m_i/c_i) start each pair of roots next to
// where an isolated star's critical points lie, far closer than the generic z_i +- 1
// (Sec. 3.2), so the cold Aberth solve takes fewer sweeps; the roots it converges to are
// the same.  A scale 1 + (i mod 64) 2^-12 keeps the guesses of coincident stars apart.
// Fallback (rectangular field, no table and N > CT<T>::TS, or |c_i| ~ 0): the star guesses
// z_i +- (1 + i/64), [2i] = z_i + (1 + i/64), [2i+1] = z_i - (1 + i/64).  The tilt breaks
// the mirror symmetry about the line through a star parallel to the real axis, which FP32
// arithmetic keeps exactly (an isolated star at phi = pi would otherwise never leave that
// line).  A guess equal to an earlier one moves by 1e-3 (1 + i) per earlier copy.
template <typename T>
__device__ __forceinline__ void seed_guesses(const Ctx<T>& x, int d, T cph, T sph) {
    using C = typename CT<T>::C;
    using Star = typename CT<T>::Star;
    const TK& K = *x.k;
    const int nr = K.nr, n = K.n;
    const Star* gs = (const Star*)K.stars;
    const int n2 = 2 * K.n;
    const T oms = (T)(1.0 - K.kappa_s);
    const T c0x = (T)K.gamma - oms * cph, c0y = oms * sph;
    // the other stars' terms: near stars + the cell's expansion where the FP32 tables exist
    // (a few dozen terms), else summed one by one from the shared star tile
    const bool tabled = !K.poly && sizeof(T) == 4 && K.tfmm.ok;
    const bool direct = !K.poly && !tabled && n <= CT<T>::TS;
    for (int k = x.lo + threadIdx.x; k < x.hi; k += blockDim.x) {
        const int key = d * nr + k;
        if (k >= n2) {
            // rectangular field: the t - 1 further roots start evenly spread on the circle of
            // radius |c| around the field (Sec. 3.2), at angles 2 pi (k - 2N + 1/2) / (t - 1)
            const float a = 6.2831853f * ((float)(k - n2) + 0.5f) / (float)(nr - n2);
            float sa, ca;
            __sincosf(a, &sa, &ca);  // a starting guess: the fast intrinsic is accurate enough
            C z;
            z.x = (T)(K.poly->rg * (double)ca);
            z.y = (T)(K.poly->rg * (double)sa);
            x.cur[key] = z;
            x.conv[key] = 0;
            x.it[key] = 0;
            x.dprev[key] = FLT_MAX;
            continue;
        }
        const int i = k >> 1;
        const Star si = gs[i];
        const T sg = (k & 1) ? (T)-1 : (T)1;
        const int cell = tabled ? far_cell<T>(K, (T)si.x, (T)si.y) : -1;
        if (direct || cell >= 0) {
            T ax = c0x, ay = c0y;
            auto add = [&](const Star& sj, int j) {
                const T dx = (T)si.x - (T)sj.x, dy = (T)si.y - (T)sj.y;
                const T r2 = dx * dx + dy * dy;
                if (j == i || !(r2 > (T)0)) return;
                const T inv = (T)1 / r2;
                const T ux = dx * inv, uy = -dy * inv;
                ax += (T)sj.z * (ux * ux - uy * uy);
                ay += (T)sj.z * ((T)2 * ux * uy);
            };
            if (direct) {
                for (int j = 0; j < n; j++) add(x.resident ? x.s_star[j] : gs[j], j);
            } else {
                // the cell's near stars, then its expansion of the far stars' S1 about the
                // cell centre: sum_far m_j/(z - z_j)^2 = -S1'(t), t = z - centre
                const TCell tc = K.tcells[cell];
                const int* nl = K.tnear + (size_t)cell * TFMM_NEAR_MAX;
                for (int q = 0; q < tc.near_cnt; q++) add(gs[nl[q]], nl[q]);
                float ux, uy, sx, sy, hx, hy;
                far_eval(K.tcoeff + (size_t)cell * TFMM_P, (float)si.x - tc.cx, (float)si.y - tc.cy, ux, uy, sx, sy,
                         hx, hy);
                ax -= (T)sx;
                ay -= (T)sy;
            }
            const T den = ax * ax + ay * ay;
            // w = -m_i / c_i, and its principal square root
            const T wx = -(T)si.z * ax / den, wy = (T)si.z * ay / den;
            const T r = sqrt(wx * wx + wy * wy);
            const T sr = sqrt((T)0.5 * (r + wx)), sq = copysign(sqrt((T)0.5 * fmax(r - wx, (T)0)), wy);
            if (den > (T)1e-12 && sr == sr && sq == sq && r < (T)1e12) {
                const T sc = sg * ((T)1 + (T)(i & 63) * (T)2.44140625e-4);
                C z;
                z.x = (T)si.x + sc * sr;
                z.y = (T)si.y + sc * sq;
                x.cur[key] = z;
                x.conv[key] = 0;
                x.it[key] = 0;
                x.dprev[key] = FLT_MAX;
                continue;
            }
        }
        const T gx = (T)si.x + sg, gy = (T)si.y + sg * (T)0.015625;
        int dup = 0;
        for (int a = 0; a < k; a++) {
            const Star sa = gs[a >> 1];
            const T sa_g = (a & 1) ? (T)-1 : (T)1;
            const T ax = (T)sa.x + sa_g, ay = (T)sa.y + sa_g * (T)0.015625;
            dup += (ax == gx && ay == gy);
        }
        C z;
        z.x = gx + (T)1e-3 * (T)dup;
        z.y = gy + (T)1e-3 * (T)dup;
        x.cur[key] = z;
        x.conv[key] = 0;
        x.it[key] = 0;
        x.dprev[key] = FLT_MAX;
    }
}

// One sub-range s of one field, start to end, by the whole CTA: cold start at its centre
// row, then both directions row by row.  w: this CTA's Jacobi scratch.
template <typename T, bool WIDE>
__device__ __forceinline__ void run_subchain(const TK& K, const int s, char* w, unsigned char* smem,
                                             int* s_count_p, int* s_maxit_p, unsigned long long* n_terms_p,
                                             unsigned long long* n_far_p, unsigned long long* n_root_p,
                                             int* s_red = nullptr,
                                             int* s_tot = nullptr, int* red_parity = nullptr, int rank = 0,
                                             int G = 1) {
    using C = typename CT<T>::C;
    using Star = typename CT<T>::Star;
    constexpr int TS = CT<T>::TS;
    int* s_count = s_count_p;  // [2]: active roots per direction
    int& s_maxit = *s_maxit_p;
    const int tid = threadIdx.x, P = blockDim.x;
    const int nr = K.nr, n = K.n;
    const int64_t b0 = subchain_begin(s, K.m, K.S), b1 = subchain_begin(s + 1, K.m, K.S);
    const int64_t c = (b0 + b1) / 2;

    Ctx<T> x;
    x.k = &K;
    x.s_star = (Star*)smem;
    x.s_root = (C*)(smem + sizeof(Star) * (size_t)min(n, TS));  // star tile of min(n, TS) stars
    x.cur = (C*)w;
    x.nxt = x.cur + 2 * nr;
    x.prev = x.nxt + 2 * nr;
    x.prev2 = x.prev + 2 * nr;
    x.dprev = (float*)(x.prev2 + 2 * nr);
    x.conv = (int*)(x.dprev + 2 * nr);
    x.it = x.conv + 2 * nr;
    x.act = x.it + 2 * nr;
    {
        char* nb = (char*)(x.act + 2 * nr);
        x.ncm = near_cells_max(nr);
        x.nfar = (float2*)nb;
        nb += sizeof(float2) * 2 * (size_t)nr;
        x.npos = (float2*)nb;
        nb += sizeof(float2) * 2 * (size_t)nr;
        x.nkey = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)nr;
        x.nord = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)nr;
        x.ncst = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)(x.ncm + 1);
        x.nfill = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)x.ncm;
        nb = (char*)(((uintptr_t)nb + 15) & ~(uintptr_t)15);
        x.nref = (float2*)nb;
        nb += sizeof(float2) * 2 * (size_t)nr;
        x.npred = (float2*)nb;
        nb += sizeof(float2) * 2 * (size_t)nr;
        x.nrank = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)nr;
        x.act2 = (int*)nb;
        nb += sizeof(int) * 2 * (size_t)nr;
        x.ncell = (int*)nb;
        if (nr <= K.near_cap) {
            // ordered positions and cell starts in shared memory, after the root tiles, and
            // (near_ext) the far parts, refresh positions and cells after them
            unsigned char* ns = (unsigned char*)(x.s_root + 2 * TR);
            x.npos = (float2*)ns;
            x.ncst = (int*)(ns + sizeof(float2) * 2 * (size_t)nr);
            if (K.near_ext) {
                float2* ne = (float2*)(((uintptr_t)(x.ncst + 2 * (size_t)(x.ncm + 1)) + 15) & ~(uintptr_t)15);
                x.nfar = ne;
                x.nref = ne + 2 * (size_t)nr;
                x.ncell = (int*)(ne + 4 * (size_t)nr);
            }
        }
    }
    __shared__ int s_ngrid[4], s_nesc;
    __shared__ float s_nlim2[2];
    x.s_ngrid = s_ngrid;
    x.s_nlim2 = s_nlim2;
    x.s_nesc = &s_nesc;
    x.resident = n <= TS;
    {
        const int Wd = (nr + G - 1) / G;
        x.lo = min(nr, rank * Wd);
        x.hi = min(nr, x.lo + Wd);
    }
    x.s_red = s_red;
    x.s_tot = s_tot;
    x.red_parity = red_parity;
    x.n_terms = n_terms_p;
    x.n_far = n_far_p;
    x.n_root = n_root_p;
    const int lo = x.lo, hi = x.hi;
    const Star* gs = (const Star*)K.stars;
    if (x.resident)
        for (int j = tid; j < n; j += P) x.s_star[j] = gs[j];
    __syncthreads();  // the guesses read the star tile
    {
        const double2 ph = K.phase[c];
        seed_guesses<T>(x, 0, (T)ph.x, (T)ph.y);
    }
    for (int k = lo + tid; k < hi; k += P) x.conv[nr + k] = 1;
    const int KR = sizeof(T) == 4 ? K.root_refresh : 0;
    // the cold row splits its root sum too: cells and far parts at the guesses, refreshed
    // whenever an iterate leaves its limit
    solve_rows<T, WIDE>(x, true, false, c, -1, K.max_iter_cold, true, true, s_count, &s_maxit,
                        KR >= 2 ? SUM_CAPTURE : SUM_FULL);

    C* zrows = (C*)K.zrows;
    C* seam = (C*)K.seam;
    auto dst = [&](int64_t row) -> C* {
        return (row == b1 && s < K.S - 1) ? seam + (size_t)s * nr : zrows + (size_t)row * nr;
    };
    // extent of the points written to zrows (FP32 form; the far-field polish grids them):
    // each output pass folds its values per thread, then per warp into order-preserving
    // integer keys in shared memory (min x, min y, -max x, -max y; flag of a non-finite point)
    __shared__ int s_ek[5];
    if (tid < 4) s_ek[tid] = 0x7fffffff;
    if (tid == 4) s_ek[4] = 0;
    __syncthreads();
    const bool want_ext = sizeof(T) == 4 && K.ext != nullptr;
    auto fold = [&](const C* vals, int n_lo, int n_hi) {  // called by every thread
        float e[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f};
        int bad = 0;
        for (int k = n_lo + tid; k < n_hi; k += P) {
            const C v = vals[k];
            const float vx = (float)v.x, vy = (float)v.y;
            if (!(isfinite(vx) && isfinite(vy))) {
                bad = 1;
                continue;
            }
            e[0] = fminf(e[0], vx);
            e[1] = fminf(e[1], vy);
            e[2] = fminf(e[2], -vx);
            e[3] = fminf(e[3], -vy);
        }
#pragma unroll
        for (int q = 0; q < 4; q++)
            for (int off = 16; off > 0; off >>= 1) e[q] = fminf(e[q], __shfl_xor_sync(0xffffffffu, e[q], off));
        bad = __any_sync(0xffffffffu, bad);
        if ((tid & 31) == 0) {
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const int b = __float_as_int(e[q]);
                atomicMin(&s_ek[q], b >= 0 ? b : b ^ 0x7fffffff);  // float order as int order
            }
            if (bad) s_ek[4] = 1;
        }
    };
    {
        C* o = dst(c);
        const bool into_rows = !(c == b1 && s < K.S - 1);
        for (int k = lo + tid; k < hi; k += P) {
            o[k] = x.cur[k];
            x.cur[nr + k] = x.cur[k];
            K.iters[(size_t)c * nr + k] = x.it[k];
        }
        if (want_ext && into_rows) fold(x.cur, lo, hi);
    }
    // s_hist[d]: rows of direction d already behind the current one that belong to the same
    // chains (a row re-solved from the star guesses has new column labels: history restarts)
    __shared__ int s_hist[2];
    // s_refresh: the near/far split needs new cells (first warm row, or a row after a restart)
    __shared__ int s_refresh;
    if (tid == 0) s_hist[0] = s_hist[1] = 0;
    if (tid == 0) s_refresh = 1;
    for (int64_t t = 1;; t++) {
        const bool a0 = c - t >= b0, a1 = c + t <= b1;
        if (!a0 && !a1) break;
        const int64_t r0 = c - t, r1 = c + t;
        __syncthreads();
        const bool refresh_due = s_refresh != 0;
        int mode = SUM_FULL;
        if (KR >= 2) mode = (refresh_due || (t - 1) % max(KR, 1) == 0) ? SUM_CAPTURE : SUM_LIGHT;
        bool out = false;  // a prediction beyond its displacement limit (light rows)
        for (int i = tid; i < 2 * (hi - lo); i += P) {
            const int dd = i >= hi - lo;
            const int k = dd * nr + lo + (i - dd * (hi - lo));
            const bool on = k < nr ? a0 : a1;
            if (!on) {
                x.conv[k] = 1;
                continue;
            }
            const int h = s_hist[k < nr ? 0 : 1];
            const C zc = x.cur[k];
            C g = zc;
            if (K.predictor >= 2 && h >= 2) {
                // quadratic extrapolation through the last three rows: 3 z_c - 3 z_p + z_pp
                const C zp = x.prev[k], zpp = x.prev2[k];
                g.x = zpp.x + (T)3 * (zc.x - zp.x);
                g.y = zpp.y + (T)3 * (zc.y - zp.y);
            } else if (K.predictor >= 1 && h >= 1) {
                const C zp = x.prev[k];
                g.x = zc.x + (zc.x - zp.x);
                g.y = zc.y + (zc.y - zp.y);
            }
            if (h >= 1) x.prev2[k] = x.prev[k];
            x.prev[k] = zc;
            x.cur[k] = g;
            if constexpr (sizeof(T) == 4) {
                if (KR >= 2) {
                    x.npred[k] = g;
                    // cells from an earlier refresh: the prediction goes to its place in cell
                    // order (a refresh row gathers all positions again after its new cells)
                    if (!refresh_due) {
                        const int code = (k >= nr ? nr : 0) + ldw<WIDE>(x.nrank + k);
                        x.npos[code] = g;
                        if (mode == SUM_LIGHT) {
                            const float2 r = ldw<WIDE>(x.nref + code);
                            const float ex = g.x - r.x, ey = g.y - r.y;
                            out |= !(ex * ex + ey * ey <= s_nlim2[dd]);
                        }
                    }
                }
            }
            x.conv[k] = 0;
            x.it[k] = 0;
            x.dprev[k] = FLT_MAX;
        }
        // a prediction beyond its displacement limit: refresh at this row (over a cluster: any
        // CTA's, a cluster-uniform decision; mode itself is uniform)
        if (mode == SUM_LIGHT) {
            int o = __syncthreads_or(out);
            if constexpr (WIDE) {
                int z1 = 0, z2 = 0;
                cluster_sum3(x, o, z1, z2);
            }
            if (o) mode = SUM_CAPTURE;
        }
        // the first rows either side of the cold row start from its positions (no history yet):
        // one capture sweep serves both directions when every root of both is swept
        const bool twin = sizeof(T) == 4 && !WIDE && t == 1 && a0 && a1 && mode == SUM_CAPTURE && nr >= P &&
                          lo == 0 && hi == nr;
        int bad = solve_rows<T, WIDE>(x, a0, a1, r0, r1, K.max_iter_warm, false, false, s_count, &s_maxit, mode,
                                      twin);
        if (bad & 4) {
            // an iterate went beyond its limit: this row again from its predictions, with the
            // exact root sum in every sweep
            __syncthreads();
            for (int i = tid; i < 2 * (hi - lo); i += P) {
                const int dd = i >= hi - lo;
                if (!(dd ? a1 : a0)) continue;
                const int k = dd * nr + lo + (i - dd * (hi - lo));
                if constexpr (sizeof(T) == 4) x.cur[k] = x.npred[k];
                x.conv[k] = 0;
                x.it[k] = 0;
                x.dprev[k] = FLT_MAX;
            }
            bad = solve_rows<T, WIDE>(x, a0, a1, r0, r1, K.max_iter_warm, false, false, s_count, &s_maxit);
            if (tid == 0) atomicAdd(&K.rep->split_redone_rows, 1ull);
        }
        if (tid == 0) {  // read again only after the next row's opening barrier
            if (a0) s_hist[0] = min(s_hist[0] + 1, 2);
            if (a1) s_hist[1] = min(s_hist[1] + 1, 2);
            if (bad & 1) s_hist[0] = 0;
            if (bad & 2) s_hist[1] = 0;
            s_refresh = (bad & 3) ? 1 : 0;
        }
        bad &= 3;
        if (bad) {
            // A warm start that does not settle (e.g. a phase step so large that the previous
            // row sits on a symmetric, non-converging configuration) restarts that row from
            // the star guesses.
            __syncthreads();
            if (bad & 1) seed_guesses<T>(x, 0, (T)K.phase[r0].x, (T)K.phase[r0].y);
            if (bad & 2) seed_guesses<T>(x, 1, (T)K.phase[r1].x, (T)K.phase[r1].y);
            solve_rows<T, WIDE>(x, bad & 1, (bad & 2) != 0, r0, r1, K.max_iter_cold, true, true, s_count, &s_maxit);
        }
        if (a0) {
            C* o = dst(r0);
            for (int k = lo + tid; k < hi; k += P) {
                o[k] = x.cur[k];
                K.iters[(size_t)r0 * nr + k] = x.it[k];
            }
            if (want_ext) fold(x.cur, lo, hi);
        }
        if (a1) {
            C* o = dst(r1);
            const bool into_rows = !(r1 == b1 && s < K.S - 1);
            for (int k = lo + tid; k < hi; k += P) {
                o[k] = x.cur[nr + k];
                if (into_rows) K.iters[(size_t)r1 * nr + k] = x.it[nr + k];
            }
            if (want_ext && into_rows) fold(x.cur + nr, lo, hi);
        }
    }
    __syncthreads();
    if (want_ext && tid == 0) {
        float e[4];
        for (int q = 0; q < 4; q++) {
            const int b = s_ek[q];
            e[q] = __int_as_float(b >= 0 ? b : b ^ 0x7fffffff);
        }
        // a NaN marks a non-finite point
        K.ext[blockIdx.x] = make_float4(s_ek[4] ? __int_as_float(0x7fc00000) : e[0], e[1], -e[2], -e[3]);
    }
    __syncthreads();
}

// Per-thread work counters summed over the warp, one atomic per warp.
__device__ __forceinline__ void add_work_counters(DevReport* rep, unsigned long long n_terms,
                                                  unsigned long long n_far, unsigned long long n_root) {
    for (int off = 16; off > 0; off >>= 1) {
        n_terms += __shfl_xor_sync(0xffffffffu, n_terms, off);
        n_far += __shfl_xor_sync(0xffffffffu, n_far, off);
        n_root += __shfl_xor_sync(0xffffffffu, n_root, off);
    }
    if ((threadIdx.x & 31) == 0) {
        if (n_terms) atomicAdd(&rep->star_terms, n_terms);
        if (n_far) atomicAdd(&rep->far_evals, n_far);
        if (n_root) atomicAdd(&rep->root_terms, n_root);
    }
}

template <typename T>
__global__ void __launch_bounds__(512, 1) trace_kernel(TK K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_count[2], s_maxit;
    if (threadIdx.x == 0) s_maxit = 0;
    unsigned long long n_terms = 0, n_far = 0, n_root = 0;
    run_subchain<T, false>(K, blockIdx.x, K.work + (size_t)blockIdx.x * K.work_stride, smem, s_count, &s_maxit,
                           &n_terms, &n_far, &n_root);
    add_work_counters(K.rep, n_terms, n_far, n_root);
    if (threadIdx.x == 0) atomicMax(&K.rep->max_iter_row, s_maxit);
}

// One phi sub-range per thread-block cluster (grid = S clusters of G CTAs): for rows so wide
// (many roots) that one SM per sub-range would leave most of the GPU idle on a small m.  Both
// arithmetics: the FP32 tracer and the plain FP64 form.
template <typename T>
__global__ void __launch_bounds__(512, 1) trace_wide_kernel(TK K) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_count[2], s_maxit, s_red[8], s_tot[4], s_parity;
    if (threadIdx.x == 0) {
        s_maxit = 0;
        s_parity = 0;
    }
    const int G = (int)cluster_size(), rank = (int)cluster_rank();
    const int s = (int)blockIdx.x / G;
    unsigned long long n_terms = 0, n_far = 0, n_root = 0;
    __syncthreads();
    run_subchain<T, true>(K, s, K.work + (size_t)s * K.work_stride, smem, s_count, &s_maxit, &n_terms, &n_far,
                          &n_root, s_red, s_tot, &s_parity, rank, G);
    add_work_counters(K.rep, n_terms, n_far, n_root);
    if (threadIdx.x == 0) atomicMax(&K.rep->max_iter_row, s_maxit);
    cluster_sync();  // no CTA leaves while another may still read its shared memory
}

// Many fields in one persistent launch: resident CTAs take (field, sub-range) items from a
// global counter, most expensive first, until the list is exhausted (a bounded loop).
template <typename T>
__global__ void __launch_bounds__(512, 1) trace_batch_kernel(BatchTraceArgs B) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_count[2], s_maxit, s_item;
    unsigned long long n_terms = 0, n_far = 0, n_root = 0;
    char* w = (char*)B.work + (size_t)blockIdx.x * B.work_stride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(B.queue, 1u);
        __syncthreads();
        const int item = s_item;
        if (item >= B.nitems) break;
        const int2 fs = B.items[item];
        const TraceTask& t = B.tasks[fs.x];
        TK K;
        K.stars = t.stars;
        K.poly = t.poly;
        K.n = t.n;
        K.nr = t.nr;
        K.kappa_s = t.kappa_s;
        K.gamma = t.gamma;
        K.m = t.m;
        K.S = t.S;
        K.phase = t.phase;
        K.zrows = t.zrows;
        K.seam = t.seam;
        K.iters = t.iters;
        K.work = nullptr;
        K.work_stride = 0;
        K.rep = t.rep;
        K.tol_abs = B.tol_abs;
        K.mu_max = 0.0;
        K.max_iter_cold = B.max_iter_cold;
        K.max_iter_warm = B.max_iter_warm;
        K.predictor = B.predictor;
        K.tfmm = t.tfmm;
        K.tcells = t.tcells;
        K.tnear = t.tnear;
        K.tcoeff = t.tcoeff;
        K.root_refresh = B.root_refresh;
        K.near_cap = B.near_cap;
        K.ext = nullptr;
        K.near_ext = B.near_ext;
        if (threadIdx.x == 0) s_maxit = 0;
        n_terms = 0;
        n_far = 0;
        n_root = 0;
        run_subchain<T, false>(K, fs.y, w, smem, s_count, &s_maxit, &n_terms, &n_far, &n_root);
        add_work_counters(K.rep, n_terms, n_far, n_root);
        if (threadIdx.x == 0) atomicMax(&K.rep->max_iter_row, s_maxit);
    }
}

// Shared memory of a tracing CTA: a star tile of min(n, TS) stars, then the root tiles, then
// (near_cap > 0) the split's ordered positions and cell starts for rows of up to near_cap roots,
// then, when they fit in an SM's 227 KB (tracer_near_ext), its far parts, refresh positions and
// cells.
static size_t tracer_smem_base(bool fp64, int64_t n, int near_cap) {
    const int64_t ts = std::min<int64_t>(n, fp64 ? CT<double>::TS : CT<float>::TS);
    size_t b = fp64 ? ts * sizeof(StarD) + 2 * TR * sizeof(double2) : ts * sizeof(float4) + 2 * TR * sizeof(float2);
    if (near_cap > 0)
        b += sizeof(float2) * 2 * (size_t)near_cap + sizeof(int) * 2 * (size_t)(near_cells_max(near_cap) + 1);
    return b;
}

static size_t near_ext_bytes(int near_cap) {
    return 16 + (size_t)2 * near_cap * (2 * sizeof(float2) + sizeof(int));
}

bool tracer_near_ext(int64_t n, int near_cap) {
    return near_cap > 0 && tracer_smem_base(false, n, near_cap) + near_ext_bytes(near_cap) <= (size_t)227 * 1024;
}

size_t tracer_smem_bytes(bool fp64, int64_t n, int near_cap) {
    size_t b = tracer_smem_base(fp64, n, near_cap);
    if (!fp64 && tracer_near_ext(n, near_cap)) b += near_ext_bytes(near_cap);
    return b;
}

size_t tracer_work_stride(int64_t nr, size_t elem) {
    size_t b = (size_t)(2 * nr) * (4 * elem + 4 * 4);
    // near/far split of the root sum: far part, ordered, refresh and predicted positions
    // (float2), cell by key, ordered index, rank, a second active list and cell by code (int)
    // per root; cell starts and scatter counters per direction
    b += (size_t)(2 * nr) * (4 * sizeof(float2) + 5 * sizeof(int)) +
         (size_t)2 * (2 * (size_t)near_cells_max((int)nr) + 1) * sizeof(int) + 16;
    return (b + 255) / 256 * 256;
}

// Tracing CTAs that fit on one SM at once (registers and shared memory).
int tracer_blocks_per_sm(bool fp64, int threads, int64_t n) {
    int b = 0;
    const size_t smem = tracer_smem_bytes(fp64, n);
    cudaError_t e;
    if (fp64) {
        e = cudaFuncSetAttribute(trace_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel<double>, threads, smem);
    } else {
        e = cudaFuncSetAttribute(trace_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_kernel<float>, threads, smem);
    }
    if (e != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

// CTAs per sub-range.  Wide rows need a cluster per sub-range when there are too few rows to
// give every SM a sub-range of its own; with enough rows (at least 8 per SM) one CTA per
// sub-range is faster when the root sum is split (its cold starts cost one SM each, but
// every warm row takes a small fraction of the exact sum: N = 20000, m = 2e4 traces in
// 0.77 s against 9.2 s with clusters).
int tracer_cluster_size(const cc_options& o, int64_t nr, bool fp64, int64_t m, int sms) {
    if (o.row_ctas > 0) return o.row_ctas;
    if (nr < WIDE_MIN_NR) return 1;
    // with enough rows one CTA per sub-range wins: the FP32 tracer's root-sum split makes
    // warm rows cheap, and the FP64 form's rows then already fill every SM
    if ((fp64 || o.root_refresh >= 2) && m >= 8 * (int64_t)sms) return 1;
    return 8;
}

template <typename T>
static cudaError_t wide_attributes(int G, size_t smem) {
    cudaError_t e = cudaFuncSetAttribute(trace_wide_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess && G > 8)
        e = cudaFuncSetAttribute(trace_wide_kernel<T>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

int tracer_max_clusters(int G, int threads, bool fp64) {
    const size_t smem =
        fp64 ? tracer_smem_bytes(true, (int64_t)CT<double>::TS) : tracer_smem_bytes(false, (int64_t)CT<float>::TS);
    cudaError_t e = fp64 ? wide_attributes<double>(G, smem) : wide_attributes<float>(G, smem);
    int n = 0;
    if (e == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)G);
        cfg.blockDim = dim3((unsigned)threads);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)G;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = fp64 ? cudaOccupancyMaxActiveClusters(&n, trace_wide_kernel<double>, &cfg)
                 : cudaOccupancyMaxActiveClusters(&n, trace_wide_kernel<float>, &cfg);
    }
    if (e != cudaSuccess) cudaGetLastError();
    return n > 0 ? n : 1;
}

int subchain_count(int64_t m, int64_t nr, const cc_options& o, int sms, int blocks_per_sm) {
    int64_t S = o.subchains;
    if (S <= 0) {
        // one wave of tracing CTAs (every sub-range pays one cold start); each sub-range
        // keeps at least 8 rows
        S = (int64_t)sms * (blocks_per_sm < 1 ? 1 : blocks_per_sm);
        if (S > m / 8) S = m / 8;
    }
    if (S > m / 2) S = m / 2;
    if (S < 1) S = 1;
    return (int)S;
}

cudaError_t launch_trace(const TraceArgs& a, bool fp64, cudaStream_t st) {
    TK K;
    K.n = (int)a.f->n;
    K.nr = (int)a.f->nr;
    K.poly = a.f->poly;
    K.stars = fp64 ? (const void*)a.f->star64 : (const void*)a.f->star32;
    K.kappa_s = a.f->kappa_s;
    K.gamma = a.f->gamma;
    K.m = a.m;
    K.S = a.S;
    K.phase = a.phase;
    K.zrows = a.zrows;
    K.seam = a.seam;
    K.iters = a.iters;
    K.work = (char*)a.work;
    K.work_stride = a.work_stride;
    K.rep = a.rep;
    K.tol_abs = a.tol_abs;
    K.mu_max = a.mu_max;
    K.max_iter_cold = a.max_iter_cold;
    K.max_iter_warm = a.max_iter_warm;
    K.predictor = a.predictor;
    K.root_refresh = a.root_refresh;
    K.tfmm = a.f->tfmm;
    if (fp64) K.tfmm.ok = 0;
    K.tcells = a.f->tcells;
    K.tnear = a.f->tnear;
    K.tcoeff = a.f->tcoeff;
    K.ext = fp64 ? nullptr : a.ext;
    K.near_cap = (!fp64 && a.cluster <= 1 && a.root_refresh >= 2 && a.f->nr <= NEAR_SMEM_NR) ? (int)a.f->nr : 0;
    K.near_ext = tracer_near_ext(a.f->n, K.near_cap) ? 1 : 0;
    const size_t smem = tracer_smem_bytes(fp64, a.f->n, K.near_cap);
    cudaError_t e;
    if (a.cluster > 1) {
        e = fp64 ? wide_attributes<double>(a.cluster, smem) : wide_attributes<float>(a.cluster, smem);
        if (e != cudaSuccess) return e;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(a.S * a.cluster));
        cfg.blockDim = dim3((unsigned)a.threads);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)a.cluster;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        e = fp64 ? cudaLaunchKernelEx(&cfg, trace_wide_kernel<double>, K) : cudaLaunchKernelEx(&cfg, trace_wide_kernel<float>, K);
        if (e != cudaSuccess) return e;
        return cudaGetLastError();
    }
    if (fp64) {
        e = cudaFuncSetAttribute(trace_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        trace_kernel<double><<<a.S, a.threads, smem, st>>>(K);
    } else {
        e = cudaFuncSetAttribute(trace_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        trace_kernel<float><<<a.S, a.threads, smem, st>>>(K);
    }
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Joining the subchains: the up-end row of subchain s and the first row of subchain s+1
// are the same root set (Sec. 4.3 footnote: the end of one chain is the start of the
// next); each of s's columns is matched to its nearest root of s+1's row, and the column
// permutations are composed so that global column g follows one chain across all rows.
// ----------------------------------------------------------------------------------
// Each of seam s's columns k (one thread each) against the first row of sub-range s + 1,
// read through shared-memory tiles of SM_TILE roots that the whole block shares.  Distances
// in the tracer's own precision: roots of one row are separated by far more than the
// tracer's rounding error, so FP32 suffices for the mixed form.
constexpr int SM_TILE = 1024;
template <typename C, typename T>
__device__ __forceinline__ void seam_match_block(const C* zrows, const C* seam, int64_t m, int S, int nr, int s,
                                                 int32_t* match, int32_t* hits, DevReport* rep, C* tile) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t row = subchain_begin(s + 1, m, S);
    const C* B = zrows + (size_t)row * nr;
    const C q = k < nr ? seam[(size_t)s * nr + k] : C{};
    T best = (T)3.0e38, second = (T)3.0e38;
    int bi = 0;
    for (int t0 = 0; t0 < nr; t0 += SM_TILE) {
        const int tn = min(SM_TILE, nr - t0);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += blockDim.x) tile[j] = B[t0 + j];
        __syncthreads();
        for (int j = 0; j < tn; j++) {
            const C b = tile[j];
            const T dx = b.x - q.x, dy = b.y - q.y;
            const T d2 = dx * dx + dy * dy;
            if (d2 < best) {
                second = best;
                best = d2;
                bi = t0 + j;
            } else if (d2 < second) {
                second = d2;
            }
        }
    }
    if (k >= nr) return;
    match[(size_t)s * nr + k] = bi;
    atomicAdd(&hits[(size_t)s * nr + bi], 1);
    if (!(best <= (T)1e-4 * second)) atomicAdd(&rep->seam_ambiguous, 1ull);
}

template <typename C, typename T>
__global__ void seam_match_kernel(const C* zrows, const C* seam, int64_t m, int S, int nr,
                                  int32_t* match, int32_t* hits, DevReport* rep) {
    __shared__ C tile[SM_TILE];
    if ((int)(blockIdx.x * blockDim.x) >= nr) return;  // block-uniform
    seam_match_block<C, T>(zrows, seam, m, S, nr, blockIdx.y, match, hits, rep, tile);
}

// Batched: blockIdx.y indexes all seams of all fields.
__global__ void seam_match_batch_kernel(const TraceTask* tasks, const int2* seams) {
    __shared__ float2 tile[SM_TILE];
    const int2 fs = seams[blockIdx.y];
    const TraceTask& t = tasks[fs.x];
    if ((int)(blockIdx.x * blockDim.x) >= t.nr) return;  // block-uniform
    seam_match_block<float2, float>((const float2*)t.zrows, (const float2*)t.seam, t.m, t.S, t.nr, fs.y, t.match,
                                    t.hits, t.rep, tile);
}

// Chain permutations: perm_{s+1}[g] = match_s[perm_s[g]], perm_0 = identity.  Each column g
// is an independent chain through the seams, so one thread carries it in a register.
__device__ __forceinline__ void compose_perm_body(int S, int nr, const int32_t* match, const int32_t* hits,
                                                  int32_t* perm, DevReport* rep, int g0, int gstride) {
    int bad = 0;
    for (int g = g0; g < nr; g += gstride) {
        int p = g;
        perm[g] = g;
        for (int s = 0; s + 1 < S; s++) {
            p = match[(size_t)s * nr + p];
            perm[(size_t)(s + 1) * nr + g] = p;
            bad += hits[(size_t)s * nr + g] != 1;
        }
    }
    if (bad) atomicAdd(&rep->seam_ambiguous, (unsigned long long)bad);
}

__global__ void compose_perm_kernel(int S, int nr, const int32_t* match, const int32_t* hits,
                                    int32_t* perm, DevReport* rep) {
    compose_perm_body(S, nr, match, hits, perm, rep, blockIdx.x * blockDim.x + threadIdx.x, gridDim.x * blockDim.x);
}

__global__ void compose_perm_batch_kernel(const TraceTask* tasks) {
    const TraceTask& t = tasks[blockIdx.x];
    compose_perm_body(t.S, t.nr, t.match, t.hits, t.perm, t.rep, threadIdx.x, blockDim.x);
}

// Seam join of the FP32 tracer by a grid, one CTA per seam.  The later sub-range's first row B
// is binned into square cells of side h over its bounding box (about 2 roots per cell, at most
// SEAM_G^2 cells) in scratch that the tracer no longer needs (the work area of sub-range s);
// each root q of the seam row then looks at the 3x3 cells around its own.  Any root of B closer
// than 0.9 h to q lies in those cells (FP32 cell assignment errs far below 0.1 h), so the nearest
// root, with the full scan's tie rule (the lowest index among equal distances), is the full
// scan's whenever it is closer than 0.9 h, and the ambiguity test is settled whenever the best
// distance is below 1e-4 of min(second found, (0.9 h)^2).  Otherwise, and for a q outside the
// grid or not finite, that q takes the full scan of seam_match_block.
constexpr int SEAM_G = 256;
constexpr int SEAM_T = 512;

// Cells per side of a seam's grid: about 2 roots per cell, at most SEAM_G.
static int seam_grid_cells(int64_t nr) {
    return (int)std::max<int64_t>(1, std::min<int64_t>(SEAM_G, (int64_t)std::ceil(std::sqrt(0.5 * (double)nr))));
}

__device__ __forceinline__ void seam_consider(float2 b, float2 q, int j, float& best, float& second, int& bi) {
    const float dx = b.x - q.x, dy = b.y - q.y;  // (this unit contracts no a*b + c: as the full scan)
    const float d2 = dx * dx + dy * dy;
    if (d2 < best || (d2 == best && j < bi)) {
        second = best;
        best = d2;
        bi = j;
    } else if (d2 < second) {
        second = d2;
    }
}

__global__ void __launch_bounds__(SEAM_T) seam_grid_kernel(const float2* zrows, const float2* seam, int64_t m, int S,
                                                           int nr, int G, char* work, size_t work_stride,
                                                           int32_t* match, int32_t* hits, DevReport* rep) {
    __shared__ float s_box[4][SEAM_T / 32];
    __shared__ float s_g[4];  // x0, y0, 1/h, h
    __shared__ int s_scan[32];
    __shared__ int s_amb;
    const int tid = threadIdx.x, P = blockDim.x, lane = tid & 31, wid = tid >> 5, nw = P >> 5;
    const int s = blockIdx.x;
    const float2* B = zrows + (size_t)subchain_begin(s + 1, m, S) * nr;
    const float2* Q = seam + (size_t)s * nr;
    // G: cells per side, from seam_grid_cells (the size the host checked the scratch for)
    const int nc = G * G;
    float2* pos = (float2*)(work + (size_t)s * work_stride);
    int* idx = (int*)(pos + nr);
    int* cst = idx + nr;   // nc + 1 cell starts
    int* fill = cst + nc + 1;
    // bounding box of the finite roots of B
    float b[4] = {3.0e38f, 3.0e38f, 3.0e38f, 3.0e38f};  // min x, min y, -max x, -max y
    for (int j = tid; j < nr; j += P) {
        const float2 v = B[j];
        if (isfinite(v.x) && isfinite(v.y)) {
            b[0] = fminf(b[0], v.x);
            b[1] = fminf(b[1], v.y);
            b[2] = fminf(b[2], -v.x);
            b[3] = fminf(b[3], -v.y);
        }
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        for (int o = 16; o > 0; o >>= 1) b[q] = fminf(b[q], __shfl_xor_sync(0xffffffffu, b[q], o));
        if (lane == 0) s_box[q][wid] = b[q];
    }
    if (tid == 0) s_amb = 0;
    __syncthreads();
    if (tid == 0) {
        for (int w = 1; w < nw; w++)
            for (int q = 0; q < 4; q++) b[q] = fminf(b[q], s_box[q][w]);
        const float span = fmaxf(fmaxf(-b[2] - b[0], -b[3] - b[1]), 0.f);
        float h = span > 0.f && span < 1.0e38f ? span / (float)G * (1.f + 1.f / 1024.f) : 1.f;
        if (!(h > 0.f)) h = 1.f;
        s_g[0] = b[0] <= -b[2] ? b[0] : 0.f;
        s_g[1] = b[1] <= -b[3] ? b[1] : 0.f;
        s_g[2] = 1.f / h;
        s_g[3] = h;
    }
    for (int c = tid; c < nc; c += P) fill[c] = 0;
    __syncthreads();
    const float x0 = s_g[0], y0 = s_g[1], ih = s_g[2], h = s_g[3];
    auto cell_of = [&](float2 v, int& cx, int& cy) -> bool {
        const float fx = (v.x - x0) * ih, fy = (v.y - y0) * ih;
        if (!(fx >= 0.f && fy >= 0.f && fx < (float)G && fy < (float)G)) return false;
        cx = min((int)fx, G - 1);
        cy = min((int)fy, G - 1);
        return true;
    };
    for (int j = tid; j < nr; j += P) {
        int cx, cy;
        if (cell_of(B[j], cx, cy)) atomicAdd(&fill[cy * G + cx], 1);
    }
    __syncthreads();
    for (int c = tid; c < nc; c += P) cst[c + 1] = fill[c];
    if (tid == 0) cst[0] = 0;
    __syncthreads();
    block_scan_inclusive(cst + 1, nc, s_scan);
    for (int c = tid; c < nc; c += P) fill[c] = 0;
    __syncthreads();
    for (int j = tid; j < nr; j += P) {
        const float2 v = B[j];
        int cx, cy;
        if (cell_of(v, cx, cy)) {
            const int c = cy * G + cx;
            const int at = cst[c] + atomicAdd(&fill[c], 1);
            idx[at] = j;
            pos[at] = v;
        }
    }
    __syncthreads();
    const float lim = 0.81f * h * h;  // (0.9 h)^2
    int amb = 0;
    for (int k = tid; k < nr; k += P) {
        const float2 q = Q[k];
        float best = 3.0e38f, second = 3.0e38f;
        int bi = 0;
        int cx, cy;
        bool full = !cell_of(q, cx, cy);
        if (!full) {
            for (int yy = max(cy - 1, 0); yy <= min(cy + 1, G - 1); yy++) {
                const int a = cst[yy * G + max(cx - 1, 0)], e = cst[yy * G + min(cx + 1, G - 1) + 1];
                for (int t = a; t < e; t++) seam_consider(pos[t], q, idx[t], best, second, bi);
            }
            full = !(best < lim) || !(best <= 1e-4f * fminf(second, lim));
        }
        if (full) {
            best = 3.0e38f;
            second = 3.0e38f;
            bi = 0;
            for (int j = 0; j < nr; j++) {
                const float2 v = B[j];
                const float dx = v.x - q.x, dy = v.y - q.y;
                const float d2 = dx * dx + dy * dy;
                if (d2 < best) {
                    second = best;
                    best = d2;
                    bi = j;
                } else if (d2 < second) {
                    second = d2;
                }
            }
        }
        match[(size_t)s * nr + k] = bi;
        atomicAdd(&hits[(size_t)s * nr + bi], 1);
        amb += !(best <= 1e-4f * second);
    }
    if (amb) atomicAdd(&s_amb, amb);
    __syncthreads();
    if (tid == 0 && s_amb) atomicAdd(&rep->seam_ambiguous, (unsigned long long)s_amb);
}

// Chain permutations in three passes over blocks of SEAM_BLK seams: each block's composition
// L_b = match_(e-1) o ... o match_(b0), then the block starts perm_(b0) in sequence, then each
// block's rows: 2 SEAM_BLK + S / SEAM_BLK dependent gathers per column instead of S.
constexpr int SEAM_BLK = 16;

__global__ void compose_local_kernel(int S, int nr, const int32_t* match, const int32_t* hits, int32_t* local,
                                     DevReport* rep) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x, bk = blockIdx.y;
    const int s0 = bk * SEAM_BLK, s1 = min(S - 1, s0 + SEAM_BLK);
    int bad = 0;
    if (g < nr) {
        int p = g;
        for (int s = s0; s < s1; s++) {
            p = match[(size_t)s * nr + p];
            bad += hits[(size_t)s * nr + g] != 1;
        }
        local[(size_t)bk * nr + g] = p;
    }
    for (int o = 16; o > 0; o >>= 1) bad += __shfl_xor_sync(0xffffffffu, bad, o);
    if ((threadIdx.x & 31) == 0 && bad) atomicAdd(&rep->seam_ambiguous, (unsigned long long)bad);
}

__global__ void compose_starts_kernel(int nb, int nr, const int32_t* local, int32_t* start) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nr) return;
    int p = g;
    start[g] = p;
    for (int bk = 0; bk < nb; bk++) {
        p = local[(size_t)bk * nr + p];
        start[(size_t)(bk + 1) * nr + g] = p;
    }
}

__global__ void compose_fill_kernel(int S, int nr, const int32_t* match, const int32_t* start, int32_t* perm) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x, bk = blockIdx.y;
    if (g >= nr) return;
    const int s0 = bk * SEAM_BLK, s1 = min(S - 1, s0 + SEAM_BLK);
    int p = start[(size_t)bk * nr + g];
    if (bk == 0) perm[g] = g;
    for (int s = s0; s < s1; s++) {
        p = match[(size_t)s * nr + p];
        perm[(size_t)(s + 1) * nr + g] = p;
    }
}

cudaError_t launch_seam_join(const void* zrows, const void* seam, int64_t m, int S, int64_t nr,
                             bool fp64, int32_t* match, int32_t* hits, int32_t* perm,
                             DevReport* rep, cudaStream_t st, void* work, size_t work_stride) {
    // the FP32 form joins through a grid in the sub-ranges' work areas (free once traced)
    const bool grid_ok = !fp64 && work && work_stride >= seam_grid_bytes(nr) &&
                         work_stride >= (size_t)(2 * ((S - 1 + SEAM_BLK - 1) / SEAM_BLK) + 1) * nr * sizeof(int32_t);
    if (S > 1) {
        cudaError_t e = cudaMemsetAsync(hits, 0, sizeof(int32_t) * (size_t)(S - 1) * nr, st);
        if (e != cudaSuccess) return e;
        if (grid_ok) {
            seam_grid_kernel<<<(unsigned)(S - 1), SEAM_T, 0, st>>>((const float2*)zrows, (const float2*)seam, m, S,
                                                                 (int)nr, seam_grid_cells(nr), (char*)work,
                                                                 work_stride, match, hits, rep);
        } else {
            dim3 grid((unsigned)((nr + 255) / 256), (unsigned)(S - 1));
            if (fp64)
                seam_match_kernel<double2, double><<<grid, 256, 0, st>>>((const double2*)zrows, (const double2*)seam,
                                                                  m, S, (int)nr, match, hits, rep);
            else
                seam_match_kernel<float2, float><<<grid, 256, 0, st>>>((const float2*)zrows, (const float2*)seam,
                                                                 m, S, (int)nr, match, hits, rep);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (grid_ok && S > 1) {
        // (work area 0 again: the grids are done by stream order)
        const int nb = (S - 1 + SEAM_BLK - 1) / SEAM_BLK;
        int32_t* local = (int32_t*)work;
        int32_t* start = local + (size_t)nb * nr;
        const dim3 g2((unsigned)((nr + 127) / 128), (unsigned)nb);
        compose_local_kernel<<<g2, 128, 0, st>>>(S, (int)nr, match, hits, local, rep);
        compose_starts_kernel<<<(unsigned)((nr + 127) / 128), 128, 0, st>>>(nb, (int)nr, local, start);
        compose_fill_kernel<<<g2, 128, 0, st>>>(S, (int)nr, match, start, perm);
        return cudaGetLastError();
    }
    compose_perm_kernel<<<(unsigned)((nr + 127) / 128), 128, 0, st>>>(S, (int)nr, match, hits, perm, rep);
    return cudaGetLastError();
}

// Scratch of one seam's grid: positions and indices of the row, cell starts and counters.
size_t seam_grid_bytes(int64_t nr) {
    const int64_t G = seam_grid_cells(nr);
    return (size_t)nr * (sizeof(float2) + sizeof(int)) + (size_t)(2 * G * G + 1) * sizeof(int);
}

// ----------------------------------------------------------------------------------
// Rescue of points the polish could not certify: one warp per point runs FP64 Aberth
// (the paper's arithmetic, stop at |dz| < tol_abs) on that root alone, the other roots of
// its row held at their polished positions (Aberth's root sum keeps it from the others'
// basins), then recomputes its caustic point with the FP64 lens equation.  An empty list
// costs one small launch.
// ----------------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(256) rescue_kernel(RescueTask t0, const RescueTask* tasks, const int4* list,
                                                      const int* nlist, int max_list, double tol_abs, int max_iter) {
    const int lane = threadIdx.x & 31;
    const int nwarp = (gridDim.x * blockDim.x) >> 5;
    const int nl = min(*nlist, max_list);
    for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < nl; e += nwarp) {
        const int4 ent = list[e];
        const RescueTask& t = tasks ? tasks[ent.x] : t0;
        const int64_t row = ent.y;
        const int col = ent.z;
        const int nr = t.nr, n = t.n;
        const double2* zr = t.z + (size_t)row * nr;
        double zx = zr[col].x, zy = zr[col].y;
        const double oms = 1.0 - t.kappa_s;
        const double2 ph = t.phase[row];
        bool conv = false;
        for (int it = 0; it < max_iter && !conv; it++) {
            double Cx = 0, Cy = 0, Ax = 0, Ay = 0, Bx = 0, By = 0, Dx = 0, Dy = 0;
            for (int i = lane; i < n; i += 32) {
                const StarD st = t.stars[i];
                const double dx = zx - st.x, dy = zy - st.y;
                const double inv = 1.0 / (dx * dx + dy * dy);
                const double ux = dx * inv, uy = -dy * inv;
                Cx += ux;
                Cy += uy;
                const double tx = ux * ux - uy * uy, ty = 2.0 * ux * uy;
                const double mx = st.z * tx, my = st.z * ty;
                Ax += mx;
                Ay += my;
                Bx += mx * ux - my * uy;
                By += mx * uy + my * ux;
            }
            for (int r = lane; r < nr; r += 32) {
                if (r == col) continue;
                const double2 q = zr[r];
                const double dx = zx - q.x, dy = zy - q.y;
                const double r2 = dx * dx + dy * dy;
                if (r2 > 0.0) {
                    Dx += dx / r2;
                    Dy -= dy / r2;
                }
            }
            Cx = warp_sum_d(Cx);
            Cy = warp_sum_d(Cy);
            Ax = warp_sum_d(Ax);
            Ay = warp_sum_d(Ay);
            Bx = warp_sum_d(Bx);
            By = warp_sum_d(By);
            Dx = warp_sum_d(Dx);
            Dy = warp_sum_d(Dy);
            double Fx = t.gamma + Ax - oms * ph.x, Fy = Ay + oms * ph.y;
            double dFx = -2.0 * Bx, dFy = -2.0 * By;
            if (t.poly) {
                double Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa;
                poly_eval<double>(t.poly, zx, zy, Qx, Qy, Q1x, Q1y, Q2x, Q2y, qa);
                Fx -= Qx;
                Fy -= Qy;
                dFx -= Q1x;
                dFy -= Q1y;
            }
            if (Fx == 0.0 && Fy == 0.0) {
                conv = true;
                break;
            }
            const double fd = Fx * Fx + Fy * Fy;
            const double px = (dFx * Fx + dFy * Fy) / fd + 2.0 * Cx - Dx;
            const double py = (dFy * Fx - dFx * Fy) / fd + 2.0 * Cy - Dy;
            const double pd = px * px + py * py;
            const double delx = px / pd, dely = -py / pd;
            zx -= delx;
            zy -= dely;
            conv = delx * delx + dely * dely < tol_abs * tol_abs;
        }
        // caustic point of the new position: w = (1-kappa_s) z + gamma conj(z) - conj(sum m/(z - z_i))
        double Sx = 0, Sy = 0;
        for (int i = lane; i < n; i += 32) {
            const StarD st = t.stars[i];
            const double dx = zx - st.x, dy = zy - st.y;
            const double q = st.z / (dx * dx + dy * dy);
            Sx += q * dx;
            Sy -= q * dy;
        }
        Sx = warp_sum_d(Sx);
        Sy = warp_sum_d(Sy);
        if (lane == 0) {
            t.z[(size_t)row * nr + col] = make_double2(zx, zy);
            double Vx = 0.0, Vy = 0.0;
            if (t.poly) {
                const double2 V = poly_V(t.poly, zx, zy);
                Vx = V.x;
                Vy = V.y;
            }
            if (t.w)
                t.w[(size_t)row * nr + col] =
                    make_double2(oms * zx + t.gamma * zx - Sx + Vx, oms * zy - t.gamma * zy + Sy + Vy);
            if (conv) {
                atomicAdd(&t.rep->uncertified, (unsigned long long)(-1LL));
                atomicAdd(&t.rep->rescued_points, 1ull);
            }
        }
    }
}

cudaError_t launch_rescue(const RescueTask* host_task, const RescueTask* dev_tasks, const int4* list, const int* nlist,
                          int max_list, double tol_abs, int max_iter, cudaStream_t st) {
    RescueTask t0;
    memset(&t0, 0, sizeof t0);
    if (host_task) t0 = *host_task;
    rescue_kernel<<<64, 256, 0, st>>>(t0, dev_tasks, list, nlist, max_list, tol_abs, max_iter);
    return cudaGetLastError();
}

cudaError_t launch_trace_batch(const BatchTraceArgs& b, int grid, int threads, cudaStream_t st) {
    const size_t smem = tracer_smem_bytes(false, (int64_t)CT<float>::TS, b.near_cap);
    cudaError_t e = cudaFuncSetAttribute(trace_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    BatchTraceArgs a = b;
    a.near_ext = tracer_near_ext((int64_t)CT<float>::TS, b.near_cap) ? 1 : 0;  // as the size above
    trace_batch_kernel<float><<<grid, threads, smem, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_seam_join_batch(const TraceTask* tasks, int count, const int2* seams, int nseams, int max_nr,
                                   cudaStream_t st) {
    if (nseams > 0) {
        dim3 grid((unsigned)((max_nr + 255) / 256), (unsigned)nseams);
        seam_match_batch_kernel<<<grid, 256, 0, st>>>(tasks, seams);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    compose_perm_batch_kernel<<<count, 1024, 0, st>>>(tasks);
    return cudaGetLastError();
}

int tracer_batch_blocks_per_sm(int threads, int near_cap) {
    int b = 0;
    const size_t smem = tracer_smem_bytes(false, (int64_t)CT<float>::TS, near_cap);
    cudaError_t e = cudaFuncSetAttribute(trace_batch_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, trace_batch_kernel<float>, threads, smem);
    if (e != cudaSuccess || b < 1) {
        cudaGetLastError();
        b = 1;
    }
    return b;
}

__global__ void phase_batch_kernel(const TraceTask* tasks, int count) {
    const TraceTask& t = tasks[blockIdx.y];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j > t.m) return;
    const double p = 2.0 * 3.14159265358979323846 * (double)j / (double)t.m;
    double sn, cs;
    sincos(p, &sn, &cs);
    ((double2*)t.phase)[j] = make_double2(cs, sn);
}

cudaError_t launch_phase_batch(const TraceTask* tasks, int count, int64_t max_m, cudaStream_t st) {
    dim3 grid((unsigned)((max_m + 1 + 255) / 256), (unsigned)count);
    phase_batch_kernel<<<grid, 256, 0, st>>>(tasks, count);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------------
// Tracer far-field tables (built once per field): one warp per cell.  Near stars (the 5x5
// block of cells around it) are listed in star order; every other star (at least 2.5
// cells from the centre, while a root in the cell is within 0.71 cells) adds to the FP32
// local expansions U_k = -sum 1/(z_i - c)^(k+1) and L_k = -sum m_i/(z_i - c)^(k+1); the
// table keeps U_k and the coefficients S1'_k = (k + 1) L_(k+1) of the derivative of S1, packed
// as far_eval reads them.
// ----------------------------------------------------------------------------------
__global__ void tracer_far_field_kernel(const float4* s32, int n, TfmmParams P, TCell* cells, int* near,
                                        float4* coeff) {
    const int lane = threadIdx.x & 31;
    const int cell = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (cell >= P.nbx * P.nby) return;  // whole warp
    const int bx = cell % P.nbx, by = cell / P.nbx;
    const float cx = P.x0 + ((float)bx + 0.5f) * P.b, cy = P.y0 + ((float)by + 0.5f) * P.b;
    float ux[TFMM_P], uy[TFMM_P], lx[TFMM_P], ly[TFMM_P];
#pragma unroll
    for (int k = 0; k < TFMM_P; k++) ux[k] = uy[k] = lx[k] = ly[k] = 0.f;
    float r2 = 0.f;
    int cnt = 0;
    bool over = false;
    for (int j0 = 0; j0 < n; j0 += 32) {
        const int j = j0 + lane;
        bool nr_ = false;
        float4 sp = make_float4(0.f, 0.f, 0.f, 0.f);
        if (j < n) {
            sp = s32[j];
            const int sx = (int)fminf(fmaxf(floorf((sp.x - P.x0) * P.inv_b), -1e6f), 1e6f);
            const int sy = (int)fminf(fmaxf(floorf((sp.y - P.y0) * P.inv_b), -1e6f), 1e6f);
            nr_ = abs(sx - bx) <= 2 && abs(sy - by) <= 2;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, nr_);
        if (nr_) {
            const int q = cnt + __popc(bal & ((1u << lane) - 1u));
            if (q < TFMM_NEAR_MAX) near[(size_t)cell * TFMM_NEAR_MAX + q] = j;
        }
        cnt += __popc(bal);
        if (j < n && !nr_) {
            const float dx = sp.x - cx, dy = sp.y - cy;
            const float d2 = dx * dx + dy * dy;
            const float inv = 1.0f / d2;
            const float vx = dx * inv, vy = -dy * inv;  // 1/(z_i - c)
            float wx = vx, wy = vy;
            r2 += sp.z * inv;
#pragma unroll
            for (int k = 0; k < TFMM_P; k++) {
                ux[k] -= wx;
                uy[k] -= wy;
                lx[k] = fmaf(-sp.z, wx, lx[k]);
                ly[k] = fmaf(-sp.z, wy, ly[k]);
                const float nx = wx * vx - wy * vy, ny = wx * vy + wy * vx;
                wx = nx;
                wy = ny;
            }
        }
    }
    over = cnt > TFMM_NEAR_MAX;
#pragma unroll
    for (int k = 0; k < TFMM_P; k++) {
        for (int off = 16; off > 0; off >>= 1) {
            ux[k] += __shfl_xor_sync(0xffffffffu, ux[k], off);
            uy[k] += __shfl_xor_sync(0xffffffffu, uy[k], off);
            lx[k] += __shfl_xor_sync(0xffffffffu, lx[k], off);
            ly[k] += __shfl_xor_sync(0xffffffffu, ly[k], off);
        }
    }
    for (int off = 16; off > 0; off >>= 1) r2 += __shfl_xor_sync(0xffffffffu, r2, off);
    if (lane < TFMM_P) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = 0; k < TFMM_P; k++)
            if (k == lane) {
                const float dx = k + 1 < TFMM_P ? (float)(k + 1) * lx[k + 1 < TFMM_P ? k + 1 : k] : 0.f;
                const float dy = k + 1 < TFMM_P ? (float)(k + 1) * ly[k + 1 < TFMM_P ? k + 1 : k] : 0.f;
                v = make_float4(ux[k], dx, uy[k], dy);
            }
        coeff[(size_t)cell * TFMM_P + lane] = v;
    }
    if (lane == 0) {
        TCell c;
        c.cx = cx;
        c.cy = cy;
        c.near_cnt = over ? -1 : cnt;
        c.far_m_d2 = r2;
        cells[cell] = c;
    }
}

cudaError_t launch_tracer_far_field(const float4* s32, int n, const TfmmParams& P, TCell* cells, int* near,
                                    float4* coeff, cudaStream_t st) {
    const int64_t threads = (int64_t)P.nbx * P.nby * 32;
    tracer_far_field_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(s32, n, P, cells, near, coeff);
    return cudaGetLastError();
}

// cos(phi_j), sin(phi_j) with phi_j = 2 pi j / m (Sec. 4.3), FP64.
__global__ void phase_kernel(double2* ph, int64_t m) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j > m) return;
    const double p = 2.0 * 3.14159265358979323846 * (double)j / (double)m;
    double sn, cs;
    sincos(p, &sn, &cs);
    ph[j] = make_double2(cs, sn);
}

cudaError_t launch_phase_table(double2* phase, int64_t m, cudaStream_t st) {
    const int64_t rows = m + 1;
    phase_kernel<<<(unsigned)((rows + 255) / 256), 256, 0, st>>>(phase, m);
    return cudaGetLastError();
}

}  // namespace ccg
