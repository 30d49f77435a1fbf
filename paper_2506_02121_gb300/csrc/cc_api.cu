// C ABI of libccgpu (declared in include/cc.h): argument checks, field set-up, workspace
// layout and the order of kernel launches.  Every compute step runs in the kernels of
// aberth.cu, polish.cu and raster.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "cc_internal.h"

using namespace ccg;

struct cc_field {
    FieldDev dev;
    cc_options opt;
    int device;
    void* block = nullptr;      // the one device allocation of the field
    DevReport* d_rep = nullptr;
    cudaEvent_t ready = nullptr;  // stars and tables on the device
    cudaEvent_t done = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // stage boundaries: start, after trace, after join, end
    bool solved;
    int64_t last_m;
    int last_S;
};

namespace {

thread_local std::string g_err;

int fail(int code, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(CC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CC_CUDA(call, what)                          \
    do {                                             \
        cudaError_t e_ = (call);                     \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

int sm_count(int device) {
    static std::mutex mu;
    static std::vector<int> cache;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)cache.size() <= device) cache.resize(device + 1, 0);
    if (cache[device] == 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || v <= 0) v = 1;
        cache[device] = v;
    }
    return cache[device];
}

// Resident tracing CTAs per SM, per (device, precision, block size); cached.
int tracer_occupancy(int device, bool fp64, int threads, int64_t n) {
    static std::mutex mu;
    static std::vector<std::pair<int64_t, int>> cache;  // (key, CTAs per SM)
    const int64_t ts = std::min<int64_t>(n, 4096);
    const int64_t key = (((int64_t)device * 2 + (fp64 ? 1 : 0)) * 17 + threads / 32) * 8192 + ts;
    std::lock_guard<std::mutex> lk(mu);
    for (const auto& kv : cache)
        if (kv.first == key) return kv.second;
    const int b = tracer_blocks_per_sm(fp64, threads, n);
    cache.push_back({key, b});
    return b;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

// Workspace layout of cc_critical_curves.
CurveLayout curve_layout(const cc_field* f, int64_t m) {
    CurveLayout L;
    const int64_t nr = f->dev.nr;
    const bool fp64 = f->opt.precision == CC_FP64;
    L.elem = fp64 ? sizeof(double2) : sizeof(float2);
    L.threads = f->opt.block_threads > 0 ? f->opt.block_threads : 512;
    L.G = tracer_cluster_size(f->opt, nr, fp64, m, sm_count(f->device));
    if (L.G > 1) {
        // one wave of clusters; a sub-range keeps >= 8 rows
        cc_options o = f->opt;
        o.subchains = f->opt.subchains > 0 ? f->opt.subchains : std::max(1, tracer_max_clusters(L.G, L.threads, fp64));
        L.S = subchain_count(m, nr, o, 1, 1);
    } else {
        L.S = subchain_count(m, nr, f->opt, sm_count(f->device), tracer_occupancy(f->device, fp64, L.threads, f->dev.n));
    }
    L.work_stride = tracer_work_stride(nr, L.elem);
    size_t o = 0;
    L.off_report = o;
    o += align256(sizeof(DevReport));
    L.off_phase = o;
    o += align256(sizeof(double2) * (size_t)(m + 1));
    L.off_zrows = o;
    o += align256(L.elem * (size_t)(m + 1) * nr);
    L.off_seam = o;
    o += align256(L.elem * (size_t)L.S * nr);
    L.off_iters = o;
    o += align256(sizeof(int32_t) * (size_t)(m + 1) * nr);
    L.off_match = o;
    o += align256(sizeof(int32_t) * (size_t)L.S * nr);
    L.off_hits = o;
    o += align256(sizeof(int32_t) * (size_t)L.S * nr);
    L.off_perm = o;
    o += align256(sizeof(int32_t) * (size_t)L.S * nr);
    L.off_list = o;
    o += align256(sizeof(int4) * (size_t)RESCUE_MAX_POINTS);
    L.off_nlist = o;
    o += 256;
    L.off_work = o;
    o += L.work_stride * (size_t)L.S;
    L.off_ext = o;
    o += align256(sizeof(float4) * (size_t)L.S * (size_t)std::max(1, L.G));
    L.fmm = !fp64 && f->opt.far_field && f->opt.hp_arith == CC_HP_DFLOAT && f->dev.n >= FMM_MIN_STARS;
    L.off_fmm = o;
    if (L.fmm) o += align256(fmm_workspace_bytes((m + 1) * nr));
    L.total = o;
    return L;
}

// Copy n doubles from a host or device pointer to host memory.  Host (or unregistered)
// memory is copied directly, so argument checks need no device.
int fetch_host(double* dst, const double* src, int64_t n, const char* what) {
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, src);
    if (e != cudaSuccess) {
        cudaGetLastError();
        memcpy(dst, src, sizeof(double) * (size_t)n);
        return CC_OK;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        e = cudaMemcpy(dst, src, sizeof(double) * (size_t)n, cudaMemcpyDefault);
        if (e != cudaSuccess) return cuda_fail(e, what);
        return CC_OK;
    }
    memcpy(dst, src, sizeof(double) * (size_t)n);
    return CC_OK;
}

bool finite3(double a, double b, double c) { return std::isfinite(a) && std::isfinite(b) && std::isfinite(c); }

// A stream-ordered memory pool per device, owned by the library, for the fields' device
// blocks: a field created and destroyed in a loop reuses cached memory instead of paying
// cudaMalloc / cudaFree and their device-wide synchronisation each time.
cudaError_t field_pool(int device, cudaMemPool_t* pool) {
    static std::mutex mu;
    static std::vector<cudaMemPool_t> pools;
    std::lock_guard<std::mutex> lk(mu);
    if ((int)pools.size() <= device) pools.resize(device + 1, nullptr);
    if (!pools[device]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = device;
        cudaMemPool_t p;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return e;
        uint64_t keep = ~0ull;  // keep freed blocks for reuse
        e = cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        if (e != cudaSuccess) return e;
        pools[device] = p;
    }
    *pool = pools[device];
    return cudaSuccess;
}

}  // namespace

int ccg::api_error(int code, const char* msg) { return fail(code, "%s", msg); }

const FieldDev* ccg::field_dev(const cc_field* f, int* device, cc_options* opt) {
    if (device) *device = f->device;
    if (opt) *opt = f->opt;
    return &f->dev;
}

extern "C" {

int cc_options_default(cc_options* opt) {
    if (!opt) return fail(CC_EINVAL, "cc_options_default: opt is NULL");
    opt->tol_abs = 1e-9;
    opt->mu_max = 0.0;
    opt->tol_cert = 1e-10;
    opt->max_iter_cold = 500;
    opt->max_iter_warm = 200;
    opt->max_polish = 8;
    opt->precision = CC_MIXED;
    opt->hp_arith = CC_HP_DFLOAT;
    opt->subchains = 0;
    opt->predictor = 1;
    opt->block_threads = 0;
    opt->far_field = 1;
    opt->field_shape = CC_FIELD_DISC;
    opt->rect_t = 0;
    opt->kappa_star = 0.0;
    opt->rect_c1 = 0.0;
    opt->rect_c2 = 0.0;
    opt->rect_eps = 1e-9;
    opt->rect_s = 2.0;
    opt->row_ctas = 0;
    opt->root_refresh = 64;
    return CC_OK;
}

namespace {

constexpr double kPi = 3.14159265358979323846;

// Truncation order of the rectangle's logarithm series (Appendix B): the smallest odd
// t >= 3 whose bound (kappa_*/pi) (4/(t+1)) s^-(t+1) |c| (s+1)/(s-1) on the error of alpha_s
// for |z| s < |c| is <= eps, then t + 2 while (t - 1) Arg(c) is within 0.1 pi of a
// multiple of pi (the leading coefficient of the polynomial vanishes or nearly so).
int rect_order(double kappa_star, double c1, double c2, double eps, double s) {
    const double ac = std::hypot(c1, c2), th = std::atan2(c2, c1);
    int t = 3;
    while (t <= CC_RECT_MAX_T &&
           (kappa_star / kPi) * (4.0 / (t + 1)) * std::pow(s, -(double)(t + 1)) * ac * (s + 1.0) / (s - 1.0) > eps)
        t += 2;
    for (; t <= CC_RECT_MAX_T; t += 2) {
        const double r = std::fmod((t - 1) * th, kPi);
        if (r > 0.1 * kPi && r < 0.9 * kPi) break;
    }
    return t;
}

// Coefficients of the rectangle's smooth-sheet polynomial, normalised by |c|.
void rect_poly(double kappa_star, double c1, double c2, int t, SmoothPoly& P) {
    std::memset(&P, 0, sizeof P);
    const double ac = std::hypot(c1, c2), th = std::atan2(c2, c1);
    P.K = (t - 1) / 2;
    P.ac = ac;
    P.inv_ac = 1.0 / ac;
    P.acf = (float)ac;
    P.inv_acf = (float)(1.0 / ac);
    P.inv_acdf = make_float2((float)(1.0 / ac), (float)(1.0 / ac - (double)(float)(1.0 / ac)));
    P.rg = ac;
    for (int k = 0; k <= P.K; k++) {
        const double q = k == 0 ? kappa_star * (1.0 - 4.0 * th / kPi)
                                : -(4.0 * kappa_star / kPi) * std::sin(2.0 * k * th) / (2.0 * k);
        const double v = q / (2.0 * k + 1.0);
        P.q[k] = q;
        P.v[k] = v;
        P.qf[k] = (float)q;
        const float qh = (float)q, vh = (float)v;
        P.qdf[k] = make_float2(qh, (float)(q - (double)qh));
        P.vdf[k] = make_float2(vh, (float)(v - (double)vh));
    }
}

}  // namespace

int cc_field_create(const double* x, const double* y, const double* mass, int64_t n, double kappa_s,
                    double gamma, const cc_options* opt, cc_field** out) {
    if (!out) return fail(CC_EINVAL, "cc_field_create: out is NULL");
    *out = nullptr;
    if (!x || !y || !mass) return fail(CC_EINVAL, "cc_field_create: NULL star array");
    if (n < 1 || n > (int64_t)1 << 26) return fail(CC_EINVAL, "cc_field_create: n = %lld out of range [1, 2^26]", (long long)n);
    if (!std::isfinite(kappa_s) || !std::isfinite(gamma))
        return fail(CC_EINVAL, "cc_field_create: kappa_s and gamma must be finite");
    cc_options o;
    cc_options_default(&o);
    if (opt) o = *opt;
    if (o.field_shape != CC_FIELD_DISC && o.field_shape != CC_FIELD_RECT)
        return fail(CC_EINVAL, "cc_field_create: field_shape must be CC_FIELD_DISC or CC_FIELD_RECT");
    if (std::fabs(1.0 - kappa_s) < 1e-12 ||
        (o.field_shape == CC_FIELD_DISC && std::fabs(std::fabs(1.0 - kappa_s) - std::fabs(gamma)) < 1e-12))
        return fail(CC_EDEGENERATE,
                    "cc_field_create: |1 - kappa_s| = |gamma| (or 1 - kappa_s = 0): a critical point runs to infinity");
    SmoothPoly hpoly;
    std::memset(&hpoly, 0, sizeof hpoly);
    bool rect = o.field_shape == CC_FIELD_RECT;
    if (rect) {
        if (!(o.kappa_star > 0) || !std::isfinite(o.kappa_star) || !(o.rect_c1 > 0) || !(o.rect_c2 > 0) ||
            !std::isfinite(o.rect_c1) || !std::isfinite(o.rect_c2))
            return fail(CC_EINVAL, "cc_field_create: a rectangular field needs kappa_star > 0 and corner c1, c2 > 0");
        int t = o.rect_t;
        if (t == 0) {
            if (!(o.rect_eps > 0) || !(o.rect_s > 1) || !std::isfinite(o.rect_s))
                return fail(CC_EINVAL, "cc_field_create: rect_eps must be > 0 and rect_s > 1");
            t = rect_order(o.kappa_star, o.rect_c1, o.rect_c2, o.rect_eps, o.rect_s);
        }
        if (t < 3 || !(t & 1) || t > CC_RECT_MAX_T)
            return fail(CC_EINVAL, "cc_field_create: rect_t = %d must be odd in [3, %d]", t, CC_RECT_MAX_T);
        if (std::fabs(std::sin((t - 1) * std::atan2(o.rect_c2, o.rect_c1))) < 1e-6)
            return fail(CC_EDEGENERATE,
                        "cc_field_create: (t - 1) Arg(c) is a multiple of pi: the sheet polynomial loses its degree");
        o.rect_t = t;
        rect_poly(o.kappa_star, o.rect_c1, o.rect_c2, t, hpoly);
    }
    if (o.precision != CC_MIXED && o.precision != CC_FP64) return fail(CC_EINVAL, "cc_field_create: bad precision");
    if (o.hp_arith != CC_HP_DFLOAT && o.hp_arith != CC_HP_FP64) return fail(CC_EINVAL, "cc_field_create: bad hp_arith");
    if (!(o.tol_abs > 0) || !(o.tol_cert > 0) || o.max_iter_cold < 1 || o.max_iter_warm < 1 || o.max_polish < 1 ||
        o.mu_max < 0 || o.subchains < 0)
        return fail(CC_EINVAL, "cc_field_create: bad options");
    if (o.far_field != 0 && o.far_field != 1) return fail(CC_EINVAL, "cc_field_create: far_field must be 0 or 1");
    if (o.predictor < 0 || o.predictor > 2) return fail(CC_EINVAL, "cc_field_create: predictor must be 0, 1 or 2");
    if (o.row_ctas < 0 || o.row_ctas > 16) return fail(CC_EINVAL, "cc_field_create: row_ctas must be in [0, 16]");
    if (o.root_refresh < 0 || o.root_refresh > 4096)
        return fail(CC_EINVAL, "cc_field_create: root_refresh must be in [0, 4096]");
    if (o.block_threads != 0 && (o.block_threads < 32 || o.block_threads > 512 || (o.block_threads & 31)))
        return fail(CC_EINVAL, "cc_field_create: block_threads must be 0 or a multiple of 32 in [32, 512]");

    std::vector<double> hx(n), hy(n), hm(n);
    if (int r = fetch_host(hx.data(), x, n, "x")) return r;
    if (int r = fetch_host(hy.data(), y, n, "y")) return r;
    if (int r = fetch_host(hm.data(), mass, n, "mass")) return r;
    bool unit = true;
    for (int64_t i = 0; i < n; i++) {
        if (!finite3(hx[i], hy[i], hm[i])) return fail(CC_EINVAL, "cc_field_create: star %lld is not finite", (long long)i);
        if (!(hm[i] > 0)) return fail(CC_EINVAL, "cc_field_create: star %lld has mass <= 0", (long long)i);
        unit = unit && hm[i] == 1.0;
    }
    std::vector<float4> s32(n), sdp(n);
    std::vector<float2> sdm(n), stf(n);
    std::vector<StarD> s64(n);
    auto split = [](double v, float& hi, float& lo) {
        hi = (float)v;
        lo = (float)(v - (double)hi);
    };
    for (int64_t i = 0; i < n; i++) {
        s32[i] = make_float4((float)hx[i], (float)hy[i], (float)hm[i], 0.f);
        s64[i] = StarD{hx[i], hy[i], hm[i], 0.0};
        float a, b, c, d, e, g;
        split(hx[i], a, b);
        split(hy[i], c, d);
        split(hm[i], e, g);
        sdp[i] = make_float4(a, b, c, d);
        sdm[i] = make_float2(e, g);
        stf[i] = make_float2((float)(hx[i] - (double)a - (double)b), (float)(hy[i] - (double)c - (double)d));
    }
    // far-field cell: about 6 stars in a 5x5 block of cells at the mean star density of the
    // field's bounding disc
    double mx = 0.0, my = 0.0;
    for (int64_t i = 0; i < n; i++) {
        mx += hx[i];
        my += hy[i];
    }
    mx /= (double)n;
    my /= (double)n;
    double r2max = 0.0;
    for (int64_t i = 0; i < n; i++) r2max = std::max(r2max, (hx[i] - mx) * (hx[i] - mx) + (hy[i] - my) * (hy[i] - my));
    const double density = r2max > 0.0 ? (double)n / (3.14159265358979323846 * r2max) : 0.0;
    const float fmm_cell = density > 0.0 ? (float)std::sqrt(6.0 / (25.0 * density)) : 1.0f;
    // tracer far-field grid: cells of the polish cell size over the stars' bounding box
    // plus three cells on every side (roots outside sum every star directly)
    TfmmParams tp;
    std::memset(&tp, 0, sizeof tp);
    size_t tcells = 0;
    if (o.far_field && n >= FMM_MIN_STARS) {
        float xmn = s32[0].x, xmx = s32[0].x, ymn = s32[0].y, ymx = s32[0].y;
        for (int64_t i = 1; i < n; i++) {
            xmn = std::min(xmn, s32[i].x);
            xmx = std::max(xmx, s32[i].x);
            ymn = std::min(ymn, s32[i].y);
            ymx = std::max(ymx, s32[i].y);
        }
        float b = fmm_cell > 0.f ? fmm_cell : 1.0f;
        const float span = std::max(xmx - xmn, ymx - ymn);
        if (span / b + 8.0f > 512.0f) b = span / 504.0f;
        tp.b = b;
        tp.inv_b = 1.0f / b;
        tp.x0 = xmn - 3.0f * b;
        tp.y0 = ymn - 3.0f * b;
        tp.nbx = (int)std::ceil((xmx - tp.x0) * tp.inv_b) + 4;
        tp.nby = (int)std::ceil((ymx - tp.y0) * tp.inv_b) + 4;
        tp.ok = 1;
        tcells = (size_t)tp.nbx * tp.nby;
    }
    // one device block for everything the field holds: the uploaded star layouts (and the
    // rectangle's polynomial) first, then the report and the far-field tables
    size_t off = 0;
    auto region = [&](size_t bytes) {
        const size_t o2 = off;
        off += align256(bytes);
        return o2;
    };
    const size_t o32 = region(sizeof(float4) * n), o64 = region(sizeof(StarD) * n), odp = region(sizeof(float4) * n),
                 odm = region(sizeof(float2) * n), otf = region(sizeof(float2) * n),
                 opoly = rect ? region(sizeof(SmoothPoly)) : off;
    const size_t upload = off;
    const size_t orep = region(sizeof(DevReport)), ocell = region(sizeof(TCell) * tcells),
                 onear = region(sizeof(int) * tcells * TFMM_NEAR_MAX), ocoef = region(sizeof(float4) * tcells * TFMM_P);
    std::vector<unsigned char> host(upload);
    std::memcpy(host.data() + o32, s32.data(), sizeof(float4) * n);
    std::memcpy(host.data() + o64, s64.data(), sizeof(StarD) * n);
    std::memcpy(host.data() + odp, sdp.data(), sizeof(float4) * n);
    std::memcpy(host.data() + odm, sdm.data(), sizeof(float2) * n);
    std::memcpy(host.data() + otf, stf.data(), sizeof(float2) * n);
    if (rect) std::memcpy(host.data() + opoly, &hpoly, sizeof(SmoothPoly));

    cc_field* f = new cc_field();
    f->opt = o;
    f->dev.fmm_cell = fmm_cell;
    f->dev.n = n;
    f->dev.nr = 2 * n + (rect ? 2 * hpoly.K : 0);
    f->dev.poly = nullptr;
    f->dev.poly_K = rect ? hpoly.K : 0;
    f->dev.kappa_s = kappa_s;
    f->dev.gamma = gamma;
    f->dev.unit_mass = unit;
    f->dev.tfmm.ok = 0;
    f->solved = false;
    cudaGetDevice(&f->device);
    cudaMemPool_t pool;
    cudaError_t e = field_pool(f->device, &pool);
    e = e ? e : cudaMallocFromPoolAsync(&f->block, off, pool, 0);
    e = e ? e : cudaEventCreateWithFlags(&f->done, cudaEventDisableTiming);
    e = e ? e : cudaEventCreateWithFlags(&f->ready, cudaEventDisableTiming);
    for (int i = 0; i < 4; i++) e = e ? e : cudaEventCreate(&f->ev[i]);
    if (e != cudaSuccess) {
        cc_field_destroy(f);
        return fail(e == cudaErrorMemoryAllocation ? CC_ENOMEM : CC_ECUDA, "cc_field_create: %s", cudaGetErrorString(e));
    }
    char* base = (char*)f->block;
    f->dev.star32 = (float4*)(base + o32);
    f->dev.star64 = (StarD*)(base + o64);
    f->dev.star_dfp = (float4*)(base + odp);
    f->dev.star_dfm = (float2*)(base + odm);
    f->dev.star_tf = (float2*)(base + otf);
    if (rect) f->dev.poly = (const SmoothPoly*)(base + opoly);
    f->d_rep = (DevReport*)(base + orep);
    // stream 0: ordered with the caller's later work through the ready event, with no
    // host wait here
    e = cudaMemcpyAsync(base, host.data(), upload, cudaMemcpyHostToDevice, 0);
    e = e ? e : cudaMemsetAsync(f->d_rep, 0, sizeof(DevReport), 0);
    if (e == cudaSuccess && tp.ok) {
        f->dev.tcells = (TCell*)(base + ocell);
        f->dev.tnear = (int*)(base + onear);
        f->dev.tcoeff = (float4*)(base + ocoef);
        e = launch_tracer_far_field(f->dev.star32, (int)n, tp, f->dev.tcells, f->dev.tnear, f->dev.tcoeff, 0);
        f->dev.tfmm = tp;
    }
    // (a pageable upload has copied the host buffer by the time cudaMemcpyAsync returns)
    e = e ? e : cudaEventRecord(f->ready, 0);
    f->dev.ready = f->ready;
    if (e != cudaSuccess) {
        cc_field_destroy(f);
        return cuda_fail(e, "cc_field_create upload");
    }
    *out = f;
    return CC_OK;
}

int cc_field_destroy(cc_field* f) {
    if (!f) return CC_OK;
    if (f->done) cudaEventSynchronize(f->done);
    if (f->ready) cudaEventSynchronize(f->ready);
    if (f->block) cudaFreeAsync(f->block, 0);
    if (f->done) cudaEventDestroy(f->done);
    if (f->ready) cudaEventDestroy(f->ready);
    for (int i = 0; i < 4; i++)
        if (f->ev[i]) cudaEventDestroy(f->ev[i]);
    delete f;
    return CC_OK;
}

int cc_field_size(const cc_field* f, int64_t* n_stars, int64_t* n_roots) {
    if (!f) return fail(CC_EINVAL, "cc_field_size: field is NULL");
    if (n_stars) *n_stars = f->dev.n;
    if (n_roots) *n_roots = f->dev.nr;
    return CC_OK;
}

static int check_m(int64_t m) {
    if (m < 2 || (m & 1)) return fail(CC_EINVAL, "m = %lld must be even and >= 2", (long long)m);
    if (m > ((int64_t)1 << 30)) return fail(CC_EINVAL, "m = %lld too large", (long long)m);
    return CC_OK;
}

int cc_critical_curves_workspace_bytes(const cc_field* f, int64_t m, size_t* bytes) {
    if (!f || !bytes) return fail(CC_EINVAL, "cc_critical_curves_workspace_bytes: NULL argument");
    if (int r = check_m(m)) return r;
    *bytes = curve_layout(f, m).total;
    return CC_OK;
}

int cc_critical_curves(cc_field* f, int64_t m, double* z_out, double* w_out, int32_t* iters_out,
                       void* workspace, size_t workspace_bytes, cc_stream_t stream) {
    if (!f) return fail(CC_EINVAL, "cc_critical_curves: field is NULL");
    if (int r = check_m(m)) return r;
    if (!z_out) return fail(CC_EINVAL, "cc_critical_curves: z_out is NULL");
    if (!workspace) return fail(CC_EINVAL, "cc_critical_curves: workspace is NULL");
    if ((uintptr_t)workspace % 256) return fail(CC_EINVAL, "cc_critical_curves: workspace must be 256-byte aligned");
    const CurveLayout L = curve_layout(f, m);
    if (workspace_bytes < L.total)
        return fail(CC_ENOMEM, "cc_critical_curves: workspace has %zu bytes, needs %zu", workspace_bytes, L.total);
    CC_CUDA(cudaSetDevice(f->device), "cudaSetDevice");
    cudaStream_t st = (cudaStream_t)stream;
    CC_CUDA(cudaStreamWaitEvent(st, f->ready, 0), "wait for the field");
    char* ws = (char*)workspace;
    const int64_t nr = f->dev.nr;
    const bool fp64 = f->opt.precision == CC_FP64;
    DevReport* rep = f->d_rep;
    CC_CUDA(cudaMemsetAsync(rep, 0, sizeof(DevReport), st), "clear report");
    double2* phase = (double2*)(ws + L.off_phase);
    CC_CUDA(cudaEventRecord(f->ev[0], st), "event record");
    CC_CUDA(launch_phase_table(phase, m, st), "phase table");
    TraceArgs ta;
    ta.f = &f->dev;
    ta.m = m;
    ta.S = L.S;
    ta.phase = phase;
    ta.zrows = ws + L.off_zrows;
    ta.seam = ws + L.off_seam;
    ta.iters = (int32_t*)(ws + L.off_iters);
    ta.work = ws + L.off_work;
    ta.work_stride = L.work_stride;
    ta.rep = rep;
    ta.tol_abs = f->opt.tol_abs;
    ta.mu_max = f->opt.mu_max;
    ta.max_iter_cold = f->opt.max_iter_cold;
    ta.max_iter_warm = f->opt.max_iter_warm;
    ta.predictor = f->opt.predictor;
    ta.root_refresh = f->opt.root_refresh;
    ta.threads = L.threads;
    ta.cluster = L.G;
    ta.ext = fp64 ? nullptr : (float4*)(ws + L.off_ext);
    CC_CUDA(launch_trace(ta, fp64, st), "trace");
    CC_CUDA(cudaEventRecord(f->ev[1], st), "event record");
    int32_t* perm = (int32_t*)(ws + L.off_perm);
    CC_CUDA(launch_seam_join(ws + L.off_zrows, ws + L.off_seam, m, L.S, nr, fp64, (int32_t*)(ws + L.off_match),
                             (int32_t*)(ws + L.off_hits), perm, rep, st, ws + L.off_work, L.work_stride),
            "seam join");
    CC_CUDA(cudaEventRecord(f->ev[2], st), "event record");
    if (fp64) {
        FinalizeArgs fa;
        fa.m = m;
        fa.S = L.S;
        fa.nr = nr;
        fa.zrows = (const double2*)(ws + L.off_zrows);
        fa.perm = perm;
        fa.iters_in = (const int32_t*)(ws + L.off_iters);
        fa.z_out = (double2*)z_out;
        fa.iters_out = iters_out;
        CC_CUDA(launch_finalize_fp64(fa, st), "finalize");
        if (w_out)
            CC_CUDA(launch_map_caustics(f->dev, (const double2*)z_out, (m + 1) * nr, (double2*)w_out,
                                        f->opt.hp_arith == CC_HP_FP64, st),
                    "map caustics");
    } else {
        PolishArgs pa;
        pa.ext = (const float4*)(ws + L.off_ext);
        pa.ext_n = L.S * std::max(1, L.G);
        pa.f = &f->dev;
        pa.m = m;
        pa.S = L.S;
        pa.nr = nr;
        pa.phase = phase;
        pa.zrows = (const float2*)(ws + L.off_zrows);
        pa.perm = perm;
        pa.iters_in = (const int32_t*)(ws + L.off_iters);
        pa.z_out = (double2*)z_out;
        pa.w_out = (double2*)w_out;
        pa.iters_out = iters_out;
        pa.rep = rep;
        pa.tol_cert = f->opt.tol_cert;
        pa.max_polish = f->opt.max_polish;
        pa.hp_fp64 = f->opt.hp_arith == CC_HP_FP64;
        pa.rescue_list = (int4*)(ws + L.off_list);
        pa.rescue_count = (int*)(ws + L.off_nlist);
        pa.field_id = 0;
        pa.skip_if = nullptr;
        CC_CUDA(cudaMemsetAsync(pa.rescue_count, 0, sizeof(int), st), "clear rescue count");
        if (L.fmm)
            CC_CUDA(launch_polish_fmm(pa, ws + L.off_fmm, st), "far-field polish");
        else
            CC_CUDA(launch_polish(pa, st), "polish");
        RescueTask rt;
        rt.stars = f->dev.star64;
        rt.poly = f->dev.poly;
        rt.n = (int)f->dev.n;
        rt.nr = (int)nr;
        rt.kappa_s = f->dev.kappa_s;
        rt.gamma = f->dev.gamma;
        rt.m = m;
        rt.phase = phase;
        rt.z = (double2*)z_out;
        rt.w = (double2*)w_out;
        rt.rep = rep;
        CC_CUDA(launch_rescue(&rt, nullptr, pa.rescue_list, pa.rescue_count, RESCUE_MAX_POINTS, f->opt.tol_abs,
                              f->opt.max_iter_warm, st),
                "rescue");
    }
    CC_CUDA(cudaEventRecord(f->ev[3], st), "event record");
    CC_CUDA(cudaEventRecord(f->done, st), "event record");
    f->solved = true;
    f->last_m = m;
    f->last_S = L.S;
    return CC_OK;
}

int cc_field_report(cc_field* f, cc_report* out) {
    if (!f || !out) return fail(CC_EINVAL, "cc_field_report: NULL argument");
    if (!f->solved) return fail(CC_EINVAL, "cc_field_report: no cc_critical_curves call on this field yet");
    CC_CUDA(cudaEventSynchronize(f->done), "wait");
    DevReport r;
    CC_CUDA(cudaMemcpy(&r, f->d_rep, sizeof r, cudaMemcpyDeviceToHost), "read report");
    memset(out, 0, sizeof *out);
    out->rows = f->last_m + 1;
    out->n_roots = f->dev.nr;
    out->subchains = f->last_S;
    out->root_iterations = (int64_t)r.root_iterations;
    out->cold_root_iterations = (int64_t)r.cold_root_iterations;
    out->unconverged = (int64_t)r.unconverged;
    out->polish_passes = (int64_t)r.polish_passes;
    out->uncertified = (int64_t)r.uncertified;
    out->seam_ambiguous = (int64_t)r.seam_ambiguous;
    out->max_iter_row = r.max_iter_row;
    out->max_err_est = r.max_err_est;
    out->rescued_points = (int64_t)r.rescued_points;
    out->jumped = (int64_t)r.jumped;
    out->star_terms = (int64_t)r.star_terms;
    out->far_evals = (int64_t)r.far_evals;
    out->root_terms = (int64_t)r.root_terms;
    out->split_redone_rows = (int64_t)r.split_redone_rows;
    CC_CUDA(cudaEventElapsedTime(&out->trace_ms, f->ev[0], f->ev[1]), "stage time");
    CC_CUDA(cudaEventElapsedTime(&out->join_ms, f->ev[1], f->ev[2]), "stage time");
    CC_CUDA(cudaEventElapsedTime(&out->polish_ms, f->ev[2], f->ev[3]), "stage time");
    if (r.unconverged || r.uncertified)
        return fail(CC_ENOCONV, "%lld root-rows hit the iteration cap, %lld points uncertified",
                    (long long)r.unconverged, (long long)r.uncertified);
    return CC_OK;
}

int cc_map_caustics(cc_field* f, const double* z, int64_t count, double* w_out, cc_stream_t stream) {
    if (!f) return fail(CC_EINVAL, "cc_map_caustics: field is NULL");
    if (count < 0) return fail(CC_EINVAL, "cc_map_caustics: count < 0");
    if (count == 0) return CC_OK;
    if (!z || !w_out) return fail(CC_EINVAL, "cc_map_caustics: NULL buffer");
    CC_CUDA(cudaSetDevice(f->device), "cudaSetDevice");
    CC_CUDA(cudaStreamWaitEvent((cudaStream_t)stream, f->ready, 0), "wait for the field");
    CC_CUDA(launch_map_caustics(f->dev, (const double2*)z, count, (double2*)w_out, f->opt.hp_arith == CC_HP_FP64,
                                (cudaStream_t)stream),
            "map caustics");
    return CC_OK;
}

int cc_crossing_map(const double* w, int64_t rows, int64_t n_r, double x0, double x1, double y0, double y1,
                    int32_t W, int32_t H, int32_t* ncc_out, cc_stream_t stream) {
    if (!ncc_out) return fail(CC_EINVAL, "cc_crossing_map: ncc_out is NULL");
    if (W < 1 || H < 1) return fail(CC_EINVAL, "cc_crossing_map: W, H must be >= 1");
    if (!(std::isfinite(x0) && std::isfinite(x1) && std::isfinite(y0) && std::isfinite(y1)) || !(x1 > x0) ||
        !(y1 > y0))
        return fail(CC_EINVAL, "cc_crossing_map: need finite x0 < x1 and y0 < y1");
    if (rows < 0 || n_r < 0) return fail(CC_EINVAL, "cc_crossing_map: rows, n_r must be >= 0");
    if (rows * n_r > 0 && !w) return fail(CC_EINVAL, "cc_crossing_map: w is NULL");
    CC_CUDA(launch_crossing_map((const double2*)w, rows, n_r, x0, x1, y0, y1, W, H, ncc_out, (cudaStream_t)stream),
            "crossing map");
    return CC_OK;
}

int cc_distance_map_workspace_bytes(int32_t W, int32_t H, size_t* bytes) {
    if (!bytes || W < 1 || H < 1) return fail(CC_EINVAL, "cc_distance_map_workspace_bytes: bad argument");
    *bytes = distance_workspace_bytes(W, H);
    return CC_OK;
}

int cc_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, double* d_out, void* workspace,
                    size_t workspace_bytes, cc_stream_t stream) {
    if (!ncc || !d_out || !workspace) return fail(CC_EINVAL, "cc_distance_map: NULL buffer");
    if (W < 1 || H < 1) return fail(CC_EINVAL, "cc_distance_map: W, H must be >= 1");
    if (!(pixel > 0) || !std::isfinite(pixel)) return fail(CC_EINVAL, "cc_distance_map: pixel must be finite and > 0");
    if ((uintptr_t)workspace % 256) return fail(CC_EINVAL, "cc_distance_map: workspace must be 256-byte aligned");
    if (workspace_bytes < distance_workspace_bytes(W, H))
        return fail(CC_ENOMEM, "cc_distance_map: workspace has %zu bytes, needs %zu", workspace_bytes,
                    distance_workspace_bytes(W, H));
    CC_CUDA(launch_distance_map(ncc, W, H, pixel, d_out, workspace, (cudaStream_t)stream), "distance map");
    return CC_OK;
}

int cc_moving_distance_map(const int32_t* ncc, int32_t W, int32_t H, double pixel, double angle, double* d_out,
                           cc_stream_t stream) {
    if (!ncc || !d_out) return fail(CC_EINVAL, "cc_moving_distance_map: NULL buffer");
    if (W < 1 || H < 1) return fail(CC_EINVAL, "cc_moving_distance_map: W, H must be >= 1");
    if (!(pixel > 0) || !std::isfinite(pixel)) return fail(CC_EINVAL, "cc_moving_distance_map: pixel must be finite and > 0");
    if (!std::isfinite(angle)) return fail(CC_EINVAL, "cc_moving_distance_map: angle must be finite");
    const float c = (float)std::cos(angle), s = (float)std::sin(angle);
    CC_CUDA(launch_moving_distance_map(ncc, W, H, pixel, c, s, d_out, (cudaStream_t)stream), "moving distance map");
    return CC_OK;
}

const char* cc_last_error(void) { return g_err.c_str(); }

const char* cc_version(void) { return "ccgpu 0.1 (sm_103a)"; }

}  // extern "C"
