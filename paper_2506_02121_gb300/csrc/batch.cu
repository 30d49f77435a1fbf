// Batched critical curves: many fields of uneven N in one persistent tracing launch, one
// batched seam join, then the polish (far-field polish per field for fields with enough
// stars, one batched direct polish for the rest), optionally replayed as a CUDA graph.
//
// Work items are (field, sub-range) pairs.  Each field gets a number of phi sub-ranges in
// proportion to its estimated work (rows x n_r x (N + n_r)), so that items are of similar
// size, and the items are handed out most expensive first (longest-processing-time order)
// from a global counter to the resident CTAs of one persistent launch.  Tables, scratch
// and per-field reports all live in the caller's workspace; the library allocates nothing
// after cc_batch_create.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "cc_internal.h"

using namespace ccg;


struct cc_batch {
    int count = 0;
    std::vector<const cc_field*> fields;
    std::vector<FieldDev> dev;
    std::vector<int64_t> m, nr, rows;
    std::vector<int> S;
    int device = 0;
    cc_options opt;
    int threads = 512, grid = 1;
    int nitems = 0, nseams = 0, max_nr = 0;
    int near_cap = 0;  // rows of up to near_cap roots keep the tracer's split in shared memory
    int64_t max_m = 0, total_blocks = 0;
    // workspace layout
    std::vector<size_t> off_phase, off_zrows, off_seam, off_iters, off_match, off_perm, off_hits;
    size_t hits_begin = 0, hits_bytes = 0;
    size_t off_rtasks = 0, off_list = 0, off_nlist = 0;
    size_t off_tasks = 0, off_items = 0, off_seams = 0, off_ptasks = 0, off_reps = 0, off_queue = 0, off_work = 0;
    // far-field polish: fields with enough stars run it one after another in stream order,
    // sharing one scratch region; the others share one batched direct polish launch
    std::vector<char> use_fmm;
    std::vector<PolishArgs> fmm_args;
    size_t off_fmm = 0;
    int direct_count = 0;
    size_t work_stride = 0, total = 0;
    // bound buffers
    bool bound = false;
    char* ws = nullptr;
    // graph
    bool graph_ok = false;
    cudaStream_t graph_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool launched = false;
    cudaStream_t last_stream = nullptr;
};

namespace {

size_t a256(size_t x) { return (x + 255) / 256 * 256; }

int berr(int code, const char* msg) { return api_error(code, msg); }

void drop_graph(cc_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->graph_ok = false;
}

// Event records inside a stream capture become external event-record nodes, so that they
// also fire when the graph is replayed.
cudaError_t rec(cudaEvent_t ev, cudaStream_t st, bool capturing) {
    return capturing ? cudaEventRecordWithFlags(ev, st, cudaEventRecordExternal) : cudaEventRecord(ev, st);
}

cudaError_t enqueue(cc_batch* b, cudaStream_t st, bool capturing) {
    char* ws = b->ws;
    cudaError_t e;
    if ((e = rec(b->ev[0], st, capturing)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + b->off_reps, 0, sizeof(DevReport) * b->count, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + b->off_queue, 0, 256, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + b->hits_begin, 0, b->hits_bytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(ws + b->off_nlist, 0, 256, st)) != cudaSuccess) return e;
    const TraceTask* tasks = (const TraceTask*)(ws + b->off_tasks);
    if ((e = launch_phase_batch(tasks, b->count, b->max_m, st)) != cudaSuccess) return e;
    BatchTraceArgs a;
    a.tasks = tasks;
    a.items = (const int2*)(ws + b->off_items);
    a.nitems = b->nitems;
    a.queue = (unsigned int*)(ws + b->off_queue);
    a.work = ws + b->off_work;
    a.work_stride = b->work_stride;
    a.tol_abs = b->opt.tol_abs;
    a.max_iter_cold = b->opt.max_iter_cold;
    a.max_iter_warm = b->opt.max_iter_warm;
    a.predictor = b->opt.predictor;
    a.root_refresh = b->opt.root_refresh;
    a.near_cap = b->near_cap;
    a.near_ext = 0;  // set by launch_trace_batch
    if ((e = launch_trace_batch(a, b->grid, b->threads, st)) != cudaSuccess) return e;
    if ((e = rec(b->ev[1], st, capturing)) != cudaSuccess) return e;
    if ((e = launch_seam_join_batch(tasks, b->count, (const int2*)(ws + b->off_seams), b->nseams, b->max_nr, st)) !=
        cudaSuccess)
        return e;
    if ((e = rec(b->ev[2], st, capturing)) != cudaSuccess) return e;
    if (b->direct_count > 0 &&
        (e = launch_polish_batch(ws + b->off_ptasks, b->direct_count, b->total_blocks, st)) != cudaSuccess)
        return e;
    for (const PolishArgs& pa : b->fmm_args)
        if ((e = launch_polish_fmm(pa, ws + b->off_fmm, st)) != cudaSuccess) return e;
    if ((e = launch_rescue(nullptr, (const RescueTask*)(ws + b->off_rtasks), (const int4*)(ws + b->off_list),
                           (const int*)(ws + b->off_nlist), RESCUE_MAX_POINTS, b->opt.tol_abs, b->opt.max_iter_warm, st)) !=
        cudaSuccess)
        return e;
    return rec(b->ev[3], st, capturing);
}

}  // namespace

extern "C" {

int cc_batch_create(cc_field* const* fields, int32_t count, const int64_t* m, int32_t block_threads,
                    int32_t items_per_cta, cc_batch** out) {
    if (!out) return berr(CC_EINVAL, "cc_batch_create: out is NULL");
    *out = nullptr;
    if (!fields || !m || count < 1) return berr(CC_EINVAL, "cc_batch_create: need count >= 1 fields and m values");
    if (block_threads != 0 && (block_threads < 32 || block_threads > 512 || (block_threads & 31)))
        return berr(CC_EINVAL, "cc_batch_create: block_threads must be 0 or a multiple of 32 in [32, 512]");
    if (items_per_cta < 0 || items_per_cta > 64) return berr(CC_EINVAL, "cc_batch_create: items_per_cta in [0, 64]");
    cc_batch* b = new cc_batch();
    b->count = count;
    double total_cost = 0;
    std::vector<double> cost(count);
    for (int f = 0; f < count; f++) {
        if (!fields[f]) {
            delete b;
            return berr(CC_EINVAL, "cc_batch_create: NULL field");
        }
        int dev = 0;
        cc_options o;
        const FieldDev* fd = field_dev(fields[f], &dev, &o);
        if (o.precision != CC_MIXED) {
            delete b;
            return berr(CC_EINVAL, "cc_batch_create: batched launches use the mixed (FP32 + polish) form");
        }
        if (m[f] < 2 || (m[f] & 1) || m[f] > ((int64_t)1 << 30)) {
            delete b;
            return berr(CC_EINVAL, "cc_batch_create: every m must be even and >= 2");
        }
        if (f == 0) {
            b->device = dev;
            b->opt = o;
        } else if (dev != b->device) {
            delete b;
            return berr(CC_EINVAL, "cc_batch_create: all fields must live on one device");
        }
        // the field's uploads and tables were enqueued on stream 0: finished before any
        // batched launch (which may be captured into a graph)
        if (fd->ready && cudaEventSynchronize(fd->ready) != cudaSuccess) {
            delete b;
            return berr(CC_ECUDA, "cc_batch_create: field set-up failed");
        }
        b->fields.push_back(fields[f]);
        b->dev.push_back(*fd);
        b->m.push_back(m[f]);
        b->nr.push_back(fd->nr);
        b->rows.push_back(m[f] + 1);
        cost[f] = (double)(m[f] + 1) * (double)fd->nr * (double)(fd->n + fd->nr);
        total_cost += cost[f];
        b->max_nr = std::max<int>(b->max_nr, (int)fd->nr);
        b->max_m = std::max<int64_t>(b->max_m, m[f]);
    }
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) {
        delete b;
        return berr(CC_ECUDA, "cc_batch_create: cudaSetDevice failed");
    }
    b->threads = block_threads > 0 ? block_threads : (b->opt.block_threads > 0 ? b->opt.block_threads : 512);
    int sms = 1;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->near_cap = b->opt.root_refresh >= 2 ? std::min(b->max_nr, NEAR_SMEM_NR) : 0;
    b->grid = sms * tracer_batch_blocks_per_sm(b->threads, b->near_cap);
    // sub-ranges per field: about items_per_cta (default 4) items per resident CTA overall,
    // each field's items of similar size; a sub-range keeps >= 32 rows so its cold start
    // stays a small overhead
    const double target = total_cost / ((items_per_cta > 0 ? items_per_cta : 4) * (double)b->grid);
    for (int f = 0; f < count; f++) {
        int64_t Sf = b->opt.subchains > 0 ? b->opt.subchains : (int64_t)std::ceil(cost[f] / std::max(target, 1.0));
        Sf = std::min<int64_t>(Sf, std::max<int64_t>(1, b->m[f] / 32));
        Sf = std::min<int64_t>(Sf, b->m[f] / 2);
        Sf = std::max<int64_t>(Sf, 1);
        b->S.push_back((int)Sf);
        b->nitems += (int)Sf;
    }
    // workspace layout
    size_t o = 0;
    b->off_reps = o;
    o += a256(sizeof(DevReport) * count);
    b->off_queue = o;
    o += 256;
    b->off_tasks = o;
    o += a256(sizeof(TraceTask) * count);
    b->off_items = o;
    o += a256(sizeof(int2) * b->nitems);
    for (int f = 0; f < count; f++) b->nseams += b->S[f] - 1;
    b->off_seams = o;
    o += a256(sizeof(int2) * std::max(1, b->nseams));
    b->off_ptasks = o;
    o += a256(polish_task_bytes() * count);
    int64_t fmm_points = 0;
    for (int f = 0; f < count; f++) {
        const bool u = b->opt.far_field && b->dev[f].n >= FMM_MIN_STARS;
        b->use_fmm.push_back(u ? 1 : 0);
        if (u) fmm_points = std::max<int64_t>(fmm_points, b->rows[f] * b->nr[f]);
    }
    b->off_fmm = o;
    if (fmm_points > 0) o += a256(fmm_workspace_bytes(fmm_points));
    b->hits_begin = o;
    for (int f = 0; f < count; f++) {
        b->off_hits.push_back(o);
        o += a256(sizeof(int32_t) * (size_t)b->S[f] * b->nr[f]);
    }
    b->hits_bytes = o - b->hits_begin;
    b->off_rtasks = o;
    o += a256(sizeof(RescueTask) * count);
    b->off_list = o;
    o += a256(sizeof(int4) * (size_t)RESCUE_MAX_POINTS);
    b->off_nlist = o;
    o += 256;
    for (int f = 0; f < count; f++) {
        const size_t nrf = (size_t)b->nr[f];
        b->off_phase.push_back(o);
        o += a256(sizeof(double2) * (size_t)b->rows[f]);
        b->off_zrows.push_back(o);
        o += a256(sizeof(float2) * (size_t)b->rows[f] * nrf);
        b->off_seam.push_back(o);
        o += a256(sizeof(float2) * (size_t)b->S[f] * nrf);
        b->off_iters.push_back(o);
        o += a256(sizeof(int32_t) * (size_t)b->rows[f] * nrf);
        b->off_match.push_back(o);
        o += a256(sizeof(int32_t) * (size_t)b->S[f] * nrf);
        b->off_perm.push_back(o);
        o += a256(sizeof(int32_t) * (size_t)b->S[f] * nrf);
    }
    b->work_stride = tracer_work_stride(b->max_nr, sizeof(float2));
    b->off_work = o;
    o += b->work_stride * (size_t)b->grid;
    b->total = o;
    for (int i = 0; i < 4; i++) {
        if (cudaEventCreate(&b->ev[i]) != cudaSuccess) {
            cc_batch_destroy(b);
            return berr(CC_ECUDA, "cc_batch_create: cudaEventCreate failed");
        }
    }
    *out = b;
    return CC_OK;
}

int cc_batch_destroy(cc_batch* b) {
    if (!b) return CC_OK;
    drop_graph(b);
    for (int i = 0; i < 4; i++)
        if (b->ev[i]) cudaEventDestroy(b->ev[i]);
    delete b;
    return CC_OK;
}

int cc_batch_workspace_bytes(const cc_batch* b, size_t* bytes) {
    if (!b || !bytes) return berr(CC_EINVAL, "cc_batch_workspace_bytes: NULL argument");
    *bytes = b->total;
    return CC_OK;
}

int cc_batch_bind(cc_batch* b, double* const* z_out, double* const* w_out, void* workspace, size_t workspace_bytes) {
    if (!b || !z_out || !workspace) return berr(CC_EINVAL, "cc_batch_bind: NULL argument");
    if ((uintptr_t)workspace % 256) return berr(CC_EINVAL, "cc_batch_bind: workspace must be 256-byte aligned");
    if (workspace_bytes < b->total) return berr(CC_ENOMEM, "cc_batch_bind: workspace too small");
    for (int f = 0; f < b->count; f++)
        if (!z_out[f]) return berr(CC_EINVAL, "cc_batch_bind: NULL z_out entry");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return berr(CC_ECUDA, "cc_batch_bind: cudaSetDevice failed");
    char* ws = (char*)workspace;
    std::vector<TraceTask> tasks(b->count);
    std::vector<RescueTask> rtasks(b->count);
    std::vector<unsigned char> ptasks(polish_task_bytes() * b->count);
    b->fmm_args.clear();
    b->direct_count = 0;
    std::vector<int2> seams;
    std::vector<std::pair<double, int2>> items;
    int64_t block0 = 0;
    for (int f = 0; f < b->count; f++) {
        const FieldDev& fd = b->dev[f];
        TraceTask& t = tasks[f];
        t.stars = fd.star32;
        t.poly = fd.poly;
        t.tfmm = fd.tfmm;
        t.tcells = fd.tcells;
        t.tnear = fd.tnear;
        t.tcoeff = fd.tcoeff;
        t.n = (int)fd.n;
        t.nr = (int)b->nr[f];
        t.kappa_s = fd.kappa_s;
        t.gamma = fd.gamma;
        t.m = b->m[f];
        t.S = b->S[f];
        t.phase = (const double2*)(ws + b->off_phase[f]);
        t.zrows = ws + b->off_zrows[f];
        t.seam = ws + b->off_seam[f];
        t.iters = (int32_t*)(ws + b->off_iters[f]);
        t.match = (int32_t*)(ws + b->off_match[f]);
        t.hits = (int32_t*)(ws + b->off_hits[f]);
        t.perm = (int32_t*)(ws + b->off_perm[f]);
        t.rep = (DevReport*)(ws + b->off_reps) + f;
        for (int s = 0; s + 1 < b->S[f]; s++) seams.push_back(make_int2(f, s));
        const double cost = (double)b->rows[f] * (double)b->nr[f] * (double)(fd.n + b->nr[f]);
        const double per = cost / (double)b->S[f] + 20.0 * (double)b->nr[f] * (double)(fd.n + b->nr[f]);
        for (int s = 0; s < b->S[f]; s++) items.push_back({per, make_int2(f, s)});
        PolishArgs pa;
        pa.ext = nullptr;
        pa.ext_n = 0;
        pa.f = &b->dev[f];
        pa.m = b->m[f];
        pa.S = b->S[f];
        pa.nr = b->nr[f];
        pa.phase = t.phase;
        pa.zrows = (const float2*)t.zrows;
        pa.perm = t.perm;
        pa.iters_in = t.iters;
        pa.z_out = (double2*)z_out[f];
        pa.w_out = w_out ? (double2*)w_out[f] : nullptr;
        pa.iters_out = nullptr;
        pa.rep = t.rep;
        pa.tol_cert = b->opt.tol_cert;
        pa.max_polish = b->opt.max_polish;
        pa.hp_fp64 = 0;
        pa.rescue_list = (int4*)(ws + b->off_list);
        pa.rescue_count = (int*)(ws + b->off_nlist);
        pa.field_id = f;
        pa.skip_if = nullptr;
        if (b->use_fmm[f]) {
            b->fmm_args.push_back(pa);
        } else {
            polish_task_fill(pa, block0, ptasks.data() + polish_task_bytes() * b->direct_count);
            b->direct_count++;
            block0 += polish_blocks(b->rows[f] * b->nr[f]);
        }
        RescueTask& rt = rtasks[f];
        rt.stars = fd.star64;
        rt.poly = fd.poly;
        rt.n = (int)fd.n;
        rt.nr = (int)b->nr[f];
        rt.kappa_s = fd.kappa_s;
        rt.gamma = fd.gamma;
        rt.m = b->m[f];
        rt.phase = t.phase;
        rt.z = pa.z_out;
        rt.w = pa.w_out;
        rt.rep = t.rep;
    }
    b->total_blocks = block0;
    std::stable_sort(items.begin(), items.end(), [](const std::pair<double, int2>& x, const std::pair<double, int2>& y) {
        return x.first > y.first;
    });
    std::vector<int2> it(items.size());
    for (size_t i = 0; i < items.size(); i++) it[i] = items[i].second;
    b->nseams = (int)seams.size();
    if ((e = cudaMemcpy(ws + b->off_tasks, tasks.data(), sizeof(TraceTask) * b->count, cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(ws + b->off_items, it.data(), sizeof(int2) * it.size(), cudaMemcpyHostToDevice)) ||
        (seams.size() && (e = cudaMemcpy(ws + b->off_seams, seams.data(), sizeof(int2) * seams.size(),
                                         cudaMemcpyHostToDevice))) ||
        (e = cudaMemcpy(ws + b->off_ptasks, ptasks.data(), ptasks.size(), cudaMemcpyHostToDevice)) ||
        (e = cudaMemcpy(ws + b->off_rtasks, rtasks.data(), sizeof(RescueTask) * b->count, cudaMemcpyHostToDevice)))
        return berr(CC_ECUDA, cudaGetErrorString(e));
    b->ws = ws;
    b->bound = true;
    drop_graph(b);
    return CC_OK;
}

int cc_batch_launch(cc_batch* b, int32_t use_graph, cc_stream_t stream) {
    if (!b) return berr(CC_EINVAL, "cc_batch_launch: batch is NULL");
    if (!b->bound) return berr(CC_EINVAL, "cc_batch_launch: call cc_batch_bind first");
    cudaError_t e = cudaSetDevice(b->device);
    if (e != cudaSuccess) return berr(CC_ECUDA, "cc_batch_launch: cudaSetDevice failed");
    cudaStream_t st = (cudaStream_t)stream;
    if (!use_graph) {
        e = enqueue(b, st, false);
        if (e != cudaSuccess) return berr(CC_ECUDA, cudaGetErrorString(e));
        b->launched = true;
        b->last_stream = st;
        return CC_OK;
    }
    if (!st) return berr(CC_EINVAL, "cc_batch_launch: graph replay needs a non-default stream");
    if (!b->graph_ok || b->graph_stream != st) {
        drop_graph(b);
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return berr(CC_ECUDA, cudaGetErrorString(e));
        cudaError_t eq = enqueue(b, st, true);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (eq != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return berr(CC_ECUDA, cudaGetErrorString(eq != cudaSuccess ? eq : e));
        }
        b->graph = g;
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            drop_graph(b);
            return berr(CC_ECUDA, cudaGetErrorString(e));
        }
        b->graph_ok = true;
        b->graph_stream = st;
    }
    e = cudaGraphLaunch(b->exec, st);
    if (e != cudaSuccess) return berr(CC_ECUDA, cudaGetErrorString(e));
    b->launched = true;
    b->last_stream = st;
    return CC_OK;
}

int cc_batch_report(cc_batch* b, cc_report* per_field, cc_report* total) {
    if (!b) return berr(CC_EINVAL, "cc_batch_report: batch is NULL");
    if (!b->launched) return berr(CC_EINVAL, "cc_batch_report: nothing launched yet");
    cudaError_t e = cudaStreamSynchronize(b->last_stream);
    if (e != cudaSuccess) return berr(CC_ECUDA, cudaGetErrorString(e));
    std::vector<DevReport> r(b->count);
    e = cudaMemcpy(r.data(), b->ws + b->off_reps, sizeof(DevReport) * b->count, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return berr(CC_ECUDA, cudaGetErrorString(e));
    float t01 = 0, t12 = 0, t23 = 0;
    if (cudaEventElapsedTime(&t01, b->ev[0], b->ev[1]) != cudaSuccess ||
        cudaEventElapsedTime(&t12, b->ev[1], b->ev[2]) != cudaSuccess ||
        cudaEventElapsedTime(&t23, b->ev[2], b->ev[3]) != cudaSuccess) {
        cudaGetLastError();  // stage times unavailable: leave them at zero
        t01 = t12 = t23 = 0;
    }
    cc_report tot;
    memset(&tot, 0, sizeof tot);
    bool bad = false;
    for (int f = 0; f < b->count; f++) {
        cc_report q;
        memset(&q, 0, sizeof q);
        q.rows = b->rows[f];
        q.n_roots = b->nr[f];
        q.subchains = b->S[f];
        q.root_iterations = (int64_t)r[f].root_iterations;
        q.cold_root_iterations = (int64_t)r[f].cold_root_iterations;
        q.unconverged = (int64_t)r[f].unconverged;
        q.polish_passes = (int64_t)r[f].polish_passes;
        q.uncertified = (int64_t)r[f].uncertified;
        q.seam_ambiguous = (int64_t)r[f].seam_ambiguous;
        q.max_iter_row = r[f].max_iter_row;
        q.max_err_est = r[f].max_err_est;
        q.rescued_points = (int64_t)r[f].rescued_points;
        q.jumped = (int64_t)r[f].jumped;
        q.star_terms = (int64_t)r[f].star_terms;
        q.far_evals = (int64_t)r[f].far_evals;
        q.root_terms = (int64_t)r[f].root_terms;
        q.split_redone_rows = (int64_t)r[f].split_redone_rows;
        if (per_field) per_field[f] = q;
        tot.rows += q.rows;
        tot.n_roots += q.n_roots;
        tot.subchains += q.subchains;
        tot.root_iterations += q.root_iterations;
        tot.cold_root_iterations += q.cold_root_iterations;
        tot.unconverged += q.unconverged;
        tot.polish_passes += q.polish_passes;
        tot.uncertified += q.uncertified;
        tot.seam_ambiguous += q.seam_ambiguous;
        tot.max_iter_row = std::max(tot.max_iter_row, q.max_iter_row);
        tot.max_err_est = std::max(tot.max_err_est, q.max_err_est);
        tot.rescued_points += q.rescued_points;
        tot.jumped += q.jumped;
        tot.star_terms += q.star_terms;
        tot.far_evals += q.far_evals;
        tot.root_terms += q.root_terms;
        tot.split_redone_rows += q.split_redone_rows;
        bad = bad || q.unconverged || q.uncertified;
    }
    tot.trace_ms = t01;
    tot.join_ms = t12;
    tot.polish_ms = t23;
    if (total) *total = tot;
    if (bad) return berr(CC_ENOCONV, "some fields have unconverged or uncertified points");
    return CC_OK;
}

int cc_batch_info(const cc_batch* b, int32_t* items, int32_t* grid, int32_t* threads) {
    if (!b) return berr(CC_EINVAL, "cc_batch_info: batch is NULL");
    if (items) *items = b->nitems;
    if (grid) *grid = b->grid;
    if (threads) *threads = b->threads;
    return CC_OK;
}

}  // extern "C"
