// C ABI of libei.so (declared in include/ei.h): geometry set-up, layouts and
// the stream-ordered entry points.  All compute runs in the CUDA kernels of
// this library; there is no CPU fallback.
#include <cstdarg>
#include <math.h>
#include <string.h>

#include <stdio.h>
#include <stdlib.h>
#include <sys/stat.h>

#include <algorithm>
#include <string>
#include <vector>

#include "ei_internal.h"
#include "lib_alloc.h"

#include <atomic>

namespace ei {

static std::atomic<int> g_fail_alloc{-1};      // allocations to pass before one fails
static std::atomic<int64_t> g_live_allocs{0};

cudaError_t lib_malloc(void **p, size_t bytes)
{
    *p = nullptr;
    int n = g_fail_alloc.load();
    while (n >= 0 && !g_fail_alloc.compare_exchange_weak(n, n - 1)) {
    }
    if (n == 0) return cudaErrorMemoryAllocation;      // the armed failure (now disarmed)
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) ++g_live_allocs;
    return e;
}

void lib_free(void *p)
{
    if (!p) return;
    cudaFree(p);
    --g_live_allocs;
}

cudaError_t ic_set_smem_limit();
cudaError_t project_set_smem_limit();

static int round_up4(int n) { return (n + 3) / 4 * 4; }

template <class T>
static cudaError_t dev_alloc(ei_geometry *g, T **p, size_t count)
{
    void *ptr = nullptr;
    size_t bytes = std::max<size_t>(count * sizeof(T), 16);
    cudaError_t e = lib_malloc(&ptr, bytes);
    if (e != cudaSuccess) return e;
    g->allocs.push_back(ptr);
    g->workspace_bytes += (int64_t)bytes;
    *p = static_cast<T *>(ptr);
    return cudaSuccess;
}

template <class T>
static cudaError_t upload(ei_geometry *g, T **p, const std::vector<T> &h)
{
    EI_CUDA_TRY(dev_alloc(g, p, h.size()));
    if (!h.empty())
        EI_CUDA_TRY(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return cudaSuccess;
}

// Copy `count` floats from host or device memory to a host vector.
static cudaError_t fetch_floats(const float *src, size_t count, std::vector<float> &dst)
{
    dst.resize(count);
    if (count == 0) return cudaSuccess;
    return cudaMemcpy(dst.data(), src, count * sizeof(float), cudaMemcpyDefault);
}

static thread_local char g_last_error[256] = "";

void record_error(cudaError_t e)
{
    snprintf(g_last_error, sizeof g_last_error, "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
}

void record_message(const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
}

// Read and clear the device-side status word that kernels with bounded waits
// set; synchronises `st`.
static int take_device_status(ei_geometry *g, cudaStream_t st)
{
    int h = 0;
    if (cudaMemcpyAsync(&h, g->dev_status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EI_ERR_CUDA;
    if (h == 0) return EI_OK;
    cudaMemsetAsync(g->dev_status, 0, sizeof(int), st);
    if (h == EI_ERR_DEVICE_CHECK)
        record_message("a kernel's index bounds check fired (build with device checks)");
    else
        record_message("a kernel's bounded wait for its input rows ran out (status %d)", h);
    return h;
}

void select_variants(ei_geometry *g, int fwd_id, int adj_id, int persistent)
{
    g->fwd_variant.id = fwd_id;
    g->fwd_variant.prefix = g->fwd_prefixes[fwd_id];
    g->fwd_variant.total = g->fwd_totals[fwd_id];
    g->adj_variant.id = adj_id;
    g->adj_variant.prefix = g->adj_prefixes[adj_id];
    g->adj_variant.total = g->adj_totals[adj_id];
    g->dg.gmirror = adj_mirror_layout(adj_id) ? 1 : 0;
    g->persistent = persistent;
}

cudaEvent_t trace_begin(ei_geometry *g, cudaStream_t st)
{
    if (!g->prof_on) return nullptr;
    cudaEvent_t e = nullptr;
    if (!g->ev_pool.empty()) {
        e = g->ev_pool.back();
        g->ev_pool.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    cudaEventRecord(e, st);
    return e;
}

void trace_end(ei_geometry *g, TracedKernel k, cudaEvent_t begin, cudaStream_t st)
{
    if (!begin) return;
    cudaEvent_t e = trace_begin(g, st);
    if (e) g->ev_pairs[k].push_back({begin, e});
}

// Launch helpers that count and (when tracing) time the three path kernels.
static cudaError_t traced_project(ei_geometry *g, float *proj, float link, const int *active,
                                  cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_project(g, proj, link, active, st);
    trace_end(g, TK_PROJECT, b, st);
    count_launches(g, 1);
    return e;
}

static cudaError_t traced_ic(ei_geometry *g, const float *proj, const float *meas, float *s_mod,
                             double *part, IcMode mode, float link, const int *active,
                             cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_ic(g, proj, meas, s_mod, part, mode, link, active, st);
    trace_end(g, TK_IC, b, st);
    count_launches(g, 1);
    return e;
}

static cudaError_t traced_backproject(ei_geometry *g, const float4 *v, float4 *out,
                                      float4 out_mult, float4 reg2, float link, const int *active,
                                      cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_backproject(g, v, out, out_mult, reg2, link, active, st);
    trace_end(g, TK_BACKPROJECT, b, st);
    count_launches(g, 1);
    return e;
}

static cudaError_t counted_prep(ei_geometry *g, const float4 *vol, float4 mult, bool linked,
                                const int *active, cudaStream_t st)
{
    count_launches(g, 1);
    return launch_prep(g, vol, mult, linked, active, st);
}

// Staging multipliers of a physical volume for the model: (1, 1, 1), or in
// linked mode (1, gamma, 0) applied to the mu lane's h.
static float4 physical_mult(const ei_geometry *g)
{
    return g->link_gamma > 0.f ? make_float4(1.f, g->link_gamma, 0.f, 0.f)
                               : make_float4(1.f, 1.f, 1.f, 0.f);
}

EvalConsts eval_consts(const ei_geometry *g, bool scaled)
{
    // linked mode: the unknown is h in the mu lane, mu = h, delta = gamma h,
    // sigma = 0, regularised by lambda_mu only (Eq. 4, Eq. 5)
    const bool linked = g->link_gamma > 0.f;
    const float gam = g->link_gamma;
    const float on1 = linked ? 0.f : 1.f;
    EvalConsts c;
    if (scaled) {
        c.mult = linked ? make_float4(g->scale[0], gam * g->scale[0], 0.f, 0.f)
                        : make_float4(g->scale[0], g->scale[1], g->scale[2], 0.f);
        c.out_mult = make_float4(g->scale[0], on1 * g->scale[1], on1 * g->scale[2], 0.f);
        c.reg2 = make_float4(2.f * g->lambda[0], on1 * 2.f * g->lambda[1], on1 * 2.f * g->lambda[2], 0.f);
        c.reg1 = make_float4(g->lambda[0], on1 * g->lambda[1], on1 * g->lambda[2], 0.f);
    } else {
        c.mult = physical_mult(g);
        c.out_mult = make_float4(1.f, on1, on1, 0.f);
        float k[3];
        for (int i = 0; i < 3; ++i) k[i] = (float)(1.0 / ((double)g->scale[i] * g->scale[i]));
        c.reg2 = make_float4(2.f * g->lambda[0] * k[0], on1 * 2.f * g->lambda[1] * k[1],
                             on1 * 2.f * g->lambda[2] * k[2], 0.f);
        c.reg1 = make_float4(g->lambda[0] * k[0], on1 * g->lambda[1] * k[1],
                             on1 * g->lambda[2] * k[2], 0.f);
    }
    // linked: single-channel staging, projection and adjoint (the IC kernel
    // combines the gradient sinogram into g_mu + gamma g_delta)
    c.link = linked ? gam : 0.f;
    return c;
}

cudaError_t evaluate(ei_geometry *g, const float4 *v, const float *meas, double *S_dev,
                     float4 *grad, bool scaled, const int *active, cudaStream_t st)
{
    NvtxRange range(grad ? "objective and gradient" : "objective");
    const EvalConsts c = eval_consts(g, scaled);
    const bool linked = c.link > 0.f;
    EI_CUDA_TRY(counted_prep(g, v, c.mult, linked, active, st));
    EI_CUDA_TRY(traced_project(g, g->proj, c.link, active, st));
    EI_CUDA_TRY(traced_ic(g, g->proj, meas, nullptr, g->part_ic,
                          grad ? IC_OBJECTIVE_GRAD : IC_OBJECTIVE, c.link, active, st));
    count_launches(g, 2);
    EI_CUDA_TRY(launch_reg_partials(g->dg, v, c.reg1, g->part_reg, active, st));
    EI_CUDA_TRY(launch_finalize_objective(g, g->part_ic, g->dg.vec_prefix, g->part_reg, S_dev,
                                          active, st));
    if (grad) EI_CUDA_TRY(traced_backproject(g, v, grad, c.out_mult, c.reg2, c.link, active, st));
    return cudaSuccess;
}

}  // namespace ei

using namespace ei;

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

extern "C" {

const char *ei_last_error(void) { return g_last_error; }

const char *ei_status_string(int status)
{
    switch (status) {
    case EI_OK: return "EI_OK";
    case EI_ERR_ARG: return "EI_ERR_ARG: invalid argument";
    case EI_ERR_CUDA: return "EI_ERR_CUDA: a CUDA call failed";
    case EI_ERR_NONFINITE: return "EI_ERR_NONFINITE: non-finite objective";
    case EI_ERR_LINESEARCH: return "EI_ERR_LINESEARCH: no acceptable step";
    case EI_ERR_TIMEOUT: return "EI_ERR_TIMEOUT: a bounded wait ran out";
    case EI_ERR_DEVICE_CHECK: return "EI_ERR_DEVICE_CHECK: a kernel bounds check fired";
    case EI_ERR_ALLOC: return "EI_ERR_ALLOC: workspace allocation failed";
    default: return "unknown ei_status";
    }
}

void ei_default_solve_opts(ei_solve_opts *o)
{
    if (!o) return;
    o->tol = 1e-6;
    o->max_iter = 100;
    o->lbfgs_m = 10;
    o->c1 = 1e-4;
    o->max_trials = 20;
    o->curv_eps = 1e-10;
    o->use_graph = 1;
    o->resume = 0;
    o->max_seconds = 0.0;
}

int ei_fail_alloc_after(int n)
{
    if (n < -1) return EI_ERR_ARG;
    ei::g_fail_alloc.store(n);
    return EI_OK;
}

int ei_fail_alloc_pending(int *n)
{
    if (!n) return EI_ERR_ARG;
    *n = std::max(-1, ei::g_fail_alloc.load());
    return EI_OK;
}

int ei_live_allocations(int64_t *n)
{
    if (!n) return EI_ERR_ARG;
    *n = ei::g_live_allocs.load();
    return EI_OK;
}

static void release_events(ei_geometry *g)
{
    for (int k = 0; k < 3; ++k) {
        for (auto &p : g->ev_pairs[k]) {
            g->ev_pool.push_back(p.first);
            g->ev_pool.push_back(p.second);
        }
        g->ev_pairs[k].clear();
    }
}

int ei_profile_enable(ei_geometry *g, int on)
{
    if (!g) return EI_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return EI_ERR_CUDA;
    release_events(g);
    g->launches = 0;
    g->prof_on = on != 0;
    return EI_OK;
}

int ei_profile_read(ei_geometry *g, ei_profile *o)
{
    if (!g || !o) return EI_ERR_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return EI_ERR_CUDA;
    double ms[3] = {0, 0, 0};
    for (int k = 0; k < 3; ++k)
        for (auto &p : g->ev_pairs[k]) {
            float t = 0.f;
            if (cudaEventElapsedTime(&t, p.first, p.second) != cudaSuccess) return EI_ERR_CUDA;
            ms[k] += t;
        }
    o->launches = g->launches;
    o->project_launches = (int64_t)g->ev_pairs[TK_PROJECT].size();
    o->ic_launches = (int64_t)g->ev_pairs[TK_IC].size();
    o->backproject_launches = (int64_t)g->ev_pairs[TK_BACKPROJECT].size();
    o->project_ms = ms[TK_PROJECT];
    o->ic_ms = ms[TK_IC];
    o->backproject_ms = ms[TK_BACKPROJECT];
    return EI_OK;
}

void ei_destroy_geometry(ei_geometry *g)
{
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    release_events(g);
    for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
    ei::destroy_solver(g);
    for (void *p : g->allocs) ei::lib_free(p);
    cudaSetDevice(prev);
    delete g;
}

int ei_setup_geometry(const ei_geometry_desc *d, int n_slices, const ei_slice_dims *per_slice,
                      ei_geometry **out)
{
    if (!d || !out || n_slices < 1) return EI_ERR_ARG;
    *out = nullptr;
    NvtxRange range("ei_setup_geometry");
    if (d->n_m < 1 || d->n_m > EI_MAX_NM || !d->m) return EI_ERR_ARG;
    if (!(d->z_cm >= 0) || !(d->period_cm > 0) || !(d->kappa_sigma >= 0)) return EI_ERR_ARG;
    if (!d->flat_A || !d->flat_c || !d->flat_w) return EI_ERR_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(d->scale[c] > 0) || !(d->lambda[c] >= 0) || !isfinite(d->lambda[c])) return EI_ERR_ARG;
    std::vector<ei_slice_dims> dims(n_slices);
    for (int s = 0; s < n_slices; ++s) {
        dims[s] = per_slice ? per_slice[s]
                            : ei_slice_dims{d->n, d->n_theta, d->n_det, d->pitch_cm};
        const ei_slice_dims &q = dims[s];
        if (q.n < 1 || q.n > 16384 || q.n_theta < 1 || q.n_det < 1 || q.n_det > EI_MAX_NDET ||
            !(q.pitch_cm > 0) || !isfinite(q.pitch_cm))
            return EI_ERR_ARG;
    }
    ei_geometry *g = new ei_geometry();
    cudaGetDevice(&g->device);
    g->n_slices = n_slices;
    g->n_m = d->n_m;
    for (int c = 0; c < 3; ++c) {
        g->lambda[c] = (float)d->lambda[c];
        g->scale[c] = (float)d->scale[c];
    }
    // ---- host tables
    const bool uniform = per_slice == nullptr;
    int64_t ang_total = 0, pix_total = 0, pix_in_total = 0;
    for (auto &q : dims) {
        ang_total += q.n_theta;
        pix_total += round_up4(q.n_det);
        pix_in_total += q.n_det;
    }
    const size_t flat_count = uniform ? (size_t)d->n_det : (size_t)pix_in_total;
    std::vector<float> fA, fc, fw, fmr, fmo;
    cudaError_t ce = fetch_floats(d->flat_A, flat_count, fA);
    if (ce == cudaSuccess) ce = fetch_floats(d->flat_c, flat_count, fc);
    if (ce == cudaSuccess) ce = fetch_floats(d->flat_w, flat_count, fw);
    if (ce == cudaSuccess && d->m_r) ce = fetch_floats(d->m_r, flat_count, fmr);
    const size_t mo_count = uniform ? (size_t)d->n_theta : (size_t)ang_total;
    if (ce == cudaSuccess && d->m_o) ce = fetch_floats(d->m_o, mo_count, fmo);
    if (ce != cudaSuccess) {
        delete g;
        return EI_ERR_ARG;   // a pointer that is neither host nor device memory
    }
    for (size_t i = 0; i < flat_count; ++i)
        if (!(fw[i] > 0) || !isfinite(fA[i]) || !isfinite(fc[i])) {
            delete g;
            return EI_ERR_ARG;
        }

    std::vector<AngleInfo> ang;
    std::vector<float> m_o;
    std::vector<float4> pix;
    ang.reserve(ang_total);
    pix.reserve(pix_total);
    std::vector<int> ic_p(1, 0), prep_p(1, 0), vec_p(1, 0);
    std::vector<std::vector<int>> fwd_p(N_FWD_VARIANTS, std::vector<int>(1, 0));
    std::vector<std::vector<int>> adj_p(N_ADJ_VARIANTS, std::vector<int>(1, 0));
    uint64_t hash = 1469598103934665603ULL;          // FNV-1a over the slice sizes
    auto mix = [&hash](uint64_t v) {
        for (int b = 0; b < 8; ++b) {
            hash ^= (v >> (8 * b)) & 0xff;
            hash *= 1099511628211ULL;
        }
    };
    int64_t vol_off = 0, pp_off = 0, gp_off = 0, sino_off = 0, proj_off = 0, meas_off = 0;
    int ang_off = 0, pix_off = 0, pix_in_off = 0, max_ndp = 4, max_nth = 1;
    for (int s = 0; s < n_slices; ++s) {
        const ei_slice_dims &q = dims[s];
        SliceInfo si{};
        si.n = q.n;
        si.n_theta = q.n_theta;
        si.n_det = q.n_det;
        si.n_dp = round_up4(q.n_det);
        si.pitch = (float)q.pitch_cm;
        si.inv_pitch = (float)(1.0 / q.pitch_cm);
        si.ang_off = ang_off;
        si.pix_off = pix_off;
        si.det_off = (int)pix_in_off;
        // zero margin of the packed gradient-sinogram rows: every voxel of the adjoint's
        // (padded) tile grid projects within [hd - R, hd + R] pixels
        {
            const double hn_ = 0.5 * (q.n - 1);
            const int cpad = (q.n + ADJ_TC - 1) / ADJ_TC * ADJ_TC;
            const int rpad = (q.n + ADJ_MAX_TR - 1) / ADJ_MAX_TR * ADJ_MAX_TR;
            const double mdx = std::max(hn_, cpad - 1 - hn_), mdy = std::max(hn_, rpad - 1 - hn_);
            const double R = sqrt(mdx * mdx + mdy * mdy);
            si.marg = std::max(2, (int)ceil(R - 0.5 * (q.n_det - 1)) + 3);
        }
        si.gw = si.n_dp + 2 * si.marg;
        si.vol_off = vol_off;
        si.pp_off = pp_off;
        si.gp_off = gp_off;
        si.sino_off = sino_off;
        si.proj_off = proj_off;
        si.meas_off = meas_off;
        g->h_slices.push_back(si);
        for (int a = 0; a < q.n_theta; ++a) {
            double th = d->theta ? d->theta[(uniform ? 0 : ang_off) + a] : a * M_PI / q.n_theta;
            ang.push_back(make_angle_info(th, q.n, q.pitch_cm));
            m_o.push_back(d->m_o ? fmo[(uniform ? 0 : ang_off) + a] : 0.f);
        }
        const int src_off = uniform ? 0 : pix_in_off;
        for (int j = 0; j < si.n_dp; ++j) {
            if (j < q.n_det)
                pix.push_back(make_float4(fA[src_off + j], fc[src_off + j], fw[src_off + j],
                                          d->m_r ? fmr[src_off + j] : 0.f));
            else
                pix.push_back(make_float4(0.f, 0.f, 1.f, 0.f));
        }
        for (int v = 0; v < N_FWD_VARIANTS; ++v) {
            int rays, angles;
            project_variant_shape(v, &rays, &angles);
            const int nrb = (si.n_dp + rays - 1) / rays;
            const int nab = (q.n_theta + angles - 1) / angles;
            fwd_p[v].push_back(fwd_p[v].back() + nab * nrb);
        }
        for (int v = 0; v < N_ADJ_VARIANTS; ++v)
            adj_p[v].push_back(adj_p[v].back() + backproject_variant_items(v, q.n));
        mix((uint64_t)q.n), mix((uint64_t)q.n_theta), mix((uint64_t)q.n_det);
        ic_p.push_back(ic_p.back() + q.n_theta);
        const int pt = (q.n + 1 + PREP_TILE - 1) / PREP_TILE;
        prep_p.push_back(prep_p.back() + pt * pt);
        const int64_t nvox = (int64_t)q.n * q.n;
        vec_p.push_back(vec_p.back() + (int)((nvox + VEC_BLK - 1) / VEC_BLK));
        vol_off += nvox;
        pp_off += (int64_t)q.n * (q.n + 1);
        gp_off += (int64_t)q.n_theta * si.gw;
        sino_off += (int64_t)q.n_theta * si.n_dp;
        proj_off += 3LL * q.n_theta * si.n_dp;
        meas_off += (int64_t)d->n_m * q.n_theta * si.n_dp;
        ang_off += q.n_theta;
        pix_off += si.n_dp;
        pix_in_off += q.n_det;
        max_ndp = std::max(max_ndp, si.n_dp);
        max_nth = std::max(max_nth, q.n_theta);
    }
    g->vol_count = vol_off;
    g->pp_count = pp_off;
    g->gp_count = gp_off;
    g->sino4_count = sino_off;
    g->proj_count = proj_off;
    g->meas_count = meas_off;
    g->h_vec_prefix = vec_p;

    DevGeom &dg = g->dg;
    dg.n_slices = n_slices;
    dg.total_ic = ic_p.back();
    dg.total_prep = prep_p.back();
    dg.total_vec = vec_p.back();
    dg.max_ndp = max_ndp;
    dg.max_n_theta = max_nth;
    dg.mc.z_over_p = (float)(d->z_cm / d->period_cm);
    dg.mc.kappa = (float)d->kappa_sigma;
    dg.mc.n_m = d->n_m;
    for (int k = 0; k < d->n_m; ++k) {
        if (!isfinite(d->m[k])) {
            delete g;
            return EI_ERR_ARG;
        }
        dg.mc.m[k] = (float)d->m[k];
    }

    // ---- device tables and workspace
    cudaError_t e = cudaSuccess;
    SliceInfo *d_sl = nullptr;
    AngleInfo *d_ang = nullptr;
    float *d_mo = nullptr;
    float4 *d_pix = nullptr;
    int *d_ic = nullptr, *d_prep = nullptr, *d_vec = nullptr;
    for (int v = 0; v < N_FWD_VARIANTS; ++v) {
        int *dp = nullptr;
        if (e == cudaSuccess) e = upload(g, &dp, fwd_p[v]);
        g->fwd_prefixes[v] = dp;
        g->fwd_totals[v] = fwd_p[v].back();
    }
    for (int v = 0; v < N_ADJ_VARIANTS; ++v) {
        int *dp = nullptr;
        if (e == cudaSuccess) e = upload(g, &dp, adj_p[v]);
        g->adj_prefixes[v] = dp;
        g->adj_totals[v] = adj_p[v].back();
    }
    g->shape_hash = hash ^ (uint64_t)n_slices;
    if (e == cudaSuccess) e = upload(g, &d_sl, g->h_slices);
    if (e == cudaSuccess) e = upload(g, &d_ang, ang);
    if (e == cudaSuccess) e = upload(g, &d_mo, m_o);
    if (e == cudaSuccess) e = upload(g, &d_pix, pix);
    if (e == cudaSuccess) e = upload(g, &d_ic, ic_p);
    if (e == cudaSuccess) e = upload(g, &d_prep, prep_p);
    if (e == cudaSuccess) e = upload(g, &d_vec, vec_p);
    if (e == cudaSuccess) e = dev_alloc(g, &g->xpA, (size_t)g->pp_count);
    // the B copies get one pair of entries more: the staged projector copies
    // them in 16-byte-aligned pairs and may read one entry past a row's end
    if (e == cudaSuccess) e = dev_alloc(g, &g->xpB, (size_t)g->pp_count + 2);
    if (e == cudaSuccess) e = dev_alloc(g, &g->xtA, (size_t)g->pp_count);
    if (e == cudaSuccess) e = dev_alloc(g, &g->xtB, (size_t)g->pp_count + 2);
    if (e == cudaSuccess) e = dev_alloc(g, &g->proj, (size_t)g->proj_count);
    if (e == cudaSuccess) e = dev_alloc(g, &g->gA, (size_t)g->gp_count);
    if (e == cudaSuccess) e = dev_alloc(g, &g->gB, (size_t)g->gp_count);
    if (e == cudaSuccess) e = dev_alloc(g, &g->part_ic, (size_t)dg.total_ic);
    if (e == cudaSuccess) e = dev_alloc(g, &g->part_reg, (size_t)std::max(1, dg.total_vec));
    if (e == cudaSuccess) e = dev_alloc(g, &g->work_counter, 2);
    if (e == cudaSuccess) e = dev_alloc(g, &g->sm_counters, MAX_SM_CHUNKS);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    if (e == cudaSuccess) e = dev_alloc(g, &g->S_dev, (size_t)n_slices);
    if (e == cudaSuccess) e = dev_alloc(g, &g->dev_status, 1);
    if (e == cudaSuccess) e = cudaMemset(g->dev_status, 0, sizeof(int));
    // the packed gradient sinogram's margins and padding pixels must read as zero
    if (e == cudaSuccess) e = cudaMemset(g->gA, 0, (size_t)g->gp_count * sizeof(float4));
    if (e == cudaSuccess) e = cudaMemset(g->gB, 0, (size_t)g->gp_count * sizeof(float2));
    if (e == cudaSuccess) e = ic_set_smem_limit();
    if (e == cudaSuccess) e = project_set_smem_limit();
    if (e == cudaSuccess) e = single_shot_set_smem_limit();
    if (e != cudaSuccess) {
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        ei_destroy_geometry(g);
        return oom ? EI_ERR_ALLOC : EI_ERR_CUDA;
    }
    dg.slices = d_sl;
    dg.ang = d_ang;
    dg.m_o = d_mo;
    dg.pix = d_pix;
    dg.ic_prefix = d_ic;
    dg.prep_prefix = d_prep;
    dg.vec_prefix = d_vec;
    dg.status = g->dev_status;
    select_variants(g, 0, 0, LAUNCH_PER_ITEM);
    g->ic_variant = ic_pipe_fits(dg.max_ndp, dg.mc.n_m) ? 1 : 0;
    *out = g;
    return EI_OK;
}

int ei_set_ic_variant(ei_geometry *g, int variant)
{
    if (!g || variant < 0 || variant > 1) return EI_ERR_ARG;
    if (variant == 1 && !ic_pipe_fits(g->dg.max_ndp, g->dg.mc.n_m)) {
        record_message("ei_set_ic_variant: rows of %d pixels with M = %d do not fit the "
                     "bulk-copy variant's shared-memory buffers", g->dg.max_ndp, g->dg.mc.n_m);
        return EI_ERR_ARG;
    }
    g->ic_variant = variant;
    return EI_OK;
}

int ei_get_ic_variant(const ei_geometry *g, int *variant)
{
    if (!g || !variant) return EI_ERR_ARG;
    *variant = g->ic_variant;
    return EI_OK;
}

int ei_set_variant(ei_geometry *g, int fwd_variant, int adj_variant, int persistent)
{
    if (!g || fwd_variant < 0 || fwd_variant >= N_FWD_VARIANTS || adj_variant < 0 ||
        adj_variant >= N_ADJ_VARIANTS || persistent < 0 || persistent >= N_LAUNCH_MODES)
        return EI_ERR_ARG;
    select_variants(g, fwd_variant, adj_variant, persistent);
    return EI_OK;
}

int ei_get_variant(const ei_geometry *g, int *fwd_variant, int *adj_variant, int *persistent)
{
    if (!g || !fwd_variant || !adj_variant || !persistent) return EI_ERR_ARG;
    *fwd_variant = g->fwd_variant.id;
    *adj_variant = g->adj_variant.id;
    *persistent = g->persistent;
    return EI_OK;
}

static std::string tune_cache_path()
{
    const char *p = getenv("EI_TUNE_CACHE");
    if (p && *p) return p;
    const char *home = getenv("HOME");
    return std::string(home && *home ? home : "/tmp") + "/.cache/ei_gb300_autotune.txt";
}

static std::string tune_key(const ei_geometry *g)
{
    cudaDeviceProp prop{};
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, g->device) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    char buf[80];
    // linked geometries run the single-channel kernels: tuned separately; the
    // variant counts make entries tuned before a variant was added stale
    snprintf(buf, sizeof buf, "|%016llx|v1f%da%d%s", (unsigned long long)g->shape_hash,
             N_FWD_VARIANTS, N_ADJ_VARIANTS, g->link_gamma > 0.f ? "L" : "");
    return name + buf;
}

// Mean duration (ms) of `reps` launches of the selected projector or adjoint variant.
static int time_kernel(ei_geometry *g, bool adjoint, float4 *adj_out, cudaStream_t st, int reps,
                       double *ms)
{
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return EI_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return EI_ERR_CUDA;
    }
    const float4 one = make_float4(1.f, 1.f, 1.f, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
    const float link = g->link_gamma;              // the kernels this geometry's evaluations run
    auto launch = [&]() {
        return adjoint ? launch_backproject(g, nullptr, adj_out, one, zero, link, nullptr, st)
                       : launch_project(g, g->proj, link, nullptr, st);
    };
    cudaError_t e = launch();                       // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, st);
    for (int r = 0; r < reps && e == cudaSuccess; ++r) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float t = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = t / reps;
    return e == cudaSuccess ? EI_OK : EI_ERR_CUDA;
}

// A candidate replaces the incumbent (the lower id, or one-block-per-item
// launches) only when it is at least 1% faster: variants within timing noise
// of each other then get the same, reproducible choice.
static const double kTuneMargin = 0.99;
static thread_local double g_tune_last[2];     // the chosen variants' times (ms)
static int autotune_timed(ei_geometry *g, float4 *adj_out, cudaStream_t st);

int ei_autotune(ei_geometry *g, int flags, void *stream)
{
    if (!g) return EI_ERR_ARG;
    NvtxRange range("ei_autotune");
    const std::string key = tune_key(g), path = tune_cache_path();
    if (!(flags & EI_TUNE_FORCE)) {
        FILE *f = fopen(path.c_str(), "r");
        if (f) {
            char k[512];
            int fv, av, pv;
            double fm, am;
            bool found = false;
            while (fscanf(f, "%511s %d %d %d %lf %lf", k, &fv, &av, &pv, &fm, &am) == 6)
                if (key == k && fv >= 0 && fv < N_FWD_VARIANTS && av >= 0 && av < N_ADJ_VARIANTS &&
                    pv >= 0 && pv < N_LAUNCH_MODES) {
                    select_variants(g, fv, av, pv);          // the last matching line wins
                    found = true;
                }
            fclose(f);
            if (found) return EI_OK;
        }
    }
    cudaStream_t st = (cudaStream_t)stream;
    // the adjoint's output while it is timed (a volume, freed below)
    float4 *adj_out = nullptr;
    {
        void *p = nullptr;
        const cudaError_t e = lib_malloc(&p, (size_t)std::max<int64_t>(1, g->vol_count) * sizeof(float4));
        if (e != cudaSuccess) {
            record_error(e);
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
        }
        adj_out = static_cast<float4 *>(p);
    }
    const int rc = autotune_timed(g, adj_out, st);
    lib_free(adj_out);
    if (rc != EI_OK) return rc;
    const int bf = g->fwd_variant.id, ba = g->adj_variant.id, bp = g->persistent;
    if (!(flags & EI_TUNE_NO_CACHE_WRITE)) {
        const size_t slash = path.find_last_of('/');
        if (slash != std::string::npos && slash > 0) mkdir(path.substr(0, slash).c_str(), 0755);
        FILE *f = fopen(path.c_str(), "a");       // best effort: no cache if not writable
        if (f) {
            fprintf(f, "%s %d %d %d %.6f %.6f\n", key.c_str(), bf, ba, bp, g_tune_last[0],
                    g_tune_last[1]);
            fclose(f);
        }
    }
    return EI_OK;
}

// The timed part of ei_autotune: selects the fastest variants and launch mode
// (their times in g_tune_last).
static int autotune_timed(ei_geometry *g, float4 *adj_out, cudaStream_t st)
{
    // stage 1: every projector and adjoint variant in launch modes 0 and 1, 3
    // launches each (the SM-chunked mode 2 stays selectable but is not
    // tuned: on the benchmark batch it was 43 % slower for the projector and
    // 47 % for the adjoint, since the SMs then work on ~150 slices at once and
    // their data no longer stays in L2)
    constexpr int L = 2;
    int fid[L] = {}, aid[L] = {};
    for (int pers = 0; pers < L; ++pers) {
        double fbest = 1e300, abest = 1e300;
        for (int v = 0; v < N_FWD_VARIANTS; ++v) {
            select_variants(g, v, 0, pers);
            double ms = 0;
            const int rc = time_kernel(g, false, adj_out, st, 3, &ms);
            if (rc != EI_OK) return rc;
            if (ms < fbest * kTuneMargin) fbest = ms, fid[pers] = v;
        }
        for (int v = 0; v < N_ADJ_VARIANTS; ++v) {
            select_variants(g, fid[pers], v, pers);
            double ms = 0;
            const int rc = time_kernel(g, true, adj_out, st, 3, &ms);
            if (rc != EI_OK) return rc;
            if (ms < abest * kTuneMargin) abest = ms, aid[pers] = v;
        }
    }
    // stage 2: the launch modes' winners re-timed alternately, 3 rounds, each
    // keeping its fastest round (variants within a few % of each other are
    // otherwise decided by noise)
    double tf[L], ta[L];
    for (int k = 0; k < L; ++k) tf[k] = ta[k] = 1e300;
    for (int round = 0; round < 3; ++round)
        for (int pers = 0; pers < L; ++pers) {
            select_variants(g, fid[pers], aid[pers], pers);
            double mf = 0, ma = 0;
            int rc = time_kernel(g, false, adj_out, st, 2, &mf);
            if (rc == EI_OK) rc = time_kernel(g, true, adj_out, st, 2, &ma);
            if (rc != EI_OK) return rc;
            tf[pers] = std::min(tf[pers], mf);
            ta[pers] = std::min(ta[pers], ma);
        }
    int bp = 0;                                   // the incumbent: one block per item
    for (int k = 1; k < L; ++k)
        if (tf[k] + ta[k] < (tf[bp] + ta[bp]) * kTuneMargin) bp = k;
    select_variants(g, fid[bp], aid[bp], bp);
    g_tune_last[0] = tf[bp];
    g_tune_last[1] = ta[bp];
    return EI_OK;
}

int ei_get_layout(const ei_geometry *g, ei_layout *o)
{
    if (!g || !o) return EI_ERR_ARG;
    o->n_slices = g->n_slices;
    o->n_m = g->n_m;
    o->vol_count = g->vol_count;
    o->proj_count = g->proj_count;
    o->sino4_count = g->sino4_count;
    o->meas_count = g->meas_count;
    o->workspace_bytes = g->workspace_bytes;
    return EI_OK;
}

int ei_get_slice_layout(const ei_geometry *g, int s, ei_slice_layout *o)
{
    if (!g || !o || s < 0 || s >= g->n_slices) return EI_ERR_ARG;
    const SliceInfo &si = g->h_slices[s];
    o->n = si.n;
    o->n_theta = si.n_theta;
    o->n_det = si.n_det;
    o->n_dp = si.n_dp;
    o->n_m = g->n_m;
    o->pitch_cm = si.pitch;
    o->vol_offset = si.vol_off;
    o->vol_count = (int64_t)si.n * si.n;
    o->proj_offset = si.proj_off;
    o->proj_count = 3LL * si.n_theta * si.n_dp;
    o->sino4_offset = si.sino_off;
    o->sino4_count = (int64_t)si.n_theta * si.n_dp;
    o->meas_offset = si.meas_off;
    o->meas_count = (int64_t)g->n_m * si.n_theta * si.n_dp;
    return EI_OK;
}

static int status_from(cudaError_t e)
{
    if (e == cudaSuccess) return EI_OK;
    ei::record_error(e);
    return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
}

int ei_project(const ei_geometry *gc, const float *vol, float *proj, void *stream)
{
    if (!gc || !vol || !proj || !aligned16(vol) || !aligned16(proj)) return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = counted_prep(g, (const float4 *)vol, make_float4(1.f, 1.f, 1.f, 0.f), false,
                                 nullptr, st);
    if (e == cudaSuccess) e = traced_project(g, proj, 0.f, nullptr, st);
    return status_from(e);
}

int ei_backproject(const ei_geometry *gc, const float *sino4, float *vol, void *stream)
{
    if (!gc || !sino4 || !vol || !aligned16(sino4) || !aligned16(vol)) return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    const float4 one = make_float4(1.f, 1.f, 1.f, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
    cudaStream_t st = (cudaStream_t)stream;
    count_launches(g, 1);
    cudaError_t e = launch_pack_sino(g, (const float4 *)sino4, st);
    if (e == cudaSuccess)
        e = traced_backproject(g, nullptr, (float4 *)vol, one, zero, 0.f, nullptr, st);
    return status_from(e);
}

int ei_ic_model(const ei_geometry *gc, const float *proj, float *s_mod, void *stream)
{
    if (!gc || !proj || !s_mod || !aligned16(proj) || !aligned16(s_mod)) return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    return status_from(traced_ic(g, proj, nullptr, s_mod, g->part_ic, IC_MODEL, 0.f, nullptr,
                                 (cudaStream_t)stream));
}

int ei_single_shot_fbp(const ei_geometry *gc, const float *s_exp, float *vol_out, void *stream)
{
    if (!gc || !s_exp || !vol_out || !aligned16(s_exp) || !aligned16(vol_out)) return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    const float4 one = make_float4(1.f, 1.f, 1.f, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
    count_launches(g, 1);
    cudaError_t e = launch_single_shot(g, s_exp, st);
    if (e == cudaSuccess)
        e = traced_backproject(g, nullptr, (float4 *)vol_out, one, zero, 0.f, nullptr, st);
    return status_from(e);
}

int ei_single_shot_eq3(ei_geometry *g, const float *s_exp, int m_index, double gamma,
                       float *vol_out, void *stream)
{
    if (!g || !s_exp || !vol_out || !aligned16(s_exp) || !aligned16(vol_out) || m_index < 0 ||
        m_index >= g->n_m || !(gamma >= 0.0) || !isfinite(gamma))
        return EI_ERR_ARG;
    if (!single_shot_eq3_fits(g)) {
        record_message("ei_single_shot_eq3: rows of %d pixels exceed its shared-memory rows",
                       g->dg.max_ndp);
        return EI_ERR_ARG;
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!g->eq3_ker) {
        int64_t n_px = 0;
        for (const SliceInfo &si : g->h_slices) n_px += si.n_det;
        e = dev_alloc(g, &g->eq3_ker, (size_t)n_px);
        if (e != cudaSuccess) {
            record_error(e);
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
        }
    }
    const float4 one = make_float4(1.f, 1.f, 1.f, 0.f), zero = make_float4(0.f, 0.f, 0.f, 0.f);
    count_launches(g, 2);
    e = launch_single_shot_eq3(g, s_exp, m_index, (float)gamma, g->eq3_ker, st);
    if (e == cudaSuccess)
        e = traced_backproject(g, nullptr, (float4 *)vol_out, one, zero, 0.f, nullptr, st);
    return status_from(e);
}

int ei_forward(const ei_geometry *gc, const float *vol, float *s_mod, void *stream)
{
    if (!gc || !vol || !s_mod || !aligned16(vol) || !aligned16(s_mod)) return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = counted_prep(g, (const float4 *)vol, physical_mult(g), g->link_gamma > 0.f,
                                 nullptr, st);
    if (e == cudaSuccess) e = traced_project(g, g->proj, g->link_gamma, nullptr, st);
    if (e == cudaSuccess)
        e = traced_ic(g, g->proj, nullptr, s_mod, g->part_ic, IC_MODEL, 0.f, nullptr, st);
    return status_from(e);
}

int ei_set_offset_unknowns(ei_geometry *g, int which, double scale)
{
    if (!g || (which & ~(EI_OFFSET_MO | EI_OFFSET_MR)) || !(scale > 0.0) || !isfinite(scale))
        return EI_ERR_ARG;
    g->off_which = which;
    g->off_scale = (float)scale;
    return EI_OK;
}

int ei_set_ring_modes(ei_geometry *g, int K)
{
    if (!g || K < 0 || K > EI_MAX_RING_MODES) return EI_ERR_ARG;
    for (const SliceInfo &si : g->h_slices)
        if (K > si.n_det) return EI_ERR_ARG;
    g->ring_modes = K;
    return EI_OK;
}

int ei_get_offsets(const ei_geometry *g, float *m_o, float *m_r)
{
    if (!g) return EI_ERR_ARG;
    cudaError_t e = cudaSuccess;
    int n_th = 0;
    for (const SliceInfo &si : g->h_slices) n_th += si.n_theta;
    if (m_o) e = cudaMemcpy(m_o, g->dg.m_o, (size_t)n_th * sizeof(float), cudaMemcpyDefault);
    if (m_r)
        for (const SliceInfo &si : g->h_slices) {
            if (e != cudaSuccess) break;
            // the w lane of the slice's pixel table entries
            e = cudaMemcpy2D(m_r + si.det_off, sizeof(float),
                             reinterpret_cast<const char *>(g->dg.pix + si.pix_off) + 3 * sizeof(float),
                             sizeof(float4), sizeof(float), (size_t)si.n_det, cudaMemcpyDefault);
        }
    if (e != cudaSuccess) {
        record_error(e);
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    return EI_OK;
}

int ei_set_flat_table(ei_geometry *g, const float *table, int K)
{
    if (!g) return EI_ERR_ARG;
    if (!table || K == 0) {
        g->dg.flat_tab = nullptr;
        g->dg.flat_k = 0;
        return EI_OK;
    }
    if (K < 4 || K > 65536) return EI_ERR_ARG;
    int64_t n_px = 0;
    for (const SliceInfo &si : g->h_slices) n_px += si.n_det;
    const int64_t count = n_px * K;
    // no kernel of any stream may read the old table while it is overwritten
    cudaError_t e = cudaDeviceSynchronize();
    g->dg.flat_tab = nullptr;
    g->dg.flat_k = 0;
    if (e == cudaSuccess && count > g->flat_cap) {
        e = dev_alloc(g, &g->flat_buf, (size_t)count);
        g->flat_cap = e == cudaSuccess ? count : 0;
    }
    if (e == cudaSuccess)
        e = cudaMemcpy(g->flat_buf, table, (size_t)count * sizeof(float), cudaMemcpyDefault);
    if (e != cudaSuccess) {
        record_error(e);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
    }
    g->dg.flat_tab = g->flat_buf;
    g->dg.flat_k = K;
    return EI_OK;
}

int ei_set_linked(ei_geometry *g, double gamma)
{
    if (!g || !(gamma >= 0.0) || !isfinite(gamma)) return EI_ERR_ARG;
    g->link_gamma = (float)gamma;
    return EI_OK;
}

int ei_offset_grad(ei_geometry *g, const float *vol, const float *s_exp, float *g_mo, float *g_mr,
                   void *stream)
{
    if (!g || !vol || !s_exp || !aligned16(vol) || !aligned16(s_exp)) return EI_ERR_ARG;
    if (!g_mo && !g_mr) return EI_OK;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!g->shift_scratch) {
        e = dev_alloc(g, &g->shift_scratch, (size_t)g->sino4_count);
        if (e == cudaSuccess) e = dev_alloc(g, &g->row_sums, (size_t)std::max(1, g->dg.total_ic));
        if (e != cudaSuccess) {
            record_error(e);
            cudaGetLastError();
            return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
        }
    }
    e = counted_prep(g, (const float4 *)vol, physical_mult(g), g->link_gamma > 0.f, nullptr, st);
    if (e == cudaSuccess) e = traced_project(g, g->proj, g->link_gamma, nullptr, st);
    if (e == cudaSuccess) {
        count_launches(g, 2);
        e = launch_offset_grads(g, g->proj, s_exp, g->shift_scratch, g->row_sums, g_mo, g_mr, st);
    }
    return status_from(e);
}

int ei_objective_grad(const ei_geometry *gc, const float *vol, const float *s_exp,
                      double *S_out, float *grad, void *stream)
{
    if (!gc || !vol || !s_exp || !S_out || !aligned16(vol) || !aligned16(s_exp) ||
        (grad && !aligned16(grad)))
        return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = evaluate(g, (const float4 *)vol, s_exp, g->S_dev, (float4 *)grad, false,
                             nullptr, st);
    if (e != cudaSuccess) return status_from(e);
    cudaPointerAttributes attr{};
    e = cudaPointerGetAttributes(&attr, S_out);
    if (e != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    e = cudaMemcpyAsync(S_out, g->S_dev, sizeof(double) * g->n_slices, cudaMemcpyDefault, st);
    if (e != cudaSuccess) return status_from(e);
    if (attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        return take_device_status(g, st);        // synchronous call: report device errors too
    return EI_OK;
}

int ei_solver_state_size(const ei_geometry *g, int lbfgs_m, size_t *bytes)
{
    if (!g || !bytes || lbfgs_m < 1 || lbfgs_m > 32) return EI_ERR_ARG;
    *bytes = ei::solver_state_size(g, lbfgs_m);
    return EI_OK;
}

int ei_solver_save(const ei_geometry *g, void *buf, size_t bytes)
{
    if (!g || !buf) return EI_ERR_ARG;
    return ei::solver_save(g, buf, bytes);
}

int ei_solver_load(ei_geometry *g, int lbfgs_m, const void *buf, size_t bytes)
{
    if (!g || !buf || lbfgs_m < 1 || lbfgs_m > 32) return EI_ERR_ARG;
    return ei::solver_load(g, lbfgs_m, buf, bytes);
}

int ei_reconstruct(const ei_geometry *gc, const float *s_exp, float *vol_inout,
                   const ei_solve_opts *opts, ei_solve_report *report, void *stream)
{
    if (!gc || !s_exp || !vol_inout || !aligned16(s_exp) || !aligned16(vol_inout)) return EI_ERR_ARG;
    ei_solve_opts o;
    ei_default_solve_opts(&o);
    if (opts) o = *opts;
    if (!(o.tol >= 0) || o.max_iter < 0 || o.lbfgs_m < 1 || o.lbfgs_m > 32 || !(o.c1 > 0) ||
        o.c1 >= 1 || o.max_trials < 1 || !(o.curv_eps >= 0) || (o.resume != 0 && o.resume != 1) ||
        !(o.max_seconds >= 0))
        return EI_ERR_ARG;
    ei_geometry *g = const_cast<ei_geometry *>(gc);
    const int r = ei::reconstruct(g, s_exp, vol_inout, &o, report, (cudaStream_t)stream);
    const int d = take_device_status(g, (cudaStream_t)stream);
    return r != EI_OK ? r : d;
}

}  // extern "C"
