// ei_objective_grad_noalloc: S and its gradient for one slice without any
// device allocation.  Every intermediate (geometry tables, staged volume,
// projections, gradient sinogram, partial sums) lives in one file-scope
// __device__ array of EI_NOALLOC_SCRATCH_BYTES; the kernels are the same ones
// ei_objective_grad runs (variant 0 of each).
//
// Who needs this: callers that may not allocate GPU memory themselves, such
// as frameworks that have reserved the device memory for their own pool and
// forbid allocations outside it, and latency-sensitive loops that cannot
// afford cudaMalloc's implicit device synchronisation.  Such callers cannot
// call ei_setup_geometry either (it allocates the workspace), so this entry
// point takes the geometry description directly.
#include <math.h>

#include <algorithm>
#include <vector>

#include "ei_internal.h"

namespace ei {

cudaError_t ic_set_smem_limit();

namespace {

// The scratch array.  In host code `g_scratch` only names the symbol; its
// device address in the current context comes from cudaGetSymbolAddress,
// which every call asks for (a cached address would outlive a context reset).
__device__ __align__(256) unsigned char g_scratch[EI_NOALLOC_SCRATCH_BYTES];

// Bump allocator over the scratch array (256-byte aligned pieces).
struct Carver {
    size_t used = 0;
    size_t take(size_t bytes)
    {
        const size_t off = used;
        used += (bytes + 255) / 256 * 256;
        return off;
    }
};

// n floats from host or device memory into dst, ordered after the work queued
// on st (false: not a valid pointer, or the copy failed).
bool fetch(const float *src, int n, std::vector<float> &dst, cudaStream_t st)
{
    dst.resize(n);
    cudaError_t e = cudaMemcpyAsync(dst.data(), src, (size_t)n * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return true;
}

int status_of(cudaError_t e)
{
    return e == cudaSuccess ? EI_OK : EI_ERR_CUDA;
}

}  // namespace
}  // namespace ei

using namespace ei;

extern "C" int ei_objective_grad_noalloc(const ei_geometry_desc *d, const float *vol,
                                         const float *s_exp, double *S_out, float *grad,
                                         void *stream)
{
    // ---- arguments (nothing is queued on the GPU before these pass; the same
    // checks as ei_setup_geometry)
    if (!d || !vol || !s_exp || !S_out) return EI_ERR_ARG;
    if ((((uintptr_t)vol) & 15u) || (((uintptr_t)s_exp) & 15u) || (grad && (((uintptr_t)grad) & 15u)))
        return EI_ERR_ARG;
    if (d->n < 1 || d->n > 16384 || d->n_theta < 1 || d->n_det < 1 || d->n_det > EI_MAX_NDET ||
        !(d->pitch_cm > 0) || !isfinite(d->pitch_cm) || d->n_m < 1 || d->n_m > EI_MAX_NM || !d->m ||
        !(d->z_cm >= 0) || !isfinite(d->z_cm) || !(d->period_cm > 0) || !isfinite(d->period_cm) ||
        !(d->kappa_sigma >= 0) || !isfinite(d->kappa_sigma) || !d->flat_A || !d->flat_c ||
        !d->flat_w)
        return EI_ERR_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(d->scale[c] > 0) || !isfinite(d->scale[c]) || !(d->lambda[c] >= 0) ||
            !isfinite(d->lambda[c]))
            return EI_ERR_ARG;
    for (int k = 0; k < d->n_m; ++k)
        if (!isfinite(d->m[k])) return EI_ERR_ARG;
    if (d->theta)
        for (int a = 0; a < d->n_theta; ++a)
            if (!isfinite(d->theta[a])) return EI_ERR_ARG;

    const int n = d->n, nth = d->n_theta, nd = d->n_det, ndp = (nd + 3) / 4 * 4;
    SliceInfo si{};
    si.n = n;
    si.n_theta = nth;
    si.n_det = nd;
    si.n_dp = ndp;
    si.pitch = (float)d->pitch_cm;
    si.inv_pitch = (float)(1.0 / d->pitch_cm);
    {
        const double hn = 0.5 * (n - 1);
        const int cpad = (n + ADJ_TC - 1) / ADJ_TC * ADJ_TC;
        const int rpad = (n + ADJ_MAX_TR - 1) / ADJ_MAX_TR * ADJ_MAX_TR;
        const double mdx = std::max(hn, cpad - 1 - hn), mdy = std::max(hn, rpad - 1 - hn);
        si.marg = std::max(2, (int)ceil(sqrt(mdx * mdx + mdy * mdy) - 0.5 * (nd - 1)) + 3);
    }
    si.gw = ndp + 2 * si.marg;
    // default kernel variants (0): their work decompositions
    int rays = 0, angles = 0;
    project_variant_shape(0, &rays, &angles);
    const int n_fwd = ((nth + angles - 1) / angles) * ((ndp + rays - 1) / rays);
    const int n_adj = backproject_variant_items(0, n);
    const int pt = (n + 1 + PREP_TILE - 1) / PREP_TILE;
    const int n_prep = pt * pt;
    const int n_vec = (int)(((int64_t)n * n + VEC_BLK - 1) / VEC_BLK);
    const int64_t pp = (int64_t)n * (n + 1), gp = (int64_t)nth * si.gw;

    // ---- scratch layout; sizes beyond the array are rejected before any GPU work
    Carver cv;
    const size_t o_slice = cv.take(sizeof(SliceInfo));
    const size_t o_pref = cv.take(10 * sizeof(int));
    const size_t o_ang = cv.take((size_t)nth * sizeof(AngleInfo));
    const size_t o_mo = cv.take((size_t)nth * sizeof(float));
    const size_t o_pix = cv.take((size_t)ndp * sizeof(float4));
    const size_t o_xpA = cv.take((size_t)pp * sizeof(float4));
    const size_t o_xtA = cv.take((size_t)pp * sizeof(float4));
    const size_t o_xpB = cv.take((size_t)pp * sizeof(float2));
    const size_t o_xtB = cv.take((size_t)pp * sizeof(float2));
    const size_t o_proj = cv.take((size_t)3 * nth * ndp * sizeof(float));
    const size_t o_gA = cv.take((size_t)gp * sizeof(float4));
    const size_t o_gB = cv.take((size_t)gp * sizeof(float2));
    const size_t o_pic = cv.take((size_t)nth * sizeof(double));
    const size_t o_preg = cv.take((size_t)n_vec * sizeof(double));
    const size_t o_S = cv.take(sizeof(double));
    const size_t o_status = cv.take(sizeof(int));
    if (cv.used > (size_t)EI_NOALLOC_SCRATCH_BYTES) return EI_ERR_ARG;

    // ---- the per-pixel and per-angle inputs (host or device arrays), checked
    // and tabulated on the host exactly as ei_setup_geometry does
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<float> fA, fc, fw, fmo, fmr;
    if (!fetch(d->flat_A, nd, fA, st) || !fetch(d->flat_c, nd, fc, st) || !fetch(d->flat_w, nd, fw, st) ||
        (d->m_o && !fetch(d->m_o, nth, fmo, st)) || (d->m_r && !fetch(d->m_r, nd, fmr, st)))
        return EI_ERR_ARG;
    for (int j = 0; j < nd; ++j)
        if (!(fw[j] > 0) || !isfinite(fA[j]) || !isfinite(fc[j])) return EI_ERR_ARG;
    std::vector<AngleInfo> ang(nth);
    std::vector<float> m_o(nth);
    for (int a = 0; a < nth; ++a) {
        const double th = d->theta ? d->theta[a] : a * M_PI / nth;
        ang[a] = make_angle_info(th, n, d->pitch_cm);
        m_o[a] = d->m_o ? fmo[a] : 0.f;
    }
    std::vector<float4> pix(ndp);
    for (int j = 0; j < ndp; ++j)
        pix[j] = j < nd ? make_float4(fA[j], fc[j], fw[j], d->m_r ? fmr[j] : 0.f)
                        : make_float4(0.f, 0.f, 1.f, 0.f);
    si.ang_off = 0;
    si.pix_off = 0;
    si.det_off = 0;
    si.vol_off = 0;
    si.pp_off = 0;
    si.gp_off = 0;
    si.sino_off = 0;
    si.proj_off = 0;
    si.meas_off = 0;
    // work-item prefix tables [0, count] of the projector, IC rows, adjoint,
    // staging tiles and vector blocks
    const int pref_h[10] = {0, n_fwd, 0, nth, 0, n_adj, 0, n_prep, 0, n_vec};

    // ---- the scratch array's address in the current context
    unsigned char *base = nullptr;
    {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
            cudaGetLastError();
            return EI_ERR_CUDA;
        }
        base = static_cast<unsigned char *>(p);
    }
    if (ic_set_smem_limit() != cudaSuccess) {
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return EI_ERR_CUDA;

    // ---- tables into the scratch (the host buffers may be released once a
    // pageable copy returns); the gradient sinogram's margins and padding must
    // read as zero, and the scratch keeps whatever the previous call left, so
    // clear it
    cudaError_t e = cudaMemcpyAsync(base + o_slice, &si, sizeof si, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_pref, pref_h, sizeof pref_h, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_ang, ang.data(), nth * sizeof(AngleInfo), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_mo, m_o.data(), nth * sizeof(float), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(base + o_pix, pix.data(), ndp * sizeof(float4), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_gA, 0, (size_t)gp * sizeof(float4), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_gB, 0, (size_t)gp * sizeof(float2), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_status, 0, sizeof(int), st);
    if (e != cudaSuccess) return status_of(e);

    // ---- a geometry view over the scratch (no host or device allocation)
    ei_geometry g;
    g.n_slices = 1;
    g.n_m = d->n_m;
    g.device = dev;
    for (int c = 0; c < 3; ++c) {
        g.lambda[c] = (float)d->lambda[c];
        g.scale[c] = (float)d->scale[c];
    }
    int *pref = (int *)(base + o_pref);
    DevGeom &dg = g.dg;
    dg.slices = (const SliceInfo *)(base + o_slice);
    dg.ang = (const AngleInfo *)(base + o_ang);
    dg.m_o = (const float *)(base + o_mo);
    dg.pix = (const float4 *)(base + o_pix);
    dg.ic_prefix = pref + 2;
    dg.prep_prefix = pref + 6;
    dg.vec_prefix = pref + 8;
    dg.n_slices = 1;
    dg.total_ic = nth;
    g.fwd_variant.id = 0;
    g.fwd_variant.prefix = pref + 0;
    g.fwd_variant.total = n_fwd;
    g.adj_variant.id = 0;
    g.adj_variant.prefix = pref + 4;
    g.adj_variant.total = n_adj;
    dg.total_prep = n_prep;
    dg.total_vec = n_vec;
    dg.max_ndp = ndp;
    dg.max_n_theta = nth;
    dg.status = (int *)(base + o_status);
    dg.mc.z_over_p = (float)(d->z_cm / d->period_cm);
    dg.mc.kappa = (float)d->kappa_sigma;
    dg.mc.n_m = d->n_m;
    for (int k = 0; k < d->n_m; ++k) dg.mc.m[k] = (float)d->m[k];
    g.xpA = (float4 *)(base + o_xpA);
    g.xtA = (float4 *)(base + o_xtA);
    g.xpB = (float2 *)(base + o_xpB);
    g.xtB = (float2 *)(base + o_xtB);
    g.proj = (float *)(base + o_proj);
    g.gA = (float4 *)(base + o_gA);
    g.gB = (float2 *)(base + o_gB);
    g.part_ic = (double *)(base + o_pic);
    g.part_reg = (double *)(base + o_preg);
    g.S_dev = (double *)(base + o_S);
    g.vol_count = (int64_t)n * n;

    e = evaluate(&g, (const float4 *)vol, s_exp, g.S_dev, (float4 *)grad, false, nullptr, st);
    if (e != cudaSuccess) return status_of(e);
    cudaPointerAttributes attr{};
    if (cudaPointerGetAttributes(&attr, S_out) != cudaSuccess) {
        cudaGetLastError();
        attr.type = cudaMemoryTypeUnregistered;
    }
    e = cudaMemcpyAsync(S_out, g.S_dev, sizeof(double), cudaMemcpyDefault, st);
    if (e == cudaSuccess && attr.type != cudaMemoryTypeDevice && attr.type != cudaMemoryTypeManaged)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && kDeviceChecks) {      // check builds: report a fired bounds check
        int h = 0;
        e = cudaMemcpyAsync(&h, base + o_status, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess && h != 0) return h;
    }
    return status_of(e);
}
