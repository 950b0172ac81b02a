// ei_objective_grad_noalloc: S and its gradient for one slice without any
// device allocation.  Every intermediate (geometry tables, staged volume,
// projections, gradient sinogram, partial sums) lives in one file-scope
// __device__ array of EI_NOALLOC_SCRATCH_BYTES; the kernels are the same ones
// ei_objective_grad runs.
//
// Who needs this: code that runs while a CUDA stream is being captured into a
// graph (cudaMalloc cannot be captured), frameworks that have reserved the
// device memory in their own pool and forbid allocations outside it, and
// latency-sensitive loops that cannot afford cudaMalloc's implicit device
// synchronisation.  Such callers cannot call ei_setup_geometry either (it
// allocates the workspace), so this entry point takes the geometry
// description directly.
#include <math.h>

#include <algorithm>
#include <mutex>

#include "ei_internal.h"

namespace ei {

cudaError_t ic_set_smem_limit();

namespace {

// The scratch array.  In host code `g_scratch` only names the symbol; its
// device address comes from cudaGetSymbolAddress (see scratch_for_device).
__device__ __align__(256) unsigned char g_scratch[EI_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
unsigned char *g_dev_ptr[kMaxDevices] = {};

// Once per device, with that device current: resolve the scratch address and
// raise the IC kernel's shared-memory limit.
cudaError_t scratch_for_device(int dev, unsigned char **out)
{
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_dev_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return e;
        e = ic_set_smem_limit();
        if (e != cudaSuccess) return e;
        g_dev_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_dev_ptr[dev];
    return cudaSuccess;
}

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

struct Counts {
    int c[5];   // work items of the projector, IC rows, adjoint tiles, staging tiles, vector blocks
};

// Geometry tables of one slice, written on the device from the description
// (same formulas as ei_setup_geometry's host code).
__global__ void k_noalloc_tables(SliceInfo si, double pitch, const double *theta, int uniform_theta,
                                 const float *fA, const float *fc, const float *fw,
                                 const float *mo, const float *mr, AngleInfo *ang, float *m_o,
                                 float4 *pix, SliceInfo *slices, int *prefixes, Counts counts)
{
    const int tid = blockIdx.x * blockDim.x + threadIdx.x;
    const int stride = gridDim.x * blockDim.x;
    for (int a = tid; a < si.n_theta; a += stride) {
        const double th = uniform_theta ? a * 3.141592653589793 / si.n_theta : theta[a];
        ang[a] = make_angle_info(th, si.n, pitch);
        m_o[a] = mo ? mo[a] : 0.f;
    }
    for (int j = tid; j < si.n_dp; j += stride)
        pix[j] = j < si.n_det ? make_float4(fA[j], fc[j], fw[j], mr ? mr[j] : 0.f)
                              : make_float4(0.f, 0.f, 1.f, 0.f);
    if (tid == 0) {
        slices[0] = si;
        for (int k = 0; k < 5; ++k) {
            prefixes[2 * k] = 0;
            prefixes[2 * k + 1] = counts.c[k];
        }
    }
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
    // ---- arguments (nothing touches the GPU before these pass)
    if (!d || !vol || !s_exp || !S_out) return EI_ERR_ARG;
    if ((((uintptr_t)vol) & 15u) || (((uintptr_t)s_exp) & 15u) || (grad && (((uintptr_t)grad) & 15u)))
        return EI_ERR_ARG;
    if (d->n < 1 || d->n > 16384 || d->n_theta < 1 || d->n_det < 1 || d->n_det > EI_MAX_NDET ||
        !(d->pitch_cm > 0) || !isfinite(d->pitch_cm) || d->n_m < 1 || d->n_m > EI_MAX_NM || !d->m ||
        !(d->z_cm >= 0) || !(d->period_cm > 0) || !(d->kappa_sigma >= 0) || !d->flat_A ||
        !d->flat_c || !d->flat_w)
        return EI_ERR_ARG;
    for (int c = 0; c < 3; ++c)
        if (!(d->scale[c] > 0) || !(d->lambda[c] >= 0) || !isfinite(d->lambda[c])) return EI_ERR_ARG;
    for (int k = 0; k < d->n_m; ++k)
        if (!isfinite(d->m[k])) return EI_ERR_ARG;

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
    const int adj_rows = backproject_variant_rows(0);
    const int n_fwd = ((nth + angles - 1) / angles) * ((ndp + rays - 1) / rays);
    const int n_adj = ((n + ADJ_TC - 1) / ADJ_TC) * ((n + adj_rows - 1) / adj_rows);
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
    const size_t o_theta = cv.take(d->theta ? (size_t)nth * sizeof(double) : 0);
    const size_t o_flat = cv.take((size_t)3 * nd * sizeof(float));
    const size_t o_mos = cv.take(d->m_o ? (size_t)nth * sizeof(float) : 0);
    const size_t o_mrs = cv.take(d->m_r ? (size_t)nd * sizeof(float) : 0);
    const size_t o_xpA = cv.take((size_t)pp * sizeof(float4));
    const size_t o_xtA = cv.take((size_t)pp * sizeof(float4));
    const size_t o_xpB = cv.take((size_t)pp * sizeof(float2));
    const size_t o_xtB = cv.take((size_t)pp * sizeof(float2));
    const size_t o_proj = cv.take((size_t)3 * nth * ndp * sizeof(float));
    const size_t o_gA = cv.take((size_t)gp * sizeof(float4));
    const size_t o_gB = cv.take((size_t)gp * sizeof(float2));
    const size_t o_pic = cv.take((size_t)nth * sizeof(double));
    const size_t o_pad = cv.take((size_t)n_adj * sizeof(double));
    const size_t o_S = cv.take(sizeof(double));
    if (cv.used > (size_t)EI_NOALLOC_SCRATCH_BYTES) return EI_ERR_ARG;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return EI_ERR_CUDA;
    unsigned char *base = nullptr;
    e = scratch_for_device(dev, &base);
    if (e != cudaSuccess) return EI_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)stream;

    // ---- inputs of the tables (host or device arrays) into the scratch
    float *flat = (float *)(base + o_flat);
    e = cudaMemcpyAsync(flat, d->flat_A, nd * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flat + nd, d->flat_c, nd * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(flat + 2 * nd, d->flat_w, nd * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess && d->theta)
        e = cudaMemcpyAsync(base + o_theta, d->theta, nth * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d->m_o)
        e = cudaMemcpyAsync(base + o_mos, d->m_o, nth * sizeof(float), cudaMemcpyDefault, st);
    if (e == cudaSuccess && d->m_r)
        e = cudaMemcpyAsync(base + o_mrs, d->m_r, nd * sizeof(float), cudaMemcpyDefault, st);
    // the gradient sinogram's margins and padding must read as zero; the scratch keeps
    // whatever the previous call left, so clear it
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_gA, 0, (size_t)gp * sizeof(float4), st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base + o_gB, 0, (size_t)gp * sizeof(float2), st);
    if (e != cudaSuccess) return status_of(e);

    si.ang_off = 0;
    si.pix_off = 0;
    si.vol_off = 0;
    si.pp_off = 0;
    si.gp_off = 0;
    si.sino_off = 0;
    si.proj_off = 0;
    si.meas_off = 0;
    int *pref = (int *)(base + o_pref);
    const Counts counts{{n_fwd, nth, n_adj, n_prep, n_vec}};
    k_noalloc_tables<<<std::max(1, (std::max(nth, ndp) + 255) / 256), 256, 0, st>>>(
        si, d->pitch_cm, d->theta ? (const double *)(base + o_theta) : nullptr, d->theta ? 0 : 1,
        flat, flat + nd, flat + 2 * nd, d->m_o ? (const float *)(base + o_mos) : nullptr,
        d->m_r ? (const float *)(base + o_mrs) : nullptr, (AngleInfo *)(base + o_ang),
        (float *)(base + o_mo), (float4 *)(base + o_pix), (SliceInfo *)(base + o_slice), pref,
        counts);
    e = cudaGetLastError();
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
    g.part_adj = (double *)(base + o_pad);
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
    return status_of(e);
}
