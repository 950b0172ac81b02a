// Illumination-curve (IC) model, residual and per-pixel gradient, fused
// (Eq. 2 with the Eq. 4 offsets, the cost of Eq. 5 and its analytic gradient).
//
// One block per sinogram row (slice, angle).  Per pixel t of the row:
//   shift = (z/period) D R[delta] + m_o(theta) + m_r(t)      (D: finite difference)
//   V     = w^2 + kappa R[sigma]
//   s_m   = A (w / sqrt(V)) exp(-R[mu] - (m - c - shift)^2 / (2 V))   for every m
//   e_m   = s_m - s_exp_m ;  objective partial sum_m e_m^2 (FP64 per block)
//   G_mu  = -sum 2 e s,  G_sh = sum 2 e s q / V,  G_V = sum 2 e s (q^2 - V) / (2 V^2)
// and the gradient sinogram row
//   g = (G_mu, (z/period) D^T G_sh, kappa G_V),
// written pair-packed (the adjoint's input layout, see ei_internal.h).
// D needs R[delta] at t +- 1 and D^T needs G_sh at t +- 1, so the whole row
// is staged in shared memory (no halo recompute, no atomics).
//
// Memory traffic per pixel (M = n_m): 12 B of projections + 4M B of s_exp
// read, 24 B of packed g written; the per-pixel flat IC table is shared by all angles
// and stays in L2.  The kernel is HBM-bound.
#include "ei_internal.h"

namespace ei {

__device__ __forceinline__ double block_sum_double(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

// (D^T g)[j] for a row of n entries (see the oracle's row-by-row definition):
// row 0 = (-1, 1)/h, row n-1 = (-1, 1)/h at (n-2, n-1), interior rows
// (-1/2, 0, 1/2)/h.
__device__ __forceinline__ float deriv_T_at(const float *gs, int j, int n, float inv_h)
{
    if (n == 1) return 0.f;
    float acc = 0.f;
    if (j == 0) acc -= gs[0] * inv_h;                     // diagonal of row 0
    if (j == n - 1) acc += gs[n - 1] * inv_h;             // diagonal of row n-1
    if (j - 1 >= 0) acc += gs[j - 1] * (j - 1 == 0 ? inv_h : 0.5f * inv_h);        // row j-1
    if (j + 1 <= n - 1) acc -= gs[j + 1] * (j + 1 == n - 1 ? inv_h : 0.5f * inv_h); // row j+1
    return acc;
}

__device__ __forceinline__ float deriv_at(const float *ps, int j, int n, float inv_h)
{
    if (n == 1) return 0.f;
    if (j == 0) return (ps[1] - ps[0]) * inv_h;
    if (j == n - 1) return (ps[n - 1] - ps[n - 2]) * inv_h;
    return (ps[j + 1] - ps[j - 1]) * (0.5f * inv_h);
}

template <int MODE>
__global__ void k_ic(DevGeom dg, const float *__restrict__ proj, const float *__restrict__ meas,
                     float *__restrict__ s_mod, float4 *__restrict__ gA, float2 *__restrict__ gB,
                     double *__restrict__ part, const int *__restrict__ active)
{
    extern __shared__ float sm[];
    __shared__ double red[32];
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const int nd = si.n_det, ndp = si.n_dp;
    const int64_t plane = (int64_t)si.n_theta * ndp;
    const int64_t rbase = (int64_t)a * ndp;
    const float *Pmu = proj + si.proj_off + rbase;
    const float *Pde = Pmu + plane;
    const float *Psg = Pde + plane;
    const float *Sx = meas + si.meas_off + rbase;      // plane k at Sx + k * plane
    const float4 *pix = dg.pix + si.pix_off;
    const float mo = dg.m_o[si.ang_off + a];
    const int n_m = dg.mc.n_m;
    const float zp = dg.mc.z_over_p, kappa = dg.mc.kappa;

    float *s_pd = sm;                  // R[delta] of the row
    float *s_gsh = sm + dg.max_ndp;    // G_shift, G_mu, G_V of the row
    float *s_gmu = s_gsh + dg.max_ndp;
    float *s_gv = s_gmu + dg.max_ndp;

    for (int gi = threadIdx.x; gi < (ndp >> 2); gi += blockDim.x)
        reinterpret_cast<float4 *>(s_pd)[gi] = __ldg(reinterpret_cast<const float4 *>(Pde) + gi);
    __syncthreads();

    double e2 = 0.0;
    bool out_of_domain = false;
    for (int j = threadIdx.x; j < ndp; j += blockDim.x) {
        float gmu = 0.f, gsh = 0.f, gvv = 0.f;
        if (j < nd) {
            const float4 fl = __ldg(pix + j);     // A, c, w, m_r
            const float shift = zp * deriv_at(s_pd, j, nd, si.inv_pitch) + mo + fl.w;
            const float V = fmaf(kappa, __ldg(Psg + j), fl.z * fl.z);
            if (!(V > 0.01f * fl.z * fl.z)) out_of_domain = true;
            const float Vs = fmaxf(V, 1e-30f);
            const float iV = 1.0f / Vs;
            const float amp = fl.x * fl.z * rsqrtf(Vs);
            const float pmu = __ldg(Pmu + j);
            float st = 0.f, stq = 0.f, stq2 = 0.f, e2f = 0.f;
            for (int k = 0; k < n_m; ++k) {
                const float qd = dg.mc.m[k] - fl.y - shift;
                const float sv = amp * expf(-pmu - 0.5f * qd * qd * iV);
                if (MODE == IC_MODEL) {
                    s_mod[si.meas_off + rbase + (int64_t)k * plane + j] = sv;
                } else {
                    const float e = sv - __ldcs(Sx + (int64_t)k * plane + j);
                    e2f = fmaf(e, e, e2f);
                    if (MODE == IC_OBJECTIVE_GRAD) {
                        const float t = 2.f * e * sv;
                        st += t;
                        stq = fmaf(t, qd, stq);
                        stq2 = fmaf(t * qd, qd, stq2);
                    }
                }
            }
            e2 += (double)e2f;
            gmu = -st;
            gsh = stq * iV;
            gvv = 0.5f * iV * (stq2 * iV - st);
        } else if (MODE == IC_MODEL) {
            for (int k = 0; k < n_m; ++k) s_mod[si.meas_off + rbase + (int64_t)k * plane + j] = 0.f;
        }
        if (MODE == IC_OBJECTIVE_GRAD) {
            s_gsh[j] = gsh;
            s_gmu[j] = gmu;
            s_gv[j] = gvv;
        }
    }
    if (MODE == IC_MODEL) return;
    if (MODE == IC_OBJECTIVE_GRAD) {
        // g_delta = (z/period) D^T G_shift (into the R[delta] row, no longer needed) and
        // g_sigma = kappa G_V; then the packed row: entry of pixel j holds g(j), g(j + 1)
        __syncthreads();
        for (int j = threadIdx.x; j < nd; j += blockDim.x) {
            s_pd[j] = zp * deriv_T_at(s_gsh, j, nd, si.inv_pitch);
            s_gv[j] *= kappa;
        }
        __syncthreads();
        const int64_t dst = si.gp_off + (int64_t)a * si.gw + si.marg;
        for (int j = (int)threadIdx.x - 1; j < nd; j += blockDim.x) {
            float lx = 0.f, ly = 0.f, lz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
            if (j >= 0) lx = s_gmu[j], ly = s_pd[j], lz = s_gv[j];
            if (j + 1 < nd) hx = s_gmu[j + 1], hy = s_pd[j + 1], hz = s_gv[j + 1];
            gA[dst + j] = make_float4(lx, ly, lz, hx);
            gB[dst + j] = make_float2(hy, hz);
        }
    }
    const int bad = __syncthreads_or(out_of_domain ? 1 : 0);
    const double tot = block_sum_double(e2, red);
    if (threadIdx.x == 0) part[row] = bad ? __longlong_as_double(0x7ff0000000000000LL) : tot;
}

cudaError_t launch_ic(const ei_geometry *g, const float *proj, const float *meas, float *s_mod,
                      double *part, IcMode mode, const int *active, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    int threads = (g->dg.max_ndp + 31) / 32 * 32;
    if (threads > 256) threads = 256;
    const size_t smem = (size_t)4 * g->dg.max_ndp * sizeof(float);
    switch (mode) {
    case IC_MODEL:
        k_ic<IC_MODEL><<<g->dg.total_ic, threads, smem, st>>>(g->dg, proj, meas, s_mod, g->gA,
                                                               g->gB, part, active);
        break;
    case IC_OBJECTIVE:
        k_ic<IC_OBJECTIVE><<<g->dg.total_ic, threads, smem, st>>>(g->dg, proj, meas, s_mod,
                                                                   g->gA, g->gB, part, active);
        break;
    default:
        k_ic<IC_OBJECTIVE_GRAD><<<g->dg.total_ic, threads, smem, st>>>(g->dg, proj, meas, s_mod,
                                                                        g->gA, g->gB, part, active);
        break;
    }
    return cudaGetLastError();
}

cudaError_t ic_set_smem_limit()
{
    const int bytes = 4 * EI_MAX_NDET * (int)sizeof(float);
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_MODEL>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_OBJECTIVE>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_OBJECTIVE_GRAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return cudaSuccess;
}

}  // namespace ei
