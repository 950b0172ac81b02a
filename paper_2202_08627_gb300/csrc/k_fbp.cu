// Non-iterative (single-shot) reconstruction: the warm-start input.
//
// The paper's non-iterative baseline retrieves the projection from a single
// mask position by Eq. 3 and inverts the Radon transform with a filtered
// back-projection (scikit-image).  With M mask positions and three channels,
// the retrieval here uses the moments of the measured IC over m against those
// of the flat IC, per pixel:
//   T = sum s / sum f               -> R[mu]    = -ln T
//   shift = mean(s) - mean(f)       -> R[delta] = (period/z) pitch cumsum_t(shift),
//                                      minus the line that makes both row ends 0
//   dv = max(0, var(s) - var(f))    -> R[sigma] = dv / kappa
// then every channel is ramp-filtered along t (the spatial Ram-Lak kernel:
// 1/(4 pitch^2) at 0, -1/(pi^2 d^2 pitch^2) at odd offsets d) and
// back-projected with the library's adjoint, scaled by pi / n_theta / pitch.
//
// One block per sinogram row; the row lives in shared memory: the moments,
// a deterministic block scan for the running sum, the filter (a direct
// convolution over the row, O(n_det^2 / 2) per row), and the packed write-out
// that the adjoint kernel reads.
#include "ei_internal.h"

namespace ei {

namespace {

// Inclusive prefix sum of v[0..n) in place, fixed order, accumulated in FP64
// (chunk per thread: its total, a scan of the totals, then the chunk's running
// sums from its offset), each result rounded once to FP32.
__device__ void block_inclusive_scan(float *v, int n, double *tot)
{
    const int T = blockDim.x, t = threadIdx.x;
    const int chunk = (n + T - 1) / T;
    const int b = t * chunk, e = min(n, b + chunk);
    double acc = 0.0;
    for (int i = b; i < e; ++i) acc += (double)v[i];
    tot[t] = acc;
    __syncthreads();
    if (t == 0) {
        double run = 0.0;
        for (int i = 0; i < T; ++i) {
            const double x = tot[i];
            tot[i] = run;        // exclusive offsets
            run += x;
        }
    }
    __syncthreads();
    double run = tot[t];
    for (int i = b; i < e; ++i) {
        run += (double)v[i];
        v[i] = (float)run;
    }
    __syncthreads();
}

// Ram-Lak filter with the FBP scale, q = (pi / n_theta) / pitch^2
// (p/4 - sum_odd p(j-d) / (pi^2 d^2)), of three rows (w[d] = 1/(pi^2 d^2) at odd
// d, prepared by the caller), then the write for the adjoint in the layout
// the selected adjoint variant reads: pair-packed (the entry of pixel j holds
// q(j) and q(j + 1)) or, with `mirror`, mirror-interleaved (pixel j and pixel
// n_det - 1 - j).  Ends with the block's writes.
__device__ void ramp_filter_write(const SliceInfo &si, int a, const float *pm, const float *pd,
                                  const float *ps, float *qm, float *qd, float *qs,
                                  const float *w, float4 *gA, float2 *gB, bool mirror)
{
    const int nd = si.n_det;
    const float K = 3.14159265358979f / (float)si.n_theta / (si.pitch * si.pitch);
    for (int j = threadIdx.x; j < nd; j += blockDim.x) {
        float am = 0.25f * pm[j], ad = 0.25f * pd[j], as = 0.25f * ps[j];
        for (int d = 1; d < nd; d += 2) {
            const float wd = w[d];
            if (j - d >= 0) am -= wd * pm[j - d], ad -= wd * pd[j - d], as -= wd * ps[j - d];
            if (j + d < nd) am -= wd * pm[j + d], ad -= wd * pd[j + d], as -= wd * ps[j + d];
        }
        qm[j] = K * am, qd[j] = K * ad, qs[j] = K * as;
    }
    __syncthreads();
    const int64_t dst = si.gp_off + (int64_t)a * si.gw + si.marg;
    for (int j = (int)threadIdx.x - 1; j < nd; j += blockDim.x) {
        if (mirror) {
            const int jm = nd - 1 - j;
            gA[dst + j] = j >= 0 ? make_float4(qm[j], qm[jm], qd[j], qd[jm])
                                 : make_float4(0.f, 0.f, 0.f, 0.f);
            gB[dst + j] = j >= 0 ? make_float2(qs[j], qs[jm]) : make_float2(0.f, 0.f);
            continue;
        }
        float lx = 0.f, ly = 0.f, lz = 0.f, hx = 0.f, hy = 0.f, hz = 0.f;
        if (j >= 0) lx = qm[j], ly = qd[j], lz = qs[j];
        if (j + 1 < nd) hx = qm[j + 1], hy = qd[j + 1], hz = qs[j + 1];
        gA[dst + j] = make_float4(lx, ly, lz, hx);
        gB[dst + j] = make_float2(hy, hz);
    }
}

}  // namespace

__global__ void k_single_shot(DevGeom dg, const float *__restrict__ meas, float4 *__restrict__ gA,
                              float2 *__restrict__ gB)
{
    extern __shared__ float sm[];
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const int nd = si.n_det, ndp = si.n_dp;
    const int64_t plane = (int64_t)si.n_theta * ndp;
    const float *Sx = meas + si.meas_off + (int64_t)a * ndp;
    const float4 *pix = dg.pix + si.pix_off;
    const float mo = dg.m_o[si.ang_off + a];
    const int n_m = dg.mc.n_m;
    const int mx = dg.max_ndp;
    float *pm = sm, *pd = sm + mx, *ps = sm + 2 * mx, *w = sm + 3 * mx;
    double *tot = reinterpret_cast<double *>(sm + 4 * mx);     // blockDim doubles

    // ---- moments of the measured and of the flat IC, per pixel, in FP64 (the
    // variance difference cancels)
    for (int j = threadIdx.x; j < nd; j += blockDim.x) {
        const float4 fl = __ldg(pix + j);            // A, c, w, m_r
        double S0 = 0.0, S1 = 0.0, S2 = 0.0, F0 = 0.0, F1 = 0.0, F2 = 0.0;
        for (int k = 0; k < n_m; ++k) {
            const double mk = dg.mc.m[k];
            const double sv = __ldg(Sx + (int64_t)k * plane + j);
            const float dm = (dg.mc.m[k] - fl.y) / fl.z;
            const double fv = (double)(fl.x * expf(-0.5f * dm * dm));
            S0 += sv, S1 = fma(mk, sv, S1), S2 = fma(mk * mk, sv, S2);
            F0 += fv, F1 = fma(mk, fv, F1), F2 = fma(mk * mk, fv, F2);
        }
        const double T = S0 / F0;
        const double cs = S0 != 0.0 ? S1 / S0 : 0.0, cf = F1 / F0;
        const double vs = S0 != 0.0 ? S2 / S0 - cs * cs : 0.0, vf = F2 / F0 - cf * cf;
        pm[j] = (float)(-log(fmax(T, 1e-6)));
        pd[j] = (float)(cs - cf) - mo - fl.w;
        ps[j] = dg.mc.kappa > 0.f ? (float)(fmax(vs - vf, 0.0) / dg.mc.kappa) : 0.f;
    }
    // filter weights 1/(pi^2 d^2) for odd d
    for (int d = threadIdx.x; d < nd; d += blockDim.x)
        w[d] = (d & 1) ? 1.f / (9.8696044010893586f * (float)d * (float)d) : 0.f;
    __syncthreads();

    // ---- R[delta] = (period/z) pitch running sum of the shift, ends pinned to 0
    block_inclusive_scan(pd, nd, tot);
    {
        const float k = si.pitch / dg.mc.z_over_p;
        const float last = pd[nd - 1];
        for (int j = threadIdx.x; j < nd; j += blockDim.x)
            pd[j] = k * (pd[j] - last * (float)(j + 1) / (float)nd);
    }
    __syncthreads();

    // ---- ramp filter and FBP scale, written pair-packed for the adjoint
    float *qm = reinterpret_cast<float *>(tot + blockDim.x);   // filtered rows (3 x max_ndp)
    ramp_filter_write(si, a, pm, pd, ps, qm, qm + mx, qm + 2 * mx, w, gA, gB, dg.gmirror != 0);
}

// ---------------------------------------------------------------------------
// The paper's single-shot retrieval (Eq. 3) for the linked unknown
// (mu = h, delta = gamma h).  Linearising Eq. 4 at one mask position m gives
// s / f = (1 + a d/dt) T with T = exp(-R[h]) and a = (z/period) gamma f'(m)/f(m)
// (f: the flat IC averaged over the pixels); Eq. 3 divides by (1 + i q a) in
// Fourier space.  That division is a circular convolution along t with the
// real kernel k_n = Re (1/N) sum_j e^{2 pi i j n / N} / (1 + i a q_j),
// q_j = 2 pi f_j / (N pitch) (f_j the signed DFT frequency index), built per
// slice (FP64 sums) and applied per row in shared memory; then R[h] = -ln T,
// ramp filter and the adjoint's FBP as for the moment retrieval.
// ---------------------------------------------------------------------------
__global__ void k_eq3_kernel(DevGeom dg, int m_index, float gamma, float *__restrict__ ker)
{
    __shared__ double red[2][32];
    const SliceInfo si = dg.slices[blockIdx.x];
    const int N = si.n_det;
    const float4 *pix = dg.pix + si.pix_off;
    const double m = dg.mc.m[m_index];
    // pixel-averaged flat IC and its derivative in m at m
    double sf = 0.0, sdf = 0.0;
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float4 fl = pix[j];                        // A, c, w, m_r
        const double d = m - fl.y, w2 = (double)fl.z * fl.z;
        const double f = fl.x * exp(-d * d / (2.0 * w2));
        sf += f;
        sdf -= f * d / w2;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sf += __shfl_down_sync(0xffffffffu, sf, o);
        sdf += __shfl_down_sync(0xffffffffu, sdf, o);
    }
    if ((threadIdx.x & 31) == 0) red[0][threadIdx.x >> 5] = sf, red[1][threadIdx.x >> 5] = sdf;
    __syncthreads();
    if (threadIdx.x < 32) {
        const int nw = blockDim.x >> 5;
        double a0 = threadIdx.x < nw ? red[0][threadIdx.x] : 0.0;
        double a1 = threadIdx.x < nw ? red[1][threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            a0 += __shfl_down_sync(0xffffffffu, a0, o);
            a1 += __shfl_down_sync(0xffffffffu, a1, o);
        }
        if (threadIdx.x == 0) red[0][0] = a0, red[1][0] = a1;
    }
    __syncthreads();
    const double a = (double)dg.mc.z_over_p * gamma * red[1][0] / red[0][0];
    const double dq = 2.0 * 3.14159265358979323846 / ((double)N * si.pitch);
    for (int n = threadIdx.x; n < N; n += blockDim.x) {
        double acc = 0.0;
        for (int j = 0; j < N; ++j) {
            const int fj = 2 * j < N ? j : j - N;           // signed frequency index
            const double aq = a * dq * fj;
            const int r = (int)(((long long)j * n) % N);     // exact phase reduction
            float sn, cn;
            sincospif(2.0f * (float)r / (float)N, &sn, &cn);
            acc += ((double)cn + aq * sn) / (1.0 + aq * aq);
        }
        ker[si.det_off + n] = (float)(acc / N);
    }
}

__global__ void k_single_shot_eq3(DevGeom dg, const float *__restrict__ meas, int m_index,
                                  float gamma, const float *__restrict__ ker,
                                  float4 *__restrict__ gA, float2 *__restrict__ gB)
{
    extern __shared__ float sm[];
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const int N = si.n_det;
    const int mx = dg.max_ndp;
    float *y = sm, *kr = sm + mx, *ph = sm + 2 * mx, *pd = sm + 3 * mx, *zero = sm + 4 * mx;
    float *w = sm + 5 * mx, *q = sm + 6 * mx;              // q: 3 x mx filtered rows
    const float *Sx = meas + si.meas_off + (int64_t)m_index * si.n_theta * si.n_dp +
                      (int64_t)a * si.n_dp;
    const float4 *pix = dg.pix + si.pix_off;
    const float m = dg.mc.m[m_index];
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        const float4 fl = __ldg(pix + j);
        const float d = (m - fl.y) / fl.z;
        y[j] = Sx[j] / (fl.x * expf(-0.5f * d * d));       // s / f at this mask position
        kr[j] = ker[si.det_off + j];
        zero[j] = 0.f;
        w[j] = (j & 1) ? 1.f / (9.8696044010893586f * (float)j * (float)j) : 0.f;
    }
    __syncthreads();
    // T = k (*) y (circular), R[h] = -ln T, R[delta] = gamma R[h]
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
        float T = 0.f;
        int i = j;                                          // (j - n) mod N, n = 0, 1, ...
        for (int n = 0; n < N; ++n) {
            T = fmaf(kr[n], y[i], T);
            i = i == 0 ? N - 1 : i - 1;
        }
        const float p = -logf(fmaxf(T, 1e-6f));
        ph[j] = p;
        pd[j] = gamma * p;
    }
    __syncthreads();
    ramp_filter_write(si, a, ph, pd, zero, q, q + mx, q + 2 * mx, w, gA, gB, dg.gmirror != 0);
}

static const int kEq3SmemLimit = 220 * 1024;     // 9 rows: n_det up to 6257 pixels

size_t single_shot_eq3_smem(const ei_geometry *g)
{
    return (size_t)9 * g->dg.max_ndp * sizeof(float);
}

cudaError_t launch_single_shot_eq3(const ei_geometry *g, const float *meas, int m_index,
                                   float gamma, float *ker, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    k_eq3_kernel<<<g->n_slices, 256, 0, st>>>(g->dg, m_index, gamma, ker);
    EI_CUDA_TRY(cudaGetLastError());
    k_single_shot_eq3<<<g->dg.total_ic, 256, single_shot_eq3_smem(g), st>>>(
        g->dg, meas, m_index, gamma, ker, g->gA, g->gB);
    return cudaGetLastError();
}

static const int kSingleShotThreads = 256;

size_t single_shot_smem(const ei_geometry *g)
{
    return (size_t)(7 * g->dg.max_ndp + 2 * kSingleShotThreads) * sizeof(float);
}

cudaError_t single_shot_set_smem_limit()
{
    const int bytes = (7 * EI_MAX_NDET + 2 * kSingleShotThreads) * (int)sizeof(float);
    EI_CUDA_TRY(cudaFuncSetAttribute(k_single_shot, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes));
    return cudaFuncSetAttribute(k_single_shot_eq3, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                kEq3SmemLimit);
}

bool single_shot_eq3_fits(const ei_geometry *g)
{
    return single_shot_eq3_smem(g) <= (size_t)kEq3SmemLimit;
}

cudaError_t launch_single_shot(const ei_geometry *g, const float *meas, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    k_single_shot<<<g->dg.total_ic, kSingleShotThreads, single_shot_smem(g), st>>>(g->dg, meas,
                                                                                  g->gA, g->gB);
    return cudaGetLastError();
}

}  // namespace ei
