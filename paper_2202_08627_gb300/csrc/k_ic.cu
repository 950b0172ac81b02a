// Illumination-curve (IC) model, residual and per-pixel gradient, fused
// (Eq. 2 with the Eq. 4 offsets, the cost of Eq. 5 and its analytic gradient).
//
// Work unit: one sinogram row (slice, angle); variant 0 runs one block per
// row, variant 1 (below) persistent blocks that stream rows through shared
// memory with bulk asynchronous copies.  Per pixel t of the row:
//   shift = (z/period) D R[delta] + m_o(theta) + m_r(t)      (D: finite difference)
//   V     = w^2 + kappa R[sigma]
//   s_m   = A (w / sqrt(V)) exp(-R[mu] - (m - c - shift)^2 / (2 V))   for every m
//   e_m   = s_m - s_exp_m ;  objective partial sum_m e_m^2 (FP32 within a warp,
//           FP64 across the warps of a row)
//   G_mu  = -sum 2 e s,  G_sh = sum 2 e s q / V,  G_V = sum 2 e s (q^2 - V) / (2 V^2)
// and the gradient sinogram row
//   g = (G_mu, (z/period) D^T G_sh, kappa G_V),
// written pair-packed (the adjoint's input layout, see ei_internal.h).
// D needs R[delta] at t +- 1 and D^T needs G_sh at t +- 1, so the whole row
// is staged in shared memory (no halo recompute, no atomics).
//
// With a sampled flat IC (ei_set_flat_table) variant 0 runs with the Gaussian
// replaced by f(t, m - shift), f interpolated in m by periodic Catmull-Rom
// splines of the pixel's K samples over one period:
//   s_m = exp(-R[mu]) f(m - shift),  ds_m/dshift = -exp(-R[mu]) f'(m - shift)
// and R[sigma] has no effect (its gradient is 0).
//
// Memory traffic per pixel (M = n_m): 12 B of projections + 4M B of s_exp
// read, 24 B of packed g written; the per-pixel flat IC table is shared by all angles
// and stays in L2.  The kernel is HBM-bound.
#include "async_copy.h"
#include "ei_internal.h"

namespace ei {

// Row objective: each warp sums its lanes' FP32 partials (a fixed shuffle
// tree over at most a few hundred squared residuals), and the warp sums are
// added in FP64 by warp 0.  FP64 arithmetic runs at a small fraction of the
// FP32 rate on this GPU, so it is kept to one add per warp and level rather
// than one per lane.
__device__ __forceinline__ double block_sum_rows(float v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = (double)v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        t = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;   // valid in thread 0
}

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

// Periodic Catmull-Rom interpolation of one pixel's K samples p_k = f(k / K)
// at x (in periods): with u = x K = i + r (0 <= r < 1) the cubic Hermite
// segment between p_i and p_{i+1} whose end slopes are the central
// differences (p_{i+1} - p_{i-1}) / 2 and (p_{i+2} - p_i) / 2; indices mod K.
// f and df = df/dx.  Every index stays in [0, K) for any x, NaN included.
__device__ __forceinline__ void flat_table_eval(const float *__restrict__ tab, int K, float x,
                                                float &f, float &df)
{
    const float u = x * (float)K;
    const float fl = floorf(u);
    const float r = u - fl;
    int i = (int)fl % K;                     // cvt saturates (NaN -> 0): i in (-K, K)
    if (i < 0) i += K;
    const int im = i == 0 ? K - 1 : i - 1;
    const int i1 = i + 1 == K ? 0 : i + 1;
    const int i2 = i1 + 1 == K ? 0 : i1 + 1;
    const float p0 = __ldg(tab + im), p1 = __ldg(tab + i), p2 = __ldg(tab + i1), p3 = __ldg(tab + i2);
    const float m1 = 0.5f * (p2 - p0), m2 = 0.5f * (p3 - p1), d = p2 - p1;
    // Hermite form: f = p1 + r (m1 + r (3d - 2 m1 - m2 + r (m1 + m2 - 2d)))
    const float c2 = 3.f * d - 2.f * m1 - m2, c3 = m1 + m2 - 2.f * d;
    f = fmaf(r, fmaf(r, fmaf(r, c3, c2), m1), p1);
    df = (float)K * fmaf(r, fmaf(r, 3.f * c3, 2.f * c2), m1);
}

template <int MODE, bool TABLE>
__global__ void k_ic(DevGeom dg, const float *__restrict__ proj, const float *__restrict__ meas,
                     float *__restrict__ s_mod, float4 *__restrict__ gA, float2 *__restrict__ gB,
                     double *__restrict__ part, const int *__restrict__ active, float link)
{
    extern __shared__ float4 sm4[];
    __shared__ double red[32];
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const int nd = si.n_det, ndp = si.n_dp, ng = ndp >> 2;
    const int64_t plane = (int64_t)si.n_theta * ndp;
    const int64_t rbase = (int64_t)a * ndp;
    // every row starts on a 16-byte boundary (n_dp is a multiple of 4)
    const float4 *Pmu = reinterpret_cast<const float4 *>(proj + si.proj_off + rbase);
    const float4 *Pde = reinterpret_cast<const float4 *>(proj + si.proj_off + plane + rbase);
    const float4 *Psg = reinterpret_cast<const float4 *>(proj + si.proj_off + 2 * plane + rbase);
    const int64_t plane4 = plane >> 2;
    const float4 *pix = dg.pix + si.pix_off;
    const float mo = dg.m_o[si.ang_off + a];
    const int n_m = dg.mc.n_m;
    const float zp = dg.mc.z_over_p, kappa = dg.mc.kappa;

    const int mq = dg.max_ndp >> 2;
    float4 *s_pd4 = sm4;               // R[delta] of the row, later g_delta
    float4 *s_gsh4 = sm4 + mq;         // G_shift, G_mu, G_V of the row
    float4 *s_gmu4 = s_gsh4 + mq;
    float4 *s_gv4 = s_gmu4 + mq;
    const float *s_pd = reinterpret_cast<const float *>(s_pd4);
    const float *s_gsh = reinterpret_cast<const float *>(s_gsh4);

    for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) s_pd4[gi] = __ldg(Pde + gi);
    __syncthreads();

    float e2 = 0.f;
    bool out_of_domain = false;
    for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
        const float4 pm4 = __ldg(Pmu + gi), ps4 = __ldg(Psg + gi);
        const float pmv[4] = {pm4.x, pm4.y, pm4.z, pm4.w};
        const float psv[4] = {ps4.x, ps4.y, ps4.z, ps4.w};
        float c[4], shift[4], iV[4], amp[4];
        const float *tab[4];
        bool ok[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * gi + q;
            ok[q] = j < nd;
            const float4 fl = ok[q] ? __ldg(pix + j) : make_float4(0.f, 0.f, 1.f, 0.f);  // A, c, w, m_r
            c[q] = fl.y;
            shift[q] = ok[q] ? zp * deriv_at(s_pd, j, nd, si.inv_pitch) + mo + fl.w : 0.f;
            if (TABLE) {
                // amp = transmission; the padding pixels read the slice's first row
                tab[q] = dg.flat_tab + (int64_t)(si.det_off + (ok[q] ? j : 0)) * dg.flat_k;
                iV[q] = 1.f;
                amp[q] = ok[q] ? expf(-pmv[q]) : 0.f;
            } else {
                const float V = fmaf(kappa, psv[q], fl.z * fl.z);
                if (ok[q] && !(V > 0.01f * fl.z * fl.z)) out_of_domain = true;
                const float Vs = fmaxf(V, 1e-30f);
                iV[q] = 1.0f / Vs;
                amp[q] = ok[q] ? fl.x * fl.z * rsqrtf(Vs) : 0.f;
            }
        }
        float st[4] = {0.f, 0.f, 0.f, 0.f}, stq[4] = {0.f, 0.f, 0.f, 0.f},
              stq2[4] = {0.f, 0.f, 0.f, 0.f};
        float e2f = 0.f;
#pragma unroll 4
        for (int k = 0; k < n_m; ++k) {
            const float mk = dg.mc.m[k];
            float sv[4], qd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                if (TABLE) {
                    // qd = ds/dshift = -T f' (the Gaussian's s q / V with V = 1)
                    float f, df;
                    flat_table_eval(tab[q], dg.flat_k, mk - shift[q], f, df);
                    sv[q] = amp[q] * f;
                    qd[q] = -amp[q] * df;
                } else {
                    qd[q] = mk - c[q] - shift[q];
                    sv[q] = amp[q] * expf(-pmv[q] - 0.5f * qd[q] * qd[q] * iV[q]);
                }
            }
            if (MODE == IC_MODEL) {
                reinterpret_cast<float4 *>(s_mod + si.meas_off + rbase)[k * plane4 + gi] =
                    make_float4(sv[0], sv[1], sv[2], sv[3]);
            } else {
                const float4 x4 = __ldcs(reinterpret_cast<const float4 *>(meas + si.meas_off + rbase) +
                                         k * plane4 + gi);
                const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float e = ok[q] ? sv[q] - xv[q] : 0.f;
                    e2f = fmaf(e, e, e2f);
                    if (MODE == IC_OBJECTIVE_GRAD) {
                        const float t = 2.f * e * sv[q];
                        st[q] += t;
                        if (TABLE) {
                            stq[q] = fmaf(2.f * e, qd[q], stq[q]);
                        } else {
                            stq[q] = fmaf(t, qd[q], stq[q]);
                            stq2[q] = fmaf(t * qd[q], qd[q], stq2[q]);
                        }
                    }
                }
            }
        }
        if (MODE != IC_MODEL) e2 += e2f;
        if (MODE == IC_OBJECTIVE_GRAD) {
            float gsh[4], gvv[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                gsh[q] = stq[q] * iV[q];
                gvv[q] = TABLE ? 0.f : kappa * 0.5f * iV[q] * (stq2[q] * iV[q] - st[q]);
            }
            s_gsh4[gi] = make_float4(gsh[0], gsh[1], gsh[2], gsh[3]);
            s_gmu4[gi] = make_float4(-st[0], -st[1], -st[2], -st[3]);
            s_gv4[gi] = make_float4(gvv[0], gvv[1], gvv[2], gvv[3]);
        }
    }
    if (MODE == IC_MODEL) return;
    if (MODE == IC_OBJECTIVE_GRAD) {
        // g_delta = (z/period) D^T G_shift into the R[delta] row (no longer needed); then
        // the packed row: the entry of pixel j holds g(j) and g(j + 1)
        __syncthreads();
        for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
            float gd[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int j = 4 * gi + q;
                gd[q] = j < nd ? zp * deriv_T_at(s_gsh, j, nd, si.inv_pitch) : 0.f;
            }
            s_pd4[gi] = make_float4(gd[0], gd[1], gd[2], gd[3]);
        }
        __syncthreads();
        const float *gmu = reinterpret_cast<const float *>(s_gmu4);
        const float *gdl = reinterpret_cast<const float *>(s_pd4);
        const float *gsg = reinterpret_cast<const float *>(s_gv4);
        const int64_t dst = si.gp_off + (int64_t)a * si.gw + si.marg;
        if (dg.gmirror) {
            // mirror-interleaved row: entry j holds pixel j and pixel nd - 1 - j
            // (zero outside [0, nd)); linked: g_mu + gamma g_delta only
            for (int j = (int)threadIdx.x - 1; j < ndp; j += blockDim.x) {
                const bool in = j >= 0 && j < nd;
                const int jm = nd - 1 - j;
                if (link > 0.f) {
                    gB[dst + j] = in ? make_float2(fmaf(link, gdl[j], gmu[j]),
                                                   fmaf(link, gdl[jm], gmu[jm]))
                                     : make_float2(0.f, 0.f);
                } else {
                    gA[dst + j] = in ? make_float4(gmu[j], gmu[jm], gdl[j], gdl[jm])
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
                    gB[dst + j] = in ? make_float2(gsg[j], gsg[jm]) : make_float2(0.f, 0.f);
                }
            }
        } else if (link > 0.f) {
            // linked unknown (Eq. 4): the single sinogram g_mu + gamma g_delta,
            // pair-packed in gB, is all the adjoint needs
            for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * gi + q;
                    const bool nx = j + 1 < ndp;
                    gB[dst + j] = make_float2(fmaf(link, gdl[j], gmu[j]),
                                              nx ? fmaf(link, gdl[j + 1], gmu[j + 1]) : 0.f);
                }
            }
            if (threadIdx.x == 0) gB[dst - 1] = make_float2(0.f, fmaf(link, gdl[0], gmu[0]));
        } else {
            for (int gi = threadIdx.x; gi < ng; gi += blockDim.x) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int j = 4 * gi + q;
                    const bool nx = j + 1 < ndp;
                    gA[dst + j] = make_float4(gmu[j], gdl[j], gsg[j], nx ? gmu[j + 1] : 0.f);
                    gB[dst + j] = make_float2(nx ? gdl[j + 1] : 0.f, nx ? gsg[j + 1] : 0.f);
                }
            }
            if (threadIdx.x == 0) {                 // entry of pixel -1: (0, g(0))
                gA[dst - 1] = make_float4(0.f, 0.f, 0.f, gmu[0]);
                gB[dst - 1] = make_float2(gdl[0], gsg[0]);
            }
        }
    }
    const int bad = __syncthreads_or(out_of_domain ? 1 : 0);
    const double tot = block_sum_rows(e2, red);
    if (threadIdx.x == 0) part[row] = bad ? __longlong_as_double(0x7ff0000000000000LL) : tot;
}

// ---------------------------------------------------------------------------
// Variant 1: persistent blocks, rows staged by bulk asynchronous copies.
//
// Each block walks the rows blockIdx.x, blockIdx.x + gridDim.x, ... and keeps
// NST (3, else 2) row buffers in shared memory: while it computes row r, the
// bulk copies of its next NST - 1 rows (three projection rows and M measured
// rows, one copy each) are in flight, so every SM keeps up to ~120 KB of reads
// outstanding independently of its register budget.  One thread issues the
// copies and publishes each row's slice constants in shared memory from a
// warp of its own, so its latency stays off the consumers' path.  Two
// pixels per consumer thread; two block barriers per row (before D^T, which reads
// neighbours' G_shift, and the objective reduction, which also releases the
// row's buffer).  Per pixel the arithmetic is variant 0's, arranged to issue
// fewer instructions: 1/V as rsqrt(V)^2, the exponential as 2^(log2(e) x) by
// the PTX ex2 instruction on a pre-scaled argument, D and D^T without
// branches (D^T from G_shift pre-weighted by its row of D), padding pixels'
// measured values zeroed once per row, the factor 2 of the residual applied
// once per pixel.  Results agree with variant 0 to FP32 rounding.
// ---------------------------------------------------------------------------
constexpr float kLog2e = 1.4426950408889634f;
constexpr uint64_t kIcWaitNs = 2000000000ull;     // 2 s bound on one row's copies
constexpr int kIcPipeMaxStages = 3;

// A row's constants, written by the issuing thread next to its buffer.
struct IcRow {
    int row;                 // -1: the block has no further row
    int a, nd, ndp;
    int pix_off, pad_;
    float inv_pitch, mo;
    int64_t meas_off, gp_off, plane;
};

__device__ __forceinline__ int ic_next_row(const DevGeom &dg, const int *active, int r, int step)
{
    if (active)
        while (r < dg.total_ic && !__ldg(active + find_slice(dg.ic_prefix, dg.n_slices, r))) r += step;
    return r;
}

// The producer's walk over its block's rows r0, r0 + step, ...: rows only
// increase, so the owning slice is tracked incrementally (a load per slice
// boundary instead of a binary search per row).
struct IcRowWalker {
    int r, s, s_end, step;

    __device__ void start(const DevGeom &dg, const int *active, int r0, int stride)
    {
        r = r0, step = stride, s = 0, s_end = __ldg(dg.ic_prefix + 1);
        skip_inactive(dg, active);
    }
    // advance s to the slice owning r (r < total_ic)
    __device__ void seek(const DevGeom &dg)
    {
        while (r >= s_end) {
            ++s;
            s_end = __ldg(dg.ic_prefix + s + 1);
        }
    }
    // move r to the first row >= r (same residue) of an active slice
    __device__ void skip_inactive(const DevGeom &dg, const int *active)
    {
        while (r < dg.total_ic) {
            seek(dg);
            if (!active || __ldg(active + s)) return;
            r += (s_end - r + step - 1) / step * step;
        }
    }
    __device__ void next(const DevGeom &dg, const int *active)
    {
        r += step;
        skip_inactive(dg, active);
    }
};

// Producer: publish row w.r's constants in *meta (row = -1 when past the end)
// and, for a real row, arm `bar` and issue the copies of the row into the
// buffer `stage` (slots of mx floats: P_mu, P_delta, P_sigma, then the M
// measured rows).
__device__ __forceinline__ void ic_issue_row(const DevGeom &dg, const IcRowWalker &w,
                                             const float *proj, const float *meas, float *stage,
                                             int mx, int n_in, unsigned bar, IcRow *meta)
{
    const int r = w.r;
    if (r >= dg.total_ic) {
        meta->row = -1;
        return;
    }
    const int s = w.s;
    const SliceInfo &si = dg.slices[s];
    const int a = r - dg.ic_prefix[s];
    IcRow m;
    m.row = r, m.a = a, m.nd = si.n_det, m.ndp = si.n_dp;
    m.pix_off = si.pix_off, m.pad_ = 0;
    m.inv_pitch = si.inv_pitch, m.mo = dg.m_o[si.ang_off + a];
    m.meas_off = si.meas_off + (int64_t)a * si.n_dp;                 // row start, plane m = 0
    m.gp_off = si.gp_off + (int64_t)a * si.gw + si.marg;             // entry of pixel 0
    const int64_t plane = (int64_t)si.n_theta * si.n_dp;
    m.plane = plane;
    *meta = m;
    const unsigned bytes = (unsigned)si.n_dp * 4u;
    const int64_t rbase = (int64_t)a * si.n_dp;
    mbar_arrive_expect_tx(bar, bytes * (unsigned)n_in);
    for (int c = 0; c < 3; ++c)
        bulk_copy_g2s(stage + c * mx, proj + si.proj_off + c * plane + rbase, bytes, bar);
    for (int k = 0; k < n_in - 3; ++k)
        bulk_copy_g2s(stage + (3 + k) * mx, meas + si.meas_off + k * plane + rbase, bytes, bar);
}

template <int MODE, int NM>
__global__ void __launch_bounds__(1024)
k_ic_pipe(DevGeom dg, const float *__restrict__ proj, const float *__restrict__ meas,
          float *__restrict__ s_mod, float4 *__restrict__ gA, float2 *__restrict__ gB,
          double *__restrict__ part, const int *__restrict__ active, int *__restrict__ status,
          int nst, float link)
{
    extern __shared__ float4 sm4[];
    __shared__ uint64_t bars[kIcPipeMaxStages];
    __shared__ IcRow metas[kIcPipeMaxStages];
    __shared__ double red[2][32];        // alternate rows: no barrier between one
                                         // row's final read and the next row's writes
    // a row that never landed, per iteration parity: set before the row's
    // barrier, read after it, so every thread takes the same decision
    __shared__ int s_abort[2];
    const int mx = dg.max_ndp;
    const int n_m = NM > 0 ? NM : dg.mc.n_m;     // NM > 0: M known at compile time
    const int n_in = MODE == IC_MODEL ? 3 : 3 + n_m;
    float *const bufs = reinterpret_cast<float *>(sm4);           // nst buffers of n_in * mx
    // per row parity b: G_shift weighted by its row of D (one zero entry in
    // front, two behind), G_mu, G_V; two sets, so that a row's packing loop and
    // the next row's computation do not share them
    float *const gbase = bufs + nst * n_in * mx;
    const int gspan = 3 * mx + 8;
    const int step = gridDim.x;
    const float zp = dg.mc.z_over_p, kappa = dg.mc.kappa;
    // the last warp produces (its lane 0 issues the copies and runs ahead over
    // the rows); the others consume, two pixels per thread
    const int n_cons = (int)blockDim.x - 32;
    const bool producer = threadIdx.x == (unsigned)n_cons;
    IcRowWalker walk;
    unsigned issued = 0;                 // iterations whose row the producer has published
    if (producer) {
        for (int i = 0; i < nst; ++i) mbar_init(smem_addr(&bars[i]), 1);
        mbar_init_fence();
        s_abort[0] = s_abort[1] = 0;
        gbase[3] = 0.f;                            // g_sw[-1] of both sets
        gbase[gspan + 3] = 0.f;
        walk.start(dg, active, blockIdx.x, step);
        while (issued < (unsigned)nst - 1) {
            ic_issue_row(dg, walk, proj, meas, bufs + issued * n_in * mx, mx, n_in,
                         smem_addr(&bars[issued]), &metas[issued]);
            if (walk.r < dg.total_ic) walk.next(dg, active);
            ++issued;
        }
    }
    __syncthreads();
    int prev_row = -1;                   // gradient mode: the row whose objective is pending
    unsigned prev_it = 0;                // and its iteration (the parity of its warp sums)
    for (unsigned it = 0;; ++it) {
        const unsigned slot = it % nst;
        const IcRow m = metas[slot];
        if (m.row < 0) break;
        float *const stg = bufs + slot * n_in * mx;
        float *const g_sw = gbase + (it & 1u) * gspan + 4;
        float *const g_mu = g_sw + mx + 4;
        float *const g_v = g_mu + mx;
        // the buffer of iteration it - 1 was released by that row's last barrier
        if (producer) {
            const unsigned sl = issued % nst;
            ic_issue_row(dg, walk, proj, meas, bufs + sl * n_in * mx, mx, n_in,
                         smem_addr(&bars[sl]), &metas[sl]);
            if (walk.r < dg.total_ic) walk.next(dg, active);
            ++issued;
        }
        const bool landed = mbar_wait_bounded(smem_addr(&bars[slot]), (it / nst) & 1u, kIcWaitNs);
        if (!landed) s_abort[it & 1u] = 1;   // finish the row on whatever is there; reported below

        const int nd = m.nd, ndp = m.ndp, nh = ndp >> 1;
        const float *Pd = stg + mx;
        const float2 *Pm2 = reinterpret_cast<const float2 *>(stg);
        const float2 *Ps2 = reinterpret_cast<const float2 *>(stg + 2 * mx);
        const float4 *pix = dg.pix + m.pix_off;
        const float h_in = zp * m.inv_pitch;                 // (z/period) / pitch
        float e2 = landed ? 0.f : __int_as_float(0x7fc00000);     // NaN if the row never landed
        for (int h = threadIdx.x; h < nh && (int)threadIdx.x < n_cons; h += n_cons) {
            const float2 pm = Pm2[h], ps = Ps2[h];
            const float pmv[2] = {pm.x, pm.y}, psv[2] = {ps.x, ps.y};
            float cs[2], r2[2], amp[2], a2[2], b2[2];
            float e2f = 0.f;
            if (MODE != IC_MODEL && 2 * h + 1 >= nd) {
                // padding pixels of this pair: their measured values count as 0
                for (int q = 0; q < 2; ++q)
                    if (2 * h + q >= nd)
                        for (int k = 0; k < n_m; ++k) stg[(3 + k) * mx + 2 * h + q] = 0.f;
                proxy_fence_async();             // ordered before the buffer's next bulk copy
            }
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const int j = 2 * h + q;
                const bool ok = j < nd;
                const float4 fl = ok ? __ldg(pix + j) : make_float4(0.f, 0.f, 1.f, 0.f);  // A, c, w, m_r
                // D R[delta]: central difference, one-sided at the row ends
                const int jl = max(j - 1, 0), jr = min(j + 1, nd - 1);
                const float dd = (Pd[jr] - Pd[jl]) * (jr - jl == 2 ? 0.5f : 1.0f);
                cs[q] = fl.y + (ok ? fmaf(h_in, dd, m.mo + fl.w) : 0.f);
                const float V = fmaf(kappa, psv[q], fl.z * fl.z);
                if (ok && !(V > 0.01f * fl.z * fl.z)) e2f = __int_as_float(0x7f800000);
                const float rs = rsqrtf(fmaxf(V, 1e-30f));
                r2[q] = rs * rs;                                  // 1 / V
                amp[q] = ok ? fl.x * fl.z * rs : 0.f;
                a2[q] = -kLog2e * pmv[q];
                b2[q] = (0.5f * kLog2e) * r2[q];
            }
            float st[2] = {0.f, 0.f}, stq[2] = {0.f, 0.f}, stq2[2] = {0.f, 0.f};
#pragma unroll(NM > 0 ? NM : 4)
            for (int k = 0; k < n_m; ++k) {
                const float mk = dg.mc.m[k];
                float sv[2], qd[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    qd[q] = mk - cs[q];
                    sv[q] = amp[q] * ex2_approx(fmaf(-b2[q], qd[q] * qd[q], a2[q]));
                }
                if (MODE == IC_MODEL) {
                    reinterpret_cast<float2 *>(s_mod + m.meas_off + k * m.plane)[h] =
                        make_float2(sv[0], sv[1]);
                } else {
                    const float2 x2 = reinterpret_cast<const float2 *>(stg + (3 + k) * mx)[h];
                    const float xv[2] = {x2.x, x2.y};
#pragma unroll
                    for (int q = 0; q < 2; ++q) {
                        const float e = sv[q] - xv[q];
                        e2f = fmaf(e, e, e2f);
                        if (MODE == IC_OBJECTIVE_GRAD) {
                            const float t = e * sv[q];          // half of d(e^2)/d(s)
                            const float tq = t * qd[q];
                            st[q] += t;
                            stq[q] += tq;
                            stq2[q] = fmaf(tq, qd[q], stq2[q]);
                        }
                    }
                }
            }
            if (MODE != IC_MODEL) e2 += e2f;
            if (MODE == IC_OBJECTIVE_GRAD) {
                float gsw[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int j = 2 * h + q;
                    // weight of G_shift(j) in its row of D: 1/pitch at the ends, 1/(2 pitch) inside
                    const float wd = nd == 1 || j >= nd ? 0.f : (j == 0 || j == nd - 1 ? 2.f : 1.f);
                    gsw[q] = wd * (2.f * stq[q] * r2[q]);    // row weight x 2 pitch x G_shift
                }
                reinterpret_cast<float2 *>(g_sw)[h] = make_float2(gsw[0], gsw[1]);
                reinterpret_cast<float2 *>(g_mu)[h] = make_float2(-2.f * st[0], -2.f * st[1]);
                reinterpret_cast<float2 *>(g_v)[h] =
                    make_float2(kappa * r2[0] * (stq2[0] * r2[0] - st[0]),
                                kappa * r2[1] * (stq2[1] * r2[1] - st[1]));
            }
        }
        if (MODE == IC_OBJECTIVE_GRAD) {
            if (threadIdx.x == 0) g_sw[ndp] = g_sw[ndp + 1] = 0.f;   // D^T reads past the row
            // every G_shift of the row is in place; every read of the row's staged
            // inputs is done (its buffer may be refilled); the previous row's warp
            // sums are written
            __syncthreads();
            if (prev_row >= 0 && threadIdx.x < 32) {
                double t = (int)threadIdx.x < ((int)blockDim.x >> 5) ? red[prev_it & 1u][threadIdx.x] : 0.0;
                for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
                if (threadIdx.x == 0) part[prev_row] = t;
            }
            if (s_abort[it & 1u]) {
                // the row never arrived: report it, poison this block's remaining
                // rows, and give the copies still in flight a bounded chance to land
                // before the block's shared memory is released
                if (producer) {
                    atomicExch(status, (int)EI_ERR_TIMEOUT);
                    for (int q = m.row; q < dg.total_ic; q = ic_next_row(dg, active, q + step, step))
                        part[q] = __longlong_as_double(0x7ff8000000000000LL);
                    for (unsigned i = it; i < issued; ++i)
                        if (metas[i % nst].row >= 0)
                            mbar_wait_bounded(smem_addr(&bars[i % nst]), (i / nst) & 1u, kIcWaitNs);
                }
                return;
            }
            // packed row: the entry of pixel j holds g(j) and g(j + 1), with
            // g_delta(j) = (z/period) (D^T G_shift)(j)
            //            = (z/period)/(2 pitch) (gsw(j-1) - gsw(j+1) + e(j) gsw(j)),
            // e(j) = +1 at j = nd - 1, -1 at j = 0 (gsw(-1) = gsw(nd) = 0)
            const float kdt = 0.5f * h_in;
            if (dg.gmirror) {
                // mirror-interleaved row: entry j holds pixel j and pixel nd - 1 - j
                // (zero outside [0, nd)), each value as the pair-packed row has it
                auto gdelta = [&](int i) {
                    const float ei = (i == nd - 1 ? 1.f : 0.f) - (i == 0 ? 1.f : 0.f);
                    return kdt * fmaf(ei, g_sw[i], g_sw[i - 1] - g_sw[i + 1]);
                };
                for (int j = (int)threadIdx.x - 1; j < ndp && (int)threadIdx.x < n_cons; j += n_cons) {
                    const bool in = j >= 0 && j < nd;
                    const int jm = in ? nd - 1 - j : 0;
                    const int jj = in ? j : 0;
                    const float dj = gdelta(jj), dm = gdelta(jm);
                    if (link > 0.f) {
                        gB[m.gp_off + j] = in ? make_float2(fmaf(link, dj, g_mu[jj]),
                                                            fmaf(link, dm, g_mu[jm]))
                                              : make_float2(0.f, 0.f);
                    } else {
                        gA[m.gp_off + j] = in ? make_float4(g_mu[jj], g_mu[jm], dj, dm)
                                              : make_float4(0.f, 0.f, 0.f, 0.f);
                        gB[m.gp_off + j] = in ? make_float2(g_v[jj], g_v[jm]) : make_float2(0.f, 0.f);
                    }
                }
            }
            for (int j = (int)threadIdx.x - 1; j < ndp && (int)threadIdx.x < n_cons && !dg.gmirror;
                 j += n_cons) {
                const float gm1 = g_sw[j - 1], g0 = g_sw[j], g1 = g_sw[j + 1], g2 = g_sw[j + 2];
                const float e0 = (j == nd - 1 ? 1.f : 0.f) - (j == 0 ? 1.f : 0.f);
                const float e1 = (j + 1 == nd - 1 ? 1.f : 0.f) - (j + 1 == 0 ? 1.f : 0.f);
                const float d0 = j >= 0 && j < nd ? kdt * fmaf(e0, g0, gm1 - g1) : 0.f;
                const float d1 = j + 1 < nd ? kdt * fmaf(e1, g1, g0 - g2) : 0.f;
                const bool cur = j >= 0, nx = j + 1 < ndp;
                if (link > 0.f) {        // linked unknown: g_mu + gamma g_delta only
                    gB[m.gp_off + j] = make_float2(fmaf(link, d0, cur ? g_mu[j] : 0.f),
                                                   fmaf(link, d1, nx ? g_mu[j + 1] : 0.f));
                } else {
                    gA[m.gp_off + j] = make_float4(cur ? g_mu[j] : 0.f, d0, cur ? g_v[j] : 0.f,
                                                   nx ? g_mu[j + 1] : 0.f);
                    gB[m.gp_off + j] = make_float2(d1, nx ? g_v[j + 1] : 0.f);
                }
            }
        }
        if (MODE == IC_OBJECTIVE_GRAD) {
            // this row's warp sums; warp 0 adds them after the next row's barrier
            float v = e2;
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if ((threadIdx.x & 31) == 0) red[it & 1u][threadIdx.x >> 5] = (double)v;
            prev_row = m.row;
            prev_it = it;
            continue;
        }
        if (MODE != IC_MODEL) {
            const double tot = block_sum_rows(e2, red[it & 1u]);    // its barrier releases the row
            if (threadIdx.x == 0) part[m.row] = tot;
        } else {
            __syncthreads();
        }
        if (s_abort[it & 1u]) {
            // a row never arrived: report it, poison this block's remaining rows,
            // and give the copies still in flight a bounded chance to land before
            // the block's shared memory is released
            if (producer) {
                atomicExch(status, (int)EI_ERR_TIMEOUT);
                if (MODE != IC_MODEL)
                    for (int q = m.row; q < dg.total_ic; q = ic_next_row(dg, active, q + step, step))
                        part[q] = __longlong_as_double(0x7ff8000000000000LL);
                for (unsigned i = it; i < issued; ++i)
                    if (metas[i % nst].row >= 0)
                        mbar_wait_bounded(smem_addr(&bars[i % nst]), (i / nst) & 1u, kIcWaitNs);
            }
            return;
        }
    }
    if (MODE == IC_OBJECTIVE_GRAD) {
        __syncthreads();                           // the last row's warp sums are written
        if (prev_row >= 0 && threadIdx.x < 32) {
            double t = (int)threadIdx.x < ((int)blockDim.x >> 5) ? red[prev_it & 1u][threadIdx.x] : 0.0;
            for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
            if (threadIdx.x == 0) part[prev_row] = t;
        }
    }
}

static const int kIcPipeSmemLimit = 220 * 1024;

// Threads for the row kernels: one per 4 (variant 0) or 2 (variant 1) pixels
// of the widest row, capped (threads then loop over the row).
static int ic_threads(const ei_geometry *g, int px, int cap)
{
    const int threads = (g->dg.max_ndp / px + 31) / 32 * 32;
    return threads > cap ? cap : threads;
}

static size_t ic_pipe_smem_stages(int max_ndp, int n_m, IcMode mode, int nst)
{
    const int n_in = mode == IC_MODEL ? 3 : 3 + n_m;
    return ((size_t)(nst * n_in + 6) * max_ndp + 16) * sizeof(float);   // + two gradient sets
}

// Row buffers of the bulk-copy variant: 3 when they fit, else 2, else 0.
static int ic_pipe_stages(int max_ndp, int n_m)
{
    for (int nst = kIcPipeMaxStages; nst >= 2; --nst)
        if (ic_pipe_smem_stages(max_ndp, n_m, IC_OBJECTIVE_GRAD, nst) <= (size_t)kIcPipeSmemLimit)
            return nst;
    return 0;
}

bool ic_pipe_fits(int max_ndp, int n_m) { return ic_pipe_stages(max_ndp, n_m) > 0; }

template <int MODE, int NM>
static cudaError_t launch_ic_pipe_nm(const ei_geometry *g, const float *proj, const float *meas,
                                     float *s_mod, double *part, const int *active, float link,
                                     cudaStream_t st)
{
    const int threads = ic_threads(g, 2, 1024 - 32) + 32;      // consumers + one producer warp
    const int nst = ic_pipe_stages(g->dg.max_ndp, g->dg.mc.n_m);
    const size_t smem = ic_pipe_smem_stages(g->dg.max_ndp, g->dg.mc.n_m, (IcMode)MODE, nst);
    int per_sm = 0;
    EI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ic_pipe<MODE, NM>, threads, smem));
    const int grid = std::max(1, std::min(g->dg.total_ic, std::max(1, per_sm) * g->num_sms));
    k_ic_pipe<MODE, NM><<<grid, threads, smem, st>>>(g->dg, proj, meas, s_mod, g->gA, g->gB, part,
                                                     active, g->dev_status, nst, link);
    return cudaGetLastError();
}

// M = 7 (the paper's scans) and M = 5 get fully unrolled loops over m.
template <int MODE>
static cudaError_t launch_ic_pipe(const ei_geometry *g, const float *proj, const float *meas,
                                  float *s_mod, double *part, const int *active, float link,
                                  cudaStream_t st)
{
    switch (g->dg.mc.n_m) {
    case 7: return launch_ic_pipe_nm<MODE, 7>(g, proj, meas, s_mod, part, active, link, st);
    case 5: return launch_ic_pipe_nm<MODE, 5>(g, proj, meas, s_mod, part, active, link, st);
    default: return launch_ic_pipe_nm<MODE, 0>(g, proj, meas, s_mod, part, active, link, st);
    }
}

template <int MODE>
static cudaError_t ic_pipe_set_smem_limit()
{
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic_pipe<MODE, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kIcPipeSmemLimit));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic_pipe<MODE, 5>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kIcPipeSmemLimit));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic_pipe<MODE, 7>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     kIcPipeSmemLimit));
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Gradient with respect to Eq. 4's drift m_o(theta) and ring term m_r(t).
// Both add to the shift of pixel (theta, t) with coefficient 1, so the
// gradients are sums of dS/dshift = sum_m 2 e s q / V over t (m_o) and over
// theta (m_r).  k_shift_grad: one block per row, dS/dshift of every pixel
// into `shift` (sino layout) and the row's FP64 sum into row_sum;
// k_offset_sums: one block per slice, FP64 sums over the slice's angles in
// angle order.  Deterministic; not on the solver's path.
// ---------------------------------------------------------------------------
template <bool TABLE>
__global__ void k_shift_grad(DevGeom dg, const float *__restrict__ proj,
                             const float *__restrict__ meas, float *__restrict__ shift,
                             double *__restrict__ row_sum, const int *__restrict__ active)
{
    extern __shared__ float s_pd[];                   // R[delta] of the row
    __shared__ double red[32];
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const int nd = si.n_det, ndp = si.n_dp;
    const int64_t plane = (int64_t)si.n_theta * ndp, rbase = (int64_t)a * ndp;
    const float *Pm = proj + si.proj_off + rbase;
    const float *Ps = Pm + 2 * plane;
    const float *Sx = meas + si.meas_off + rbase;
    for (int j = threadIdx.x; j < ndp; j += blockDim.x) s_pd[j] = Pm[plane + j];
    __syncthreads();
    const float4 *pix = dg.pix + si.pix_off;
    const float mo = dg.m_o[si.ang_off + a];
    const float zp = dg.mc.z_over_p, kappa = dg.mc.kappa;
    double acc = 0.0;
    for (int j = threadIdx.x; j < ndp; j += blockDim.x) {
        float g = 0.f;
        if (j < nd) {
            const float4 fl = __ldg(pix + j);           // A, c, w, m_r
            const float shift = zp * deriv_at(s_pd, j, nd, si.inv_pitch) + mo + fl.w;
            const float pm = Pm[j];
            if (TABLE) {                                // ds/dshift = -T f'(m - shift)
                const float *tab = dg.flat_tab + (int64_t)(si.det_off + j) * dg.flat_k;
                const float T = expf(-pm);
                float acc2 = 0.f;
                for (int k = 0; k < dg.mc.n_m; ++k) {
                    float f, df;
                    flat_table_eval(tab, dg.flat_k, dg.mc.m[k] - shift, f, df);
                    acc2 = fmaf(T * f - Sx[k * plane + j], -T * df, acc2);
                }
                g = 2.f * acc2;
            } else {
                const float cs = fl.y + shift;
                const float Vs = fmaxf(fmaf(kappa, Ps[j], fl.z * fl.z), 1e-30f);
                const float iV = 1.0f / Vs;
                const float amp = fl.x * fl.z * rsqrtf(Vs);
                float stq = 0.f;
                for (int k = 0; k < dg.mc.n_m; ++k) {
                    const float q = dg.mc.m[k] - cs;
                    const float sv = amp * expf(-pm - 0.5f * q * q * iV);
                    stq = fmaf((sv - Sx[k * plane + j]) * sv, q, stq);
                }
                g = 2.f * stq * iV;
            }
        }
        shift[si.sino_off + rbase + j] = g;
        acc += (double)g;
    }
    const double tot = block_sum_double(acc, red);
    if (threadIdx.x == 0) row_sum[row] = tot;
}

__global__ void k_offset_sums(DevGeom dg, const float *__restrict__ shift,
                              const double *__restrict__ row_sum, float *__restrict__ g_mo,
                              float *__restrict__ g_mr)
{
    const SliceInfo si = dg.slices[blockIdx.x];
    const int r0 = dg.ic_prefix[blockIdx.x];
    if (g_mo)
        for (int a = threadIdx.x; a < si.n_theta; a += blockDim.x)
            g_mo[si.ang_off + a] = (float)row_sum[r0 + a];
    if (g_mr)
        for (int j = threadIdx.x; j < si.n_det; j += blockDim.x) {
            double acc = 0.0;
            for (int a = 0; a < si.n_theta; ++a) acc += (double)shift[si.sino_off + (int64_t)a * si.n_dp + j];
            g_mr[si.det_off + j] = (float)acc;
        }
}

cudaError_t launch_offset_grads(const ei_geometry *g, const float *proj, const float *meas,
                                float *shift, double *row_sum, float *g_mo, float *g_mr,
                                cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    EI_CUDA_TRY(launch_shift_grad(g, proj, meas, shift, row_sum, nullptr, st));
    k_offset_sums<<<g->n_slices, 256, 0, st>>>(g->dg, shift, row_sum, g_mo, g_mr);
    return cudaGetLastError();
}

cudaError_t launch_shift_grad(const ei_geometry *g, const float *proj, const float *meas,
                              float *shift, double *row_sum, const int *active, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    const size_t smem = (size_t)g->dg.max_ndp * sizeof(float);
    if (g->dg.flat_tab)
        k_shift_grad<true><<<g->dg.total_ic, 256, smem, st>>>(g->dg, proj, meas, shift, row_sum, active);
    else
        k_shift_grad<false><<<g->dg.total_ic, 256, smem, st>>>(g->dg, proj, meas, shift, row_sum, active);
    return cudaGetLastError();
}

template <bool TABLE>
static void launch_ic_rows(const ei_geometry *g, const float *proj, const float *meas, float *s_mod,
                           double *part, IcMode mode, const int *active, float link,
                           cudaStream_t st)
{
    const int threads = ic_threads(g, 4, 512);
    const size_t smem = (size_t)4 * g->dg.max_ndp * sizeof(float);
    switch (mode) {
    case IC_MODEL:
        k_ic<IC_MODEL, TABLE><<<g->dg.total_ic, threads, smem, st>>>(g->dg, proj, meas, s_mod, g->gA,
                                                                      g->gB, part, active, link);
        break;
    case IC_OBJECTIVE:
        k_ic<IC_OBJECTIVE, TABLE><<<g->dg.total_ic, threads, smem, st>>>(
            g->dg, proj, meas, s_mod, g->gA, g->gB, part, active, link);
        break;
    default:
        k_ic<IC_OBJECTIVE_GRAD, TABLE><<<g->dg.total_ic, threads, smem, st>>>(
            g->dg, proj, meas, s_mod, g->gA, g->gB, part, active, link);
        break;
    }
}

cudaError_t launch_ic(const ei_geometry *g, const float *proj, const float *meas, float *s_mod,
                      double *part, IcMode mode, float link, const int *active, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    if (g->dg.flat_tab) {                        // the sampled flat runs one block per row
        launch_ic_rows<true>(g, proj, meas, s_mod, part, mode, active, link, st);
        return cudaGetLastError();
    }
    if (g->ic_variant == 1) {
        switch (mode) {
        case IC_MODEL: return launch_ic_pipe<IC_MODEL>(g, proj, meas, s_mod, part, active, link, st);
        case IC_OBJECTIVE:
            return launch_ic_pipe<IC_OBJECTIVE>(g, proj, meas, s_mod, part, active, link, st);
        default: return launch_ic_pipe<IC_OBJECTIVE_GRAD>(g, proj, meas, s_mod, part, active, link, st);
        }
    }
    launch_ic_rows<false>(g, proj, meas, s_mod, part, mode, active, link, st);
    return cudaGetLastError();
}

template <bool TABLE>
static cudaError_t ic_rows_set_smem_limit(int bytes)
{
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_MODEL, TABLE>, a, bytes));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_OBJECTIVE, TABLE>, a, bytes));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_ic<IC_OBJECTIVE_GRAD, TABLE>, a, bytes));
    return cudaSuccess;
}

cudaError_t ic_set_smem_limit()
{
    const int bytes = 4 * EI_MAX_NDET * (int)sizeof(float);
    EI_CUDA_TRY(ic_rows_set_smem_limit<false>(bytes));
    EI_CUDA_TRY(ic_rows_set_smem_limit<true>(bytes));
    EI_CUDA_TRY(ic_pipe_set_smem_limit<IC_MODEL>());
    EI_CUDA_TRY(ic_pipe_set_smem_limit<IC_OBJECTIVE>());
    EI_CUDA_TRY(ic_pipe_set_smem_limit<IC_OBJECTIVE_GRAD>());
    return cudaSuccess;
}

}  // namespace ei
