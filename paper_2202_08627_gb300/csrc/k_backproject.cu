// Adjoint R^T of the projector (the transpose the analytic gradient of Eq. 5
// needs), in gather form: every thread owns voxels and sums, over all angles,
// their two detector taps — no atomics and a fixed summation order, so the
// result is deterministic.
//
// Matrix entry (same matrix as the ray-driven projector):
//   R[(a, j), (r, c)] = (pitch / ch) * max(0, 1 - |u - j| / ch),
//   u = (c - hn) cos + (hn - r) sin + hd,   ch = max(|cos|, |sin|),
// so voxel (r, c) reads pixels floor(u) and floor(u) + 1 of every angle.
//
// Like the projector, this kernel is bound by the bytes loads bring from L1
// into registers.  Per voxel and angle it loads one pair-packed entry (both
// taps, 24 B) of the gradient sinogram; the rows carry zero margins wide
// enough for every voxel, so there are no bounds checks; each thread owns 8
// voxels so the per-angle constants (read from shared memory) are shared by 8
// voxel-angle updates; a warp covers an 8 x 4 voxel patch per pass so its
// lanes read a compact run of pixels.
//
// Accuracy: u reaches ~n_det, where an FP32 product would carry ~1e-4 pixel
// of rounding.  Per angle the block computes u at its tile origin in 32.32
// fixed point and splits it into an integer J and a fraction phi; each voxel
// adds only its small local offset dc cos - dr sin in FP32.
//
// Also fused: out = out_mult * R^T g + reg2 * v (the regulariser's gradient)
// and per-tile FP64 partial sums of sum_c reg1_c v_c^2 (its value); v may be
// null (no regulariser).
#include "ei_internal.h"

namespace ei {

constexpr int ADJ_PASSES = EI_ADJ_PASSES;   // 8 rows per pass (8 warps: 4 columns x 2 rows of 8x4)
constexpr int ADJ_CHUNK = 128;           // angles staged per shared-memory chunk

__device__ __forceinline__ double block_sum_double_adj(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(ADJ_THREADS, EI_ADJ_MINBLOCKS)
k_backproject(DevGeom dg, const float4 *__restrict__ gA, const float2 *__restrict__ gB,
              bool with_sino, const float4 *__restrict__ v, float4 *__restrict__ out,
              float4 out_mult, float4 reg2, float4 reg1, double *__restrict__ part,
              const int *__restrict__ active)
{
    __shared__ float4 s_cs[ADJ_CHUNK];   // cos, sin, pitch/(ch*ch), pitch/ch
    __shared__ float4 s_jp[ADJ_CHUNK];   // J (int bits), phi, pitch/ch - pitch/(ch*ch), -
    __shared__ double red[32];

    const int item = blockIdx.x;
    const int s = find_slice(dg.adj_prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int ntc = (n + ADJ_TC - 1) / ADJ_TC;
    const int local = item - dg.adj_prefix[s];
    const int r_t = (local / ntc) * ADJ_TR, c_t = (local % ntc) * ADJ_TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int dc = (warp & 3) * 8 + (lane & 7);        // column offset in the tile
    const int dr0 = (warp >> 2) * 4 + (lane >> 3);     // row offset of pass 0 (passes add 8)

    float acc[ADJ_PASSES][3];
#pragma unroll
    for (int p = 0; p < ADJ_PASSES; ++p) acc[p][0] = acc[p][1] = acc[p][2] = 0.f;

    if (with_sino) {
        const float4 *rowA0 = gA + si.gp_off + si.marg;
        const float2 *rowB0 = gB + si.gp_off + si.marg;
        const long long two_ct = 2LL * c_t - (n - 1);              // 2 (c_t - hn)
        const long long two_rt = (long long)(n - 1) - 2LL * r_t;   // 2 (hn - r_t)
        const long long hd2 = (long long)(si.n_det - 1) << 32;     // 2 hd in 32.32
        const float fx = (float)dc, fy = (float)dr0;
        for (int a0 = 0; a0 < si.n_theta; a0 += ADJ_CHUNK) {
            const int na = min(ADJ_CHUNK, si.n_theta - a0);
            __syncthreads();
            if ((int)threadIdx.x < na) {
                const AngleInfo an = dg.ang[si.ang_off + a0 + threadIdx.x];
                const long long U = (two_ct * an.cos_fx + two_rt * an.sin_fx + hd2) >> 1;
                const float pi = an.pch * an.inv_ch;
                s_cs[threadIdx.x] = make_float4(an.cosf, an.sinf, pi, an.pch);
                s_jp[threadIdx.x] = make_float4(
                    __int_as_float((int)(U >> 32)),
                    (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f, an.pch - pi, 0.f);
            }
            __syncthreads();
            const float4 *rowA = rowA0 + (int64_t)a0 * si.gw;
            const float2 *rowB = rowB0 + (int64_t)a0 * si.gw;
            for (int k = 0; k < na; ++k) {
                const float4 cs = s_cs[k];
                const float4 jp = s_jp[k];
                const int J = __float_as_int(jp.x);
                const float v0 = fmaf(fx, cs.x, fmaf(-fy, cs.y, jp.y));
                const float step = -8.f * cs.y;
                const float4 *rA = rowA + J;
                const float2 *rB = rowB + J;
#pragma unroll
                for (int p = 0; p < ADJ_PASSES; ++p) {
                    const float vl = fmaf((float)p, step, v0);
                    const float fl = floorf(vl);
                    const int jj = (int)fl;
                    const float d0 = vl - fl;
                    const float4 ta = __ldg(rA + jj);
                    const float2 tb = __ldg(rB + jj);
                    const float w0 = fmaxf(0.f, fmaf(-d0, cs.z, cs.w));
                    const float w1 = fmaxf(0.f, fmaf(d0, cs.z, jp.z));
                    acc[p][0] = fmaf(w0, ta.x, fmaf(w1, ta.w, acc[p][0]));
                    acc[p][1] = fmaf(w0, ta.y, fmaf(w1, tb.x, acc[p][1]));
                    acc[p][2] = fmaf(w0, ta.z, fmaf(w1, tb.y, acc[p][2]));
                }
                rowA += si.gw;
                rowB += si.gw;
            }
        }
    }

    double regv = 0.0;
    const int c = c_t + dc;
#pragma unroll
    for (int p = 0; p < ADJ_PASSES; ++p) {
        const int r = r_t + dr0 + 8 * p;
        if (r < n && c < n) {
            const int64_t idx = si.vol_off + (int64_t)r * n + c;
            const float4 x = v ? v[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
            regv += (double)(reg1.x * x.x * x.x) + (double)(reg1.y * x.y * x.y) +
                    (double)(reg1.z * x.z * x.z);
            if (with_sino && out != nullptr)
                out[idx] = make_float4(fmaf(out_mult.x, acc[p][0], reg2.x * x.x),
                                       fmaf(out_mult.y, acc[p][1], reg2.y * x.y),
                                       fmaf(out_mult.z, acc[p][2], reg2.z * x.z), 0.f);
        }
    }
    const double tot = block_sum_double_adj(regv, red);
    if (threadIdx.x == 0) part[item] = tot;
}

cudaError_t launch_backproject(const ei_geometry *g, bool with_sino, const float4 *v,
                               float4 *out, float4 out_mult, float4 reg2, float4 reg1,
                               double *part, const int *active, cudaStream_t st)
{
    if (g->dg.total_adj == 0) return cudaSuccess;
    k_backproject<<<g->dg.total_adj, ADJ_THREADS, 0, st>>>(g->dg, g->gA, g->gB, with_sino, v, out,
                                                            out_mult, reg2, reg1, part, active);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// Packed gradient sinogram from a user sino4 array ([n_theta][n_dp] float4 per
// slice): entries of pixels j = -1 .. n_det - 1 of every row; the margins are
// zero from set-up.  One block per row.
// ----------------------------------------------------------------------------
__global__ void k_pack_sino(DevGeom dg, const float4 *__restrict__ sino4, float4 *__restrict__ gA,
                            float2 *__restrict__ gB)
{
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const float4 *src = sino4 + si.sino_off + (int64_t)a * si.n_dp;
    const int64_t dst = si.gp_off + (int64_t)a * si.gw + si.marg;
    for (int j = (int)threadIdx.x - 1; j < si.n_det; j += blockDim.x) {
        const float4 lo = j >= 0 ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float4 hi = j + 1 < si.n_det ? src[j + 1] : make_float4(0.f, 0.f, 0.f, 0.f);
        gA[dst + j] = make_float4(lo.x, lo.y, lo.z, hi.x);
        gB[dst + j] = make_float2(hi.y, hi.z);
    }
}

cudaError_t launch_pack_sino(const ei_geometry *g, const float4 *sino4, cudaStream_t st)
{
    if (g->dg.total_ic == 0) return cudaSuccess;
    k_pack_sino<<<g->dg.total_ic, 256, 0, st>>>(g->dg, sino4, g->gA, g->gB);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// S[s] = sum_rows part_ic + sum_tiles part_adj, one block per slice, fixed order.
// ----------------------------------------------------------------------------
__global__ void k_finalize_objective(DevGeom dg, const double *__restrict__ part_ic,
                                     const double *__restrict__ part_adj, double *__restrict__ S,
                                     const int *__restrict__ active)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (active && !active[s]) return;
    double acc = 0.0;
    for (int i = dg.ic_prefix[s] + threadIdx.x; i < dg.ic_prefix[s + 1]; i += blockDim.x)
        acc += part_ic[i];
    for (int i = dg.adj_prefix[s] + threadIdx.x; i < dg.adj_prefix[s + 1]; i += blockDim.x)
        acc += part_adj[i];
    const double tot = block_sum_double_adj(acc, red);
    if (threadIdx.x == 0) S[s] = tot;
}

cudaError_t launch_finalize_objective(const ei_geometry *g, const double *part_ic,
                                      const double *part_adj, double *S, const int *active,
                                      cudaStream_t st)
{
    k_finalize_objective<<<g->n_slices, 256, 0, st>>>(g->dg, part_ic, part_adj, S, active);
    return cudaGetLastError();
}

}  // namespace ei
