// Adjoint R^T of the projector (the transpose the analytic gradient of Eq. 5
// needs), in gather form: every thread owns one voxel and sums, over all
// angles, its two detector taps — no atomics, a fixed summation order, so the
// result is deterministic.
//
// Matrix entry (same matrix as the ray-driven projector):
//   R[(a, j), (r, c)] = (pitch / ch) * max(0, 1 - |u - j| / ch),
//   u = (c - hn) cos + (hn - r) sin + hd,   ch = max(|cos|, |sin|),
// so voxel (r, c) reads pixels floor(u) and floor(u) + 1 of every angle.
//
// Accuracy: u reaches ~n_det, where an FP32 product would carry ~1e-4 pixel
// of rounding.  The block therefore computes, per angle, u at its tile origin
// in 32.32 fixed point and splits it into an integer J and a fraction phi;
// each voxel adds only its small local offset dc cos - dr sin in FP32.
//
// Also fused: out = out_mult * R^T g + reg2 * v (the regulariser's gradient)
// and per-tile FP64 partial sums of sum_c reg1_c v_c^2 (its value); v may be
// null (no regulariser).
#include "ei_internal.h"

namespace ei {

constexpr int ADJ_THREADS = ADJ_TILE * ADJ_TILE;

__device__ __forceinline__ double block_sum_double_adj(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = lane < (ADJ_THREADS / 32) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    return t;
}

__global__ void __launch_bounds__(ADJ_THREADS)
k_backproject(DevGeom dg, const float4 *__restrict__ sino4, const float4 *__restrict__ v,
              float4 *__restrict__ out, float4 out_mult, float4 reg2, float4 reg1,
              double *__restrict__ part, const int *__restrict__ active)
{
    __shared__ int s_J[ADJ_THREADS];
    __shared__ float s_phi[ADJ_THREADS];
    __shared__ float4 s_cs[ADJ_THREADS];     // cos, sin, 1/ch, pitch/ch
    __shared__ double red[32];

    const int item = blockIdx.x;
    const int s = find_slice(dg.adj_prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int nt = (n + ADJ_TILE - 1) / ADJ_TILE;
    const int local = item - dg.adj_prefix[s];
    const int r_t = (local / nt) * ADJ_TILE, c_t = (local % nt) * ADJ_TILE;
    const int tx = threadIdx.x % ADJ_TILE, ty = threadIdx.x / ADJ_TILE;
    const int r = r_t + ty, c = c_t + tx;
    const bool inside = r < n && c < n;
    const int nd = si.n_det;

    float ax = 0.f, ay = 0.f, az = 0.f;
    if (sino4 != nullptr) {
        const float4 *gs = sino4 + si.sino_off;
        const long long two_ct = 2LL * c_t - (n - 1);      // 2 (c_t - hn)
        const long long two_rt = (long long)(n - 1) - 2LL * r_t;   // 2 (hn - r_t)
        const long long hd2 = (long long)(nd - 1) << 32;   // 2 hd in fixed point
        const float fx = (float)tx, fy = (float)ty;
        for (int a0 = 0; a0 < si.n_theta; a0 += ADJ_THREADS) {
            const int na = min(ADJ_THREADS, si.n_theta - a0);
            if ((int)threadIdx.x < na) {
                const AngleInfo an = dg.ang[si.ang_off + a0 + threadIdx.x];
                const long long U2 = two_ct * an.cos_fx + two_rt * an.sin_fx + hd2;
                const long long U = U2 >> 1;           // u at the tile origin, 32.32
                s_J[threadIdx.x] = (int)(U >> 32);
                s_phi[threadIdx.x] = (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f;
                s_cs[threadIdx.x] = make_float4(an.cosf, an.sinf, an.inv_ch, an.pch);
            }
            __syncthreads();
            for (int k = 0; k < na; ++k) {
                const float4 cs = s_cs[k];
                const float vloc = fmaf(fx, cs.x, fmaf(-fy, cs.y, s_phi[k]));
                const float fl = floorf(vloc);
                const int j0 = s_J[k] + (int)fl;
                const float d0 = vloc - fl;
                const float w0 = cs.w * fmaxf(0.f, fmaf(-d0, cs.z, 1.f));
                const float w1 = cs.w * fmaxf(0.f, fmaf(d0 - 1.f, cs.z, 1.f));
                const float4 *grow = gs + (int64_t)(a0 + k) * si.n_dp;
                float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0;
                if (j0 >= 0 && j0 < nd) g0 = __ldg(grow + j0);
                if (j0 + 1 >= 0 && j0 + 1 < nd) g1 = __ldg(grow + j0 + 1);
                ax = fmaf(w0, g0.x, fmaf(w1, g1.x, ax));
                ay = fmaf(w0, g0.y, fmaf(w1, g1.y, ay));
                az = fmaf(w0, g0.z, fmaf(w1, g1.z, az));
            }
            __syncthreads();
        }
    }

    double regv = 0.0;
    if (inside) {
        const int64_t idx = si.vol_off + (int64_t)r * n + c;
        const float4 x = v ? v[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
        regv = (double)(reg1.x * x.x * x.x) + (double)(reg1.y * x.y * x.y) +
               (double)(reg1.z * x.z * x.z);
        if (sino4 != nullptr && out != nullptr)
            out[idx] = make_float4(fmaf(out_mult.x, ax, reg2.x * x.x),
                                   fmaf(out_mult.y, ay, reg2.y * x.y),
                                   fmaf(out_mult.z, az, reg2.z * x.z), 0.f);
    }
    const double tot = block_sum_double_adj(regv, red);
    if (threadIdx.x == 0) part[item] = tot;
}

cudaError_t launch_backproject(const ei_geometry *g, const float4 *sino4, const float4 *v,
                               float4 *out, float4 out_mult, float4 reg2, float4 reg1,
                               double *part, const int *active, cudaStream_t st)
{
    if (g->dg.total_adj == 0) return cudaSuccess;
    k_backproject<<<g->dg.total_adj, ADJ_THREADS, 0, st>>>(g->dg, sino4, v, out, out_mult, reg2,
                                                            reg1, part, active);
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
    k_finalize_objective<<<g->n_slices, ADJ_THREADS, 0, st>>>(g->dg, part_ic, part_adj, S, active);
    return cudaGetLastError();
}

}  // namespace ei
