// Forward projection R (Eq. 1) of the three channels (mu, delta, sigma).
//
// Ray-driven linear interpolation: the ray of pixel j at angle a samples one
// voxel per row (per column when |sin| > |cos|) at the crossing point and
// interpolates the two voxels it falls between; every sample carries the
// path length pitch / max(|cos|, |sin|).
//
// Layout for the inner loop: the volume is first staged as two zero-padded
// copies, row-major xp[r][1 + c] and transposed xt[c][1 + r] (n rows of
// n + 2 float4), so that a ray always walks the contiguous ("inner") axis of
// one of them: neighbouring rays read neighbouring float4, and the zero
// border removes every bounds check from the loop.  The crossing position is
// carried in 32.32 fixed point (int64): one integer add per sample, the
// integer part is the voxel index and the low word the interpolation weight,
// exact to ~1e-7 voxel for any slice size.
#include "ei_internal.h"

namespace ei {

// --------------------------------------------------------------------------
// Staging: xp = mult * vol (padded), xt = its transpose (padded).
// One block per 32 x 32 tile of a slice.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(PREP_TILE * 8)
k_prep(DevGeom dg, const float4 *__restrict__ vol, float4 mult, float4 *__restrict__ xp,
       float4 *__restrict__ xt, const int *__restrict__ active)
{
    __shared__ float4 tile[PREP_TILE][PREP_TILE + 1];
    const int item = blockIdx.x;
    const int s = find_slice(dg.prep_prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int nt = (n + PREP_TILE - 1) / PREP_TILE;
    const int local = item - dg.prep_prefix[s];
    const int r0 = (local / nt) * PREP_TILE, c0 = (local % nt) * PREP_TILE;
    const float4 *v = vol + si.vol_off;
    float4 *p = xp + si.pad_off;
    float4 *t = xt + si.pad_off;
    const int64_t w = n + 2;
    for (int dy = threadIdx.y; dy < PREP_TILE; dy += blockDim.y) {
        const int r = r0 + dy, c = c0 + threadIdx.x;
        float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
        if (r < n && c < n) {
            float4 x = v[(int64_t)r * n + c];
            val = make_float4(x.x * mult.x, x.y * mult.y, x.z * mult.z, 0.f);
            p[(int64_t)r * w + 1 + c] = val;
        }
        tile[dy][threadIdx.x] = val;
    }
    __syncthreads();
    for (int dx = threadIdx.y; dx < PREP_TILE; dx += blockDim.y) {
        const int c = c0 + dx, r = r0 + threadIdx.x;
        if (r < n && c < n) t[(int64_t)c * w + 1 + r] = tile[threadIdx.x][dx];
    }
}

// --------------------------------------------------------------------------
// Projector: one thread per ray (slice, angle, pixel); a work item is
// FWD_RAYS consecutive pixels of one angle.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(FWD_RAYS)
k_project(DevGeom dg, const float4 *__restrict__ xp, const float4 *__restrict__ xt,
          float *__restrict__ proj, const int *__restrict__ active)
{
    const int item = blockIdx.x;
    const int s = find_slice(dg.fwd_prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int nb = (si.n_dp + FWD_RAYS - 1) / FWD_RAYS;
    const int local = item - dg.fwd_prefix[s];
    const int a = local / nb;
    const int j = (local - a * nb) * FWD_RAYS + threadIdx.x;
    if (j >= si.n_dp) return;
    const int64_t plane = (int64_t)si.n_theta * si.n_dp;
    float *out = proj + si.proj_off + (int64_t)a * si.n_dp + j;
    if (j >= si.n_det) {
        out[0] = 0.f;
        out[plane] = 0.f;
        out[2 * plane] = 0.f;
        return;
    }
    const AngleInfo an = dg.ang[si.ang_off + a];
    const int n = si.n;
    const double hd = 0.5 * (si.n_det - 1);
    // inner position at o = 0, in 32.32 fixed point
    const double P0 = (j - hd) * an.inv_dom + an.k0;
    const double TWO32 = 4294967296.0;
    const long long base = __double2ll_rn(P0 * TWO32);
    const long long p1 = an.p1_fx;
    const long long lo_lim = -(1LL << 32);               // s >= -1
    const long long hi_lim = (long long)n << 32;         // s <  n
    // valid outer range [o_lo, o_hi]: first an FP64 estimate, then exact checks
    int o_lo, o_hi;
    if (p1 == 0) {
        const bool in = base >= lo_lim && base < hi_lim;
        o_lo = in ? 0 : 1;
        o_hi = in ? n - 1 : 0;
    } else {
        double e1 = (-1.0 - P0) * an.inv_p1, e2 = (n - P0) * an.inv_p1;
        double lo = fmin(e1, e2), hi = fmax(e1, e2);
        o_lo = (int)fmax(0.0, fmin((double)n, ceil(lo)));
        o_hi = (int)fmin((double)(n - 1), fmax(-1.0, floor(hi)));
        auto inr = [&](int o) {
            long long v = base + (long long)o * p1;
            return v >= lo_lim && v < hi_lim;
        };
        while (o_lo <= o_hi && !inr(o_lo)) ++o_lo;
        while (o_hi >= o_lo && !inr(o_hi)) --o_hi;
        while (o_lo > 0 && inr(o_lo - 1)) --o_lo;
        while (o_hi < n - 1 && inr(o_hi + 1)) ++o_hi;
    }
    const float4 *src = (an.col_dom ? xt : xp) + si.pad_off;
    const int64_t w = n + 2;
    float ax = 0.f, ay = 0.f, az = 0.f;
    long long pos = base + (long long)o_lo * p1;
    const float inv32 = 2.3283064365386963e-10f;   // 2^-32
    const float4 *row = src + (int64_t)o_lo * w + 1;
    for (int o = o_lo; o <= o_hi; ++o) {
        const int i0 = (int)(pos >> 32);                       // floor of the position
        const float f = (float)(unsigned)(pos & 0xffffffffLL) * inv32;
        const float4 v0 = __ldg(row + i0);
        const float4 v1 = __ldg(row + i0 + 1);
        ax += fmaf(f, v1.x - v0.x, v0.x);
        ay += fmaf(f, v1.y - v0.y, v0.y);
        az += fmaf(f, v1.z - v0.z, v0.z);
        pos += p1;
        row += w;
    }
    out[0] = ax * an.pch;
    out[plane] = ay * an.pch;
    out[2 * plane] = az * an.pch;
}

cudaError_t launch_prep(const ei_geometry *g, const float4 *vol, float4 mult, float4 *xp,
                        float4 *xt, const int *active, cudaStream_t st)
{
    if (g->dg.total_prep == 0) return cudaSuccess;
    k_prep<<<g->dg.total_prep, dim3(PREP_TILE, 8), 0, st>>>(g->dg, vol, mult, xp, xt, active);
    return cudaGetLastError();
}

cudaError_t launch_project(const ei_geometry *g, const float4 *xp, const float4 *xt,
                           float *proj, const int *active, cudaStream_t st)
{
    if (g->dg.total_fwd == 0) return cudaSuccess;
    k_project<<<g->dg.total_fwd, FWD_RAYS, 0, st>>>(g->dg, xp, xt, proj, active);
    return cudaGetLastError();
}

}  // namespace ei
