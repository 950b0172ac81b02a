// Forward projection R (Eq. 1) of the three channels (mu, delta, sigma).
//
// Ray-driven linear interpolation: the ray of pixel j at angle a samples one
// voxel per row (per column when |sin| > |cos|) at the crossing point and
// interpolates the two voxels it falls between; every sample carries the
// path length pitch / max(|cos|, |sin|).
//
// What bounds this kernel is the bytes the samples bring from L1 into
// registers (a warp-wide load returns 16 B per lane per load, whatever the
// addresses), not HBM: a 1024^2 slice with 1800 angles takes ~1.7e9 samples
// from a 17 MB volume.  So:
//  - the volume is staged once per evaluation as two pair-packed copies
//    (row-major for rows-first rays, transposed for columns-first rays): one
//    sample = one float4 + one float2 load (24 B instead of 32 B) holding a
//    voxel and its difference to the next, so the interpolation is one FMA
//    per channel, and the zero border of the copies removes every bounds
//    check from the loop;
//  - a warp covers 8 neighbouring rays x 4 neighbouring angles, so at each
//    row its lanes touch a compact run of voxels (few cache lines per load),
//    and a block covers FWD_ANGLES angles so its warps re-use each other's
//    lines in L1;
//  - several samples per loop iteration keep independent loads in flight;
//  - for the linked unknown of Eq. 4 (mu = h, delta = gamma h, sigma = 0) the
//    copies hold h alone, 8 B per entry, and R[delta] = gamma R[h] is written
//    from the same sum: a third of the bytes per sample;
//  - the crossing position is carried in 32.32 fixed point (int64): one
//    integer add per sample; the integer part is the voxel index and the low
//    word the interpolation weight, exact to ~1e-7 voxel at any slice size.
#include <algorithm>

#include "ei_internal.h"

namespace ei {

// --------------------------------------------------------------------------
// Staging: packed row-major and transposed copies of mult * vol, or with
// `linked` (the single unknown h of Eq. 4 in the mu lane) single-channel
// copies of mult.x h, 8 bytes per entry in the B arrays (the linked projector
// derives R[delta] = gamma R[mu]).  One block per 32 x 32 tile of entries; the tile
// loads the voxels it needs (with a one-voxel halo above and to the left)
// into shared memory.
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(PREP_TILE * 8)
k_prep(DevGeom dg, const float4 *__restrict__ vol, float4 mult, bool linked, float4 *__restrict__ xpA,
       float2 *__restrict__ xpB, float4 *__restrict__ xtA, float2 *__restrict__ xtB,
       const int *__restrict__ active)
{
    __shared__ float4 T[PREP_TILE + 1][PREP_TILE + 2];
    const int item = blockIdx.x;
    const int s = find_slice(dg.prep_prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int nt = (n + 1 + PREP_TILE - 1) / PREP_TILE;      // tiles over n + 1 entries
    const int local = item - dg.prep_prefix[s];
    const int R0 = (local / nt) * PREP_TILE, C0 = (local % nt) * PREP_TILE;
    const float4 *v = vol + si.vol_off;
    // T[y][x] = voxel (R0 - 1 + y, C0 - 1 + x), zero outside the slice
    for (int y = threadIdx.y; y < PREP_TILE + 1; y += blockDim.y) {
        const int r = R0 - 1 + y;
        for (int x = threadIdx.x; x < PREP_TILE + 1; x += blockDim.x) {
            const int c = C0 - 1 + x;
            float4 val = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r >= 0 && r < n && c >= 0 && c < n) {
                const float4 q = v[(int64_t)r * n + c];
                val = linked ? make_float4(q.x * mult.x, q.x * mult.y, 0.f, 0.f)
                             : make_float4(q.x * mult.x, q.y * mult.y, q.z * mult.z, 0.f);
            }
            T[y][x] = val;
        }
    }
    __syncthreads();
    const int64_t w = n + 1;
    // row-major entries (r, e): voxels (r, e - 1) and (r, e); linked: the
    // single channel's (value, difference) in the B copy only
    for (int dy = threadIdx.y; dy < PREP_TILE; dy += blockDim.y) {
        const int r = R0 + dy, e = C0 + threadIdx.x;
        if (r < n && e <= n) {
            const float4 a = T[dy + 1][threadIdx.x], b = T[dy + 1][threadIdx.x + 1];
            const int64_t k = si.pp_off + (int64_t)r * w + e;
            if (linked) {
                xpB[k] = make_float2(a.x, b.x - a.x);
            } else {
                xpA[k] = make_float4(a.x, a.y, a.z, b.x - a.x);
                xpB[k] = make_float2(b.y - a.y, b.z - a.z);
            }
        }
    }
    // transposed entries (c, e): voxels (e - 1, c) and (e, c)
    for (int dx = threadIdx.y; dx < PREP_TILE; dx += blockDim.y) {
        const int c = C0 + dx, e = R0 + threadIdx.x;
        if (c < n && e <= n) {
            const float4 a = T[threadIdx.x][dx + 1], b = T[threadIdx.x + 1][dx + 1];
            const int64_t k = si.pp_off + (int64_t)c * w + e;
            if (linked) {
                xtB[k] = make_float2(a.x, b.x - a.x);
            } else {
                xtA[k] = make_float4(a.x, a.y, a.z, b.x - a.x);
                xtB[k] = make_float2(b.y - a.y, b.z - a.z);
            }
        }
    }
}

// --------------------------------------------------------------------------
// Projector: one thread per ray; a work item is ANGLES angles x RAYS pixels of
// one slice; a warp covers WRAYS neighbouring pixels x 32 / WRAYS neighbouring
// angles, with consecutive lanes on neighbouring pixels or (AFAST) on
// neighbouring angles.  The order matters because L1 serves a 16-byte load of
// 8 consecutive lanes in one pass only when their addresses share a 128-byte
// line: neighbouring angles of one ray sample nearly the same voxels, while
// neighbouring rays sample voxels 1 to 1.4 entries apart.  Templated on the
// tile shape, the warp shape and the unroll so the autotuner can choose among
// instantiations.
// --------------------------------------------------------------------------
// Ray (pixel j, angle an) through an n x n slice: its inner position at outer
// index o is (base + o p1) / 2^32 voxels (32.32 fixed point), and it samples
// the rows o_lo .. o_hi, those whose position lies in [-1, n) (empty when
// o_lo > o_hi).
struct RaySetup {
    long long base, p1;
    int o_lo, o_hi;
};

__device__ __forceinline__ RaySetup ray_setup(const AngleInfo &an, int j, int n, int n_det)
{
    const double hd = 0.5 * (n_det - 1);
    // inner position at o = 0, in 32.32 fixed point
    const double P0 = (j - hd) * an.inv_dom + an.k0;
    const double TWO32 = 4294967296.0;
    RaySetup r;
    r.base = __double2ll_rn(P0 * TWO32);
    r.p1 = an.p1_fx;
    const long long base = r.base, p1 = r.p1;
    const long long lo_lim = -(1LL << 32);               // position >= -1
    const long long hi_lim = (long long)n << 32;         // position <  n
    // valid outer range [o_lo, o_hi]: an FP64 estimate, then exact int64 checks
    int o_lo, o_hi;
    if (p1 == 0) {
        const bool in = base >= lo_lim && base < hi_lim;
        o_lo = in ? 0 : 1;
        o_hi = in ? n - 1 : 0;
    } else {
        const double e1 = (-1.0 - P0) * an.inv_p1, e2 = (n - P0) * an.inv_p1;
        o_lo = (int)fmax(0.0, fmin((double)n, ceil(fmin(e1, e2))));
        o_hi = (int)fmin((double)(n - 1), fmax(-1.0, floor(fmax(e1, e2))));
        auto inr = [&](int o) {
            const long long q = base + (long long)o * p1;
            return q >= lo_lim && q < hi_lim;
        };
        while (o_lo <= o_hi && !inr(o_lo)) ++o_lo;
        while (o_hi >= o_lo && !inr(o_hi)) --o_hi;
        while (o_lo > 0 && inr(o_lo - 1)) --o_lo;
        while (o_hi < n - 1 && inr(o_hi + 1)) ++o_hi;
    }
    r.o_lo = o_lo;
    r.o_hi = o_hi;
    return r;
}

// Adds the samples of rows o0 .. o1 of one ray to acc (row order, so any split
// of a ray's rows into consecutive segments gives the same sums).  A, B: the
// packed copy's entries of position 0 of row 0 (entry i0 + 1 holds the voxel
// at i0 and its difference to the next).
template <int UNROLL, bool LINKED>
__device__ __forceinline__ void ray_rows(const RaySetup &rs, int o0, int o1, const float4 *A,
                                         const float2 *B, int64_t w, float (&acc)[3],
                                         int *status)
{
    // the sampled position lies in [-1, n) by construction (ray_setup): entry
    // i0 + 1 of the row's n + 1; check builds verify it
    const int n = (int)w - 1;
    if (o0 > o1) return;
    const float inv32 = 2.3283064365386963e-10f;   // 2^-32
    long long pos = rs.base + (long long)o0 * rs.p1;
    const float4 *rowA = A + o0 * w;
    const float2 *rowB = B + o0 * w;
    const long long p1 = rs.p1;
    int o = o0;
    for (; o + UNROLL - 1 <= o1; o += UNROLL) {
        float4 va[UNROLL];
        float2 vb[UNROLL];
        float f[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            const long long q = pos + u * p1;
            const int i0 = checked_index((int)(q >> 32), -1, n - 1, status);   // floor of the position
            f[u] = (float)(unsigned)(q & 0xffffffffLL) * inv32;
            if (!LINKED) va[u] = __ldg(rowA + u * w + i0);
            vb[u] = __ldg(rowB + u * w + i0);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            if (LINKED) {
                acc[0] += fmaf(f[u], vb[u].y, vb[u].x);
            } else {
                acc[0] += fmaf(f[u], va[u].w, va[u].x);
                acc[1] += fmaf(f[u], vb[u].x, va[u].y);
                acc[2] += fmaf(f[u], vb[u].y, va[u].z);
            }
        }
        pos += UNROLL * p1;
        rowA += UNROLL * w;
        rowB += UNROLL * w;
    }
    for (; o <= o1; ++o) {
        const int i0 = checked_index((int)(pos >> 32), -1, n - 1, status);
        const float f = (float)(unsigned)(pos & 0xffffffffLL) * inv32;
        const float2 vb = __ldg(rowB + i0);
        if (LINKED) {
            acc[0] += fmaf(f, vb.y, vb.x);
        } else {
            const float4 va = __ldg(rowA + i0);
            acc[0] += fmaf(f, va.w, va.x);
            acc[1] += fmaf(f, vb.x, va.y);
            acc[2] += fmaf(f, vb.y, va.z);
        }
        pos += p1;
        rowA += w;
        rowB += w;
    }
}

// The three output planes of one ray: (R[mu], R[delta], R[sigma]), or linked
// (R[h], gamma R[h], 0).
template <bool LINKED>
__device__ __forceinline__ void ray_store(float *out, int64_t plane, const float (&acc)[3],
                                          float pch, float link)
{
    if (LINKED) {
        const float pm = acc[0] * pch;
        out[0] = pm;
        out[plane] = link * pm;
        out[2 * plane] = 0.f;
    } else {
        out[0] = acc[0] * pch;
        out[plane] = acc[1] * pch;
        out[2 * plane] = acc[2] * pch;
    }
}

// The full ray of pixel j at angle an.
template <int UNROLL, bool LINKED>
__device__ __forceinline__ void project_ray(const SliceInfo &si, const AngleInfo &an, int j,
                                            const float4 *__restrict__ xpA,
                                            const float2 *__restrict__ xpB,
                                            const float4 *__restrict__ xtA,
                                            const float2 *__restrict__ xtB, float *out,
                                            int64_t plane, float link, int *status)
{
    const RaySetup rs = ray_setup(an, j, si.n, si.n_det);
    const int64_t off = si.pp_off + 1;
    float acc[3] = {0.f, 0.f, 0.f};
    if (kDeviceChecks && rs.o_lo <= rs.o_hi)       // rows of the slice
        if (checked_index(rs.o_lo, 0, si.n - 1, status) != rs.o_lo ||
            checked_index(rs.o_hi, 0, si.n - 1, status) != rs.o_hi)
            return;
    ray_rows<UNROLL, LINKED>(rs, rs.o_lo, rs.o_hi, (an.col_dom ? xtA : xpA) + off,
                             (an.col_dom ? xtB : xpB) + off, si.n + 1, acc, status);
    ray_store<LINKED>(out, plane, acc, an.pch, link);
}

template <int RAYS, int ANGLES, int UNROLL, int WRAYS, bool AFAST, bool LINKED, int QUADS = 0>
__device__ __forceinline__ void project_item(const DevGeom &dg, const int *prefix, int item,
                                             const float4 *__restrict__ xpA,
                                             const float2 *__restrict__ xpB,
                                             const float4 *__restrict__ xtA,
                                             const float2 *__restrict__ xtB,
                                             float *__restrict__ proj, float link,
                                             const int *__restrict__ active)
{
    const int s = find_slice(prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int nrb = (si.n_dp + RAYS - 1) / RAYS;
    const int local = item - prefix[s];
    const int ab = local / nrb, rb = local - ab * nrb;
    static_assert(RAYS % WRAYS == 0 && 32 % WRAYS == 0 && ANGLES % (32 / WRAYS) == 0,
                  "block tile must be a whole number of warp tiles");
    static_assert(QUADS == 0 || WRAYS == 4, "2 x 4 lane groups need warps of 4 rays x 8 angles");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int WR = RAYS / WRAYS;                   // warps along the rays
    constexpr int WA = 32 / WRAYS;                     // angles per warp
    // lane order within the warp's WRAYS x WA tile: rays first, angles first
    // (AFAST), or (QUADS, for 4 x 8 warps) groups of 8 lanes on 2 rays x 4
    // angles, their pairs on 2 rays x 8 angles (QUADS == 1) or 4 rays x 4
    // angles (QUADS == 2)
    int la, lr;
    if (QUADS == 1) {
        la = (lane & 3) | (((lane >> 3) & 1) << 2);
        lr = ((lane >> 2) & 1) | (((lane >> 4) & 1) << 1);
    } else if (QUADS == 2) {
        la = (lane & 3) | (((lane >> 4) & 1) << 2);
        lr = (lane >> 2) & 3;
    } else {
        la = AFAST ? lane % WA : lane / WRAYS;
        lr = AFAST ? lane / WA : lane % WRAYS;
    }
    const int a = ab * ANGLES + (warp / WR) * WA + la;
    const int j = rb * RAYS + (warp % WR) * WRAYS + lr;
    if (a >= si.n_theta || j >= si.n_dp) return;
    const int64_t plane = (int64_t)si.n_theta * si.n_dp;
    float *out = proj + si.proj_off + (int64_t)a * si.n_dp + j;
    if (j >= si.n_det) {
        out[0] = 0.f;
        out[plane] = 0.f;
        out[2 * plane] = 0.f;
        return;
    }
    project_ray<UNROLL, LINKED>(si, dg.ang[si.ang_off + a], j, xpA, xpB, xtA, xtB, out, plane, link,
                                dg.status);
}

// One block per work item.
template <int RAYS, int ANGLES, int UNROLL, int WRAYS, bool AFAST, bool LINKED, int QUADS>
__global__ void __launch_bounds__(RAYS * ANGLES)
k_project(DevGeom dg, const int *__restrict__ prefix, const float4 *__restrict__ xpA,
          const float2 *__restrict__ xpB, const float4 *__restrict__ xtA,
          const float2 *__restrict__ xtB, float *__restrict__ proj, float link,
          const int *__restrict__ active)
{
    project_item<RAYS, ANGLES, UNROLL, WRAYS, AFAST, LINKED, QUADS>(dg, prefix, blockIdx.x, xpA, xpB, xtA,
                                                             xtB, proj, link, active);
}

// Persistent: a GPU-sized grid whose blocks take work items from a counter
// (set to 0 before the launch) until the list is exhausted; no block waits on
// another.
template <int RAYS, int ANGLES, int UNROLL, int WRAYS, bool AFAST, bool LINKED, int QUADS>
__global__ void __launch_bounds__(RAYS * ANGLES)
k_project_persistent(DevGeom dg, const int *__restrict__ prefix, int total, int *counter,
                     const float4 *__restrict__ xpA, const float2 *__restrict__ xpB,
                     const float4 *__restrict__ xtA, const float2 *__restrict__ xtB,
                     float *__restrict__ proj, float link, const int *__restrict__ active)
{
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item >= total) return;
        project_item<RAYS, ANGLES, UNROLL, WRAYS, AFAST, LINKED, QUADS>(dg, prefix, item, xpA, xpB, xtA, xtB,
                                                                 proj, link, active);
    }
}

// Persistent, SM-chunked: the blocks resident on one SM take consecutive work
// items (neighbouring ray groups of the same angles) from their SM's chunk of
// the list, then items of the other chunks; the chunk counters are 0 before
// the launch.  No block waits on another.
template <int RAYS, int ANGLES, int UNROLL, int WRAYS, bool AFAST, bool LINKED, int QUADS>
__global__ void __launch_bounds__(RAYS * ANGLES, 1280 / (RAYS * ANGLES))   // 5 blocks of 256
k_project_sm(DevGeom dg, const int *__restrict__ prefix, int total, int *counters,
             const float4 *__restrict__ xpA, const float2 *__restrict__ xpB,
             const float4 *__restrict__ xtA, const float2 *__restrict__ xtB,
             float *__restrict__ proj, float link, const int *__restrict__ active)
{
    __shared__ int s_item, s_k;
    const int sm = sm_id(), nchunk = sm_id_count();
    if (threadIdx.x == 0) s_k = 0;
    for (;;) {
        if (threadIdx.x == 0) s_item = sm_chunk_next(total, counters, sm % nchunk, nchunk, &s_k);
        __syncthreads();
        const int item = s_item;
        __syncthreads();
        if (item < 0) return;
        project_item<RAYS, ANGLES, UNROLL, WRAYS, AFAST, LINKED, QUADS>(dg, prefix, item, xpA, xpB, xtA, xtB,
                                                                 proj, link, active);
    }
}

template <int R, int A, int U, int W, bool F, bool L, int Q>
static cudaError_t launch_project_mode(const ei_geometry *g, float *proj, float link,
                                       const int *active, cudaStream_t st)
{
    const FwdVariant &v = g->fwd_variant;
    if (v.total == 0) return cudaSuccess;
    if (g->persistent == LAUNCH_PER_ITEM) {
        k_project<R, A, U, W, F, L, Q><<<v.total, R * A, 0, st>>>(g->dg, v.prefix, g->xpA, g->xpB,
                                                              g->xtA, g->xtB, proj, link, active);
    } else if (g->persistent == LAUNCH_SM_CHUNKS) {
        static int per_sm = 0;          // resident blocks per SM (same for every GB300)
        if (per_sm == 0)
            EI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_project_sm<R, A, U, W, F, L, Q>, R * A, 0));
        const int grid = std::max(1, std::min(v.total, per_sm * g->num_sms));
        EI_CUDA_TRY(cudaMemsetAsync(g->sm_counters, 0, MAX_SM_CHUNKS * sizeof(int), st));
        k_project_sm<R, A, U, W, F, L, Q><<<grid, R * A, 0, st>>>(
            g->dg, v.prefix, v.total, g->sm_counters, g->xpA, g->xpB, g->xtA, g->xtB, proj, link,
            active);
    } else {
        static int per_sm = 0;          // resident blocks per SM (same for every GB300)
        if (per_sm == 0)
            EI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_project_persistent<R, A, U, W, F, L, Q>, R * A, 0));
        const int grid = std::max(1, std::min(v.total, per_sm * g->num_sms));
        EI_CUDA_TRY(cudaMemsetAsync(g->work_counter, 0, sizeof(int), st));
        k_project_persistent<R, A, U, W, F, L, Q><<<grid, R * A, 0, st>>>(
            g->dg, v.prefix, v.total, g->work_counter, g->xpA, g->xpB, g->xtA, g->xtB, proj, link,
            active);
    }
    return cudaGetLastError();
}

template <int R, int A, int U, int W, bool F, int Q = 0>
static cudaError_t launch_project_variant(const ei_geometry *g, float *proj, float link,
                                          const int *active, cudaStream_t st)
{
    return link > 0.f ? launch_project_mode<R, A, U, W, F, true, Q>(g, proj, link, active, st)
                      : launch_project_mode<R, A, U, W, F, false, Q>(g, proj, 0.f, active, st);
}

cudaError_t launch_prep(const ei_geometry *g, const float4 *vol, float4 mult, bool linked,
                        const int *active, cudaStream_t st)
{
    if (g->dg.total_prep == 0) return cudaSuccess;
    k_prep<<<g->dg.total_prep, dim3(PREP_TILE, 8), 0, st>>>(g->dg, vol, mult, linked, g->xpA, g->xpB,
                                                             g->xtA, g->xtB, active);
    return cudaGetLastError();
}

cudaError_t launch_project(const ei_geometry *g, float *proj, float link, const int *active,
                           cudaStream_t st)
{
    switch (g->fwd_variant.id) {
    case 0: return launch_project_variant<16, 16, 4, 8, false>(g, proj, link, active, st);
    case 1: return launch_project_variant<32, 8, 4, 8, false>(g, proj, link, active, st);
    case 2: return launch_project_variant<32, 16, 4, 8, false>(g, proj, link, active, st);
    case 3: return launch_project_variant<16, 16, 2, 8, false>(g, proj, link, active, st);
    case 4: return launch_project_variant<32, 8, 4, 32, false>(g, proj, link, active, st);
    case 5: return launch_project_variant<16, 16, 4, 16, false>(g, proj, link, active, st);
    case 6: return launch_project_variant<32, 16, 4, 32, false>(g, proj, link, active, st);
    case 7: return launch_project_variant<16, 16, 4, 4, true>(g, proj, link, active, st);
    case 8: return launch_project_variant<8, 32, 4, 4, true>(g, proj, link, active, st);
    case 9: return launch_project_variant<32, 8, 4, 4, true>(g, proj, link, active, st);
    case 10: return launch_project_variant<16, 16, 4, 2, true>(g, proj, link, active, st);
    // groups of 8 lanes on 2 rays x 4 angles (pairs of groups on 2 x 8 or 4 x 4)
    case 11: return launch_project_variant<8, 32, 4, 4, true, 1>(g, proj, link, active, st);
    default: return launch_project_variant<8, 32, 4, 4, true, 2>(g, proj, link, active, st);
    }
}

// Tile shape (rays, angles) of projector variant `id` (see launch_project).
void project_variant_shape(int id, int *rays, int *angles)
{
    static const int R[N_FWD_VARIANTS] = {16, 32, 32, 16, 32, 16, 32, 16, 8, 32, 16, 8, 8},
                     A[N_FWD_VARIANTS] = {16, 8, 16, 16, 8, 16, 16, 16, 32, 8, 16, 32, 32};
    *rays = R[id];
    *angles = A[id];
}

}  // namespace ei
