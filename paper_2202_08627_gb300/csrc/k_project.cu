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
#include <climits>

#include "async_copy.h"
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

// --------------------------------------------------------------------------
// Staged variant: the rows a block samples go through shared memory.
//
// A block covers STG_RAYS rays x STG_ANGLES angles, each thread STG_RPT rays
// of one angle (rays j, j + 4, ...), so that at every step a warp's lanes sit
// on 4 neighbouring rays x 8 neighbouring angles in the lane order of variant
// 12.  All its rays step through the rows together.  At row o every position
// the block samples lies in a window of W entries starting at
// floor((L + o pc) / 2^32) + 1: pc is the slope of the block's middle angle and
// L (H) the least (largest) value of P(o) - o pc over the block's rays, taken
// at the first and last row each ray samples (P(o) - o pc is linear in o, so
// those two rows bound it); W = floor((H - L) / 2^32) + 2.  On 1024^2 and
// 512^2 slices with 1800 angles W is 24..95 entries, 5-7% of the block's
// samples per row.  Warp 0 copies the windows into a ring of STG_NS stages of
// STG_ROWS rows with bulk asynchronous copies (one lane per row, one mbarrier
// per stage) while the block samples the stage before; it also writes each
// staged row's shared-memory offsets into a row table, so a sample's address
// is one multiply-add of the position's integer part.  A stage that every ray
// of a warp samples throughout runs without per-sample tests.  With
// STG_WMAX = 88 a block needs 43 KB of shared memory and four blocks (32
// warps) fit an SM; 2-3% of the blocks of 1024^2 slices have wider windows.
//
// Why: an L1 load costs one pass of the data path for every 128-byte line its
// quarter warp (16-byte loads) touches, and the 4 to 7 entries of a quarter
// warp straddle a line boundary about half the time; a shared-memory load of
// the same entries is one pass whenever they lie within 8 consecutive 16-byte
// slots, since the banks wrap around.  Blocks whose angles mix row- and
// column-first rays, or whose window exceeds STG_WMAX, read global memory as
// the other variants do.  Every ray adds the same samples in the same order
// with the same arithmetic, so the projections equal the other variants' bit
// for bit.
// --------------------------------------------------------------------------
#ifndef EI_STG_RAYS
#define EI_STG_RAYS 32               // block tile: rays x angles, rays per thread
#endif
#ifndef EI_STG_ANGLES
#define EI_STG_ANGLES 32
#endif
#ifndef EI_STG_RPT
#define EI_STG_RPT 4
#endif
#ifndef EI_STG_WMAX
#define EI_STG_WMAX 88               // widest staged window (entries)
#endif
constexpr int STG_RAYS = EI_STG_RAYS, STG_ANGLES = EI_STG_ANGLES, STG_RPT = EI_STG_RPT;
constexpr int STG_THREADS = STG_RAYS * STG_ANGLES / STG_RPT;     // 256
// Compile-time tunables (measured defaults): rows per stage, stages in the
// ring, row-loop unroll, how a buffer is released for refilling (0: a block
// barrier after each stage; 1: per-stage "empty" mbarriers, warp 0 waiting for
// every warp), and how a ray outside its rows is skipped (1: a select of the
// zero entry; 0: a branch).
#ifndef EI_STG_ROWS
#define EI_STG_ROWS 10
#endif
#ifndef EI_STG_NS
#define EI_STG_NS 2
#endif
#ifndef EI_STG_UNROLL
#define EI_STG_UNROLL 1
#endif
#ifndef EI_STG_SYNC
#define EI_STG_SYNC 0
#endif
#ifndef EI_STG_SEL
#define EI_STG_SEL 0
#endif
#ifndef EI_STG_MINB
#define EI_STG_MINB 4                // resident blocks per SM the registers are sized for
#endif
constexpr int STG_ROWS = EI_STG_ROWS, STG_NS = EI_STG_NS, STG_WMAX = EI_STG_WMAX;
constexpr int STG_UNROLL = EI_STG_UNROLL;
constexpr uint64_t kStageWaitNs = 2000000000ull;                  // 2 s bound on a stage's copies

template <bool LINKED>
struct StageLayout {
    static constexpr int kBars = 0;                               // full[STG_NS], empty[STG_NS]
    static constexpr int kRed = 128;                              // 8 warps x 4 int64
    static constexpr int kRow = 384;                              // STG_NS x STG_ROWS int4
    static constexpr int kPar = (kRow + STG_NS * STG_ROWS * 16 + 127) / 128 * 128;   // StageParams
    static constexpr int kZero = kPar + 64;                       // one zero A / B entry
    static constexpr int kA = kPar + 128;
    static constexpr int kRowA = STG_WMAX * 16;                   // float4 entries of a row
    static constexpr int kRowB = (STG_WMAX + 2) * 8;              // float2 entries, even start
    static constexpr int kB = kA + (LINKED ? 0 : STG_NS * STG_ROWS * kRowA);
    static constexpr int kBytes = kB + STG_NS * STG_ROWS * kRowB;
};
static_assert(STG_THREADS == 256 && STG_RAYS % (4 * STG_RPT) == 0 && STG_ANGLES % 8 == 0 &&
              (STG_RAYS / (4 * STG_RPT)) * (STG_ANGLES / 8) * 32 == STG_THREADS,
              "warps of 4 rays x 8 angles, STG_RPT rays per thread");
static_assert(STG_ROWS <= 32 && StageLayout<false>::kRowB % 16 == 0, "one lane per staged row");
static_assert(2 * STG_NS * 8 <= 128, "barriers fit their region");
static_assert(StageLayout<false>::kBytes <= 227 * 1024, "one block fits an SM's shared memory");

// What warp 0 needs to copy a stage (kept in shared memory, not in every
// thread's registers).
struct StageParams {
    long long L, pc, pp_off;
    const float4 *gA;
    const float2 *gB;
    int O_lo, O_hi, W, w;
};
static_assert(sizeof(StageParams) <= 64, "StageParams sits before the zero entry");

template <typename T>
__device__ __forceinline__ T warp_min(T v)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v)
{
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// The samples of rows o0 .. o1 (one stage) of a thread's rays from the staged
// windows; rt: the stage's row table (A and B byte offsets, window start).
// With TEST a ray adds only the rows in [lo, lo + span]: at other rows it
// skips the sample (EI_STG_SEL 0) or reads the zero entry (kZero), whose
// sample fmaf(f, 0, 0) is +0; adding +0 leaves the sum's bits unchanged (a sum
// that starts at +0 is never -0).  Without TEST the caller has checked that
// every ray samples every row of the stage.
template <bool LINKED, bool TEST>
__device__ __forceinline__ void stage_rows(const int4 *rt, int o0, int o1, const char *sbytes,
                                           long long (&pos)[STG_RPT], long long p1,
                                           const int (&lo)[STG_RPT], const int (&span)[STG_RPT],
                                           int W, float (&acc)[STG_RPT][3], int *status)
{
    constexpr int kZero = StageLayout<LINKED>::kZero;
    const float inv32 = 2.3283064365386963e-10f;   // 2^-32
#pragma unroll STG_UNROLL
    for (int o = o0; o <= o1; ++o) {
        const int4 ro = rt[o - o0];
#pragma unroll
        for (int t = 0; t < STG_RPT; ++t) {
            const bool act = !TEST || (unsigned)(o - lo[t]) <= (unsigned)span[t];
            if (!EI_STG_SEL && !act) {
                pos[t] += p1;
                continue;
            }
            const long long q = pos[t];
            int i0 = (int)(q >> 32);                                 // floor of the position
            if (kDeviceChecks && act)                                // window slot i0 + 1 - start
                i0 = checked_index(i0 + 1 - ro.z, 0, W - 1, status) + ro.z - 1;
            const int addrA = act ? ro.x + i0 * 16 : kZero, addrB = act ? ro.y + i0 * 8 : kZero;
            const float f = (float)(unsigned)(q & 0xffffffffLL) * inv32;
            const float2 vb = *reinterpret_cast<const float2 *>(sbytes + addrB);
            if (LINKED) {
                acc[t][0] += fmaf(f, vb.y, vb.x);
            } else {
                const float4 va = *reinterpret_cast<const float4 *>(sbytes + addrA);
                acc[t][0] += fmaf(f, va.w, va.x);
                acc[t][1] += fmaf(f, vb.x, va.y);
                acc[t][2] += fmaf(f, vb.y, va.z);
            }
            pos[t] += p1;
        }
    }
}

template <bool LINKED>
__global__ void __launch_bounds__(STG_THREADS, LINKED ? 4 : EI_STG_MINB)
k_project_staged(DevGeom dg, const int *__restrict__ prefix, const float4 *__restrict__ xpA,
                 const float2 *__restrict__ xpB, const float4 *__restrict__ xtA,
                 const float2 *__restrict__ xtB, float *__restrict__ proj, float link,
                 const int *__restrict__ active)
{
    using Lay = StageLayout<LINKED>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + Lay::kBars);
    long long *red = reinterpret_cast<long long *>(smem + Lay::kRed);
    int4 *rowtab = reinterpret_cast<int4 *>(smem + Lay::kRow);
    float4 *sA = reinterpret_cast<float4 *>(smem + Lay::kA);
    float2 *sB = reinterpret_cast<float2 *>(smem + Lay::kB);

    const int item = blockIdx.x;
    const int s = find_slice(prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int nrb = (si.n_dp + STG_RAYS - 1) / STG_RAYS;
    const int local = item - prefix[s];
    const int ab = local / nrb, rb = local - ab * nrb;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    constexpr int WR = STG_RAYS / (4 * STG_RPT);                 // warps along the rays
    const int la = (lane & 3) | (((lane >> 4) & 1) << 2), lr = (lane >> 2) & 3;
    const int a = ab * STG_ANGLES + (warp / WR) * 8 + la;
    const int j0 = rb * STG_RAYS + (warp % WR) * (4 * STG_RPT) + lr;
    const bool a_ok = a < si.n_theta;
    const AngleInfo an = dg.ang[si.ang_off + (a_ok ? a : si.n_theta - 1)];
    const int a_mid = min(ab * STG_ANGLES + STG_ANGLES / 2, si.n_theta - 1);
    const long long pc = dg.ang[si.ang_off + a_mid].p1_fx;
    const int mid_col = dg.ang[si.ang_off + a_mid].col_dom;
    const int n = si.n, w = si.n + 1;

    // the rays: first row (lo; 2^30 when the ray misses the slice), rows after
    // it (span), fixed-point position at the row the block starts on (pos)
    int lo[STG_RPT], span[STG_RPT];
    long long pos[STG_RPT];
    int o_min = INT_MAX, o_max = -1;
    long long d_min = LLONG_MAX, d_max = LLONG_MIN;
    const long long p1 = an.p1_fx;
#pragma unroll
    for (int t = 0; t < STG_RPT; ++t) {
        const int j = j0 + 4 * t;
        RaySetup rs{0, 0, 1, 0};
        if (a_ok && j < si.n_det) rs = ray_setup(an, j, n, si.n_det);
        pos[t] = rs.base;
        if (rs.o_lo <= rs.o_hi) {
            lo[t] = rs.o_lo;
            span[t] = rs.o_hi - rs.o_lo;
            o_min = min(o_min, rs.o_lo);
            o_max = max(o_max, rs.o_hi);
            const long long d1 = rs.base + (long long)rs.o_lo * (p1 - pc);
            const long long d2 = rs.base + (long long)rs.o_hi * (p1 - pc);
            d_min = min(d_min, min(d1, d2));
            d_max = max(d_max, max(d1, d2));
        } else {
            lo[t] = 1 << 30;
            span[t] = 0;
        }
    }
    const bool any = o_min <= o_max;
    o_min = warp_min(o_min);
    o_max = warp_max(o_max);
    d_min = warp_min(d_min);
    d_max = warp_max(d_max);
    if (lane == 0) {
        red[4 * warp + 0] = o_min;
        red[4 * warp + 1] = o_max;
        red[4 * warp + 2] = d_min;
        red[4 * warp + 3] = d_max;
    }
    if (threadIdx.x == 0) {
        for (int b = 0; b < STG_NS; ++b) {
            mbar_init(smem_addr(&bars[b]), 1);                        // full: the copies
            mbar_init(smem_addr(&bars[STG_NS + b]), STG_THREADS / 32); // empty: every warp
        }
        mbar_init_fence();
        *reinterpret_cast<float4 *>(smem + Lay::kZero) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const int mixed = __syncthreads_or(any && an.col_dom != mid_col);
    int O_lo = INT_MAX, O_hi = -1;
    long long L = LLONG_MAX, H = LLONG_MIN;
#pragma unroll
    for (int q = 0; q < STG_THREADS / 32; ++q) {
        O_lo = min(O_lo, (int)red[4 * q + 0]);
        O_hi = max(O_hi, (int)red[4 * q + 1]);
        L = min(L, red[4 * q + 2]);
        H = max(H, red[4 * q + 3]);
    }
    const int W = O_lo <= O_hi ? (int)((H - L) >> 32) + 2 : 0;
    const bool staged = O_lo <= O_hi && !mixed && W <= STG_WMAX;

    float acc[STG_RPT][3];
#pragma unroll
    for (int t = 0; t < STG_RPT; ++t) acc[t][0] = acc[t][1] = acc[t][2] = 0.f;
    bool failed = false;

    if (staged) {
        // every sampling ray of the block has the middle angle's orientation
        const float4 *gA = mid_col ? xtA : xpA;
        const float2 *gB = mid_col ? xtB : xpB;
        // absolute entries: entry e of row o is pp_off + o w + e
        const int nrows = O_hi - O_lo + 1, nst = (nrows + STG_ROWS - 1) / STG_ROWS;
        StageParams *sp = reinterpret_cast<StageParams *>(smem + Lay::kPar);
        if (threadIdx.x == 0) *sp = StageParams{L, pc, si.pp_off, gA, gB, O_lo, O_hi, W, w};
        __syncwarp();
        // warp 0: arm stage k's barrier with its byte count, then copy its rows
        auto issue = [&](int k) {
            const StageParams prm = *sp;
            const long long L = prm.L, pc = prm.pc;
            const float4 *gA = prm.gA;
            const float2 *gB = prm.gB;
            const int O_lo = prm.O_lo, O_hi = prm.O_hi, W = prm.W, w = prm.w;
            const int buf = k % STG_NS, o = O_lo + k * STG_ROWS + lane;
            unsigned bytesA = 0, bytesB = 0;
            const float4 *srcA = nullptr;
            const float2 *srcB = nullptr;
            float4 *dstA = nullptr;
            float2 *dstB = nullptr;
            if (lane < STG_ROWS && o <= O_hi) {
                const int start = (int)((L + (long long)o * pc) >> 32) + 1;
                const int e0 = max(start, 0), e1 = min(start + W, w);
                // byte offsets from the start of shared memory at which the
                // entry e = i0 + 1 of the sampled position's floor i0 sits:
                // offA + 16 i0 (A) and offB + 8 i0 (B)
                const long long rb0 = prm.pp_off + (long long)o * w;
                const int par = (int)((rb0 + start) & 1LL);
                const int r0 = buf * STG_ROWS + lane;
                rowtab[r0] = make_int4(Lay::kA + r0 * Lay::kRowA + (1 - start) * 16,
                                       Lay::kB + r0 * Lay::kRowB + (1 - start + par) * 8, start, 0);
                if (e1 > e0) {
                    const long long b0 = (rb0 + e0) & ~1LL, b1 = (rb0 + e1 + 1) & ~1LL;
                    const long long sb = (rb0 + start) & ~1LL;    // slot 0 of the B row
                    if (!LINKED) {
                        bytesA = (unsigned)(e1 - e0) * 16u;
                        srcA = gA + rb0 + e0;
                        dstA = sA + (buf * STG_ROWS + lane) * STG_WMAX + (e0 - start);
                    }
                    bytesB = (unsigned)(b1 - b0) * 8u;
                    srcB = gB + b0;
                    dstB = sB + (buf * STG_ROWS + lane) * (STG_WMAX + 2) + (int)(b0 - sb);
                }
            }
            unsigned tot = bytesA + bytesB;
            for (int q = 16; q > 0; q >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, q);
            const unsigned bar = smem_addr(&bars[buf]);
            __syncwarp();             // the row table's writes precede the (releasing) arrive
            if (lane == 0) mbar_arrive_expect_tx(bar, tot);
            __syncwarp();
            if (bytesA) bulk_copy_g2s(dstA, srcA, bytesA, bar);
            if (bytesB) bulk_copy_g2s(dstB, srcB, bytesB, bar);
        };
        int issued = 0;
        if (warp == 0)
            for (; issued < STG_NS && issued < nst; ++issued) issue(issued);
#pragma unroll
        for (int t = 0; t < STG_RPT; ++t) pos[t] += (long long)O_lo * p1;
        // rows every ray of the thread samples: stages inside them need no
        // per-sample test
        int lo_max = 0, hi_min = INT_MAX;
#pragma unroll
        for (int t = 0; t < STG_RPT; ++t) {
            lo_max = max(lo_max, lo[t]);
            hi_min = min(hi_min, lo[t] + span[t]);
        }
        const char *sbytes = reinterpret_cast<const char *>(smem);
        // Each warp waits for a stage's copies (full) and samples it.  Then
        // either the block meets at a barrier (EI_STG_SYNC 0) or each warp
        // arrives on the stage's empty barrier and warp 0 waits for all of them
        // (EI_STG_SYNC 1); after that warp 0 refills the buffer with stage
        // k + STG_NS.
        int k = 0;
        bool ok = true;
        for (; k < nst; ++k) {
            const int buf = k % STG_NS;
            const unsigned ph = (unsigned)(k / STG_NS) & 1u;
            ok = __all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(&bars[buf]), ph, kStageWaitNs));
            if (ok) {
                const int o0 = O_lo + k * STG_ROWS, o1 = min(O_hi, o0 + STG_ROWS - 1);
                const int4 *rt = rowtab + buf * STG_ROWS;
                if (__all_sync(0xffffffffu, o0 >= lo_max && o1 <= hi_min))
                    stage_rows<LINKED, false>(rt, o0, o1, sbytes, pos, p1, lo, span, W, acc, dg.status);
                else
                    stage_rows<LINKED, true>(rt, o0, o1, sbytes, pos, p1, lo, span, W, acc, dg.status);
            }
            if (EI_STG_SYNC == 0) {
                ok = __syncthreads_and(ok);
                if (!ok) break;
            } else {
                if (!ok) break;
                __syncwarp();
                if (lane == 0) mbar_arrive(smem_addr(&bars[STG_NS + buf]));
                if (warp == 0 && issued < nst) {
                    ok = __all_sync(0xffffffffu, mbar_wait_bounded(smem_addr(&bars[STG_NS + buf]), ph,
                                                                   kStageWaitNs));
                    if (!ok) break;
                }
            }
            if (warp == 0 && issued < nst) issue(issued++);
        }
        if (!ok) {
            // a wait ran out: report it; warp 0 gives the copies it issued that
            // no wait has seen land a bounded chance to do so before the block's
            // shared memory is released
            failed = true;
            if (lane == 0) atomicExch(dg.status, (int)EI_ERR_TIMEOUT);
            if (threadIdx.x == 0)
                for (int i = k; i < issued; ++i)
                    mbar_wait_bounded(smem_addr(&bars[i % STG_NS]), (unsigned)(i / STG_NS) & 1u,
                                      kStageWaitNs);
        }
    } else if (O_lo <= O_hi) {
        // mixed row- and column-first angles, or a window too wide: global loads
        const int64_t off = si.pp_off + 1;
        const float4 *gA = an.col_dom ? xtA : xpA;
        const float2 *gB = an.col_dom ? xtB : xpB;
#pragma unroll
        for (int t = 0; t < STG_RPT; ++t) {
            if (lo[t] > n) continue;
            RaySetup rs{pos[t], p1, lo[t], lo[t] + span[t]};
            ray_rows<4, LINKED>(rs, rs.o_lo, rs.o_hi, gA + off, gB + off, w, acc[t], dg.status);
        }
    }

    if (!a_ok) return;
    const int64_t plane = (int64_t)si.n_theta * si.n_dp;
    const float nan = __int_as_float(0x7fc00000);
#pragma unroll
    for (int t = 0; t < STG_RPT; ++t) {
        const int j = j0 + 4 * t;
        if (j >= si.n_dp) continue;
        float *out = proj + si.proj_off + (int64_t)a * si.n_dp + j;
        if (j >= si.n_det || failed) {
            const float v = failed ? nan : 0.f;
            out[0] = v;
            out[plane] = v;
            out[2 * plane] = v;
        } else {
            ray_store<LINKED>(out, plane, acc[t], an.pch, link);
        }
    }
}

template <bool LINKED>
static cudaError_t launch_project_staged(const ei_geometry *g, float *proj, float link,
                                         const int *active, cudaStream_t st)
{
    const FwdVariant &v = g->fwd_variant;
    if (v.total == 0) return cudaSuccess;
    k_project_staged<LINKED><<<v.total, STG_THREADS, StageLayout<LINKED>::kBytes, st>>>(
        g->dg, v.prefix, g->xpA, g->xpB, g->xtA, g->xtB, proj, link, active);
    return cudaGetLastError();
}

// Raises the staged projector's dynamic shared-memory limit (once per device
// context, before its first launch).
cudaError_t project_set_smem_limit()
{
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    EI_CUDA_TRY(cudaFuncSetAttribute(k_project_staged<false>, a, StageLayout<false>::kBytes));
    EI_CUDA_TRY(cudaFuncSetAttribute(k_project_staged<true>, a, StageLayout<true>::kBytes));
    return cudaSuccess;
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
    case 12: return launch_project_variant<8, 32, 4, 4, true, 2>(g, proj, link, active, st);
    // rows staged in shared memory (one block per item in every launch mode)
    default:
        return link > 0.f ? launch_project_staged<true>(g, proj, link, active, st)
                          : launch_project_staged<false>(g, proj, 0.f, active, st);
    }
}

// Tile shape (rays, angles) of projector variant `id` (see launch_project).
void project_variant_shape(int id, int *rays, int *angles)
{
    static const int R[N_FWD_VARIANTS] = {16, 32, 32, 16, 32, 16, 32, 16, 8, 32, 16, 8, 8, STG_RAYS},
                     A[N_FWD_VARIANTS] = {16, 8, 16, 16, 8, 16, 16, 16, 32, 8, 16, 32, 32, STG_ANGLES};
    *rays = R[id];
    *angles = A[id];
}

}  // namespace ei
