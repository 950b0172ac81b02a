// Batched L-BFGS for the cost S of Eq. 5 (the paper minimises S with SciPy's
// L-BFGS, [Byrd 1995]); every slice is an independent problem with its own
// memory, step length and stop test.
//
// Per slice k, in the solver's scaled variables u = x / scale:
//   1. d = -H g: two-loop recursion over the kept (s_i, y_i) pairs, newest
//      first then oldest first, H0 = (s.y / y.y) I of the newest pair, run
//      on coefficients (below);
//   2. Armijo backtracking: alpha0 = 1/|g| while no pair is kept, else 1;
//      accept when S(u + alpha d) <= S(u) + c1 alpha g.d, else halve;
//   3. s = alpha d, y = g_new - g; keep the pair when s.y > eps |s| |y|;
//   4. stop when (f - f_new) / max(|f|, |f_new|, 1) < tol or after max_iter.
//
// Execution: one "round" per host iteration = direction for the slices that
// need one, one trial step + objective evaluation for every slice in line
// search, Armijo test, the gradient and the memory update of accepted slices.
// All per-slice decisions are taken on the device by one-thread-per-slice
// scalar kernels; the host reads back one summary word per round to stop.
//
// Radon calls per iteration (the paper removes superfluous ones, "Algorithmic
// improvements"): R is linear, so along a search direction the projection of
// a trial u + alpha d is P(u) + alpha P(d).  The solver keeps per slice Pu,
// the projections at the current iterate, and Pt, those at the latest trial:
// the first trial of an iteration is projected (prep + projector), and every
// backtracking trial takes Pt <- Pu + (alpha / alpha_prev) (Pt - Pu), a
// sinogram axpy, so the cost of a rejected trial is the IC kernel alone.  The
// regulariser's value is summed by the trial-point kernel, and the adjoint
// (the gradient) runs only for slices whose trial was accepted; Pu <- Pt then.
// Each iteration's first trial is a fresh projection, so no rounding drift
// accumulates in Pu across iterations.
//
// The two-loop recursion runs on coefficients, not on vectors: d is a
// combination of the basis b = (s_i, y_i of the kept pairs, g), and every
// dot product the recursion takes (s_i . q, y_i . r) is one of the basis'
// Gram matrix, kept per slice in FP64 (2 ring + 1 rows).  An accepted step
// adds one pass over the kept pairs: the new pair's dot products with them
// and with itself; the new gradient's entries follow (g_new = g + y).  Forming
// d from its coefficients is one more pass.  (A vector two-loop reads and
// writes ~4 vectors per pair and direction, ~90 vector passes per iteration
// with ten pairs; this takes ~45.)
//
// Vectors are the batched vol layout (float4 per voxel, pad lane kept at 0);
// vector kernels work on VEC_BLK-element blocks that each belong to one slice
// and write FP64 partial dot products per block.  With Eq. 4's offsets
// among the unknowns, every vector continues after the volumes with one
// offsets segment per slice (m_o(theta) then m_r(t), scaled by 1/off_scale,
// three values per float4), whose blocks belong to their slice too.  A consumer block sums its
// slice's partials itself in a fixed order (deterministic, no atomics); the
// partial buffers alternate between launches so no kernel reads what it writes.
#include <math.h>

#include <algorithm>
#include <chrono>
#include <vector>

#include "ei_internal.h"
#include "lib_alloc.h"

namespace ei {

struct SliceState {
    double f, f_t, gd, gg, alpha, gamma, f0;   // gamma: H0 scaling of the last direction
    double alpha_p;             // the step of the trial whose projections Pt holds
    double ratio;               // backtracking trial: alpha / alpha_p of the previous trial
    int k, count, head, trials;
    int status, converged, reset, evals;
    int projections, adjoints;  // projector and adjoint evaluations of the slice
    int pad_;
};

struct Solver {
    int m = 0, ring = 0;
    int64_t vol_count = 0;              // vector length in float4 (volumes + offsets)
    int off_which = 0;                  // offsets among the unknowns (EI_OFFSET_* bits)
    DevGeom dgx{};                      // solver view of the geometry (extended blocks)
    float *shift = nullptr;             // [sino pixels] dS/dshift (offsets mode)
    double *row_sum = nullptr;          // [rows]
    float4 *u = nullptr, *g = nullptr, *d = nullptr, *xt = nullptr, *gt = nullptr;
    float4 *Sr = nullptr, *Yr = nullptr;    // rings of `ring` slots
    float *Pu = nullptr, *Pt = nullptr;     // proj layout: projections of u and of the trial
    double *part_reg = nullptr;             // [solver blocks] regulariser partial sums
    double *part_gd = nullptr;              // [solver blocks] g . d partial sums
    float *meas_stage = nullptr;            // device copy of host s_exp
    float4 *vol_stage = nullptr;            // device copy of host x0 / solution
    double *part_dots = nullptr;            // [solver blocks][KD] partial dot products
    double *gram = nullptr;                 // [S][GD][GD] basis Gram matrix per slice
    double *coef = nullptr;                 // [S][GD] d's coefficients on the basis
    SliceState *st = nullptr;               // [S]
    int *mask_dir = nullptr, *mask_ls = nullptr, *mask_acc = nullptr;
    int *mask_first = nullptr, *mask_bt = nullptr;   // trial projected / interpolated
    int *summary = nullptr;                 // [2]: slices still running, slices in line search
    int *summary_h = nullptr;               // pinned host copy
    cudaStream_t stream = nullptr;          // the solver's own stream (capturable)
    bool has_state = false;                 // a completed solve (or a loaded checkpoint)
    std::vector<void *> allocs;
};

struct SolverDev {
    float4 *u, *g, *d, *xt, *gt, *Sr, *Yr;
    int64_t vol_count;
    int m, ring;
    double *gram, *coef, *part_dots;
    SliceState *st;
    int *mask_dir, *mask_ls, *mask_acc, *mask_first, *mask_bt;
};

// Basis of the coefficient two-loop: s of ring slot i is index i, y of slot i
// is ring + i, the gradient g is 2 ring; GD = 2 ring + 1 indices.  Partial
// dot products per vector block of an accepted step: KD = 4 ring + 5 (per
// kept slot i: s . s_i, s . y_i, y . s_i, y . y_i at 4 i .. 4 i + 3; then
// s . s, s . y, y . y, g_old . s, g_old . y).
__host__ __device__ __forceinline__ int basis_dim(int ring) { return 2 * ring + 1; }
__host__ __device__ __forceinline__ int dots_per_block(int ring) { return 4 * ring + 5; }

static SolverDev dev_view(const Solver *s)
{
    return SolverDev{s->u,  s->g,  s->d,   s->xt,     s->gt,      s->Sr,   s->Yr,
                     s->vol_count, s->m, s->ring, s->gram, s->coef, s->part_dots, s->st,
                     s->mask_dir, s->mask_ls, s->mask_acc, s->mask_first, s->mask_bt};
}

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------
struct VecBlock {
    int s;            // slice
    int64_t begin;    // first float4 (batched vol layout)
    int64_t end;      // one past the last
    bool off;         // a block of the slice's offsets segment (not voxels)
};

__device__ __forceinline__ VecBlock vec_block(const DevGeom &dg)
{
    VecBlock b;
    b.s = find_slice(dg.vec_prefix, dg.n_slices, blockIdx.x);
    const SliceInfo &si = dg.slices[b.s];
    const int64_t nvox = (int64_t)si.n * si.n;
    int64_t lb = blockIdx.x - dg.vec_prefix[b.s];
    if (dg.vec_nvb && lb >= dg.vec_nvb[b.s]) {        // a block of the slice's offsets segment
        lb -= dg.vec_nvb[b.s];
        b.begin = dg.off_start[b.s] + lb * VEC_BLK;
        b.end = dg.off_start[b.s] + min((int64_t)dg.off_len[b.s], (lb + 1) * (int64_t)VEC_BLK);
        b.off = true;
        return b;
    }
    b.off = false;
    b.begin = si.vol_off + lb * VEC_BLK;
    b.end = si.vol_off + min(nvox, (lb + 1) * (int64_t)VEC_BLK);
    return b;
}

__device__ __forceinline__ double dot3(float4 a, float4 b)
{
    return (double)(a.x * b.x + a.y * b.y + a.z * b.z);
}

// Block-wide sum, result broadcast to every thread.
__device__ double block_allsum(double v, double *red)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        double t = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (lane == 0) red[0] = t;
    }
    __syncthreads();
    return red[0];
}

// Sum of a slice's per-block partials, fixed order, broadcast to the block.
__device__ double slice_partials(const DevGeom &dg, const double *part, int s, double *red)
{
    double acc = 0.0;
    for (int b = dg.vec_prefix[s] + threadIdx.x; b < dg.vec_prefix[s + 1]; b += blockDim.x)
        acc += part[b];
    return block_allsum(acc, red);
}

__device__ __forceinline__ int slot_of(const SolverDev &sv, int s, int i)
{
    const int h = sv.st[s].head;
    return ((h - 1 - i) % sv.ring + sv.ring) % sv.ring;
}

__device__ __forceinline__ float4 f4(float x, float y, float z) { return make_float4(x, y, z, 0.f); }

// One voxel's regulariser term sum_c reg1_c x_c^2 (Eq. 5) in FP64; a lane
// with a zero weight (the delta and sigma lanes of the linked unknown) adds
// nothing, whatever it holds.
__device__ __forceinline__ double reg_term(float4 x, float4 reg1)
{
    double r = (double)(reg1.x * x.x * x.x);
    if (reg1.y != 0.f) r += (double)(reg1.y * x.y * x.y);
    if (reg1.z != 0.f) r += (double)(reg1.z * x.z * x.z);
    return r;
}

// The regulariser's value per vector block (0 for an offsets block).
__global__ void k_reg_partials(DevGeom dg, const float4 *__restrict__ v, float4 reg1,
                               double *__restrict__ part, const int *__restrict__ active)
{
    __shared__ double red[32];
    const VecBlock b = vec_block(dg);
    if (active && !active[b.s]) return;
    double acc = 0.0;
    if (!b.off)
        for (int64_t i = b.begin + threadIdx.x; i < b.end; i += blockDim.x) acc += reg_term(v[i], reg1);
    const double t = block_allsum(acc, red);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t launch_reg_partials(const DevGeom &dg, const float4 *v, float4 reg1, double *part,
                                const int *active, cudaStream_t st)
{
    if (dg.total_vec == 0) return cudaSuccess;
    k_reg_partials<<<dg.total_vec, VEC_THREADS, 0, st>>>(dg, v, reg1, part, active);
    return cudaGetLastError();
}

// Sinogram rows of the trial projections Pt (one block per row (slice, angle),
// all three planes; slices with mask[s], all when null):
//   k_sino_backtrack: Pt = Pu + ratio (Pt - Pu), the projections of
//     u + alpha d from those of u and of u + alpha_p d (R is linear);
//   k_sino_commit:    Pu = Pt (the trial was accepted).
template <bool COMMIT>
__global__ void k_sino_rows(DevGeom dg, SolverDev sv, float *__restrict__ Pu,
                            float *__restrict__ Pt, const int *__restrict__ mask)
{
    const int row = blockIdx.x;
    const int s = find_slice(dg.ic_prefix, dg.n_slices, row);
    if (mask && !mask[s]) return;
    const SliceInfo si = dg.slices[s];
    const int a = row - dg.ic_prefix[s];
    const float r = COMMIT ? 0.f : (float)sv.st[s].ratio;
    const int64_t plane = (int64_t)si.n_theta * si.n_dp;
    const int nq = si.n_dp >> 2;
    for (int c = 0; c < 3; ++c) {
        // rows start on 16-byte boundaries (n_dp and every offset are multiples of 4)
        float4 *u4 = reinterpret_cast<float4 *>(Pu + si.proj_off + c * plane + (int64_t)a * si.n_dp);
        float4 *t4 = reinterpret_cast<float4 *>(Pt + si.proj_off + c * plane + (int64_t)a * si.n_dp);
        for (int i = threadIdx.x; i < nq; i += blockDim.x) {
            const float4 pt = t4[i];
            if (COMMIT) {
                u4[i] = pt;
            } else {
                const float4 pu = u4[i];
                t4[i] = make_float4(fmaf(r, pt.x - pu.x, pu.x), fmaf(r, pt.y - pu.y, pu.y),
                                    fmaf(r, pt.z - pu.z, pu.z), fmaf(r, pt.w - pu.w, pu.w));
            }
        }
    }
}

// --------------------------------------------------------------------------
// vector kernels
// --------------------------------------------------------------------------
// u = x0 / scale (x0 in vol layout)
__global__ void k_to_scaled(DevGeom dg, const float4 *__restrict__ x0, float4 *__restrict__ u, float4 inv)
{
    const VecBlock b = vec_block(dg);
    for (int64_t i = b.begin + threadIdx.x; i < b.end; i += blockDim.x) {
        const float4 x = x0[i];
        // a zero factor clears its lane (linked mode ignores the delta and sigma lanes)
        u[i] = f4(x.x * inv.x, inv.y != 0.f ? x.y * inv.y : 0.f, inv.z != 0.f ? x.z * inv.z : 0.f);
    }
}

// x = u * scale
__global__ void k_from_scaled(DevGeom dg, const float4 *__restrict__ u, float4 *__restrict__ x, float4 sc)
{
    const VecBlock b = vec_block(dg);
    for (int64_t i = b.begin + threadIdx.x; i < b.end; i += blockDim.x) {
        const float4 v = u[i];
        x[i] = f4(v.x * sc.x, v.y * sc.y, v.z * sc.z);
    }
}

// --------------------------------------------------------------------------
// Eq. 4's offsets among the unknowns.  Offsets segment of slice s: element k
// (k < n_mo: m_o of angle k; then m_r of pixel k - n_mo) is lane k % 3 of
// float4 k / 3 from off_start[s].  One block per slice.
// --------------------------------------------------------------------------
__device__ __forceinline__ float &off_elem(float4 *v, int64_t start, int k)
{
    return reinterpret_cast<float *>(v + start + k / 3)[k % 3];
}

// u's offsets segments from the geometry's current m_o / m_r tables
__global__ void k_offsets_to_u(DevGeom dg, int which, float inv_scale, float4 *__restrict__ u)
{
    const int s = blockIdx.x;
    const SliceInfo si = dg.slices[s];
    const int n_mo = (which & EI_OFFSET_MO) ? si.n_theta : 0;
    const int n_mr = (which & EI_OFFSET_MR) ? si.n_det : 0;
    const int64_t st = dg.off_start[s];
    for (int i = threadIdx.x; i < dg.off_len[s]; i += blockDim.x) u[st + i] = f4(0.f, 0.f, 0.f);
    __syncthreads();
    for (int k = threadIdx.x; k < n_mo + n_mr; k += blockDim.x)
        off_elem(u, st, k) = (k < n_mo ? dg.m_o[si.ang_off + k] : dg.pix[si.pix_off + k - n_mo].w) *
                             inv_scale;
}

// the geometry's m_o / m_r tables from the offsets segments of v (slices with
// active[s], all when null): the model then evaluates at v's offsets
__global__ void k_offsets_apply(DevGeom dg, int which, float scale, const float4 *__restrict__ v,
                                const int *__restrict__ active)
{
    const int s = blockIdx.x;
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n_mo = (which & EI_OFFSET_MO) ? si.n_theta : 0;
    const int n_mr = (which & EI_OFFSET_MR) ? si.n_det : 0;
    float *m_o = const_cast<float *>(dg.m_o);
    float4 *pix = const_cast<float4 *>(dg.pix);
    float4 *vv = const_cast<float4 *>(v);
    for (int k = threadIdx.x; k < n_mo + n_mr; k += blockDim.x) {
        const float val = off_elem(vv, dg.off_start[s], k) * scale;
        if (k < n_mo) m_o[si.ang_off + k] = val;
        else pix[si.pix_off + k - n_mo].w = val;
    }
}

// Orthonormal DCT-II vector k of length n at j (the ring-mode basis).
__device__ __forceinline__ double dct2_basis(int k, int j, int n)
{
    return sqrt((k == 0 ? 1.0 : 2.0) / n) * cospi((double)k * (j + 0.5) / n);
}

// the offsets segments of the gradient gv: scale * dS/dm_o (row sums of
// dS/dshift) and scale * dS/dm_r (FP64 sums over the slice's angles in
// order).  The latter is then restricted to ring frequencies, minus its
// components along the ring_k lowest DCT-II modes (FP64 sums in a fixed
// order), or with ring_k = 0 and both offsets unknowns minus its mean over
// the slice (the gauge (m_o + a, m_r - a) leaves S unchanged, so the
// iteration keeps the mean of m_r fixed).
__global__ void k_offsets_grad(DevGeom dg, int which, int ring_k, float scale,
                               const float *__restrict__ shift, const double *__restrict__ row_sum,
                               float4 *__restrict__ gv, const int *__restrict__ active)
{
    __shared__ double red[32];
    __shared__ double coef[EI_MAX_RING_MODES];
    const int s = blockIdx.x;
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n_mo = (which & EI_OFFSET_MO) ? si.n_theta : 0;
    const int n_mr = (which & EI_OFFSET_MR) ? si.n_det : 0;
    const int64_t st = dg.off_start[s];
    const int r0 = dg.ic_prefix[s];
    for (int a = threadIdx.x; a < n_mo; a += blockDim.x)
        off_elem(gv, st, a) = (float)(row_sum[r0 + a] * scale);
    if (n_mr == 0) return;
    double part = 0.0;
    for (int j = threadIdx.x; j < n_mr; j += blockDim.x) {
        double acc = 0.0;
        for (int a = 0; a < si.n_theta; ++a) acc += (double)shift[si.sino_off + (int64_t)a * si.n_dp + j];
        off_elem(gv, st, n_mo + j) = (float)acc;     // unscaled for now
        part += acc;
    }
    if (ring_k > 0) {
        __syncthreads();                             // every column sum is in place
        for (int k = threadIdx.x; k < ring_k; k += blockDim.x) {
            double c = 0.0;
            for (int j = 0; j < n_mr; ++j) c += (double)off_elem(gv, st, n_mo + j) * dct2_basis(k, j, n_mr);
            coef[k] = c;
        }
        __syncthreads();
        for (int j = threadIdx.x; j < n_mr; j += blockDim.x) {
            float &e = off_elem(gv, st, n_mo + j);
            double r = (double)e;
            for (int k = 0; k < ring_k; ++k) r -= coef[k] * dct2_basis(k, j, n_mr);
            e = (float)(r * scale);
        }
        return;
    }
    // fixed-order block reduction of the column sums
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = part;
    __syncthreads();
    if (threadIdx.x < 32) {
        double t = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) red[0] = t;
    }
    __syncthreads();
    const double mean = n_mo > 0 ? red[0] / n_mr : 0.0;
    for (int j = threadIdx.x; j < n_mr; j += blockDim.x) {
        float &e = off_elem(gv, st, n_mo + j);
        e = (float)(((double)e - mean) * scale);
    }
}

// g . g per block after the initial evaluation (the Gram matrix's first entry)
__global__ void k_gram_gg(DevGeom dg, SolverDev sv)
{
    __shared__ double red[32];
    const VecBlock b = vec_block(dg);
    double acc = 0.0;
    for (int64_t e = b.begin + threadIdx.x; e < b.end; e += blockDim.x) {
        const float4 gv = sv.g[e];
        acc += dot3(gv, gv);
    }
    const double t = block_allsum(acc, red);
    if (threadIdx.x == 0) sv.part_dots[(int64_t)blockIdx.x * dots_per_block(sv.ring)] = t;
}

// trial point xt = u + alpha d, and the regulariser's value at it (part_reg);
// an iteration's first trial first forms d = sum_j coef_j b_j over the basis
// (the kept pairs' s and y, and g) and its slope g . d (part_gd), which the
// Armijo test takes from the d it steps along
__global__ void k_trial(DevGeom dg, SolverDev sv, float4 reg1, double *__restrict__ part_reg,
                        double *__restrict__ part_gd)
{
    __shared__ double red[32];
    __shared__ float cS[EI_MAX_LBFGS_M + 1], cY[EI_MAX_LBFGS_M + 1];
    __shared__ int slots[EI_MAX_LBFGS_M + 1];
    const VecBlock b = vec_block(dg);
    const int s = b.s;
    if (!sv.mask_ls[s]) return;
    const SliceState &q = sv.st[s];
    const float al = (float)q.alpha;
    const bool first = q.trials == 0;
    const int cnt = q.count, R = sv.ring, GD = basis_dim(R);
    const double *co = sv.coef + (int64_t)s * GD;
    if (first && (int)threadIdx.x < cnt) {
        const int sl = slot_of(sv, s, threadIdx.x);
        slots[threadIdx.x] = sl;
        cS[threadIdx.x] = (float)co[sl];
        cY[threadIdx.x] = (float)co[R + sl];
    }
    const float cg = (float)co[2 * R];
    __syncthreads();
    double acc = 0.0, gd = 0.0;
    for (int64_t e = b.begin + threadIdx.x; e < b.end; e += blockDim.x) {
        float4 dv;
        if (first) {
            const float4 gv = sv.g[e];
            dv = f4(cg * gv.x, cg * gv.y, cg * gv.z);
            for (int k = 0; k < cnt; ++k) {
                const int64_t off = (int64_t)slots[k] * sv.vol_count + e;
                const float4 sv4 = sv.Sr[off], yv4 = sv.Yr[off];
                dv = f4(fmaf(cS[k], sv4.x, fmaf(cY[k], yv4.x, dv.x)),
                        fmaf(cS[k], sv4.y, fmaf(cY[k], yv4.y, dv.y)),
                        fmaf(cS[k], sv4.z, fmaf(cY[k], yv4.z, dv.z)));
            }
            sv.d[e] = dv;
            gd += dot3(gv, dv);
        } else {
            dv = sv.d[e];
        }
        const float4 uv = sv.u[e];
        const float4 x = f4(fmaf(al, dv.x, uv.x), fmaf(al, dv.y, uv.y), fmaf(al, dv.z, uv.z));
        sv.xt[e] = x;
        if (!b.off) acc += reg_term(x, reg1);
    }
    const double t = block_allsum(acc, red);
    if (threadIdx.x == 0) part_reg[blockIdx.x] = t;
    if (first) {
        const double tg = block_allsum(gd, red);
        if (threadIdx.x == 0) part_gd[blockIdx.x] = tg;
    }
}

// A dot product accumulated by one thread: FP32 over chunks of 4 elements
// (12 products), FP64 across chunks.  FP64 runs at a small fraction of the
// FP32 rate on this GPU; chunks of 4 keep the rounding within ~2x that of an
// FP64 sum of per-element FP32 dots.
struct ChunkedDot {
    double total = 0.0;
    float chunk = 0.f;
    __device__ __forceinline__ void add(float4 a, float4 b, int e_count)
    {
        chunk = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, chunk)));
        if ((e_count & 3) == 3) total += (double)chunk, chunk = 0.f;
    }
    __device__ __forceinline__ double value() const { return total + (double)chunk; }
};

// accepted step: S_head = s = xt - u, Y_head = y = gt - g, u = xt, g = gt; and
// the new pair's dot products with the kept pairs (before this update), with
// itself and with the old gradient, per block (ChunkedDot per thread, FP64
// across threads): part_dots[block] = (s . s_i, s . y_i, y . s_i, y . y_i at
// 4 i; s . s, s . y, y . y, g_old . s, g_old . y at 4 ring).  Taken directly
// from s and y, so a small y near convergence loses no precision.
__global__ void k_accept(DevGeom dg, SolverDev sv)
{
    __shared__ double red[32];
    const VecBlock b = vec_block(dg);
    const int s = b.s;
    if (!sv.mask_acc[s]) return;
    const int head = sv.st[s].head, cnt = sv.st[s].count, R = sv.ring;
    double *out = sv.part_dots + (int64_t)blockIdx.x * dots_per_block(R);
    float4 *Sv = sv.Sr + (int64_t)head * sv.vol_count;
    float4 *Yv = sv.Yr + (int64_t)head * sv.vol_count;
    ChunkedDot a_ss, a_sy, a_yy, a_gs, a_gy;
    int ec = 0;
    for (int64_t e = b.begin + threadIdx.x; e < b.end; e += blockDim.x, ++ec) {
        const float4 x = sv.xt[e], uv = sv.u[e], gn = sv.gt[e], go = sv.g[e];
        const float4 sd = f4(x.x - uv.x, x.y - uv.y, x.z - uv.z);
        const float4 yd = f4(gn.x - go.x, gn.y - go.y, gn.z - go.z);
        Sv[e] = sd;
        Yv[e] = yd;
        sv.u[e] = x;
        sv.g[e] = gn;
        a_ss.add(sd, sd, ec);
        a_sy.add(sd, yd, ec);
        a_yy.add(yd, yd, ec);
        a_gs.add(go, sd, ec);
        a_gy.add(go, yd, ec);
    }
    const double tail[5] = {a_ss.value(), a_sy.value(), a_yy.value(), a_gs.value(), a_gy.value()};
    for (int j = 0; j < 5; ++j) {
        const double t = block_allsum(tail[j], red);
        if (threadIdx.x == 0) out[4 * R + j] = t;
    }
    for (int k = 0; k < cnt; ++k) {           // the kept pairs (head is never one of them)
        const int sl = slot_of(sv, s, k);
        const float4 *Sk = sv.Sr + (int64_t)sl * sv.vol_count;
        const float4 *Yk = sv.Yr + (int64_t)sl * sv.vol_count;
        ChunkedDot a0, a1, a2, a3;
        int ek = 0;
        for (int64_t e = b.begin + threadIdx.x; e < b.end; e += blockDim.x, ++ek) {
            const float4 sd = Sv[e], yd = Yv[e], sk = Sk[e], yk = Yk[e];
            a0.add(sd, sk, ek);
            a1.add(sd, yk, ek);
            a2.add(yd, sk, ek);
            a3.add(yd, yk, ek);
        }
        const double four[4] = {a0.value(), a1.value(), a2.value(), a3.value()};
        for (int j = 0; j < 4; ++j) {
            const double t = block_allsum(four[j], red);
            if (threadIdx.x == 0) out[4 * sl + j] = t;
        }
    }
}

// --------------------------------------------------------------------------
// scalar kernels (one block, one thread per slice)
// --------------------------------------------------------------------------
struct Opts {
    double tol, c1, curv_eps;
    int max_iter, max_trials;
};

// Sum over a slice's vector blocks of entry k of their partials (stride KD),
// in block order.
__device__ double serial_sum(const DevGeom &dg, const double *part, int stride, int k, int s)
{
    double acc = 0.0;
    for (int b = dg.vec_prefix[s]; b < dg.vec_prefix[s + 1]; ++b) acc += part[(int64_t)b * stride + k];
    return acc;
}

// initial evaluation done: f0 = S, state reset, Gram matrix (g . g only)
__global__ void k_init_state(DevGeom dg, SolverDev sv, const double *__restrict__ S, int *summary)
{
    int running = 0;
    const int R = sv.ring, GD = basis_dim(R), KD = dots_per_block(R);
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        SliceState &q = sv.st[s];
        q = SliceState{};
        double *G = sv.gram + (int64_t)s * GD * GD;
        G[2 * R * GD + 2 * R] = serial_sum(dg, sv.part_dots, KD, 0, s);
        q.f = q.f0 = S[s];
        q.gamma = 1.0;
        q.evals = 1;
        q.projections = 1;
        q.adjoints = 1;
        const bool ok = isfinite(q.f);
        q.status = ok ? EI_OK : EI_ERR_NONFINITE;
        sv.mask_dir[s] = ok;
        sv.mask_ls[s] = 0;
        sv.mask_acc[s] = 0;
        running += ok;
    }
    __shared__ int acc;
    if (threadIdx.x == 0) acc = 0;
    __syncthreads();
    atomicAdd(&acc, running);
    __syncthreads();
    if (threadIdx.x == 0) summary[0] = acc, summary[1] = 0;
}

// resume from a kept or loaded state: slices that stopped at max_iter (between
// steps, not converged, no error) need a direction again under the new limit
__global__ void k_resume_state(DevGeom dg, SolverDev sv, int max_iter, int *summary)
{
    int running = 0, in_ls = 0;
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        const SliceState &q = sv.st[s];
        sv.mask_acc[s] = 0;
        if (q.status == EI_OK && !q.converged && !sv.mask_ls[s] && q.k < max_iter)
            sv.mask_dir[s] = 1;
        running += sv.mask_dir[s] | sv.mask_ls[s];
        in_ls += sv.mask_ls[s];
    }
    __shared__ int a0, a1;
    if (threadIdx.x == 0) a0 = 0, a1 = 0;
    __syncthreads();
    atomicAdd(&a0, running);
    atomicAdd(&a1, in_ls);
    __syncthreads();
    if (threadIdx.x == 0) summary[0] = a0, summary[1] = a1;
}

// The two-loop recursion on coefficients (one thread per slice in line for a
// direction): q = g; newest pair first a_i = rho_i s_i . q, q -= a_i y_i;
// r = gamma q (gamma = s.y / y.y of the newest pair, 1 without pairs); oldest
// first beta = rho_i y_i . r, r += (a_i - beta) s_i; d = -r.  Every dot
// product is a row of the Gram matrix applied to coefficients.  Then the
// first trial step, as before: alpha0 = 1/|g| without pairs, else 1; a
// direction that is not a descent one restarts from -g.
__global__ void k_ls_start(DevGeom dg, SolverDev sv)
{
    const int R = sv.ring, GD = basis_dim(R), IG = 2 * R;
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        SliceState &q = sv.st[s];
        q.reset = 0;
        if (!sv.mask_dir[s]) continue;
        sv.mask_dir[s] = 0;
        const double *G = sv.gram + (int64_t)s * GD * GD;
        double *c = sv.coef + (int64_t)s * GD;
        for (int j = 0; j < GD; ++j) c[j] = 0.0;
        const int cnt = q.count;
        int sl[EI_MAX_LBFGS_M];
        for (int k = 0; k < cnt; ++k) sl[k] = slot_of(sv, s, k);
        // (G row a) . c over the basis indices in use: the kept pairs and g
        auto row_dot = [&](int a) {
            double t = G[(int64_t)a * GD + IG] * c[IG];
            for (int k = 0; k < cnt; ++k)
                t += G[(int64_t)a * GD + sl[k]] * c[sl[k]] + G[(int64_t)a * GD + R + sl[k]] * c[R + sl[k]];
            return t;
        };
        double al[EI_MAX_LBFGS_M];
        c[IG] = 1.0;                                             // q = g
        for (int k = 0; k < cnt; ++k) {                          // newest first
            const int i = sl[k];
            const double rho = 1.0 / G[(int64_t)i * GD + R + i];
            al[k] = rho * row_dot(i);
            c[R + i] -= al[k];
        }
        double gam = 1.0;
        if (cnt > 0) {
            const int n = sl[0];
            gam = G[(int64_t)n * GD + R + n] / G[(int64_t)(R + n) * GD + R + n];
        }
        for (int j = 0; j < GD; ++j) c[j] *= gam;                // r = gamma q
        for (int k = cnt - 1; k >= 0; --k) {                     // oldest first
            const int i = sl[k];
            const double rho = 1.0 / G[(int64_t)i * GD + R + i];
            const double beta = rho * row_dot(R + i);
            c[i] += al[k] - beta;
        }
        for (int j = 0; j < GD; ++j) c[j] = -c[j];               // d = -r
        q.gamma = gam;
        const double gd = row_dot(IG), gg = G[(int64_t)IG * GD + IG];
        q.gg = gg;
        q.gd = gd;
        if (!(gd < 0.0)) {
            if (!(gg > 0.0)) {            // zero gradient: stationary point
                q.converged = 1;
                continue;
            }
            q.reset = 1;                  // not a descent direction: restart from -g
            q.count = 0;
            for (int j = 0; j < GD; ++j) c[j] = 0.0;
            c[IG] = -1.0;
            q.gd = -gg;
        }
        q.alpha = q.count == 0 ? 1.0 / sqrt(gg) : 1.0;
        q.trials = 0;
        sv.mask_ls[s] = 1;
    }
    // the trial of every slice in line search in the current solver round: an
    // iteration's first trial is projected, a backtracking one interpolated
    // from Pu and Pt
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        sv.mask_first[s] = 0;
        sv.mask_bt[s] = 0;
        if (!sv.mask_ls[s]) continue;
        SliceState &q = sv.st[s];
        if (q.trials == 0) {
            sv.mask_first[s] = 1;
            q.projections += 1;
        } else {
            sv.mask_bt[s] = 1;
            q.ratio = q.alpha / q.alpha_p;
        }
        q.alpha_p = q.alpha;
    }
}

// Armijo test of the trial point; at an iteration's first trial the slope
// g . d comes from the d the trial stepped along (part_gd)
__global__ void k_armijo(DevGeom dg, SolverDev sv, const double *__restrict__ S,
                         const double *__restrict__ part_gd, Opts o)
{
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        if (!sv.mask_ls[s]) continue;
        SliceState &q = sv.st[s];
        if (q.trials == 0) q.gd = serial_sum(dg, part_gd, 1, 0, s);
        const double ft = S[s];
        q.evals += 1;
        if (isfinite(ft) && ft <= q.f + o.c1 * q.alpha * q.gd) {
            q.f_t = ft;
            q.adjoints += 1;
            sv.mask_ls[s] = 0;
            sv.mask_acc[s] = 1;
        } else {
            q.alpha *= 0.5;
            if (++q.trials >= o.max_trials) {
                q.status = EI_ERR_LINESEARCH;
                sv.mask_ls[s] = 0;
            }
        }
    }
}

// Memory and Gram update and stop test of accepted slices; summary of what
// still runs.  The new pair (s, y) has its dot products with the kept pairs
// and with itself from the accepted step's pass; the new gradient
// g_new = g + y has g_new . b = g . b + y . b (g . b: the old gradient column)
// and g_new . g_new = g . g + 2 g . y + y . y.  The pair is kept when
// s.y > eps |s| |y|.
__global__ void k_update(DevGeom dg, SolverDev sv, Opts o, int *summary)
{
    int running = 0, in_ls = 0;
    const int R = sv.ring, GD = basis_dim(R), KD = dots_per_block(R), IG = 2 * R;
    for (int s = threadIdx.x; s < dg.n_slices; s += blockDim.x) {
        SliceState &q = sv.st[s];
        if (sv.mask_acc[s]) {
            sv.mask_acc[s] = 0;
            double *G = sv.gram + (int64_t)s * GD * GD;
            const int cnt = q.count, h = q.head;
            const double s_s = serial_sum(dg, sv.part_dots, KD, 4 * R, s);
            const double s_y = serial_sum(dg, sv.part_dots, KD, 4 * R + 1, s);
            const double y_y = serial_sum(dg, sv.part_dots, KD, 4 * R + 2, s);
            const double g_s = serial_sum(dg, sv.part_dots, KD, 4 * R + 3, s);
            const double g_y = serial_sum(dg, sv.part_dots, KD, 4 * R + 4, s);
            const double gn_gn = G[(int64_t)IG * GD + IG] + 2.0 * g_y + y_y;
            const bool keep = s_y > o.curv_eps * sqrt(fmax(s_s, 0.0)) * sqrt(fmax(y_y, 0.0));
            // the old pairs kept after this update (newest first; with the new
            // pair m in all)
            const int kept_old = keep ? min(cnt, sv.m - 1) : cnt;
            for (int k = 0; k < kept_old; ++k) {
                const int j = slot_of(sv, s, k);
                const double yS = serial_sum(dg, sv.part_dots, KD, 4 * j + 2, s);
                const double yY = serial_sum(dg, sv.part_dots, KD, 4 * j + 3, s);
                if (keep) {
                    const double sS = serial_sum(dg, sv.part_dots, KD, 4 * j, s);
                    const double sY = serial_sum(dg, sv.part_dots, KD, 4 * j + 1, s);
                    G[(int64_t)h * GD + j] = G[(int64_t)j * GD + h] = sS;
                    G[(int64_t)h * GD + R + j] = G[(int64_t)(R + j) * GD + h] = sY;
                    G[(int64_t)(R + h) * GD + j] = G[(int64_t)j * GD + R + h] = yS;
                    G[(int64_t)(R + h) * GD + R + j] = G[(int64_t)(R + j) * GD + R + h] = yY;
                }
                // the gradient column: g_new . s_j, g_new . y_j
                const double gS = G[(int64_t)IG * GD + j] + yS, gY = G[(int64_t)IG * GD + R + j] + yY;
                G[(int64_t)j * GD + IG] = G[(int64_t)IG * GD + j] = gS;
                G[(int64_t)(R + j) * GD + IG] = G[(int64_t)IG * GD + R + j] = gY;
            }
            if (keep) {
                G[(int64_t)h * GD + h] = s_s;
                G[(int64_t)h * GD + R + h] = G[(int64_t)(R + h) * GD + h] = s_y;
                G[(int64_t)(R + h) * GD + R + h] = y_y;
                G[(int64_t)h * GD + IG] = G[(int64_t)IG * GD + h] = g_s + s_y;
                G[(int64_t)(R + h) * GD + IG] = G[(int64_t)IG * GD + R + h] = g_y + y_y;
                q.head = (h + 1) % sv.ring;
                q.count = min(cnt + 1, sv.m);
            }
            G[(int64_t)IG * GD + IG] = gn_gn;
            const double rel = (q.f - q.f_t) / fmax(fmax(fabs(q.f), fabs(q.f_t)), 1.0);
            q.f = q.f_t;
            q.k += 1;
            if (rel < o.tol) q.converged = 1;
            else if (q.k < o.max_iter) sv.mask_dir[s] = 1;
        }
        running += sv.mask_dir[s] | sv.mask_ls[s];
        in_ls += sv.mask_ls[s];
    }
    __shared__ int a0, a1;
    if (threadIdx.x == 0) a0 = 0, a1 = 0;
    __syncthreads();
    atomicAdd(&a0, running);
    atomicAdd(&a1, in_ls);
    __syncthreads();
    if (threadIdx.x == 0) summary[0] = a0, summary[1] = a1;
}

// --------------------------------------------------------------------------
// host side: allocation, rounds, checkpoints
// --------------------------------------------------------------------------
template <class T>
static cudaError_t salloc(Solver *s, T **p, size_t count)
{
    void *ptr = nullptr;
    cudaError_t e = lib_malloc(&ptr, std::max<size_t>(count * sizeof(T), 16));
    if (e != cudaSuccess) return e;
    s->allocs.push_back(ptr);
    *p = static_cast<T *>(ptr);
    return cudaSuccess;
}

void destroy_solver(ei_geometry *g)
{
    if (!g->solver) return;
    for (void *p : g->solver->allocs) lib_free(p);
    if (g->solver->summary_h) cudaFreeHost(g->solver->summary_h);
    if (g->solver->stream) cudaStreamDestroy(g->solver->stream);
    delete g->solver;
    g->solver = nullptr;
}

static cudaError_t ensure_solver(ei_geometry *g, int m)
{
    if (g->solver && g->solver->m == m && g->solver->off_which == g->off_which) return cudaSuccess;
    destroy_solver(g);
    Solver *s = new Solver();
    g->solver = s;
    s->m = m;
    s->ring = m + 1;
    s->off_which = g->off_which;
    s->dgx = g->dg;
    int64_t ext = g->vol_count;
    if (g->off_which) {
        // the offsets segments after the volumes, and the solver's block table
        std::vector<int> prefix(1, 0), nvb, len;
        std::vector<int64_t> start;
        for (int k = 0; k < g->n_slices; ++k) {
            const SliceInfo &si = g->h_slices[k];
            const int nv = g->h_vec_prefix[k + 1] - g->h_vec_prefix[k];
            const int K = ((g->off_which & EI_OFFSET_MO) ? si.n_theta : 0) +
                          ((g->off_which & EI_OFFSET_MR) ? si.n_det : 0);
            const int L = (K + 2) / 3;
            nvb.push_back(nv);
            len.push_back(L);
            start.push_back(ext);
            ext += L;
            prefix.push_back(prefix.back() + nv + (L + VEC_BLK - 1) / VEC_BLK);
        }
        int *d_prefix = nullptr, *d_nvb = nullptr, *d_len = nullptr;
        int64_t *d_start = nullptr;
        EI_CUDA_TRY(salloc(s, &d_prefix, prefix.size()));
        EI_CUDA_TRY(salloc(s, &d_nvb, nvb.size()));
        EI_CUDA_TRY(salloc(s, &d_len, len.size()));
        EI_CUDA_TRY(salloc(s, &d_start, start.size()));
        EI_CUDA_TRY(cudaMemcpy(d_prefix, prefix.data(), prefix.size() * sizeof(int), cudaMemcpyHostToDevice));
        EI_CUDA_TRY(cudaMemcpy(d_nvb, nvb.data(), nvb.size() * sizeof(int), cudaMemcpyHostToDevice));
        EI_CUDA_TRY(cudaMemcpy(d_len, len.data(), len.size() * sizeof(int), cudaMemcpyHostToDevice));
        EI_CUDA_TRY(cudaMemcpy(d_start, start.data(), start.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
        s->dgx.vec_prefix = d_prefix;
        s->dgx.total_vec = prefix.back();
        s->dgx.vec_nvb = d_nvb;
        s->dgx.off_len = d_len;
        s->dgx.off_start = d_start;
        EI_CUDA_TRY(salloc(s, &s->shift, (size_t)g->sino4_count));
        EI_CUDA_TRY(salloc(s, &s->row_sum, (size_t)std::max(1, g->dg.total_ic)));
    }
    s->vol_count = ext;
    const size_t V = (size_t)ext, S = (size_t)g->n_slices;
    const size_t NB = (size_t)s->dgx.total_vec;
    EI_CUDA_TRY(salloc(s, &s->u, V));
    EI_CUDA_TRY(salloc(s, &s->g, V));
    EI_CUDA_TRY(salloc(s, &s->d, V));
    EI_CUDA_TRY(salloc(s, &s->xt, V));
    EI_CUDA_TRY(salloc(s, &s->gt, V));
    EI_CUDA_TRY(salloc(s, &s->Sr, V * s->ring));
    EI_CUDA_TRY(salloc(s, &s->Yr, V * s->ring));
    const size_t GD = (size_t)basis_dim(s->ring), KD = (size_t)dots_per_block(s->ring);
    EI_CUDA_TRY(salloc(s, &s->part_dots, NB * KD));
    EI_CUDA_TRY(salloc(s, &s->gram, S * GD * GD));
    EI_CUDA_TRY(salloc(s, &s->coef, S * GD));
    EI_CUDA_TRY(salloc(s, &s->st, S));
    EI_CUDA_TRY(salloc(s, &s->mask_dir, S));
    EI_CUDA_TRY(salloc(s, &s->mask_ls, S));
    EI_CUDA_TRY(salloc(s, &s->mask_acc, S));
    EI_CUDA_TRY(salloc(s, &s->mask_first, S));
    EI_CUDA_TRY(salloc(s, &s->mask_bt, S));
    EI_CUDA_TRY(salloc(s, &s->Pu, (size_t)g->proj_count));
    EI_CUDA_TRY(salloc(s, &s->Pt, (size_t)g->proj_count));
    EI_CUDA_TRY(salloc(s, &s->part_reg, NB));
    EI_CUDA_TRY(salloc(s, &s->part_gd, NB));
    EI_CUDA_TRY(salloc(s, &s->summary, 2));
    EI_CUDA_TRY(cudaMallocHost(&s->summary_h, 2 * sizeof(int)));
    EI_CUDA_TRY(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
    // pad lanes of every vector stay 0: start from zeroed memory
    EI_CUDA_TRY(cudaMemset(s->u, 0, V * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->g, 0, V * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->xt, 0, V * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->gt, 0, V * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->d, 0, V * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->Sr, 0, V * s->ring * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->Yr, 0, V * s->ring * sizeof(float4)));
    EI_CUDA_TRY(cudaMemset(s->gram, 0, S * GD * GD * sizeof(double)));
    EI_CUDA_TRY(cudaMemset(s->coef, 0, S * GD * sizeof(double)));
    return cudaSuccess;
}

static bool is_device_ptr(const void *p)
{
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Traced launches of the solver's Radon-class and IC kernels (events when
// tracing is on, every launch counted).
static cudaError_t solver_project(ei_geometry *g, float *proj, float link, const int *active,
                                  cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_project(g, proj, link, active, st);
    trace_end(g, TK_PROJECT, b, st);
    count_launches(g, 1);
    return e;
}

static cudaError_t solver_ic(ei_geometry *g, const float *proj, const float *meas, float link,
                             const int *active, cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_ic(g, proj, meas, nullptr, g->part_ic, IC_OBJECTIVE_GRAD, link, active, st);
    trace_end(g, TK_IC, b, st);
    count_launches(g, 1);
    return e;
}

static cudaError_t solver_adjoint(ei_geometry *g, const float4 *v, float4 *out, const EvalConsts &c,
                                  const int *active, cudaStream_t st)
{
    cudaEvent_t b = trace_begin(g, st);
    cudaError_t e = launch_backproject(g, v, out, c.out_mult, c.reg2, c.link, active, st);
    trace_end(g, TK_BACKPROJECT, b, st);
    count_launches(g, 1);
    return e;
}

// deadline: the time budget's end (opts->max_seconds > 0), checked before each
// round; *timed_out tells whether it stopped the rounds
static cudaError_t run_solver(ei_geometry *g, const float *meas, float4 *x_dev,
                              const ei_solve_opts *opts, int *evals, cudaStream_t st,
                              std::chrono::steady_clock::time_point deadline, bool *timed_out)
{
    Solver *sv = g->solver;
    const SolverDev dv = dev_view(sv);
    const DevGeom &dg = sv->dgx;              // the solver's blocks (with offsets segments)
    const int NB = dg.total_vec;
    const int NBv = g->dg.total_vec;          // the volumes' blocks only
    const int NR = g->dg.total_ic;            // sinogram rows
    const int T = VEC_THREADS;
    const int ow = sv->off_which;
    const float os = g->off_scale;
    const EvalConsts ec = eval_consts(g, true);   // the solver's scaled unknowns
    const bool linked = g->link_gamma > 0.f;
    // the gradient's offsets segments at the points whose projections are in Pt
    // (after the model's tables hold their offsets)
    auto offsets_gradient = [&](float4 *gv, const int *active) -> cudaError_t {
        EI_CUDA_TRY(launch_shift_grad(g, sv->Pt, meas, sv->shift, sv->row_sum, active, st));
        k_offsets_grad<<<g->n_slices, 256, 0, st>>>(dg, ow, (ow & EI_OFFSET_MR) ? g->ring_modes : 0,
                                                    os, sv->shift, sv->row_sum, gv, active);
        count_launches(g, 2);
        return cudaGetLastError();
    };
    // linked mode iterates on h alone: the other lanes of u start and stay at 0
    const float on1 = linked ? 0.f : 1.f;
    const float4 inv = make_float4(1.f / g->scale[0], on1 / g->scale[1], on1 / g->scale[2], 0.f);
    const float4 sc = make_float4(g->scale[0], on1 * g->scale[1], on1 * g->scale[2], 0.f);
    Opts o{opts->tol, opts->c1, opts->curv_eps, opts->max_iter, opts->max_trials};
    const int scalar_threads = 256;

    sv->has_state = false;                    // until this solve completes
    if (opts->resume) {
        // continue from the kept state: u, its gradient and projections, the memory,
        // the slices' records
        k_resume_state<<<1, scalar_threads, 0, st>>>(dg, dv, opts->max_iter, sv->summary);
        count_launches(g, 1);
        EI_CUDA_TRY(cudaGetLastError());
        *evals = 0;
    } else {
        NvtxRange init("initial evaluation");
        k_to_scaled<<<NBv, T, 0, st>>>(g->dg, x_dev, sv->u, inv);
        count_launches(g, 1);
        if (ow) {
            k_offsets_to_u<<<g->n_slices, 256, 0, st>>>(dg, ow, 1.f / os, sv->u);
            k_offsets_apply<<<g->n_slices, 256, 0, st>>>(dg, ow, os, sv->u, nullptr);
            count_launches(g, 2);
        }
        EI_CUDA_TRY(cudaGetLastError());
        // the initial evaluation: S, the gradient and the projections Pu at u
        EI_CUDA_TRY(launch_reg_partials(dg, sv->u, ec.reg1, sv->part_reg, nullptr, st));
        EI_CUDA_TRY(launch_prep(g, sv->u, ec.mult, linked, nullptr, st));
        count_launches(g, 2);
        EI_CUDA_TRY(solver_project(g, sv->Pt, ec.link, nullptr, st));
        EI_CUDA_TRY(solver_ic(g, sv->Pt, meas, ec.link, nullptr, st));
        EI_CUDA_TRY(launch_finalize_objective(g, g->part_ic, dg.vec_prefix, sv->part_reg,
                                              g->S_dev, nullptr, st));
        count_launches(g, 1);
        EI_CUDA_TRY(solver_adjoint(g, sv->u, sv->g, ec, nullptr, st));
        if (ow) EI_CUDA_TRY(offsets_gradient(sv->g, nullptr));
        if (NR > 0) k_sino_rows<true><<<NR, 256, 0, st>>>(g->dg, dv, sv->Pu, sv->Pt, nullptr);
        k_gram_gg<<<NB, T, 0, st>>>(dg, dv);
        k_init_state<<<1, scalar_threads, 0, st>>>(dg, dv, g->S_dev, sv->summary);
        count_launches(g, 3);
        EI_CUDA_TRY(cudaGetLastError());
        *evals = 1;
    }
    EI_CUDA_TRY(cudaMemcpyAsync(sv->summary_h, sv->summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st));
    EI_CUDA_TRY(cudaStreamSynchronize(st));

    // one round: direction for the slices that need one; a trial step and its
    // objective for every slice in line search (projected when it is the
    // iteration's first trial, interpolated otherwise); Armijo; the gradient,
    // projections and memory update of accepted slices; summary
    auto round = [&]() -> cudaError_t {
        // direction (coefficients, for the slices that need one) and first step
        k_ls_start<<<1, scalar_threads, 0, st>>>(dg, dv);
        k_trial<<<NB, T, 0, st>>>(dg, dv, ec.reg1, sv->part_reg, sv->part_gd);
        count_launches(g, 2);
        EI_CUDA_TRY(cudaGetLastError());
        // the trial's projections: first trials projected, later ones interpolated
        EI_CUDA_TRY(launch_prep(g, sv->xt, ec.mult, linked, sv->mask_first, st));
        count_launches(g, 1);
        EI_CUDA_TRY(solver_project(g, sv->Pt, ec.link, sv->mask_first, st));
        if (NR > 0) k_sino_rows<false><<<NR, 256, 0, st>>>(g->dg, dv, sv->Pu, sv->Pt, sv->mask_bt);
        count_launches(g, 1);
        if (ow) {
            k_offsets_apply<<<g->n_slices, 256, 0, st>>>(dg, ow, os, sv->xt, sv->mask_ls);
            count_launches(g, 1);
        }
        // the objective at the trial: data term (its per-pixel gradient too) + regulariser
        EI_CUDA_TRY(solver_ic(g, sv->Pt, meas, ec.link, sv->mask_ls, st));
        EI_CUDA_TRY(launch_finalize_objective(g, g->part_ic, dg.vec_prefix, sv->part_reg,
                                              g->S_dev, sv->mask_ls, st));
        k_armijo<<<1, scalar_threads, 0, st>>>(dg, dv, g->S_dev, sv->part_gd, o);
        count_launches(g, 2);
        EI_CUDA_TRY(cudaGetLastError());
        // accepted trials: the gradient, the projections Pu, the memory update
        EI_CUDA_TRY(solver_adjoint(g, sv->xt, sv->gt, ec, sv->mask_acc, st));
        if (ow) EI_CUDA_TRY(offsets_gradient(sv->gt, sv->mask_acc));
        if (NR > 0) k_sino_rows<true><<<NR, 256, 0, st>>>(g->dg, dv, sv->Pu, sv->Pt, sv->mask_acc);
        k_accept<<<NB, T, 0, st>>>(dg, dv);
        k_update<<<1, scalar_threads, 0, st>>>(dg, dv, o, sv->summary);
        count_launches(g, 3);
        EI_CUDA_TRY(cudaGetLastError());
        return cudaMemcpyAsync(sv->summary_h, sv->summary, 2 * sizeof(int), cudaMemcpyDeviceToHost, st);
    };

    // CUDA graph: capture the round once, replay it every round.  While
    // tracing is on, rounds run eagerly so that every traced launch is timed.
    cudaGraphExec_t exec = nullptr;
    int64_t launches_per_round = 0;
    if (opts->use_graph && !g->prof_on) {
        const int64_t l0 = g->launches;
        cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        cudaGraph_t graph = nullptr;
        if (ce == cudaSuccess) {
            ce = round();
            const cudaError_t ee = cudaStreamEndCapture(st, &graph);
            if (ce == cudaSuccess) ce = ee;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        launches_per_round = g->launches - l0;
        g->launches = l0;
        if (ce != cudaSuccess) {            // capture not possible here: run the rounds eagerly
            cudaGetLastError();
            exec = nullptr;
        }
    }
    cudaError_t err = cudaSuccess;
    const long long max_rounds = (long long)opts->max_iter * (opts->max_trials + 1) + 2;
    *timed_out = false;
    for (long long r = 0; sv->summary_h[0] > 0 && r < max_rounds; ++r) {
        if (opts->max_seconds > 0 && std::chrono::steady_clock::now() >= deadline) {
            *timed_out = true;                // between rounds: nothing in flight
            break;
        }
        NvtxRange rr("solver round");
        if (exec) {
            err = cudaGraphLaunch(exec, st);
            g->launches += launches_per_round;
        } else {
            err = round();
        }
        if (err == cudaSuccess) err = cudaStreamSynchronize(st);
        if (err != cudaSuccess) break;
        *evals += 1;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (err != cudaSuccess) return err;
    sv->has_state = true;
    k_from_scaled<<<NBv, T, 0, st>>>(g->dg, sv->u, x_dev, sc);
    count_launches(g, 1);
    if (ow) {                                 // the solution's offsets stay in the geometry
        k_offsets_apply<<<g->n_slices, 256, 0, st>>>(dg, ow, os, sv->u, nullptr);
        count_launches(g, 1);
    }
    return cudaGetLastError();
}

int reconstruct(ei_geometry *g, const float *s_exp, float *vol_inout, const ei_solve_opts *opts,
                ei_solve_report *report, cudaStream_t st)
{
    NvtxRange range("ei_reconstruct");
    const auto t0 = std::chrono::steady_clock::now();
    if (opts->resume && !(g->solver && g->solver->has_state && g->solver->m == opts->lbfgs_m &&
                          g->solver->off_which == g->off_which)) {
        record_message("ei_reconstruct: resume needs the state of a completed solve or a "
                       "loaded checkpoint with the same lbfgs_m and unknowns");
        return EI_ERR_ARG;
    }
    cudaError_t e = ensure_solver(g, opts->lbfgs_m);
    if (e != cudaSuccess) {
        record_error(e);
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        destroy_solver(g);
        return oom ? EI_ERR_ALLOC : EI_ERR_CUDA;
    }
    Solver *sv = g->solver;
    // the call is synchronous: finish the caller's queued work, then run on the
    // solver's own stream (a legacy default stream could not be captured)
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        record_error(e);
        return EI_ERR_CUDA;
    }
    st = sv->stream;
    const bool meas_dev = is_device_ptr(s_exp), vol_dev = is_device_ptr(vol_inout);
    const float *meas = s_exp;
    float4 *x = (float4 *)vol_inout;
    if (!meas_dev) {
        if (!sv->meas_stage) e = salloc(sv, &sv->meas_stage, (size_t)g->meas_count);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sv->meas_stage, s_exp, (size_t)g->meas_count * sizeof(float),
                                cudaMemcpyHostToDevice, st);
        meas = sv->meas_stage;
    }
    if (e == cudaSuccess && !vol_dev) {
        if (!sv->vol_stage) e = salloc(sv, &sv->vol_stage, (size_t)g->vol_count);
        if (e == cudaSuccess && !opts->resume)     // resume: vol_inout is output only
            e = cudaMemcpyAsync(sv->vol_stage, vol_inout, (size_t)g->vol_count * sizeof(float4),
                                cudaMemcpyHostToDevice, st);
        x = sv->vol_stage;
    }
    int evals = 0;
    bool timed_out = false;
    const auto deadline = t0 + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                   std::chrono::duration<double>(std::min(opts->max_seconds, 1e9)));
    if (e == cudaSuccess) e = run_solver(g, meas, x, opts, &evals, st, deadline, &timed_out);
    if (e == cudaSuccess && !vol_dev)
        e = cudaMemcpyAsync(vol_inout, sv->vol_stage, (size_t)g->vol_count * sizeof(float4),
                            cudaMemcpyDeviceToHost, st);
    std::vector<SliceState> hs(g->n_slices);
    std::vector<int> still_dir(timed_out ? g->n_slices : 0), still_ls(still_dir.size());
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hs.data(), sv->st, sizeof(SliceState) * g->n_slices,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && timed_out)        // which slices the budget stopped
        e = cudaMemcpyAsync(still_dir.data(), sv->mask_dir, sizeof(int) * g->n_slices,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && timed_out)
        e = cudaMemcpyAsync(still_ls.data(), sv->mask_ls, sizeof(int) * g->n_slices,
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        record_error(e);
        return e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA;
    }
    int first_err = EI_OK;
    for (int s = 0; s < g->n_slices; ++s) {
        int status = hs[s].status;
        if (status == EI_OK && isnan(hs[s].f)) status = EI_ERR_NONFINITE;
        if (status == EI_OK && timed_out && (still_dir[s] | still_ls[s])) status = EI_ERR_TIMEOUT;
        if (status != EI_OK && first_err == EI_OK) first_err = status;
        if (report) {
            if (report->iterations) report->iterations[s] = hs[s].k;
            if (report->status) report->status[s] = status;
            if (report->converged) report->converged[s] = hs[s].converged;
            if (report->f_final) report->f_final[s] = hs[s].f;
            if (report->f_initial) report->f_initial[s] = hs[s].f0;
            if (report->slice_evaluations) report->slice_evaluations[s] = hs[s].evals;
            if (report->slice_projections) report->slice_projections[s] = hs[s].projections;
            if (report->slice_adjoints) report->slice_adjoints[s] = hs[s].adjoints;
        }
    }
    if (report) {
        report->evaluations = evals;
        report->seconds =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return first_err;
}

// --------------------------------------------------------------------------
// checkpoint: the state a solve leaves (or a resumed solve continues from),
// behind a header that names the geometry it belongs to
// --------------------------------------------------------------------------
struct StateHeader {
    uint64_t magic;          // "EISOLVER" + layout version
    int n_slices, m, ring, off_which;
    int linked, slice_state_bytes;
    int64_t vol_count;       // float4 per solver vector (volumes + offsets segments)
    uint64_t shape_hash;
};

static const uint64_t kStateMagic = 0x4549534f4c564533ull;   // "EISOLVE3"

static int64_t solver_vol_count(const ei_geometry *g)
{
    int64_t ext = g->vol_count;
    if (g->off_which)
        for (const SliceInfo &si : g->h_slices) {
            const int K = ((g->off_which & EI_OFFSET_MO) ? si.n_theta : 0) +
                          ((g->off_which & EI_OFFSET_MR) ? si.n_det : 0);
            ext += (K + 2) / 3;
        }
    return ext;
}

static StateHeader state_header(const ei_geometry *g, int m)
{
    StateHeader h{};
    h.magic = kStateMagic;
    h.n_slices = g->n_slices;
    h.m = m;
    h.ring = m + 1;
    h.off_which = g->off_which;
    h.linked = g->link_gamma > 0.f ? 1 : 0;
    h.slice_state_bytes = (int)sizeof(SliceState);
    h.vol_count = solver_vol_count(g);
    h.shape_hash = g->shape_hash;
    return h;
}

// The state's pieces in checkpoint order: device pointer and bytes.
static std::vector<std::pair<void *, size_t>> state_pieces(const Solver *s, const ei_geometry *g)
{
    const size_t V = (size_t)s->vol_count * sizeof(float4), S = (size_t)g->n_slices;
    const size_t P = (size_t)g->proj_count * sizeof(float);
    return {{s->u, V},
            {s->Pu, P},
            {s->Pt, P},
            {s->g, V},
            {s->d, V},
            {s->Sr, V * s->ring},
            {s->Yr, V * s->ring},
            {s->gram, sizeof(double) * S * basis_dim(s->ring) * basis_dim(s->ring)},
            {s->coef, sizeof(double) * S * basis_dim(s->ring)},
            {s->st, sizeof(SliceState) * S},
            {s->mask_dir, sizeof(int) * S},
            {s->mask_ls, sizeof(int) * S},
            {s->mask_acc, sizeof(int) * S}};
}

size_t solver_state_size(const ei_geometry *g, int m)
{
    const size_t V = (size_t)solver_vol_count(g) * sizeof(float4), S = (size_t)g->n_slices;
    const size_t ring = (size_t)m + 1;
    const size_t GD = (size_t)basis_dim((int)ring);
    return sizeof(StateHeader) + V * (3 + 2 * ring) + 2 * sizeof(float) * (size_t)g->proj_count +
           sizeof(double) * S * GD * (GD + 1) + sizeof(SliceState) * S + 3 * sizeof(int) * S;
}

int solver_save(const ei_geometry *g, void *buf, size_t bytes)
{
    const Solver *s = g->solver;
    if (!s || !s->has_state) {
        record_message("ei_solver_save: no completed solve on this geometry");
        return EI_ERR_ARG;
    }
    if (bytes < solver_state_size(g, s->m)) return EI_ERR_ARG;
    const StateHeader h = state_header(g, s->m);
    char *p = static_cast<char *>(buf);
    cudaError_t e = cudaMemcpy(p, &h, sizeof h, cudaMemcpyDefault);
    p += sizeof h;
    for (const auto &pc : state_pieces(s, g)) {
        if (e != cudaSuccess) break;
        e = cudaMemcpy(p, pc.first, pc.second, cudaMemcpyDefault);
        p += pc.second;
    }
    if (e != cudaSuccess) {
        record_error(e);
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    return EI_OK;
}

int solver_load(ei_geometry *g, int m, const void *buf, size_t bytes)
{
    if (bytes < solver_state_size(g, m)) return EI_ERR_ARG;
    StateHeader h{};
    const char *p = static_cast<const char *>(buf);
    cudaError_t e = cudaMemcpy(&h, p, sizeof h, cudaMemcpyDefault);
    if (e != cudaSuccess) {
        record_error(e);
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    const StateHeader want = state_header(g, m);
    if (h.magic != want.magic || h.n_slices != want.n_slices || h.m != want.m ||
        h.ring != want.ring || h.off_which != want.off_which || h.linked != want.linked ||
        h.slice_state_bytes != want.slice_state_bytes || h.vol_count != want.vol_count ||
        h.shape_hash != want.shape_hash) {
        record_message("ei_solver_load: the checkpoint belongs to another geometry, mode or lbfgs_m");
        return EI_ERR_ARG;
    }
    e = ensure_solver(g, m);
    if (e != cudaSuccess) {
        record_error(e);
        const bool oom = e == cudaErrorMemoryAllocation;
        cudaGetLastError();
        destroy_solver(g);
        return oom ? EI_ERR_ALLOC : EI_ERR_CUDA;
    }
    Solver *s = g->solver;
    s->has_state = false;
    p += sizeof h;
    for (const auto &pc : state_pieces(s, g)) {
        if (e != cudaSuccess) break;
        e = cudaMemcpy(pc.first, p, pc.second, cudaMemcpyDefault);
        p += pc.second;
    }
    if (e != cudaSuccess) {
        record_error(e);
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    s->has_state = true;
    return EI_OK;
}

}  // namespace ei
