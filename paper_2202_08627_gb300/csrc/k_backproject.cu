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
// Linked unknown of Eq. 4 (mu = h, delta = gamma h): by linearity
// R^T g_mu + gamma R^T g_delta = R^T (g_mu + gamma g_delta), so the IC kernel
// writes that single sinogram, pair-packed, and the linked instantiation loads
// one 8-B entry per voxel and angle (a third of the bytes) and does 2 FMAs.
//
// Also fused: out = out_mult * R^T g + reg2 * v (the regulariser's gradient;
// v may be null).  The regulariser's value sum_c lambda_c ||u_c||^2 is summed
// elsewhere (k_reg_partials, or the solver's trial-point kernel), so that the
// objective at a point never needs this kernel: the solver runs it only where
// a line-search trial was accepted.
#include <algorithm>

#include "ei_internal.h"

namespace ei {

constexpr int ADJ_CHUNK = 128;           // angles staged per shared-memory chunk

__device__ __forceinline__ double block_sum_double_fin(double v, double *red)
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

struct AdjShared {
    float4 cs[ADJ_CHUNK];   // cos, sin, pitch/(ch*ch), pitch/ch
    float4 jp[ADJ_CHUNK];   // J (int bits), phi, pitch/ch - pitch/(ch*ch), mirror variant: phi_B
    int jb[ADJ_CHUNK];      // mirror variant: J_B
};

// Check builds: the entries J + jj .. J + jj + span of a packed gradient row
// lie within its margins, [-marg, n_dp + marg - 1] (pixel units); returns
// the (clamped) jj.  Regular builds: jj.
__device__ __forceinline__ int row_entry(int jj, int J, int span, const SliceInfo &si, int *status)
{
    if (!kDeviceChecks) return jj;
    return checked_index(J + jj, -si.marg, si.n_dp + si.marg - 1 - span, status) - J;
}

// One voxel's output: out = out_mult R^T g + reg2 v; linked: the unknown h
// in the mu lane, dS/dh = R^T (g_mu + link g_delta), the sinogram the IC
// kernel combined.
template <bool LINKED>
__device__ __forceinline__ void adj_store(float4 *__restrict__ out, int64_t idx,
                                          const float4 *__restrict__ v, const float (&acc)[3],
                                          float4 out_mult, float4 reg2)
{
    const float4 x = v ? v[idx] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (LINKED)
        out[idx] = make_float4(fmaf(out_mult.x, acc[0], reg2.x * x.x), 0.f, 0.f, 0.f);
    else
        out[idx] = make_float4(fmaf(out_mult.x, acc[0], reg2.x * x.x),
                               fmaf(out_mult.y, acc[1], reg2.y * x.y),
                               fmaf(out_mult.z, acc[2], reg2.z * x.z), 0.f);
}

// One work item: a 32-column x (8 PASSES)-row voxel tile, 8 x 4 voxel patch per
// warp and pass, one voxel per thread and pass.  Lanes run along the patch's
// rows of 8 voxels, or (QUAD) each group of 8 consecutive lanes covers a 2 x 4
// sub-patch, whose detector positions lie closer together (L1 serves the
// group's 16-byte loads in one pass when they share a 128-byte line).  A
// voxel's computation does not depend on the lane order, and angles are
// summed in order whatever PASSES.
template <int PASSES, bool QUAD, bool LINKED>
__device__ __forceinline__ void backproject_single_item(
    const DevGeom &dg, const int *prefix, int item, AdjShared &sh, const float4 *__restrict__ gA,
    const float2 *__restrict__ gB, const float4 *__restrict__ v, float4 *__restrict__ out,
    float4 out_mult, float4 reg2, const int *__restrict__ active)
{
    constexpr int TR = 8 * PASSES;
    const int s = find_slice(prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int ntc = (n + ADJ_TC - 1) / ADJ_TC;
    const int local = item - prefix[s];
    const int r_t = (local / ntc) * TR, c_t = (local % ntc) * ADJ_TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // column offset in the tile, row offset of pass 0 (passes add 8)
    const int dc = (warp & 3) * 8 + (QUAD ? 2 * (lane >> 3) + (lane & 1) : lane & 7);
    const int dr0 = (warp >> 2) * 4 + (QUAD ? (lane >> 1) & 3 : lane >> 3);

    float acc[PASSES][3];
#pragma unroll
    for (int p = 0; p < PASSES; ++p) acc[p][0] = acc[p][1] = acc[p][2] = 0.f;

    {
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
                sh.cs[threadIdx.x] = make_float4(an.cosf, an.sinf, pi, an.pch);
                sh.jp[threadIdx.x] = make_float4(
                    __int_as_float((int)(U >> 32)),
                    (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f, an.pch - pi, 0.f);
            }
            __syncthreads();
            const float4 *rowA = rowA0 + (int64_t)a0 * si.gw;
            const float2 *rowB = rowB0 + (int64_t)a0 * si.gw;
            for (int k = 0; k < na; ++k) {
                const float4 cs = sh.cs[k];
                const float4 jp = sh.jp[k];
                const int J = __float_as_int(jp.x);
                const float v0 = fmaf(fx, cs.x, fmaf(-fy, cs.y, jp.y));
                const float step = -8.f * cs.y;
                const float4 *rA = rowA + J;
                const float2 *rB = rowB + J;
#pragma unroll
                for (int p = 0; p < PASSES; ++p) {
                    const float vl = fmaf((float)p, step, v0);
                    const float fl = floorf(vl);
                    const int jj = row_entry((int)fl, J, 0, si, dg.status);
                    const float d0 = vl - fl;
                    const float w0 = fmaxf(0.f, fmaf(-d0, cs.z, cs.w));
                    const float w1 = fmaxf(0.f, fmaf(d0, cs.z, jp.z));
                    if (LINKED) {                   // one 8-byte entry: g(j), g(j + 1)
                        const float2 tb = __ldg(rB + jj);
                        acc[p][0] = fmaf(w0, tb.x, fmaf(w1, tb.y, acc[p][0]));
                    } else {
                        const float4 ta = __ldg(rA + jj);
                        const float2 tb = __ldg(rB + jj);
                        acc[p][0] = fmaf(w0, ta.x, fmaf(w1, ta.w, acc[p][0]));
                        acc[p][1] = fmaf(w0, ta.y, fmaf(w1, tb.x, acc[p][1]));
                        acc[p][2] = fmaf(w0, ta.z, fmaf(w1, tb.y, acc[p][2]));
                    }
                }
                rowA += si.gw;
                rowB += si.gw;
            }
        }
    }

    const int c = c_t + dc;
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
        const int r = r_t + dr0 + 8 * p;
        if (r < n && c < n) {
            const int64_t idx = si.vol_off + (int64_t)r * n + c;
            adj_store<LINKED>(out, idx, v, acc[p], out_mult, reg2);
        }
    }
}

// Voxel pairs.  Two horizontally adjacent voxels project |cos| <= 1 pixel
// apart, so at every angle their four taps lie among three consecutive pixels
// j, j + 1, j + 2 (j: the lower tap of the pair's lower-u voxel), and the
// packed sinogram already holds g(j + 2) in the second half of entry j + 1.
// A thread owns a pair: per angle it loads entry j, and of entry j + 1 only the
// second half (3 of its 6 floats), 36 B for two voxels instead of 48, and
// shares the index arithmetic.  The lower-u voxel adds its two taps as the
// single-voxel kernel does; the other one, whose lower tap is j + o with
// o = [d + |cos| >= 1], adds the three slots with weights (w0, w1, 0) or
// (0, w0, w1): the same FMAs in the same order, plus one with a zero weight.
// Warp: 8 pairs x 4 rows; a tile is 32 columns x 16 PASSES rows.
template <int PASSES, bool LINKED, bool SWAP>
__device__ __forceinline__ void pair_angle(float (&acc)[PASSES][2][3], const float4 *rA,
                                           const float2 *rB, float v0, float step, float a,
                                           float4 cs, float4 jp, int J, const SliceInfo &si,
                                           int *status)
{
    constexpr int LO = SWAP ? 1 : 0, HI = SWAP ? 0 : 1;    // lower-u voxel: left unless cos < 0
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
        const float vl = fmaf((float)p, step, v0);
        const float fl = floorf(vl);
        const int jj = row_entry((int)fl, J, 1, si, status);
        const float d0 = vl - fl;
        float dh = d0 + a;
        const bool o = dh >= 1.f;
        dh = o ? dh - 1.f : dh;
        const float w0l = fmaxf(0.f, fmaf(-d0, cs.z, cs.w)), w1l = fmaxf(0.f, fmaf(d0, cs.z, jp.z));
        const float w0h = fmaxf(0.f, fmaf(-dh, cs.z, cs.w)), w1h = fmaxf(0.f, fmaf(dh, cs.z, jp.z));
        const float s0 = o ? 0.f : w0h, s1 = o ? w0h : w1h, s2 = o ? w1h : 0.f;
        if (LINKED) {
            const float2 t = __ldg(rB + jj);                                  // g(j), g(j + 1)
            const float g2 = __ldg(reinterpret_cast<const float *>(rB + jj + 1) + 1);   // g(j + 2)
            acc[p][LO][0] = fmaf(w0l, t.x, fmaf(w1l, t.y, acc[p][LO][0]));
            acc[p][HI][0] = fmaf(s0, t.x, fmaf(s1, t.y, fmaf(s2, g2, acc[p][HI][0])));
        } else {
            const float4 ta = __ldg(rA + jj);       // mu(j), delta(j), sigma(j), mu(j + 1)
            const float2 tb = __ldg(rB + jj);       // delta(j + 1), sigma(j + 1)
            const float m2 = __ldg(reinterpret_cast<const float *>(rA + jj + 1) + 3);  // mu(j + 2)
            const float2 tc = __ldg(rB + jj + 1);   // delta(j + 2), sigma(j + 2)
            acc[p][LO][0] = fmaf(w0l, ta.x, fmaf(w1l, ta.w, acc[p][LO][0]));
            acc[p][LO][1] = fmaf(w0l, ta.y, fmaf(w1l, tb.x, acc[p][LO][1]));
            acc[p][LO][2] = fmaf(w0l, ta.z, fmaf(w1l, tb.y, acc[p][LO][2]));
            acc[p][HI][0] = fmaf(s0, ta.x, fmaf(s1, ta.w, fmaf(s2, m2, acc[p][HI][0])));
            acc[p][HI][1] = fmaf(s0, ta.y, fmaf(s1, tb.x, fmaf(s2, tc.x, acc[p][HI][1])));
            acc[p][HI][2] = fmaf(s0, ta.z, fmaf(s1, tb.y, fmaf(s2, tc.y, acc[p][HI][2])));
        }
    }
}

template <int PASSES, bool LINKED, int COMPACT>
__device__ __forceinline__ void backproject_pair_item(
    const DevGeom &dg, const int *prefix, int item, AdjShared &sh, const float4 *__restrict__ gA,
    const float2 *__restrict__ gB, const float4 *__restrict__ v, float4 *__restrict__ out,
    float4 out_mult, float4 reg2, const int *__restrict__ active)
{
    constexpr int TR = 16 * PASSES;
    const int s = find_slice(prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int ntc = (n + ADJ_TC - 1) / ADJ_TC;
    const int local = item - prefix[s];
    const int r_t = (local / ntc) * TR, c_t = (local % ntc) * ADJ_TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // left voxel of the pair and its row at pass 0 (passes add 16): 8 lanes cover
    // 8 pairs of one row (COMPACT 0) or 2 pairs x 4 rows; a warp covers 16
    // columns x 4 rows (COMPACT 0, 1) or 8 columns x 8 rows (COMPACT 2)
    int dc, dr0;
    if (COMPACT == 2) {
        dc = (warp & 3) * 8 + 2 * (lane & 1) + 4 * ((lane >> 3) & 1);
        dr0 = (warp >> 2) * 8 + ((lane >> 1) & 3) + 4 * (lane >> 4);
    } else {
        dc = (warp & 1) * 16 + (COMPACT ? 4 * (lane >> 3) + 2 * (lane & 1) : 2 * (lane & 7));
        dr0 = (warp >> 1) * 4 + (COMPACT ? (lane >> 1) & 3 : lane >> 3);
    }

    float acc[PASSES][2][3];
#pragma unroll
    for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int h = 0; h < 2; ++h) acc[p][h][0] = acc[p][h][1] = acc[p][h][2] = 0.f;

    {
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
                sh.cs[threadIdx.x] = make_float4(an.cosf, an.sinf, pi, an.pch);
                sh.jp[threadIdx.x] = make_float4(
                    __int_as_float((int)(U >> 32)),
                    (float)(unsigned)(U & 0xffffffffLL) * 2.3283064365386963e-10f, an.pch - pi, 0.f);
            }
            __syncthreads();
            const float4 *rowA = rowA0 + (int64_t)a0 * si.gw;
            const float2 *rowB = rowB0 + (int64_t)a0 * si.gw;
            for (int k = 0; k < na; ++k) {
                const float4 cs = sh.cs[k];
                const float4 jp = sh.jp[k];
                const int J = __float_as_int(jp.x);
                // detector position of the pair's lower-u voxel at pass 0
                const float v0 = fmaf(fx, cs.x, fmaf(-fy, cs.y, jp.y)) + fminf(cs.x, 0.f);
                const float step = -16.f * cs.y;
                if (cs.x >= 0.f)
                    pair_angle<PASSES, LINKED, false>(acc, rowA + J, rowB + J, v0, step, cs.x, cs, jp,
                                                      J, si, dg.status);
                else
                    pair_angle<PASSES, LINKED, true>(acc, rowA + J, rowB + J, v0, step, -cs.x, cs, jp,
                                                     J, si, dg.status);
                rowA += si.gw;
                rowB += si.gw;
            }
        }
    }

#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
        const int r = r_t + dr0 + 16 * p;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c_t + dc + h;
            if (r < n && c < n) {
                const int64_t idx = si.vol_off + (int64_t)r * n + c;
                adj_store<LINKED>(out, idx, v, acc[p][h], out_mult, reg2);
            }
        }
    }
}

// Mirror images.  Voxel (x, y) of a slice, in pitch units about its centre,
// projects to u(x, y) = hd + x cos + y sin; its point mirror (-x, -y) to
// 2 hd - u = (n_det - 1) - u.  With u = j + d the mirror's taps are pixels
// n_det - 1 - j and n_det - 2 - j with the SAME hat weights (the entry
// weights depend on |u - j| only), so one detector-coordinate split and one
// weight computation serve a voxel and its point mirror.  A thread owns a
// voxel pair of the slice's top-left quadrant (rows r < ceil(n / 2), columns
// c < ceil(n / 2)) and the pair's three images: family A = the pair and its
// point mirror, family B = its row mirror (x, -y) and that one's point mirror
// (-x, y); each family needs one split per angle (two per 8 voxels instead
// of four).  The point mirror of a pair is again a horizontally adjacent
// pair, so its loads keep the pair shape (one entry and the second half of
// the next), taken from the mirrored end of the row: the slot of pixel j + k
// of the pair is pixel n_det - 1 - j - k of its image.  Every voxel is written
// by exactly one (thread, image): the pair itself where it lies in the
// quadrant, an image where it lies in the other half (an odd slice's centre
// row and column belong to the quadrant).  The mirrored detector coordinate
// is exact only up to FP32 rounding of d, so results agree with the other
// variants to FP32 rounding, not bit for bit.
template <bool LINKED, bool SWAP, int q0, int q1>
__device__ __forceinline__ void mirror_pair_angle(float (&acc)[4][2][3], const float4 *row_a,
                                                  const float2 *row_b, float vl, float a,
                                                  float4 cs, float4 jp, int J, int JM,
                                                  const SliceInfo &si, int *status)
{
    // vl: detector position of the pair's lower-u voxel (relative to J); a =
    // |cos|; q0, q1: the acc indices of the pair (direct) and of its point
    // mirror; row_a / row_b: the row's entry of pixel 0; the image of entry
    // J + jj is JM - jj, JM = n_det - 3 - J
    const float fl = floorf(vl);
    const int ed = J + row_entry((int)fl, J, 1, si, status);          // the pair's entry
    const int em = JM + row_entry(-(int)fl, JM, 1, si, status);       // its image's entry
    const float d0 = vl - fl;
    float dh = d0 + a;
    const bool o = dh >= 1.f;
    dh = o ? dh - 1.f : dh;
    const float w0l = fmaxf(0.f, fmaf(-d0, cs.z, cs.w)), w1l = fmaxf(0.f, fmaf(d0, cs.z, jp.z));
    const float w0h = fmaxf(0.f, fmaf(-dh, cs.z, cs.w)), w1h = fmaxf(0.f, fmaf(dh, cs.z, jp.z));
    const float s0 = o ? 0.f : w0h, s1 = o ? w0h : w1h, s2 = o ? w1h : 0.f;
    // lower-u voxel: left unless cos < 0; acc[q1][h] holds the image of voxel h,
    // which takes voxel h's weights at the mirrored pixels
    constexpr int LO = SWAP ? 1 : 0, HI = SWAP ? 0 : 1;
    if (LINKED) {
        const float2 t = __ldg(row_b + ed);                                      // slots 0, 1
        const float g2 = __ldg(reinterpret_cast<const float *>(row_b + ed + 1) + 1);   // slot 2
        acc[q0][LO][0] = fmaf(w0l, t.x, fmaf(w1l, t.y, acc[q0][LO][0]));
        acc[q0][HI][0] = fmaf(s0, t.x, fmaf(s1, t.y, fmaf(s2, g2, acc[q0][HI][0])));
        const float2 u = __ldg(row_b + em);                                      // slots 2, 1
        const float g0 = __ldg(reinterpret_cast<const float *>(row_b + em + 1) + 1);   // slot 0
        acc[q1][LO][0] = fmaf(w0l, g0, fmaf(w1l, u.y, acc[q1][LO][0]));
        acc[q1][HI][0] = fmaf(s0, g0, fmaf(s1, u.y, fmaf(s2, u.x, acc[q1][HI][0])));
    } else {
        const float4 ta = __ldg(row_a + ed);       // slot 0 (mu, delta, sigma), slot 1 mu
        const float2 tb = __ldg(row_b + ed);       // slot 1 (delta, sigma)
        const float m2 = __ldg(reinterpret_cast<const float *>(row_a + ed + 1) + 3);  // slot 2 mu
        const float2 tc = __ldg(row_b + ed + 1);   // slot 2 (delta, sigma)
        acc[q0][LO][0] = fmaf(w0l, ta.x, fmaf(w1l, ta.w, acc[q0][LO][0]));
        acc[q0][LO][1] = fmaf(w0l, ta.y, fmaf(w1l, tb.x, acc[q0][LO][1]));
        acc[q0][LO][2] = fmaf(w0l, ta.z, fmaf(w1l, tb.y, acc[q0][LO][2]));
        acc[q0][HI][0] = fmaf(s0, ta.x, fmaf(s1, ta.w, fmaf(s2, m2, acc[q0][HI][0])));
        acc[q0][HI][1] = fmaf(s0, ta.y, fmaf(s1, tb.x, fmaf(s2, tc.x, acc[q0][HI][1])));
        acc[q0][HI][2] = fmaf(s0, ta.z, fmaf(s1, tb.y, fmaf(s2, tc.y, acc[q0][HI][2])));
        const float4 ma = __ldg(row_a + em);       // slot 2 (mu, delta, sigma), slot 1 mu
        const float2 mb = __ldg(row_b + em);       // slot 1 (delta, sigma)
        const float n0 = __ldg(reinterpret_cast<const float *>(row_a + em + 1) + 3);  // slot 0 mu
        const float2 mc = __ldg(row_b + em + 1);   // slot 0 (delta, sigma)
        acc[q1][LO][0] = fmaf(w0l, n0, fmaf(w1l, ma.w, acc[q1][LO][0]));
        acc[q1][LO][1] = fmaf(w0l, mc.x, fmaf(w1l, mb.x, acc[q1][LO][1]));
        acc[q1][LO][2] = fmaf(w0l, mc.y, fmaf(w1l, mb.y, acc[q1][LO][2]));
        acc[q1][HI][0] = fmaf(s0, n0, fmaf(s1, ma.w, fmaf(s2, ma.x, acc[q1][HI][0])));
        acc[q1][HI][1] = fmaf(s0, mc.x, fmaf(s1, mb.x, fmaf(s2, ma.y, acc[q1][HI][1])));
        acc[q1][HI][2] = fmaf(s0, mc.y, fmaf(s1, mb.y, fmaf(s2, ma.z, acc[q1][HI][2])));
    }
}

// Two FP32 lanes in one 64-bit register: fma.rn.f32x2 computes each lane as
// a single correctly rounded fmaf, so a pair of accumulators advanced with it
// holds exactly what two fmaf chains would.
using f32x2 = unsigned long long;

__device__ __forceinline__ f32x2 fma_x2(f32x2 a, f32x2 b, f32x2 c)
{
    f32x2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

__device__ __forceinline__ f32x2 splat_x2(float w)
{
    f32x2 d;
    asm("mov.b64 %0, {%1, %1};" : "=l"(d) : "f"(w));
    return d;
}

__device__ __forceinline__ float2 unpack_x2(f32x2 v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// The mirror-interleaved layout (written by the IC kernels and k_pack_sino
// when a variant below is selected): entry j of a row holds pixel j and its
// mirror pixel n_det - 1 - j, A = (mu_j, mu_m, delta_j, delta_m) and
// B = (sigma_j, sigma_m) (linked: B = (g_j, g_m)), zero outside [0, n_det).
// A voxel's taps j..j+2 and its point mirror's taps n_det-1-j.. are then the
// two lanes of the same three entries, and both take the same weights, so
// one fma.rn.f32x2 advances a channel of the voxel and of its image: half the
// FMA instructions of mirror_pair_angle, and 6 loads instead of 8 for the same
// 72 bytes.  The sums are formed in mirror_pair_angle's order, so the results
// equal its bit for bit.
template <bool LINKED, bool SWAP>
__device__ __forceinline__ void mirror_pair_angle_x2(f32x2 (&acc)[2][3], const ulonglong2 *row_a,
                                                     const f32x2 *row_b, float vl, float a,
                                                     float4 cs, float4 jp, int J,
                                                     const SliceInfo &si, int *status)
{
    const float fl = floorf(vl);
    const int e = J + row_entry((int)fl, J, 2, si, status);           // entries e .. e + 2
    const float d0 = vl - fl;
    float dh = d0 + a;
    const bool o = dh >= 1.f;
    dh = o ? dh - 1.f : dh;
    const float w0l = fmaxf(0.f, fmaf(-d0, cs.z, cs.w)), w1l = fmaxf(0.f, fmaf(d0, cs.z, jp.z));
    const float w0h = fmaxf(0.f, fmaf(-dh, cs.z, cs.w)), w1h = fmaxf(0.f, fmaf(dh, cs.z, jp.z));
    constexpr int LO = SWAP ? 1 : 0, HI = SWAP ? 0 : 1;
    // tap by tap, last tap first (each sum keeps mirror_pair_angle's order:
    // the tap of pixel j + 2, then j + 1, then j), so that only one entry's
    // data and its weights are live at a time
    {
        const f32x2 S2 = splat_x2(o ? w1h : 0.f);
        if (LINKED) {
            acc[HI][0] = fma_x2(S2, __ldg(row_b + e + 2), acc[HI][0]);
        } else {
            const ulonglong2 t = __ldg(row_a + e + 2);
            const f32x2 u = __ldg(row_b + e + 2);
            acc[HI][0] = fma_x2(S2, t.x, acc[HI][0]);
            acc[HI][1] = fma_x2(S2, t.y, acc[HI][1]);
            acc[HI][2] = fma_x2(S2, u, acc[HI][2]);
        }
    }
    {
        const f32x2 W1 = splat_x2(w1l), S1 = splat_x2(o ? w0h : w1h);
        if (LINKED) {
            const f32x2 t = __ldg(row_b + e + 1);
            acc[LO][0] = fma_x2(W1, t, acc[LO][0]);
            acc[HI][0] = fma_x2(S1, t, acc[HI][0]);
        } else {
            const ulonglong2 t = __ldg(row_a + e + 1);
            const f32x2 u = __ldg(row_b + e + 1);
            acc[LO][0] = fma_x2(W1, t.x, acc[LO][0]);
            acc[LO][1] = fma_x2(W1, t.y, acc[LO][1]);
            acc[LO][2] = fma_x2(W1, u, acc[LO][2]);
            acc[HI][0] = fma_x2(S1, t.x, acc[HI][0]);
            acc[HI][1] = fma_x2(S1, t.y, acc[HI][1]);
            acc[HI][2] = fma_x2(S1, u, acc[HI][2]);
        }
    }
    {
        const f32x2 W0 = splat_x2(w0l), S0 = splat_x2(o ? 0.f : w0h);
        if (LINKED) {
            const f32x2 t = __ldg(row_b + e);
            acc[LO][0] = fma_x2(W0, t, acc[LO][0]);
            acc[HI][0] = fma_x2(S0, t, acc[HI][0]);
        } else {
            const ulonglong2 t = __ldg(row_a + e);
            const f32x2 u = __ldg(row_b + e);
            acc[LO][0] = fma_x2(W0, t.x, acc[LO][0]);
            acc[LO][1] = fma_x2(W0, t.y, acc[LO][1]);
            acc[LO][2] = fma_x2(W0, u, acc[LO][2]);
            acc[HI][0] = fma_x2(S0, t.x, acc[HI][0]);
            acc[HI][1] = fma_x2(S0, t.y, acc[HI][1]);
            acc[HI][2] = fma_x2(S0, u, acc[HI][2]);
        }
    }
}

// Voxel rows of a mirror-variant tile: 16 per pass.  X2: the gradient rows
// are in the mirror-interleaved layout and a voxel and its point mirror share
// fma.rn.f32x2 instructions (mirror_pair_angle_x2).
template <int PASSES, bool LINKED, bool X2>
__device__ __forceinline__ void backproject_mirror_item(
    const DevGeom &dg, const int *prefix, int item, AdjShared &sh, const float4 *__restrict__ gA,
    const float2 *__restrict__ gB, const float4 *__restrict__ v, float4 *__restrict__ out,
    float4 out_mult, float4 reg2, const int *__restrict__ active)
{
    constexpr int TR = 16 * PASSES;
    const int s = find_slice(prefix, dg.n_slices, item);
    if (active && !active[s]) return;
    const SliceInfo si = dg.slices[s];
    const int n = si.n;
    const int hq = (n + 1) >> 1;                        // quadrant: rows and columns [0, hq)
    const int ntc = (hq + ADJ_TC - 1) / ADJ_TC;
    const int local = item - prefix[s];
    const int r_t = (local / ntc) * TR, c_t = (local % ntc) * ADJ_TC;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // left voxel of the pair and its row at pass 0 (passes add 16): warps of
    // 4 pairs x 8 rows, lanes in groups of 8 on 2 pairs x 4 rows
    const int dc = (warp & 3) * 8 + 2 * (lane & 1) + 4 * ((lane >> 3) & 1);
    const int dr0 = (warp >> 2) * 8 + ((lane >> 1) & 3) + 4 * (lane >> 4);

    // acc[p][image][voxel of the pair (0 = left column)][channel]; images:
    // 0 the pair (r, c..c+1), 1 its point mirror (n-1-r, n-1-c-h),
    // 2 its row mirror (n-1-r, c..c+1), 3 that one's point mirror (r, n-1-c-h)
    float acc[PASSES][4][2][3];
#pragma unroll
    for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) acc[p][q][h][0] = acc[p][q][h][1] = acc[p][q][h][2] = 0.f;
    // X2: acc2[p][family][voxel of the pair][channel] holds images (0, 1) of
    // family A and (2, 3) of family B as the two lanes
    f32x2 acc2[PASSES][2][2][3];
#pragma unroll
    for (int p = 0; p < PASSES; ++p)
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int h = 0; h < 2; ++h) acc2[p][q][h][0] = acc2[p][q][h][1] = acc2[p][q][h][2] = 0ull;

    {
        const float4 *rowA0 = gA + si.gp_off + si.marg;
        const float2 *rowB0 = gB + si.gp_off + si.marg;
        const long long two_ct = 2LL * c_t - (n - 1);              // 2 (c_t - hn)
        const long long two_rt = (long long)(n - 1) - 2LL * r_t;   // 2 (hn - r_t): family A
        const long long hd2 = (long long)(si.n_det - 1) << 32;     // 2 hd in 32.32
        const float fx = (float)dc, fy = (float)dr0;
        const int nm3 = si.n_det - 3;                              // image of entry j: nm3 - j
        for (int a0 = 0; a0 < si.n_theta; a0 += ADJ_CHUNK) {
            const int na = min(ADJ_CHUNK, si.n_theta - a0);
            __syncthreads();
            if ((int)threadIdx.x < na) {
                const AngleInfo an = dg.ang[si.ang_off + a0 + threadIdx.x];
                // the detector coordinate at the two families' tile origins: family
                // A's at row r_t, family B's at the mirrored row n - 1 - r_t
                const long long UA = (two_ct * an.cos_fx + two_rt * an.sin_fx + hd2) >> 1;
                const long long UB = (two_ct * an.cos_fx - two_rt * an.sin_fx + hd2) >> 1;
                const float pi = an.pch * an.inv_ch;
                sh.cs[threadIdx.x] = make_float4(an.cosf, an.sinf, pi, an.pch);
                sh.jp[threadIdx.x] = make_float4(
                    __int_as_float((int)(UA >> 32)),
                    (float)(unsigned)(UA & 0xffffffffLL) * 2.3283064365386963e-10f, an.pch - pi,
                    (float)(unsigned)(UB & 0xffffffffLL) * 2.3283064365386963e-10f);
                sh.jb[threadIdx.x] = (int)(UB >> 32);
            }
            __syncthreads();
            const float4 *rowA = rowA0 + (int64_t)a0 * si.gw;
            const float2 *rowB = rowB0 + (int64_t)a0 * si.gw;
            for (int k = 0; k < na; ++k) {
                const float4 cs = sh.cs[k];
                const float4 jp = sh.jp[k];
                const int JA = __float_as_int(jp.x), JB = sh.jb[k];
                // lower-u voxel of the pair at pass 0, family A (rows go down: y falls)
                // and family B (the mirrored rows go up: y rises)
                const float lo = fminf(cs.x, 0.f);
                const float vA = fmaf(fx, cs.x, fmaf(-fy, cs.y, jp.y)) + lo;
                const float vB = fmaf(fx, cs.x, fmaf(fy, cs.y, jp.w)) + lo;
                const float step = 16.f * cs.y;
                const float a = fabsf(cs.x);
                const int JMA = nm3 - JA, JMB = nm3 - JB;
                int *const st = dg.status;
                if constexpr (X2) {
                    const ulonglong2 *ra = reinterpret_cast<const ulonglong2 *>(rowA);
                    const f32x2 *rb = reinterpret_cast<const f32x2 *>(rowB);
                    if (cs.x >= 0.f) {
#pragma unroll
                        for (int p = 0; p < PASSES; ++p) {
                            mirror_pair_angle_x2<LINKED, false>(acc2[p][0], ra, rb,
                                                                fmaf((float)p, -step, vA), a, cs,
                                                                jp, JA, si, st);
                            mirror_pair_angle_x2<LINKED, false>(acc2[p][1], ra, rb,
                                                                fmaf((float)p, step, vB), a, cs,
                                                                jp, JB, si, st);
                        }
                    } else {
#pragma unroll
                        for (int p = 0; p < PASSES; ++p) {
                            mirror_pair_angle_x2<LINKED, true>(acc2[p][0], ra, rb,
                                                               fmaf((float)p, -step, vA), a, cs,
                                                               jp, JA, si, st);
                            mirror_pair_angle_x2<LINKED, true>(acc2[p][1], ra, rb,
                                                               fmaf((float)p, step, vB), a, cs,
                                                               jp, JB, si, st);
                        }
                    }
                } else if (cs.x >= 0.f) {
#pragma unroll
                    for (int p = 0; p < PASSES; ++p) {
                        mirror_pair_angle<LINKED, false, 0, 1>(acc[p], rowA, rowB,
                                                               fmaf((float)p, -step, vA), a, cs, jp,
                                                               JA, JMA, si, st);
                        mirror_pair_angle<LINKED, false, 2, 3>(acc[p], rowA, rowB,
                                                               fmaf((float)p, step, vB), a, cs, jp,
                                                               JB, JMB, si, st);
                    }
                } else {
#pragma unroll
                    for (int p = 0; p < PASSES; ++p) {
                        mirror_pair_angle<LINKED, true, 0, 1>(acc[p], rowA, rowB,
                                                              fmaf((float)p, -step, vA), a, cs, jp,
                                                              JA, JMA, si, st);
                        mirror_pair_angle<LINKED, true, 2, 3>(acc[p], rowA, rowB,
                                                              fmaf((float)p, step, vB), a, cs, jp,
                                                              JB, JMB, si, st);
                    }
                }
                rowA += si.gw;
                rowB += si.gw;
            }
        }
    }

    if constexpr (X2) {
#pragma unroll
        for (int p = 0; p < PASSES; ++p)
#pragma unroll
            for (int f = 0; f < 2; ++f)
#pragma unroll
                for (int h = 0; h < 2; ++h)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        const float2 u = unpack_x2(acc2[p][f][h][c]);
                        acc[p][2 * f][h][c] = u.x;
                        acc[p][2 * f + 1][h][c] = u.y;
                    }
    }
#pragma unroll
    for (int p = 0; p < PASSES; ++p) {
        const int r = r_t + dr0 + 16 * p, rm = n - 1 - r;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = c_t + dc + h, cm = n - 1 - c;
            const int64_t base = si.vol_off;
            if (r < hq && c < hq) adj_store<LINKED>(out, base + (int64_t)r * n + c, v, acc[p][0][h], out_mult, reg2);
            if (rm >= hq && cm >= hq) adj_store<LINKED>(out, base + (int64_t)rm * n + cm, v, acc[p][1][h], out_mult, reg2);
            if (rm >= hq && c < hq) adj_store<LINKED>(out, base + (int64_t)rm * n + c, v, acc[p][2][h], out_mult, reg2);
            if (r < hq && cm >= hq) adj_store<LINKED>(out, base + (int64_t)r * n + cm, v, acc[p][3][h], out_mult, reg2);
        }
    }
}

// LAY: 0 lanes along rows of 8 voxels, 1 lanes on 2 x 4 sub-patches, 2 voxel
// pairs along rows, 3 voxel pairs on 4 x 4 sub-patches (warps of 16 x 4), 4 the
// same sub-patches in warps of 8 x 8, 5 pairs with their mirror images, 6 the
// same over mirror-interleaved gradient rows with paired FMAs.
template <int PASSES, int LAY, bool LINKED>
__device__ __forceinline__ void backproject_item(
    const DevGeom &dg, const int *prefix, int item, AdjShared &sh, const float4 *__restrict__ gA,
    const float2 *__restrict__ gB, const float4 *__restrict__ v, float4 *__restrict__ out,
    float4 out_mult, float4 reg2, const int *__restrict__ active)
{
    if constexpr (LAY >= 5)
        backproject_mirror_item<PASSES, LINKED, LAY == 6>(dg, prefix, item, sh, gA, gB, v, out,
                                                          out_mult, reg2, active);
    else if constexpr (LAY >= 2)
        backproject_pair_item<PASSES, LINKED, LAY - 2>(dg, prefix, item, sh, gA, gB, v, out,
                                                       out_mult, reg2, active);
    else
        backproject_single_item<PASSES, LAY == 1, LINKED>(dg, prefix, item, sh, gA, gB, v, out,
                                                          out_mult, reg2, active);
}

template <int PASSES, int MINB, int LAY, bool LINKED>
__global__ void __launch_bounds__(ADJ_THREADS, MINB)
k_backproject(DevGeom dg, const int *__restrict__ prefix, const float4 *__restrict__ gA,
              const float2 *__restrict__ gB, const float4 *__restrict__ v,
              float4 *__restrict__ out, float4 out_mult, float4 reg2,
              const int *__restrict__ active)
{
    __shared__ AdjShared sh;
    backproject_item<PASSES, LAY, LINKED>(dg, prefix, blockIdx.x, sh, gA, gB, v, out, out_mult,
                                          reg2, active);
}

// Persistent: GPU-sized grid, blocks take tiles from a counter (0 before the
// launch) until the list is exhausted; no block waits on another.
template <int PASSES, int MINB, int LAY, bool LINKED>
__global__ void __launch_bounds__(ADJ_THREADS, MINB)
k_backproject_persistent(DevGeom dg, const int *__restrict__ prefix, int total, int *counter,
                         const float4 *__restrict__ gA, const float2 *__restrict__ gB,
                         const float4 *__restrict__ v, float4 *__restrict__ out,
                         float4 out_mult, float4 reg2, const int *__restrict__ active)
{
    __shared__ AdjShared sh;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= total) return;
        backproject_item<PASSES, LAY, LINKED>(dg, prefix, item, sh, gA, gB, v, out, out_mult,
                                              reg2, active);
    }
}

// Persistent, SM-chunked: the blocks resident on one SM take consecutive
// tiles (neighbouring column tiles of the same rows, whose voxels read
// neighbouring pixels) from their SM's chunk of the list, then tiles of the
// other chunks; the chunk counters are 0 before the launch.
template <int PASSES, int MINB, int LAY, bool LINKED>
__global__ void __launch_bounds__(ADJ_THREADS, MINB)
k_backproject_sm(DevGeom dg, const int *__restrict__ prefix, int total, int *counters,
                 const float4 *__restrict__ gA, const float2 *__restrict__ gB,
                 const float4 *__restrict__ v, float4 *__restrict__ out, float4 out_mult,
                 float4 reg2, const int *__restrict__ active)
{
    __shared__ AdjShared sh;
    __shared__ int s_item, s_k;
    const int sm = sm_id(), nchunk = sm_id_count();
    if (threadIdx.x == 0) s_k = 0;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = sm_chunk_next(total, counters, sm % nchunk, nchunk, &s_k);
        __syncthreads();
        const int item = s_item;
        if (item < 0) return;
        backproject_item<PASSES, LAY, LINKED>(dg, prefix, item, sh, gA, gB, v, out, out_mult,
                                              reg2, active);
    }
}

template <int P, int M, int Q, bool L>
static cudaError_t launch_bp_mode(const ei_geometry *g, const float4 *v, float4 *out,
                                  float4 out_mult, float4 reg2, const int *active, cudaStream_t st)
{
    const AdjVariant &av = g->adj_variant;
    if (av.total == 0) return cudaSuccess;
    if (g->persistent == LAUNCH_PER_ITEM) {
        k_backproject<P, M, Q, L><<<av.total, ADJ_THREADS, 0, st>>>(
            g->dg, av.prefix, g->gA, g->gB, v, out, out_mult, reg2, active);
    } else if (g->persistent == LAUNCH_SM_CHUNKS) {
        static int per_sm = 0;          // resident blocks per SM (same for every GB300)
        if (per_sm == 0)
            EI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_backproject_sm<P, M, Q, L>, ADJ_THREADS, 0));
        const int grid = std::max(1, std::min(av.total, per_sm * g->num_sms));
        EI_CUDA_TRY(cudaMemsetAsync(g->sm_counters, 0, MAX_SM_CHUNKS * sizeof(int), st));
        k_backproject_sm<P, M, Q, L><<<grid, ADJ_THREADS, 0, st>>>(
            g->dg, av.prefix, av.total, g->sm_counters, g->gA, g->gB, v, out, out_mult, reg2,
            active);
    } else {
        static int per_sm = 0;          // resident blocks per SM (same for every GB300)
        if (per_sm == 0)
            EI_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                &per_sm, k_backproject_persistent<P, M, Q, L>, ADJ_THREADS, 0));
        const int grid = std::max(1, std::min(av.total, per_sm * g->num_sms));
        EI_CUDA_TRY(cudaMemsetAsync(g->work_counter + 1, 0, sizeof(int), st));
        k_backproject_persistent<P, M, Q, L><<<grid, ADJ_THREADS, 0, st>>>(
            g->dg, av.prefix, av.total, g->work_counter + 1, g->gA, g->gB, v, out, out_mult, reg2,
            active);
    }
    return cudaGetLastError();
}

template <int P, int M, int Q>
static cudaError_t launch_bp_variant(const ei_geometry *g, const float4 *v, float4 *out,
                                     float4 out_mult, float4 reg2, float link, const int *active,
                                     cudaStream_t st)
{
    // link > 0: the linked single-channel gather over the combined sinogram
    return link > 0.f ? launch_bp_mode<P, M, Q, true>(g, v, out, out_mult, reg2, active, st)
                      : launch_bp_mode<P, M, Q, false>(g, v, out, out_mult, reg2, active, st);
}

cudaError_t launch_backproject(const ei_geometry *g, const float4 *v, float4 *out,
                               float4 out_mult, float4 reg2, float link, const int *active,
                               cudaStream_t st)
{
    switch (g->adj_variant.id) {
    case 0: return launch_bp_variant<8, 4, 0>(g, v, out, out_mult, reg2, link, active, st);
    case 1: return launch_bp_variant<4, 1, 0>(g, v, out, out_mult, reg2, link, active, st);
    case 2: return launch_bp_variant<16, 2, 0>(g, v, out, out_mult, reg2, link, active, st);
    case 3: return launch_bp_variant<8, 4, 1>(g, v, out, out_mult, reg2, link, active, st);
    case 4: return launch_bp_variant<16, 2, 1>(g, v, out, out_mult, reg2, link, active, st);
    // voxel pairs, 4 passes of 16 rows
    case 5: return launch_bp_variant<4, 4, 2>(g, v, out, out_mult, reg2, link, active, st);
    case 6: return launch_bp_variant<4, 4, 3>(g, v, out, out_mult, reg2, link, active, st);
    case 7: return launch_bp_variant<4, 4, 4>(g, v, out, out_mult, reg2, link, active, st);
    // voxel pairs with their three mirror images, quadrant tiles of 16 or 32 rows
    case 8: return launch_bp_variant<1, 4, 5>(g, v, out, out_mult, reg2, link, active, st);
    case 9: return launch_bp_variant<1, 3, 5>(g, v, out, out_mult, reg2, link, active, st);
    case 10: return launch_bp_variant<2, 2, 5>(g, v, out, out_mult, reg2, link, active, st);
    // the same with the mirror-interleaved gradient rows and paired FMAs
    case 11: return launch_bp_variant<1, 4, 6>(g, v, out, out_mult, reg2, link, active, st);
    case 12: return launch_bp_variant<1, 3, 6>(g, v, out, out_mult, reg2, link, active, st);
    default: return launch_bp_variant<2, 2, 6>(g, v, out, out_mult, reg2, link, active, st);
    }
}

// Voxel rows per tile of adjoint variant `id` (see launch_backproject).
int backproject_variant_rows(int id)
{
    static const int R[N_ADJ_VARIANTS] = {64, 32, 128, 64, 128, 64, 64, 64, 16, 16, 32, 16, 16, 32};
    return R[id];
}

// Work items (tiles) of adjoint variant `id` for an n x n slice: tiles of 32
// columns over the slice, or (the mirror variants) over its top-left quadrant.
int backproject_variant_items(int id, int n)
{
    const int tr = backproject_variant_rows(id);
    const int ext = id >= 8 ? (n + 1) / 2 : n;
    return ((ext + ADJ_TC - 1) / ADJ_TC) * ((ext + tr - 1) / tr);
}

// ----------------------------------------------------------------------------
// Packed gradient sinogram from a user sino4 array ([n_theta][n_dp] float4 per
// slice): entries of pixels j = -1 .. n_det - 1 of every row, pair-packed or
// (dg.gmirror) mirror-interleaved; the margins are zero from set-up.  One
// block per row.
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
        if (dg.gmirror) {              // pixel j and its mirror n_det - 1 - j
            const float4 d = j >= 0 ? src[j] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 m = j >= 0 ? src[si.n_det - 1 - j] : make_float4(0.f, 0.f, 0.f, 0.f);
            gA[dst + j] = make_float4(d.x, m.x, d.y, m.y);
            gB[dst + j] = make_float2(d.z, m.z);
            continue;
        }
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
// S[s] = sum over the slice's rows of part_ic (the data term) + sum over its
// blocks reg_prefix[s] .. reg_prefix[s + 1] - 1 of part_reg (the regulariser),
// one block per slice, fixed order.
// ----------------------------------------------------------------------------
__global__ void k_finalize_objective(DevGeom dg, const int *__restrict__ reg_prefix,
                                     const double *__restrict__ part_ic,
                                     const double *__restrict__ part_reg, double *__restrict__ S,
                                     const int *__restrict__ active)
{
    __shared__ double red[32];
    const int s = blockIdx.x;
    if (active && !active[s]) return;
    double acc = 0.0;
    for (int i = dg.ic_prefix[s] + threadIdx.x; i < dg.ic_prefix[s + 1]; i += blockDim.x)
        acc += part_ic[i];
    for (int i = reg_prefix[s] + threadIdx.x; i < reg_prefix[s + 1]; i += blockDim.x)
        acc += part_reg[i];
    const double tot = block_sum_double_fin(acc, red);
    if (threadIdx.x == 0) S[s] = tot;
}

cudaError_t launch_finalize_objective(const ei_geometry *g, const double *part_ic,
                                      const int *reg_prefix, const double *part_reg, double *S,
                                      const int *active, cudaStream_t st)
{
    k_finalize_objective<<<g->n_slices, 256, 0, st>>>(g->dg, reg_prefix, part_ic, part_reg, S,
                                                       active);
    return cudaGetLastError();
}

}  // namespace ei
