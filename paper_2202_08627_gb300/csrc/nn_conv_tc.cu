// Implicit-GEMM convolution of the learned warm start on the 5th-generation
// tensor cores (tcgen05, kind::f16: BF16 operands, FP32 accumulation in
// tensor memory).
//
//   Y[p][co] = sum_{tap, ci} X_tap[p][ci] W[tap][ci][co]   (+ bias, ReLU)
//
// One CTA computes a tile of 128 pixels (GEMM rows, M = 128) x NT output
// channels (N = NT <= 256).  The reduction runs over (tap, 32-channel chunk):
// every chunk, the 4 warps stage the chunk's 128 x 32 activations (the tap's
// shifted pixels, zero outside the image) and NT x 32 weights in shared memory
// in the canonical K-major layout without swizzle (core matrices of 8 rows x
// 16 bytes; 128 bytes between core matrices along K, 512 between groups of 8
// rows), then one thread issues two tcgen05.mma (K = 16 each) into the
// accumulator in tensor memory and commits them to the stage's mbarrier.
// Four stages, filled by cp.async two chunks ahead of the MMAs: the global
// loads of later chunks overlap the tensor-core work on earlier ones; a stage
// is refilled only after the MMAs that read it have completed.  The
// epilogue reads the accumulator with tcgen05.ld (each warp its 32 lanes =
// pixels), adds the bias, applies the ReLU, optionally accumulates into the
// destination, and stores BF16 NHWC; output channels below `split` go to Y1,
// the others to Y2 (dgrad into a concatenation's two inputs).
//
// Weights are read K-major, W_k[taps - 1 - tap][n][k]: for the forward pass
// that is the flipped, transposed copy the WMMA kernel uses for dgrad, and for
// dgrad (a forward convolution of dY with the flipped, transposed weights) it
// is the forward copy itself, so no extra weight layout exists.
//
// 3 x 3 layers run on k_conv3_tc (below), which stages input pixels per row
// patch (or whole halo) once for several taps; 1 x 1 layers on k_conv_tc.
// The weight gradients (k_conv_wgrad_tc, below) run on the same pipeline with
// the pixels as the reduction dimension and MN-major operand tiles.
//
// Every wait on an mbarrier is bounded (1 s); a wait that runs out sets
// *status, skips the rest of the tile, waits (bounded) for the MMAs already
// issued, frees the tensor memory and returns.
#include <cuda_bf16.h>

#include "async_copy.h"
#include "nn_internal.h"

namespace ei {
namespace nn {

namespace {

constexpr int TC_M = 128;            // pixels per CTA (tcgen05 M)
constexpr int TC_BK = 32;            // input channels per stage
// stages of the operand ring and chunks copied ahead of the MMAs (compile-time
// tunables; DEPTH < STAGES)
#ifndef EI_TC_STAGES
#define EI_TC_STAGES 4
#endif
#ifndef EI_TC_DEPTH
#define EI_TC_DEPTH 2
#endif
constexpr int TC_STAGES = EI_TC_STAGES;
constexpr uint64_t kTcWaitNs = 1000000000ull;

// shared-memory descriptor: start, LBO (K direction), SBO (8-row groups),
// version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(unsigned addr)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}

// byte offset of element (row, k) of a stage tile (k < 32)
__device__ __forceinline__ int tile_off(int row, int kg)
{
    return (row >> 3) * 512 + kg * 128 + (row & 7) * 16;
}

__device__ __forceinline__ void tc_mma(unsigned tmem_d, uint64_t ad, uint64_t bd, unsigned idesc,
                                       unsigned accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(unsigned bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_ld16(unsigned taddr, unsigned (&v)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
          "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

}  // namespace

template <int KS, int NT>
__global__ void __launch_bounds__(128)
k_conv_tc(const bf16 *__restrict__ X1, int C1, const bf16 *__restrict__ X2, int C2,
          const bf16 *__restrict__ Wk, const float *__restrict__ bias, int Cout, int B, int H,
          int W, int relu, bf16 *__restrict__ Y1, int split, int acc1, bf16 *__restrict__ Y2,
          int acc2, int *__restrict__ status)
{
    constexpr int A_BYTES = TC_M * TC_BK * 2, B_BYTES = NT * TC_BK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_mma[TC_STAGES];
    __shared__ __align__(8) uint64_t bar_done;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = B * H * W;
    const int p0 = blockIdx.x * TC_M, co0 = blockIdx.y * NT;
    const int Cin = C1 + C2;
    const int chunks = Cin / TC_BK;
    const int nK = KS * KS * chunks;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(smem_addr(&bar_mma[s]), 1);
        mbar_init(smem_addr(&bar_done), 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    // D f32, A bf16, B bf16, both K-major, N >> 3, M >> 4
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NT >> 3) << 17) |
                           ((unsigned)(TC_M >> 4) << 24);

    // this thread's pixel (row of the A tile)
    const int p = p0 + tid;
    int pb = 0, py = 0, px = 0;
    if (p < P) {
        pb = p / (H * W);
        const int r = p - pb * H * W;
        py = r / W;
        px = r - py * W;
    }
    // chunk kc into stage kc % TC_STAGES with cp.async (one commit group per chunk)
    auto issue = [&](int kc) {
        unsigned char *As = tc_smem + (kc % TC_STAGES) * STAGE_BYTES;
        unsigned char *Bs = As + A_BYTES;
        const int tap = kc / chunks, c0 = (kc - tap * chunks) * TC_BK;
        // A: 128 pixels x 32 channels of the tap's shifted input (zero outside)
        const int dy = KS == 3 ? tap / 3 - 1 : 0, dx = KS == 3 ? tap % 3 - 1 : 0;
        const int yy = py + dy, xx = px + dx;
        const bool inb = p < P && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const int64_t q = ((int64_t)pb * H + yy) * W + xx;
        const bf16 *src = X1;
        if (inb) src = c0 < C1 ? X1 + q * C1 + c0 : X2 + q * C2 + (c0 - C1);
#pragma unroll
        for (int kg = 0; kg < 4; ++kg)
            cp_async16(As + tile_off(tid, kg), inb ? src + kg * 8 : X1, inb ? 16u : 0u);
        // B: NT output channels x 32 input channels, K-major, tap flipped
        const bf16 *wsrc = Wk + ((int64_t)(KS * KS - 1 - tap) * Cout + co0) * Cin + c0;
#pragma unroll
        for (int i = 0; i < NT * 4 / 128; ++i) {
            const int e = tid + i * 128;                    // (row, kg) = (e / 4, e % 4)
            const int n = e >> 2, kg = e & 3;
            cp_async16(Bs + tile_off(n, kg), wsrc + (int64_t)n * Cin + kg * 8, 16u);
        }
    };
    constexpr int DEPTH = EI_TC_DEPTH;         // chunks in flight ahead of the MMA
    static_assert(DEPTH < TC_STAGES, "a stage must be free before its refill");
#pragma unroll
    for (int i = 0; i < DEPTH; ++i) {
        if (i < nK) issue(i);
        cp_async_commit();
    }
    bool aborted = false;
    for (int kc = 0; kc < nK; ++kc) {
        // refill: chunk kc + DEPTH into the stage that chunk kc + DEPTH - STAGES used,
        // once the MMAs that read it have completed
        bool ok = true;
        const int kn = kc + DEPTH;
        if (kn < nK) {
            if (kn >= TC_STAGES)
                ok = mbar_wait_bounded(smem_addr(&bar_mma[kn % TC_STAGES]),
                                       ((kn / TC_STAGES) - 1) & 1, kTcWaitNs);
            if (ok) issue(kn);
        }
        cp_async_commit();
        cp_async_wait<DEPTH>();                // this thread's copies of chunk kc landed
        proxy_fence_async();                   // the tensor core reads what the copies wrote
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned a_addr = smem_addr(tc_smem + (kc % TC_STAGES) * STAGE_BYTES);
            const unsigned b_addr = a_addr + A_BYTES;
            tc_mma(tmem, smem_desc(a_addr), smem_desc(b_addr), idesc, kc > 0 ? 1u : 0u);
            tc_mma(tmem, smem_desc(a_addr + 256), smem_desc(b_addr + 256), idesc, 1u);
            tc_commit(smem_addr(&bar_mma[kc % TC_STAGES]));
        }
    }
    cp_async_wait<0>();                        // no copy outlives the block
    // all issued MMAs complete -> bar_done
    if (tid == 0) tc_commit(smem_addr(&bar_done));
    const bool done = mbar_wait_bounded(smem_addr(&bar_done), 0, kTcWaitNs);
    // one decision for the whole block: the accumulator loads below are
    // warp-collective, so no lane may skip them while another takes them
    const bool failed = __syncthreads_or(aborted || !done);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (failed) {
        if (tid == 0) atomicExch(status, 1);
    } else {
        // warp w reads lanes 32w .. 32w + 31 (its pixels); the loads are
        // warp-collective, the stores only for pixels inside the image
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        for (int c = 0; c < NT; c += 16) {
            unsigned v[16];
            tc_ld16(lane_base + c, v);
            if (p >= P) continue;
            const int co = co0 + c;
            const bool first = co < split;
            bf16 *dst = first ? Y1 + (int64_t)p * split + co
                              : Y2 + (int64_t)p * (Cout - split) + (co - split);
            const int acc_mode = first ? acc1 : acc2;
            __align__(16) __nv_bfloat162 outv[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float a = __uint_as_float(v[j]), b = __uint_as_float(v[j + 1]);
                if (bias) a += bias[co + j], b += bias[co + j + 1];
                if (relu) a = fmaxf(a, 0.f), b = fmaxf(b, 0.f);
                if (acc_mode) {
                    const float2 o = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(dst)[j / 2]);
                    a += o.x, b += o.y;
                }
                outv[j / 2] = __floats2bfloat162_rn(a, b);
            }
            reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(outv)[0];
            reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(outv)[1];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

template <int KS, int NT>
static cudaError_t launch_tc(const Tensor &x1, const Tensor *x2, int cout, const bf16 *Wk,
                             const float *bias, bool relu, bf16 *y1, int split, bool acc1,
                             bf16 *y2, bool acc2, int *status, cudaStream_t st)
{
    constexpr int smem = TC_STAGES * (TC_M * TC_BK * 2 + NT * TC_BK * 2);
    // set on every launch: the attribute belongs to the current context
    EI_NN_TRY(cudaFuncSetAttribute(k_conv_tc<KS, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int P = x1.B * x1.H * x1.W;
    dim3 grid((P + TC_M - 1) / TC_M, cout / NT);
    k_conv_tc<KS, NT><<<grid, 128, smem, st>>>(x1.d, x1.C, x2 ? x2->d : nullptr, x2 ? x2->C : 0,
                                               Wk, bias, cout, x1.B, x1.H, x1.W, relu, y1, split,
                                               acc1, y2, acc2, status);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Weight gradient on the tensor cores:
//   dW[tap][ci][co] = sum_p X_tap[p][ci] G[p][co]
// as a GEMM whose rows are r = tap Cin + ci (M = 128 rows per CTA; rows past
// KS^2 Cin are zero), whose columns are the output channels (N = NT), and
// whose reduction runs over the pixels in chunks of 32, split over the grid's
// z dimension (FP32 partials, summed by k_sum_splits in a fixed order).  Both
// operands are read straight from the NHWC activations: with the pixels as the
// reduction dimension the channels are the contiguous one, so the tiles are
// MN-major (tcgen05 instruction descriptor bits 15 and 16): core matrices of
// 8 pixels x 8 channels whose 16-byte rows are 8 consecutive channels of one
// pixel, 128 bytes between core matrices along the pixels and 512 between
// groups of 8 rows, the same descriptor strides as the K-major tiles.  The
// pipeline, the bounded waits and the tensor-memory handling are those of
// k_conv_tc.
// ---------------------------------------------------------------------------
template <int KS, int NT>
__global__ void __launch_bounds__(128)
k_conv_wgrad_tc(const bf16 *__restrict__ X1, int C1, const bf16 *__restrict__ X2, int C2,
                const bf16 *__restrict__ G, int Cout, int B, int H, int W, int per_split,
                float *__restrict__ partial, int *__restrict__ status)
{
    constexpr int A_BYTES = TC_M * TC_BK * 2, B_BYTES = NT * TC_BK * 2;
    constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_mma[TC_STAGES];
    __shared__ __align__(8) uint64_t bar_done;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int P = B * H * W;
    const int Cin = C1 + C2;
    const int R = KS * KS * Cin;
    const int r0 = blockIdx.x * TC_M, co0 = blockIdx.y * NT, split = blockIdx.z;
    const int pa = split * per_split, pe = min(P, pa + per_split);
    const int nK = pe > pa ? (pe - pa + TC_BK - 1) / TC_BK : 0;

    if (tid == 0) {
        for (int s = 0; s < TC_STAGES; ++s) mbar_init(smem_addr(&bar_mma[s]), 1);
        mbar_init(smem_addr(&bar_done), 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    // D f32, A bf16, B bf16, both MN-major, N >> 3, M >> 4
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                           ((unsigned)(NT >> 3) << 17) | ((unsigned)(TC_M >> 4) << 24);

    // this thread stages, in every chunk, pixel kp of the chunk for the A row
    // groups gq, gq + 4, gq + 8, gq + 12 and the B column groups gq + 4 j
    const int kp = tid & 31, gq = tid >> 5;
    int g_dy[4], g_dx[4], g_ci[4];
    bool g_ok[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int r = r0 + 8 * (gq + 4 * i);
        g_ok[i] = r < R;
        const int tap = g_ok[i] ? r / Cin : 0;
        g_ci[i] = g_ok[i] ? r - tap * Cin : 0;
        g_dy[i] = KS == 3 ? tap / 3 - 1 : 0;
        g_dx[i] = KS == 3 ? tap % 3 - 1 : 0;
    }
    const int cell = (kp >> 3) * 128 + (kp & 7) * 16;       // this pixel's 16 bytes in a row group
    auto issue = [&](int kc) {
        unsigned char *As = tc_smem + (kc % TC_STAGES) * STAGE_BYTES;
        unsigned char *Bs = As + A_BYTES;
        const int p = pa + kc * TC_BK + kp;
        const bool pin = p < pe;
        int pb = 0, py = 0, px = 0;
        if (pin) {
            pb = p / (H * W);
            const int rr = p - pb * H * W;
            py = rr / W;
            px = rr - py * W;
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int yy = py + g_dy[i], xx = px + g_dx[i];
            const bool inb = pin && g_ok[i] && yy >= 0 && yy < H && xx >= 0 && xx < W;
            const int64_t q = ((int64_t)pb * H + yy) * W + xx;
            const int ci = g_ci[i];
            const bf16 *src = X1;
            if (inb) src = ci < C1 ? X1 + q * C1 + ci : X2 + q * C2 + (ci - C1);
            cp_async16(As + (gq + 4 * i) * 512 + cell, src, inb ? 16u : 0u);
        }
#pragma unroll
        for (int j = 0; j < NT / 32; ++j) {
            const int g = gq + 4 * j;
            cp_async16(Bs + g * 512 + cell, pin ? G + (int64_t)p * Cout + co0 + 8 * g : G,
                       pin ? 16u : 0u);
        }
    };
    constexpr int DEPTH = EI_TC_DEPTH;         // chunks in flight ahead of the MMA
    static_assert(DEPTH < TC_STAGES, "a stage must be free before its refill");
#pragma unroll
    for (int i = 0; i < DEPTH; ++i) {
        if (i < nK) issue(i);
        cp_async_commit();
    }
    bool aborted = false;
    for (int kc = 0; kc < nK; ++kc) {
        bool ok = true;
        const int kn = kc + DEPTH;
        if (kn < nK) {
            if (kn >= TC_STAGES)
                ok = mbar_wait_bounded(smem_addr(&bar_mma[kn % TC_STAGES]),
                                       ((kn / TC_STAGES) - 1) & 1, kTcWaitNs);
            if (ok) issue(kn);
        }
        cp_async_commit();
        cp_async_wait<DEPTH>();
        proxy_fence_async();
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned a_addr = smem_addr(tc_smem + (kc % TC_STAGES) * STAGE_BYTES);
            const unsigned b_addr = a_addr + A_BYTES;
            tc_mma(tmem, smem_desc(a_addr), smem_desc(b_addr), idesc, kc > 0 ? 1u : 0u);
            tc_mma(tmem, smem_desc(a_addr + 256), smem_desc(b_addr + 256), idesc, 1u);
            tc_commit(smem_addr(&bar_mma[kc % TC_STAGES]));
        }
    }
    cp_async_wait<0>();
    bool done = true;
    if (nK > 0) {
        if (tid == 0) tc_commit(smem_addr(&bar_done));
        done = mbar_wait_bounded(smem_addr(&bar_done), 0, kTcWaitNs);
    }
    const bool failed = __syncthreads_or(aborted || !done);   // block-uniform, as above
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int r = r0 + warp * 32 + (tid & 31);                // this thread's row (its lane)
    float *dst = partial + ((int64_t)split * R + r) * Cout + co0;
    if (failed) {
        if (tid == 0) atomicExch(status, 1);
    } else if (nK == 0) {                      // an empty pixel range: zero partials
        if (r < R)
            for (int c = 0; c < NT; c += 4) reinterpret_cast<float4 *>(dst + c)[0] = make_float4(0.f, 0.f, 0.f, 0.f);
    } else {
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        for (int c = 0; c < NT; c += 16) {
            unsigned v[16];
            tc_ld16(lane_base + c, v);
            if (r >= R) continue;
#pragma unroll
            for (int j = 0; j < 16; j += 4)
                reinterpret_cast<float4 *>(dst + c + j)[0] =
                    make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]),
                                __uint_as_float(v[j + 2]), __uint_as_float(v[j + 3]));
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

template <int KS, int NT>
static cudaError_t launch_wgrad_tc(const Tensor &x1, const Tensor *x2, const bf16 *g, int cout,
                                   float *partial, int nsplit, int *status, cudaStream_t st)
{
    constexpr int smem = TC_STAGES * (TC_M * TC_BK * 2 + NT * TC_BK * 2);
    // set on every launch: the attribute belongs to the current context
    EI_NN_TRY(cudaFuncSetAttribute(k_conv_wgrad_tc<KS, NT>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int P = x1.B * x1.H * x1.W;
    const int cin = x1.C + (x2 ? x2->C : 0);
    const int R = KS * KS * cin;
    const int per = ((P + nsplit - 1) / nsplit + TC_BK - 1) / TC_BK * TC_BK;
    dim3 grid((R + TC_M - 1) / TC_M, cout / NT, nsplit);
    k_conv_wgrad_tc<KS, NT><<<grid, 128, smem, st>>>(x1.d, x1.C, x2 ? x2->d : nullptr,
                                                     x2 ? x2->C : 0, g, cout, x1.B, x1.H, x1.W,
                                                     per, partial, status);
    return cudaGetLastError();
}

// ----------------------------------------------------------------------------
// 3 x 3 convolutions by row patches.  A CTA computes 16 output rows x 8
// output columns of one image (GEMM rows r = 8 y + x, M = 128) x NT output
// channels.  The reduction runs over (32-channel chunk, kernel row dy): a stage
// holds the 16 x 10 input pixels of the chunk at rows y + dy, columns
// x - 1 .. x + 8, in the K-major no-swizzle layout (core matrices of 8
// consecutive pixels of a row x 16 bytes; 2560 bytes between 8-channel groups,
// 160 between output rows), and the three taps' weights.  Tap dx's A operand
// is the same tile started dx + 1 pixels (16 bytes each) further, so an input
// pixel is staged 3 times instead of 9 (once per tap) and each stage feeds 6
// MMAs instead of 2.  Partial patches at the image's bottom and right edges
// read zeros and store nothing for the missing pixels.
// ----------------------------------------------------------------------------
constexpr int C3_PR = 16, C3_PC = 8, C3_PW = C3_PC + 2;   // patch rows, columns, staged columns
constexpr int C3_LBO = C3_PR * C3_PW * 16;                // 2560: next 8 input channels
constexpr int C3_SBO = C3_PW * 16;                        // 160: next output row
constexpr int C3_A_BYTES = 4 * C3_LBO;                    // 10240: 32 channels
static_assert(C3_PR * C3_PC == TC_M, "a patch is one tcgen05 M tile");

#ifndef EI_C3_STAGES
#define EI_C3_STAGES 3               // stages (measured: 3 beats 4, more resident CTAs)
#endif
// HALO: a stage holds one 32-channel chunk's 18 x 10 input pixels (rows
// y - 1 .. y + 16) and all nine taps' weights; tap (dy, dx) reads the tile
// started dy + 1 rows and dx + 1 pixels further, so each input pixel is staged
// once per chunk and a stage feeds 18 MMAs.
constexpr int C3H_LBO = (C3_PR + 2) * C3_PW * 16;         // 2880
constexpr int C3H_A_BYTES = 4 * C3H_LBO;                  // 11520
#ifndef EI_C3_HALO_MAXNT
#define EI_C3_HALO_MAXNT 64          // largest NT that stages whole halos (0: none)
#endif
template <int NT, bool HALO = false>
struct Conv3Shape {
    static constexpr int kStages = HALO ? (NT >= 64 ? 2 : 3) : (NT >= 256 ? 3 : EI_C3_STAGES);
    static constexpr int kTaps = HALO ? 9 : 3;
    static constexpr int kLBO = HALO ? C3H_LBO : C3_LBO;
    static constexpr int kABytes = HALO ? C3H_A_BYTES : C3_A_BYTES;
    static constexpr int kBTap = NT * TC_BK * 2;
    static constexpr int kStageBytes = kABytes + kTaps * kBTap;
    static constexpr int kSmem = kStages * kStageBytes;
};

// shared-memory descriptor with explicit strides (no swizzle)
__device__ __forceinline__ uint64_t smem_desc_s(unsigned addr, int lbo, int sbo)
{
    return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

template <int NT, bool HALO>
__global__ void __launch_bounds__(128)
k_conv3_tc(const bf16 *__restrict__ X1, int C1, const bf16 *__restrict__ X2, int C2,
           const bf16 *__restrict__ Wk, const float *__restrict__ bias, int Cout, int B, int H,
           int W, int relu, bf16 *__restrict__ Y1, int split, int acc1, bf16 *__restrict__ Y2,
           int acc2, int *__restrict__ status)
{
    using S = Conv3Shape<NT, HALO>;
    constexpr int STAGES = S::kStages;
    extern __shared__ __align__(1024) unsigned char tc_smem[];
    __shared__ __align__(8) uint64_t bar_mma[STAGES];
    __shared__ __align__(8) uint64_t bar_done;
    __shared__ unsigned tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5;
    const int tiles_y = (H + C3_PR - 1) / C3_PR, tiles_x = (W + C3_PC - 1) / C3_PC;
    const int t_img = blockIdx.x / (tiles_y * tiles_x), t_rem = blockIdx.x - t_img * tiles_y * tiles_x;
    const int y0 = (t_rem / tiles_x) * C3_PR, x0 = (t_rem % tiles_x) * C3_PC;
    const int co0 = blockIdx.y * NT;
    const int Cin = C1 + C2;
    const int chunks = Cin / TC_BK;
    const int nK = HALO ? chunks : 3 * chunks;

    if (tid == 0) {
        for (int s = 0; s < STAGES; ++s) mbar_init(smem_addr(&bar_mma[s]), 1);
        mbar_init(smem_addr(&bar_done), 1);
        mbar_init_fence();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_base)),
                     "r"(NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const unsigned tmem = tmem_base;
    // D f32, A bf16, B bf16, both K-major, N >> 3, M >> 4
    const unsigned idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(NT >> 3) << 17) |
                           ((unsigned)(TC_M >> 4) << 24);

    // stage kc = (chunk kc / 3, kernel row dy = kc % 3 - 1), cp.async, one commit group each
    auto issue = [&](int kc) {
        unsigned char *As = tc_smem + (kc % STAGES) * S::kStageBytes;
        unsigned char *Bs = As + S::kABytes;
        const int c = HALO ? kc : kc / 3, dyi = HALO ? 0 : kc - 3 * c, dy = dyi - 1;
        const int c0 = c * TC_BK;
        // A: 16 (HALO: 18) x 10 pixels x 32 channels (zero outside the image)
        constexpr int AROWS = HALO ? C3_PR + 2 : C3_PR;
        for (int e = tid; e < AROWS * C3_PW * 4; e += 128) {
            const int pi = e >> 2, kg = e & 3;
            const int yy = pi / C3_PW, xx = pi - yy * C3_PW;
            const int iy = y0 + yy + dy, ix = x0 + xx - 1;
            const bool inb = iy >= 0 && iy < H && ix >= 0 && ix < W;
            const int64_t q = ((int64_t)t_img * H + iy) * W + ix;
            const bf16 *src = X1;
            if (inb) src = c0 < C1 ? X1 + q * C1 + c0 : X2 + q * C2 + (c0 - C1);
            cp_async16(As + kg * S::kLBO + pi * 16, inb ? src + kg * 8 : X1, inb ? 16u : 0u);
        }
        // B: the three taps (dy, dx = -1, 0, 1), NT output x 32 input channels,
        // K-major, tap flipped as in k_conv_tc
#pragma unroll
        for (int t = 0; t < S::kTaps; ++t) {
            const int tap = HALO ? t : dyi * 3 + t;
            const bf16 *wsrc = Wk + ((int64_t)(8 - tap) * Cout + co0) * Cin + c0;
            unsigned char *Bt = Bs + t * S::kBTap;
#pragma unroll
            for (int i = 0; i < NT * 4 / 128; ++i) {
                const int e = tid + i * 128;
                const int n = e >> 2, kg = e & 3;
                cp_async16(Bt + tile_off(n, kg), wsrc + (int64_t)n * Cin + kg * 8, 16u);
            }
        }
    };
    constexpr int DEPTH = EI_TC_DEPTH < STAGES ? EI_TC_DEPTH : STAGES - 1;
    static_assert(DEPTH < STAGES, "a stage must be free before its refill");
#pragma unroll
    for (int i = 0; i < DEPTH; ++i) {
        if (i < nK) issue(i);
        cp_async_commit();
    }
    bool aborted = false;
    for (int kc = 0; kc < nK; ++kc) {
        bool ok = true;
        const int kn = kc + DEPTH;
        if (kn < nK) {
            if (kn >= STAGES)
                ok = mbar_wait_bounded(smem_addr(&bar_mma[kn % STAGES]), ((kn / STAGES) - 1) & 1,
                                       kTcWaitNs);
            if (ok) issue(kn);
        }
        cp_async_commit();
        cp_async_wait<DEPTH>();                // this thread's copies of stage kc landed
        proxy_fence_async();                   // the tensor core reads what the copies wrote
        if (__syncthreads_or(!ok)) {
            aborted = true;
            break;
        }
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const unsigned a_addr = smem_addr(tc_smem + (kc % STAGES) * S::kStageBytes);
            const unsigned b_addr = a_addr + S::kABytes;
#pragma unroll
            for (int t = 0; t < S::kTaps; ++t) {
                // tap t's tile: HALO (dy, dx) = (t / 3 - 1, t % 3 - 1) starts dy + 1 rows
                // and dx + 1 pixels into the halo; otherwise dx = t - 1
                const unsigned at = a_addr + (HALO ? (t / 3) * C3_SBO + (t % 3) * 16 : t * 16);
                const unsigned bt = b_addr + t * S::kBTap;
                tc_mma(tmem, smem_desc_s(at, S::kLBO, C3_SBO), smem_desc(bt), idesc,
                       kc > 0 || t > 0 ? 1u : 0u);
                tc_mma(tmem, smem_desc_s(at + 2 * S::kLBO, S::kLBO, C3_SBO), smem_desc(bt + 256),
                       idesc, 1u);
            }
            tc_commit(smem_addr(&bar_mma[kc % STAGES]));
        }
    }
    cp_async_wait<0>();                        // no copy outlives the block
    if (tid == 0) tc_commit(smem_addr(&bar_done));
    const bool done = mbar_wait_bounded(smem_addr(&bar_done), 0, kTcWaitNs);
    const bool failed = __syncthreads_or(aborted || !done);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (failed) {
        if (tid == 0) atomicExch(status, 1);
    } else {
        // warp w reads lanes 32w .. 32w + 31 (rows r = 8 y + x); the loads are
        // warp-collective, the stores only for pixels inside the image
        const int r = tid, yy = y0 + (r >> 3), xx = x0 + (r & 7);
        const bool in = yy < H && xx < W;
        const int64_t p = ((int64_t)t_img * H + yy) * W + xx;
        const unsigned lane_base = tmem + ((unsigned)(warp * 32) << 16);
        for (int c = 0; c < NT; c += 16) {
            unsigned v[16];
            tc_ld16(lane_base + c, v);
            if (!in) continue;
            const int co = co0 + c;
            const bool first = co < split;
            bf16 *dst = first ? Y1 + p * split + co : Y2 + p * (Cout - split) + (co - split);
            const int acc_mode = first ? acc1 : acc2;
            __align__(16) __nv_bfloat162 outv[8];
#pragma unroll
            for (int j = 0; j < 16; j += 2) {
                float a = __uint_as_float(v[j]), b = __uint_as_float(v[j + 1]);
                if (bias) a += bias[co + j], b += bias[co + j + 1];
                if (relu) a = fmaxf(a, 0.f), b = fmaxf(b, 0.f);
                if (acc_mode) {
                    const float2 o = __bfloat1622float2(reinterpret_cast<const __nv_bfloat162 *>(dst)[j / 2]);
                    a += o.x, b += o.y;
                }
                outv[j / 2] = __floats2bfloat162_rn(a, b);
            }
            reinterpret_cast<uint4 *>(dst)[0] = reinterpret_cast<const uint4 *>(outv)[0];
            reinterpret_cast<uint4 *>(dst)[1] = reinterpret_cast<const uint4 *>(outv)[1];
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NT));
}

template <int NT>
static cudaError_t launch_conv3_tc(const Tensor &x1, const Tensor *x2, int cout, const bf16 *Wk,
                                   const float *bias, bool relu, bf16 *y1, int split, bool acc1,
                                   bf16 *y2, bool acc2, int *status, cudaStream_t st)
{
    constexpr bool HALO = NT <= EI_C3_HALO_MAXNT;
    constexpr int smem = Conv3Shape<NT, HALO>::kSmem;
    // set on every launch: the attribute belongs to the current context
    EI_NN_TRY(cudaFuncSetAttribute(k_conv3_tc<NT, HALO>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    const int tiles = ((x1.H + C3_PR - 1) / C3_PR) * ((x1.W + C3_PC - 1) / C3_PC);
    dim3 grid(x1.B * tiles, cout / NT);
    k_conv3_tc<NT, HALO><<<grid, 128, smem, st>>>(x1.d, x1.C, x2 ? x2->d : nullptr, x2 ? x2->C : 0, Wk,
                                            bias, cout, x1.B, x1.H, x1.W, relu, y1, split, acc1, y2,
                                            acc2, status);
    return cudaGetLastError();
}

bool wgrad_tc_supported(int cin, int cout, int c1)
{
    const int nt = cout >= 256 ? 256 : cout;
    return cin % TC_BK == 0 && c1 % 8 == 0 && (nt == 32 || nt == 64 || nt == 128 || nt == 256) &&
           cout % nt == 0;
}

cudaError_t conv_wgrad_tc(const Tensor &x1, const Tensor *x2, const bf16 *g, int cout, int ks,
                          float *partial, int nsplit, int *status, cudaStream_t st)
{
    const int nt = cout >= 256 ? 256 : cout;
#define EI_WG_CASE(K, N)                                                                     \
    if (ks == K && nt == N) return launch_wgrad_tc<K, N>(x1, x2, g, cout, partial, nsplit, status, st);
    EI_WG_CASE(3, 32) EI_WG_CASE(3, 64) EI_WG_CASE(3, 128) EI_WG_CASE(3, 256)
    EI_WG_CASE(1, 32) EI_WG_CASE(1, 64) EI_WG_CASE(1, 128) EI_WG_CASE(1, 256)
#undef EI_WG_CASE
    return cudaErrorInvalidValue;
}

bool conv_tc_supported(int cin, int cout, int c1, int split)
{
    const int nt = cout >= 256 ? 256 : cout;
    return cin % TC_BK == 0 && c1 % TC_BK == 0 && split % 16 == 0 &&
           (nt == 32 || nt == 64 || nt == 128 || nt == 256) && cout % nt == 0;
}

cudaError_t conv_forward_tc(const Tensor &x1, const Tensor *x2, int cout, int ks, const bf16 *Wk,
                            const float *bias, bool relu, bf16 *y1, int split, bool acc1, bf16 *y2,
                            bool acc2, int *status, cudaStream_t st)
{
    const int nt = cout >= 256 ? 256 : cout;
#define EI_TC_CASE(K, N)                                                                     \
    if (ks == K && nt == N)                                                                  \
        return launch_tc<K, N>(x1, x2, cout, Wk, bias, relu, y1, split, acc1, y2, acc2, status, st);
#ifndef EI_CONV3_TAPWISE
    // 3 x 3: row patches (each input pixel staged once per kernel row)
    if (ks == 3) {
        if (nt == 32) return launch_conv3_tc<32>(x1, x2, cout, Wk, bias, relu, y1, split, acc1, y2, acc2, status, st);
        if (nt == 64) return launch_conv3_tc<64>(x1, x2, cout, Wk, bias, relu, y1, split, acc1, y2, acc2, status, st);
        if (nt == 128) return launch_conv3_tc<128>(x1, x2, cout, Wk, bias, relu, y1, split, acc1, y2, acc2, status, st);
        if (nt == 256) return launch_conv3_tc<256>(x1, x2, cout, Wk, bias, relu, y1, split, acc1, y2, acc2, status, st);
    }
#endif
    EI_TC_CASE(3, 32) EI_TC_CASE(3, 64) EI_TC_CASE(3, 128) EI_TC_CASE(3, 256)
    EI_TC_CASE(1, 32) EI_TC_CASE(1, 64) EI_TC_CASE(1, 128) EI_TC_CASE(1, 256)
#undef EI_TC_CASE
    return cudaErrorInvalidValue;
}

}  // namespace nn
}  // namespace ei
