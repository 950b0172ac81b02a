// Kernels of the learned warm start: a small U-Net on NHWC BF16 activations
// with FP32 accumulation (tensor cores through WMMA 16x16x16 BF16 fragments).
//
// Convolutions are implicit GEMMs (no im2col buffer):
//   forward  Y[p][co] = sum_{tap, ci} X_tap[p][ci] W[tap][ci][co]    (+ bias, ReLU)
//   dgrad    dX[p][ci] = sum_{tap, co} dY_{flip tap}[p][co] W[tap][ci][co]
//            (the forward kernel on the flipped, transposed weights)
//   wgrad    dW[tap][ci][co] = sum_p X_tap[p][ci] dY[p][co]        (split over pixels,
//            partial tiles summed in a fixed order: deterministic)
// X_tap is the input shifted by the tap's offset with zero padding.  A
// convolution can read its input channels from two tensors (the decoder's
// concatenation of the upsampled path and the skip connection), and dgrad can
// write its two channel ranges to two tensors, so no concatenated copy exists.
#include <cuda_bf16.h>
#include <mma.h>

#include "nn_internal.h"

namespace ei {
namespace nn {

using namespace nvcuda;
typedef __nv_bfloat16 bf16;

constexpr int CONV_BM = 128;     // pixels per block
constexpr int CONV_BN = 32;      // output channels per block
constexpr int CONV_BK = 16;      // input channels per step
constexpr int A_LD = CONV_BK + 8;
constexpr int B_LD = CONV_BN + 8;
constexpr int C_LD = CONV_BN + 4;

// ---------------------------------------------------------------------------
// Forward convolution (also dgrad).  Grid (ceil(P / 128), Cout / 32), 128 threads.
// ---------------------------------------------------------------------------
template <int KS>
__global__ void __launch_bounds__(128)
k_conv(const bf16 *__restrict__ X1, int C1, const bf16 *__restrict__ X2, int C2,
       const bf16 *__restrict__ Wt, const float *__restrict__ bias, int Cout, int B, int H, int W,
       int relu, bf16 *__restrict__ Y1, int split, int acc1, bf16 *__restrict__ Y2, int acc2)
{
    __shared__ __align__(32) bf16 As[CONV_BM * A_LD];
    __shared__ __align__(32) bf16 Bs[CONV_BK * B_LD];
    __shared__ __align__(32) float Cs[CONV_BM * C_LD];
    const int P = B * H * W;
    const int p0 = blockIdx.x * CONV_BM, co0 = blockIdx.y * CONV_BN;
    const int warp = threadIdx.x >> 5;
    const int Cin = C1 + C2;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc[2][2];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j) wmma::fill_fragment(acc[i][j], 0.f);

    // this thread's pixel for the A loads
    const int p = p0 + threadIdx.x;
    int pb = 0, py = 0, px = 0;
    if (p < P) {
        pb = p / (H * W);
        const int r = p - pb * H * W;
        py = r / W;
        px = r - py * W;
    }
    for (int tap = 0; tap < KS * KS; ++tap) {
        const int dy = KS == 3 ? tap / 3 - 1 : 0, dx = KS == 3 ? tap % 3 - 1 : 0;
        const int yy = py + dy, xx = px + dx;
        const bool inb = p < P && yy >= 0 && yy < H && xx >= 0 && xx < W;
        const int64_t q = ((int64_t)pb * H + yy) * W + xx;
        for (int c0 = 0; c0 < Cin; c0 += CONV_BK) {
            // A: 128 pixels x 16 channels
            uint4 v0 = make_uint4(0, 0, 0, 0), v1 = v0;
            if (inb) {
                const bf16 *src = c0 < C1 ? X1 + q * C1 + c0 : X2 + q * C2 + (c0 - C1);
                v0 = *reinterpret_cast<const uint4 *>(src);
                v1 = *reinterpret_cast<const uint4 *>(src + 8);
            }
            *reinterpret_cast<uint4 *>(As + threadIdx.x * A_LD) = v0;
            *reinterpret_cast<uint4 *>(As + threadIdx.x * A_LD + 8) = v1;
            // B: 16 input channels x 32 output channels (8 bytes per thread)
            {
                const int r = threadIdx.x >> 3, c = (threadIdx.x & 7) * 4;
                const bf16 *src = Wt + ((int64_t)tap * Cin + c0 + r) * Cout + co0 + c;
                *reinterpret_cast<uint2 *>(Bs + r * B_LD + c) = *reinterpret_cast<const uint2 *>(src);
            }
            __syncthreads();
            wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::row_major> fa[2];
            wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb[2];
#pragma unroll
            for (int i = 0; i < 2; ++i) wmma::load_matrix_sync(fa[i], As + (warp * 32 + i * 16) * A_LD, A_LD);
#pragma unroll
            for (int j = 0; j < 2; ++j) wmma::load_matrix_sync(fb[j], Bs + j * 16, B_LD);
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 2; ++j) wmma::mma_sync(acc[i][j], fa[i], fb[j], acc[i][j]);
            __syncthreads();
        }
    }
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 2; ++j)
            wmma::store_matrix_sync(Cs + (warp * 32 + i * 16) * C_LD + j * 16, acc[i][j], C_LD,
                                    wmma::mem_row_major);
    __syncthreads();
    if (p < P) {
        // output channels [co0, co0 + 32) of pixel p: to Y1 below `split`, to Y2 above
        const bool first = co0 < split;
        bf16 *dst = first ? Y1 + (int64_t)p * split + co0
                          : Y2 + (int64_t)p * (Cout - split) + (co0 - split);
        const int acc_mode = first ? acc1 : acc2;
        for (int c = 0; c < CONV_BN; c += 2) {
            float a = Cs[threadIdx.x * C_LD + c], b = Cs[threadIdx.x * C_LD + c + 1];
            if (bias) a += bias[co0 + c], b += bias[co0 + c + 1];
            if (relu) a = fmaxf(a, 0.f), b = fmaxf(b, 0.f);
            __nv_bfloat162 *d2 = reinterpret_cast<__nv_bfloat162 *>(dst + c);
            if (acc_mode) {
                const float2 o = __bfloat1622float2(*d2);
                a += o.x, b += o.y;
            }
            *d2 = __floats2bfloat162_rn(a, b);
        }
    }
}

// ---------------------------------------------------------------------------
// Weight gradient: partial[split][tap][ci][co] over a pixel range.
// Grid (Cin/32 * Cout/32, KS*KS, nsplit), 128 threads: 4 warps = 2 x 2
// fragments of the 32 x 32 tile.
// ---------------------------------------------------------------------------
template <int KS>
__global__ void __launch_bounds__(128)
k_conv_wgrad(const bf16 *__restrict__ X1, int C1, const bf16 *__restrict__ X2, int C2,
             const bf16 *__restrict__ G, int Cout, int B, int H, int W, int per_split,
             float *__restrict__ partial)
{
    __shared__ __align__(32) bf16 Xs[16 * (32 + 8)];
    __shared__ __align__(32) bf16 Gs[16 * (32 + 8)];
    const int Cin = C1 + C2;
    const int nco = Cout / 32;
    const int ci0 = (blockIdx.x / nco) * 32, co0 = (blockIdx.x % nco) * 32;
    const int tap = blockIdx.y, split = blockIdx.z;
    const int dy = KS == 3 ? tap / 3 - 1 : 0, dx = KS == 3 ? tap % 3 - 1 : 0;
    const int P = B * H * W;
    const int pa = split * per_split, pe = min(P, pa + per_split);
    const int warp = threadIdx.x >> 5;
    const int fi = warp >> 1, fj = warp & 1;
    wmma::fragment<wmma::accumulator, 16, 16, 16, float> acc;
    wmma::fill_fragment(acc, 0.f);
    for (int pc = pa; pc < pe; pc += 16) {
        // 16 pixels x 32 input channels (shifted input) and x 32 output-gradient channels
        {
            const int r = threadIdx.x >> 3, c = (threadIdx.x & 7) * 4;   // 16 rows x 8 quads
            const int p = pc + r;
            uint2 xv = make_uint2(0, 0), gv = make_uint2(0, 0);
            if (p < pe) {
                const int b = p / (H * W), rr = p - b * H * W, y = rr / W, x = rr - y * W;
                const int yy = y + dy, xx = x + dx;
                if (yy >= 0 && yy < H && xx >= 0 && xx < W) {
                    const int64_t q = ((int64_t)b * H + yy) * W + xx;
                    const int ci = ci0 + c;
                    const bf16 *src = ci < C1 ? X1 + q * C1 + ci : X2 + q * C2 + (ci - C1);
                    xv = *reinterpret_cast<const uint2 *>(src);
                }
                gv = *reinterpret_cast<const uint2 *>(G + (int64_t)p * Cout + co0 + c);
            }
            *reinterpret_cast<uint2 *>(Xs + r * 40 + c) = xv;
            *reinterpret_cast<uint2 *>(Gs + r * 40 + c) = gv;
        }
        __syncthreads();
        // C[ci][co] += sum_p Xs[p][ci] Gs[p][co]: A = Xs^T (col-major), B = Gs (row-major)
        wmma::fragment<wmma::matrix_a, 16, 16, 16, bf16, wmma::col_major> fa;
        wmma::fragment<wmma::matrix_b, 16, 16, 16, bf16, wmma::row_major> fb;
        wmma::load_matrix_sync(fa, Xs + fi * 16, 40);
        wmma::load_matrix_sync(fb, Gs + fj * 16, 40);
        wmma::mma_sync(acc, fa, fb, acc);
        __syncthreads();
    }
    float *dst = partial + (((int64_t)split * KS * KS + tap) * Cin + ci0 + fi * 16) * Cout + co0 + fj * 16;
    wmma::store_matrix_sync(dst, acc, Cout, wmma::mem_row_major);
}

// out[i] = sum_s partial[s][i] (fixed order)
__global__ void k_sum_splits(const float *__restrict__ partial, int nsplit, int64_t n,
                             float *__restrict__ out, int accumulate)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        float a = 0.f;
        for (int s = 0; s < nsplit; ++s) a += partial[(int64_t)s * n + i];
        out[i] = accumulate ? out[i] + a : a;
    }
}

// dbias partials: block b sums pixels [b per, (b+1) per) of every channel;
// with 256 threads and C | 256, thread t always meets channel t % C
__global__ void k_bias_grad(const bf16 *__restrict__ G, int C, int64_t P, int64_t per,
                            float *__restrict__ partial)
{
    __shared__ float red[256];
    const int64_t p0 = blockIdx.x * per, p1 = min(P, p0 + per);
    float a = 0.f;
    for (int64_t i = p0 * C + threadIdx.x; i < p1 * C; i += blockDim.x) a += __bfloat162float(G[i]);
    red[threadIdx.x] = a;
    __syncthreads();
    if ((int)threadIdx.x < C) {
        float s = 0.f;
        for (int k = threadIdx.x; k < (int)blockDim.x; k += C) s += red[k];
        partial[(int64_t)blockIdx.x * C + threadIdx.x] = s;
    }
}

// Wf[flip tap][co][ci] = W[tap][ci][co] (dgrad weights) and the BF16 copy of W.
__global__ void k_prepare_weights(const float *__restrict__ Wm, int taps, int Cin, int Cout,
                                  bf16 *__restrict__ Wb, bf16 *__restrict__ Wf)
{
    const int64_t n = (int64_t)taps * Cin * Cout;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int co = (int)(i % Cout);
        const int ci = (int)((i / Cout) % Cin);
        const int t = (int)(i / ((int64_t)Cout * Cin));
        const bf16 v = __float2bfloat16_rn(Wm[i]);
        Wb[i] = v;
        Wf[((int64_t)(taps - 1 - t) * Cout + co) * Cin + ci] = v;
    }
}

// ---------------------------------------------------------------------------
// Elementwise and small kernels
// ---------------------------------------------------------------------------
// x: FP32 NHWC with 3 channels -> BF16 NHWC with 32 channels (zeros beyond 3)
__global__ void k_pack_input(const float *__restrict__ x, int64_t P, bf16 *__restrict__ y)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        __align__(16) bf16 v[32];
        for (int c = 0; c < 32; ++c) v[c] = __float2bfloat16_rn(c < 3 ? x[p * 3 + c] : 0.f);
        for (int k = 0; k < 4; ++k)
            reinterpret_cast<uint4 *>(y + p * 32)[k] = reinterpret_cast<uint4 *>(v)[k];
    }
}

// 2x2 average pooling, NHWC (H, W even)
__global__ void k_pool2(const bf16 *__restrict__ x, int B, int H, int W, int C, bf16 *__restrict__ y)
{
    const int Ho = H / 2, Wo = W / 2;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        int64_t r = i / C;
        const int xo = (int)(r % Wo);
        r /= Wo;
        const int yo = (int)(r % Ho);
        const int b = (int)(r / Ho);
        const int64_t base = (((int64_t)b * H + 2 * yo) * W + 2 * xo) * C + c;
        const float s = __bfloat162float(x[base]) + __bfloat162float(x[base + C]) +
                        __bfloat162float(x[base + (int64_t)W * C]) +
                        __bfloat162float(x[base + (int64_t)W * C + C]);
        y[i] = __float2bfloat16_rn(0.25f * s);
    }
}

// backward of the pooling: gx (+)= gy / 4 at each of the 4 inputs
__global__ void k_pool2_back(const bf16 *__restrict__ gy, int B, int H, int W, int C,
                             bf16 *__restrict__ gx, int accumulate)
{
    const int64_t n = (int64_t)B * H * W * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        int64_t r = i / C;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const int b = (int)(r / H);
        float v = 0.25f * __bfloat162float(gy[(((int64_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c]);
        if (accumulate) v += __bfloat162float(gx[i]);
        gx[i] = __float2bfloat16_rn(v);
    }
}

// nearest 2x upsampling: y[2i+a][2j+b] = x[i][j]
__global__ void k_up2(const bf16 *__restrict__ x, int B, int H, int W, int C, bf16 *__restrict__ y)
{
    const int Ho = 2 * H, Wo = 2 * W;
    const int64_t n = (int64_t)B * Ho * Wo * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        int64_t r = i / C;
        const int xo = (int)(r % Wo);
        r /= Wo;
        const int yo = (int)(r % Ho);
        const int b = (int)(r / Ho);
        y[i] = x[(((int64_t)b * H + yo / 2) * W + xo / 2) * C + c];
    }
}

// backward of the upsampling: gx = sum of the 4 copies
__global__ void k_up2_back(const bf16 *__restrict__ gy, int B, int H, int W, int C, bf16 *__restrict__ gx)
{
    const int64_t n = (int64_t)B * H * W * C;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i % C);
        int64_t r = i / C;
        const int x = (int)(r % W);
        r /= W;
        const int y = (int)(r % H);
        const int b = (int)(r / H);
        const int64_t base = (((int64_t)b * 2 * H + 2 * y) * 2 * W + 2 * x) * C + c;
        const int64_t row = (int64_t)2 * W * C;
        const float s = __bfloat162float(gy[base]) + __bfloat162float(gy[base + C]) +
                        __bfloat162float(gy[base + row]) + __bfloat162float(gy[base + row + C]);
        gx[i] = __float2bfloat16_rn(s);
    }
}

// g *= (y > 0): backward of a ReLU, in place
__global__ void k_relu_mask(bf16 *__restrict__ g, const bf16 *__restrict__ y, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!(__bfloat162float(y[i]) > 0.f)) g[i] = __float2bfloat16_rn(0.f);
}

// head: out[p][k] = x_in[p][k] + b[k] + sum_c h[p][c] w[c][k]   (1x1 conv, FP32 out, 3 channels)
__global__ void k_head(const bf16 *__restrict__ h, int C, const float *__restrict__ w,
                       const float *__restrict__ b, const float *__restrict__ xin, int64_t P,
                       float *__restrict__ out)
{
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        float o0 = b[0], o1 = b[1], o2 = b[2];
        for (int c = 0; c < C; ++c) {
            const float v = __bfloat162float(h[p * C + c]);
            o0 = fmaf(v, w[c * 3 + 0], o0);
            o1 = fmaf(v, w[c * 3 + 1], o1);
            o2 = fmaf(v, w[c * 3 + 2], o2);
        }
        out[p * 3 + 0] = xin[p * 3 + 0] + o0;
        out[p * 3 + 1] = xin[p * 3 + 1] + o1;
        out[p * 3 + 2] = xin[p * 3 + 2] + o2;
    }
}

// MSE loss pieces: go[p][k] = 2 (out - target) / n ; per-block FP64 partial sums of the squares
__global__ void k_mse(const float *__restrict__ out, const float *__restrict__ target, int64_t n,
                      float *__restrict__ go, double *__restrict__ part)
{
    __shared__ double red[256];
    double a = 0.0;
    const float inv = 2.f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = out[i] - target[i];
        a += (double)d * d;
        if (go) go[i] = inv * d;
    }
    red[threadIdx.x] = a;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// head backward: gh[p][c] = sum_k go[p][k] w[c][k] (BF16); per-block partials of dw, db
__global__ void k_head_back(const bf16 *__restrict__ h, int C, const float *__restrict__ w,
                            const float *__restrict__ go, int64_t P, bf16 *__restrict__ gh,
                            float *__restrict__ part_w /*[blocks][C*3]*/, float *__restrict__ part_b)
{
    extern __shared__ float sh[];   // C*3 + 3 accumulators
    for (int i = threadIdx.x; i < C * 3 + 3; i += blockDim.x) sh[i] = 0.f;
    __syncthreads();
    float lw[64 * 3];               // C <= 64
    float lb[3] = {0.f, 0.f, 0.f};
    for (int i = 0; i < C * 3; ++i) lw[i] = 0.f;
    for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < P;
         p += (int64_t)gridDim.x * blockDim.x) {
        const float g0 = go[p * 3], g1 = go[p * 3 + 1], g2 = go[p * 3 + 2];
        lb[0] += g0, lb[1] += g1, lb[2] += g2;
        for (int c = 0; c < C; ++c) {
            const float v = __bfloat162float(h[p * C + c]);
            gh[p * C + c] = __float2bfloat16_rn(g0 * w[c * 3] + g1 * w[c * 3 + 1] + g2 * w[c * 3 + 2]);
            lw[c * 3] += v * g0, lw[c * 3 + 1] += v * g1, lw[c * 3 + 2] += v * g2;
        }
    }
    // fixed-order block reduction through shared memory, one thread at a time per slot
    for (int t = 0; t < (int)blockDim.x; ++t) {
        if ((int)threadIdx.x == t) {
            for (int i = 0; i < C * 3; ++i) sh[i] += lw[i];
            for (int k = 0; k < 3; ++k) sh[C * 3 + k] += lb[k];
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < C * 3; i += blockDim.x) part_w[(int64_t)blockIdx.x * C * 3 + i] = sh[i];
    if (threadIdx.x < 3) part_b[blockIdx.x * 3 + threadIdx.x] = sh[C * 3 + threadIdx.x];
}

// Adam on FP32 master parameters (bias-corrected)
__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps,
                       float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi, v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int grid_for(int64_t n, int threads = 256)
{
    int64_t g = (n + threads - 1) / threads;
    return (int)std::min<int64_t>(std::max<int64_t>(g, 1), 152 * 32);
}

cudaError_t conv_forward(const Tensor &x1, const Tensor *x2, const ConvParams &cp, int ks,
                         const bf16 *Wb, const float *bias, bool relu, bf16 *y1, int split,
                         bool acc1, bf16 *y2, bool acc2, cudaStream_t st)
{
    const int P = x1.B * x1.H * x1.W;
    dim3 grid((P + CONV_BM - 1) / CONV_BM, cp.cout / CONV_BN);
    const int c2 = x2 ? x2->C : 0;
    const bf16 *p2 = x2 ? x2->d : nullptr;
    if (ks == 3)
        k_conv<3><<<grid, 128, 0, st>>>(x1.d, x1.C, p2, c2, Wb, bias, cp.cout, x1.B, x1.H, x1.W,
                                        relu, y1, split, acc1, y2, acc2);
    else
        k_conv<1><<<grid, 128, 0, st>>>(x1.d, x1.C, p2, c2, Wb, bias, cp.cout, x1.B, x1.H, x1.W,
                                        relu, y1, split, acc1, y2, acc2);
    return cudaGetLastError();
}

cudaError_t conv_wgrad(const Tensor &x1, const Tensor *x2, const bf16 *g, int cout, int ks,
                       float *partial, int nsplit, float *dw, bool accumulate, cudaStream_t st)
{
    const int P = x1.B * x1.H * x1.W;
    const int cin = x1.C + (x2 ? x2->C : 0);
    const int per = ((P + nsplit - 1) / nsplit + 15) / 16 * 16;
    dim3 grid((cin / 32) * (cout / 32), ks * ks, nsplit);
    const int c2 = x2 ? x2->C : 0;
    const bf16 *p2 = x2 ? x2->d : nullptr;
    if (ks == 3)
        k_conv_wgrad<3><<<grid, 128, 0, st>>>(x1.d, x1.C, p2, c2, g, cout, x1.B, x1.H, x1.W, per, partial);
    else
        k_conv_wgrad<1><<<grid, 128, 0, st>>>(x1.d, x1.C, p2, c2, g, cout, x1.B, x1.H, x1.W, per, partial);
    const int64_t n = (int64_t)ks * ks * cin * cout;
    k_sum_splits<<<grid_for(n), 256, 0, st>>>(partial, nsplit, n, dw, accumulate);
    return cudaGetLastError();
}

cudaError_t sum_splits(const float *partial, int nsplit, int64_t n, float *out, bool accumulate,
                       cudaStream_t st)
{
    k_sum_splits<<<grid_for(n), 256, 0, st>>>(partial, nsplit, n, out, accumulate);
    return cudaGetLastError();
}

cudaError_t bias_grad(const bf16 *g, int C, int64_t P, float *db, float *partial, cudaStream_t st)
{
    const int blocks = (int)std::min<int64_t>(256, std::max<int64_t>(1, P / 1024));
    const int64_t per = (P + blocks - 1) / blocks;
    k_bias_grad<<<blocks, 256, 0, st>>>(g, C, P, per, partial);
    k_sum_splits<<<grid_for(C), 256, 0, st>>>(partial, blocks, C, db, 0);
    return cudaGetLastError();
}

cudaError_t prepare_weights(const float *Wm, int taps, int cin, int cout, bf16 *Wb, bf16 *Wf,
                            cudaStream_t st)
{
    const int64_t n = (int64_t)taps * cin * cout;
    k_prepare_weights<<<grid_for(n), 256, 0, st>>>(Wm, taps, cin, cout, Wb, Wf);
    return cudaGetLastError();
}

cudaError_t pack_input(const float *x, int64_t P, bf16 *y, cudaStream_t st)
{
    k_pack_input<<<grid_for(P), 256, 0, st>>>(x, P, y);
    return cudaGetLastError();
}

cudaError_t pool2(const Tensor &x, bf16 *y, cudaStream_t st)
{
    k_pool2<<<grid_for((int64_t)x.B * x.H * x.W * x.C / 4), 256, 0, st>>>(x.d, x.B, x.H, x.W, x.C, y);
    return cudaGetLastError();
}

cudaError_t pool2_back(const bf16 *gy, const Tensor &x, bf16 *gx, bool acc, cudaStream_t st)
{
    k_pool2_back<<<grid_for((int64_t)x.B * x.H * x.W * x.C), 256, 0, st>>>(gy, x.B, x.H, x.W, x.C, gx, acc);
    return cudaGetLastError();
}

cudaError_t up2(const Tensor &x, bf16 *y, cudaStream_t st)
{
    k_up2<<<grid_for((int64_t)x.B * x.H * x.W * x.C * 4), 256, 0, st>>>(x.d, x.B, x.H, x.W, x.C, y);
    return cudaGetLastError();
}

cudaError_t up2_back(const bf16 *gy, const Tensor &x, bf16 *gx, cudaStream_t st)
{
    k_up2_back<<<grid_for((int64_t)x.B * x.H * x.W * x.C), 256, 0, st>>>(gy, x.B, x.H, x.W, x.C, gx);
    return cudaGetLastError();
}

cudaError_t relu_mask(bf16 *g, const bf16 *y, int64_t n, cudaStream_t st)
{
    k_relu_mask<<<grid_for(n), 256, 0, st>>>(g, y, n);
    return cudaGetLastError();
}

cudaError_t head_forward(const Tensor &h, const float *w, const float *b, const float *xin,
                         float *out, cudaStream_t st)
{
    const int64_t P = (int64_t)h.B * h.H * h.W;
    k_head<<<grid_for(P), 256, 0, st>>>(h.d, h.C, w, b, xin, P, out);
    return cudaGetLastError();
}

cudaError_t mse(const float *out, const float *target, int64_t n, float *go, double *part,
                int blocks, cudaStream_t st)
{
    k_mse<<<blocks, 256, 0, st>>>(out, target, n, go, part);
    return cudaGetLastError();
}

cudaError_t head_backward(const Tensor &h, const float *w, const float *go, bf16 *gh,
                          float *part_w, float *part_b, int blocks, cudaStream_t st)
{
    const int64_t P = (int64_t)h.B * h.H * h.W;
    k_head_back<<<blocks, 128, (h.C * 3 + 3) * sizeof(float), st>>>(h.d, h.C, w, go, P, gh,
                                                                      part_w, part_b);
    return cudaGetLastError();
}

cudaError_t sum_blocks(const float *part, int nblocks, int64_t n, float *out, cudaStream_t st)
{
    k_sum_splits<<<grid_for(n), 256, 0, st>>>(part, nblocks, n, out, 0);
    return cudaGetLastError();
}

cudaError_t adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t st)
{
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    k_adam<<<grid_for(n), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace ei
