// Internal declarations of the U-Net kernels (nn_kernels.cu) used by the
// network orchestration (nn_unet.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#define EI_NN_TRY(expr)                         \
    do {                                        \
        cudaError_t _e = (expr);                \
        if (_e != cudaSuccess) return _e;       \
    } while (0)

namespace ei {
namespace nn {

typedef __nv_bfloat16 bf16;

// NHWC BF16 activation tensor (capacity fixed at creation; B may be smaller).
struct Tensor {
    bf16 *d = nullptr;
    int B = 0, H = 0, W = 0, C = 0;
    int64_t count() const { return (int64_t)B * H * W * C; }
};

struct ConvParams {
    int cout;
};

cudaError_t conv_forward(const Tensor &x1, const Tensor *x2, const ConvParams &cp, int ks,
                         const bf16 *Wb, const float *bias, bool relu, bf16 *y1, int split,
                         bool acc1, bf16 *y2, bool acc2, cudaStream_t st);
// The same convolution on the tcgen05 tensor cores (nn_conv_tc.cu): Wk is the
// K-major weight copy read with the tap order flipped (the forward pass passes
// the dgrad copy, dgrad the forward copy); *status is set if a bounded wait
// ran out.  conv_tc_supported: channel counts the kernel handles.
bool conv_tc_supported(int cin, int cout, int c1, int split);
cudaError_t conv_forward_tc(const Tensor &x1, const Tensor *x2, int cout, int ks, const bf16 *Wk,
                            const float *bias, bool relu, bf16 *y1, int split, bool acc1, bf16 *y2,
                            bool acc2, int *status, cudaStream_t st);
cudaError_t conv_wgrad(const Tensor &x1, const Tensor *x2, const bf16 *g, int cout, int ks,
                       float *partial, int nsplit, float *dw, bool accumulate, cudaStream_t st);
// The weight gradient's per-split partials on the tcgen05 tensor cores
// (nn_conv_tc.cu): partial[split][tap Cin + ci][co], the layout conv_wgrad's
// partials have; sum them with sum_splits.  *status is set if a bounded wait ran out.
bool wgrad_tc_supported(int cin, int cout, int c1);
cudaError_t conv_wgrad_tc(const Tensor &x1, const Tensor *x2, const bf16 *g, int cout, int ks,
                          float *partial, int nsplit, int *status, cudaStream_t st);
// out[i] (+)= sum_s partial[s][i] over nsplit splits of n values, in split order.
cudaError_t sum_splits(const float *partial, int nsplit, int64_t n, float *out, bool accumulate,
                       cudaStream_t st);
// db[c] = sum_p g[p][c] through per-block partials (C divides 256)
cudaError_t bias_grad(const bf16 *g, int C, int64_t P, float *db, float *partial, cudaStream_t st);
cudaError_t prepare_weights(const float *Wm, int taps, int cin, int cout, bf16 *Wb, bf16 *Wf,
                            cudaStream_t st);
// FP32 NHWC 3 channels -> BF16 NHWC 32 channels (zeros beyond 3)
cudaError_t pack_input(const float *x, int64_t P, bf16 *y, cudaStream_t st);
cudaError_t pool2(const Tensor &x, bf16 *y, cudaStream_t st);
cudaError_t pool2_back(const bf16 *gy, const Tensor &x, bf16 *gx, bool acc, cudaStream_t st);
cudaError_t up2(const Tensor &x, bf16 *y, cudaStream_t st);
cudaError_t up2_back(const bf16 *gy, const Tensor &x, bf16 *gx, cudaStream_t st);
cudaError_t relu_mask(bf16 *g, const bf16 *y, int64_t n, cudaStream_t st);
cudaError_t head_forward(const Tensor &h, const float *w, const float *b, const float *xin,
                         float *out, cudaStream_t st);
cudaError_t mse(const float *out, const float *target, int64_t n, float *go, double *part,
                int blocks, cudaStream_t st);
cudaError_t head_backward(const Tensor &h, const float *w, const float *go, bf16 *gh,
                          float *part_w, float *part_b, int blocks, cudaStream_t st);
cudaError_t sum_blocks(const float *part, int nblocks, int64_t n, float *out, cudaStream_t st);
cudaError_t adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1,
                 float b2, float eps, int step, cudaStream_t st);

}  // namespace nn
}  // namespace ei
