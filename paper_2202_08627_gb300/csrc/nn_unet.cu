// The learned warm start: a U-Net that maps the non-iterative (single-shot)
// reconstruction to a start close to the converged iterative one, trained on
// pairs the plain method generates.  Residual output: y = x + net(x).
//
// Topology (levels L, base width c0; c_l = c0 2^l): per encoder level two
// 3x3 conv + ReLU (the first of level l > 0 reads the 2x2 average pool of the
// level above); per decoder level (from L-2 up to 0) a nearest 2x upsample,
// a 3x3 conv + ReLU to c_l channels, a 3x3 conv + ReLU over the concatenation
// with the encoder's skip tensor, and a 3x3 conv + ReLU; a 1x1 head to the 3
// channels.  Activations are BF16 NHWC; weights are kept in FP32 (Adam) and
// copied to BF16 for the tensor-core convolutions after every update.
// Everything runs in this library's kernels (nn_kernels.cu).
#include <math.h>
#include <string.h>

#include <random>
#include <vector>

#include "../../include/ei.h"
#include "lib_alloc.h"
#include "nn_internal.h"

using namespace ei::nn;

namespace {

struct Conv {
    int ks = 3, cin1 = 0, cin2 = 0, cout = 0;
    bool relu = true;
    float *W = nullptr, *b = nullptr, *gW = nullptr, *gb = nullptr;
    float *mW = nullptr, *vW = nullptr, *mb = nullptr, *vb = nullptr;
    bf16 *Wb = nullptr, *Wf = nullptr;
    int cin() const { return cin1 + cin2; }
    int64_t nw() const { return (int64_t)ks * ks * cin() * cout; }
};

constexpr int kInC = 32;           // input channels after padding (3 used)

}  // namespace

struct ei_unet {
    int L = 0, base = 0, Bmax = 0, H = 0, W = 0, step = 0;
    std::vector<Conv> convs;
    std::vector<int> enc1, enc2, dup, da, db;
    float *hw = nullptr, *hb = nullptr, *ghw = nullptr, *ghb = nullptr;
    float *mhw = nullptr, *vhw = nullptr, *mhb = nullptr, *vhb = nullptr;
    Tensor in, E1[8], E2[8], POOL[8], U[8], DUP[8], DA[8], DB[8];
    Tensor GE1[8], GE2[8], GPOOL[8], GU[8], GDUP[8], GDA[8], GDB[8];
    float *out = nullptr, *go = nullptr, *partial = nullptr, *head_pw = nullptr, *head_pb = nullptr;
    float *bias_part = nullptr;        // [256 blocks][max channels]
    double *mse_part = nullptr, *mse_host = nullptr;
    int64_t partial_count = 0;
    int mse_blocks = 256, head_blocks = 152;
    int use_tc = 1;                    // convolutions on tcgen05 (1) or WMMA mma.sync (0)
    int *status = nullptr;             // device: set by a tcgen05 wait that ran out
    std::vector<void *> allocs;
};

namespace {

template <class T>
cudaError_t dalloc(ei_unet *n, T **p, int64_t count)
{
    void *q = nullptr;
    cudaError_t e = ei::lib_malloc(&q, std::max<int64_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return e;
    n->allocs.push_back(q);
    *p = static_cast<T *>(q);
    return cudaSuccess;
}

cudaError_t tensor(ei_unet *n, Tensor &t, int B, int H, int W, int C)
{
    t.B = B, t.H = H, t.W = W, t.C = C;
    return dalloc(n, &t.d, (int64_t)B * H * W * C);
}

int add_conv(ei_unet *n, int ks, int cin1, int cin2, int cout, bool relu)
{
    Conv c;
    c.ks = ks, c.cin1 = cin1, c.cin2 = cin2, c.cout = cout, c.relu = relu;
    n->convs.push_back(c);
    return (int)n->convs.size() - 1;
}

int nsplit_for(int64_t P) { return (int)std::min<int64_t>(128, std::max<int64_t>(1, P / 2048)); }

void set_batch(ei_unet *n, int B)
{
    n->in.B = B;
    for (int l = 0; l < n->L; ++l) {
        Tensor *ts[] = {&n->E1[l], &n->E2[l], &n->POOL[l], &n->U[l], &n->DUP[l], &n->DA[l],
                        &n->DB[l], &n->GE1[l], &n->GE2[l], &n->GPOOL[l], &n->GU[l], &n->GDUP[l],
                        &n->GDA[l], &n->GDB[l]};
        for (Tensor *t : ts) t->B = B;
    }
}

// One convolution: tcgen05 when enabled and the channel counts allow, else
// WMMA.  Wmn: the [tap][k][n] copy (WMMA); Wk: the flipped K-major copy.
cudaError_t conv(ei_unet *n, const Tensor &x1, const Tensor *x2, int cout, int ks,
                 const bf16 *Wmn, const bf16 *Wk, const float *bias, bool relu, bf16 *y1,
                 int split, bool acc1, bf16 *y2, bool acc2, cudaStream_t st)
{
    const int cin = x1.C + (x2 ? x2->C : 0);
    if (n->use_tc && conv_tc_supported(cin, cout, x1.C, split))
        return conv_forward_tc(x1, x2, cout, ks, Wk, bias, relu, y1, split, acc1, y2, acc2,
                               n->status, st);
    return conv_forward(x1, x2, {cout}, ks, Wmn, bias, relu, y1, split, acc1, y2, acc2, st);
}

cudaError_t forward(ei_unet *n, const float *x, float *y, cudaStream_t st)
{
    const int L = n->L;
    const int64_t P0 = (int64_t)n->in.B * n->H * n->W;
    EI_NN_TRY(pack_input(x, P0, n->in.d, st));
    for (int l = 0; l < L; ++l) {
        const Conv &c1 = n->convs[n->enc1[l]], &c2 = n->convs[n->enc2[l]];
        const Tensor &src = l == 0 ? n->in : n->POOL[l];
        EI_NN_TRY(conv(n, src, nullptr, c1.cout, 3, c1.Wb, c1.Wf, c1.b, true, n->E1[l].d, c1.cout,
                       false, nullptr, false, st));
        EI_NN_TRY(conv(n, n->E1[l], nullptr, c2.cout, 3, c2.Wb, c2.Wf, c2.b, true, n->E2[l].d,
                       c2.cout, false, nullptr, false, st));
        if (l < L - 1) EI_NN_TRY(pool2(n->E2[l], n->POOL[l + 1].d, st));
    }
    const Tensor *cur = &n->E2[L - 1];
    for (int d = L - 2; d >= 0; --d) {
        const Conv &cu = n->convs[n->dup[d]], &ca = n->convs[n->da[d]], &cb = n->convs[n->db[d]];
        EI_NN_TRY(up2(*cur, n->U[d].d, st));
        EI_NN_TRY(conv(n, n->U[d], nullptr, cu.cout, 3, cu.Wb, cu.Wf, cu.b, true, n->DUP[d].d,
                       cu.cout, false, nullptr, false, st));
        EI_NN_TRY(conv(n, n->DUP[d], &n->E2[d], ca.cout, 3, ca.Wb, ca.Wf, ca.b, true, n->DA[d].d,
                       ca.cout, false, nullptr, false, st));
        EI_NN_TRY(conv(n, n->DA[d], nullptr, cb.cout, 3, cb.Wb, cb.Wf, cb.b, true, n->DB[d].d,
                       cb.cout, false, nullptr, false, st));
        cur = &n->DB[d];
    }
    return head_forward(*cur, n->hw, n->hb, x, y, st);
}

// Backward of one conv (+ReLU): g (gradient of its output, masked in place by
// the ReLU), weight and bias gradients, and (if gx1) the input gradient(s).
cudaError_t conv_backward(ei_unet *n, const Conv &c, const Tensor &x1, const Tensor *x2,
                          const Tensor &y, bf16 *g, bf16 *gx1, bool acc1, bf16 *gx2, bool acc2,
                          cudaStream_t st)
{
    const int64_t P = (int64_t)y.B * y.H * y.W;
    if (c.relu) EI_NN_TRY(relu_mask(g, y.d, P * c.cout, st));
    const int nsplit = nsplit_for(P);
    if (n->use_tc && wgrad_tc_supported(c.cin(), c.cout, x1.C)) {
        EI_NN_TRY(conv_wgrad_tc(x1, x2, g, c.cout, c.ks, n->partial, nsplit, n->status, st));
        EI_NN_TRY(sum_splits(n->partial, nsplit, (int64_t)c.ks * c.ks * c.cin() * c.cout, c.gW,
                             false, st));
    } else {
        EI_NN_TRY(conv_wgrad(x1, x2, g, c.cout, c.ks, n->partial, nsplit, c.gW, false, st));
    }
    EI_NN_TRY(bias_grad(g, c.cout, P, c.gb, n->bias_part, st));
    if (gx1) {
        Tensor gt;
        gt.d = g, gt.B = y.B, gt.H = y.H, gt.W = y.W, gt.C = c.cout;
        EI_NN_TRY(conv(n, gt, nullptr, c.cin(), c.ks, c.Wf, c.Wb, nullptr, false, gx1, c.cin1,
                       acc1, gx2, acc2, st));
    }
    return cudaSuccess;
}

cudaError_t backward(ei_unet *n, const float *x, cudaStream_t st)
{
    const int L = n->L;
    const Tensor &top = L >= 2 ? n->DB[0] : n->E2[0];
    EI_NN_TRY(head_backward(top, n->hw, n->go, L >= 2 ? n->GDB[0].d : n->GE2[0].d, n->head_pw,
                            n->head_pb, n->head_blocks, st));
    EI_NN_TRY(sum_blocks(n->head_pw, n->head_blocks, (int64_t)n->base * 3, n->ghw, st));
    EI_NN_TRY(sum_blocks(n->head_pb, n->head_blocks, 3, n->ghb, st));
    for (int d = 0; d <= L - 2; ++d) {
        const Conv &cu = n->convs[n->dup[d]], &ca = n->convs[n->da[d]], &cb = n->convs[n->db[d]];
        EI_NN_TRY(conv_backward(n, cb, n->DA[d], nullptr, n->DB[d], n->GDB[d].d, n->GDA[d].d, false,
                                nullptr, false, st));
        EI_NN_TRY(conv_backward(n, ca, n->DUP[d], &n->E2[d], n->DA[d], n->GDA[d].d, n->GDUP[d].d,
                                false, n->GE2[d].d, false, st));
        EI_NN_TRY(conv_backward(n, cu, n->U[d], nullptr, n->DUP[d], n->GDUP[d].d, n->GU[d].d, false,
                                nullptr, false, st));
        const Tensor &below = d == L - 2 ? n->E2[L - 1] : n->DB[d + 1];
        bf16 *gbelow = d == L - 2 ? n->GE2[L - 1].d : n->GDB[d + 1].d;
        EI_NN_TRY(up2_back(n->GU[d].d, below, gbelow, st));
    }
    for (int l = L - 1; l >= 0; --l) {
        const Conv &c1 = n->convs[n->enc1[l]], &c2 = n->convs[n->enc2[l]];
        EI_NN_TRY(conv_backward(n, c2, n->E1[l], nullptr, n->E2[l], n->GE2[l].d, n->GE1[l].d, false,
                                nullptr, false, st));
        const Tensor &src = l == 0 ? n->in : n->POOL[l];
        EI_NN_TRY(conv_backward(n, c1, src, nullptr, n->E1[l], n->GE1[l].d,
                                l > 0 ? n->GPOOL[l].d : nullptr, false, nullptr, false, st));
        if (l > 0) EI_NN_TRY(pool2_back(n->GPOOL[l].d, n->E2[l - 1], n->GE2[l - 1].d, true, st));
    }
    (void)x;
    return cudaSuccess;
}

cudaError_t refresh_bf16(ei_unet *n, cudaStream_t st)
{
    for (Conv &c : n->convs)
        EI_NN_TRY(prepare_weights(c.W, c.ks * c.ks, c.cin(), c.cout, c.Wb, c.Wf, st));
    return cudaSuccess;
}

// parameters in export order: every conv's W then b (creation order), head W, head b
template <class F>
void for_each_param(ei_unet *n, F f)
{
    for (Conv &c : n->convs) {
        f(c.W, c.gW, c.mW, c.vW, c.nw());
        f(c.b, c.gb, c.mb, c.vb, (int64_t)c.cout);
    }
    f(n->hw, n->ghw, n->mhw, n->vhw, (int64_t)n->base * 3);
    f(n->hb, n->ghb, n->mhb, n->vhb, (int64_t)3);
}

int status(cudaError_t e) { return e == cudaSuccess ? EI_OK : (e == cudaErrorMemoryAllocation ? EI_ERR_ALLOC : EI_ERR_CUDA); }

}  // namespace

extern "C" {

int ei_unet_create(int levels, int base, int batch, int height, int width,
                   unsigned long long seed, ei_unet **out)
{
    if (!out || levels < 1 || levels > 6 || base < 32 || base > 64 || base % 32 || batch < 1 ||
        height < 1 || width < 1 || height % (1 << (levels - 1)) || width % (1 << (levels - 1)))
        return EI_ERR_ARG;
    *out = nullptr;
    ei_unet *n = new ei_unet();
    n->L = levels, n->base = base, n->Bmax = batch, n->H = height, n->W = width;
    const int L = levels;
    auto ch = [&](int l) { return base << l; };
    n->enc1.resize(L), n->enc2.resize(L), n->dup.resize(L), n->da.resize(L), n->db.resize(L);
    for (int l = 0; l < L; ++l) {
        n->enc1[l] = add_conv(n, 3, l == 0 ? kInC : ch(l - 1), 0, ch(l), true);
        n->enc2[l] = add_conv(n, 3, ch(l), 0, ch(l), true);
    }
    for (int d = L - 2; d >= 0; --d) {
        n->dup[d] = add_conv(n, 3, ch(d + 1), 0, ch(d), true);
        n->da[d] = add_conv(n, 3, ch(d), ch(d), ch(d), true);
        n->db[d] = add_conv(n, 3, ch(d), 0, ch(d), true);
    }
    cudaError_t e = cudaSuccess;
    int64_t maxpart = 0;
    for (Conv &c : n->convs) {
        if (e == cudaSuccess) e = dalloc(n, &c.W, c.nw());
        if (e == cudaSuccess) e = dalloc(n, &c.gW, c.nw());
        if (e == cudaSuccess) e = dalloc(n, &c.mW, c.nw());
        if (e == cudaSuccess) e = dalloc(n, &c.vW, c.nw());
        if (e == cudaSuccess) e = dalloc(n, &c.b, c.cout);
        if (e == cudaSuccess) e = dalloc(n, &c.gb, c.cout);
        if (e == cudaSuccess) e = dalloc(n, &c.mb, c.cout);
        if (e == cudaSuccess) e = dalloc(n, &c.vb, c.cout);
        if (e == cudaSuccess) e = dalloc(n, &c.Wb, c.nw());
        if (e == cudaSuccess) e = dalloc(n, &c.Wf, c.nw());
    }
    for (int l = 0; l < L; ++l) {
        const int h = height >> l, w = width >> l;
        const int64_t P = (int64_t)batch * h * w;
        maxpart = std::max<int64_t>(maxpart, (int64_t)nsplit_for(P) * 9 * 2 * ch(l) * ch(l));
        maxpart = std::max<int64_t>(maxpart, (int64_t)nsplit_for(P) * 9 * (l + 1 < L ? ch(l + 1) : 1) * ch(l));
        maxpart = std::max<int64_t>(maxpart, (int64_t)nsplit_for(P) * 9 * kInC * ch(l));
    }
    if (e == cudaSuccess) e = tensor(n, n->in, batch, height, width, kInC);
    for (int l = 0; l < L && e == cudaSuccess; ++l) {
        const int h = height >> l, w = width >> l, c = ch(l);
        e = tensor(n, n->E1[l], batch, h, w, c);
        if (e == cudaSuccess) e = tensor(n, n->E2[l], batch, h, w, c);
        if (e == cudaSuccess) e = tensor(n, n->GE1[l], batch, h, w, c);
        if (e == cudaSuccess) e = tensor(n, n->GE2[l], batch, h, w, c);
        if (l > 0 && e == cudaSuccess) e = tensor(n, n->POOL[l], batch, h, w, ch(l - 1));
        if (l > 0 && e == cudaSuccess) e = tensor(n, n->GPOOL[l], batch, h, w, ch(l - 1));
        if (l < L - 1) {
            if (e == cudaSuccess) e = tensor(n, n->U[l], batch, h, w, ch(l + 1));
            if (e == cudaSuccess) e = tensor(n, n->GU[l], batch, h, w, ch(l + 1));
            if (e == cudaSuccess) e = tensor(n, n->DUP[l], batch, h, w, c);
            if (e == cudaSuccess) e = tensor(n, n->GDUP[l], batch, h, w, c);
            if (e == cudaSuccess) e = tensor(n, n->DA[l], batch, h, w, c);
            if (e == cudaSuccess) e = tensor(n, n->GDA[l], batch, h, w, c);
            if (e == cudaSuccess) e = tensor(n, n->DB[l], batch, h, w, c);
            if (e == cudaSuccess) e = tensor(n, n->GDB[l], batch, h, w, c);
        }
    }
    const int64_t n_out = (int64_t)batch * height * width * 3;
    n->partial_count = maxpart;
    if (e == cudaSuccess) e = dalloc(n, &n->out, n_out);
    if (e == cudaSuccess) e = dalloc(n, &n->go, n_out);
    if (e == cudaSuccess) e = dalloc(n, &n->partial, maxpart);
    if (e == cudaSuccess) e = dalloc(n, &n->bias_part, (int64_t)256 * ch(L - 1));
    if (e == cudaSuccess) e = dalloc(n, &n->head_pw, (int64_t)n->head_blocks * base * 3);
    if (e == cudaSuccess) e = dalloc(n, &n->head_pb, (int64_t)n->head_blocks * 3);
    if (e == cudaSuccess) e = dalloc(n, &n->mse_part, n->mse_blocks);
    if (e == cudaSuccess) e = cudaMallocHost(&n->mse_host, n->mse_blocks * sizeof(double));
    if (e == cudaSuccess) e = dalloc(n, &n->status, 1);
    if (e == cudaSuccess) e = cudaMemset(n->status, 0, sizeof(int));
    for (float **p : {&n->hw, &n->ghw, &n->mhw, &n->vhw})
        if (e == cudaSuccess) e = dalloc(n, p, (int64_t)base * 3);
    for (float **p : {&n->hb, &n->ghb, &n->mhb, &n->vhb})
        if (e == cudaSuccess) e = dalloc(n, p, 3);
    // He-normal weights, zero biases, a small head so that the net starts near the identity
    if (e == cudaSuccess) {
        std::mt19937_64 rng(seed);
        std::normal_distribution<float> nd(0.f, 1.f);
        for (Conv &c : n->convs) {
            std::vector<float> w(c.nw());
            const float sd = sqrtf(2.f / (float)(c.ks * c.ks * c.cin()));
            for (float &v : w) v = sd * nd(rng);
            if (e == cudaSuccess) e = cudaMemcpy(c.W, w.data(), w.size() * 4, cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemset(c.b, 0, c.cout * 4);
        }
        std::vector<float> hw((size_t)base * 3);
        for (float &v : hw) v = 1e-3f * nd(rng);
        if (e == cudaSuccess) e = cudaMemcpy(n->hw, hw.data(), hw.size() * 4, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(n->hb, 0, 12);
        for_each_param(n, [&](float *, float *, float *m, float *v, int64_t cnt) {
            if (e == cudaSuccess) e = cudaMemset(m, 0, cnt * 4);
            if (e == cudaSuccess) e = cudaMemset(v, 0, cnt * 4);
        });
        if (e == cudaSuccess) e = refresh_bf16(n, 0);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        ei_unet_destroy(n);
        return status(e);
    }
    *out = n;
    return EI_OK;
}

void ei_unet_destroy(ei_unet *n)
{
    if (!n) return;
    cudaDeviceSynchronize();
    for (void *p : n->allocs) ei::lib_free(p);
    if (n->mse_host) cudaFreeHost(n->mse_host);
    delete n;
}

int ei_unet_forward(ei_unet *n, const float *x, float *y, int batch, void *stream)
{
    if (!n || !x || !y || batch < 1 || batch > n->Bmax) return EI_ERR_ARG;
    set_batch(n, batch);
    return status(forward(n, x, y, (cudaStream_t)stream));
}

int ei_unet_train_step(ei_unet *n, const float *x, const float *target, int batch, double lr,
                       double *loss, void *stream)
{
    if (!n || !x || !target || batch < 1 || batch > n->Bmax || !(lr > 0)) return EI_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    set_batch(n, batch);
    const int64_t cnt = (int64_t)batch * n->H * n->W * 3;
    cudaError_t e = forward(n, x, n->out, st);
    if (e == cudaSuccess) e = mse(n->out, target, cnt, n->go, n->mse_part, n->mse_blocks, st);
    if (e == cudaSuccess) e = backward(n, x, st);
    n->step += 1;
    for_each_param(n, [&](float *p, float *g, float *m, float *v, int64_t c) {
        if (e == cudaSuccess) e = adam(p, g, m, v, c, (float)lr, 0.9f, 0.999f, 1e-8f, n->step, st);
    });
    if (e == cudaSuccess) e = refresh_bf16(n, st);
    if (e == cudaSuccess && loss) {
        e = cudaMemcpyAsync(n->mse_host, n->mse_part, n->mse_blocks * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e == cudaSuccess) {
            double s = 0.0;
            for (int i = 0; i < n->mse_blocks; ++i) s += n->mse_host[i];
            *loss = s / (double)cnt;
        }
    }
    if (e == cudaSuccess && loss) {                 // synchronised: report a timed-out wait
        int h = 0;
        e = cudaMemcpy(&h, n->status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && h) {
            cudaMemset(n->status, 0, sizeof(int));
            return EI_ERR_TIMEOUT;
        }
    }
    return status(e);
}

int ei_unet_set_tensor_path(ei_unet *n, int path)
{
    if (!n || (path != 0 && path != 1)) return EI_ERR_ARG;
    n->use_tc = path;
    return EI_OK;
}

int64_t ei_unet_num_params(const ei_unet *n)
{
    if (!n) return -1;
    int64_t c = 0;
    for_each_param(const_cast<ei_unet *>(n), [&](float *, float *, float *, float *, int64_t k) { c += k; });
    return c;
}

static int copy_params(ei_unet *n, float *host, int which, bool to_host)
{
    if (!n || !host) return EI_ERR_ARG;
    cudaError_t e = cudaDeviceSynchronize();
    int64_t off = 0;
    for_each_param(n, [&](float *p, float *g, float *m, float *v, int64_t k) {
        float *d = which == 0 ? p : which == 1 ? g : which == 2 ? m : v;
        if (e == cudaSuccess)
            e = to_host ? cudaMemcpy(host + off, d, k * 4, cudaMemcpyDeviceToHost)
                        : cudaMemcpy(d, host + off, k * 4, cudaMemcpyHostToDevice);
        off += k;
    });
    if (e == cudaSuccess && !to_host && which == 0) e = refresh_bf16(n, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return status(e);
}

int ei_unet_get_params(const ei_unet *n, float *host) { return copy_params(const_cast<ei_unet *>(n), host, 0, true); }
int ei_unet_set_params(ei_unet *n, const float *host) { return copy_params(n, const_cast<float *>(host), 0, false); }
int ei_unet_get_grads(const ei_unet *n, float *host) { return copy_params(const_cast<ei_unet *>(n), host, 1, true); }

int ei_unet_get_optimizer(const ei_unet *n, float *m_host, float *v_host, int *step)
{
    if (!n || !m_host || !v_host || !step) return EI_ERR_ARG;
    ei_unet *u = const_cast<ei_unet *>(n);
    int r = copy_params(u, m_host, 2, true);
    if (r == EI_OK) r = copy_params(u, v_host, 3, true);
    if (r == EI_OK) *step = n->step;
    return r;
}

int ei_unet_set_optimizer(ei_unet *n, const float *m_host, const float *v_host, int step)
{
    if (!n || !m_host || !v_host || step < 0) return EI_ERR_ARG;
    int r = copy_params(n, const_cast<float *>(m_host), 2, false);
    if (r == EI_OK) r = copy_params(n, const_cast<float *>(v_host), 3, false);
    if (r == EI_OK) n->step = step;
    return r;
}

}  // extern "C"
