// On-chip throughput microbenchmarks: the denominators of the rooflines of
// the kernels that are bound on chip rather than by HBM (the projector and
// the adjoint move ~50 B per voxel-angle from L1 into registers; the IC
// kernel's arithmetic is FP32).
//
//   FP32 FMA rate      every thread runs 8 independent FMA chains
//   L1 load bandwidth  every block re-reads one 8 KB region with lane-contiguous
//                      16-byte loads (after the first pass every load hits L1)
//   shared memory      the same pattern on an 8 KB shared-memory copy
//
// Each is timed with CUDA events after a warm-up launch; the best of three
// runs is reported.  Work sizes are fixed and the loops have constant trip
// counts, so every launch ends.
#include <algorithm>

#include "async_copy.h"
#include "ei_internal.h"

namespace ei {

namespace {

constexpr int kPeakThreads = 256;
constexpr int kSpan4 = 512;                 // float4 per block region: 8 KB

__global__ void __launch_bounds__(kPeakThreads) k_peak_fma(float *out, int iters)
{
    float a[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = 1.0f + 1e-3f * (float)(threadIdx.x + i);
    const float b = 0.9999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], b, c);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.0f) out[blockIdx.x] = s;     // keeps the chains live; never true
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_l1(const float4 *__restrict__ src, float *out,
                                                          int iters)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = threadIdx.x; k < kSpan4; k += kPeakThreads) {
            // the offset moves with the iteration so no load is loop-invariant
            const float4 v = __ldg(src + ((k + it * 32) & (kSpan4 - 1)));
            acc.x += v.x, acc.y += v.y, acc.z += v.z, acc.w += v.w;
        }
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == 12345.0f) out[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kPeakThreads) k_peak_smem(const float4 *__restrict__ src, float *out,
                                                            int iters)
{
    __shared__ float4 buf[kSpan4];
    for (int k = threadIdx.x; k < kSpan4; k += kPeakThreads) buf[k] = src[k];
    __syncthreads();
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = threadIdx.x; k < kSpan4; k += kPeakThreads) {
            const float4 v = buf[(k + it * 32) & (kSpan4 - 1)];
            acc.x += v.x, acc.y += v.y, acc.z += v.z, acc.w += v.w;
        }
    }
    const float s = acc.x + acc.y + acc.z + acc.w;
    if (s == 12345.0f) out[blockIdx.x] = s;
}

template <typename F>
cudaError_t best_ms(F launch, cudaStream_t st, float *ms)
{
    cudaEvent_t e0, e1;
    EI_CUDA_TRY(cudaEventCreate(&e0));
    EI_CUDA_TRY(cudaEventCreate(&e1));
    launch();                                           // warm-up
    float best = 1e30f;
    cudaError_t e = cudaGetLastError();
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
        cudaEventRecord(e0, st);
        launch();
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        best = std::min(best, t);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return e;
}

}  // namespace

}  // namespace ei

using namespace ei;

extern "C" int ei_measure_peaks(ei_peaks *out, void *stream)
{
    if (!out) return EI_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return EI_ERR_CUDA;
    float4 *src = nullptr;
    float *sink = nullptr;
    const int grid = sms * 8;                 // 2048 threads per SM
    cudaError_t e = cudaMalloc(&src, kSpan4 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc(&sink, grid * sizeof(float));
    if (e == cudaSuccess) e = cudaMemsetAsync(src, 0, kSpan4 * sizeof(float4), st);
    const int fma_iters = 4096, mem_iters = 2048;
    float t_fma = 0.f, t_l1 = 0.f, t_sm = 0.f;
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_fma<<<grid, kPeakThreads, 0, st>>>(sink, fma_iters); }, st, &t_fma);
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_l1<<<grid, kPeakThreads, 0, st>>>(src, sink, mem_iters); }, st, &t_l1);
    if (e == cudaSuccess)
        e = best_ms([&] { k_peak_smem<<<grid, kPeakThreads, 0, st>>>(src, sink, mem_iters); }, st, &t_sm);
    cudaFree(src);
    cudaFree(sink);
    if (e != cudaSuccess) {
        record_error(e);
        return EI_ERR_CUDA;
    }
    const double threads = (double)grid * kPeakThreads;
    out->fp32_tflops = threads * fma_iters * 16 * 8 * 2 / (t_fma * 1e-3) / 1e12;
    const double bytes = (double)grid * mem_iters * kSpan4 * sizeof(float4);
    out->l1_load_tbs = bytes / (t_l1 * 1e-3) / 1e12;
    out->smem_load_tbs = bytes / (t_sm * 1e-3) / 1e12;
    out->num_sms = sms;
    return EI_OK;
}

// ---------------------------------------------------------------------------
// Failure-detection self-test: one thread initialises an mbarrier that
// nothing ever arrives on (no copy, no other thread) and waits on it with the
// same bounded wait the bulk-copy kernels use, limited to `limit_ns`; it
// records whether the wait gave up.  Nothing is in flight when it returns,
// so the context stays usable.
// ---------------------------------------------------------------------------
namespace ei {

__global__ void k_wait_selftest(uint64_t limit_ns, int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(smem_addr(&bar), 1);
    mbar_init_fence();
    const bool landed = mbar_wait_bounded(smem_addr(&bar), 0u, limit_ns);
    *status = landed ? (int)EI_OK : (int)EI_ERR_TIMEOUT;
}

}  // namespace ei

extern "C" int ei_selftest_wait_timeout(unsigned limit_us, int *status_out)
{
    using namespace ei;
    if (!status_out || limit_us == 0 || limit_us > 2000000u) return EI_ERR_ARG;
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) {
        k_wait_selftest<<<1, 32>>>((uint64_t)limit_us * 1000u, d);
        e = cudaGetLastError();
    }
    int st = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&st, d, sizeof(int), cudaMemcpyDeviceToHost);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    *status_out = st;
    return EI_OK;
}

// Bounds-check self-test: 32 threads each read element i + skew of a
// 64-float buffer through checked_index with the logical range [0, 31]; with
// skew = 8 the last eight indices fall outside that range but inside the
// buffer, so the read stays in bounds whether or not the check fires.
__global__ void k_check_selftest(const float *buf, float *out, int skew, int *status)
{
    const int i = ei::checked_index((int)threadIdx.x + skew, 0, 31, status);
    out[threadIdx.x] = buf[i];
}

extern "C" int ei_device_checks_enabled(void) { return ei::kDeviceChecks ? 1 : 0; }

extern "C" int ei_selftest_device_check(int *status_out)
{
    using namespace ei;
    if (!status_out) return EI_ERR_ARG;
    float *buf = nullptr;
    int *d = nullptr;
    cudaError_t e = cudaMalloc(&buf, 96 * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&d, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(buf, 0, 96 * sizeof(float));
    if (e == cudaSuccess) e = cudaMemset(d, 0, sizeof(int));
    if (e == cudaSuccess) {
        k_check_selftest<<<1, 32>>>(buf, buf + 64, 8, d);
        e = cudaGetLastError();
    }
    int st = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&st, d, sizeof(int), cudaMemcpyDeviceToHost);
    if (buf) cudaFree(buf);
    if (d) cudaFree(d);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return EI_ERR_CUDA;
    }
    *status_out = st;
    return EI_OK;
}
