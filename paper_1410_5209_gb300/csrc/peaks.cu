// Device peaks of the units the mode passes are bound by, measured with CUDA events on the
// current device: FP32 FMA throughput (plain and packed two-wide) and shared-memory load
// bandwidth.  The HBM copy bandwidth and the tensor-core rate are measured elsewhere; these
// two give the lean pass a roofline against its own binding units.
#include "common.cuh"

namespace tfs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kFmaChains = 8;
constexpr int kFmaIters = 4096;

// Independent FMA chains per thread (enough to cover the pipeline latency), the results
// folded into one store so that nothing is removed.
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float *out, float a, float b) {
    float x[kFmaChains];
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) x[c] = (float)(threadIdx.x + c);
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) s += x[c];
    if (s == 1.2345f) out[blockIdx.x] = s;  // never true for the inputs used; keeps the work
}

__global__ void __launch_bounds__(kPeakThreads) k_fma2_peak(float *out, float a, float b) {
    unsigned long long x[kFmaChains];
    unsigned long long av, bv;
    asm("mov.b64 %0, {%1, %1};" : "=l"(av) : "f"(a));
    asm("mov.b64 %0, {%1, %1};" : "=l"(bv) : "f"(b));
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) {
        const float v = (float)(threadIdx.x + c);
        asm("mov.b64 %0, {%1, %1};" : "=l"(x[c]) : "f"(v));
    }
    for (int it = 0; it < kFmaIters; ++it) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c)
            asm("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(x[c]) : "l"(av), "l"(bv));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kFmaChains; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    if (s == 1.2345f) out[blockIdx.x] = s;
}

constexpr int kSmemIters = 2048;
constexpr int kSmemFloats = 8192;  // 32 KB per block

// 16-byte shared-memory loads, each quarter-warp on 8 distinct 16-byte bank groups (no
// conflicts); the address moves with the iteration so that no load can be hoisted.
__global__ void __launch_bounds__(kPeakThreads) k_smem_peak(float *out) {
    __shared__ __align__(16) float buf[kSmemFloats];
    for (int i = threadIdx.x; i < kSmemFloats; i += kPeakThreads) buf[i] = (float)i;
    __syncthreads();
    const unsigned base = (unsigned)__cvta_generic_to_shared(buf);
    unsigned acc = 0;
    for (int it = 0; it < kSmemIters; ++it) {
        const unsigned idx = ((unsigned)threadIdx.x + (unsigned)it * kPeakThreads) %
                             (unsigned)(kSmemFloats / 4);
        unsigned w0, w1, w2, w3;
        asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(w0), "=r"(w1), "=r"(w2), "=r"(w3)
                     : "r"(base + 16u * idx));
        acc ^= w0 ^ w1 ^ w2 ^ w3;
    }
    if (acc == 0x12345678u) out[blockIdx.x] = (float)acc;
}

template <class F>
double time_ms(F &&launch, cudaStream_t st) {
    cudaEvent_t a, b;
    TFS_CUDA(cudaEventCreate(&a));
    TFS_CUDA(cudaEventCreate(&b));
    launch();  // warm-up
    TFS_CUDA(cudaEventRecord(a, st));
    for (int r = 0; r < 5; ++r) launch();
    TFS_CUDA(cudaEventRecord(b, st));
    TFS_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    TFS_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / 5.0;
}

}  // namespace
}  // namespace tfs

extern "C" tf_status tf_device_peaks(double *fp32_tflops, double *fp32x2_tflops,
                                     double *smem_tbytes) {
    using namespace tfs;
    try {
        int dev = 0, sms = 0;
        TFS_CUDA(cudaGetDevice(&dev));
        TFS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        float *out = nullptr;
        const int blocks = sms * 8;
        TFS_CUDA(cudaMalloc(&out, sizeof(float) * blocks));
        cudaStream_t st = nullptr;
        TFS_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        const double threads = (double)blocks * kPeakThreads;
        const double fma_ms = time_ms(
            [&] { k_fma_peak<<<blocks, kPeakThreads, 0, st>>>(out, 0.999f, 1e-3f); }, st);
        const double fma2_ms = time_ms(
            [&] { k_fma2_peak<<<blocks, kPeakThreads, 0, st>>>(out, 0.999f, 1e-3f); }, st);
        const double smem_ms = time_ms([&] { k_smem_peak<<<blocks, kPeakThreads, 0, st>>>(out); }, st);
        TFS_CUDA(cudaGetLastError());
        cudaStreamDestroy(st);
        cudaFree(out);
        const double fmas = threads * kFmaIters * kFmaChains;
        if (fp32_tflops) *fp32_tflops = 2.0 * fmas / (fma_ms * 1e-3) / 1e12;
        if (fp32x2_tflops) *fp32x2_tflops = 4.0 * fmas / (fma2_ms * 1e-3) / 1e12;
        if (smem_tbytes) *smem_tbytes = threads * kSmemIters * 16.0 / (smem_ms * 1e-3) / 1e12;
        return TF_OK;
    } catch (const CudaError &) {
        cudaGetLastError();
        return TF_ECUDA;
    }
}
