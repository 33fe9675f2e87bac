// Arithmetic peak probes: the FP32 and FP64 fused multiply-add rates of the
// device, measured (CUDA events) rather than taken from a data sheet.  They
// are the ceilings against which the ALU-bound steps of the path (the FP32
// screening and Loewdin Gram matrices, the FP64 factorisations, the FFT
// butterflies) are reported.  Every thread runs CHAINS independent chains of
// dependent FMAs, enough to hide the pipeline latency, on one CTA grid that
// fills every SM several times over.
#include <cuda_runtime.h>

#include <algorithm>

#include "../../include/lace.h"

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 16;

__device__ __forceinline__ unsigned long long pack2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                        unsigned long long c) {
    unsigned long long d;
    asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <typename T, int CHAINS>
__global__ void __launch_bounds__(kThreads) fma_probe_kernel(T* out, int iters, T a, T b) {
    T x[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma(x[c], a, b);
        }
    }
    T s = 0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += x[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Packed FP32 pairs: one fma.rn.f32x2 instruction does two FMAs.
template <int CHAINS>
__global__ void __launch_bounds__(kThreads) fma_probe_f32x2_kernel(float* out, int iters, float a, float b) {
    unsigned long long x[CHAINS];
    const unsigned long long a2 = pack2(a, a), b2 = pack2(b, b);
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = pack2((float)(threadIdx.x + c) * 1e-3f, (float)c * 1e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
            for (int c = 0; c < CHAINS; ++c) x[c] = fma_f32x2(x[c], a2, b2);
        }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
        float lo, hi;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(x[c]));
        s += lo + hi;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Best of `reps` timed launches of fn; returns FLOP/s (0 on failure).
template <class Launch>
double time_rate(Launch launch, double flops, cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, int reps) {
    launch();  // warm-up
    float best = 0.f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(e0, s);
        launch();
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) != cudaSuccess) return 0.0;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r == 0 || ms < best) best = ms;
    }
    return best > 0.f ? flops / (best * 1e-3) : 0.0;
}

}  // namespace

extern "C" lace_status lace_probe_peak_rates(int device, double* rates_out, int count) {
    if (!rates_out || count < 1) return LACE_ERR_ARG;
    if (cudaSetDevice(device) != cudaSuccess) {
        cudaGetLastError();
        return LACE_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return LACE_ERR_CUDA;
    const int blocks = sms * 8;  // 2048 threads an SM
    const size_t nthr = (size_t)blocks * kThreads;
    void* out = nullptr;
    if (cudaMalloc(&out, nthr * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return LACE_ERR_OOM;
    }
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    lace_status st = LACE_OK;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        st = LACE_ERR_CUDA;
    } else {
        constexpr int C32 = 8, C64 = 8;
        const int it32 = 4096, it64 = 256;
        double r[3] = {0.0, 0.0, 0.0};
        r[0] = time_rate(
            [&] {
                fma_probe_kernel<float, C32><<<blocks, kThreads, 0, s>>>(static_cast<float*>(out), it32, 0.999999f,
                                                                          1e-7f);
            },
            2.0 * C32 * kUnroll * (double)it32 * nthr, s, e0, e1, 5);
        r[1] = time_rate(
            [&] {
                fma_probe_f32x2_kernel<C32><<<blocks, kThreads, 0, s>>>(static_cast<float*>(out), it32 / 2,
                                                                         0.999999f, 1e-7f);
            },
            4.0 * C32 * kUnroll * (double)(it32 / 2) * nthr, s, e0, e1, 5);
        r[2] = time_rate(
            [&] {
                fma_probe_kernel<double, C64><<<blocks, kThreads, 0, s>>>(static_cast<double*>(out), it64,
                                                                           0.999999999, 1e-12);
            },
            2.0 * C64 * kUnroll * (double)it64 * nthr, s, e0, e1, 5);
        if (cudaGetLastError() != cudaSuccess) st = LACE_ERR_CUDA;
        for (int k = 0; k < count; ++k) rates_out[k] = k < 3 ? r[k] : 0.0;
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(out);
    return st;
}
