// Measured roofline denominators: FP32 FMA throughput and L2 read bandwidth.
//
// Neither is a datasheet number on this part, and the row pass is bound by
// FP32 arithmetic while the column pass reads fields that stay in L2 between
// passes, so both are measured on the device that runs the passes, with the
// same CUDA-event timing as the passes.  Nothing here changes a clock or
// any other setting of the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "plan.h"

namespace shg {

constexpr int kFmaThreads = 256;
constexpr int kFmaChains = 8;  // independent accumulator pairs per thread

// Each thread runs kFmaChains independent chains of packed two-lane FMAs
// (fma.rn.f32x2: two FP32 FMAs per instruction), `iters` rounds each.  The
// operands stay in registers and the result is written once, so the kernel
// is bound by the FMA pipe alone.
__global__ void __launch_bounds__(kFmaThreads) k_fma_peak(int iters, float seed, float* sink) {
    float2 acc[kFmaChains];
    for (int c = 0; c < kFmaChains; ++c) {
        acc[c].x = seed + 1e-3f * (threadIdx.x + c);
        acc[c].y = seed - 1e-3f * (threadIdx.x + c);
    }
    const float a = 0.9999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c) {
            asm volatile(
                "{\n .reg .b64 x, m, s;\n mov.b64 x, {%0, %1};\n mov.b64 m, {%2, %2};\n"
                " mov.b64 s, {%3, %3};\n fma.rn.f32x2 x, x, m, s;\n mov.b64 {%0, %1}, x;\n}"
                : "+f"(acc[c].x), "+f"(acc[c].y)
                : "f"(a), "f"(b));
        }
    }
    float s = 0;
    for (int c = 0; c < kFmaChains; ++c) s += acc[c].x + acc[c].y;
    // keeps the chains live; the index stays inside the 2^18-float sink
    if (s == 12345.678f) sink[(blockIdx.x * blockDim.x + threadIdx.x) & ((1u << 18) - 1)] = s;
}

// Same with scalar FMAs (fma.rn.f32), 2 x kFmaChains chains.
__global__ void __launch_bounds__(kFmaThreads) k_fma_peak_scalar(int iters, float seed,
                                                                 float* sink) {
    float acc[2 * kFmaChains];
    for (int c = 0; c < 2 * kFmaChains; ++c) acc[c] = seed + 1e-3f * (threadIdx.x + c);
    const float a = 0.9999f, b = 1e-7f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < 2 * kFmaChains; ++c)
            asm volatile("fma.rn.f32 %0, %0, %1, %2;\n" : "+f"(acc[c]) : "f"(a), "f"(b));
    }
    float s = 0;
    for (int c = 0; c < 2 * kFmaChains; ++c) s += acc[c];
    if (s == 12345.678f) sink[(blockIdx.x * blockDim.x + threadIdx.x) & ((1u << 18) - 1)] = s;
}

// Same with double-precision FMAs (fma.rn.f64), kFmaChains chains.
__global__ void __launch_bounds__(kFmaThreads) k_fma_peak_f64(int iters, double seed,
                                                              double* sink) {
    double acc[kFmaChains];
    for (int c = 0; c < kFmaChains; ++c) acc[c] = seed + 1e-3 * (threadIdx.x + c);
    const double a = 0.9999, b = 1e-7;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kFmaChains; ++c)
            asm volatile("fma.rn.f64 %0, %0, %1, %2;\n" : "+d"(acc[c]) : "d"(a), "d"(b));
    }
    double s = 0;
    for (int c = 0; c < kFmaChains; ++c) s += acc[c];
    if (s == 12345.678) sink[(blockIdx.x * blockDim.x + threadIdx.x) & ((1u << 17) - 1)] = s;
}

// Grid-stride read of `n` 16-byte words, `reps` times over the same buffer
// (small enough to stay in L2 after the first pass), summed so the loads are
// kept.
__global__ void k_l2_read(const uint4* __restrict__ buf, size_t n, int reps, unsigned* sink) {
    unsigned acc = 0;
    for (int r = 0; r < reps; ++r)
        for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
             i += size_t(gridDim.x) * blockDim.x) {
            uint4 v;
            asm volatile("ld.global.cg.v4.u32 {%0, %1, %2, %3}, [%4];\n"
                         : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                         : "l"(buf + i));
            acc ^= v.x ^ v.y ^ v.z ^ v.w;
        }
    if (acc == 0x9e3779b9u) sink[0] = acc;
}

struct Events {
    cudaEvent_t a = nullptr, b = nullptr;
    ~Events() {
        if (a) cudaEventDestroy(a);
        if (b) cudaEventDestroy(b);
    }
};

}  // namespace shg

using namespace shg;

extern "C" shg_status_t shg_measure_peaks(double* fp32_tflops, double* l2_read_gbs,
                                          double* fp32_scalar_tflops, double* fp64_tflops,
                                          shg_stream_t stream) {
    if (!fp32_tflops && !l2_read_gbs && !fp32_scalar_tflops && !fp64_tflops)
        return SHG_ERR_INVALID_ARG;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    SHG_CK(cudaGetDevice(&dev));
    SHG_CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    Events ev;
    SHG_CK(cudaEventCreate(&ev.a));
    SHG_CK(cudaEventCreate(&ev.b));
    void* sink = nullptr;
    // 1 MiB of sink: written by no thread unless a sum hits its sentinel
    SHG_CK(cudaMallocAsync(&sink, 1 << 20, st));
    auto time_best = [&](auto launch, int rounds, float* best) -> cudaError_t {
        *best = 1e30f;
        cudaError_t e = launch();  // warm-up
        for (int r = 0; r < rounds && e == cudaSuccess; ++r) {
            if ((e = cudaEventRecord(ev.a, st)) != cudaSuccess) break;
            if ((e = launch()) != cudaSuccess) break;
            if ((e = cudaEventRecord(ev.b, st)) != cudaSuccess) break;
            if ((e = cudaEventSynchronize(ev.b)) != cudaSuccess) break;
            float ms = 0;
            if ((e = cudaEventElapsedTime(&ms, ev.a, ev.b)) != cudaSuccess) break;
            *best = std::min(*best, ms);
        }
        return e;
    };
    cudaError_t e = cudaSuccess;
    // 8 CTAs of 256 threads per SM: every warp slot filled
    const int blocks = nsm * 8;
    const int iters = 4096;
    const double fma_threads = double(blocks) * kFmaThreads;
    if (fp32_tflops && e == cudaSuccess) {
        float ms = 0;
        e = time_best([&] {
            k_fma_peak<<<blocks, kFmaThreads, 0, st>>>(iters, 1.0f, static_cast<float*>(sink));
            return cudaGetLastError();
        }, 5, &ms);
        if (e == cudaSuccess) *fp32_tflops = fma_threads * iters * kFmaChains * 4.0 / (ms * 1e-3) / 1e12;
    }
    if (fp32_scalar_tflops && e == cudaSuccess) {
        float ms = 0;
        e = time_best([&] {
            k_fma_peak_scalar<<<blocks, kFmaThreads, 0, st>>>(iters, 1.0f,
                                                              static_cast<float*>(sink));
            return cudaGetLastError();
        }, 5, &ms);
        if (e == cudaSuccess)
            *fp32_scalar_tflops = fma_threads * iters * 2 * kFmaChains * 2.0 / (ms * 1e-3) / 1e12;
    }
    if (fp64_tflops && e == cudaSuccess) {
        // FP64 runs far slower than FP32 on this part: fewer rounds per thread
        const int it64 = 256;
        float ms = 0;
        e = time_best([&] {
            k_fma_peak_f64<<<blocks, kFmaThreads, 0, st>>>(it64, 1.0, static_cast<double*>(sink));
            return cudaGetLastError();
        }, 5, &ms);
        if (e == cudaSuccess) *fp64_tflops = fma_threads * it64 * kFmaChains * 2.0 / (ms * 1e-3) / 1e12;
    }
    if (l2_read_gbs && e == cudaSuccess) {
        // 32 MiB: a quarter of L2, re-read 16 times per launch
        const size_t bytes = size_t(32) << 20;
        void* buf = nullptr;
        e = cudaMallocAsync(&buf, bytes, st);
        if (e == cudaSuccess) e = cudaMemsetAsync(buf, 1, bytes, st);
        const int reps = 16;
        float ms = 0;
        if (e == cudaSuccess)
            e = time_best([&] {
                k_l2_read<<<nsm * 4, 512, 0, st>>>(static_cast<const uint4*>(buf), bytes / 16,
                                                   reps, static_cast<unsigned*>(sink));
                return cudaGetLastError();
            }, 5, &ms);
        if (e == cudaSuccess) *l2_read_gbs = double(bytes) * reps / (ms * 1e-3) / 1e9;
        if (buf) cudaFreeAsync(buf, st);
    }
    cudaFreeAsync(sink, st);
    const cudaError_t e2 = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "shg_measure_peaks");
    if (e2 != cudaSuccess) return cuda_fail(e2, "shg_measure_peaks");
    return SHG_OK;
}
