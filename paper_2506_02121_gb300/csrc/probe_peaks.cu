// Arithmetic-rate probes for the roofline denominators of the root finder: FP32 FMA lane
// operations per second (scalar FFMA and packed fma.rn.f32x2) and FP64 FMA per second, by
// a grid of independent FMA chains long enough that launch overhead does not count.
// Separate from libccgpu (built as libccprobe.so): it is a measurement tool, not part of
// the method.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

constexpr int kChains = 8;  // independent chains per thread: enough to cover the FMA latency

__global__ void ffma_loop(float* out, int iters, float a, float b) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = (float)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void ffma2_loop(float* out, int iters, float a, float b) {
    unsigned long long v[kChains];
    unsigned long long aa, bb;
    asm("mov.b64 %0, {%1, %2};" : "=l"(aa) : "f"(a), "f"(a));
    asm("mov.b64 %0, {%1, %2};" : "=l"(bb) : "f"(b), "f"(b));
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        const float x = (float)(threadIdx.x + c), y = x + 0.5f;
        asm("mov.b64 %0, {%1, %2};" : "=l"(v[c]) : "f"(x), "f"(y));
    }
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(v[c]) : "l"(aa), "l"(bb));
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kChains; c++) {
        float x, y;
        asm("mov.b64 {%0, %1}, %2;" : "=f"(x), "=f"(y) : "l"(v[c]));
        s += x + y;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void dfma_loop(double* out, int iters, double a, double b) {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; c++) v[c] = (double)(threadIdx.x + c);
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int c = 0; c < kChains; c++) v[c] = fma(v[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; c++) s += v[c];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" {

// Runs one probe on stream 0 and returns its device time in milliseconds (CUDA events),
// with *lane_ops = the FMA lane operations it executed.  kind: 0 scalar FP32 FFMA,
// 1 packed FP32 (two lane operations per instruction), 2 FP64 DFMA.  out must hold
// blocks * threads elements of the probe's type (device memory).  Returns a negative
// value on a CUDA error.
double ccprobe_fma_rate(int kind, int blocks, int threads, int iters, void* out, double* lane_ops) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1.0;
    cudaEventRecord(e0, 0);
    if (kind == 0)
        ffma_loop<<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
    else if (kind == 1)
        ffma2_loop<<<blocks, threads>>>((float*)out, iters, 0.999999f, 1e-7f);
    else
        dfma_loop<<<blocks, threads>>>((double*)out, iters, 0.9999999999, 1e-12);
    cudaEventRecord(e1, 0);
    cudaError_t err = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (err == cudaSuccess) err = cudaGetLastError();
    if (err == cudaSuccess) err = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (err != cudaSuccess) return -1.0;
    *lane_ops = (double)blocks * threads * (double)iters * kChains * (kind == 1 ? 2.0 : 1.0);
    return (double)ms;
}

}  // extern "C"
