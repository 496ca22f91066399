// Throughput probes (measurement utilities for the benchmark's roofline
// denominators; no counterpart in the paper).  Built as libinla_probe.so,
// separate from the product library; declared in include/inla_probe.h.
// Every SM runs register-resident chains of independent fused multiply-adds
// (FP64 scalar FMA, the warp-level m8n8k4 double-precision MMA instruction,
// or FP32 scalar FMA) for a fixed number of iterations; the rate is
// flops / CUDA-event time.  The loops are bounded and touch no memory except
// one store per thread at the end (so the compiler cannot drop them).
#include <cuda_runtime.h>

#include <string>

#include "../../include/inla_probe.h"

namespace {

thread_local std::string g_probe_err;
void set_error(const char *msg) { g_probe_err = msg; }

constexpr int CHAINS = 8;

__global__ void __launch_bounds__(256) dfma_probe(int iters, double *sink) {
  double a[CHAINS];
  const double x = 1.0 + 1e-9 * threadIdx.x, y = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = 0.5 * c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) dmma_probe(int iters, double *sink) {
  double acc[CHAINS][2];
  const double av = 1.0 + 1e-9 * threadIdx.x, bv = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc[c][0] = acc[c][1] = 0.25 * c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      asm volatile(
          "mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
          : "+d"(acc[c][0]), "+d"(acc[c][1])
          : "d"(av), "d"(bv));
    }
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += acc[c][0] + acc[c][1];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Both FP64 paths at once: even warps run the DFMA chains, odd warps the DMMA
// chains, to see whether the scalar FP64 pipe and the FP64 tensor path add up.
__global__ void __launch_bounds__(256) dboth_probe(int iters, double *sink) {
  const int warp = threadIdx.x >> 5;
  double s = 0.0;
  if (warp & 1) {
    double acc[CHAINS][2];
    const double av = 1.0 + 1e-9 * threadIdx.x, bv = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) acc[c][0] = acc[c][1] = 0.25 * c;
    for (int i = 0; i < iters / 4; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c)
        asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0, %1}, {%2}, {%3}, {%0, %1};\n"
                     : "+d"(acc[c][0]), "+d"(acc[c][1])
                     : "d"(av), "d"(bv));
    }
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += acc[c][0] + acc[c][1];
  } else {
    double a[CHAINS];
    const double x = 1.0 + 1e-9 * threadIdx.x, y = 1.0 - 1e-9 * blockIdx.x;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = 0.5 * c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], x, y);
    }
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
  }
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma_probe(int iters, float *sink) {
  float a[CHAINS];
  const float x = 1.0f + 1e-7f * threadIdx.x, y = 1.0f - 1e-7f * blockIdx.x;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = 0.5f * c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = fmaf(a[c], x, y);
  }
  float s = 0.0f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

extern "C" const char *inla_probe_last_error(void) { return g_probe_err.c_str(); }

extern "C" int inla_measure_fp32_peak(int device, double *tflops) {
  if (!tflops) {
    set_error("tflops is NULL");
    return INLA_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return INLA_ERR_CUDA;
  }
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  const int blocks = prop.multiProcessorCount * 8, threads = 256, iters = 1 << 16;
  float *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(float) * blocks * threads) != cudaSuccess) {
    set_error("cudaMalloc failed");
    return INLA_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    ffma_probe<<<blocks, threads>>>(iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) {
    set_error(cudaGetErrorString(err));
    return INLA_ERR_CUDA;
  }
  *tflops = (double)blocks * threads * CHAINS * 2 * iters / (best * 1e-3) / 1e12;
  return INLA_OK;
}

extern "C" int inla_measure_fp64_peak(int device, int use_tensor, double *tflops) {
  if (!tflops) {
    set_error("tflops is NULL");
    return INLA_ERR_ARG;
  }
  if (cudaSetDevice(device) != cudaSuccess) {
    set_error("cudaSetDevice failed");
    return INLA_ERR_CUDA;
  }
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, device);
  const int blocks = prop.multiProcessorCount * 4, threads = 256;
  const int iters = use_tensor ? (1 << 14) : (1 << 16);
  double *sink = nullptr;
  if (cudaMalloc(&sink, sizeof(double) * blocks * threads) != cudaSuccess) {
    set_error("cudaMalloc failed");
    return INLA_ERR_OOM;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0);
    if (use_tensor == 2) dboth_probe<<<blocks, threads>>>(1 << 16, sink);
    else if (use_tensor) dmma_probe<<<blocks, threads>>>(iters, sink);
    else dfma_probe<<<blocks, threads>>>(iters, sink);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  cudaError_t err = cudaGetLastError();
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (err != cudaSuccess) {
    set_error(cudaGetErrorString(err));
    return INLA_ERR_CUDA;
  }
  // scalar: 2 flops per FMA per thread; MMA m8n8k4: 8*8*4 FMAs per warp instruction
  double flops;
  if (use_tensor == 2)   // half the warps: 2^16 DFMA steps; the other half: 2^14 DMMA steps
    flops = (double)blocks * (threads / 2) * CHAINS * 2 * (1 << 16) +
            (double)blocks * (threads / 64) * CHAINS * 8 * 8 * 4 * 2 * (1 << 14);
  else if (use_tensor)
    flops = (double)blocks * (threads / 32) * CHAINS * 8 * 8 * 4 * 2 * iters;
  else
    flops = (double)blocks * threads * CHAINS * 2 * iters;
  *tflops = flops / (best * 1e-3) / 1e12;
  return INLA_OK;
}
