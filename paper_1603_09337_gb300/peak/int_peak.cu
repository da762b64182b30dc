// int_peak.cu -- measured issue rate of the 32-bit integer instruction
// classes the HASF kernels are built from, for the benchmark's roofline.
//
// Each probe kernel keeps eight independent dependency chains per thread and
// runs one instruction class in a fully unrolled loop, so that the
// instruction under test dominates the issue slots (the loop counter and
// branch add 2 instructions per 64 probed ones).  The grid fills every SM
// with 2,048 threads.  Timed with CUDA events; reported in lane-operations
// per second (warp instructions x 32).
#include <cstdint>
#include <cuda_runtime.h>

#include "hasf_peak.h"

namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 8;   // probed instructions per chain per loop trip

template <int KIND>
__global__ void __launch_bounds__(512) int_probe_kernel(uint32_t* out, int iters, uint32_t b,
                                                       uint32_t c) {
  uint32_t a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = threadIdx.x * 0x9E3779B9u + k * 0x85EBCA6Bu + b;
  const uint32_t sh = c & 31u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
#pragma unroll
      for (int k = 0; k < kChains; ++k) {
        if (KIND == HASF_PEAK_LOP3) a[k] = (a[k] & b) ^ (c | u);        // one LOP3
        if (KIND == HASF_PEAK_SHF) a[k] = __funnelshift_r(a[k], b, sh);  // one SHF
        if (KIND == HASF_PEAK_IADD3) a[k] = a[k] + a[(k + 1) & 7] + c;  // one IADD3
        if (KIND == HASF_PEAK_SHFL) a[k] = __shfl_xor_sync(0xFFFFFFFFu, a[k], 1 + (k & 3));
      }
    }
  }
  uint32_t x = 0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) x ^= a[k];
  if (x == 0x12345678u) out[blockIdx.x * blockDim.x + threadIdx.x] = x;  // keeps the chains live
}

template <int KIND>
cudaError_t run_probe(int sms, int iters, uint32_t* d_out, cudaEvent_t e0, cudaEvent_t e1,
                      float* ms) {
  const int grid = sms * 4, block = 512;
  int_probe_kernel<KIND><<<grid, block>>>(d_out, 16, 0x0F0F0F0Fu, 5u);  // warm-up
  cudaEventRecord(e0);
  int_probe_kernel<KIND><<<grid, block>>>(d_out, iters, 0x0F0F0F0Fu, 5u);
  cudaEventRecord(e1);
  cudaError_t e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  return e;
}

}  // namespace

extern "C" int hasf_peak_int(int kind, int device, double* lane_ops_per_s, float* ms_out) {
  if (!lane_ops_per_s || kind < HASF_PEAK_LOP3 || kind > HASF_PEAK_SHFL) return 1;
  if (cudaSetDevice(device) != cudaSuccess) return 2;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      sms < 1)
    return 2;
  const int iters = 4096;
  uint32_t* d_out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&d_out, (size_t)sms * 4 * 512 * sizeof(uint32_t)) != cudaSuccess) return 2;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  cudaError_t e = cudaErrorInvalidValue;
  switch (kind) {
    case HASF_PEAK_LOP3: e = run_probe<HASF_PEAK_LOP3>(sms, iters, d_out, e0, e1, &ms); break;
    case HASF_PEAK_SHF: e = run_probe<HASF_PEAK_SHF>(sms, iters, d_out, e0, e1, &ms); break;
    case HASF_PEAK_IADD3: e = run_probe<HASF_PEAK_IADD3>(sms, iters, d_out, e0, e1, &ms); break;
    case HASF_PEAK_SHFL: e = run_probe<HASF_PEAK_SHFL>(sms, iters, d_out, e0, e1, &ms); break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(d_out);
  if (e != cudaSuccess || ms <= 0.f) return 2;
  const double ops = (double)sms * 4 * 512 * (double)iters * kUnroll * kChains;
  *lane_ops_per_s = ops / (ms * 1e-3);
  if (ms_out) *ms_out = ms;
  return 0;
}
