// hasf_reg.cu -- the register kernel with four rows per sweep group, and the
// launchers that dispatch to the instance of the chosen sweep schedule.
#include <cstdint>
#include <cuda_runtime.h>

#include "hasf_device.cuh"
#include "hasf_reg.cuh"
#include "hasf_reg_kernel.cuh"

namespace hasf {

cudaError_t set_level_table_reg(const void* tab, size_t bytes) {
  cudaError_t e = cudaMemcpyToSymbol(c_lv, tab, bytes);
  if (e == cudaSuccess) e = set_level_table_reg_g2(tab, bytes);
  if (e == cudaSuccess) e = set_level_table_reg_g1(tab, bytes);
  return e;
}

size_t reg_kernel_smem(int w, int h) { return reg_smem_bytes(w, h); }
bool reg_kernel_ok(int w, int h, int rmax) { return reg_kernel_fits(w, h, rmax); }

int reg_ctas_per_sm(size_t smem_bytes) {
  int n = 0;
  cudaFuncSetAttribute(hasf_reg_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem_bytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hasf_reg_kernel<4>, kThreads, smem_bytes);
  return n;
}

// The one-job kernel (four rows per sweep group): its shared-memory limit is
// raised once to what the largest register-path image needs.
cudaError_t reg_one_prepare() {
  return cudaFuncSetAttribute(hasf_reg_one_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)reg_smem_bytes(32 * kRegW, kRegRows));
}
cudaError_t launch_reg_one(const Job& jb, cudaStream_t s) {
  hasf_reg_one_kernel<4><<<1, kThreads, reg_smem_bytes(jb.w, jb.h), s>>>(jb);
  return cudaGetLastError();
}

cudaError_t launch_reg(int group, const Job* d_jobs, const int* d_order, int njobs, int grid,
                       size_t smem_bytes, unsigned* d_counter, cudaStream_t s) {
  switch (group) {
    case 1: return launch_reg_g1(d_jobs, d_order, njobs, grid, smem_bytes, d_counter, s);
    case 2: return launch_reg_g2(d_jobs, d_order, njobs, grid, smem_bytes, d_counter, s);
    case 4: return reg_launch_instance<4>(d_jobs, d_order, njobs, grid, smem_bytes, d_counter, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hasf
