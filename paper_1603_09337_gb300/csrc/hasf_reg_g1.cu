// hasf_reg_g1.cu -- the register kernel with 1 row per sweep group.
#include <cstdint>
#include <cuda_runtime.h>

#include "hasf_device.cuh"
#include "hasf_reg.cuh"
#include "hasf_reg_kernel.cuh"

namespace hasf {

cudaError_t set_level_table_reg_g1(const void* tab, size_t bytes) {
  return cudaMemcpyToSymbol(c_lv, tab, bytes);
}

cudaError_t launch_reg_g1(const Job* d_jobs, const int* d_order, int njobs, int grid,
                          size_t smem_bytes, unsigned* d_counter, cudaStream_t s) {
  return reg_launch_instance<1>(d_jobs, d_order, njobs, grid, smem_bytes, d_counter, s);
}

}  // namespace hasf
