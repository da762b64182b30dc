// hasf_reg_kernel.cuh -- the register kernel (one CTA per image of at most
// 512 x 512) as a template over its sweep schedule, and the launch helpers of
// one instance.  Each schedule is compiled in its own translation unit
// (hasf_reg.cu: 4 rows per group, hasf_reg_g2.cu: 2, hasf_reg_g1.cu: 1).
#pragma once

namespace hasf {

// One job on this CTA: the register context over the dynamic shared memory,
// then the job's operators.
template <int G>
__device__ __forceinline__ void reg_run_job(const Job& jb, uint32_t* smem) {
  RegCtx k;
  Ctx<SmemMode>& g = k.g;
  g.w = jb.w;
  g.h = jb.h;
  g.wpr = jb.wpr;
  g.P = row_pitch(jb.w);
  const int rem = jb.w & 31;
  g.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
  g.S = nullptr;
  g.F = smem + 1 + kRegPadR * g.P;
  g.cand = nullptr;
  g.cap = jb.cap;
  if (threadIdx.x < STAT_COUNT) s_reg_stats[threadIdx.x] = 0u;  // ordered by the job's first barrier
  k.M = smem + reg_f_words(jb.w, jb.h);
  k.cand = k.M + kRegPlane;
  k.top = k.cand + kRegPlane;
  k.bot = k.top + (kThreads / 32) * kRegW;
  k.warp = threadIdx.x >> 5;
  k.half = (threadIdx.x >> 4) & 1;
  k.j = threadIdx.x & 15;
  k.s0 = (2 * k.warp + k.half) * kRegR;
  k.jin = k.j < jb.wpr;
  if (jb.conn == 4) reg_job<4, G>(k, jb, smem);
  else reg_job<8, G>(k, jb, smem);
}

// Persistent CTAs of kThreads threads take register-path jobs from `order`.
// G: rows of a parity tested together in a sweep (the sweep schedule).
template <int G>
__global__ void __launch_bounds__(kThreads, 2)
hasf_reg_kernel(const Job* __restrict__ jobs, const int* __restrict__ order, int njobs,
                unsigned* counter) {
  extern __shared__ uint4 smem4[];
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem4);
  __shared__ int next;
  for (;;) {
    if (threadIdx.x == 0) next = (int)atomicAdd(counter, 1u);
    __syncthreads();
    const int slot = next;
    __syncthreads();
    if (slot >= njobs) break;
    reg_run_job<G>(jobs[order[slot]], smem);
    __syncthreads();
  }
}

// One CTA, one job passed by value: the form that needs no device memory for
// its job list (the allocation-free entry point).
template <int G>
__global__ void __launch_bounds__(kThreads, 2) hasf_reg_one_kernel(const Job jb) {
  extern __shared__ uint4 smem4[];
  reg_run_job<G>(jb, reinterpret_cast<uint32_t*>(smem4));
}

template <int G>
cudaError_t reg_launch_instance(const Job* d_jobs, const int* d_order, int njobs, int grid,
                                size_t smem_bytes, unsigned* d_counter, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(hasf_reg_kernel<G>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  hasf_reg_kernel<G><<<grid, kThreads, smem_bytes, s>>>(d_jobs, d_order, njobs, d_counter);
  return cudaGetLastError();
}

}  // namespace hasf
