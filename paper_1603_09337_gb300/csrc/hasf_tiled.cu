// hasf_tiled.cu -- the tiled register kernels (images larger than one tile:
// thread-block clusters and gangs) and their launchers.  Each kernel has two
// instances.  MINB = 2 fits two CTAs per SM (64 registers, 93 KB of shared
// memory: the movable mask is read from the constraint planes instead of being
// kept in shared memory): the sweeps wait on exchanges, a second CTA per SM
// fills those waits, and a gang of more tiles than SMs fits.  MINB = 1 (128
// registers, no spills) serves plans whose CTAs all fit one per SM.
#include <cstdint>
#include <cuda_runtime.h>

#include "hasf_device.cuh"
#include "hasf_reg.cuh"
#include "hasf_tiled.cuh"

namespace hasf {

// One cluster of ntx * nty CTAs per image: cluster i works on job order[i].
// MINB as for the gang kernel below.
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
hasf_tile_cluster_kernel(const Job* __restrict__ jobs, const int* __restrict__ order) {
  extern __shared__ uint4 smem4[];
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem4);
  __shared__ int flags[3];
  cg::cluster_group cl = cg::this_cluster();
  const int csize = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const Job& jb = jobs[order[blockIdx.x / csize]];
  const int ntx = tiles_x(jb.w);
  TileCtx<ClusterX> k;
  tile_init(k, jb, smem, rank % ntx, rank / ntx);
  k.x.halo2 = k.halo2;
  k.x.Fc = k.g.F;
  k.x.flags = flags;
  k.x.slot = 0;
  for (int t = threadIdx.x; t < kTileSmemWords; t += blockDim.x) smem[t] = 0u;
  if (threadIdx.x == 0) flags[0] = flags[1] = flags[2] = 0;
  cl.sync();   // every tile's halo is zero before any neighbour stores into it
  if (jb.conn == 4) tile_job<4>(k, jb, smem);
  else tile_job<8>(k, jb, smem);
  cl.sync();   // no CTA leaves while others may still read its shared memory
}

// Gang mode with tiles: CTA b works on tile ctamap[b].y of job ctamap[b].x.
// MINB = 2 is the default; a plan whose CTAs all fit one per SM uses
// MINB = 1 (one CTA per SM with twice the registers, no spills).
template <int MINB>
__global__ void __launch_bounds__(kThreads, MINB)
hasf_tile_gang_kernel(const Job* __restrict__ jobs, const int2* __restrict__ ctamap) {
  extern __shared__ uint4 smem4[];
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem4);
  __shared__ __align__(8) int flag[4];  // gang barrier state (GangMode)
  const int2 m = ctamap[blockIdx.x];
  const Job& jb = jobs[m.x];
  if (gang_fault_leaves(jb.fault_skip, jb.gang, m.y)) {
    job_done(jb, jb.gang);
    return;
  }
  const int ntx = tiles_x(jb.w);
  TileCtx<GangX> k;
  tile_init(k, jb, smem, m.y % ntx, m.y / ntx);
  k.x.gbase = jb.planes;
  k.x.gm.init(jb.sync, jb.gang, flag, jb.deadline_ms);
  for (int t = threadIdx.x; t < kTileSmemWords; t += blockDim.x) smem[t] = 0u;
  __syncthreads();
  if (jb.conn == 4) tile_job<4>(k, jb, smem);
  else tile_job<8>(k, jb, smem);
}

cudaError_t set_level_table_tiled(const void* tab, size_t bytes) {
  return cudaMemcpyToSymbol(c_lv, tab, bytes);
}

size_t tile_kernel_smem() { return tile_smem_bytes(); }
int tile_count(int w, int h) { return tiles_x(w) * tiles_y(h); }
size_t tile_gang_words(int w, int h) { return (size_t)tile_count(w, h) * kGangTileWords; }

// Clusters of csize CTAs of the tile kernel that can run at once (0: none).
int tile_clusters_possible(int csize) {
  if (csize < 1 || csize > 16) return 0;
  const size_t smem = tile_smem_bytes();
  cudaFuncSetAttribute(hasf_tile_cluster_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaFuncSetAttribute(hasf_tile_cluster_kernel<2>,
                       cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(csize);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = csize;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, hasf_tile_cluster_kernel<2>, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_tile_cluster(const Job* d_jobs, const int* d_order, int njobs, int csize,
                                bool alone, cudaStream_t s) {
  const size_t smem = tile_smem_bytes();
  const void* fn = alone ? (const void*)hasf_tile_cluster_kernel<1>
                         : (const void*)hasf_tile_cluster_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(njobs * csize);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr;
  attr.id = cudaLaunchAttributeClusterDimension;
  attr.val.clusterDim.x = csize;
  attr.val.clusterDim.y = 1;
  attr.val.clusterDim.z = 1;
  cfg.attrs = &attr;
  cfg.numAttrs = 1;
  void* args[] = {(void*)&d_jobs, (void*)&d_order};
  return cudaLaunchKernelExC(&cfg, fn, args);
}

int max_tile_gang_ctas(int device) {
  int per_sm = 0, sms = 0;
  const size_t smem = tile_smem_bytes();
  cudaFuncSetAttribute(hasf_tile_gang_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hasf_tile_gang_kernel<2>, kThreads, smem);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

cudaError_t launch_tile_gang(const Job* d_jobs, const int2* d_ctamap, int nctas, bool alone,
                             cudaStream_t s) {
  const size_t smem = tile_smem_bytes();
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = (alone && nctas <= sms) ? (const void*)hasf_tile_gang_kernel<1>
                                           : (const void*)hasf_tile_gang_kernel<2>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {(void*)&d_jobs, (void*)&d_ctamap};
  return cudaLaunchCooperativeKernel(fn, dim3(nctas), dim3(kThreads), args, smem, s);
}

}  // namespace hasf
