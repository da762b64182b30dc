// hasf_kernels.cu -- generic HASF kernels (resident and gang modes), the
// check kernels, the level table and the allocation-free entry point.
// The device code they share with the register and tiled kernels is in
// hasf_device.cuh.
#include <cstdint>
#include <mutex>
#include <cuda_runtime.h>

#include "hasf_device.cuh"

namespace hasf {

// Resident mode: persistent CTAs take jobs from `order` through a counter.
__global__ void __launch_bounds__(kThreads, 2)
hasf_resident_kernel(const Job* __restrict__ jobs, const int* __restrict__ order, int njobs,
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
    const Job& jb = jobs[order[slot]];
    Ctx<SmemMode> k;
    init_ctx(k, jb, smem, threadIdx.x, blockDim.x);
    if (jb.conn == 4) run_job<SmemMode, 4>(k, jb, smem);
    else run_job<SmemMode, 8>(k, jb, smem);
    __syncthreads();
  }
}

// Gang mode: CTA b works on job ctamap[b].x as part ctamap[b].y of jobs[].gang.
__global__ void __launch_bounds__(kThreads, 1)
hasf_gang_kernel(const Job* __restrict__ jobs, const int2* __restrict__ ctamap) {
  __shared__ __align__(8) int flag[4];  // gang barrier state (GangMode)
  const int2 m = ctamap[blockIdx.x];
  const Job& jb = jobs[m.x];
  if (gang_fault_leaves(jb.fault_skip, jb.gang, m.y)) {
    job_done(jb, jb.gang);
    return;
  }
  Ctx<GangMode> k;
  k.m.init(jb.sync, jb.gang, flag, jb.deadline_ms);
  init_ctx(k, jb, jb.planes, m.y * blockDim.x + threadIdx.x, jb.gang * blockDim.x);
  if (jb.conn == 4) run_job<GangMode, 4>(k, jb, jb.planes);
  else run_job<GangMode, 8>(k, jb, jb.planes);
}


// All 256 neighbour codes through simple_bits: thread t builds the 3 x 3
// words whose bit 1 holds the code t's neighbourhood and reads bit 1.
__global__ void simple_table_kernel(int conn, uint8_t* out) {
  const int code = threadIdx.x;
  if (code >= 256) return;
  // Pixel under test: bit 1 of the centre word.  Neighbour k at (dx, dy).
  const int dxs[8] = {1, 1, 0, -1, -1, -1, 0, 1};
  const int dys[8] = {0, -1, -1, -1, 0, 1, 1, 1};
  uint32_t rows[3] = {0u, 0u, 0u};
  for (int k = 0; k < 8; ++k)
    if ((code >> k) & 1) rows[1 + dys[k]] |= 1u << (1 + dxs[k]);
  const uint32_t r = conn == 4 ? simple_bits<4>(0, rows[0], 0, 0, rows[1], 0, 0, rows[2], 0)
                               : simple_bits<8>(0, rows[0], 0, 0, rows[1], 0, 0, rows[2], 0);
  out[code] = (uint8_t)((r >> 1) & 1u);
}

// Priority levels of every pixel, from the same threshold walk the fused
// kernel uses (one CTA per row band, packed planes in global memory).
// Pixels past the width in the last word of a row are outside the box: they
// are packed as `pad` so that, read through xor inv, they give outv.
__global__ void levels_pack_kernel(const uint8_t* feat, int w, int h, int pitch, uint32_t* Fp,
                                   uint32_t pad) {
  const int wpr = words_per_row(w);
  const int P = row_pitch(w);
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int it = gwarp; it < h * wpr; it += nwarps) {
    const int y = it / wpr, j = it - y * wpr;
    const int x = (j << 5) + lane;
    const uint32_t v = __ballot_sync(0xFFFFFFFFu, x < w ? feat[(size_t)y * pitch + x] != 0
                                                        : ((pad >> lane) & 1u) != 0);
    if (lane == 0) Fp[1 + (y + 1) * P + j] = v;
  }
}

__global__ void levels_walk_kernel(int w, int h, int mode, int r, const uint32_t* Fbase,
                                   int32_t* d) {
  Ctx<SmemMode> k;  // geometry only; loads are plain global loads
  k.w = w;
  k.h = h;
  k.wpr = words_per_row(w);
  k.P = row_pitch(w);
  const int rem = w & 31;
  k.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
  const uint32_t inv = mode == 2 ? 0xFFFFFFFFu : 0u;
  const uint32_t outv = mode >= 1 ? 0xFFFFFFFFu : 0u;
  const uint32_t* F = Fbase + 1;
  const int nlev = c_lv.nlev[r];
  const int total = h * k.wpr;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < total; t += gridDim.x * blockDim.x) {
    const int y = t / k.wpr, j = t - y * k.wpr;
    const uint32_t valid = k.rowmask(j);
    // Level 0: the feature points themselves.
    uint32_t done = fshift(k, F, y, j, 0, inv, outv) & valid;
    int32_t* row = d + (size_t)y * w + (j << 5);
    for (int b = 0; b < 32; ++b)
      if ((valid >> b) & 1u) row[b] = ((done >> b) & 1u) ? 0 : r * r + 1;
    for (int li = 0; li < nlev && done != valid; ++li) {
      uint32_t ring = 0;
      for (int o = c_lv.start[li]; o < c_lv.start[li + 1]; ++o)
        ring |= fshift(k, F, y + c_lv.off[o][1], j, c_lv.off[o][0], inv, outv);
      uint32_t fresh = ring & valid & ~done;
      while (fresh) {
        const int b = __ffs(fresh) - 1;
        fresh &= fresh - 1u;
        row[b] = c_lv.value[li];
      }
      done |= ring & valid;
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

namespace {
// The host copy of the level table, built once (std::call_once: contexts and
// the allocation-free entry point may upload it from several threads).
LevelTable g_level_tab;
bool g_level_tab_ok = false;
std::once_flag g_level_tab_once;

void build_level_table() {
  LevelTable& tab = g_level_tab;
  // Sort the lattice vectors of the disc of radius kMaxR by squared norm.
  int n = 0;
  const int R = kMaxR;
  static int norms[kMaxOffsets];
  static int8_t vecs[kMaxOffsets][2];
  for (int dy = -R; dy <= R; ++dy)
    for (int dx = -R; dx <= R; ++dx) {
      const int q = dx * dx + dy * dy;
      if (q == 0 || q > R * R) continue;
      norms[n] = q;
      vecs[n][0] = (int8_t)dx;
      vecs[n][1] = (int8_t)dy;
      ++n;
    }
  // counting sort by norm (stable)
  static int count[kMaxR * kMaxR + 2];
  for (int i = 0; i <= R * R + 1; ++i) count[i] = 0;
  for (int i = 0; i < n; ++i) ++count[norms[i] + 1];
  for (int i = 1; i <= R * R + 1; ++i) count[i] += count[i - 1];
  static int pos[kMaxR * kMaxR + 2];
  for (int i = 0; i <= R * R + 1; ++i) pos[i] = count[i];
  for (int i = 0; i < n; ++i) {
    const int p = pos[norms[i]]++;
    tab.off[p][0] = vecs[i][0];
    tab.off[p][1] = vecs[i][1];
  }
  int nl = 0;
  for (int q = 1; q <= R * R; ++q) {
    if (count[q + 1] == count[q]) continue;
    tab.value[nl] = (uint16_t)q;
    tab.start[nl] = (uint16_t)count[q];
    ++nl;
  }
  tab.start[nl] = (uint16_t)n;
  for (int r = 0; r <= R; ++r) {
    int c = 0;
    while (c < nl && tab.value[c] <= r * r) ++c;
    tab.nlev[r] = (uint16_t)c;
  }
  g_level_tab_ok = (n == kMaxOffsets && nl == kMaxLevels);
}
}  // namespace

cudaError_t upload_level_table() {
  std::call_once(g_level_tab_once, build_level_table);
  if (!g_level_tab_ok) return cudaErrorInvalidValue;
  const LevelTable& tab = g_level_tab;
  cudaError_t e = cudaMemcpyToSymbol(c_lv, &tab, sizeof(tab));
  if (e == cudaSuccess) e = set_level_table_reg(&tab, sizeof(tab));
  if (e == cudaSuccess) e = set_level_table_tiled(&tab, sizeof(tab));
  return e;
}

size_t max_resident_smem(int device) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
  return (size_t)v;
}

int resident_ctas_per_sm(int device, size_t smem_bytes) {
  (void)device;
  int n = 0;
  cudaFuncSetAttribute(hasf_resident_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)smem_bytes);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, hasf_resident_kernel, kThreads, smem_bytes);
  return n;
}

cudaError_t launch_resident(const Job* d_jobs, const int* d_order, int njobs, int grid,
                            size_t smem_bytes, unsigned* d_counter, cudaStream_t s) {
  cudaError_t e = cudaFuncSetAttribute(hasf_resident_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes);
  if (e != cudaSuccess) return e;
  hasf_resident_kernel<<<grid, kThreads, smem_bytes, s>>>(d_jobs, d_order, njobs, d_counter);
  return cudaGetLastError();
}

int max_gang_ctas(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hasf_gang_kernel, kThreads, 0);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

cudaError_t launch_gang(const Job* d_jobs, const int2* d_ctamap, int nctas, cudaStream_t s) {
  void* args[] = {(void*)&d_jobs, (void*)&d_ctamap};
  return cudaLaunchCooperativeKernel((const void*)hasf_gang_kernel, dim3(nctas), dim3(kThreads),
                                     args, 0, s);
}

cudaError_t launch_simple_table(int conn, uint8_t* d_out256, cudaStream_t s) {
  simple_table_kernel<<<1, 256, 0, s>>>(conn, d_out256);
  return cudaGetLastError();
}

// A batch of 2D byte copies in one launch (host buffers mapped into the
// device's address space to or from device buffers): blockIdx.y is the copy,
// the blocks along x stride over its 16-byte chunks (or bytes, when a row or
// a pointer is not 16-byte aligned).
__global__ void __launch_bounds__(256) copy2d_kernel(const Copy2D* __restrict__ copies) {
  const Copy2D c = copies[blockIdx.y];
  const bool vec = ((reinterpret_cast<uintptr_t>(c.src) | reinterpret_cast<uintptr_t>(c.dst) |
                     (uintptr_t)c.spitch | (uintptr_t)c.dpitch | (uintptr_t)c.w) & 15u) == 0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (vec) {
    const int cpr = c.w >> 4;
    const long long total = (long long)c.h * cpr;
    for (long long i = first; i < total; i += stride) {
      const int y = (int)(i / cpr), k = (int)(i - (long long)y * cpr);
      reinterpret_cast<uint4*>(c.dst + (size_t)y * c.dpitch)[k] =
          reinterpret_cast<const uint4*>(c.src + (size_t)y * c.spitch)[k];
    }
  } else {
    const long long total = (long long)c.h * c.w;
    for (long long i = first; i < total; i += stride) {
      const int y = (int)(i / c.w), x = (int)(i - (long long)y * c.w);
      c.dst[(size_t)y * c.dpitch + x] = c.src[(size_t)y * c.spitch + x];
    }
  }
}

cudaError_t launch_copy2d(const Copy2D* d_copies, int n, cudaStream_t s) {
  for (int at = 0; at < n; at += 65535) {
    const int m = n - at < 65535 ? n - at : 65535;
    copy2d_kernel<<<dim3(16, m), 256, 0, s>>>(d_copies + at);
  }
  return cudaGetLastError();
}

cudaError_t launch_levels(const uint8_t* feat, int w, int h, int pitch, int mode, int r,
                          uint32_t* d_plane_f, uint32_t* d_plane_a, int32_t* d, cudaStream_t s) {
  const int pw = plane_words(w, h);
  cudaError_t e = cudaMemsetAsync(d_plane_f, 0, (size_t)pw * 4, s);
  if (e != cudaSuccess) return e;
  // mode 1 reads F as is with the outside as feature: pad bits must read 1
  const uint32_t pad = mode == 1 ? 0xFFFFFFFFu : 0u;
  (void)d_plane_a;
  levels_pack_kernel<<<256, 256, 0, s>>>(feat, w, h, pitch, d_plane_f, pad);
  levels_walk_kernel<<<512, 128, 0, s>>>(w, h, mode, r, d_plane_f, d);
  return cudaGetLastError();
}

}  // namespace hasf

// ---------------------------------------------------------------------------
// Allocation-free entry point.
//
// Some callers cannot call cudaMalloc: latency-critical loops that must not
// stall on an allocation (cudaMalloc may synchronise the device), and code
// running inside a host framework or plug-in whose device memory is owned by
// that framework's allocator and budget.  hasf_smooth_noalloc serves them: it
// runs one image on one CTA, through the register kernel (the job passed by
// value) when the image is at most 512 x 512 and rmax <= 31, else through the
// fused kernel in resident mode (bit planes in shared memory), and keeps the
// kernels' global scratch -- the operator-input snapshot and the packed C and
// D planes -- in the file-scope array below instead of memory from a context.
// The array is part of the library image: every GPU that loads the library
// holds it (about 240 KB) until the process exits.
// ---------------------------------------------------------------------------
namespace hasf {

constexpr int kStaticPlaneWords = 20480;  // h * ceil(w / 32) words per plane, at most
constexpr int kStaticWords = 3 * kStaticPlaneWords + 64;  // g0, cp, dp, status

static __device__ __align__(256) uint32_t g_noalloc_scratch[kStaticWords];

__global__ void __launch_bounds__(kThreads, 2) hasf_single_kernel(Job jb) {
  extern __shared__ uint4 smem4[];
  uint32_t* smem = reinterpret_cast<uint32_t*>(smem4);
  Ctx<SmemMode> k;
  init_ctx(k, jb, smem, threadIdx.x, blockDim.x);
  if (jb.conn == 4) run_job<SmemMode, 4>(k, jb, smem);
  else run_job<SmemMode, 8>(k, jb, smem);
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
uint32_t* g_noalloc_ptr[kMaxDevices] = {};  // device address of the array, per device
size_t g_noalloc_smem[kMaxDevices] = {};    // opt-in shared memory per block, per device
}  // namespace

}  // namespace hasf

extern "C" int hasf_smooth_noalloc(const hasf_image* img, int* status, void* stream) {
  using namespace hasf;
  if (!img || !img->in || !img->out) return HASF_EINVAL;
  const int w = img->width, h = img->height;
  if (w < 1 || w > 65536 || h < 1 || h > 65536 || img->pitch < w || img->rmax < 1 ||
      img->rmax > kMaxR || (img->connectivity != 8 && img->connectivity != 4) ||
      img->reserved != 0)
    return HASF_EINVAL;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HASF_ECUDA;
  uint32_t* base = nullptr;
  size_t smem_limit = 0;
  {
    // Set-up, once per device, with that device current: the level table and
    // the device address of the scratch array (its name is only a host-side
    // stand-in in host code).
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
      e = upload_level_table();
      if (e != cudaSuccess) return HASF_ECUDA;
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) return HASF_ECUDA;
      int v = 0;
      e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
      if (e != cudaSuccess) return HASF_ECUDA;
      e = cudaFuncSetAttribute(hasf_single_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               v - 1024);
      if (e == cudaSuccess) e = reg_one_prepare();
      if (e != cudaSuccess) return HASF_ECUDA;
      g_noalloc_smem[dev] = (size_t)v - 1024;
      g_noalloc_ptr[dev] = (uint32_t*)p;
    }
    base = g_noalloc_ptr[dev];
    smem_limit = g_noalloc_smem[dev];
  }
  const long long words = (long long)h * words_per_row(w);
  const bool reg = reg_kernel_ok(w, h, img->rmax);
  const size_t smem = reg ? reg_kernel_smem(w, h) : resident_smem_bytes(w, h);
  if (words > kStaticPlaneWords || smem > smem_limit) return HASF_EBUDGET;

  Job jb{};
  jb.in = img->in;
  jb.out = img->out;
  jb.C = img->C;
  jb.D = img->D;
  jb.g0 = base;
  jb.cp = img->C ? base + kStaticPlaneWords : nullptr;
  jb.dp = img->D ? base + 2 * kStaticPlaneWords : nullptr;
  jb.status = status ? status : (int*)(base + 3 * kStaticPlaneWords);
  jb.w = w;
  jb.h = h;
  jb.pitch = img->pitch;
  jb.wpr = words_per_row(w);
  jb.r_lo = 1;
  jb.r_hi = img->rmax;
  jb.op = OP_HASF;
  jb.conn = img->connectivity;
  jb.gang = 1;
  jb.cap = (int)(words * 32 + 2 < 0x7FFFFFFF ? words * 32 + 2 : 0x7FFFFFFF);
  jb.plane_words = plane_words(w, h);
  cudaStream_t s = (cudaStream_t)stream;
  // The status word must start at zero; the planes are fully written by the
  // kernel before they are read.
  e = cudaMemsetAsync(jb.status, 0, sizeof(int), s);
  if (e != cudaSuccess) return HASF_ECUDA;
  if (reg) {
    e = launch_reg_one(jb, s);
  } else {
    hasf_single_kernel<<<1, kThreads, smem, s>>>(jb);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? HASF_OK : HASF_ECUDA;
}
