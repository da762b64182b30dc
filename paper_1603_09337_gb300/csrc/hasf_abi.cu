// hasf_abi.cu -- host runtime behind the C ABI declared in include/hasf.h.
//
// A context owns: a device scratch arena for the synchronous entry points
// (job descriptors, per-job bit planes), pinned staging for the host-buffer
// entry point, and the continuous-batching server (a worker thread that
// admits submitted jobs against the byte budget and launches them in batches
// on a small pool of streams, so that batches overlap on the device).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <climits>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <cstdio>
#include <deque>
#include <map>
#include <mutex>
#include <tuple>
#include <thread>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include <cuda_runtime.h>

#include "hasf.h"
#include "hasf_internal.h"

using namespace hasf;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

// Public status of a device status word.
int public_status(int dev) {
  switch (dev) {
    case DEV_OK: return HASF_OK;
    case DEV_UNSTABLE: return HASF_EUNSTABLE;
    case DEV_TIMEOUT: return HASF_ETIMEOUT;
    default: return HASF_ECUDA;
  }
}

int validate(const hasf_image* im) {
  if (!im || !im->in || !im->out) return HASF_EINVAL;
  if (im->width < 1 || im->width > 65536 || im->height < 1 || im->height > 65536)
    return HASF_EINVAL;
  if (im->pitch < im->width) return HASF_EINVAL;
  if (im->rmax == 0 || im->rmax > kMaxR || im->rmax < -kMaxR) return HASF_EINVAL;
  if (im->connectivity != 8 && im->connectivity != 4) return HASF_EINVAL;
  if (im->reserved != 0) return HASF_EINVAL;
  return HASF_OK;
}

// Launch plan of a set of jobs: descriptors, resident order, gang CTA map and
// the byte layout of the scratch they need.
struct Plan {
  std::vector<Job> jobs;
  std::vector<int> order;       // resident jobs (generic kernel), largest work first
  std::vector<int> reg_order;   // resident jobs (register kernel): by sweep schedule
                                // (4, 2, 1 rows per group), then largest work first
  int reg_split[3] = {0, 0, 0}; // jobs of each schedule, in that order
  size_t reg_smem = 0;          // dynamic shared memory of the register launch
  std::map<int, std::vector<int>> tile_groups;  // tiles per image -> cluster jobs
  std::vector<int2> tctamap;    // tiled gang CTAs (job, tile)
  std::vector<int> gang_jobs;   // gang jobs
  std::vector<int2> ctamap;     // gang CTAs (job, part)
  size_t smem = 0;              // dynamic shared memory of the resident launch
  size_t bytes = 0;             // scratch bytes
  // offsets inside the scratch block
  size_t off_jobs = 0, off_order = 0, off_ctamap = 0, off_counter = 0, off_sync = 0,
         off_status = 0;
  size_t sync_bytes = 0;
};

struct Options {
  int force_gang = 0;
  int no_tiles = 0;
  int tile_force = 0;   // 2: send every tiled image to the tiled gang
  int gang_ctas = 0;
  long long round_cap = 0;
  int serve_streams = 8;
  int serve_batch = 512;
  int stats = 0;
  int generic_only = 0;
  int host_mapped = 2;  // hasf_smooth_host: 2 direct access, 1 copy kernel, 0 staged copies
  int wait_deadline_ms = 0;  // gang barrier wait limit, 0 = 4000 ms
  int fault_gang_skip = 0;   // fault injection: CTA 0 of a gang leaves before its first barrier
  int row_group = 0;         // register kernel's rows per sweep group: 0 = tuned / 4, or 1, 2, 4
  int simple3_table = 1;     // 3D simple-voxel test by the 8 MB table (1) or by flood fill (0)
};

// The server's launch resources, one per concurrent batch, made once and
// reused: a stream, a completion event, completion words in pinned
// device-mapped host memory (one per job of a batch), and device scratch that
// grows to the largest batch the slot has run.
struct ServeSlot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  int* h_status = nullptr;  // pinned and mapped, one per job: 0 running, 1 + status done
  int* d_notify = nullptr;  // device address of h_status
  int status_cap = 0;
  void* mem = nullptr;
  size_t cap = 0;
};

struct Batch {  // one server launch in flight
  ServeSlot slot;
  size_t bytes = 0;
  std::vector<uint64_t> tickets;
  std::vector<char> reported;
};

struct Pending {
  uint64_t ticket;
  hasf_image img;
  size_t bytes;
};

}  // namespace

struct hasf_ctx {
  int device = 0;
  size_t budget = 0;
  int num_sms = 0;
  size_t max_smem = 0;
  int gang_max = 0;
  int tile_gang_max = 0;
  std::vector<cudaStream_t> lanes;  // streams for the independent launches of a plan
  int tile_cluster_ok[17] = {0};  // clusters of n tiles can run (1) or not (0)
  Options opt;

  void* arena = nullptr;
  uint32_t* simple3_lut = nullptr;  // the 3D simple-voxel table, built at the first volume call
  size_t arena_bytes = 0;
  int* d_status = nullptr;
  unsigned long long* d_stats = nullptr;  // STAT_COUNT counters
  unsigned long long launches = 0;        // kernel launches issued (host count)
  int max3d = 1;                          // co-resident CTAs of the 3D kernel
  bool pageable_access = false;           // kernels may read and write any host memory (ATS)

  void* pinned = nullptr;
  size_t pinned_bytes = 0;
  void* io = nullptr;
  size_t io_bytes = 0;
  cudaStream_t host_stream = nullptr;

  std::mutex mu;
  std::condition_variable cv;
  std::deque<Pending> pending;
  std::vector<Batch> inflight;
  std::vector<ServeSlot> free_slots;
  size_t serve_retained = 0;  // device scratch held by the slots
  std::unordered_map<uint64_t, int> finished;
  std::unordered_set<uint64_t> launched;
  std::unordered_set<uint64_t> queued;
  uint64_t next_ticket = 1;
  size_t inflight_bytes = 0;
  bool stop = false;
  std::thread worker;
  bool worker_running = false;

  // fault injection: the n-th device or pinned-host allocation from now fails
  // (0 = off); counted down by every allocation of the context
  std::atomic<long long> fault_alloc{0};

  // autotuner: size bucket -> CTAs per image (0 = one-CTA generic kernel)
  std::map<std::tuple<int, int, int>, int> tune;
  // autotuner: size bucket of the register kernel -> rows per sweep group
  std::map<std::tuple<int, int, int>, int> tune_group;
  std::mutex tune_mu;  // guards tune_group (read by plans built under ctx->mu and without it)
};

struct hasf_graph {
  hasf_ctx* ctx = nullptr;
  void* mem = nullptr;
  size_t bytes = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HASF_OK;
  if (e == cudaErrorMemoryAllocation) return HASF_ENOMEM;
  return HASF_ECUDA;
}

// Whether the allocation about to be made is the injected failure.
bool alloc_fault(hasf_ctx* ctx) {
  long long n = ctx->fault_alloc.load();
  while (n > 0 && !ctx->fault_alloc.compare_exchange_weak(n, n - 1)) {
  }
  return n == 1;
}

// cudaMalloc / cudaMallocAsync / cudaHostAlloc of the context, through the
// allocation fault injection.
cudaError_t ctx_malloc(hasf_ctx* ctx, void** p, size_t bytes) {
  if (alloc_fault(ctx)) return cudaErrorMemoryAllocation;
  return cudaMalloc(p, bytes);
}
cudaError_t ctx_malloc_async(hasf_ctx* ctx, void** p, size_t bytes, cudaStream_t s) {
  if (alloc_fault(ctx)) return cudaErrorMemoryAllocation;
  return cudaMallocAsync(p, bytes, s);
}
cudaError_t ctx_host_alloc(hasf_ctx* ctx, void** p, size_t bytes, unsigned flags) {
  if (alloc_fault(ctx)) return cudaErrorMemoryAllocation;
  return cudaHostAlloc(p, bytes, flags);
}

int ceil_log2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}
std::tuple<int, int, int> tune_key(const hasf_image& im) {
  return std::make_tuple(ceil_log2(im.width), ceil_log2(im.height), im.rmax);
}

// Rows per sweep group of a register-kernel image: forced by the option, else
// the autotuner's choice for its size bucket, else 4.
int reg_group(hasf_ctx* ctx, const hasf_image& im) {
  if (ctx->opt.row_group) return ctx->opt.row_group;
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  auto it = ctx->tune_group.find(tune_key(im));
  return it != ctx->tune_group.end() ? it->second : 4;
}
int group_slot(int g) { return g == 4 ? 0 : (g == 2 ? 1 : 2); }

bool fits_resident(const hasf_ctx* ctx, const hasf_image& im) {
  // keep 1 KB of the per-block limit for the kernel's static shared memory
  return resident_smem_bytes(im.width, im.height) + 1024 <= ctx->max_smem;
}

// Path of an image that the register kernel does not take: 1 = tile
// cluster, 2 = tiled gang, 0 = the generic kernels.
int tile_path(const hasf_ctx* ctx, const hasf_image& im) {
  if (ctx->opt.force_gang || ctx->opt.generic_only || ctx->opt.no_tiles) return 0;
  if (im.rmax < 0) return 0;  // run to stability: the generic kernels
  if (im.rmax > kTileMaxR) return 0;
  auto it = ctx->tune.find(tune_key(im));
  if (it != ctx->tune.end() && it->second >= 0) return 0;  // tuned to a generic shape
  const int nt = tile_count(im.width, im.height);
  if (ctx->opt.tile_force == 2) return nt <= ctx->tile_gang_max ? 2 : 0;
  if (nt <= 16 && ctx->tile_cluster_ok[nt]) return 1;
  if (nt <= ctx->tile_gang_max) return 2;
  return 0;
}

bool wants_gang(const hasf_ctx* ctx, const hasf_image& im) {
  if (ctx->opt.force_gang) return true;
  if (!fits_resident(ctx, im)) return true;
  auto it = ctx->tune.find(tune_key(im));
  return it != ctx->tune.end() && it->second > 0 && !reg_kernel_ok(im.width, im.height, im.rmax);
}
bool uses_reg(const hasf_ctx* ctx, const hasf_image& im) {
  // a run to stability (rmax < 0) takes the register kernel when its cap fits
  return !ctx->opt.force_gang && !ctx->opt.generic_only &&
         reg_kernel_ok(im.width, im.height, im.rmax < 0 ? -im.rmax : im.rmax);
}

int gang_size(const hasf_ctx* ctx, const hasf_image& im) {
  if (ctx->opt.gang_ctas > 0) return std::min(ctx->opt.gang_ctas, ctx->gang_max);
  auto it = ctx->tune.find(tune_key(im));
  if (it != ctx->tune.end() && it->second > 0) return std::min(it->second, ctx->gang_max);
  const long long words = (long long)im.height * words_per_row(im.width);
  long long g = (words + 4095) / 4096;  // about 8 words per thread and pass
  g = std::max(1LL, std::min(g, (long long)ctx->gang_max));
  return (int)g;
}

// Size (base == nullptr) or fill (base != nullptr) the plan of n images.
// Returns the scratch bytes.
size_t build_plan(hasf_ctx* ctx, const hasf_image* imgs, int n, int op, Plan& p, char* base,
                  int* status_ptr, int* notify = nullptr) {
  p.jobs.assign(n, Job{});
  p.order.clear();
  p.reg_order.clear();
  p.reg_split[0] = p.reg_split[1] = p.reg_split[2] = 0;
  std::vector<int> reg_by_group[3];
  p.reg_smem = 0;
  p.tile_groups.clear();
  p.tctamap.clear();
  p.gang_jobs.clear();
  p.ctamap.clear();
  p.smem = 0;
  size_t off = 0;
  p.off_jobs = off;
  off = align_up(off + sizeof(Job) * (size_t)n);
  p.off_order = off;
  off = align_up(off + sizeof(int) * (size_t)n);
  // path of each image: 3 register kernel, 1 tile cluster, 2 tiled gang,
  // 4 generic gang, 0 generic one-CTA
  int gang_ctas = 0;
  std::vector<char> path(n, 0);
  for (int i = 0; i < n; ++i) {
    if (uses_reg(ctx, imgs[i])) {
      path[i] = 3;
    } else if (int tp = tile_path(ctx, imgs[i])) {
      path[i] = (char)tp;
      if (tp == 2) gang_ctas += tile_count(imgs[i].width, imgs[i].height);
    } else if (wants_gang(ctx, imgs[i])) {
      path[i] = 4;
      gang_ctas += gang_size(ctx, imgs[i]);
    }
  }
  p.off_ctamap = off;
  off = align_up(off + sizeof(int2) * (size_t)std::max(gang_ctas, 1));
  p.off_counter = off;
  off = align_up(off + 16);
  p.off_sync = off;
  p.sync_bytes = sizeof(unsigned) * 8 * (size_t)n;
  off = align_up(off + p.sync_bytes);
  p.off_status = off;
  off = align_up(off + sizeof(int) * (size_t)n);
  for (int i = 0; i < n; ++i) {
    const hasf_image& im = imgs[i];
    Job& j = p.jobs[i];
    j.in = im.in;
    j.out = im.out;
    j.C = im.C;
    j.D = (op == OP_HASF || op == OP_HF) ? im.D : nullptr;
    j.w = im.width;
    j.h = im.height;
    j.pitch = im.pitch;
    j.wpr = words_per_row(im.width);
    j.stable = (op == OP_HASF && im.rmax < 0) ? 1 : 0;
    j.r_lo = (op == OP_HASF) ? 1 : im.rmax;
    j.r_hi = im.rmax < 0 ? -im.rmax : im.rmax;
    j.op = op;
    j.conn = im.connectivity;
    j.plane_words = plane_words(im.width, im.height);
    const long long px = (long long)im.width * im.height;
    j.cap = ctx->opt.round_cap > 0 ? (int)std::min<long long>(ctx->opt.round_cap, INT_MAX)
                                   : (int)std::min<long long>(px + 2, INT_MAX);
    j.deadline_ms = ctx->opt.wait_deadline_ms;
    j.fault_skip = ctx->opt.fault_gang_skip;
    const size_t gwords = (size_t)im.height * j.wpr;
    j.g0 = base ? (uint32_t*)(base + off) : nullptr;
    off += align_up(gwords * 4);
    if (j.stable) {
      j.g1 = base ? (uint32_t*)(base + off) : nullptr;
      off += align_up(gwords * 4);
    }
    const bool need_c = (op == OP_THICK) || im.C != nullptr;
    if (need_c) {
      j.cp = base ? (uint32_t*)(base + off) : nullptr;
      off += align_up(gwords * 4);
    }
    if (j.D) {
      j.dp = base ? (uint32_t*)(base + off) : nullptr;
      off += align_up(gwords * 4);
    }
    if (path[i] == 4) {
      j.gang = gang_size(ctx, im);
      j.planes = base ? (uint32_t*)(base + off) : nullptr;
      off += align_up(state_bytes(im.width, im.height));
      j.sync = base ? (unsigned*)(base + p.off_sync) + 8 * i : nullptr;
      p.gang_jobs.push_back(i);
    } else if (path[i] == 3) {
      j.gang = 1;
      reg_by_group[group_slot(reg_group(ctx, im))].push_back(i);
      p.reg_smem = std::max(p.reg_smem, reg_kernel_smem(im.width, im.height));
    } else if (path[i] == 1) {
      j.gang = tile_count(im.width, im.height);
      p.tile_groups[j.gang].push_back(i);
    } else if (path[i] == 2) {
      j.gang = tile_count(im.width, im.height);
      j.planes = base ? (uint32_t*)(base + off) : nullptr;
      off += align_up(tile_gang_words(im.width, im.height) * 4);
      j.sync = base ? (unsigned*)(base + p.off_sync) + 8 * i : nullptr;
      for (int t = 0; t < j.gang; ++t) p.tctamap.push_back(make_int2(i, t));
    } else {
      j.gang = 1;
      p.order.push_back(i);
      p.smem = std::max(p.smem, resident_smem_bytes(im.width, im.height));
    }
    j.status = status_ptr ? status_ptr
                          : (base ? (int*)(base + p.off_status) + i : nullptr);
    j.stats = ctx->opt.stats ? ctx->d_stats : nullptr;
    j.sync = base ? (unsigned*)(base + p.off_sync) + 8 * i : nullptr;
    j.notify = notify ? notify + i : nullptr;
  }
  // Largest work first (the paper's scheduler bound: a worker never holds
  // more than its share of the largest tasks).
  auto by_work = [&](int a, int b) {
    const long long wa = (long long)imgs[a].width * imgs[a].height * std::abs(imgs[a].rmax);
    const long long wb = (long long)imgs[b].width * imgs[b].height * std::abs(imgs[b].rmax);
    return wa > wb;
  };
  std::stable_sort(p.order.begin(), p.order.end(), by_work);
  for (int gi = 0; gi < 3; ++gi) {
    std::stable_sort(reg_by_group[gi].begin(), reg_by_group[gi].end(), by_work);
    p.reg_order.insert(p.reg_order.end(), reg_by_group[gi].begin(), reg_by_group[gi].end());
    p.reg_split[gi] = (int)reg_by_group[gi].size();
  }
  for (auto& kv : p.tile_groups) std::stable_sort(kv.second.begin(), kv.second.end(), by_work);
  for (int gi : p.gang_jobs)
    for (int part = 0; part < p.jobs[gi].gang; ++part) p.ctamap.push_back(make_int2(gi, part));
  p.bytes = off;
  return off;
}

// Upload the plan's descriptors and launch it on `s`.  `base` is the scratch.
// Upload the plan's descriptors and launch it on `s`.  When the plan has
// several independent launches (kernel kinds, cluster sizes, gang chunks) and
// `fork` is set, they are issued on the context's lane streams after an event
// on `s`, and `s` waits for all of them: they overlap on the device.
int launch_plan(hasf_ctx* ctx, Plan& p, char* base, cudaStream_t s, bool upload = true,
                bool fork = true) {
  const int n = (int)p.jobs.size();
  cudaError_t e = cudaSuccess;
  if (upload) {
    std::vector<char> head(
        p.off_ctamap + sizeof(int2) * std::max<size_t>(p.ctamap.size() + p.tctamap.size(), 1), 0);
    std::memcpy(head.data() + p.off_jobs, p.jobs.data(), sizeof(Job) * n);
    if (!p.order.empty())
      std::memcpy(head.data() + p.off_order, p.order.data(), sizeof(int) * p.order.size());
    if (!p.reg_order.empty())
      std::memcpy(head.data() + p.off_order + sizeof(int) * p.order.size(), p.reg_order.data(),
                  sizeof(int) * p.reg_order.size());
    size_t at_o = p.order.size() + p.reg_order.size();
    for (const auto& kv : p.tile_groups) {
      std::memcpy(head.data() + p.off_order + sizeof(int) * at_o, kv.second.data(),
                  sizeof(int) * kv.second.size());
      at_o += kv.second.size();
    }
    if (!p.ctamap.empty())
      std::memcpy(head.data() + p.off_ctamap, p.ctamap.data(), sizeof(int2) * p.ctamap.size());
    if (!p.tctamap.empty())
      std::memcpy(head.data() + p.off_ctamap + sizeof(int2) * p.ctamap.size(), p.tctamap.data(),
                  sizeof(int2) * p.tctamap.size());
    e = cudaMemcpyAsync(base, head.data(), head.size(), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(base + p.off_counter, 0, 16, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + p.off_sync, 0, p.sync_bytes, s);
  if (e != cudaSuccess) return cuda_status(e);
  const Job* d_jobs = (const Job*)(base + p.off_jobs);
  const int groups = (p.reg_split[0] > 0) + (p.reg_split[1] > 0) + (p.reg_split[2] > 0) +
                     (p.order.empty() ? 0 : 1) +
                     (int)p.tile_groups.size() + (p.tctamap.empty() ? 0 : 1) +
                     (p.ctamap.empty() ? 0 : 1);
  const int nl = (fork && groups > 1) ? std::min<int>(groups, (int)ctx->lanes.size()) : 0;
  // A plan whose CTAs all fit one per SM runs its tiled kernels one CTA per
  // SM (the instance with twice the registers).
  long long plan_ctas = (long long)p.reg_order.size() + (long long)p.order.size() +
                        (long long)p.tctamap.size() + (long long)p.ctamap.size();
  for (const auto& kv : p.tile_groups) plan_ctas += (long long)kv.first * kv.second.size();
  const bool alone = plan_ctas <= ctx->num_sms;
  cudaEvent_t ev_fork = nullptr;
  if (nl > 0) {
    e = cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev_fork, s);
    for (int l = 0; e == cudaSuccess && l < nl; ++l) e = cudaStreamWaitEvent(ctx->lanes[l], ev_fork, 0);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int next_lane = 0;
  auto lane = [&]() -> cudaStream_t { return nl > 0 ? ctx->lanes[(next_lane++) % nl] : s; };
  auto join = [&]() -> int {
    if (nl == 0) return HASF_OK;
    cudaError_t ej = cudaSuccess;
    for (int l = 0; ej == cudaSuccess && l < nl; ++l) {
      cudaEvent_t ev;
      ej = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (ej != cudaSuccess) break;
      ej = cudaEventRecord(ev, ctx->lanes[l]);
      if (ej == cudaSuccess) ej = cudaStreamWaitEvent(s, ev, 0);
      cudaEventDestroy(ev);
    }
    cudaEventDestroy(ev_fork);
    return cuda_status(ej);
  };
  // Tile clusters: one launch per cluster size, the largest images first
  // (they run longest; launched first, they do not form the tail).
  {
    std::vector<std::pair<int, size_t>> at_of;   // (cluster size, first order slot)
    size_t at_o = p.order.size() + p.reg_order.size();
    for (const auto& kv : p.tile_groups) {
      at_of.push_back({kv.first, at_o});
      at_o += kv.second.size();
    }
    for (auto it = at_of.rbegin(); it != at_of.rend(); ++it) {
      const auto& jobs_of = p.tile_groups.at(it->first);
      e = launch_tile_cluster(d_jobs, (const int*)(base + p.off_order) + it->second,
                              (int)jobs_of.size(), it->first, alone, lane());
      if (e != cudaSuccess) return cuda_status(e);
      ++ctx->launches;
    }
  }
  // Tiled gangs: as many whole images as fit co-resident per cooperative launch
  // (the chunks of one kind run one after the other on one stream).
  if (!p.tctamap.empty()) {
    const cudaStream_t ls = lane();
    const int2* d_tmap = (const int2*)(base + p.off_ctamap) + p.ctamap.size();
    size_t at = 0;
    while (at < p.tctamap.size()) {
      size_t end = at;
      while (end < p.tctamap.size()) {
        const int gsz = p.jobs[p.tctamap[end].x].gang;
        if (end > at && (int)(end - at) + gsz > ctx->tile_gang_max) break;
        end += gsz;
      }
      e = launch_tile_gang(d_jobs, d_tmap + at, (int)(end - at), alone, ls);
      if (e != cudaSuccess) return cuda_status(e);
      ++ctx->launches;
      at = end;
    }
  }
  // Gang jobs: as many as fit co-resident per cooperative launch.
  size_t at = 0;
  const int2* d_map = (const int2*)(base + p.off_ctamap);
  const cudaStream_t gs = p.ctamap.empty() ? s : lane();
  while (at < p.ctamap.size()) {
    size_t end = at;
    while (end < p.ctamap.size()) {
      const int gsz = p.jobs[p.ctamap[end].x].gang;
      if (end > at && (int)(end - at) + gsz > ctx->gang_max) break;
      end += gsz;
    }
    e = launch_gang(d_jobs, d_map + at, (int)(end - at), gs);
    if (e != cudaSuccess) return cuda_status(e);
    ++ctx->launches;
    at = end;
  }
  for (int gi = 0, at = 0; gi < 3; at += p.reg_split[gi], ++gi) {
    if (!p.reg_split[gi]) continue;
    const int per_sm = std::max(1, reg_ctas_per_sm(p.reg_smem));
    const int grid = std::min<int>(p.reg_split[gi], per_sm * ctx->num_sms);
    e = launch_reg(gi == 0 ? 4 : (gi == 1 ? 2 : 1), d_jobs,
                   (const int*)(base + p.off_order) + p.order.size() + at, p.reg_split[gi], grid,
                   p.reg_smem, (unsigned*)(base + p.off_counter) + 1 + gi, lane());
    if (e != cudaSuccess) return cuda_status(e);
    ++ctx->launches;
  }
  if (!p.order.empty()) {
    const int per_sm = std::max(1, resident_ctas_per_sm(ctx->device, p.smem));
    const int grid = std::min<int>((int)p.order.size(), per_sm * ctx->num_sms);
    e = launch_resident(d_jobs, (const int*)(base + p.off_order), (int)p.order.size(), grid,
                        p.smem, (unsigned*)(base + p.off_counter), lane());
    if (e != cudaSuccess) return cuda_status(e);
    ++ctx->launches;
  }
  return join();
}

int ensure_arena(hasf_ctx* ctx, size_t bytes, cudaStream_t s) {
  if (bytes > ctx->budget) return HASF_EBUDGET;
  if (ctx->arena_bytes >= bytes) return HASF_OK;
  if (ctx->arena) {
    cudaStreamSynchronize(s);
    cudaDeviceSynchronize();
    cudaFree(ctx->arena);
    ctx->arena = nullptr;
    ctx->arena_bytes = 0;
  }
  if (alloc_fault(ctx)) return HASF_ENOMEM;
  size_t want = std::min(ctx->budget, std::max(bytes, bytes + bytes / 4));
  cudaError_t e = cudaMalloc(&ctx->arena, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    e = cudaMalloc(&ctx->arena, bytes);
    want = bytes;
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    ctx->arena = nullptr;
    return HASF_ENOMEM;
  }
  ctx->arena_bytes = want;
  return HASF_OK;
}

// Run n images (device pointers) with operator `op` on stream s, splitting
// into chunks that fit the budget.
int run_images(hasf_ctx* ctx, const hasf_image* imgs, int n, int op, cudaStream_t s) {
  if (n < 0 || (n > 0 && !imgs)) return HASF_EINVAL;
  for (int i = 0; i < n; ++i) {
    int v = validate(&imgs[i]);
    if (v) return v;
    if (op == OP_THICK && !imgs[i].C) return HASF_EINVAL;
  }
  if (n == 0) return HASF_OK;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_status(e);
  Plan p;
  int first = 0;
  while (first < n) {
    // grow the chunk while it fits the budget
    int cnt = n - first;
    size_t need = build_plan(ctx, imgs + first, cnt, op, p, nullptr, nullptr);
    while (need > ctx->budget && cnt > 1) {
      cnt = (cnt + 1) / 2;
      need = build_plan(ctx, imgs + first, cnt, op, p, nullptr, nullptr);
    }
    if (need > ctx->budget) return HASF_EBUDGET;
    int rc = ensure_arena(ctx, need, s);
    if (rc) return rc;
    build_plan(ctx, imgs + first, cnt, op, p, (char*)ctx->arena, ctx->d_status);
    if (cnt == 1 && p.reg_split[0] == 1) {
      // one image of the register kernel's default schedule: its descriptor
      // goes by value in the launch, with no upload and no job counter
      e = launch_reg_one(p.jobs[0], s);
      if (e != cudaSuccess) return cuda_status(e);
      ++ctx->launches;
    } else {
      rc = launch_plan(ctx, p, (char*)ctx->arena, s);
      if (rc) return rc;
    }
    first += cnt;
    if (first < n) {
      // the next chunk reuses the arena: wait for this one
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  return HASF_OK;
}

// ---------------------------------------------------------------------------
// Server.
// ---------------------------------------------------------------------------

size_t serve_job_bytes(hasf_ctx* ctx, const hasf_image& im) {
  Plan p;
  return build_plan(ctx, &im, 1, OP_HASF, p, nullptr, nullptr);
}

void retire_finished(hasf_ctx* ctx) {  // ctx->mu held
  for (size_t i = 0; i < ctx->inflight.size();) {
    Batch& b = ctx->inflight[i];
    // jobs report themselves as they finish (their CTAs write the mapped flags)
    for (size_t k = 0; k < b.tickets.size(); ++k) {
      if (b.reported[k]) continue;
      const int f = *(volatile int*)(b.slot.h_status + k);
      if (f) {
        b.reported[k] = 1;
        const int st = f - 1;
        ctx->finished[b.tickets[k]] = public_status(st);
        ctx->launched.erase(b.tickets[k]);
        ctx->cv.notify_all();
      }
    }
    cudaError_t q = cudaEventQuery(b.slot.done);
    if (q == cudaErrorNotReady) {
      ++i;
      continue;
    }
    for (size_t k = 0; k < b.tickets.size(); ++k) {
      if (b.reported[k]) continue;
      const int f = *(volatile int*)(b.slot.h_status + k);
      ctx->finished[b.tickets[k]] = (q == cudaSuccess && f) ? public_status(f - 1) : HASF_ECUDA;
      ctx->launched.erase(b.tickets[k]);
    }
    if (q != cudaSuccess) cudaGetLastError();
    ctx->free_slots.push_back(b.slot);  // its resources stay for the next batch
    ctx->inflight_bytes -= b.bytes;
    ctx->inflight.erase(ctx->inflight.begin() + i);
    ctx->cv.notify_all();
  }
}

// Admit pending jobs that fit the budget into one batch and launch it.  A
// batch holds jobs of one kind -- images the single-tile kernel takes, or
// larger ones -- taken in arrival order starting from the oldest job, so that
// short jobs never wait in a launch for a long one.
// Give a slot room for a batch of n jobs and `bytes` of scratch.  Scratch
// grows with a quarter of slack while the slots' total stays within the
// budget; idle slots give theirs back when it would not.
int slot_reserve(hasf_ctx* ctx, ServeSlot& sl, int n, size_t bytes) {  // ctx->mu held
  if (sl.status_cap < n) {
    if (sl.h_status) cudaFreeHost(sl.h_status);
    sl.h_status = nullptr;
    sl.d_notify = nullptr;
    sl.status_cap = 0;
    const int want = std::max(n, ctx->opt.serve_batch);
    cudaError_t e = ctx_host_alloc(ctx, (void**)&sl.h_status, sizeof(int) * want,
                                   cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void**)&sl.d_notify, sl.h_status, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (sl.h_status) cudaFreeHost(sl.h_status);
      sl.h_status = nullptr;
      return cuda_status(e);
    }
    sl.status_cap = want;
  }
  if (sl.cap < bytes) {
    if (sl.mem) cudaFreeAsync(sl.mem, sl.stream);
    ctx->serve_retained -= sl.cap;
    sl.mem = nullptr;
    sl.cap = 0;
    size_t want = std::max(bytes, bytes + bytes / 4);
    if (ctx->serve_retained + want > ctx->budget) want = bytes;
    for (ServeSlot& o : ctx->free_slots) {
      if (ctx->serve_retained + want <= ctx->budget) break;
      if (o.mem) {
        cudaFreeAsync(o.mem, o.stream);
        ctx->serve_retained -= o.cap;
        o.mem = nullptr;
        o.cap = 0;
      }
    }
    cudaError_t e = ctx_malloc_async(ctx, &sl.mem, want, sl.stream);
    if (e != cudaSuccess) {
      cudaGetLastError();
      sl.mem = nullptr;
      return cuda_status(e);
    }
    sl.cap = want;
    ctx->serve_retained += want;
  }
  return HASF_OK;
}

// Admit pending jobs that fit the budget into one batch and launch it.  A
// batch holds jobs of one kind -- images the single-tile kernel takes, or
// larger ones -- taken in arrival order starting from the oldest job, so that
// short jobs never wait in a launch for a long one.
bool launch_next(hasf_ctx* ctx) {  // ctx->mu held
  if (ctx->pending.empty() || ctx->free_slots.empty()) return false;
  std::vector<hasf_image> imgs;
  std::vector<uint64_t> tickets;
  size_t bytes = 0;
  const bool small = uses_reg(ctx, ctx->pending.front().img);
  for (auto it = ctx->pending.begin();
       it != ctx->pending.end() && (int)imgs.size() < ctx->opt.serve_batch;) {
    if (uses_reg(ctx, it->img) != small) {
      ++it;
      continue;
    }
    if (ctx->inflight_bytes + bytes + it->bytes + 65536 > ctx->budget) break;
    imgs.push_back(it->img);
    tickets.push_back(it->ticket);
    bytes += it->bytes;
    ctx->queued.erase(it->ticket);
    it = ctx->pending.erase(it);
  }
  if (imgs.empty()) return false;
  Batch b;
  b.slot = ctx->free_slots.back();
  ctx->free_slots.pop_back();
  b.tickets = tickets;
  Plan p;
  const int n = (int)imgs.size();
  b.bytes = build_plan(ctx, imgs.data(), n, OP_HASF, p, nullptr, nullptr);
  b.reported.assign(n, 0);
  int rc = slot_reserve(ctx, b.slot, n, b.bytes);
  if (rc == HASF_OK) {
    // the slot's last batch has finished (its event was seen complete): the
    // words may be cleared on the host
    std::memset(b.slot.h_status, 0, sizeof(int) * n);
    build_plan(ctx, imgs.data(), n, OP_HASF, p, (char*)b.slot.mem, nullptr, b.slot.d_notify);
    cudaError_t e = cudaMemsetAsync((char*)b.slot.mem + p.off_status, 0, sizeof(int) * n,
                                    b.slot.stream);
    rc = cuda_status(e);
    if (rc == HASF_OK) rc = launch_plan(ctx, p, (char*)b.slot.mem, b.slot.stream, true, false);
    if (rc == HASF_OK) rc = cuda_status(cudaEventRecord(b.slot.done, b.slot.stream));
  }
  if (rc != HASF_OK) {
    cudaGetLastError();
    cudaStreamSynchronize(b.slot.stream);
    for (uint64_t t : tickets) ctx->finished[t] = rc;
    ctx->free_slots.push_back(b.slot);
    ctx->cv.notify_all();
    return true;
  }
  for (uint64_t t : tickets) ctx->launched.insert(t);
  ctx->inflight_bytes += b.bytes;
  ctx->inflight.push_back(b);
  return true;
}

void worker_main(hasf_ctx* ctx) {
  cudaSetDevice(ctx->device);
  std::unique_lock<std::mutex> lk(ctx->mu);
  while (!ctx->stop || !ctx->inflight.empty()) {
    retire_finished(ctx);
    bool launched = false;
    if (!ctx->stop)
      while (launch_next(ctx)) launched = true;
    if (launched) continue;
    if (ctx->inflight.empty()) {
      ctx->cv.wait(lk, [&] { return ctx->stop || !ctx->pending.empty(); });
    } else {
      // batches on the device: look again shortly
      lk.unlock();
      std::this_thread::sleep_for(std::chrono::microseconds(20));
      lk.lock();
    }
  }
}

int start_server(hasf_ctx* ctx) {  // ctx->mu held
  if (ctx->worker_running) return HASF_OK;
  for (int i = 0; i < ctx->opt.serve_streams; ++i) {
    ServeSlot sl;
    cudaError_t e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      if (sl.stream) cudaStreamDestroy(sl.stream);
      return cuda_status(e);
    }
    ctx->free_slots.push_back(sl);
  }
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess) {
    uint64_t thr = ctx->budget;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  ctx->stop = false;
  ctx->worker = std::thread(worker_main, ctx);
  ctx->worker_running = true;
  return HASF_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI.
// ---------------------------------------------------------------------------

extern "C" {

int hasf_create(hasf_ctx** out, int device, size_t mem_budget_bytes) {
  if (!out) return HASF_EINVAL;
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return HASF_ECUDA;
  }
  if (device < 0 || device >= ndev) return HASF_EINVAL;
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return cuda_status(e);
  e = upload_level_table();
  if (e == cudaSuccess) e = upload_level_table_3d();
  if (e == cudaSuccess) e = reg_one_prepare();
  if (e != cudaSuccess) return cuda_status(e);
  hasf_ctx* c = new (std::nothrow) hasf_ctx();
  if (!c) return HASF_ENOMEM;
  c->device = device;
  c->budget = mem_budget_bytes ? mem_budget_bytes : (size_t)20 << 30;
  cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device);
  c->max_smem = max_resident_smem(device);
  c->gang_max = std::max(1, max_gang_ctas(device));
  c->tile_gang_max = max_tile_gang_ctas(device);
  c->max3d = std::max(1, max_3d_ctas(device));
  {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrPageableMemoryAccess, device) != cudaSuccess) {
      cudaGetLastError();
      v = 0;
    }
    c->pageable_access = v != 0;
  }
  for (int l = 0; l < 8; ++l) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess) c->lanes.push_back(st);
    else cudaGetLastError();
  }
  for (int t = 1; t <= 16; ++t) c->tile_cluster_ok[t] = tile_clusters_possible(t) > 0 ? 1 : 0;
  e = cudaMalloc(&c->d_status, 16);
  if (e == cudaSuccess) e = cudaMemset(c->d_status, 0, 16);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_stats, sizeof(unsigned long long) * STAT_COUNT);
  if (e == cudaSuccess) e = cudaMemset(c->d_stats, 0, sizeof(unsigned long long) * STAT_COUNT);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->host_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    int rc = cuda_status(e);
    if (c->d_status) cudaFree(c->d_status);
    delete c;
    return rc;
  }
  *out = c;
  return HASF_OK;
}

int hasf_destroy(hasf_ctx* ctx) {
  if (!ctx) return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  {
    std::unique_lock<std::mutex> lk(ctx->mu);
    for (const Pending& pj : ctx->pending) ctx->finished[pj.ticket] = HASF_ECANCELLED;
    ctx->pending.clear();
    ctx->queued.clear();
    ctx->stop = true;
    ctx->cv.notify_all();
  }
  if (ctx->worker_running) ctx->worker.join();
  for (ServeSlot& sl : ctx->free_slots) {
    cudaStreamSynchronize(sl.stream);
    if (sl.mem) cudaFreeAsync(sl.mem, sl.stream);
    cudaStreamSynchronize(sl.stream);
    if (sl.h_status) cudaFreeHost(sl.h_status);
    cudaEventDestroy(sl.done);
    cudaStreamDestroy(sl.stream);
  }
  ctx->free_slots.clear();
  for (cudaStream_t st : ctx->lanes) cudaStreamDestroy(st);
  cudaDeviceSynchronize();
  if (ctx->arena) cudaFree(ctx->arena);
  if (ctx->simple3_lut) cudaFree(ctx->simple3_lut);
  if (ctx->io) cudaFree(ctx->io);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_stats) cudaFree(ctx->d_stats);
  if (ctx->host_stream) cudaStreamDestroy(ctx->host_stream);
  delete ctx;
  return HASF_OK;
}

int hasf_set_option(hasf_ctx* ctx, int option, int64_t value) {
  if (!ctx) return HASF_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  switch (option) {
    case HASF_OPT_FORCE_GANG:
      if (value != 0 && value != 1) return HASF_EINVAL;
      ctx->opt.force_gang = (int)value;
      return HASF_OK;
    case HASF_OPT_GANG_CTAS:
      if (value < 0 || value > 1 << 20) return HASF_EINVAL;
      ctx->opt.gang_ctas = (int)value;
      return HASF_OK;
    case HASF_OPT_ROUND_CAP:
      if (value < 0) return HASF_EINVAL;
      ctx->opt.round_cap = value;
      return HASF_OK;
    case HASF_OPT_SERVE_STREAMS:
      if (value < 1 || value > 16 || ctx->worker_running) return HASF_EINVAL;
      ctx->opt.serve_streams = (int)value;
      return HASF_OK;
    case HASF_OPT_SERVE_BATCH:
      if (value < 1 || value > 4096) return HASF_EINVAL;
      ctx->opt.serve_batch = (int)value;
      return HASF_OK;
    case HASF_OPT_STATS:
      if (value != 0 && value != 1) return HASF_EINVAL;
      ctx->opt.stats = (int)value;
      return HASF_OK;
    case HASF_OPT_GENERIC_ONLY:
      if (value != 0 && value != 1) return HASF_EINVAL;
      ctx->opt.generic_only = (int)value;
      return HASF_OK;
    case HASF_OPT_TILES:
      if (value < 0 || value > 2) return HASF_EINVAL;
      ctx->opt.no_tiles = value == 0;
      ctx->opt.tile_force = (int)value == 2 ? 2 : 0;
      return HASF_OK;
    case HASF_OPT_HOST_MAPPED:
      if (value < 0 || value > 2) return HASF_EINVAL;
      ctx->opt.host_mapped = (int)value;
      return HASF_OK;
    case HASF_OPT_WAIT_DEADLINE_MS:
      if (value < 0 || value > 60000) return HASF_EINVAL;
      ctx->opt.wait_deadline_ms = (int)value;
      return HASF_OK;
    case HASF_OPT_FAULT_GANG_SKIP:
      if (value != 0 && value != 1) return HASF_EINVAL;
      ctx->opt.fault_gang_skip = (int)value;
      return HASF_OK;
    case HASF_OPT_FAULT_ALLOC:
      if (value < 0) return HASF_EINVAL;
      ctx->fault_alloc.store(value);
      return HASF_OK;
    case HASF_OPT_ROW_GROUP:
      if (value != 0 && value != 1 && value != 2 && value != 4) return HASF_EINVAL;
      ctx->opt.row_group = (int)value;
      return HASF_OK;
    case HASF_OPT_SIMPLE3_TABLE:
      if (value != 0 && value != 1) return HASF_EINVAL;
      ctx->opt.simple3_table = (int)value;
      return HASF_OK;
    default:
      return HASF_EINVAL;
  }
}

int hasf_smooth(hasf_ctx* ctx, const hasf_image* img, void* stream) {
  if (!ctx || !img) return HASF_EINVAL;
  return run_images(ctx, img, 1, OP_HASF, (cudaStream_t)stream);
}

int hasf_smooth_batch(hasf_ctx* ctx, const hasf_image* imgs, int n, void* stream) {
  if (!ctx) return HASF_EINVAL;
  return run_images(ctx, imgs, n, OP_HASF, (cudaStream_t)stream);
}

// ---- 3D -------------------------------------------------------------------

namespace {

int validate3d(const hasf_volume* v) {
  if (!v || !v->in || !v->out) return HASF_EINVAL;
  if (v->width < 1 || v->height < 1 || v->depth < 1 || v->width > 4096 || v->height > 4096 ||
      v->depth > 4096)
    return HASF_EINVAL;
  if ((long long)v->width * v->height * v->depth > (1LL << 31)) return HASF_EINVAL;
  if (v->rmax < 1 || v->rmax > kMaxR3D) return HASF_EINVAL;
  if (v->reserved[0] != 0 || v->reserved[1] != 0) return HASF_EINVAL;
  return HASF_OK;
}

// Scratch of one volume: seven planes (S, F, cand, M, g0, C, D).
size_t volume_bytes(const hasf_volume& v) {
  const size_t nw = (size_t)v.depth * v.height * words_per_row(v.width);
  return 7 * align_up(nw * 4);
}

// CTAs of one volume's gang: about 4 words per thread and pass, but no more
// than the batch's share of the co-resident CTAs, so that the whole batch runs
// in one launch (the gang barrier, not the words, bounds a sweep's time).
int volume_gang(const hasf_ctx* ctx, const hasf_volume& v, int nvols) {
  const long long nw = (long long)v.depth * v.height * words_per_row(v.width);
  long long g = (nw + 2047) / 2048;
  const int share = std::max(1, ctx->max3d / std::max(1, nvols));
  return (int)std::max(1LL, std::min(g, (long long)std::min({share, ctx->max3d, 64})));
}

}  // namespace

namespace {
// The 3D simple-voxel table, once per context: built on stream s and waited
// for, so that later calls on any stream find it complete.
int ensure_simple3_table(hasf_ctx* ctx, cudaStream_t s) {
  if (ctx->simple3_lut) return HASF_OK;
  void* p = nullptr;
  cudaError_t e = ctx_malloc(ctx, &p, kSimple3TableWords * 4);
  if (e != cudaSuccess) return cuda_status(e);
  e = build_simple3_table((uint32_t*)p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    cudaFree(p);
    return cuda_status(e);
  }
  ctx->simple3_lut = (uint32_t*)p;
  return HASF_OK;
}
}  // namespace

int hasf_simple3_table(hasf_ctx* ctx, uint32_t* out, void* stream) {
  if (!ctx || !out) return HASF_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_status(e);
  int rc = ensure_simple3_table(ctx, s);
  if (rc) return rc;
  e = cudaMemcpyAsync(out, ctx->simple3_lut, kSimple3TableWords * 4, cudaMemcpyDeviceToDevice, s);
  return e == cudaSuccess ? HASF_OK : cuda_status(e);
}

int hasf_smooth3d(hasf_ctx* ctx, const hasf_volume* vols, int n, void* stream) {
  if (!ctx || n < 0 || (n > 0 && !vols)) return HASF_EINVAL;
  for (int i = 0; i < n; ++i)
    if (int v = validate3d(&vols[i])) return v;
  if (n == 0) return HASF_OK;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_status(e);
  if (ctx->opt.simple3_table) {
    int rc = ensure_simple3_table(ctx, s);
    if (rc) return rc;
  }
  const uint32_t* lut = ctx->opt.simple3_table ? ctx->simple3_lut : nullptr;
  int first = 0;
  while (first < n) {
    // a chunk: co-resident gangs within the budget
    int cnt = 0, ctas = 0;
    size_t bytes = 0;
    while (first + cnt < n) {
      const hasf_volume& v = vols[first + cnt];
      const int g = volume_gang(ctx, v, n);
      const size_t b = volume_bytes(v);
      if (cnt > 0 && (ctas + g > ctx->max3d || bytes + b > ctx->budget / 2)) break;
      ctas += g;
      bytes += b;
      ++cnt;
    }
    const size_t head = align_up(sizeof(Job3) * cnt) + align_up(sizeof(int2) * ctas) +
                        align_up(sizeof(unsigned) * 8 * cnt);
    if (head + bytes > ctx->budget) return HASF_EBUDGET;
    int rc = ensure_arena(ctx, head + bytes, s);
    if (rc) return rc;
    char* base = (char*)ctx->arena;
    std::vector<Job3> jobs(cnt);
    std::vector<int2> map;
    size_t off = head;
    unsigned* d_sync = (unsigned*)(base + align_up(sizeof(Job3) * cnt) + align_up(sizeof(int2) * ctas));
    for (int k = 0; k < cnt; ++k) {
      const hasf_volume& v = vols[first + k];
      Job3& j = jobs[k];
      j = Job3{};
      j.in = v.in;
      j.out = v.out;
      j.C = v.C;
      j.D = v.D;
      j.w = v.width;
      j.h = v.height;
      j.d = v.depth;
      j.wpr = words_per_row(v.width);
      j.rmax = v.rmax;
      j.gang = volume_gang(ctx, v, n);
      const long long vox = (long long)v.width * v.height * v.depth;
      j.cap = ctx->opt.round_cap > 0 ? ctx->opt.round_cap : (int)std::min<long long>(vox + 2, INT_MAX);
      j.deadline_ms = ctx->opt.wait_deadline_ms;
      j.fault_skip = ctx->opt.fault_gang_skip;
      const size_t pb = align_up((size_t)v.depth * v.height * j.wpr * 4);
      uint32_t** planes[7] = {&j.S, &j.F, &j.cand, &j.M, &j.g0, &j.cp, &j.dp};
      for (int q = 0; q < 7; ++q) {
        *planes[q] = (uint32_t*)(base + off);
        off += pb;
      }
      if (!v.C) j.cp = nullptr;
      if (!v.D) j.dp = nullptr;
      j.sync = d_sync + 8 * k;
      j.status = ctx->d_status;
      j.stats = ctx->opt.stats ? ctx->d_stats : nullptr;
      j.simple_lut = lut;
      for (int part = 0; part < j.gang; ++part) map.push_back(make_int2(k, part));
    }
    e = cudaMemcpyAsync(base, jobs.data(), sizeof(Job3) * cnt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(base + align_up(sizeof(Job3) * cnt), map.data(), sizeof(int2) * ctas,
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_sync, 0, sizeof(unsigned) * 8 * cnt, s);
    if (e == cudaSuccess)
      e = launch_3d((const Job3*)base, (const int2*)(base + align_up(sizeof(Job3) * cnt)), ctas,
                    lut != nullptr, s);
    if (e != cudaSuccess) return cuda_status(e);
    ++ctx->launches;
    first += cnt;
    // the host vectors are copied from pageable memory (staged before return);
    // the next chunk reuses the arena: wait for this one
    if (first < n) {
      e = cudaStreamSynchronize(s);
      if (e != cudaSuccess) return cuda_status(e);
    }
  }
  return HASF_OK;
}

int hasf_operator(hasf_ctx* ctx, int op, const hasf_image* img, void* stream) {
  if (!ctx || !img || op < OP_THIN || op > OP_HF || img->rmax < 1) return HASF_EINVAL;
  return run_images(ctx, img, 1, op, (cudaStream_t)stream);
}

int hasf_status_of(hasf_ctx* ctx, void* stream) {
  if (!ctx) return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_status(e);
  int st = 0;
  e = cudaMemcpy(&st, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
  if (e != cudaSuccess) return cuda_status(e);
  return public_status(st);
}

namespace {
bool is_pinned(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// The device address of a page-locked host buffer mapped into the device's
// address space, or null.
void* mapped_ptr(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

// The image with every buffer replaced by its device mapping, if they all
// have one.
bool mapped_image(const hasf_image& im, hasf_image& out) {
  out = im;
  void* in = mapped_ptr(im.in);
  void* o = mapped_ptr(im.out);
  if (!in || !o) return false;
  out.in = (const uint8_t*)in;
  out.out = (uint8_t*)o;
  if (im.C) {
    void* c = mapped_ptr(im.C);
    if (!c) return false;
    out.C = (const uint8_t*)c;
  }
  if (im.D) {
    void* d = mapped_ptr(im.D);
    if (!d) return false;
    out.D = (const uint8_t*)d;
  }
  return true;
}

int smooth_host_staged(hasf_ctx* ctx, const hasf_image* imgs, int n);

// Images whose host buffers are all mapped (maps: the same images with the
// device addresses of those buffers): per chunk, one launch of the library's
// copy kernel gathers every input into device buffers, one batched smoothing
// runs, one copy launch scatters the results back to the callers' buffers.
int smooth_host_mapped(hasf_ctx* ctx, const hasf_image* maps, int n) {
  cudaStream_t s = ctx->host_stream;
  auto dpitch = [](const hasf_image& im) { return ((size_t)im.width + 15) & ~(size_t)15; };
  auto slots = [](const hasf_image& im) { return 2 + (im.C ? 1 : 0) + (im.D ? 1 : 0); };
  auto img_bytes = [&](const hasf_image& im) {
    return align_up(dpitch(im) * im.height) * slots(im);
  };
  const size_t io_cap = std::max<size_t>(ctx->budget / 4, 64ull << 20);
  int first = 0;
  while (first < n) {
    int cnt = 0;
    size_t io = 0;
    while (first + cnt < n && (cnt == 0 || io + img_bytes(maps[first + cnt]) <= io_cap)) {
      io += img_bytes(maps[first + cnt]);
      ++cnt;
    }
    const size_t desc_at = align_up(io);
    const size_t need = desc_at + align_up(sizeof(Copy2D) * 4 * (size_t)cnt);
    if (ctx->io_bytes < need) {
      cudaStreamSynchronize(s);
      if (ctx->io) cudaFree(ctx->io);
      ctx->io = nullptr;
      ctx->io_bytes = 0;
      if (ctx_malloc(ctx, &ctx->io, need) != cudaSuccess) {
        cudaGetLastError();
        return HASF_ENOMEM;
      }
      ctx->io_bytes = need;
    }
    char* dev = (char*)ctx->io;
    std::vector<hasf_image> dimgs(cnt);
    std::vector<Copy2D> copies;   // the gathers, then the scatters
    std::vector<Copy2D> back;
    size_t at = 0;
    for (int i = 0; i < cnt; ++i) {
      const hasf_image& m = maps[first + i];
      const size_t dp = dpitch(m), sb = align_up(dp * m.height);
      hasf_image& di = dimgs[i];
      di = m;
      di.pitch = (int32_t)dp;
      char* base = dev + at;
      di.in = (const uint8_t*)base;
      di.out = (uint8_t*)(base + sb);
      size_t k = 2;
      copies.push_back({m.in, (uint8_t*)base, m.width, m.height, m.pitch, (int)dp});
      if (m.C) {
        di.C = (const uint8_t*)(base + sb * k++);
        copies.push_back({m.C, (uint8_t*)di.C, m.width, m.height, m.pitch, (int)dp});
      }
      if (m.D) {
        di.D = (const uint8_t*)(base + sb * k++);
        copies.push_back({m.D, (uint8_t*)di.D, m.width, m.height, m.pitch, (int)dp});
      }
      back.push_back({di.out, m.out, m.width, m.height, (int)dp, m.pitch});
      at += img_bytes(m);
    }
    const int nin = (int)copies.size();
    copies.insert(copies.end(), back.begin(), back.end());
    Copy2D* d_copies = (Copy2D*)(dev + desc_at);
    cudaError_t e = cudaMemcpyAsync(d_copies, copies.data(), sizeof(Copy2D) * copies.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch_copy2d(d_copies, nin, s);
    if (e != cudaSuccess) return cuda_status(e);
    ctx->launches += (nin + 65534) / 65535;
    int rc = run_images(ctx, dimgs.data(), cnt, OP_HASF, s);
    if (rc) return rc;
    e = launch_copy2d(d_copies + nin, cnt, s);
    if (e != cudaSuccess) return cuda_status(e);
    ctx->launches += (cnt + 65534) / 65535;
    rc = hasf_status_of(ctx, s);   // also: the chunk's buffers are free again
    if (rc) return rc;
    first += cnt;
  }
  return HASF_OK;
}
}  // namespace

int hasf_smooth_host(hasf_ctx* ctx, const hasf_image* imgs, int n) {
  if (!ctx || n < 0 || (n > 0 && !imgs)) return HASF_EINVAL;
  for (int i = 0; i < n; ++i) {
    int v = validate(&imgs[i]);
    if (v) return v;
  }
  if (n == 0) return HASF_OK;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_status(e);
  // Direct access (HASF_OPT_HOST_MAPPED 2) for the images of the register
  // kernel, which reads every input byte once and writes every output byte
  // once: it reads and writes the callers' buffers itself -- any buffer when
  // the device reaches all host memory through the host's page tables, else
  // the page-locked mapped ones (through their device addresses).  The other
  // kernels read their inputs more than once (tile halos, reloads), so their
  // mapped buffers move through the copy kernel (also mode 1 for all mapped
  // buffers), and the rest are staged through the context's pinned buffer
  // with one copy per buffer.
  std::vector<hasf_image> direct, mapped, staged;
  for (int i = 0; i < n; ++i) {
    hasf_image m;
    const bool mp = ctx->opt.host_mapped && mapped_image(imgs[i], m);
    if (ctx->opt.host_mapped == 2 && uses_reg(ctx, imgs[i]) && (ctx->pageable_access || mp))
      direct.push_back(ctx->pageable_access ? imgs[i] : m);
    else if (mp)
      mapped.push_back(m);
    else
      staged.push_back(imgs[i]);
  }
  if (!direct.empty()) {
    int rc = run_images(ctx, direct.data(), (int)direct.size(), OP_HASF, ctx->host_stream);
    if (rc == HASF_OK) rc = hasf_status_of(ctx, ctx->host_stream);
    if (rc) return rc;
  }
  if (!mapped.empty()) {
    int rc = smooth_host_mapped(ctx, mapped.data(), (int)mapped.size());
    if (rc) return rc;
  }
  return staged.empty() ? HASF_OK : smooth_host_staged(ctx, staged.data(), (int)staged.size());
}

namespace {
int smooth_host_staged(hasf_ctx* ctx, const hasf_image* imgs, int n) {
  cudaError_t e = cudaSuccess;
  cudaStream_t s = ctx->host_stream;
  // Device layout of one image: in, out, [C], [D], each w*h bytes, pitch w.
  auto img_bytes = [](const hasf_image& im) {
    const size_t px = (size_t)im.width * im.height;
    return align_up(px) * (2 + (im.C ? 1 : 0) + (im.D ? 1 : 0));
  };
  size_t io_cap = std::max<size_t>(ctx->budget / 4, 64ull << 20);
  int first = 0;
  while (first < n) {
    int cnt = 0;
    size_t io = 0;
    while (first + cnt < n && (cnt == 0 || io + img_bytes(imgs[first + cnt]) <= io_cap)) {
      io += img_bytes(imgs[first + cnt]);
      ++cnt;
    }
    if (ctx->io_bytes < io) {
      cudaStreamSynchronize(s);
      if (ctx->io) cudaFree(ctx->io);
      ctx->io = nullptr;
      ctx->io_bytes = 0;
      e = ctx_malloc(ctx, &ctx->io, io);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return HASF_ENOMEM;
      }
      ctx->io_bytes = io;
    }
    // Stage through pinned memory unless the caller's buffers are pinned.
    std::vector<hasf_image> dimgs(cnt);
    std::vector<size_t> offs(cnt);
    size_t at = 0;
    for (int i = 0; i < cnt; ++i) {
      offs[i] = at;
      at += img_bytes(imgs[first + i]);
    }
    if (ctx->pinned_bytes < io) {
      if (ctx->pinned) cudaFreeHost(ctx->pinned);
      ctx->pinned = nullptr;
      ctx->pinned_bytes = 0;
      e = ctx_host_alloc(ctx, &ctx->pinned, io, 0);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return HASF_ENOMEM;
      }
      ctx->pinned_bytes = io;
    }
    char* pin = (char*)ctx->pinned;
    char* dev = (char*)ctx->io;
    // Pinned caller buffers are copied directly (2D copies honour the pitch);
    // pageable ones are staged through the context's pinned buffer.
    std::vector<char> out_pinned(cnt, 0);
    for (int i = 0; i < cnt; ++i) {
      const hasf_image& im = imgs[first + i];
      const size_t w = im.width, h = im.height, px = w * h, ap = align_up(px);
      char* d = dev + offs[i];
      char* hp = pin + offs[i];
      hasf_image& di = dimgs[i];
      di = im;
      di.pitch = im.width;
      di.in = (const uint8_t*)d;
      di.out = (uint8_t*)(d + ap);
      out_pinned[i] = is_pinned(im.out);
      const uint8_t* srcs[3] = {im.in, im.C, im.D};
      const uint8_t** dsts[3] = {&di.in, &di.C, &di.D};
      size_t slot = 2;
      for (int q = 0; q < 3; ++q) {
        if (!srcs[q]) continue;
        const size_t at_slot = q == 0 ? 0 : slot++;
        char* dd = d + ap * at_slot;
        *dsts[q] = (const uint8_t*)dd;
        if (is_pinned(srcs[q])) {
          e = cudaMemcpy2DAsync(dd, w, srcs[q], (size_t)im.pitch, w, h, cudaMemcpyHostToDevice, s);
        } else {
          char* hs = hp + ap * at_slot;
          for (size_t y = 0; y < h; ++y) std::memcpy(hs + y * w, srcs[q] + y * (size_t)im.pitch, w);
          e = cudaMemcpyAsync(dd, hs, px, cudaMemcpyHostToDevice, s);
        }
        if (e != cudaSuccess) return cuda_status(e);
      }
    }
    int rc = run_images(ctx, dimgs.data(), cnt, OP_HASF, s);
    if (rc) return rc;
    for (int i = 0; i < cnt; ++i) {
      const hasf_image& im = imgs[first + i];
      const size_t w = im.width, h = im.height, px = w * h, ap = align_up(px);
      if (out_pinned[i])
        e = cudaMemcpy2DAsync(im.out, (size_t)im.pitch, dev + offs[i] + ap, w, w, h,
                              cudaMemcpyDeviceToHost, s);
      else
        e = cudaMemcpyAsync(pin + offs[i] + ap, dev + offs[i] + ap, px, cudaMemcpyDeviceToHost, s);
      if (e != cudaSuccess) return cuda_status(e);
    }
    rc = hasf_status_of(ctx, s);
    if (rc) return rc;
    for (int i = 0; i < cnt; ++i) {
      if (out_pinned[i]) continue;
      const hasf_image& im = imgs[first + i];
      const size_t w = im.width, h = im.height, ap = align_up(w * h);
      for (size_t y = 0; y < h; ++y)
        std::memcpy(im.out + y * (size_t)im.pitch, pin + offs[i] + ap + y * w, w);
    }
    first += cnt;
  }
  return HASF_OK;
}
}  // namespace

int hasf_submit(hasf_ctx* ctx, const hasf_image* img, uint64_t* ticket) {
  if (!ctx || !img || !ticket) return HASF_EINVAL;
  int v = validate(img);
  if (v) return v;
  const size_t bytes = serve_job_bytes(ctx, *img);
  if (bytes + 65536 > ctx->budget) return HASF_EBUDGET;
  std::lock_guard<std::mutex> lk(ctx->mu);
  int rc = start_server(ctx);
  if (rc) return rc;
  const uint64_t t = ctx->next_ticket++;
  ctx->pending.push_back(Pending{t, *img, bytes});
  ctx->queued.insert(t);
  *ticket = t;
  ctx->cv.notify_all();
  return HASF_OK;
}

int hasf_poll(hasf_ctx* ctx, uint64_t ticket, int* done, int* status) {
  if (!ctx || !done || !status) return HASF_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->finished.find(ticket);
  if (it != ctx->finished.end()) {
    *done = 1;
    *status = it->second;
    ctx->finished.erase(it);
    return HASF_OK;
  }
  if (ctx->queued.count(ticket) || ctx->launched.count(ticket)) {
    *done = 0;
    *status = HASF_EPENDING;
    return HASF_OK;
  }
  return HASF_ENOTFOUND;
}

int hasf_cancel(hasf_ctx* ctx, uint64_t ticket) {
  if (!ctx) return HASF_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->queued.count(ticket)) {
    for (auto it = ctx->pending.begin(); it != ctx->pending.end(); ++it)
      if (it->ticket == ticket) {
        ctx->pending.erase(it);
        break;
      }
    ctx->queued.erase(ticket);
    ctx->finished[ticket] = HASF_ECANCELLED;
    return HASF_OK;
  }
  if (ctx->launched.count(ticket)) return HASF_EPENDING;
  return HASF_ENOTFOUND;
}

int hasf_drain(hasf_ctx* ctx) {
  if (!ctx) return HASF_EINVAL;
  std::unique_lock<std::mutex> lk(ctx->mu);
  ctx->cv.wait(lk, [&] { return ctx->pending.empty() && ctx->inflight.empty(); });
  return HASF_OK;
}

int hasf_graph_create(hasf_ctx* ctx, const hasf_image* imgs, int n, hasf_graph** out) {
  if (!ctx || !out || n < 1 || !imgs) return HASF_EINVAL;
  *out = nullptr;
  for (int i = 0; i < n; ++i) {
    int v = validate(&imgs[i]);
    if (v) return v;
  }
  cudaSetDevice(ctx->device);
  hasf_graph* g = new (std::nothrow) hasf_graph();
  if (!g) return HASF_ENOMEM;
  g->ctx = ctx;
  Plan p;
  g->bytes = build_plan(ctx, imgs, n, OP_HASF, p, nullptr, nullptr);
  if (g->bytes > ctx->budget) {
    delete g;
    return HASF_EBUDGET;
  }
  cudaError_t e = ctx_malloc(ctx, &g->mem, g->bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete g;
    return HASF_ENOMEM;
  }
  build_plan(ctx, imgs, n, OP_HASF, p, (char*)g->mem, ctx->d_status);
  // Descriptors are fixed: upload them once, outside the capture.
  cudaStream_t cs = nullptr;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  int rc = cuda_status(e);
  if (rc == HASF_OK) rc = launch_plan(ctx, p, (char*)g->mem, cs);  // also warms up
  if (rc == HASF_OK) rc = cuda_status(cudaStreamSynchronize(cs));
  if (rc == HASF_OK) rc = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed));
  if (rc == HASF_OK) {
    int lrc = launch_plan(ctx, p, (char*)g->mem, cs, /*upload=*/false);
    cudaError_t ec = cudaStreamEndCapture(cs, &g->graph);
    rc = lrc ? lrc : cuda_status(ec);
  }
  if (rc == HASF_OK) rc = cuda_status(cudaGraphInstantiate(&g->exec, g->graph, 0));
  if (cs) cudaStreamDestroy(cs);
  if (rc != HASF_OK) {
    cudaGetLastError();
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    cudaFree(g->mem);
    delete g;
    return rc;
  }
  *out = g;
  return HASF_OK;
}

int hasf_graph_launch(hasf_graph* g, void* stream) {
  if (!g) return HASF_EINVAL;
  cudaSetDevice(g->ctx->device);
  return cuda_status(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
}

int hasf_graph_destroy(hasf_graph* g) {
  if (!g) return HASF_EINVAL;
  cudaSetDevice(g->ctx->device);
  cudaDeviceSynchronize();
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  cudaFree(g->mem);
  delete g;
  return HASF_OK;
}

namespace {
// Synthetic tuning image: discs and 5 % salt-and-pepper from a 64-bit LCG.
void tune_image(std::vector<uint8_t>& img, int w, int h) {
  uint64_t st = 0x9E3779B97F4A7C15ull ^ ((uint64_t)w << 32) ^ (uint64_t)h;
  auto next = [&]() {
    st = st * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(st >> 33);
  };
  img.assign((size_t)w * h, 0);
  const int nd = std::max(1, (int)((long long)w * h / 20000));
  for (int d = 0; d < nd; ++d) {
    const int cx = (int)(next() % (uint32_t)w), cy = (int)(next() % (uint32_t)h);
    const int rr = 5 + (int)(next() % 40u);
    for (int y = std::max(0, cy - rr); y <= std::min(h - 1, cy + rr); ++y)
      for (int x = std::max(0, cx - rr); x <= std::min(w - 1, cx + rr); ++x)
        if ((x - cx) * (x - cx) + (y - cy) * (y - cy) <= rr * rr) img[(size_t)y * w + x] = 1;
  }
  for (size_t p = 0; p < img.size(); ++p)
    if (next() % 100u < 5u) img[p] ^= 1;
}
}  // namespace

namespace {
// Time the register kernel's sweep schedules (4, 2 and 1 rows per group) on a
// synthetic image of the bucket's size, in batches that fill the GPU, and
// record the fastest for the bucket.
int tune_reg_group(hasf_ctx* ctx, const hasf_image& im) {
  std::vector<uint8_t> host;
  tune_image(host, im.width, im.height);
  const size_t px = (size_t)im.width * im.height;
  const int copies = std::max(1, 2 * ctx->num_sms);
  uint8_t* dev = nullptr;
  if (ctx_malloc(ctx, (void**)&dev, px * 2 * copies) != cudaSuccess) {
    cudaGetLastError();
    return HASF_ENOMEM;
  }
  for (int c = 0; c < copies; ++c)
    cudaMemcpy(dev + px * 2 * c, host.data(), px, cudaMemcpyHostToDevice);
  std::vector<hasf_image> batch(copies, im);
  for (int c = 0; c < copies; ++c) {
    batch[c].in = dev + px * 2 * c;
    batch[c].out = dev + px * 2 * c + px;
  }
  const Options saved = ctx->opt;
  cudaStream_t s = ctx->host_stream;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  int rc = HASF_OK, best_g = 4;
  float best = 1e30f;
  for (int g : {4, 2, 1}) {
    ctx->opt = saved;
    ctx->opt.row_group = g;
    rc = run_images(ctx, batch.data(), copies, OP_HASF, s);  // warm-up
    if (rc == HASF_OK) rc = hasf_status_of(ctx, s);
    if (rc != HASF_OK) break;
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && rc == HASF_OK; ++rep) {
      cudaEventRecord(a, s);
      rc = run_images(ctx, batch.data(), copies, OP_HASF, s);
      cudaEventRecord(b, s);
      if (rc == HASF_OK) rc = hasf_status_of(ctx, s);
      float t = 0.f;
      cudaEventElapsedTime(&t, a, b);
      ms = std::min(ms, t);
    }
    if (rc != HASF_OK) break;
    if (ms < best) {
      best = ms;
      best_g = g;
    }
  }
  ctx->opt = saved;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(dev);
  if (rc != HASF_OK) return rc;
  std::lock_guard<std::mutex> lk(ctx->tune_mu);
  ctx->tune_group[tune_key(im)] = best_g;
  return HASF_OK;
}
}  // namespace

int hasf_tuning_get(hasf_ctx* ctx, int32_t width, int32_t height, int32_t rmax, int32_t* ctas,
                    int32_t* rows_per_group) {
  if (!ctx || !ctas || !rows_per_group || width < 1 || height < 1 || rmax == 0) return HASF_EINVAL;
  hasf_image im{};
  im.width = width;
  im.height = height;
  im.rmax = rmax;
  const auto key = tune_key(im);
  if (reg_kernel_ok(width, height, std::abs(rmax))) {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    auto it = ctx->tune_group.find(key);
    if (it == ctx->tune_group.end()) return HASF_ENOTFOUND;
    *ctas = 0;
    *rows_per_group = it->second;
    return HASF_OK;
  }
  std::lock_guard<std::mutex> lk(ctx->mu);
  auto it = ctx->tune.find(key);
  if (it == ctx->tune.end()) return HASF_ENOTFOUND;
  *ctas = it->second;
  *rows_per_group = 0;
  return HASF_OK;
}

int hasf_autotune(hasf_ctx* ctx, int32_t width, int32_t height, int32_t rmax, int32_t conn,
                  int32_t* ctas) {
  if (!ctx || !ctas || width < 1 || height < 1 || width > 65536 || height > 65536 || rmax < 1 ||
      rmax > kMaxR || (conn != 4 && conn != 8))
    return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  hasf_image im{};
  im.width = width;
  im.height = height;
  im.pitch = width;
  im.rmax = rmax;
  im.connectivity = conn;
  if (reg_kernel_ok(width, height, rmax)) {  // the register kernel: time its sweep schedules
    *ctas = 0;
    return tune_reg_group(ctx, im);
  }
  std::vector<uint8_t> host;
  tune_image(host, width, height);
  const size_t px = (size_t)width * height;
  uint8_t* dev = nullptr;
  // copies run side by side so that each candidate is timed at full occupancy
  const int copies_max = 16;
  if (cudaMalloc(&dev, px * 2 * copies_max) != cudaSuccess) {
    cudaGetLastError();
    return HASF_ENOMEM;
  }
  for (int c = 0; c < copies_max; ++c)
    cudaMemcpy(dev + px * 2 * c, host.data(), px, cudaMemcpyHostToDevice);
  // candidates: -1 = tiled register kernel, 0 = generic one-CTA kernel,
  // g > 0 = generic gang of g CTAs
  std::vector<int> cands;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tune.erase(tune_key(im));
  }
  if (tile_path(ctx, im)) cands.push_back(-1);
  if (fits_resident(ctx, im)) cands.push_back(0);
  for (int g = 1; g <= ctx->gang_max; g *= 2) cands.push_back(g);
  const Options saved = ctx->opt;
  cudaStream_t s = ctx->host_stream;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  double best = 1e30;
  int best_c = cands.empty() ? 1 : cands.back();
  int rc = HASF_OK;
  for (int c : cands) {
    const int nt = tile_count(width, height);
    const int per = c < 0 ? std::max(1, ctx->num_sms / std::max(1, nt))
                          : (c == 0 ? std::max(1, 2 * ctx->num_sms) : std::max(1, ctx->gang_max / c));
    const int copies = std::min(copies_max, per);
    std::vector<hasf_image> batch(copies, im);
    for (int k = 0; k < copies; ++k) {
      batch[k].in = dev + px * 2 * k;
      batch[k].out = dev + px * 2 * k + px;
    }
    ctx->opt = saved;
    if (c >= 0) {
      ctx->opt.force_gang = c > 0;
      ctx->opt.gang_ctas = c;
      ctx->opt.generic_only = 1;
    }
    rc = run_images(ctx, batch.data(), copies, OP_HASF, s);  // warm-up
    if (rc == HASF_OK) rc = hasf_status_of(ctx, s);
    if (rc != HASF_OK) break;
    cudaEventRecord(a, s);
    rc = run_images(ctx, batch.data(), copies, OP_HASF, s);
    cudaEventRecord(b, s);
    if (rc == HASF_OK) rc = hasf_status_of(ctx, s);
    if (rc != HASF_OK) break;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    const double per_image = ms / copies;
    if (per_image < best) {
      best = per_image;
      best_c = c;
    }
  }
  ctx->opt = saved;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  cudaFree(dev);
  if (rc != HASF_OK) return rc;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    ctx->tune[tune_key(im)] = best_c;
  }
  *ctas = best_c;
  return HASF_OK;
}

int hasf_tuning_save(hasf_ctx* ctx, const char* path) {
  if (!ctx || !path) return HASF_EINVAL;
  FILE* f = std::fopen(path, "w");
  if (!f) return HASF_EINVAL;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    for (const auto& kv : ctx->tune)
      std::fprintf(f, "%d %d %d %d 0\n", std::get<0>(kv.first), std::get<1>(kv.first),
                   std::get<2>(kv.first), kv.second);
  }
  {
    std::lock_guard<std::mutex> lk(ctx->tune_mu);
    for (const auto& kv : ctx->tune_group)
      std::fprintf(f, "%d %d %d 0 %d\n", std::get<0>(kv.first), std::get<1>(kv.first),
                   std::get<2>(kv.first), kv.second);
  }
  std::fclose(f);
  return HASF_OK;
}

int hasf_tuning_load(hasf_ctx* ctx, const char* path) {
  if (!ctx || !path) return HASF_EINVAL;
  FILE* f = std::fopen(path, "r");
  if (!f) return HASF_EINVAL;
  // lines "log2w log2h rmax ctas [rows_per_group]"; a group of 0 or none is a
  // choice of CTAs per image, else a register-kernel schedule
  char line[256];
  while (std::fgets(line, sizeof line, f)) {
    int a, b, c, d, g = 0;
    const int n = std::sscanf(line, "%d %d %d %d %d", &a, &b, &c, &d, &g);
    if (n < 4 || a < 0 || b < 0 || c == 0 || c > kMaxR || c < -kMaxR) continue;
    const auto key = std::make_tuple(a, b, c);
    if (g == 1 || g == 2 || g == 4) {
      std::lock_guard<std::mutex> lk(ctx->tune_mu);
      ctx->tune_group[key] = g;
    } else if (g == 0 && d >= -1) {
      std::lock_guard<std::mutex> lk(ctx->mu);
      ctx->tune[key] = d;
    }
  }
  std::fclose(f);
  return HASF_OK;
}

int hasf_read_stats(hasf_ctx* ctx, uint64_t* out, int n) {
  if (!ctx || !out || n < 1 || n > STAT_COUNT + 1) return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  cudaError_t e = cudaDeviceSynchronize();
  unsigned long long buf[STAT_COUNT] = {0};
  if (e == cudaSuccess)
    e = cudaMemcpy(buf, ctx->d_stats, sizeof(buf), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_stats, 0, sizeof(buf));
  if (e != cudaSuccess) return cuda_status(e);
  for (int i = 0; i < n && i < STAT_COUNT; ++i) out[i] = buf[i];
  if (n > STAT_COUNT) out[STAT_COUNT] = ctx->launches;
  ctx->launches = 0;
  return HASF_OK;
}

const char* hasf_strerror(int status) {
  switch (status) {
    case HASF_OK: return "ok";
    case HASF_EINVAL: return "invalid argument";
    case HASF_ENOMEM: return "out of memory";
    case HASF_EBUDGET: return "job exceeds the context's memory budget";
    case HASF_EPENDING: return "job not finished";
    case HASF_ETIMEOUT: return "device iteration cap or wait deadline reached";
    case HASF_EUNSTABLE: return "run to stability: the last allowed step still changed the image";
    case HASF_ECUDA: return "CUDA runtime error";
    case HASF_ENOTFOUND: return "unknown ticket";
    case HASF_ECANCELLED: return "job cancelled";
    default: return "unknown status";
  }
}

int hasf_simple_table(hasf_ctx* ctx, int32_t connectivity, uint8_t* out256) {
  if (!ctx || !out256 || (connectivity != 8 && connectivity != 4)) return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  uint8_t* d = nullptr;
  cudaError_t e = cudaMalloc(&d, 256);
  if (e == cudaSuccess) e = launch_simple_table(connectivity, d, ctx->host_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out256, d, 256, cudaMemcpyDeviceToHost, ctx->host_stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->host_stream);
  if (d) cudaFree(d);
  return cuda_status(e);
}

int hasf_levels(hasf_ctx* ctx, const uint8_t* feat, int32_t width, int32_t height, int32_t pitch,
                int32_t mode, int32_t r, int32_t* d, void* stream) {
  if (!ctx || !feat || !d || width < 1 || height < 1 || width > 65536 || height > 65536 ||
      pitch < width || r < 1 || r > kMaxR || mode < 0 || mode > 2)
    return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t pw = (size_t)plane_words(width, height);
  int rc = ensure_arena(ctx, 2 * pw * 4, s);
  if (rc) return rc;
  uint32_t* f = (uint32_t*)ctx->arena;
  return cuda_status(launch_levels(feat, width, height, pitch, mode, r, f, f + pw, d, s));
}

int hasf_edt(hasf_ctx* ctx, const uint8_t* feat, int32_t width, int32_t height, int32_t pitch,
             int32_t outside_is_feature, int32_t* d, void* stream) {
  if (!ctx || !feat || !d || width < 1 || height < 1 || width > 32768 || height > 32768 ||
      pitch < width)
    return HASF_EINVAL;
  cudaSetDevice(ctx->device);
  cudaStream_t s = (cudaStream_t)stream;
  const size_t g_bytes = align_up((size_t)width * height * 4);
  const size_t st_bytes = (size_t)height * 2 * (width + 2) * 4;
  int rc = ensure_arena(ctx, g_bytes + st_bytes, s);
  if (rc) return rc;
  char* base = (char*)ctx->arena;
  return cuda_status(launch_edt(feat, width, height, pitch, outside_is_feature ? 1 : 0,
                                (int32_t*)base, (int32_t*)(base + g_bytes), d, s));
}

}  // extern "C"
