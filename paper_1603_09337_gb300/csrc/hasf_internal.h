// hasf_internal.h -- types shared by the host runtime and the kernels of the
// HASF library (not part of the public C ABI).
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

namespace hasf {

constexpr int kThreads = 512;      // threads per CTA of the fused kernels
constexpr int kMaxR = 64;          // largest radius (rmax) supported
constexpr int kMaxOffsets = 12852; // lattice points v != 0 with |v|^2 <= 64^2
constexpr int kMaxLevels = 1197;   // sums of two squares in [1, 64^2]

// Operation a job runs.
enum Op : int {
  OP_HASF = 0,   // HC_r then HF_r for r = r_lo..r_hi
  OP_THIN = 1,   // H(Z, W): in = Z, C = W, levels 1..r_hi^2
  OP_THICK = 2,  // *H(Y, V): in = Y, C = V, levels 1..r_hi^2
  OP_HC = 3,     // HC_{r_hi}
  OP_HF = 4,     // HF_{r_hi}
};

// Work counters a job adds to when Job::stats is set.
enum StatIndex : int {
  STAT_WORD_TESTS = 0,  // sweep words tested, once per subfield
  STAT_RING_EVALS = 1,  // shifted feature words read by level updates
  STAT_PASSES = 2,      // subfield passes
  STAT_LEVELS = 3,      // levels that activated points
  STAT_ROUNDS = 4,      // rounds
  STAT_COUNT = 5
};

// Device status codes written by kernels (a subset of hasf_status).
// Device status of a job; jobs of one launch combine theirs with atomicMax,
// so the more serious status wins.
enum DevStatus : int { DEV_OK = 0, DEV_UNSTABLE = 1, DEV_TIMEOUT = 5 };

// One image job as the kernels see it.  Planes are bit-packed, 32 pixels per
// 32-bit word, bit b of word j of row y = pixel (32 j + b, y).
struct Job {
  const uint8_t* in;
  uint8_t* out;
  const uint8_t* C;
  const uint8_t* D;
  uint32_t* g0;      // h * wpr words: snapshot of the operator input
  uint32_t* cp;      // h * wpr words or null: kept points (C cap X) / W / V
  uint32_t* dp;      // h * wpr words or null: forbidden points (D minus X)
  uint32_t* g1;      // run to stability: h * wpr words, the image before the step
  uint32_t* planes;  // gang mode: 3 padded planes (S, F, cand); else null
  unsigned* sync;    // gang mode: 8 barrier words; else null
  int* status;       // device status word of the job
  unsigned long long* stats;  // work counters (see StatIndex) or null
  int* notify;       // host-mapped word set to 1 + status when the job is done, or null
  int w, h, pitch, wpr;
  int r_lo, r_hi;
  int op;
  int conn;
  int gang;          // CTAs cooperating on the job (gang mode)
  int cap;           // rounds allowed per level before DEV_TIMEOUT
  int plane_words;   // words per padded plane (see plane_words())
  int stable;        // 1: stop after the first step r that changes nothing
  int deadline_ms;   // gang barrier wait limit (0 = 4000 ms)
  int fault_skip;    // fault injection: 1 makes CTA 0 of a gang leave before its first barrier
};

// One volume job of the 3D filter.  Planes: d * h rows of wpr words, bit b of
// word j of row (y, z) = voxel (32 j + b, y, z); all in global memory.
struct Job3 {
  const uint8_t* in;   // dense w * h * d bytes, x fastest
  uint8_t* out;
  const uint8_t* C;
  const uint8_t* D;
  uint32_t* S;         // current set
  uint32_t* F;         // operator input (priority source)
  uint32_t* cand;      // candidates
  uint32_t* M;         // points allowed to change
  uint32_t* g0;        // input of the current HC_r / HF_r
  uint32_t* cp;        // C cap X, or null
  uint32_t* dp;        // D minus X, or null
  unsigned* sync;      // 8 barrier words (zeroed before the launch)
  int* status;
  unsigned long long* stats;
  const uint32_t* simple_lut;  // simple-voxel table (kSimple3TableWords), or null: flood fill
  int w, h, d, wpr;
  int rmax;
  int gang;            // CTAs of the gang
  int cap;             // rounds allowed per level
  int deadline_ms;     // gang barrier wait limit (0 = 4000 ms)
  int fault_skip;      // fault injection, as in Job
  int pad_[1];         // 160 bytes: descriptors stay 16-byte aligned in the array
};

// The simple-voxel table of (26, 6) adjacency: bit i of the table is 1 when
// the centre of the 3 x 3 x 3 neighbourhood with the 26 neighbour bits i (the
// 27-bit position code with the centre bit taken out) is simple.  2^26 bits.
constexpr size_t kSimple3TableWords = size_t(1) << 21;
cudaError_t build_simple3_table(uint32_t* lut, cudaStream_t s);

// Padded plane geometry shared by both modes: rows -1..h, P words per row
// (P = the first odd number above the words of a row; the extra words and
// rows are zero: outside the box), one zero word before row -1, rounded up
// to 4 words.  P odd lets two half-warps on rows 16 apart (or quarter-warps
// on rows 8 apart ...) hit disjoint shared-memory banks.
__host__ __device__ inline int words_per_row(int w) { return (w + 31) >> 5; }
__host__ __device__ inline int row_pitch(int w) {
  const int wpr = words_per_row(w);
  return wpr + 1 + (wpr & 1);
}
__host__ __device__ inline int plane_words(int w, int h) {
  long long n = (long long)(h + 2) * row_pitch(w) + 2;
  return (int)((n + 3) & ~3LL);
}
__host__ __device__ inline int dirty_words(int, int) { return 0; }
inline size_t state_bytes(int w, int h) {
  return (3ull * (size_t)plane_words(w, h) + (size_t)dirty_words(w, h)) * 4ull;
}
inline size_t resident_smem_bytes(int w, int h) { return state_bytes(w, h); }

// Host launchers (hasf_kernels.cu).
cudaError_t upload_level_table();
cudaError_t set_level_table_reg(const void* tab, size_t bytes);
cudaError_t set_level_table_tiled(const void* tab, size_t bytes);
constexpr int kMaxR3D = 12;   // largest rmax of the 3D filter
cudaError_t upload_level_table_3d();
int max_3d_ctas(int device);
// table: every job's simple_lut is set (the table instance of the kernel).
cudaError_t launch_3d(const Job3* d_jobs, const int2* d_ctamap, int nctas, bool table,
                      cudaStream_t s);
cudaError_t launch_resident(const Job* d_jobs, const int* d_order, int njobs, int grid,
                            size_t smem_bytes, unsigned* d_counter, cudaStream_t s);
cudaError_t launch_gang(const Job* d_jobs, const int2* d_ctamap, int nctas, cudaStream_t s);
size_t reg_kernel_smem(int w, int h);
bool reg_kernel_ok(int w, int h, int rmax);
int reg_ctas_per_sm(size_t smem_bytes);
// group: rows of a parity tested together by a sweep (1, 2 or 4).
cudaError_t launch_reg(int group, const Job* d_jobs, const int* d_order, int njobs, int grid,
                       size_t smem_bytes, unsigned* d_counter, cudaStream_t s);
cudaError_t launch_reg_g1(const Job* d_jobs, const int* d_order, int njobs, int grid,
                          size_t smem_bytes, unsigned* d_counter, cudaStream_t s);
cudaError_t launch_reg_g2(const Job* d_jobs, const int* d_order, int njobs, int grid,
                          size_t smem_bytes, unsigned* d_counter, cudaStream_t s);
// One image on one CTA of the register kernel, the job passed by value (no
// device memory for a job list); reg_one_prepare once per device first.
cudaError_t reg_one_prepare();
cudaError_t launch_reg_one(const Job& jb, cudaStream_t s);
cudaError_t set_level_table_reg_g1(const void* tab, size_t bytes);
cudaError_t set_level_table_reg_g2(const void* tab, size_t bytes);
size_t tile_kernel_smem();
int tile_count(int w, int h);
size_t tile_gang_words(int w, int h);
int tile_clusters_possible(int csize);
cudaError_t launch_tile_cluster(const Job* d_jobs, const int* d_order, int njobs, int csize,
                                bool alone, cudaStream_t s);
int max_tile_gang_ctas(int device);
cudaError_t launch_tile_gang(const Job* d_jobs, const int2* d_ctamap, int nctas, bool alone,
                             cudaStream_t s);
constexpr int kTileMaxR = 31;   // the tiled kernels take rmax <= 31
int max_gang_ctas(int device);
size_t max_resident_smem(int device);
int resident_ctas_per_sm(int device, size_t smem_bytes);
cudaError_t launch_simple_table(int conn, uint8_t* d_out256, cudaStream_t s);
// One 2D byte copy: h rows of w bytes, row pitches in bytes.
struct Copy2D {
  const uint8_t* src;
  uint8_t* dst;
  int w, h, spitch, dpitch;
};
cudaError_t launch_copy2d(const Copy2D* d_copies, int n, cudaStream_t s);
cudaError_t launch_levels(const uint8_t* feat, int w, int h, int pitch, int mode, int r,
                          uint32_t* d_plane_f, uint32_t* d_plane_a, int32_t* d, cudaStream_t s);
cudaError_t launch_edt(const uint8_t* feat, int w, int h, int pitch, int outside, int32_t* g,
                       int32_t* stack, int32_t* d, cudaStream_t s);

}  // namespace hasf
