// hasf_3d.cu -- HASF of 3D volumes with (26, 6) adjacency.
//
// The paper states the filter for 2D images and notes (Sec. 1) that it
// applies to 3D ones.  Here the same scheme runs on volumes: eqs. (i) and (ii)
// with B_r the ball |v|^2 <= r^2; priorities in threshold form (a voxel has
// priority <= l iff a feature voxel lies at a lattice vector of squared norm
// <= l; the levels are the sums of three squares); rounds of the eight
// subfields (x mod 2, y mod 2, z mod 2), taken in the order s = 0..7 with
// parities (s & 1, (s >> 1) & 1, s >> 2).  Voxels of one subfield differ by an
// even amount in every coordinate, so they are never 26-adjacent and a whole
// subfield is updated at once.
//
// Simple voxels: the object voxels of the 26-neighbourhood form one
// 26-connected component and the background voxels of the 18-neighbourhood
// that are 6-connected to a face neighbour form one 6-connected component.
// Both numbers are computed on the 27-bit neighbourhood code by flood fill
// with mask dilations (shifts by 1, 3, 9 for x, y, z).
//
// Layout: each plane is d * h rows of ceil(w / 32) words (bit b of word j of
// row (y, z) = voxel (32 j + b, y, z)), in global memory (L2).  A volume is
// processed by a gang of co-resident CTAs meeting at the bounded gang barrier
// after every phase.  Plain (L1-cacheable) loads and stores: within a phase no
// word is written that another thread reads, and the barrier between phases
// (fence and counter release, counter poll and fence acquire, then the CTA
// barrier) orders every write before every later read, as a grid-wide sync
// does; one thread only ever reads back its own candidate words.
#include <cstdint>
#include <algorithm>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

#include "hasf_device.cuh"

namespace hasf {

__device__ __forceinline__ void st_plain(uint32_t* p, uint32_t v) { *p = v; }

#ifndef HASF_3D_TABLE_BATCH
#define HASF_3D_TABLE_BATCH 4
#endif

constexpr int kMaxR3 = kMaxR3D;
constexpr int kMaxOff3 = 7300;   // lattice vectors with 0 < |v|^2 <= 144
constexpr int kMaxLev3 = 150;

struct LevelTable3 {
  uint16_t value[kMaxLev3];
  uint16_t start[kMaxLev3 + 1];
  uint16_t nlev[kMaxR3 + 1];
  int8_t off[kMaxOff3][3];
};
static __constant__ LevelTable3 c_lv3;

// ---------------------------------------------------------------------------
// Topology of a 3 x 3 x 3 neighbourhood.  Position of offset (dx, dy, dz):
// (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1); the centre is position 13.
// ---------------------------------------------------------------------------

constexpr uint32_t cube_mask(int axis, int val) {
  uint32_t m = 0;
  for (int i = 0; i < 27; ++i) {
    const int c = axis == 0 ? i % 3 : (axis == 1 ? (i / 3) % 3 : i / 9);
    if (c == val) m |= 1u << i;
  }
  return m;
}
constexpr uint32_t l1_mask(int lo, int hi) {
  uint32_t m = 0;
  for (int i = 0; i < 27; ++i) {
    const int a = i % 3 - 1, b = (i / 3) % 3 - 1, c = i / 9 - 1;
    const int l1 = (a < 0 ? -a : a) + (b < 0 ? -b : b) + (c < 0 ? -c : c);
    if (l1 >= lo && l1 <= hi) m |= 1u << i;
  }
  return m;
}
constexpr uint32_t kX0 = cube_mask(0, 0), kX2 = cube_mask(0, 2);
constexpr uint32_t kY0 = cube_mask(1, 0), kY2 = cube_mask(1, 2);
constexpr uint32_t kZ0 = cube_mask(2, 0), kZ2 = cube_mask(2, 2);
constexpr uint32_t kN26 = l1_mask(1, 3), kN18 = l1_mask(1, 2), kN6 = l1_mask(1, 1);

__device__ __forceinline__ uint32_t dil_x(uint32_t s) {
  return s | ((s & ~kX2) << 1) | ((s & ~kX0) >> 1);
}
__device__ __forceinline__ uint32_t dil_y(uint32_t s) {
  return s | ((s & ~kY2) << 3) | ((s & ~kY0) >> 3);
}
__device__ __forceinline__ uint32_t dil_z(uint32_t s) {
  return s | ((s & ~kZ2) << 9) | ((s & ~kZ0) >> 9);
}

__device__ __forceinline__ bool simple3(uint32_t code) {
  // one 26-component of object neighbours
  const uint32_t obj = code & kN26;
  if (!obj) return false;
  uint32_t comp = obj & (0u - obj);
  for (int it = 0; it < 27; ++it) {
    const uint32_t nc = dil_z(dil_y(dil_x(comp))) & obj;
    if (nc == comp) break;
    comp = nc;
  }
  if (comp != obj) return false;
  // one 6-component of 18-neighbourhood background touching a face neighbour
  const uint32_t bg = ~code & kN18;
  const uint32_t touch = bg & kN6;
  if (!touch) return false;
  comp = touch & (0u - touch);
  for (int it = 0; it < 27; ++it) {
    const uint32_t nc = (dil_x(comp) | dil_y(comp) | dil_z(comp)) & bg;
    if (nc == comp) break;
    comp = nc;
  }
  return (touch & ~comp) == 0u;
}

// ---------------------------------------------------------------------------
// Per-CTA view of a volume job.
// ---------------------------------------------------------------------------

struct V3 {
  int w, h, d, wpr;
  long long nw;        // words per plane
  int gtid, gthreads;  // this thread in the gang
  bool solo;
  GangMode gm;
  uint32_t lastmask;
  unsigned long long n_tests, n_ring, n_rounds, n_levels;
  __device__ __forceinline__ int bar(int v) { return solo ? __syncthreads_or(v) : gm.barrier(v); }
  __device__ __forceinline__ bool failed() const { return !solo && gm.failed(); }
  __device__ __forceinline__ uint32_t rowmask(int j) const {
    return j == wpr - 1 ? lastmask : 0xFFFFFFFFu;
  }
  __device__ __forceinline__ uint32_t ld(const uint32_t* P, int j, int y, int z) const {
    if (j < 0 || j >= wpr || y < 0 || y >= h || z < 0 || z >= d) return 0u;
    return P[((long long)z * h + y) * wpr + j];
  }
};

__device__ __forceinline__ void word_pos(const V3& v, long long t, int& j, int& y, int& z) {
  j = (int)(t % v.wpr);
  const long long row = t / v.wpr;
  y = (int)(row % v.h);
  z = (int)(row / v.h);
}

__device__ uint32_t pack3(const uint8_t* p, int n) {
  uint32_t s = 0;
  for (int b = 0; b < n; ++b) s |= (p[b] != 0 ? 1u : 0u) << b;
  return s;
}

// Load the 3 x 3 rows around row (y, z) at word j as 96-bit windows: bit i of
// win[k] is voxel x = 32 j + i - 1 of row (y + k % 3 - 1, z + k / 3 - 1).
__device__ __forceinline__ void load_window(const V3& v, const uint32_t* S, int j, int y, int z,
                                            uint64_t (&win)[9]) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int dy = k % 3 - 1, dz = k / 3 - 1;
    const uint32_t p = v.ld(S, j - 1, y + dy, z + dz);
    const uint32_t c = v.ld(S, j, y + dy, z + dz);
    const uint32_t n = v.ld(S, j + 1, y + dy, z + dz);
    win[k] = ((uint64_t)n << 33) | ((uint64_t)c << 1) | (uint64_t)(p >> 31);
  }
}

// Index of a 27-bit position code in the simple-voxel table: the 26
// neighbour bits, the centre (bit 13) taken out.
__device__ __forceinline__ uint32_t simple3_index(uint32_t code) {
  return (code & 0x1FFFu) | ((code >> 14) << 13);
}

// The table, 32 codes per thread: word i holds the codes 32 i .. 32 i + 31.
__global__ void __launch_bounds__(256) simple3_table_kernel(uint32_t* lut) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kSimple3TableWords) return;
  uint32_t word = 0;
  for (int b = 0; b < 32; ++b) {
    const uint32_t idx = (i << 5) | (uint32_t)b;
    const uint32_t code = (idx & 0x1FFFu) | ((idx >> 13) << 14);
    if (simple3(code)) word |= 1u << b;
  }
  lut[i] = word;
}

// The simple voxels among the candidate bits cw of the window's centre word:
// by the table (kTable: one read of an 8 MB table that stays in L2), else by
// the flood fills of simple3.  The kernel is compiled once for each.
// The 27-bit position code of the voxel at bit b of the window's centre word.
__device__ __forceinline__ uint32_t window_code(const uint64_t (&win)[9], int b) {
  uint32_t code = 0;
#pragma unroll
  for (int k = 0; k < 9; ++k) code |= (uint32_t)((win[k] >> b) & 7u) << (3 * k);
  return code;
}

// Table form: the candidates are taken kBatch at a time, their table words
// read together, so that a lane waits for one L2 round trip per batch rather
// than one per voxel (the voxels of one word lie in one subfield and do not
// see each other's changes, so the order does not matter).
constexpr int kTableBatch = HASF_3D_TABLE_BATCH;
__device__ __forceinline__ uint32_t test_bits_table(V3& v, const uint64_t (&win)[9], uint32_t cw,
                                                    const uint32_t* __restrict__ lut) {
  uint32_t chg = 0;
  while (cw) {
    uint32_t bit[kTableBatch], idx[kTableBatch], word[kTableBatch];
#pragma unroll
    for (int i = 0; i < kTableBatch; ++i) {
      bit[i] = cw & (0u - cw);   // the lowest candidate left, or 0
      cw ^= bit[i];
      idx[i] = simple3_index(window_code(win, bit[i] ? __ffs(bit[i]) - 1 : 0));
    }
#pragma unroll
    for (int i = 0; i < kTableBatch; ++i) word[i] = bit[i] ? __ldg(lut + (idx[i] >> 5)) : 0u;
#pragma unroll
    for (int i = 0; i < kTableBatch; ++i) {
      v.n_tests += bit[i] != 0u;
      if ((word[i] >> (idx[i] & 31u)) & 1u) chg |= bit[i];
    }
  }
  return chg;
}

template <bool kTable>
__device__ __forceinline__ uint32_t test_bits(V3& v, const uint64_t (&win)[9], uint32_t cw,
                                              const uint32_t* __restrict__ lut) {
  if (kTable) return test_bits_table(v, win, cw, lut);
  uint32_t chg = 0;
  while (cw) {
    const int b = __ffs(cw) - 1;
    cw &= cw - 1u;
    ++v.n_tests;
    if (simple3(window_code(win, b))) chg |= 1u << b;
  }
  return chg;
}

// One subfield (sx, sy, sz): every candidate voxel of it that is simple changes.
template <bool kTable>
__device__ int sweep_sub3(V3& v, const Job3& jb, bool thin, int sx, int sy, int sz) {
  const int ny = (v.h - sy + 1) >> 1, nz = (v.d - sz + 1) >> 1;
  const long long nsub = (long long)ny * nz * v.wpr;
  const uint32_t xm = sx ? 0xAAAAAAAAu : 0x55555555u;
  int changed = 0;
  for (long long q = v.gtid; q < nsub; q += v.gthreads) {
    const int j = (int)(q % v.wpr);
    const long long rr = q / v.wpr;
    const int y = sy + 2 * (int)(rr % ny), z = sz + 2 * (int)(rr / ny);
    const long long t = ((long long)z * v.h + y) * v.wpr + j;
    const uint32_t call = (*(jb.cand + t));
    const uint32_t cw = call & xm;
    if (!cw) continue;
    uint64_t win[9];
    load_window(v, jb.S, j, y, z, win);
    const uint32_t cur = (uint32_t)(win[4] >> 1);
    const uint32_t chg = test_bits<kTable>(v, win, cw, jb.simple_lut);
    if (chg) {
      st_plain(jb.S + t, thin ? (cur & ~chg) : (cur | chg));
      st_plain(jb.cand + t, call & ~chg);
      changed = 1;
    }
  }
  return changed;
}

// The two subfields (0, sy, sz) then (1, sy, sz) fused, for rows of at most 32
// words: a row is handled by wpr consecutive lanes of one warp, which test the
// even voxels, pass their updated words one lane to the left (an odd voxel at
// bit 31 sees the next word's even voxel 0 as the first subfield left it),
// then test the odd voxels.  Only the row itself changes in these two passes,
// and a warp's lanes load everything before any of them stores.
template <bool kTable>
__device__ int sweep_pair3(V3& v, const Job3& jb, bool thin, int sy, int sz) {
  const int ny = (v.h - sy + 1) >> 1, nz = (v.d - sz + 1) >> 1;
  const long long nrows = (long long)ny * nz;
  const int per_warp = 32 / v.wpr;
  const int lane = threadIdx.x & 31;
  const int rl = lane / v.wpr, j = lane - rl * v.wpr;
  const long long gw = v.gtid >> 5, nwarps = v.gthreads >> 5;
  int changed = 0;
  for (long long rb = gw * per_warp; rb < nrows; rb += nwarps * per_warp) {
    const long long row = rb + rl;
    const bool act = rl < per_warp && row < nrows;
    long long t = 0;
    uint32_t call = 0;
    if (act) {
      const int y = sy + 2 * (int)(row % ny), z = sz + 2 * (int)(row / ny);
      t = ((long long)z * v.h + y) * v.wpr + j;
      call = (*(jb.cand + t));
    }
    if (!__any_sync(0xFFFFFFFFu, call != 0u)) continue;
    uint64_t win[9];
    uint32_t cur = 0, ch0 = 0;
    if (act && call) {
      const int y = sy + 2 * (int)(row % ny), z = sz + 2 * (int)(row / ny);
      load_window(v, jb.S, j, y, z, win);
      cur = (uint32_t)(win[4] >> 1);
      ch0 = test_bits<kTable>(v, win, call & 0x55555555u, jb.simple_lut);
    } else {
      cur = act ? (*(jb.S + t)) : 0u;
    }
    const uint32_t c1 = thin ? (cur & ~ch0) : (cur | ch0);
    uint32_t east = __shfl_down_sync(0xFFFFFFFFu, c1, 1);
    if (j == v.wpr - 1) east = 0u;   // the next word is outside the box
    uint32_t ch1 = 0;
    const uint32_t cw1 = call & 0xAAAAAAAAu;
    if (act && cw1) {
      win[4] = ((uint64_t)east << 33) | ((uint64_t)c1 << 1) | (win[4] & 1u);
      ch1 = test_bits<kTable>(v, win, cw1, jb.simple_lut);
    }
    __syncwarp();
    const uint32_t chg = ch0 | ch1;
    if (act && chg) {
      st_plain(jb.S + t, thin ? (c1 & ~ch1) : (c1 | ch1));
      st_plain(jb.cand + t, call & ~chg);
      changed = 1;
    }
  }
  return changed;
}

// One constrained thinning (thin) or thickening of S at radius r; the points
// allowed to change lie in pos (if given) and not in neg (if given).
template <bool kTable>
__device__ bool op3(V3& v, const Job3& jb, int r, bool thin, const uint32_t* pos,
                    const uint32_t* neg) {
  for (long long t = v.gtid; t < v.nw; t += v.gthreads) {
    const uint32_t s = (*(jb.S + t));
    st_plain(jb.F + t, s);
    uint32_t m = v.rowmask((int)(t % v.wpr));
    if (pos) m &= (*(pos + t));
    if (neg) m &= ~(*(neg + t));
    st_plain(jb.M + t, m);
    st_plain(jb.cand + t, 0u);
  }
  v.bar(0);
  if (v.failed()) return false;
  const int nlev = c_lv3.nlev[r];
  for (int li = 0; li < nlev; ++li) {
    // new candidates: points whose priority is the level's value
    int any = 0;
    const int o0 = c_lv3.start[li], o1 = c_lv3.start[li + 1];
    for (long long t = v.gtid; t < v.nw; t += v.gthreads) {
      const uint32_t s = (*(jb.S + t)), c = (*(jb.cand + t));
      const uint32_t pend = (*(jb.M + t)) & (thin ? s : ~s) & ~c;
      if (!pend) continue;
      int j, y, z;
      word_pos(v, t, j, y, z);
      uint32_t acc = thin ? 0xFFFFFFFFu : 0u;
      for (int o = o0; o < o1; ++o) {
        const int dx = c_lv3.off[o][0], dy = c_lv3.off[o][1], dz = c_lv3.off[o][2];
        const int j0 = j + (dx >> 5), sh = dx & 31;
        const uint32_t lo = v.ld(jb.F, j0, y + dy, z + dz);
        const uint32_t val = sh ? __funnelshift_r(lo, v.ld(jb.F, j0 + 1, y + dy, z + dz), sh) : lo;
        acc = thin ? (acc & val) : (acc | val);
        ++v.n_ring;
        if (((o - o0) & 3) == 3 && !(pend & (thin ? acc : ~acc))) break;
      }
      const uint32_t add = pend & (thin ? ~acc : acc);
      if (add) {
        st_plain(jb.cand + t, c | add);
        any = 1;
      }
    }
    any = v.bar(any);
    if (v.failed()) return false;
    if (!any) continue;
    ++v.n_levels;
    // rounds of the eight subfields until a round changes nothing
    for (int round = 0;; ++round) {
      if (round >= jb.cap) return false;
      ++v.n_rounds;
      int changed = 0;
      if (v.wpr <= 32) {
        for (int m = 0; m < 4; ++m) {   // (sy, sz) = (0,0), (1,0), (0,1), (1,1)
          changed |= sweep_pair3<kTable>(v, jb, thin, m & 1, m >> 1);
          const int o = v.bar(m == 3 ? changed : 0);
          if (v.failed()) return false;
          if (m == 3) changed = o;
        }
      } else {
        for (int sub = 0; sub < 8; ++sub) {
          changed |= sweep_sub3<kTable>(v, jb, thin, sub & 1, (sub >> 1) & 1, sub >> 2);
          const int o = v.bar(sub == 7 ? changed : 0);
          if (v.failed()) return false;
          if (sub == 7) changed = o;
        }
      }
      if (!changed) break;
    }
  }
  return true;
}

__device__ void snapshot3(V3& v, const Job3& jb) {
  for (long long t = v.gtid; t < v.nw; t += v.gthreads) st_plain(jb.g0 + t, (*(jb.S + t)));
  v.bar(0);
}

// CTA b works on part ctamap[b].y of job ctamap[b].x (a gang of jobs[].gang CTAs).
// Two CTAs per SM: the sweeps wait on gang barriers, and a second CTA hides them.
template <bool kTable>
__global__ void __launch_bounds__(kThreads, 2)
hasf_3d_kernel(const Job3* __restrict__ jobs, const int2* __restrict__ ctamap) {
  __shared__ __align__(8) int flag[4];  // gang barrier state (GangMode)
  const int2 m = ctamap[blockIdx.x];
  const Job3& jb = jobs[m.x];
  if (gang_fault_leaves(jb.fault_skip, jb.gang, m.y)) return;
  V3 v;
  v.w = jb.w;
  v.h = jb.h;
  v.d = jb.d;
  v.wpr = jb.wpr;
  v.nw = (long long)jb.d * jb.h * jb.wpr;
  v.gtid = m.y * blockDim.x + threadIdx.x;
  v.gthreads = jb.gang * blockDim.x;
  v.solo = jb.gang == 1;
  v.gm.init(jb.sync, jb.gang, flag, jb.deadline_ms);
  const int rem = jb.w & 31;
  v.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
  v.n_tests = v.n_ring = v.n_rounds = v.n_levels = 0;
  // pack X (and C cap X, D minus X)
  for (long long t = v.gtid; t < v.nw; t += v.gthreads) {
    int j, y, z;
    word_pos(v, t, j, y, z);
    const long long off = ((long long)z * jb.h + y) * jb.w + 32LL * j;
    const int n = min(32, jb.w - 32 * j);
    const uint32_t x = pack3(jb.in + off, n);
    st_plain(jb.S + t, x);
    if (jb.cp) st_plain(jb.cp + t, jb.C ? (pack3(jb.C + off, n) & x) : 0u);
    if (jb.dp) st_plain(jb.dp + t, jb.D ? (pack3(jb.D + off, n) & ~x) : 0u);
  }
  v.bar(0);
  bool ok = !v.failed();
  for (int r = 1; ok && r <= jb.rmax; ++r) {
    snapshot3(v, jb);   // HC_r: thinning that keeps C, thickening inside its input
    ok = op3<kTable>(v, jb, r, true, nullptr, jb.cp) &&
         op3<kTable>(v, jb, r, false, jb.g0, nullptr);
    if (!ok) break;
    snapshot3(v, jb);   // HF_r: thickening that avoids D, thinning that keeps its input
    ok = op3<kTable>(v, jb, r, false, nullptr, jb.dp) &&
         op3<kTable>(v, jb, r, true, nullptr, jb.g0);
  }
  if (ok) {
    for (long long t = v.gtid; t < v.nw; t += v.gthreads) {
      int j, y, z;
      word_pos(v, t, j, y, z);
      const uint32_t s = (*(jb.S + t));
      uint8_t* o = jb.out + ((long long)z * jb.h + y) * jb.w + 32LL * j;
      const int n = min(32, jb.w - 32 * j);
      for (int b = 0; b < n; ++b) o[b] = (uint8_t)((s >> b) & 1u);
    }
  } else if (threadIdx.x == 0) {
    atomicMax(jb.status, (int)DEV_TIMEOUT);
  }
  if (jb.stats) {
    unsigned long long a = v.n_tests, b = v.n_ring;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xFFFFFFFFu, a, o);
      b += __shfl_down_sync(0xFFFFFFFFu, b, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(jb.stats + STAT_WORD_TESTS, a);
      atomicAdd(jb.stats + STAT_RING_EVALS, b);
    }
    if (v.gtid == 0) {
      atomicAdd(jb.stats + STAT_LEVELS, v.n_levels);
      atomicAdd(jb.stats + STAT_ROUNDS, v.n_rounds);
    }
  }
}

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------

cudaError_t upload_level_table_3d() {
  static LevelTable3 tab;
  static bool built = false;
  static std::mutex mu;
  std::lock_guard<std::mutex> lock(mu);
  if (!built) {
    struct V { int n2, dx, dy, dz; };
    std::vector<V> vs;
    const int R = kMaxR3;
    for (int dz = -R; dz <= R; ++dz)
      for (int dy = -R; dy <= R; ++dy)
        for (int dx = -R; dx <= R; ++dx) {
          const int n2 = dx * dx + dy * dy + dz * dz;
          if (n2 >= 1 && n2 <= R * R) vs.push_back({n2, dx, dy, dz});
        }
    std::stable_sort(vs.begin(), vs.end(), [](const V& a, const V& b) { return a.n2 < b.n2; });
    if ((int)vs.size() > kMaxOff3) return cudaErrorInvalidValue;
    int nl = 0;
    for (size_t i = 0; i < vs.size(); ++i) {
      if (i == 0 || vs[i].n2 != vs[i - 1].n2) {
        if (nl >= kMaxLev3) return cudaErrorInvalidValue;
        tab.value[nl] = (uint16_t)vs[i].n2;
        tab.start[nl] = (uint16_t)i;
        ++nl;
      }
      tab.off[i][0] = (int8_t)vs[i].dx;
      tab.off[i][1] = (int8_t)vs[i].dy;
      tab.off[i][2] = (int8_t)vs[i].dz;
    }
    tab.start[nl] = (uint16_t)vs.size();
    for (int r = 0; r <= R; ++r) {
      int c = 0;
      while (c < nl && tab.value[c] <= r * r) ++c;
      tab.nlev[r] = (uint16_t)c;
    }
    built = true;
  }
  return cudaMemcpyToSymbol(c_lv3, &tab, sizeof(tab));
}

cudaError_t build_simple3_table(uint32_t* lut, cudaStream_t s) {
  simple3_table_kernel<<<(unsigned)(kSimple3TableWords / 256), 256, 0, s>>>(lut);
  return cudaGetLastError();
}

int max_3d_ctas(int device) {
  int per_sm = 0, sms = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, hasf_3d_kernel<true>, kThreads, 0);
  int per_sm_flood = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_flood, hasf_3d_kernel<false>, kThreads, 0);
  per_sm = std::min(per_sm, per_sm_flood);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  return per_sm * sms;
}

cudaError_t launch_3d(const Job3* d_jobs, const int2* d_ctamap, int nctas, bool table,
                      cudaStream_t s) {
  void* args[] = {(void*)&d_jobs, (void*)&d_ctamap};
  const void* fn = table ? (const void*)hasf_3d_kernel<true> : (const void*)hasf_3d_kernel<false>;
  return cudaLaunchCooperativeKernel(fn, dim3(nctas), dim3(kThreads), args, 0, s);
}

}  // namespace hasf
