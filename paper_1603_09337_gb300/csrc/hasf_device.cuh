// hasf_device.cuh -- device code shared by the HASF kernels (sm_103a).
//
// One job = one binary image.  Its state lives in three bit-packed planes
// (32 pixels per 32-bit word):
//   S     the current set (X, then Y, Z, ... as the operators run);
//   F     a snapshot of S taken when an operator starts: its distance map
//         (to the complement of F for a thinning, to F for a thickening) is
//         the operator's priority, computed once on its input (Sec. 2);
//   cand  the points currently allowed to change (priority <= current level).
// Resident mode keeps the three planes of one image in shared memory of one
// CTA; gang mode keeps them in global memory (L2) for images too large for
// that, and a gang of co-resident CTAs shares the image, meeting at a
// global-memory barrier after every sweep.
//
// Distances appear only through their sublevel sets.  A point p has priority
// <= l iff some feature point q lies within squared distance l, i.e. iff q - p
// is a lattice vector v with |v|^2 <= l.  The kernel walks the levels l that
// are sums of two squares in increasing order and, at each, ORs the feature
// plane shifted by the vectors with |v|^2 = l: that adds exactly the points of
// priority l.  This is the clamped exact EDT of Sec. 4.1 (column distance g,
// then min over columns of dx^2 + g^2) evaluated as thresholds: values above
// r^2 are never needed, because every candidate point of every operator call
// of HC_r / HF_r has priority <= r^2 (the rest lies in the operator's
// constraint set).  The masks eps_r / delta_r of eqs. (i)-(ii) are therefore
// implied by the level bound r^2 and need no plane of their own.
//
// Simple points (Sec. 2: T = 1 and Tbar = 1) are tested 32 at a time: the
// eight neighbour planes of a word come from funnel shifts of the 3 x 3 words
// around it, and the test is the crossing count
//   sum over the 4-neighbours k in {E, N, W, S} of [x_k = 0 and (x_{k+1} or x_{k+2}) = 1]
// (cyclic neighbour order E, NE, N, NW, W, SW, S, SE) being exactly 1; for
// (4,8) adjacency the same count on the complemented neighbours.  The tests
// check this against the flood-fill definition on all 256 codes.
//
// Sweep order: for each level, rounds of the four subfields (x mod 2, y mod 2)
// = (0,0), (1,0), (0,1), (1,1) until a round changes nothing.  Points of one
// subfield are never 8-adjacent, so updating a whole subfield at once equals
// visiting it in raster order.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "hasf.h"
#include "hasf_internal.h"

namespace hasf {


struct LevelTable {
  uint16_t value[kMaxLevels];      // sums of two squares, increasing
  uint16_t start[kMaxLevels + 1];  // vectors of level i: off[start[i] .. start[i+1])
  uint16_t nlev[kMaxR + 1];        // number of levels <= r^2
  int8_t off[kMaxOffsets][2];      // (dx, dy)
};

// Every translation unit that reads the level table has its own copy in
// constant memory; upload_level_table fills all of them.
static __constant__ LevelTable c_lv;

// ---------------------------------------------------------------------------
// Memory / synchronisation policies.
// ---------------------------------------------------------------------------

struct SmemMode {
  static __device__ __forceinline__ uint32_t ld(const uint32_t* p) { return *p; }
  static __device__ __forceinline__ void st(uint32_t* p, uint32_t v) { *p = v; }
  static __device__ __forceinline__ void atomic_or(uint32_t* p, uint32_t v) { atomicOr(p, v); }
  __device__ __forceinline__ void sync() { __syncthreads(); }
  __device__ __forceinline__ int sync_or(int v) { return __syncthreads_or(v); }
  __device__ __forceinline__ bool failed() const { return false; }
};

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Gang barrier on two 64-bit counters at sync[4..5] and sync[6..7] (zeroed
// before the launch), barrier e using counter e & 1.  A CTA arrives by adding
// 1 + (its OR bit << 32) and waits until the low half reaches the arrivals
// that barrier completes; the high half then says how many CTAs had the bit
// set, and the OR is whether it grew since the last barrier on that counter.
// No CTA can arrive on a counter again before every CTA has left the barrier
// that used it, so the value a CTA reads after the wait is that barrier's
// final value.  Every wait is bounded by a deadline (4 s unless the job sets
// another); a CTA that gives up marks the gang failed and leaves the job.
struct GangMode {
  unsigned* sync_words;
  int nctas;
  // shared, 8-byte aligned: [0] broadcast of the barrier result, [2..3] the
  // wait limit in ns (thread 0 reads it only while it waits)
  int* flag_smem;
  int dead;
  unsigned epoch;        // barriers passed (thread 0's copy is the one used)
  unsigned hi0, hi1;     // high half after the last barrier on each counter

  static __device__ __forceinline__ uint32_t ld(const uint32_t* p) { return __ldcg(p); }
  static __device__ __forceinline__ void st(uint32_t* p, uint32_t v) { __stcg(p, v); }
  static __device__ __forceinline__ void atomic_or(uint32_t* p, uint32_t v) { atomicOr(p, v); }

  __device__ __forceinline__ void init(unsigned* words, int n, int* flag, int deadline_ms) {
    sync_words = words;
    nctas = n;
    flag_smem = flag;
    dead = 0;
    epoch = 0;
    hi0 = hi1 = 0;
    if (threadIdx.x == 0)
      *reinterpret_cast<unsigned long long*>(flag + 2) =
          (unsigned long long)(deadline_ms > 0 ? deadline_ms : 4000) * 1000000ull;
  }

  __device__ int barrier(int v) {
    const int any = __syncthreads_or(v);
    if (threadIdx.x == 0) {
      const unsigned par = epoch & 1u;
      unsigned long long* ctr = reinterpret_cast<unsigned long long*>(sync_words + 4) + par;
      const unsigned target = (epoch / 2u + 1u) * (unsigned)nctas;
      __threadfence();
      atomicAdd(ctr, 1ull | ((unsigned long long)(any != 0) << 32));
      unsigned long long c = *(volatile unsigned long long*)ctr;
      int res = 1;
      if ((unsigned)c < target) {
        const unsigned long long t0 = global_ns();
        unsigned spins = 0;
        do {
          __nanosleep(32);
          c = *(volatile unsigned long long*)ctr;
          if ((unsigned)c >= target) break;
          if ((++spins & 255u) == 0u &&
              global_ns() - t0 > *reinterpret_cast<const unsigned long long*>(flag_smem + 2)) {
            res = 0;
            break;
          }
        } while (true);
      }
      __threadfence();
      const unsigned hi = (unsigned)(c >> 32);
      *flag_smem = res ? (int)(hi != (par ? hi1 : hi0)) : -1;
      if (par) hi1 = hi;
      else hi0 = hi;
      ++epoch;
    }
    __syncthreads();
    const int r = *flag_smem;
    __syncthreads();
    if (r < 0) dead = 1;
    return r > 0;
  }
  __device__ __forceinline__ void sync() { barrier(0); }
  __device__ __forceinline__ int sync_or(int v) { return barrier(v); }
  __device__ __forceinline__ bool failed() const { return dead != 0; }
};

// Fault injection for tests of the failure path: with the job's fault option
// set, CTA 0 of a gang of two or more leaves its job before its first barrier,
// as a CTA that died would; it still counts itself done, so that a served
// job is reported.  The others' bounded waits run out and the job reports
// DEV_TIMEOUT, with no device fault.
__device__ __forceinline__ bool gang_fault_leaves(int fault_skip, int gang, int rank) {
  return fault_skip > 0 && gang > 1 && rank == 0;
}

// ---------------------------------------------------------------------------
// Per-job context.
// ---------------------------------------------------------------------------

// Thread-to-word walk over a set of rows (every row, or every other row).
// A warp covers 32 consecutive words of one row when rows have more than 32
// words; otherwise it splits into g = 32 / L groups of L lanes (L = the power
// of two >= words per row), group k taking the row k * delta (set indices)
// below group 0.  delta makes the groups' addresses differ by L words modulo
// 32 (the row pitch is odd, so it has an inverse modulo 32), so that the
// groups hit disjoint shared-memory banks.  Rows are visited in tuples of g;
// tuple t is block t / delta, offset t % delta; warps take tuples round robin.
struct Walk {
  int delta;   // group stride in row-set indices
  int block;   // rows per block (g * delta)
  int b0, m0;  // this warp's first tuple
  int db, dm;  // tuple advance per step (nwarps tuples)
};

template <class Mode>
struct Ctx {
  Mode m;
  uint32_t* S;
  uint32_t* F;
  uint32_t* cand;
  uint32_t* dirty;    // 2 planes of h * dwpr words
  int w, h, wpr, P, dwpr;
  uint32_t lastmask;  // valid bits of the last word of each row
  int gtid, gthreads; // thread index within the job, threads on the job
  int wid, nwarps;    // warp index within the job, warps on the job
  int L, grp, lj, nchunks;
  Walk walk1, walk2;  // every row / every other row
  int cap;
  unsigned n_tests, n_ring;          // per-thread work counters
  unsigned n_passes, n_levels, n_rounds;
  __device__ __forceinline__ int idx(int y, int j) const { return (y + 1) * P + j; }
  __device__ __forceinline__ uint32_t rowmask(int j) const {
    return j == wpr - 1 ? lastmask : 0xFFFFFFFFu;
  }
};

__device__ __forceinline__ void walk_init(Walk& wk, int step, int L, int g, int P, int wid,
                                          int nwarps) {
  if (g == 1) {
    wk.delta = 1;
  } else {
    int pinv = 1;
    while (((pinv * P) & 31) != 1) pinv += 2;  // P is odd: an inverse exists
    int d = (L * pinv) & 31;
    if (step == 2 && (d & 1) == 0) d >>= 1;
    wk.delta = d > 0 ? d : 1;
  }
  wk.block = g * wk.delta;
  wk.b0 = wid / wk.delta;
  wk.m0 = wid % wk.delta;
  wk.db = nwarps / wk.delta;
  wk.dm = nwarps % wk.delta;
}

// Three-input logic as one instruction: LUT is the truth table evaluated on
// a = 0xF0, b = 0xCC, c = 0xAA.
template <unsigned LUT>
__device__ __forceinline__ uint32_t lop3(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("lop3.b32 %0, %1, %2, %3, %4;" : "=r"(d) : "r"(a), "r"(b), "r"(c), "n"(LUT));
  return d;
}

// Simple-point test of the 32 pixels of the word `c` given the 3 x 3 words
// around it.  Bit b of the result is 1 iff pixel b is simple (removable when
// in the set, addable when not).
template <int CONN>
__device__ __forceinline__ uint32_t simple_bits(uint32_t nw, uint32_t n, uint32_t ne,
                                                uint32_t wv, uint32_t c, uint32_t e,
                                                uint32_t sw, uint32_t s, uint32_t se) {
  uint32_t x0 = __funnelshift_r(c, e, 1);   // E
  uint32_t x1 = __funnelshift_r(n, ne, 1);  // NE
  uint32_t x2 = n;                          // N
  uint32_t x3 = __funnelshift_l(nw, n, 1);  // NW
  uint32_t x4 = __funnelshift_l(wv, c, 1);  // W
  uint32_t x5 = __funnelshift_l(sw, s, 1);  // SW
  uint32_t x6 = s;                          // S
  uint32_t x7 = __funnelshift_r(s, se, 1);  // SE
  if (CONN == 4) {
    x0 = ~x0; x1 = ~x1; x2 = ~x2; x3 = ~x3;
    x4 = ~x4; x5 = ~x5; x6 = ~x6; x7 = ~x7;
  }
  const uint32_t a = ~x0 & (x1 | x2);
  const uint32_t b = ~x2 & (x3 | x4);
  const uint32_t cc = ~x4 & (x5 | x6);
  const uint32_t d = ~x6 & (x7 | x0);
  // exactly one of the four terms: d ? none of a, b, cc : exactly one of a, b, cc
  return lop3<0x3Au>(d, lop3<0xFEu>(a, b, cc), lop3<0x16u>(a, b, cc));
}

// Word whose bit b is G(32 j + b + dx, y2), where G = F xor inv inside the
// box and outv outside it.  A thinning reads the complement of its input with
// the outside as feature (inv = outv = ~0), a thickening its input with an
// empty outside (inv = outv = 0).
template <class Mode>
__device__ __forceinline__ uint32_t fshift(const Ctx<Mode>& k, const uint32_t* Fp, int y2, int j,
                                           int dx, uint32_t inv, uint32_t outv) {
  if (y2 < 0 || y2 >= k.h) return outv;
  const int j0 = j + (dx >> 5);
  const int sh = dx & 31;
  const uint32_t* row = Fp + k.idx(y2, 0);
  uint32_t lo = (j0 >= 0 && j0 < k.wpr) ? (Mode::ld(row + j0) ^ inv) : outv;
  if (sh == 0) return lo;
  uint32_t hi = (j0 + 1 >= 0 && j0 + 1 < k.wpr) ? (Mode::ld(row + j0 + 1) ^ inv) : outv;
  return __funnelshift_r(lo, hi, sh);
}

// Activate the points of priority level li: cand |= allowed & ring_li(F).
// Returns (to every thread) whether any point was activated.  Each thread
// walks its own words with no warp collective in the loop, so that lanes
// drift apart and the irregular ring loops of different words share warp
// instructions.
template <class Mode>
__device__ int level_update(Ctx<Mode>& k, int li, bool thin, const uint32_t* pos,
                            const uint32_t* neg) {
  const int o0 = c_lv.start[li], o1 = c_lv.start[li + 1];
  const uint32_t cm = thin ? 0xFFFFFFFFu : 0u;
  int act = 0;
  const int wpr = k.wpr;
  const int total = k.h * wpr;
  int y = k.gtid / wpr, j = k.gtid - y * wpr;
  const int dy = k.gthreads / wpr, dj = k.gthreads - dy * wpr;
  for (int t = k.gtid; t < total; t += k.gthreads) {
    const int yy = y, jj = j;
    y += dy;
    j += dj;
    if (j >= wpr) {
      j -= wpr;
      ++y;
    }
    const int id = k.idx(yy, jj);
    const uint32_t s = Mode::ld(k.S + id);
    const uint32_t cd = Mode::ld(k.cand + id);
    uint32_t pend = (thin ? s : (~s & k.rowmask(jj))) & ~cd;
    if (!pend) continue;
    if (pos) pend &= Mode::ld(pos + t);
    if (neg) pend &= ~Mode::ld(neg + t);
    if (!pend) continue;
    uint32_t ring = 0;
    for (int o = o0; o < o1; ++o) {
      ring |= fshift(k, k.F, yy + c_lv.off[o][1], jj, c_lv.off[o][0], cm, cm);
      ++k.n_ring;
      if (!(pend & ~ring)) break;
    }
    const uint32_t add = pend & ring;
    if (add) {
      Mode::st(k.cand + id, cd | add);
      act = 1;
    }
  }
  return k.m.sync_or(act);
}

// Test the padded-plane word `id` in the subfield with column mask pm and
// change its simple candidates.
template <class Mode, int CONN>
__device__ __forceinline__ void test_word(Ctx<Mode>& k, int id, uint32_t pm, bool thin,
                                          int& any) {
  const int P = k.P;
  uint32_t* S = k.S;
  const uint32_t cw = Mode::ld(k.cand + id);
  ++k.n_tests;
  const uint32_t ctr = Mode::ld(S + id);
  const uint32_t sm = simple_bits<CONN>(
      Mode::ld(S + id - P - 1), Mode::ld(S + id - P), Mode::ld(S + id - P + 1),
      Mode::ld(S + id - 1), ctr, Mode::ld(S + id + 1),
      Mode::ld(S + id + P - 1), Mode::ld(S + id + P), Mode::ld(S + id + P + 1));
  const uint32_t chg = cw & pm & sm;
  if (chg) {
    Mode::st(S + id, thin ? (ctr & ~chg) : (ctr | chg));
    Mode::st(k.cand + id, cw & ~chg);
    any = 1;
  }
}

// One subfield pass: change every candidate of the subfield that is simple.
// Each lane scans one word per step (a row of this pass's parity); a ballot
// compacts the words holding candidates of the subfield into a per-warp
// queue (two registers per lane: positions lane and 32 + lane), and the 3 x 3
// test runs on full batches of 32 queued words, so that its lanes all do
// useful work.  Points of one subfield are never 8-adjacent: the order in
// which words are tested does not matter.
template <class Mode, int CONN>
__device__ __forceinline__ int sweep_subfield(Ctx<Mode>& k, int sub, bool thin) {
  const int sy = sub >> 1;
  const uint32_t pm = (sub & 1) ? 0xAAAAAAAAu : 0x55555555u;
  const int nrows = (k.h - sy + 1) >> 1;
  const int wpr = k.wpr;
  const int total = nrows * wpr;
  const int lane = threadIdx.x & 31;
  int any = 0;
  int q0 = 0, q1 = 0;  // queued word indices
  int qn = 0;          // queue length (warp-uniform)
  // word t of this pass = parity row t / wpr, word t % wpr; warps take 32
  // consecutive words per step
  const int stride = k.nwarps * 32;
  int t = k.wid * 32 + lane;
  int i = t / wpr, j = t - i * wpr;
  const int di = stride / wpr, dj = stride - di * wpr;
  const int P2 = 2 * k.P;
  for (int t0 = k.wid * 32; t0 < total; t0 += stride) {   // warp-uniform loop
    int id = -1;
    if (t < total) {
      const int w = k.idx(sy + 2 * i, j);
      if (Mode::ld(k.cand + w) & pm) id = w;
    }
    t += stride;
    i += di;
    j += dj;
    if (j >= wpr) {
      j -= wpr;
      ++i;
    }
    const unsigned bal = __ballot_sync(0xFFFFFFFFu, id >= 0);
    if (!bal) continue;
    const int nnew = __popc(bal);
    const int p0 = lane - qn, p1 = lane + 32 - qn;
    const bool take0 = p0 >= 0 && p0 < nnew, take1 = p1 >= 0 && p1 < nnew;
    const int v0 = __shfl_sync(0xFFFFFFFFu, id, take0 ? __fns(bal, 0, p0 + 1) : 0);
    const int v1 = __shfl_sync(0xFFFFFFFFu, id, take1 ? __fns(bal, 0, p1 + 1) : 0);
    if (take0) q0 = v0;
    if (take1) q1 = v1;
    qn += nnew;
    if (qn >= 32) {
      test_word<Mode, CONN>(k, q0, pm, thin, any);
      q0 = q1;
      qn -= 32;
    }
  }
  (void)P2;
  if (lane < qn) test_word<Mode, CONN>(k, q0, pm, thin, any);
  return any;
}

// Rounds at one level until a round changes nothing.  False on the cap.
template <class Mode, int CONN>
__device__ bool run_level(Ctx<Mode>& k, bool thin) {
  for (int round = 0;; ++round) {
    if (round >= k.cap) return false;
    ++k.n_rounds;
    k.n_passes += 4;
    int any = 0;
    for (int sub = 0; sub < 4; ++sub) {
      any |= sweep_subfield<Mode, CONN>(k, sub, thin);
      if (sub < 3) k.m.sync();
    }
    if (!k.m.sync_or(any)) return !k.m.failed();
    if (k.m.failed()) return false;
  }
}

// One constrained thinning (thin = true, H) or thickening (*H) of S at
// radius r.  Allowed points: thin -> S minus neg; thick -> (complement of S)
// cap pos minus neg (pos / neg are unpadded global planes, may be null).
template <class Mode, int CONN>
__device__ bool run_operator(Ctx<Mode>& k, int r, bool thin, const uint32_t* pos,
                             const uint32_t* neg) {
  const int total = k.h * k.wpr;
  for (int t = k.gtid; t < total; t += k.gthreads) {
    const int y = t / k.wpr, j = t - y * k.wpr;
    const int id = k.idx(y, j);
    Mode::st(k.F + id, Mode::ld(k.S + id));
    Mode::st(k.cand + id, 0u);
  }
  k.m.sync();
  const int nlev = c_lv.nlev[r];
  for (int li = 0; li < nlev; ++li) {
    const int act = level_update(k, li, thin, pos, neg);
    if (k.m.failed()) return false;
    if (!act) continue;
    ++k.n_levels;
    if (!run_level<Mode, CONN>(k, thin)) return false;
  }
  return true;
}

template <class Mode>
__device__ void snapshot(Ctx<Mode>& k, uint32_t* g0) {
  const int total = k.h * k.wpr;
  for (int t = k.gtid; t < total; t += k.gthreads) {
    const int y = t / k.wpr, j = t - y * k.wpr;
    Mode::st(g0 + t, Mode::ld(k.S + k.idx(y, j)));
  }
  k.m.sync();
}

// Zero the three padded planes, then pack the input (and C, D) into them.
template <class Mode>
__device__ void load_job(Ctx<Mode>& k, const Job& jb, uint32_t* planes_base) {
  const int nw = 3 * jb.plane_words + dirty_words(jb.w, jb.h);
  for (int t = k.gtid; t < nw; t += k.gthreads) Mode::st(planes_base + t, 0u);
  k.m.sync();
  const int lane = threadIdx.x & 31;
  const int gwarp = k.gtid >> 5, nwarps = k.gthreads >> 5;
  const int total = k.h * k.wpr;
  const bool cx = jb.op == OP_HASF || jb.op == OP_HC;  // C is taken as C cap X
  for (int it = gwarp; it < total; it += nwarps) {
    const int y = it / k.wpr, j = it - y * k.wpr;
    const int x = (j << 5) + lane;
    const bool inb = x < k.w;
    const size_t off = (size_t)y * jb.pitch + x;
    const uint32_t xs = __ballot_sync(0xFFFFFFFFu, inb && jb.in[off] != 0);
    uint32_t cs = 0, ds = 0;
    if (jb.cp) cs = __ballot_sync(0xFFFFFFFFu, inb && jb.C != nullptr && jb.C[off] != 0);
    if (jb.dp) ds = __ballot_sync(0xFFFFFFFFu, inb && jb.D != nullptr && jb.D[off] != 0);
    if (lane == 0) {
      Mode::st(k.S + k.idx(y, j), xs);
      if (jb.cp) Mode::st(jb.cp + it, cx ? (cs & xs) : cs);
      if (jb.dp) Mode::st(jb.dp + it, ds & ~xs);
    }
  }
  k.m.sync();
}

template <class Mode>
__device__ void store_job(Ctx<Mode>& k, const Job& jb) {
  const int lane = threadIdx.x & 31;
  const int gwarp = k.gtid >> 5, nwarps = k.gthreads >> 5;
  const int total = k.h * k.wpr;
  for (int it = gwarp; it < total; it += nwarps) {
    const int y = it / k.wpr, j = it - y * k.wpr;
    const uint32_t s = Mode::ld(k.S + k.idx(y, j));
    const int x = (j << 5) + lane;
    if (x < k.w) jb.out[(size_t)y * jb.pitch + x] = (uint8_t)((s >> lane) & 1u);
  }
}

// HC_r: Y = H(X, eps_r(X) cup C), then *H(Y, delta_r(Y) cap X) (eq. (i)).
// HF_r: Z = *H(X, delta_r(X) minus D), then H(Z, eps_r(Z) cup X) (eq. (ii)).
template <class Mode, int CONN>
__device__ bool run_hc(Ctx<Mode>& k, const Job& jb, int r) {
  snapshot(k, jb.g0);
  if (!run_operator<Mode, CONN>(k, r, true, nullptr, jb.cp)) return false;
  return run_operator<Mode, CONN>(k, r, false, jb.g0, nullptr);
}
template <class Mode, int CONN>
__device__ bool run_hf(Ctx<Mode>& k, const Job& jb, int r) {
  snapshot(k, jb.g0);
  if (!run_operator<Mode, CONN>(k, r, false, nullptr, jb.dp)) return false;
  return run_operator<Mode, CONN>(k, r, true, nullptr, jb.g0);
}

// End of a job on one of its CTAs: the last of the job's CTAs to get here
// publishes the job's status to the host (1 + status), after a system-scope
// fence that orders the job's output writes before it.
__device__ __forceinline__ void job_done(const Job& jb, int gang) {
  if (!jb.notify) return;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence_system();
    const unsigned c = atomicAdd(jb.sync + 3, 1u);
    if (c + 1u == (unsigned)gang) {
      const int st = atomicAdd(jb.status, 0);
      __threadfence_system();
      *(volatile int*)jb.notify = 1 + st;
    }
  }
}

// Whether the current set differs anywhere from the plane g (h * wpr words);
// the same answer on every thread of the job.
template <class Mode>
__device__ int differs(Ctx<Mode>& k, const uint32_t* g) {
  const int total = k.h * k.wpr;
  int d = 0;
  for (int t = k.gtid; t < total; t += k.gthreads) {
    const int y = t / k.wpr, j = t - y * k.wpr;
    d |= Mode::ld(k.S + k.idx(y, j)) != Mode::ld(g + t);
  }
  return k.m.sync_or(d);
}

template <class Mode, int CONN>
__device__ void run_job(Ctx<Mode>& k, const Job& jb, uint32_t* planes_base) {
  load_job(k, jb, planes_base);
  bool ok = true;
  switch (jb.op) {
    case OP_HASF: {
      // run to stability: stop after the first step that changes nothing
      bool fixed = false;
      for (int r = jb.r_lo; ok && r <= jb.r_hi; ++r) {
        if (jb.stable) snapshot(k, jb.g1);
        ok = run_hc<Mode, CONN>(k, jb, r);
        if (ok) ok = run_hf<Mode, CONN>(k, jb, r);
        if (ok && jb.stable && !differs(k, jb.g1)) {
          fixed = true;
          break;
        }
      }
      if (ok && jb.stable && !fixed && threadIdx.x == 0) atomicMax(jb.status, (int)DEV_UNSTABLE);
      break;
    }
    case OP_THIN: ok = run_operator<Mode, CONN>(k, jb.r_hi, true, nullptr, jb.cp); break;
    case OP_THICK: ok = run_operator<Mode, CONN>(k, jb.r_hi, false, jb.cp, nullptr); break;
    case OP_HC: ok = run_hc<Mode, CONN>(k, jb, jb.r_hi); break;
    case OP_HF: ok = run_hf<Mode, CONN>(k, jb, jb.r_hi); break;
    default: ok = false;
  }
  if (ok) {
    store_job(k, jb);
  } else if (threadIdx.x == 0) {
    atomicMax(jb.status, (int)DEV_TIMEOUT);
  }
  job_done(jb, jb.gang);
  if (jb.stats) {
    unsigned long long t = k.n_tests, r = k.n_ring;
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_down_sync(0xFFFFFFFFu, t, o);
      r += __shfl_down_sync(0xFFFFFFFFu, r, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(jb.stats + STAT_WORD_TESTS, t);
      atomicAdd(jb.stats + STAT_RING_EVALS, r);
    }
    if (k.gtid == 0) {
      atomicAdd(jb.stats + STAT_PASSES, (unsigned long long)k.n_passes);
      atomicAdd(jb.stats + STAT_LEVELS, (unsigned long long)k.n_levels);
      atomicAdd(jb.stats + STAT_ROUNDS, (unsigned long long)k.n_rounds);
    }
  }
}

template <class Mode>
__device__ __forceinline__ void init_ctx(Ctx<Mode>& k, const Job& jb, uint32_t* base, int gtid,
                                         int gthreads) {
  k.w = jb.w;
  k.h = jb.h;
  k.wpr = jb.wpr;
  k.P = row_pitch(jb.w);
  k.dwpr = (jb.wpr + 31) >> 5;
  const int rem = jb.w & 31;
  k.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
  k.S = base + 1;
  k.F = base + jb.plane_words + 1;
  k.cand = base + 2 * jb.plane_words + 1;
  k.dirty = base + 3 * jb.plane_words;
  k.gtid = gtid;
  k.gthreads = gthreads;
  k.wid = gtid >> 5;
  k.nwarps = gthreads >> 5;
  int L = 1;
  while (L < jb.wpr && L < 32) L <<= 1;
  k.L = L;
  const int lane = threadIdx.x & 31;
  k.grp = lane / L;
  k.lj = lane % L;
  k.nchunks = jb.wpr > 32 ? (jb.wpr + 31) >> 5 : 1;
  walk_init(k.walk1, 1, L, 32 / L, k.P, k.wid, k.nwarps);
  walk_init(k.walk2, 2, L, 32 / L, k.P, k.wid, k.nwarps);
  k.cap = jb.cap;
  k.n_tests = k.n_ring = k.n_passes = k.n_levels = k.n_rounds = 0;
}

}  // namespace hasf
