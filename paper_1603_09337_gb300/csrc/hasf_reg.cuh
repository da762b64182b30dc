// hasf_reg.cuh -- register-resident fused HASF kernel for images up to
// 512 x 512 (device code; included by hasf_reg.cu and hasf_tiled.cu after hasf_device.cuh).
//
// The current set S lives in registers (the candidates, read once per test,
// in shared memory).  With 16 words (512 pixels) per row,
// thread (warp w, lane l) owns word column j = l & 15 of a 16-row strip:
// lanes 0-15 hold rows [32 w, 32 w + 16), lanes 16-31 the 16 rows below, so a
// CTA of 512 threads covers 512 rows.  A 3 x 3 neighbourhood then comes from
// the thread's own registers (rows above and below), the bit next to the word
// in the words left and right (exchanged as one pack of 16 rows' edge bits per
// half-round), a warp shuffle for the row across the boundary of the two
// strips of a warp, and a small shared-memory exchange of each warp's first
// and last row.
//
// A subfield pass tests the words of its rows (8 per thread) from registers.
// The two subfields of one row parity, (0, sy) and (1, sy), read only rows of
// the other parity across rows, so they run back to back without a CTA
// barrier (fused row by row, see reg_half): a round takes two barriers (after
// the even rows, after the odd rows), the second one OR-reducing the round's
// change flag.
//
// The operator's priority map (snapshot F) stays a padded plane in shared
// memory, read by the level updates exactly as in the generic kernel; the
// movable mask M = (points the operator may change, ignoring levels) and the
// candidates are two more planes there, with a row pitch of 17 words so that
// the two half-warps (16 rows apart) use disjoint banks.
#pragma once

namespace hasf {

constexpr int kRegW = 16;   // words per row handled (512 pixels)
constexpr int kRegR = 16;   // rows per thread
constexpr int kRegRows = kRegR * 2 * (kThreads / 32);  // 512 rows
constexpr int kRegPitch = kRegW + 1;                    // M and cand row pitch

constexpr int kRegPadR = 31;  // zero rows above and below the F plane (rmax <= 31)

__host__ __device__ inline bool reg_kernel_fits(int w, int h, int rmax) {
  return w <= 32 * kRegW && h <= kRegRows && rmax >= 1 && rmax <= kRegPadR;
}
// F plane of the register kernel: rows -kRegPadR .. h + kRegPadR - 1, row pitch
// row_pitch(w) (the last word of every row is zero), plus one leading word.
__host__ __device__ inline int reg_f_words(int w, int h) {
  return (((h + 2 * kRegPadR) * row_pitch(w) + 2) + 3) & ~3;
}
// Shared memory: the padded F plane, then M and cand for all kRegRows rows
// (threads whose rows lie below the image read them: zero), then the
// first/last-row exchange of each warp.
constexpr int kRegPlane = kRegRows * kRegPitch;
constexpr int kRegXchg = 2 * (kThreads / 32) * kRegW;
__host__ __device__ inline int reg_smem_words(int w, int h) {
  return reg_f_words(w, h) + 2 * kRegPlane + kRegXchg;
}
inline size_t reg_smem_bytes(int w, int h) { return (size_t)reg_smem_words(w, h) * 4; }

// Work counters of the CTA's current job (see StatIndex), in shared memory so
// that they hold no registers: thread 0 or one lane per warp adds to them.
static __shared__ unsigned s_reg_stats[STAT_COUNT];

struct RegCtx {
  Ctx<SmemMode> g;      // image geometry; g.F = F at (row 0, word 0)
  uint32_t* M;          // kRegRows rows x kRegPitch words
  uint32_t* cand;       // kRegRows rows x kRegPitch words
  uint32_t* top;        // [warp][kRegW]: first row of each warp
  uint32_t* bot;        // [warp][kRegW]: last row of each warp
  int warp, half, j, s0;  // s0 = first row of this thread's strip
  bool jin;             // j < words per row of the image
};

// Simple-point test of 32 pixels from their eight neighbour planes (bit b of
// x_k = neighbour k of pixel b, in the order E, NE, N, NW, W, SW, S, SE), by
// the crossing count of Sec. 2's T = Tbar = 1: with the four terms
// [x_k = 0 and (x_{k+1} or x_{k+2}) = 1] for k = E, N, W, S (cyclic order),
// exactly one of them holds.  (4,8) adjacency takes the complemented planes,
// folded into the terms' truth table.  Seven three-input logic instructions:
// four terms, then "exactly one of four" as d ? none of a, b, c : exactly one
// of a, b, c.
template <int CONN>
__device__ __forceinline__ uint32_t simple_planes(uint32_t x0, uint32_t x1, uint32_t x2,
                                                  uint32_t x3, uint32_t x4, uint32_t x5,
                                                  uint32_t x6, uint32_t x7) {
  constexpr unsigned T = CONN == 8 ? 0x0Eu : 0x70u;  // ~a & (b | c), or a & ~(b & c)
  const uint32_t a = lop3<T>(x0, x1, x2), b = lop3<T>(x2, x3, x4);
  const uint32_t c = lop3<T>(x4, x5, x6), d = lop3<T>(x6, x7, x0);
  // exactly one of a, b, c, d = d ? none of a, b, c : exactly one of a, b, c
  return lop3<0x3Au>(d, lop3<0xFEu>(a, b, c), lop3<0x16u>(a, b, c));
}

// A row next to the thread's strip (the last row of the strip above, or the
// first row of the strip below) with its west and east neighbour planes.
struct EdgeRow {
  uint32_t v, l, r;
};

// The two subfield passes (0, SY) then (1, SY) over this thread's rows of
// parity SY (compile-time).  They are fused row by row: within these two
// passes a row of parity SY reads only itself and the rows of the other
// parity (which do not change), so finishing (0, SY) and (1, SY) on one row
// before the next gives the same result as two full passes.  Four rows of the
// parity (r, r + 2, r + 4, r + 6) are tested together: their work is
// independent, which gives each thread four chains of instructions in flight.
//
// Neighbour planes.  A pixel's west neighbour plane is the row shifted left by
// one with bit 31 of the word to the left coming in at bit 0; the east plane is
// the row shifted right with bit 0 of the word to the right coming in at bit
// 31.  Those cross-word bits come from the packs Wb (bit q = bit 31 of the
// left neighbour's row q) and Eb (bit 16 + q = bit 0 of the right neighbour's
// row q), exchanged once per half.  The rows of the other parity do not change
// in the half: the planes of the five rows around a group of four are made
// once.  An even pixel's cross-word neighbours all lie in the left word (bit
// 31: an odd pixel, unchanged by the first pass); an odd pixel's in the right
// word (bit 0: an even pixel).  So the second test needs one fresh bit per
// row, the right word's updated bit 0: one shuffle of the four rows' bits,
// taken only when the first pass changed a pixel of the group somewhere in
// the warp (else the first test's result holds for the odd pixels too).
// The candidates are stored back unconditionally (a store costs less than
// the test that would skip it).
//
// `need` (warp-uniform, bit q = row q of either strip of the warp) says which
// rows can change at all.  A row whose last test left it stable stays stable
// until a row next to it changes or it gains candidates: after the fused test
// no remaining candidate of the row is simple, except that odd-column changes
// can re-enable even-column candidates of the same row -- then the row stays
// marked.  A change in row r marks rows r - 1 and r + 1 (the strips of a warp
// are stacked, so row 15 and row 0 are neighbours across them).  Marks are
// kept per group of four rows (a superset of the rows that changed; testing a
// stable row changes nothing).  A group without a candidate anywhere in the
// warp is skipped.  `pack` (bits q and 16 + q: bits 31 and 0 of
// row q) is rebuilt for this parity's rows at the end.  Returns non-zero when
// a pixel changed.
template <int CONN, int SY, int G>
__device__ __forceinline__ uint32_t reg_half(RegCtx& k, uint32_t (&S)[kRegR], uint32_t& pack,
                                             uint32_t Wb, uint32_t Eb, const EdgeRow& xr,
                                             uint32_t& need) {
  static_assert(G == 1 || G == 2 || G == 4, "rows per group");
  constexpr uint32_t gm = G == 4 ? 0x55u : (G == 2 ? 0x5u : 0x1u);  // the group's rows
  uint32_t* cr = k.cand + k.s0 * kRegPitch + k.j;
  const uint32_t emask = k.j == kRegW - 1 ? 0u : 0xFFFFFFFFu;
  uint32_t changed = 0;
  uint32_t rowchg = 0;
  uint32_t again = 0;
#pragma unroll
  for (int r = SY; r < kRegR; r += 2 * G) {
    if (!((need >> r) & gm)) continue;   // rows r, r + 2, ..., r + 2 (G - 1), tested together
    uint32_t cw[G], anyc = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      cw[i] = cr[(r + 2 * i) * kRegPitch];
      anyc |= cw[i];
    }
    if (!__any_sync(0xFFFFFFFFu, anyc != 0u)) continue;
    // work counter: the group's rows, both subfields, every lane
    if ((threadIdx.x & 31) == 0) atomicAdd(&s_reg_stats[STAT_WORD_TESTS], 64u * G);
    uint32_t v[G + 1], L[G + 1], R[G + 1];   // rows r - 1, r + 1, ..., r + 2 G - 1
#pragma unroll
    for (int i = 0; i <= G; ++i) {
      const int q = r - 1 + 2 * i;
      if (q < 0 || q >= kRegR) {
        v[i] = xr.v;
        L[i] = xr.l;
        R[i] = xr.r;
      } else {
        v[i] = S[q];
        L[i] = __funnelshift_l(Wb << (31 - q), v[i], 1);
        R[i] = __funnelshift_r(v[i], Eb >> (16 + q), 1);
      }
    }
    uint32_t c[G], wl[G], res[G], c0[G];
    uint32_t any = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int q = r + 2 * i;
      c[i] = S[q];
      wl[i] = Wb << (31 - q);
      res[i] = simple_planes<CONN>(__funnelshift_r(c[i], Eb >> (16 + q), 1), R[i], v[i], L[i],
                                   __funnelshift_l(wl[i], c[i], 1), L[i + 1], v[i + 1], R[i + 1]);
      c0[i] = res[i] & cw[i] & 0x55555555u;
      any |= c0[i];
    }
    if (__any_sync(0xFFFFFFFFu, any != 0u)) {
      // odd pixels: the right word's bit 0 after its even-column pass, one
      // shuffle per row
#pragma unroll
      for (int i = 0; i < G; ++i) {
        c[i] ^= c0[i];
        const uint32_t e = __shfl_down_sync(0xFFFFFFFFu, c[i], 1, 16) & emask;
        res[i] = simple_planes<CONN>(__funnelshift_r(c[i], e, 1), R[i], v[i], L[i],
                                     __funnelshift_l(wl[i], c[i], 1), L[i + 1], v[i + 1],
                                     R[i + 1]);
      }
      rowchg |= gm << r;
      changed = 1u;
    }
    uint32_t any1 = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) {
      const int q = r + 2 * i;
      const uint32_t c1 = res[i] & cw[i] & 0xAAAAAAAAu;
      S[q] = c[i] ^ c1;
      cr[q * kRegPitch] = cw[i] ^ c0[i] ^ c1;
      any1 |= c1;
    }
    if (__any_sync(0xFFFFFFFFu, any1 != 0u)) {
      rowchg |= gm << r;
      again |= gm << r;
      changed = 1u;
    }
  }
  // bits 31 and 0 of this parity's rows, rebuilt into the pack
  {
    uint32_t hb = 0, lb = 0;
#pragma unroll
    for (int q = kRegR - 2 + SY; q >= 0; q -= 2) hb = __funnelshift_l(S[q], hb, 2);
#pragma unroll
    for (int q = SY; q < kRegR; q += 2) lb = __funnelshift_r(lb, S[q], 2);
    if (SY == 0) hb >>= 1;
    else lb <<= 1;
    const uint32_t keep = SY ? 0x55555555u : 0xAAAAAAAAu;
    pack = (pack & keep) | (hb & ~keep & 0xFFFFu) | (lb & ~keep & 0xFFFF0000u);
  }
  // rows of this parity were tested: keep only those an odd-column change
  // may have re-enabled, then mark the neighbours of the changed rows
  need &= ~(SY ? 0xAAAAu : 0x5555u);
  need |= again;
  uint32_t nb = (rowchg << 1) | (rowchg >> 1);
  if (rowchg & 0x8000u) nb |= 1u;       // row 15 of strip A is above row 0 of strip B
  if (rowchg & 0x0001u) nb |= 0x8000u;  // and row 0 of strip B below row 15 of strip A
  need |= nb & 0xFFFFu;
  return changed;
}

// Bits 31 (at bit q) and 0 (at bit 16 + q) of the thread's rows q.
__device__ __forceinline__ uint32_t edge_pack(const uint32_t (&S)[kRegR]) {
  uint32_t hb = 0, lb = 0;
#pragma unroll
  for (int q = kRegR - 1; q >= 0; --q) hb = __funnelshift_l(S[q], hb, 1);  // (hb << 1) | bit 31
#pragma unroll
  for (int q = 0; q < kRegR; ++q) lb = __funnelshift_r(lb, S[q], 1);       // (lb >> 1) | bit 0 << 31
  return (hb & 0xFFFFu) | (lb & 0xFFFF0000u);
}

// A row next to the strip with its west / east planes (its neighbours' words
// come from the lanes beside this one, which hold the same row).
__device__ __forceinline__ EdgeRow edge_row(uint32_t v, bool jfirst, bool jlast) {
  uint32_t l = __shfl_up_sync(0xFFFFFFFFu, v, 1, 16);
  uint32_t r = __shfl_down_sync(0xFFFFFFFFu, v, 1, 16);
  if (jfirst) l = 0u;
  if (jlast) r = 0u;
  return EdgeRow{v, __funnelshift_l(l, v, 1), __funnelshift_r(v, r, 1)};
}

// Rounds at one level until a round changes nothing.  False on the cap.
// ab_prev / be_prev: the rows across the warp boundary as last seen.
template <int CONN, int G>
__device__ bool reg_level(RegCtx& k, uint32_t (&S)[kRegR], uint32_t& need, uint32_t& ab_prev,
                          uint32_t& be_prev) {
  const int lane = threadIdx.x & 31;
  const bool jfirst = k.j == 0, jlast = k.j == kRegW - 1;
  uint32_t pack = edge_pack(S);
  for (int round = 0;; ++round) {
    if (round >= k.g.cap) return false;
    if (threadIdx.x == 0) {
      s_reg_stats[STAT_ROUNDS] += 1;
      s_reg_stats[STAT_PASSES] += 4;
    }
    // even rows: row above the strip = last row of the strip above
    uint32_t ab = __shfl_sync(0xFFFFFFFFu, S[kRegR - 1], lane ^ 16);
    if (k.half == 0) ab = k.warp > 0 ? k.bot[(k.warp - 1) * kRegW + k.j] : 0u;
    if (__any_sync(0xFFFFFFFFu, ab != ab_prev)) need |= 1u;
    ab_prev = ab;
    uint32_t Wb = __shfl_up_sync(0xFFFFFFFFu, pack, 1, 16);
    uint32_t Eb = __shfl_down_sync(0xFFFFFFFFu, pack, 1, 16);
    if (jfirst) Wb = 0u;
    if (jlast) Eb = 0u;
    uint32_t ch = reg_half<CONN, 0, G>(k, S, pack, Wb, Eb, edge_row(ab, jfirst, jlast), need);
    if (k.half == 0) k.top[k.warp * kRegW + k.j] = S[0];
    __syncthreads();
    // odd rows: row below the strip = first row of the strip below
    uint32_t be = __shfl_sync(0xFFFFFFFFu, S[0], lane ^ 16);
    if (k.half == 1)
      be = (k.warp + 1) < (int)(blockDim.x >> 5) ? k.top[(k.warp + 1) * kRegW + k.j] : 0u;
    if (__any_sync(0xFFFFFFFFu, be != be_prev)) need |= 0x8000u;
    be_prev = be;
    Wb = __shfl_up_sync(0xFFFFFFFFu, pack, 1, 16);
    Eb = __shfl_down_sync(0xFFFFFFFFu, pack, 1, 16);
    if (jfirst) Wb = 0u;
    if (jlast) Eb = 0u;
    ch |= reg_half<CONN, 1, G>(k, S, pack, Wb, Eb, edge_row(be, jfirst, jlast), need);
    if (k.half == 1) k.bot[k.warp * kRegW + k.j] = S[kRegR - 1];
    if (!__syncthreads_or(ch != 0u)) return true;
  }
}

// Level updates read the feature plane F (the operator's input snapshot)
// shifted by each vector of the level and OR the words: a point reached by a
// vector of squared norm l has priority <= l.  A thinning's feature set is the
// complement of F (outside the box included: the zero padding and the zero
// bits past the width read as feature), so it ANDs F and complements at the
// end.  No bounds checks: the padding covers |dy| <= 31, |dx| <= 32.

// One constrained thinning (thin) or thickening at radius r; the allowed
// points are (thin ? S : complement of S) cap pos minus neg (global planes).
template <int CONN, bool thin, int G>
__device__ bool reg_operator(RegCtx& k, uint32_t (&S)[kRegR], int r,
                             const uint32_t* pos, const uint32_t* neg) {
  Ctx<SmemMode>& g = k.g;
  // snapshot F, the movable mask M, no candidates; rows with movable points
  uint32_t pendrows = 0;
#pragma unroll
  for (int q = 0; q < kRegR; ++q) {
    const int y = k.s0 + q;
    if (y < g.h) {
      uint32_t m = 0;
      if (k.jin) {
        g.F[y * g.P + k.j] = S[q];
        const int t = y * g.wpr + k.j;
        m = g.rowmask(k.j);
        if (pos) m &= pos[t];
        if (neg) m &= ~neg[t];
        if (m & (thin ? S[q] : ~S[q])) pendrows |= 1u << q;
      }
      k.M[y * kRegPitch + k.j] = m;
      k.cand[y * kRegPitch + k.j] = 0u;
    }
  }
  // first and last rows of each warp, for the first passes
  if (k.half == 0) k.top[k.warp * kRegW + k.j] = S[0];
  if (k.half == 1) k.bot[k.warp * kRegW + k.j] = S[kRegR - 1];
  __syncthreads();
  uint32_t need = 0;
  const int lane = threadIdx.x & 31;
  uint32_t ab_prev = __shfl_sync(0xFFFFFFFFu, S[kRegR - 1], lane ^ 16);
  if (k.half == 0) ab_prev = k.warp > 0 ? k.bot[(k.warp - 1) * kRegW + k.j] : 0u;
  uint32_t be_prev = __shfl_sync(0xFFFFFFFFu, S[0], lane ^ 16);
  if (k.half == 1)
    be_prev = (k.warp + 1) < (int)(blockDim.x >> 5) ? k.top[(k.warp + 1) * kRegW + k.j] : 0u;
  const int nlev = c_lv.nlev[r];
  for (int li = 0; li < nlev; ++li) {
    const int o0 = c_lv.start[li], o1 = c_lv.start[li + 1];
    uint32_t newrows = 0;
    unsigned ring = 0;  // shifted feature words read (work counter)
#pragma unroll
    for (int g4 = 0; g4 < kRegR; g4 += 4) {
      if (!((pendrows >> g4) & 0xFu)) continue;
      uint32_t pend[4], acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = g4 + u;
        pend[u] = 0u;
        if ((pendrows >> q) & 1u) {
          const int a = (k.s0 + q) * kRegPitch + k.j;
          pend[u] = k.M[a] & (thin ? S[q] : ~S[q]) & ~k.cand[a];
          if (!pend[u]) pendrows &= ~(1u << q);
        }
        acc[u] = thin ? 0xFFFFFFFFu : 0u;
      }
      if (!(pend[0] | pend[1] | pend[2] | pend[3])) continue;
      // the level's vectors, applied to the four rows at once (independent
      // chains); stop once every pending point of the four rows is reached.
      // The walk is latency-bound: unrolled eight vectors deep, with the stop
      // checked every eight, it keeps eight vectors' reads in flight.
      const uint32_t* base = g.F + (k.s0 + g4) * g.P + k.j;
#pragma unroll 8
      for (int o = o0; o < o1; ++o) {
        const int dx = c_lv.off[o][0], dy = c_lv.off[o][1];
        const uint32_t* p0 = base + dy * g.P + (dx >> 5);
        const int sh = dx & 31;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (pend[u]) {  // rows without pending points may lie past the image
            const uint32_t v = __funnelshift_r(p0[u * g.P], p0[u * g.P + 1], sh);
            acc[u] = thin ? (acc[u] & v) : (acc[u] | v);
          }
        }
        ++ring;
        if (((o - o0) & 7) == 7) {
          uint32_t left = 0;
#pragma unroll
          for (int u = 0; u < 4; ++u) left |= pend[u] & (thin ? acc[u] : ~acc[u]);
          if (!left) break;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const uint32_t add = pend[u] & (thin ? ~acc[u] : acc[u]);
        if (add) {
          const int q = g4 + u;
          const int a = (k.s0 + q) * kRegPitch + k.j;
          k.cand[a] |= add;
          newrows |= 1u << q;
          if (!(pend[u] & ~add)) pendrows &= ~(1u << q);
        }
      }
    }
    need |= __reduce_or_sync(0xFFFFFFFFu, newrows);
    ring = __reduce_add_sync(0xFFFFFFFFu, ring);
    if (lane == 0) atomicAdd(&s_reg_stats[STAT_RING_EVALS], ring);
    if (!__syncthreads_or(newrows != 0u)) continue;
    if (threadIdx.x == 0) s_reg_stats[STAT_LEVELS] += 1;
    if (!reg_level<CONN, G>(k, S, need, ab_prev, be_prev)) return false;
  }
  return true;
}

// 1 bit per byte (non-zero = 1) of n <= 32 bytes at p.
__device__ __forceinline__ uint32_t nibbles(uint32_t x) {
  uint32_t t = (x | (x >> 4)) & 0x0F0F0F0Fu;
  t = (t | (t >> 2)) & 0x03030303u;
  t = (t | (t >> 1)) & 0x01010101u;
  return (t * 0x01020408u) >> 24;  // byte i's bit to bit i
}
__device__ __forceinline__ uint32_t pack_word(const uint8_t* p, int n, bool vec) {
  if (vec && n == 32) {
    const uint4 a = __ldg(reinterpret_cast<const uint4*>(p));
    const uint4 b = __ldg(reinterpret_cast<const uint4*>(p) + 1);
    return nibbles(a.x) | (nibbles(a.y) << 4) | (nibbles(a.z) << 8) | (nibbles(a.w) << 12) |
           (nibbles(b.x) << 16) | (nibbles(b.y) << 20) | (nibbles(b.z) << 24) |
           (nibbles(b.w) << 28);
  }
  uint32_t v = 0;
  for (int i = 0; i < n; ++i) v |= (p[i] != 0 ? 1u : 0u) << i;
  return v;
}

// A job as a sequence of constrained operators.  HC_r (eq. (i)) is a
// thinning that keeps C, then a thickening inside its input g0; HF_r (eq.
// (ii)) a thickening that avoids D, then a thinning that keeps g0.  pos: the
// points that may change must lie in it; neg: they must not.  snap: g0 is
// taken (the current set) before the step.
struct OpStep {
  int r;
  bool thin, snap;
  const uint32_t* pos;
  const uint32_t* neg;
};
__device__ __forceinline__ int op_steps(const Job& jb) {
  switch (jb.op) {
    case OP_HASF: return 4 * (jb.r_hi - jb.r_lo + 1);
    case OP_HC:
    case OP_HF: return 2;
    case OP_THIN:
    case OP_THICK: return 1;
    default: return 0;
  }
}
__device__ __forceinline__ OpStep op_step(const Job& jb, int st) {
  int kind, r = jb.r_hi;  // kind 0/1: HC thin/thick, 2/3: HF thick/thin, 4: thin, 5: thick
  if (jb.op == OP_HASF) {
    kind = st & 3;
    r = jb.r_lo + (st >> 2);
  } else if (jb.op == OP_HC) {
    kind = st;
  } else if (jb.op == OP_HF) {
    kind = 2 + st;
  } else {
    kind = jb.op == OP_THIN ? 4 : 5;
  }
  OpStep s;
  s.r = r;
  s.thin = kind == 0 || kind == 3 || kind == 4;
  s.snap = kind == 0 || kind == 2;
  s.pos = kind == 1 ? jb.g0 : (kind == 5 ? jb.cp : nullptr);
  s.neg = (kind == 0 || kind == 4) ? jb.cp : (kind == 2 ? jb.dp : (kind == 3 ? jb.g0 : nullptr));
  return s;
}

template <int CONN, int G>
__device__ void reg_job(RegCtx& k, const Job& jb, uint32_t* smem) {
  Ctx<SmemMode>& g = k.g;
  uint32_t S[kRegR];
  // zero the shared planes, then read this thread's 16 words straight from
  // the input (32 bytes per word: two 16-byte loads when rows are aligned)
  {
    const int nz = reg_smem_words(jb.w, jb.h);
    for (int t = threadIdx.x; t < nz; t += blockDim.x) smem[t] = 0u;
    const bool vec = ((reinterpret_cast<uintptr_t>(jb.in) | (uintptr_t)jb.pitch |
                       reinterpret_cast<uintptr_t>(jb.C) | reinterpret_cast<uintptr_t>(jb.D)) &
                      15u) == 0;
    const bool cx = jb.op == OP_HASF || jb.op == OP_HC;
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int y = k.s0 + q;
      uint32_t xs = 0;
      if (y < g.h && k.jin) {
        const size_t off = (size_t)y * jb.pitch + (k.j << 5);
        const int n = min(32, g.w - (k.j << 5));
        xs = pack_word(jb.in + off, n, vec);
        const int t = y * g.wpr + k.j;
        if (jb.cp) {
          const uint32_t cs = jb.C ? pack_word(jb.C + off, n, vec) : 0u;
          jb.cp[t] = cx ? (cs & xs) : cs;
        }
        if (jb.dp) jb.dp[t] = (jb.D ? pack_word(jb.D + off, n, vec) : 0u) & ~xs;
      }
      S[q] = xs;
    }
    __syncthreads();
  }
  auto snapshot_g0 = [&]() {
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int y = k.s0 + q;
      if (y < g.h && k.jin) jb.g0[y * g.wpr + k.j] = S[q];
    }
    __syncthreads();
  };
  bool ok = true;
  auto hc = [&](int r) {
    snapshot_g0();
    if (!reg_operator<CONN, true, G>(k, S, r, nullptr, jb.cp)) return false;
    return reg_operator<CONN, false, G>(k, S, r, jb.g0, nullptr);
  };
  auto hf = [&](int r) {
    snapshot_g0();
    if (!reg_operator<CONN, false, G>(k, S, r, nullptr, jb.dp)) return false;
    return reg_operator<CONN, true, G>(k, S, r, nullptr, jb.g0);
  };
  switch (jb.op) {
    case OP_HASF: {
      // run to stability: keep the image before each step in g1 and stop
      // after the first step that leaves it unchanged
      bool fixed = false;
      for (int r = jb.r_lo; ok && r <= jb.r_hi; ++r) {
        if (jb.stable) {
#pragma unroll
          for (int q = 0; q < kRegR; ++q) {
            const int y = k.s0 + q;
            if (y < g.h && k.jin) jb.g1[y * g.wpr + k.j] = S[q];
          }
        }
        ok = hc(r);
        if (ok) ok = hf(r);
        if (ok && jb.stable) {
          int d = 0;
#pragma unroll
          for (int q = 0; q < kRegR; ++q) {
            const int y = k.s0 + q;
            if (y < g.h && k.jin) d |= jb.g1[y * g.wpr + k.j] != S[q];
          }
          if (!__syncthreads_or(d)) {
            fixed = true;
            break;
          }
        }
      }
      if (ok && jb.stable && !fixed && threadIdx.x == 0) atomicMax(jb.status, (int)DEV_UNSTABLE);
      break;
    }
    case OP_THIN: ok = reg_operator<CONN, true, G>(k, S, jb.r_hi, nullptr, jb.cp); break;
    case OP_THICK: ok = reg_operator<CONN, false, G>(k, S, jb.r_hi, jb.cp, nullptr); break;
    case OP_HC: ok = hc(jb.r_hi); break;
    case OP_HF: ok = hf(jb.r_hi); break;
    default: ok = false;
  }
  if (ok) {
    // unpack: 32 bytes per word, vectorised when the rows are 16-byte aligned
    const bool vec = ((reinterpret_cast<uintptr_t>(jb.out) | (uintptr_t)jb.pitch) & 15u) == 0;
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int y = k.s0 + q;
      if (y >= g.h || !k.jin) continue;
      const uint32_t v = S[q];
      uint8_t* o = jb.out + (size_t)y * jb.pitch + (k.j << 5);
      const int n = min(32, g.w - (k.j << 5));
      if (vec && n == 32) {
        uint32_t wds[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const uint32_t nib = (v >> (4 * e)) & 0xFu;
          wds[e] = (nib & 1u) | ((nib & 2u) << 7) | ((nib & 4u) << 14) | ((nib & 8u) << 21);
        }
        reinterpret_cast<uint4*>(o)[0] = make_uint4(wds[0], wds[1], wds[2], wds[3]);
        reinterpret_cast<uint4*>(o)[1] = make_uint4(wds[4], wds[5], wds[6], wds[7]);
      } else {
        for (int b = 0; b < n; ++b) o[b] = (uint8_t)((v >> b) & 1u);
      }
    }
  } else if (threadIdx.x == 0) {
    atomicMax(jb.status, (int)DEV_TIMEOUT);
  }
  job_done(jb, 1);
  if (jb.stats) {
    __syncthreads();
    if (threadIdx.x == 0)
      for (int i = 0; i < STAT_COUNT; ++i)
        atomicAdd(jb.stats + i, (unsigned long long)s_reg_stats[i]);
  }
}

}  // namespace hasf
