// hasf_reg.cuh -- register-resident fused HASF kernel for images up to
// 512 x 512 (included by hasf_kernels.cu, which defines the helpers it uses).
//
// The current set S lives in registers (the candidates, read once per test,
// in shared memory).  With 16 words (512 pixels) per row,
// thread (warp w, lane l) owns word column j = l & 15 of a 16-row strip:
// lanes 0-15 hold rows [32 w, 32 w + 16), lanes 16-31 the 16 rows below, so a
// CTA of 512 threads covers 512 rows.  A 3 x 3 neighbourhood then comes from
// the thread's own registers (rows above and below), warp shuffles (the words
// left and right, and the row across the boundary of the two strips of a
// warp), and a small shared-memory exchange of each warp's first and last row.
//
// A subfield pass tests the words of its rows (8 per thread) from registers
// and shuffles.  The two subfields of one row parity, (0, sy) and (1, sy),
// read only rows of the other parity across rows, and words of their own row
// through shuffles, so they run back to back without a CTA barrier (fused row
// by row, see reg_half): a round takes two barriers (after the even rows,
// after the odd rows), the second one OR-reducing the round's change flag.
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

__host__ __device__ inline bool reg_kernel_fits(int w, int h) {
  return w <= 32 * kRegW && h <= kRegRows;
}
// Shared memory: the padded F plane, then M and cand for all kRegRows rows
// (threads whose rows lie below the image read them: zero), then the
// first/last-row exchange of each warp.
constexpr int kRegPlane = kRegRows * kRegPitch;
constexpr int kRegXchg = 2 * (kThreads / 32) * kRegW;
__host__ __device__ inline int reg_smem_words(int w, int h) {
  return plane_words(w, h) + 2 * kRegPlane + kRegXchg;
}
inline size_t reg_smem_bytes(int w, int h) { return (size_t)reg_smem_words(w, h) * 4; }

struct RegCtx {
  Ctx<SmemMode> g;      // geometry of the padded F plane (and counters)
  uint32_t* M;          // kRegRows rows x kRegPitch words
  uint32_t* cand;       // kRegRows rows x kRegPitch words
  uint32_t* top;        // [warp][kRegW]: first row of each warp
  uint32_t* bot;        // [warp][kRegW]: last row of each warp
  int warp, half, j, s0;  // s0 = first row of this thread's strip
  bool jin;             // j < words per row of the image
};

// The two subfield passes (0, SY) then (1, SY) over this thread's rows of
// parity SY (compile-time).  They are fused row by row: within these two
// passes a row of parity SY reads only itself and the rows of the other
// parity (which do not change), so finishing (0, SY) and (1, SY) on one row
// before the next gives the same result as two full passes.  The simple mask
// of the first test is reused by the second unless a word of the warp's row
// changed in between; then only the row's own left/right words are
// re-shuffled.  Warp rows with no candidate are skipped.  Returns the OR of
// the changed bits.
template <int CONN, int SY>
__device__ __forceinline__ uint32_t reg_half(RegCtx& k, uint32_t (&S)[kRegR], bool thin,
                                             uint32_t above, uint32_t below) {
  const int j = k.j;
  uint32_t* cr = k.cand + k.s0 * kRegPitch + j;
  uint32_t changed = 0;
#pragma unroll
  for (int r = SY; r < kRegR; r += 2) {
    uint32_t cw = cr[r * kRegPitch];
    if (!__any_sync(0xFFFFFFFFu, cw != 0u)) continue;
    const uint32_t n = r > 0 ? S[r - 1] : above;
    uint32_t c = S[r];
    const uint32_t s = r + 1 < kRegR ? S[r + 1] : below;
    uint32_t nw = __shfl_up_sync(0xFFFFFFFFu, n, 1, 16);
    uint32_t wv = __shfl_up_sync(0xFFFFFFFFu, c, 1, 16);
    uint32_t sw = __shfl_up_sync(0xFFFFFFFFu, s, 1, 16);
    uint32_t ne = __shfl_down_sync(0xFFFFFFFFu, n, 1, 16);
    uint32_t e = __shfl_down_sync(0xFFFFFFFFu, c, 1, 16);
    uint32_t se = __shfl_down_sync(0xFFFFFFFFu, s, 1, 16);
    if (j == 0) nw = wv = sw = 0u;
    if (j == kRegW - 1) ne = e = se = 0u;
    uint32_t sm = simple_bits<CONN>(nw, n, ne, wv, c, e, sw, s, se);
    const uint32_t chg0 = cw & 0x55555555u & sm;
    if (__any_sync(0xFFFFFFFFu, chg0 != 0u)) {
      c = thin ? (c & ~chg0) : (c | chg0);
      cw &= ~chg0;
      wv = __shfl_up_sync(0xFFFFFFFFu, c, 1, 16);
      e = __shfl_down_sync(0xFFFFFFFFu, c, 1, 16);
      if (j == 0) wv = 0u;
      if (j == kRegW - 1) e = 0u;
      sm = simple_bits<CONN>(nw, n, ne, wv, c, e, sw, s, se);
    }
    const uint32_t chg1 = cw & 0xAAAAAAAAu & sm;
    c = thin ? (c & ~chg1) : (c | chg1);
    cw &= ~chg1;
    const uint32_t chg = chg0 | chg1;
    if (chg) {
      S[r] = c;
      cr[r * kRegPitch] = cw;
      changed |= chg;
    }
  }
  return changed;
}

// Rounds at one level until a round changes nothing.  False on the cap.
template <int CONN>
__device__ bool reg_level(RegCtx& k, uint32_t (&S)[kRegR], bool thin) {
  const int lane = threadIdx.x & 31;
  for (int round = 0;; ++round) {
    if (round >= k.g.cap) return false;
    ++k.g.n_rounds;
    k.g.n_passes += 4;
    k.g.n_tests += kRegR * 2;
    // even rows: row above the strip = last row of the strip above
    uint32_t ab = __shfl_sync(0xFFFFFFFFu, S[kRegR - 1], lane ^ 16);
    if (k.half == 0) ab = k.warp > 0 ? k.bot[(k.warp - 1) * kRegW + k.j] : 0u;
    uint32_t ch = reg_half<CONN, 0>(k, S, thin, ab, 0u);
    if (k.half == 0) k.top[k.warp * kRegW + k.j] = S[0];
    __syncthreads();
    // odd rows: row below the strip = first row of the strip below
    uint32_t be = __shfl_sync(0xFFFFFFFFu, S[0], lane ^ 16);
    if (k.half == 1)
      be = (k.warp + 1) < (int)(blockDim.x >> 5) ? k.top[(k.warp + 1) * kRegW + k.j] : 0u;
    ch |= reg_half<CONN, 1>(k, S, thin, 0u, be);
    if (k.half == 1) k.bot[k.warp * kRegW + k.j] = S[kRegR - 1];
    if (!__syncthreads_or(ch != 0u)) return true;
  }
}

// One constrained thinning (thin) or thickening at radius r; the allowed
// points are (thin ? S : complement of S) cap pos minus neg (global planes).
template <int CONN>
__device__ bool reg_operator(RegCtx& k, uint32_t (&S)[kRegR], int r, bool thin,
                             const uint32_t* pos, const uint32_t* neg) {
  Ctx<SmemMode>& g = k.g;
  // snapshot F, the movable mask M, no candidates
#pragma unroll
  for (int q = 0; q < kRegR; ++q) {
    const int y = k.s0 + q;
    if (y < g.h) {
      uint32_t m = 0;
      if (k.jin) {
        g.F[g.idx(y, k.j)] = S[q];
        const int t = y * g.wpr + k.j;
        m = g.rowmask(k.j);
        if (pos) m &= pos[t];
        if (neg) m &= ~neg[t];
      }
      k.M[y * kRegPitch + k.j] = m;
      k.cand[y * kRegPitch + k.j] = 0u;
    }
  }
  // first and last rows of each warp, for the first passes
  if (k.half == 0) k.top[k.warp * kRegW + k.j] = S[0];
  if (k.half == 1) k.bot[k.warp * kRegW + k.j] = S[kRegR - 1];
  __syncthreads();
  const uint32_t cm = thin ? 0xFFFFFFFFu : 0u;
  const int nlev = c_lv.nlev[r];
  for (int li = 0; li < nlev; ++li) {
    const int o0 = c_lv.start[li], o1 = c_lv.start[li + 1];
    uint32_t act = 0;
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int y = k.s0 + q;
      if (y >= g.h || !k.jin) continue;
      const int a = y * kRegPitch + k.j;
      const uint32_t cd = k.cand[a];
      uint32_t pend = k.M[a] & (thin ? S[q] : ~S[q]) & ~cd;
      if (!pend) continue;
      uint32_t ring = 0;
      for (int o = o0; o < o1; ++o) {
        ring |= fshift(g, g.F, y + c_lv.off[o][1], k.j, c_lv.off[o][0], cm, cm);
        ++g.n_ring;
        if (!(pend & ~ring)) break;
      }
      const uint32_t add = pend & ring;
      if (add) {
        k.cand[a] = cd | add;
        act = 1;
      }
    }
    if (!__syncthreads_or(act != 0u)) continue;
    ++g.n_levels;
    if (!reg_level<CONN>(k, S, thin)) return false;
  }
  return true;
}

template <int CONN>
__device__ void reg_job(RegCtx& k, const Job& jb, uint32_t* smem) {
  Ctx<SmemMode>& g = k.g;
  uint32_t S[kRegR];
  // pack the input (and C, D) through the F plane
  {
    const int nz = reg_smem_words(jb.w, jb.h);
    for (int t = threadIdx.x; t < nz; t += blockDim.x) smem[t] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int total = g.h * g.wpr;
    const bool cx = jb.op == OP_HASF || jb.op == OP_HC;
    for (int it = wid; it < total; it += nw) {
      const int y = it / g.wpr, j = it - y * g.wpr;
      const int x = (j << 5) + lane;
      const bool inb = x < g.w;
      const size_t off = (size_t)y * jb.pitch + x;
      const uint32_t xs = __ballot_sync(0xFFFFFFFFu, inb && jb.in[off] != 0);
      uint32_t cs = 0, ds = 0;
      if (jb.cp) cs = __ballot_sync(0xFFFFFFFFu, inb && jb.C != nullptr && jb.C[off] != 0);
      if (jb.dp) ds = __ballot_sync(0xFFFFFFFFu, inb && jb.D != nullptr && jb.D[off] != 0);
      if (lane == 0) {
        g.F[g.idx(y, j)] = xs;
        if (jb.cp) jb.cp[it] = cx ? (cs & xs) : cs;
        if (jb.dp) jb.dp[it] = ds & ~xs;
      }
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int y = k.s0 + q;
      S[q] = (y < g.h && k.jin) ? g.F[g.idx(y, k.j)] : 0u;
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
    if (!reg_operator<CONN>(k, S, r, true, nullptr, jb.cp)) return false;
    return reg_operator<CONN>(k, S, r, false, jb.g0, nullptr);
  };
  auto hf = [&](int r) {
    snapshot_g0();
    if (!reg_operator<CONN>(k, S, r, false, nullptr, jb.dp)) return false;
    return reg_operator<CONN>(k, S, r, true, nullptr, jb.g0);
  };
  switch (jb.op) {
    case OP_HASF:
      for (int r = jb.r_lo; ok && r <= jb.r_hi; ++r) {
        ok = hc(r);
        if (ok) ok = hf(r);
      }
      break;
    case OP_THIN: ok = reg_operator<CONN>(k, S, jb.r_hi, true, nullptr, jb.cp); break;
    case OP_THICK: ok = reg_operator<CONN>(k, S, jb.r_hi, false, jb.cp, nullptr); break;
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
  if (jb.stats) {
    unsigned long long t = g.n_tests, rr = g.n_ring;
    for (int o = 16; o > 0; o >>= 1) {
      t += __shfl_down_sync(0xFFFFFFFFu, t, o);
      rr += __shfl_down_sync(0xFFFFFFFFu, rr, o);
    }
    if ((threadIdx.x & 31) == 0) {
      atomicAdd(jb.stats + STAT_WORD_TESTS, t);
      atomicAdd(jb.stats + STAT_RING_EVALS, rr);
    }
    if (threadIdx.x == 0) {
      atomicAdd(jb.stats + STAT_PASSES, (unsigned long long)g.n_passes);
      atomicAdd(jb.stats + STAT_LEVELS, (unsigned long long)g.n_levels);
      atomicAdd(jb.stats + STAT_ROUNDS, (unsigned long long)g.n_rounds);
    }
  }
}

// Persistent CTAs of kThreads threads take register-path jobs from `order`.
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
    const Job& jb = jobs[order[slot]];
    RegCtx k;
    Ctx<SmemMode>& g = k.g;
    g.w = jb.w;
    g.h = jb.h;
    g.wpr = jb.wpr;
    g.P = row_pitch(jb.w);
    const int rem = jb.w & 31;
    g.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
    g.S = nullptr;
    g.F = smem + 1;
    g.cand = nullptr;
    g.cap = jb.cap;
    g.n_tests = g.n_ring = g.n_passes = g.n_levels = g.n_rounds = 0;
    k.M = smem + jb.plane_words;
    k.cand = k.M + kRegPlane;
    k.top = k.cand + kRegPlane;
    k.bot = k.top + (kThreads / 32) * kRegW;
    k.warp = threadIdx.x >> 5;
    k.half = (threadIdx.x >> 4) & 1;
    k.j = threadIdx.x & 15;
    k.s0 = (2 * k.warp + k.half) * kRegR;
    k.jin = k.j < jb.wpr;
    if (jb.conn == 4) reg_job<4>(k, jb, smem);
    else reg_job<8>(k, jb, smem);
    __syncthreads();
  }
}

}  // namespace hasf
