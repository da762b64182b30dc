// hasf_tiled.cuh -- register-resident HASF for images larger than one tile
// (device code; included by hasf_tiled.cu after hasf_reg.cuh, whose helpers it uses).
//
// The image is cut into tiles of 512 x 512 pixels (16 words x 512 rows), one
// CTA per tile, each running the register scheme of the single-tile kernel:
// thread (warp w, lane l) owns word column l & 15 of a 16-row strip.  Tiles
// exchange what crosses their borders:
//   - after every half-round (all rows of one parity updated) and every level
//     update, their first and last word columns, the candidates of their first
//     column, and their first and last rows, into the neighbours' halo arrays
//     (left/right columns with the corner words, the rows above and below);
//   - at the start of every operator, the 31 rows and the word column around
//     the tile of the priority snapshot F, for the ring reads of the level
//     updates (the kernel takes rmax <= 31).
// Inside a fused half-round the rightmost word's odd pixel 31 needs its right
// neighbour's even pixel 0 as updated by the neighbour's own even-column pass;
// that one bit is computed here again from the halo (the neighbour computes the
// same bit from the same data), so a half-round needs no extra barrier.
// An exchange moves the boundaries, ORs one flag over all tiles (level
// activated anything, round changed anything) and is one barrier.  Two
// policies: a thread-block cluster for images of up to 16 tiles, where each
// tile stores its boundary straight into its neighbours' shared memory before
// the hardware cluster barrier; or, for larger images, a gang that publishes
// boundaries to global memory, meets at a bounded gang barrier and then reads
// its neighbours'.
#pragma once

#include <cooperative_groups.h>

namespace hasf {

namespace cg = cooperative_groups;

constexpr int kTW = 16;                  // words per tile row
constexpr int kTH = kRegRows;            // rows per tile (512)
constexpr int kTPad = kRegPadR;          // F halo rows (31)
constexpr int kFP = kTW + 3;             // F row pitch: words -1..16, one pad (odd)
constexpr int kFR = kTH + 2 * kTPad;     // F rows: -31 .. 542
constexpr int kTileF = ((kFR * kFP + 2) + 3) & ~3;
// boundary published to global memory by the gang policy (double-buffered)
constexpr int kPubCol0 = 0, kPubCol15 = kTH, kPubCand0 = 2 * kTH, kPubTop = 3 * kTH,
              kPubBot = 3 * kTH + kTW, kPubWords = 3 * kTH + 2 * kTW;
// halo array: left / right neighbour column at rows -1..512 (index row + 1),
// right neighbour's column-0 candidates, rows above and below.  A strip's 16
// rows start on a 16-byte boundary, so they move as four 16-byte stores.
constexpr int kHLcol = 3, kHRcol = kHLcol + kTH + 4, kHRcand = kHRcol + kTH + 5,
              kHAbove = kHRcand + kTH, kHBelow = kHAbove + kTW, kHaloWords = kHBelow + kTW;
static_assert((kHLcol + 1) % 4 == 0 && (kHRcol + 1) % 4 == 0 && kHRcand % 4 == 0 &&
                  kHaloWords % 4 == 0,
              "halo strips must be 16-byte aligned");
// Both policies double-buffer the halo: exchange n fills buffer n & 1; every
// read of a buffer happens between the barriers of exchanges n and n + 1, and
// the next write to it comes after the barrier of exchange n + 1.
constexpr int kTileSmemWords = kTileF + kRegPlane + kRegXchg + 2 * kHaloWords + 8;

__host__ __device__ inline int tiles_x(int w) { return (words_per_row(w) + kTW - 1) / kTW; }
__host__ __device__ inline int tiles_y(int h) { return (h + kTH - 1) / kTH; }
inline size_t tile_smem_bytes() { return (size_t)kTileSmemWords * 4; }
// global words per tile of the gang policy: published boundary (two buffers) + F centre
constexpr int kGangTileWords = 2 * kPubWords + kTH * kTW;

// ---------------------------------------------------------------------------
// Exchange policies.
// ---------------------------------------------------------------------------

struct ClusterX {
  uint32_t* halo2;  // this CTA's two halo buffers; the same offset in every CTA
  uint32_t* Fc;     // this CTA's F plane at (row 0, word 0)
  int* flags;       // three OR slots (shared memory), exchange n uses slot n % 3
  int slot;
  int ntx, nty, tx, ty;
  __device__ __forceinline__ bool has(int x, int y) const {
    return x >= 0 && x < ntx && y >= 0 && y < nty;
  }
  __device__ __forceinline__ int rank_of(int x, int y) const { return y * ntx + x; }
  __device__ __forceinline__ uint32_t* remote(int dx, int dy, int idx) const {
    return cg::this_cluster().map_shared_rank(halo2 + idx, rank_of(tx + dx, ty + dy));
  }
  __device__ __forceinline__ uint32_t f_ld(int x, int y, int row, int word) const {
    return *cg::this_cluster().map_shared_rank(Fc + row * kFP + word, rank_of(x, y));
  }
  __device__ __forceinline__ void f_publish(int, int, uint32_t) {}  // F is read in place
  __device__ __forceinline__ bool failed() const { return false; }
};

struct GangX {
  uint32_t* gbase;  // kGangTileWords per tile of this image, row-major tiles
  GangMode gm;
  int ntx, nty, tx, ty;
  __device__ __forceinline__ bool has(int x, int y) const {
    return x >= 0 && x < ntx && y >= 0 && y < nty;
  }
  __device__ __forceinline__ uint32_t* tile(int x, int y) const {
    return gbase + (size_t)(y * ntx + x) * kGangTileWords;
  }
  __device__ __forceinline__ uint32_t pub_ld(int x, int y, int off) const {
    return __ldcg(tile(x, y) + off);
  }
  __device__ __forceinline__ uint32_t f_ld(int x, int y, int row, int word) const {
    return __ldcg(tile(x, y) + 2 * kPubWords + row * kTW + word);
  }
  __device__ __forceinline__ void pub_st(int off, uint32_t v) { __stcg(tile(tx, ty) + off, v); }
  __device__ __forceinline__ void f_publish(int row, int word, uint32_t v) {
    __stcg(tile(tx, ty) + 2 * kPubWords + row * kTW + word, v);
  }
  __device__ __forceinline__ bool failed() const { return gm.failed(); }
};

template <class X>
struct TileCtx {
  X x;
  Ctx<SmemMode> g;   // image geometry and counters; g.F = F plane at (row 0, word 0)
  uint32_t* cand;    // 512 x kRegPitch
  uint32_t* xtop;    // [warp][16] first row of each warp of this tile
  uint32_t* xbot;    // [warp][16] last row of each warp
  uint32_t* halo2;   // two halo buffers of kHaloWords
  uint32_t* halo;    // the buffer filled by the last exchange
  int warp, half, j, s0;
  int pb;            // buffer of the next exchange (0 or 1)
  int x0w, y0;       // first word and row of the tile in the image
  bool jin;          // this thread's word lies inside the image
  __device__ __forceinline__ bool row_in(int R) const { return y0 + R < g.h; }
};

// Gang policy: write this tile's boundary (columns 0 and 15, the candidates
// of column 0, rows 0 and 511) to its published area pb in global memory.
__device__ __forceinline__ void gang_publish(TileCtx<GangX>& k, const uint32_t (&S)[kRegR]) {
  const int b = k.pb * kPubWords;
  if (k.j == 0 || k.j == kTW - 1) {
    const int off = b + (k.j == 0 ? kPubCol0 : kPubCol15);
#pragma unroll
    for (int q = 0; q < kRegR; ++q) k.x.pub_st(off + k.s0 + q, S[q]);
    if (k.j == 0)
#pragma unroll
      for (int q = 0; q < kRegR; ++q)
        k.x.pub_st(b + kPubCand0 + k.s0 + q, k.cand[(k.s0 + q) * kRegPitch]);
  }
  if (k.warp == 0 && k.half == 0) k.x.pub_st(b + kPubTop + k.j, S[0]);
  if (k.warp == (int)(blockDim.x >> 5) - 1 && k.half == 1)
    k.x.pub_st(b + kPubBot + k.j, S[kRegR - 1]);
}

// Gang policy: copy the neighbours' published area pb into halo buffer pb.
__device__ void gang_fetch(TileCtx<GangX>& k) {
  uint32_t* h = k.halo2 + k.pb * kHaloWords;
  const int tx = k.x.tx, ty = k.x.ty;
  const int b = k.pb * kPubWords;
  for (int i = threadIdx.x; i < kTH + 2; i += blockDim.x) {
    const int R = i - 1;
    const int dy = R < 0 ? -1 : (R >= kTH ? 1 : 0);
    const int rr = R - dy * kTH;
    h[kHLcol + i] =
        k.x.has(tx - 1, ty + dy) ? k.x.pub_ld(tx - 1, ty + dy, b + kPubCol15 + rr) : 0u;
    h[kHRcol + i] =
        k.x.has(tx + 1, ty + dy) ? k.x.pub_ld(tx + 1, ty + dy, b + kPubCol0 + rr) : 0u;
    if (R >= 0 && R < kTH)
      h[kHRcand + R] = k.x.has(tx + 1, ty) ? k.x.pub_ld(tx + 1, ty, b + kPubCand0 + R) : 0u;
  }
  for (int i = threadIdx.x; i < kTW; i += blockDim.x) {
    h[kHAbove + i] = k.x.has(tx, ty - 1) ? k.x.pub_ld(tx, ty - 1, b + kPubBot + i) : 0u;
    h[kHBelow + i] = k.x.has(tx, ty + 1) ? k.x.pub_ld(tx, ty + 1, b + kPubTop + i) : 0u;
  }
  __syncthreads();
}

// One exchange: every tile's boundary into its neighbours' halo buffer pb and
// the OR of v over all threads of all tiles, at the cost of one barrier.
// Gang policy: publish, gang barrier (which carries the OR), read.
__device__ int tile_exchange(TileCtx<GangX>& k, const uint32_t (&S)[kRegR], int v) {
  gang_publish(k, S);
  const int any = k.x.gm.barrier(v);
  if (k.x.failed()) return 0;
  gang_fetch(k);
  k.halo = k.halo2 + k.pb * kHaloWords;
  k.pb ^= 1;
  return any;
}

__device__ __forceinline__ void st4(uint32_t* d, uint32_t a, uint32_t b, uint32_t c,
                                    uint32_t e) {
  *reinterpret_cast<uint4*>(d) = make_uint4(a, b, c, e);
}

// Cluster policy: stores into the neighbours' shared memory, OR flags, one
// hardware cluster barrier (release / acquire: the stores are visible after it).
__device__ int tile_exchange(TileCtx<ClusterX>& k, const uint32_t (&S)[kRegR], int v) {
  const ClusterX& x = k.x;
  const int o = k.pb * kHaloWords;
  const int tx = x.tx, ty = x.ty;
  const bool top = k.s0 == 0, bot = k.s0 + kRegR == kTH;
  if (k.j == 0 && x.has(tx - 1, ty)) {
    // left neighbour: its right column and its right column's candidates
    uint32_t* d = x.remote(-1, 0, o + kHRcol + 1 + k.s0);
#pragma unroll
    for (int q = 0; q < kRegR; q += 4) st4(d + q, S[q], S[q + 1], S[q + 2], S[q + 3]);
    const uint32_t* c = k.cand + k.s0 * kRegPitch;
    uint32_t* e = x.remote(-1, 0, o + kHRcand + k.s0);
#pragma unroll
    for (int q = 0; q < kRegR; q += 4)
      st4(e + q, c[q * kRegPitch], c[(q + 1) * kRegPitch], c[(q + 2) * kRegPitch],
          c[(q + 3) * kRegPitch]);
  }
  if (k.j == kTW - 1 && x.has(tx + 1, ty)) {
    uint32_t* d = x.remote(1, 0, o + kHLcol + 1 + k.s0);
#pragma unroll
    for (int q = 0; q < kRegR; q += 4) st4(d + q, S[q], S[q + 1], S[q + 2], S[q + 3]);
  }
  // corner words (row 0 or 511 of column 0 or 15) for the diagonal tiles
  if (k.j == 0 && top && x.has(tx - 1, ty - 1)) *x.remote(-1, -1, o + kHRcol + kTH + 1) = S[0];
  if (k.j == 0 && bot && x.has(tx - 1, ty + 1)) *x.remote(-1, 1, o + kHRcol) = S[kRegR - 1];
  if (k.j == kTW - 1 && top && x.has(tx + 1, ty - 1))
    *x.remote(1, -1, o + kHLcol + kTH + 1) = S[0];
  if (k.j == kTW - 1 && bot && x.has(tx + 1, ty + 1)) *x.remote(1, 1, o + kHLcol) = S[kRegR - 1];
  if (top && x.has(tx, ty - 1)) *x.remote(0, -1, o + kHBelow + k.j) = S[0];
  if (bot && x.has(tx, ty + 1)) *x.remote(0, 1, o + kHAbove + k.j) = S[kRegR - 1];
  // OR flag: every warp that saw v sets slot n % 3 in every tile (all write the
  // same value, so plain stores do); each tile clears the slot of exchange
  // n + 2, whose last reads came before this barrier and whose next writes
  // come after the next one.
  const int lane = threadIdx.x & 31;
  if (__any_sync(0xFFFFFFFFu, v) && lane < x.ntx * x.nty)
    *cg::this_cluster().map_shared_rank(x.flags + x.slot, lane) = 1;
  cg::this_cluster().sync();
  const int any = *(volatile int*)(x.flags + x.slot);
  if (threadIdx.x == 0) x.flags[x.slot == 0 ? 2 : x.slot - 1] = 0;
  k.x.slot = x.slot == 2 ? 0 : x.slot + 1;
  k.halo = k.halo2 + o;
  k.pb ^= 1;
  return any;
}

// The two subfield passes (0, SY), (1, SY) over this thread's rows of parity SY,
// fused row by row as in the single-tile kernel, with the tile's left/right
// neighbour words from the halo and the right neighbour's even pixel 0
// recomputed for the odd pass.
template <int CONN, int SY, bool thin, class X>
__device__ __forceinline__ uint32_t tile_half(TileCtx<X>& k, uint32_t (&S)[kRegR],
                                              uint32_t above, uint32_t below) {
  const int j = k.j;
  const uint32_t* lcol = k.halo + kHLcol;   // index = tile row + 1
  const uint32_t* rcol = k.halo + kHRcol;
  const uint32_t* rcand = k.halo + kHRcand;
  uint32_t* cr = k.cand + k.s0 * kRegPitch + j;
  uint32_t changed = 0;
#pragma unroll
  for (int r = SY; r < kRegR; r += 2) {
    uint32_t cw = cr[r * kRegPitch];
    const int R = k.s0 + r;
    const bool redge = j == kTW - 1 && (rcand[R] & 1u);
    if (!__any_sync(0xFFFFFFFFu, cw != 0u || redge)) continue;
    const uint32_t n = r > 0 ? S[r - 1] : above;
    uint32_t c = S[r];
    const uint32_t s = r + 1 < kRegR ? S[r + 1] : below;
    uint32_t nw = __shfl_up_sync(0xFFFFFFFFu, n, 1, 16);
    uint32_t wv = __shfl_up_sync(0xFFFFFFFFu, c, 1, 16);
    uint32_t sw = __shfl_up_sync(0xFFFFFFFFu, s, 1, 16);
    uint32_t ne = __shfl_down_sync(0xFFFFFFFFu, n, 1, 16);
    uint32_t e = __shfl_down_sync(0xFFFFFFFFu, c, 1, 16);
    uint32_t se = __shfl_down_sync(0xFFFFFFFFu, s, 1, 16);
    if (j == 0) {
      nw = lcol[R];
      wv = lcol[R + 1];
      sw = lcol[R + 2];
    }
    if (j == kTW - 1) {
      ne = rcol[R];
      e = rcol[R + 1];
      se = rcol[R + 2];
    }
    uint32_t sm = simple_bits<CONN>(nw, n, ne, wv, c, e, sw, s, se);
    const uint32_t chg0 = cw & 0x55555555u & sm;
    // the right neighbour's pixel 0 after its even-column pass: its 3 x 3
    // words are (n, ne, -), (c, e, -), (s, se, -) seen from its side
    uint32_t e1 = e;
    if (redge) {
      const uint32_t smr = simple_bits<CONN>(n, ne, 0u, c, e, 0u, s, se, 0u);
      const uint32_t cr0 = rcand[R] & 1u & smr;
      e1 = thin ? (e & ~cr0) : (e | cr0);
    }
    if (__any_sync(0xFFFFFFFFu, chg0 != 0u || e1 != e)) {
      // odd pixels see only their own word's even pixels on the left
      c = thin ? (c & ~chg0) : (c | chg0);
      cw &= ~chg0;
      uint32_t e2 = __shfl_down_sync(0xFFFFFFFFu, c, 1, 16);
      if (j == kTW - 1) e2 = e1;
      sm = simple_bits<CONN>(nw, n, ne, wv, c, e2, sw, s, se);
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

// Row above / below this thread's strip at its column: the other strip of the
// warp, the neighbouring warp, or the tile above / below (halo).
template <class X>
__device__ __forceinline__ uint32_t tile_above(TileCtx<X>& k, const uint32_t (&S)[kRegR]) {
  const int lane = threadIdx.x & 31;
  uint32_t v = __shfl_sync(0xFFFFFFFFu, S[kRegR - 1], lane ^ 16);
  if (k.half == 0)
    v = k.warp > 0 ? k.xbot[(k.warp - 1) * kTW + k.j] : k.halo[kHAbove + k.j];
  return v;
}
template <class X>
__device__ __forceinline__ uint32_t tile_below(TileCtx<X>& k, const uint32_t (&S)[kRegR]) {
  const int lane = threadIdx.x & 31;
  uint32_t v = __shfl_sync(0xFFFFFFFFu, S[0], lane ^ 16);
  if (k.half == 1)
    v = (k.warp + 1) < (int)(blockDim.x >> 5) ? k.xtop[(k.warp + 1) * kTW + k.j]
                                             : k.halo[kHBelow + k.j];
  return v;
}

template <int CONN, bool thin, class X>
__device__ bool tile_level(TileCtx<X>& k, uint32_t (&S)[kRegR]) {
  for (int round = 0;; ++round) {
    if (round >= k.g.cap) return false;
    ++k.g.n_rounds;
    k.g.n_passes += 4;
    k.g.n_tests += 2 * kRegR;
    uint32_t ch = tile_half<CONN, 0, thin>(k, S, tile_above(k, S), 0u);
    if (k.half == 0) k.xtop[k.warp * kTW + k.j] = S[0];
    tile_exchange(k, S, 0);
    if (k.x.failed()) return false;
    ch |= tile_half<CONN, 1, thin>(k, S, 0u, tile_below(k, S));
    if (k.half == 1) k.xbot[k.warp * kTW + k.j] = S[kRegR - 1];
    const int any = tile_exchange(k, S, ch != 0u);
    if (k.x.failed()) return false;
    if (!any) return true;
  }
}

template <int CONN, bool thin, class X>
__device__ bool tile_operator(TileCtx<X>& k, uint32_t (&S)[kRegR], int r,
                              const uint32_t* pos, const uint32_t* neg) {
  Ctx<SmemMode>& g = k.g;
  uint32_t pendrows = 0;
  // snapshot F (centre), movable mask, no candidates
#pragma unroll
  for (int q = 0; q < kRegR; ++q) {
    const int R = k.s0 + q;
    uint32_t m = 0;
    if (k.row_in(R) && k.jin) {
      const int t = (k.y0 + R) * g.wpr + k.x0w + k.j;
      m = g.rowmask(k.x0w + k.j);
      if (pos) m &= pos[t];
      if (neg) m &= ~neg[t];
      if (m & (thin ? S[q] : ~S[q])) pendrows |= 1u << q;
    }
    g.F[R * kFP + k.j] = S[q];
    k.x.f_publish(R, k.j, S[q]);
    k.cand[R * kRegPitch + k.j] = 0u;
  }
  if (k.half == 0) k.xtop[k.warp * kTW + k.j] = S[0];
  if (k.half == 1) k.xbot[k.warp * kTW + k.j] = S[kRegR - 1];
  tile_exchange(k, S, 0);
  if (k.x.failed()) return false;
  // F halo: 31 rows above and below (words -1..16), words -1 and 16 beside
  {
    const int tx = k.x.tx, ty = k.x.ty;
    const int band = kTPad * (kTW + 2);
    for (int i = threadIdx.x; i < 2 * band + 2 * kTH; i += blockDim.x) {
      int R, w;
      if (i < 2 * band) {
        const int b = i < band ? i : i - band;
        R = i < band ? -kTPad + b / (kTW + 2) : kTH + b / (kTW + 2);
        w = b % (kTW + 2) - 1;
      } else {
        const int b = i - 2 * band;
        R = b % kTH;
        w = b < kTH ? -1 : kTW;
      }
      const int dx = w < 0 ? -1 : (w >= kTW ? 1 : 0);
      const int dy = R < 0 ? -1 : (R >= kTH ? 1 : 0);
      const uint32_t v = k.x.has(tx + dx, ty + dy)
                             ? k.x.f_ld(tx + dx, ty + dy, R - dy * kTH, w - dx * kTW)
                             : 0u;
      g.F[R * kFP + w] = v;
    }
  }
  __syncthreads();
  const int nlev = c_lv.nlev[r];
  for (int li = 0; li < nlev; ++li) {
    const int o0 = c_lv.start[li], o1 = c_lv.start[li + 1];
    uint32_t newrows = 0;
#pragma unroll
    for (int g4 = 0; g4 < kRegR; g4 += 4) {
      if (!((pendrows >> g4) & 0xFu)) continue;
      uint32_t pend[4], acc[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = g4 + u;
        pend[u] = 0u;
        if ((pendrows >> q) & 1u) {
          // the movable mask, read again from the constraint planes rather
          // than kept in shared memory (this tile's words of them are written
          // by this CTA only, so cached loads see its own writes)
          const int R = k.s0 + q;
          const int t = (k.y0 + R) * g.wpr + k.x0w + k.j;
          uint32_t m = g.rowmask(k.x0w + k.j);
          if (pos) m &= pos[t];
          if (neg) m &= ~neg[t];
          pend[u] = m & (thin ? S[q] : ~S[q]) & ~k.cand[R * kRegPitch + k.j];
          if (!pend[u]) pendrows &= ~(1u << q);
        }
        acc[u] = thin ? 0xFFFFFFFFu : 0u;
      }
      if (!(pend[0] | pend[1] | pend[2] | pend[3])) continue;
      const uint32_t* base = g.F + (k.s0 + g4) * kFP + k.j;
      // unrolled eight vectors deep, the stop checked every eight (as in the
      // register kernel's walk: latency-bound)
#pragma unroll 8
      for (int o = o0; o < o1; ++o) {
        const int dx = c_lv.off[o][0], dy = c_lv.off[o][1];
        const uint32_t* p0 = base + dy * kFP + (dx >> 5);
        const int sh = dx & 31;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (pend[u]) {
            const uint32_t v = __funnelshift_r(p0[u * kFP], p0[u * kFP + 1], sh);
            acc[u] = thin ? (acc[u] & v) : (acc[u] | v);
          }
        }
        ++g.n_ring;
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
          k.cand[(k.s0 + q) * kRegPitch + k.j] |= add;
          newrows |= 1u << q;
          if (!(pend[u] & ~add)) pendrows &= ~(1u << q);
        }
      }
    }
    const int any = tile_exchange(k, S, newrows != 0u);   // column-0 candidates changed
    if (k.x.failed()) return false;
    if (!any) continue;
    ++g.n_levels;
    if (!tile_level<CONN, thin>(k, S)) return false;
  }
  return true;
}

template <int CONN, class X>
__device__ __forceinline__ void tile_job(TileCtx<X>& k, const Job& jb, uint32_t* smem) {
  Ctx<SmemMode>& g = k.g;
  uint32_t S[kRegR];
  {
    const bool vec = ((reinterpret_cast<uintptr_t>(jb.in) | (uintptr_t)jb.pitch |
                       reinterpret_cast<uintptr_t>(jb.C) | reinterpret_cast<uintptr_t>(jb.D)) &
                      15u) == 0;
    const bool cx = jb.op == OP_HASF || jb.op == OP_HC;
    const int wimg = k.x0w + k.j;
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int R = k.s0 + q;
      uint32_t xs = 0;
      if (k.row_in(R) && k.jin) {
        const size_t off = (size_t)(k.y0 + R) * jb.pitch + (wimg << 5);
        const int n = min(32, g.w - (wimg << 5));
        xs = pack_word(jb.in + off, n, vec);
        const int t = (k.y0 + R) * g.wpr + wimg;
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
      const int R = k.s0 + q;
      if (k.row_in(R) && k.jin) jb.g0[(k.y0 + R) * g.wpr + k.x0w + k.j] = S[q];
    }
    __syncthreads();
  };
  // one call site per operator kind keeps the kernel small
  const int nst = op_steps(jb);
  bool ok = nst > 0;
  for (int st = 0; ok && st < nst; ++st) {
    const OpStep o = op_step(jb, st);
    if (o.snap) snapshot_g0();
    ok = o.thin ? tile_operator<CONN, true>(k, S, o.r, o.pos, o.neg)
                : tile_operator<CONN, false>(k, S, o.r, o.pos, o.neg);
  }
  if (ok) {
    const bool vec = ((reinterpret_cast<uintptr_t>(jb.out) | (uintptr_t)jb.pitch) & 15u) == 0;
    const int wimg = k.x0w + k.j;
#pragma unroll
    for (int q = 0; q < kRegR; ++q) {
      const int R = k.s0 + q;
      if (!k.row_in(R) || !k.jin) continue;
      const uint32_t v = S[q];
      uint8_t* o = jb.out + (size_t)(k.y0 + R) * jb.pitch + (wimg << 5);
      const int n = min(32, g.w - (wimg << 5));
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
  job_done(jb, k.x.ntx * k.x.nty);
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
    if (threadIdx.x == 0 && k.x.tx == 0 && k.x.ty == 0) {
      atomicAdd(jb.stats + STAT_PASSES, (unsigned long long)g.n_passes);
      atomicAdd(jb.stats + STAT_LEVELS, (unsigned long long)g.n_levels);
      atomicAdd(jb.stats + STAT_ROUNDS, (unsigned long long)g.n_rounds);
    }
  }
}

template <class X>
__device__ __forceinline__ void tile_init(TileCtx<X>& k, const Job& jb, uint32_t* smem, int tx,
                                          int ty) {
  Ctx<SmemMode>& g = k.g;
  g.w = jb.w;
  g.h = jb.h;
  g.wpr = jb.wpr;
  g.P = kFP;
  const int rem = jb.w & 31;
  g.lastmask = rem ? ((1u << rem) - 1u) : 0xFFFFFFFFu;
  g.S = nullptr;
  g.cand = nullptr;
  g.F = smem + 1 + kTPad * kFP + 1;   // row 0, word 0 (word -1 is one to the left)
  g.cap = jb.cap;
  g.n_tests = g.n_ring = g.n_passes = g.n_levels = g.n_rounds = 0;
  k.cand = smem + kTileF;
  k.xtop = k.cand + kRegPlane;
  k.xbot = k.xtop + (kThreads / 32) * kTW;
  k.halo2 = k.xbot + (kThreads / 32) * kTW;
  k.halo = k.halo2 + kHaloWords;
  k.pb = 0;
  k.warp = threadIdx.x >> 5;
  k.half = (threadIdx.x >> 4) & 1;
  k.j = threadIdx.x & 15;
  k.s0 = (2 * k.warp + k.half) * kRegR;
  k.x0w = tx * kTW;
  k.y0 = ty * kTH;
  k.jin = k.x0w + k.j < jb.wpr;
  k.x.ntx = tiles_x(jb.w);
  k.x.nty = tiles_y(jb.h);
  k.x.tx = tx;
  k.x.ty = ty;
}

}  // namespace hasf
