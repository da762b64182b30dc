// hasf_edt.cu -- exact squared Euclidean distance transform on the GPU
// (Sec. 4.1: Meijster's algorithm in its two independent phases).
//
// Phase 1 (Algorithm 1): one thread per column computes g, the vertical
// distance to the nearest feature pixel of its column, with a downward and an
// upward scan.  Neighbouring threads own neighbouring columns, so every row
// step is one coalesced load of consecutive bytes and one coalesced store.
//
// Phase 2 (Algorithm 2): one thread per row builds the lower envelope of the
// parabolas i -> (x - i)^2 + g(i)^2 left to right (a stack of apex columns and
// of the first column where each parabola takes over), then reads it back
// right to left.  The separator of two parabolas i < u is the last x where i
// is no worse: floor((u^2 - i^2 + g(u)^2 - g(i)^2) / (2 (u - i))).
//
// When the outside of the box counts as feature, the envelope also holds the
// columns -1 and w (whose g is 0) and the vertical scans start from a feature
// just above row 0 and just below row h - 1.
#include <cstdint>
#include <cuda_runtime.h>

#include "hasf_internal.h"

namespace hasf {

__global__ void edt_columns_kernel(const uint8_t* __restrict__ feat, int w, int h, int pitch,
                                   int outside, int32_t* __restrict__ g) {
  const int none = w + h + 2;
  for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < w; x += gridDim.x * blockDim.x) {
    int above = outside ? 0 : none;  // distance of the row above to its nearest feature
    for (int y = 0; y < h; ++y) {
      const int v = feat[(size_t)y * pitch + x] ? 0 : min(above + 1, none);
      g[(size_t)y * w + x] = v;
      above = v;
    }
    int below = outside ? 0 : none;
    for (int y = h - 1; y >= 0; --y) {
      int v = g[(size_t)y * w + x];
      const int cand = min(below + 1, none);
      if (cand < v) {
        v = cand;
        g[(size_t)y * w + x] = v;
      }
      below = v;
    }
  }
}

__global__ void edt_rows_kernel(const int32_t* __restrict__ g, int w, int h, int outside,
                                int32_t* __restrict__ stack, int32_t* __restrict__ d) {
  const long long none = (long long)w + h + 2;
  const int c0 = outside ? -1 : 0, c1 = outside ? w + 1 : w;
  const int span = w + 2;
  for (int y = blockIdx.x * blockDim.x + threadIdx.x; y < h; y += gridDim.x * blockDim.x) {
    const int32_t* gr = g + (size_t)y * w;
    int32_t* apex = stack + (size_t)y * 2 * span;
    int32_t* from = apex + span;
    auto gv = [&](int i) -> long long { return (i < 0 || i >= w) ? 0LL : (long long)gr[i]; };
    auto par = [&](long long x, int i) -> long long {
      const long long dx = x - i, gi = gv(i);
      return dx * dx + gi * gi;
    };
    int top = 0;
    apex[0] = c0;
    from[0] = c0;
    for (int u = c0 + 1; u < c1; ++u) {
      while (top >= 0 && par(from[top], apex[top]) > par(from[top], u)) --top;
      if (top < 0) {
        top = 0;
        apex[0] = u;
        from[0] = c0;
        continue;
      }
      const int i = apex[top];
      const long long gi = gv(i), gu = gv(u);
      const long long num = (long long)u * u - (long long)i * i + gu * gu - gi * gi;
      const long long den = 2LL * (u - i);
      long long q = num / den;
      if (num % den != 0 && num < 0) --q;
      const long long first = q + 1;
      if (first < c1) {
        ++top;
        apex[top] = u;
        from[top] = (int32_t)first;
      }
    }
    for (int u = c1 - 1; u >= c0; --u) {
      if (u >= 0 && u < w) {
        const long long v = par(u, apex[top]);
        d[(size_t)y * w + u] = v >= none * none ? -1 : (int32_t)v;
      }
      if (u == from[top]) --top;
    }
  }
}

cudaError_t launch_edt(const uint8_t* feat, int w, int h, int pitch, int outside, int32_t* g,
                       int32_t* stack, int32_t* d, cudaStream_t s) {
  edt_columns_kernel<<<(w + 127) / 128, 128, 0, s>>>(feat, w, h, pitch, outside, g);
  edt_rows_kernel<<<(h + 63) / 64, 64, 0, s>>>(g, w, h, outside, stack, d);
  return cudaGetLastError();
}

}  // namespace hasf
