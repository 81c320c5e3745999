// common.cuh -- shared device helpers of libsfc (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "sfc.h"

namespace sfc {

// Device-side status bits (ORed into a library-owned word, read by sfc_status).
enum : uint32_t { ST_BAD_CENTRE = 1u, ST_TIMEOUT = 2u, ST_OVERFLOW = 4u };

// Upper bound of the spin iterations of any wait on another CTA's flag.
constexpr long long kSpinLimit = 1ll << 24;

// Geometry as the kernels see it.
struct Geo {
  int ndim, ch, K, r, P;  // P = K^ndim pixels per patch
  int64_t X, Y, Z;
  int n;                  // values per patch, P * ch
};

__host__ __device__ inline int64_t lin_of(const Geo& g, int64_t x, int64_t y, int64_t z) {
  return (z * g.Y + y) * g.X + x;
}

// Linear pixel offset of patch pixel pp relative to the centre.
__host__ __device__ inline int64_t patch_off(const Geo& g, int pp) {
  int px = pp % g.K, py = (pp / g.K) % g.K, pz = g.ndim == 3 ? pp / (g.K * g.K) : g.r;
  return ((int64_t)(pz - g.r) * g.Y + (py - g.r)) * g.X + (px - g.r);
}

// Valid centre: the whole patch inside the grid.
__device__ inline bool centre_ok(const Geo& g, int64_t x, int64_t y, int64_t z) {
  if (x < g.r || x > g.X - 1 - g.r || y < g.r || y > g.Y - 1 - g.r) return false;
  if (g.ndim == 3) return z >= g.r && z <= g.Z - 1 - g.r;
  return z == 0;
}

// ---------------------------------------------------------------------------
// packed (cost, id) keys: non-negative IEEE values order like their bit
// patterns, so min over (bits << 32 | id) is argmin with ties to the lowest id.
__device__ inline unsigned long long pack_min(float c, uint32_t id) {
  return ((unsigned long long)__float_as_uint(c) << 32) | id;
}

template <typename T>
__device__ inline T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    T w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}

__device__ inline float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Lexicographic (c64, id) minimum across a warp.
__device__ inline void warp_argmin64(double& c, int64_t& id) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    double c2 = __shfl_xor_sync(0xffffffffu, c, o);
    int64_t i2 = __shfl_xor_sync(0xffffffffu, id, o);
    if (c2 < c || (c2 == c && i2 < id)) {
      c = c2;
      id = i2;
    }
  }
}

// Exact cost of one (target, source) pair in FP64: known elements of the target
// in patch raster order, channel innermost, d = t - p in FP64 (operands widened
// from FP32), term = w * (d * d), sequential sum, no fused multiply-add.
// `tv`/`tm` hold the target's values and per-pixel known flags; `eoff` the
// element offsets (pixel offset * ch + channel) relative to centre * ch.
__device__ inline double exact_cost64(const float* __restrict__ grid, int64_t src_base, const float* tv,
                                      const uint8_t* tm, const int* eoff, int P, int ch, const float* w,
                                      bool l1 = false) {
  double acc = 0.0;
  for (int pp = 0; pp < P; ++pp) {
    if (!tm[pp]) continue;
    for (int c = 0; c < ch; ++c) {
      int e = pp * ch + c;
      double d = __dsub_rn((double)tv[e], (double)grid[src_base + eoff[e]]);
      double sq = l1 ? fabs(d) : __dmul_rn(d, d);  // L1 (Sec. III.K): |d|
      double term = __dmul_rn((double)w[c], sq);
      acc = __dadd_rn(acc, term);
    }
  }
  return acc;
}

// Upper end of the FP32 band around the FP32 minimum: |c32 - c| <= gamma * c
// for a sum of n non-negative terms, each d^2 or |d| (d rounded once) times a
// rounded weight, summed by FMA or addition, with gamma = (n + 8) * 2^-24.  A candidate can be the
// exact argmin only if c32 <= min32 * (1 + 3 gamma) + n * 2^-126 (absolute
// slack for underflow).  Every operation rounds up, so the float returned is >=
// that bound and the band it defines contains the exact one.
__device__ inline float band_limit32(float min32, int n) {
  const float g3 = __fmul_ru((float)(n + 8), 1.78813934326171875e-7f);  // 3 * 2^-24
  const float t = __fmaf_ru(min32, g3, min32);
  return __fadd_ru(t, __fmul_ru((float)n, 1.1754943508222875e-38f));
}

// Quantised coordinate (same arithmetic for dictionary entries and queries):
// clamp(floor((y - lo) * scale), 0, 2^b - 1), subtraction and product rounded to
// FP32 separately.
__device__ inline uint32_t quantise_one(float y, float lo, float scale, int bits) {
  float t = __fsub_rn(y, lo);
  float u = __fmul_rn(t, scale);
  float f = floorf(u);
  float top = (float)((1u << bits) - 1u);
  if (!(f >= 0.0f)) f = 0.0f;
  if (f > top) f = top;
  return (uint32_t)f;
}

// Morton / z-address: bit planes from the highest, dimension 0 first inside a
// plane; the first 64 bits emitted when D * bp > 64.
__device__ inline uint64_t morton_key(const uint32_t* q, int D, int bp) {
  uint64_t key = 0;
  int n = 0;
  for (int p = bp - 1; p >= 0 && n < 64; --p)
    for (int k = 0; k < D && n < 64; ++k, ++n) key = (key << 1) | (uint64_t)((q[k] >> p) & 1u);
  return key;
}

// Packed pairs of FP32 values for fma.rn.f32x2 (sm_100+): each half is the
// same IEEE round-to-nearest fused multiply-add as the scalar one (the
// projections it computes are bit-identical to the scalar chains).
__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

// morton_key for D = 8: the key is the top min(bp, 8) bit planes of the eight
// coordinates, one byte per plane (dimension 0 its most significant bit), i.e.
// the transpose of the 8 x 8 bit matrix whose row 7 - k holds coordinate k's
// top eight bits.  The transpose is the three-step swap of 1 x 1, 2 x 2 and
// 4 x 4 blocks across the diagonal (Hacker's Delight, Sec. 7-3).
__host__ __device__ inline uint64_t morton_key8(const uint32_t* q, int bp) {
  const int sh = bp > 8 ? bp - 8 : 0;
  const uint32_t m = bp >= 8 ? 0xffu : (1u << bp) - 1u;
  uint64_t x = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) x |= (uint64_t)((q[k] >> sh) & m) << (8 * (7 - k));
  uint64_t t;
  t = (x ^ (x >> 7)) & 0x00AA00AA00AA00AAull;
  x ^= t ^ (t << 7);
  t = (x ^ (x >> 14)) & 0x0000CCCC0000CCCCull;
  x ^= t ^ (t << 14);
  t = (x ^ (x >> 28)) & 0x00000000F0F0F0F0ull;
  x ^= t ^ (t << 28);
  return x;
}

// morton_key with D known at compile time (q stays in registers): each bit
// plane's D bits form a group, dimension 0 its most significant bit.
template <int D>
__device__ inline uint64_t morton_key_t(const uint32_t* q, int bp) {
  if constexpr (D == 8) return morton_key8(q, bp);
  uint64_t key = 0;
  int n = 0;
  for (int p = bp - 1; p >= 0 && n < 64; --p) {
    uint32_t grp = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) grp = (grp << 1) | ((q[k] >> p) & 1u);
    const int take = 64 - n < D ? 64 - n : D;
    key = (key << take) | (uint64_t)(grp >> (D - take));
    n += take;
  }
  return key;
}

// Hilbert key (Skilling 2004, transpose method): the coordinates q[0..D) of bp
// bits are rewritten into the transposed Hilbert index -- from the top bit
// plane down, coordinate 0's bits below the plane are inverted where
// coordinate i has the plane's bit, else exchanged with coordinate i's (undoing
// the sub-cube rotations and reflections); then a Gray code across the
// coordinates and a final xor with the low-bit masks of the planes where the
// last coordinate is set -- and interleaved as morton_key does.  q is modified.
__device__ inline uint64_t hilbert_key(uint32_t* q, int D, int bp) {
  const uint32_t top = 1u << (bp - 1);
  for (uint32_t plane = top; plane > 1; plane >>= 1) {
    const uint32_t low = plane - 1;
    for (int i = 0; i < D; ++i) {
      if (q[i] & plane) {
        q[0] ^= low;
      } else {
        const uint32_t t = (q[0] ^ q[i]) & low;
        q[0] ^= t;
        q[i] ^= t;
      }
    }
  }
  for (int i = 1; i < D; ++i) q[i] ^= q[i - 1];
  uint32_t mask = 0;
  for (uint32_t plane = top; plane > 1; plane >>= 1)
    if (q[D - 1] & plane) mask ^= plane - 1;
  for (int i = 0; i < D; ++i) q[i] ^= mask;
  return morton_key(q, D, bp);
}

// hilbert_key with D known at compile time (the same steps)
template <int D>
__device__ inline uint64_t hilbert_key_t(uint32_t* q, int bp) {
  const uint32_t top = 1u << (bp - 1);
  for (uint32_t plane = top; plane > 1; plane >>= 1) {
    const uint32_t low = plane - 1;
#pragma unroll
    for (int i = 0; i < D; ++i) {
      if (q[i] & plane) {
        q[0] ^= low;
      } else {
        const uint32_t t = (q[0] ^ q[i]) & low;
        q[0] ^= t;
        q[i] ^= t;
      }
    }
  }
#pragma unroll
  for (int i = 1; i < D; ++i) q[i] ^= q[i - 1];
  uint32_t mask = 0;
  for (uint32_t plane = top; plane > 1; plane >>= 1)
    if (q[D - 1] & plane) mask ^= plane - 1;
#pragma unroll
  for (int i = 0; i < D; ++i) q[i] ^= mask;
  return morton_key_t<D>(q, bp);
}

}  // namespace sfc
