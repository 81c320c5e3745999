// k_fullscan.cu -- exact full scan (Sec. I: the cost of every dictionary patch,
// then the global minimum) for a batch of queries.
//
// Pass 1 (FP32, CUDA cores): a CTA takes QT queries x (256 * EPT) dictionary
// entries; every thread keeps an EPT x QT register tile of costs, the queries'
// per-element (known, known * value) pairs sit in shared memory (read as
// broadcasts), the source patch values are gathered from the grid (L2-resident).
// Per element: d = fma(-k, p, k t) (exactly k (t - p) for k in {0,1}), acc =
// fma(d, d, acc); weighted: acc = fma(w d, d, acc).  The CTA writes its per-query
// minimum (tile minimum) and folds it into a per-query global minimum.
// Pass 2 (one CTA per query): every tile whose minimum lies inside the FP32
// error band of the global minimum is re-evaluated with the identical FP32
// arithmetic and its in-band entries listed.  One entry in the band is the exact
// argmin; with several (near-ties) each is rescored with the exact FP64
// sequential cost and the argmin over (cost, id) taken.  The reported cost is
// the FP32 cost of the pick.  Costs are non-negative, so float bit patterns order
// like their values.
#include <atomic>

#include "internal.cuh"

namespace sfc {

namespace {

constexpr int kFsThreads = 256;
constexpr int kBandCap = 64;  // in-band entries listed per query before the fallback

// CM (cost mode): bit 0 = channel weights, bit 1 = L1 norm (Sec. III.K) instead of
// the squared L2 norm.  One accumulation step of the FP32 cost for the
// difference d: w d^2 or d^2 by FMA (L2), w |d| by FMA or + |d| (L1).
template <int CM>
__device__ __forceinline__ float cost_step(float acc, float d, float w) {
  if (CM & 2) return (CM & 1) ? __fmaf_rn(w, fabsf(d), acc) : __fadd_rn(acc, fabsf(d));
  return (CM & 1) ? __fmaf_rn(__fmul_rn(w, d), d, acc) : __fmaf_rn(d, d, acc);
}

// CM (cost mode): bit 0 = channel weights, bit 1 = L1 norm.
template <int QT, int EPT, int CM>
__global__ void __launch_bounds__(kFsThreads) k_fs_scan(const float* __restrict__ grid,
                                                        const uint8_t* __restrict__ mask, Geo g,
                                                        const uint32_t* __restrict__ dict, int64_t N,
                                                        const int* __restrict__ eoff_all,
                                                        const float* __restrict__ weights,
                                                        const int64_t* __restrict__ centre_lin, int64_t Q,
                                                        int64_t qbase, float* __restrict__ tilemin,
                                                        unsigned int* __restrict__ gmin, int64_t ntiles) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, ch = g.ch;
  float2* am = reinterpret_cast<float2*>(smem_raw);  // [ne][QT]: (known, known * t)
  int* eo = reinterpret_cast<int*>(am + (size_t)n * QT);
  float* we = reinterpret_cast<float*>(eo + n);       // [ne] weights (WEIGHTED)
  __shared__ int s_wcnt[kFsThreads / 32];
  const int64_t q0 = qbase + (int64_t)blockIdx.y * QT;
  // the elements known to at least one query of the tile, in patch order: an
  // element unknown to every query adds exactly 0 to every cost, so it is left out
  const int lane0 = threadIdx.x & 31, warp0 = threadIdx.x >> 5;
  int ne = 0;
  for (int r0 = 0; r0 < n; r0 += kFsThreads) {
    const int e = r0 + threadIdx.x;
    int o = 0, pixo = 0;
    bool any = false;
    if (e < n) {
      o = eoff_all[e];
      pixo = eoff_all[e - e % ch] / ch;
#pragma unroll
      for (int qi = 0; qi < QT; ++qi) {
        const int64_t q = q0 + qi;
        if (q < Q) any |= mask[centre_lin[q] + pixo] != 0;
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, any);
    if (lane0 == 0) s_wcnt[warp0] = __popc(bal);
    __syncthreads();
    int off = ne, tot = 0;
    for (int w = 0; w < kFsThreads / 32; ++w) {
      if (w < warp0) off += s_wcnt[w];
      tot += s_wcnt[w];
    }
    if (any) {
      const int at = off + __popc(bal & ((1u << lane0) - 1u));
      eo[at] = o;
      if (CM & 1) we[at] = weights[e % ch];
#pragma unroll
      for (int qi = 0; qi < QT; ++qi) {
        const int64_t q = q0 + qi;
        float2 v = make_float2(0.0f, 0.0f);
        if (q < Q) {
          const int64_t tc = centre_lin[q];
          const float k = mask[tc + pixo] ? 1.0f : 0.0f;
          v = make_float2(k, k * grid[tc * ch + o]);
        }
        am[(size_t)at * QT + qi] = v;
      }
    }
    __syncthreads();
    ne += tot;
  }
  const int64_t j0 = (int64_t)blockIdx.x * kFsThreads * EPT + threadIdx.x;
  int64_t sb[EPT];
#pragma unroll
  for (int k = 0; k < EPT; ++k) {
    int64_t j = j0 + (int64_t)k * kFsThreads;
    sb[k] = j < N ? (int64_t)dict[j] * ch : -1;
  }
  float acc[EPT][QT];
#pragma unroll
  for (int k = 0; k < EPT; ++k)
#pragma unroll
    for (int qi = 0; qi < QT; ++qi) acc[k][qi] = 0.0f;
  for (int e = 0; e < ne; ++e) {
    const int o = eo[e];
    float p[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) p[k] = sb[k] >= 0 ? __ldg(grid + sb[k] + o) : 0.0f;
    float w = (CM & 1) ? we[e] : 1.0f;
#pragma unroll
    for (int qi = 0; qi < QT; ++qi) {
      const float2 v = am[(size_t)e * QT + qi];
#pragma unroll
      for (int k = 0; k < EPT; ++k) {
        float d = __fmaf_rn(-v.x, p[k], v.y);
        acc[k][qi] = cost_step<CM>(acc[k][qi], d, w);
      }
    }
  }
  __shared__ float red[kFsThreads / 32][QT];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int qi = 0; qi < QT; ++qi) {
    float m = INFINITY;
#pragma unroll
    for (int k = 0; k < EPT; ++k)
      if (sb[k] >= 0) m = fminf(m, acc[k][qi]);
    m = warp_min(m);
    if (lane == 0) red[warp][qi] = m;
  }
  __syncthreads();
  if (threadIdx.x < QT) {
    const int qi = threadIdx.x;
    float m = red[0][qi];
    for (int w = 1; w < kFsThreads / 32; ++w) m = fminf(m, red[w][qi]);
    int64_t q = q0 + qi;
    if (q < Q) {
      tilemin[q * ntiles + blockIdx.x] = m;
      atomicMin(&gmin[q], __float_as_uint(m));
    }
  }
}

// Same FP32 arithmetic for one query and one entry (bit-identical to pass 1).
template <int CM>
__device__ inline float cost32_one(const float* __restrict__ grid, int64_t sb, const float2* am, const int* eo,
                                   const float* we, int n) {
  float acc = 0.0f;
  for (int e = 0; e < n; ++e) {
    float p = __ldg(grid + sb + eo[e]);
    float d = __fmaf_rn(-am[e].x, p, am[e].y);
    acc = cost_step<CM>(acc, d, (CM & 1) ? we[e] : 1.0f);
  }
  return acc;
}

// RANGE: the band pass of one shard of a dictionary split (the entries dict[0,
// N) are ids id_base + [0, N) of the whole dictionary, gmin is the minimum over
// every shard): every in-band entry of the shard is rescored in FP64 (no
// single-entry shortcut, since other shards may hold band entries too) and the
// shard's (FP64 cost, id, FP32 cost) minimum is written to cost64 / pick / cost
// (+inf, -1, +inf when the shard holds no band entry).
template <int EPT, int CM, bool RANGE = false>
__global__ void __launch_bounds__(kFsThreads) k_fs_band(const float* __restrict__ grid,
                                                        const uint8_t* __restrict__ mask, Geo g,
                                                        const uint32_t* __restrict__ dict, int64_t N,
                                                        const int* __restrict__ eoff_all,
                                                        const float* __restrict__ weights,
                                                        const int64_t* __restrict__ centre_lin,
                                                        const float* __restrict__ tilemin,
                                                        const unsigned int* __restrict__ gmin, int64_t ntiles,
                                                        int64_t* __restrict__ pick, float* __restrict__ cost,
                                                        double* __restrict__ cost64 = nullptr, int64_t id_base = 0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, ch = g.ch, P = g.P;
  float2* am = reinterpret_cast<float2*>(smem_raw);
  float* tv = reinterpret_cast<float*>(am + n);
  int* eo = reinterpret_cast<int*>(tv + n);
  float* we = reinterpret_cast<float*>(eo + n);
  uint8_t* tm = reinterpret_cast<uint8_t*>(we + n);
  const int64_t q = blockIdx.x;
  const int64_t tc = centre_lin[q];
  for (int e = threadIdx.x; e < n; e += kFsThreads) {
    int o = eoff_all[e];
    eo[e] = o;
    we[e] = weights[e % ch];
    float t = grid[tc * ch + o];
    float k = mask[tc + eoff_all[e - e % ch] / ch] ? 1.0f : 0.0f;
    tv[e] = t;
    am[e] = make_float2(k, k * t);
  }
  for (int pp = threadIdx.x; pp < P; pp += kFsThreads) tm[pp] = mask[tc + eoff_all[pp * ch] / ch];
  __syncthreads();
  const float m32 = __uint_as_float(gmin[q]);
  const float T = band_limit32(m32, n);
  // pass A: collect the in-band entries (usually exactly one)
  __shared__ int s_cnt;
  __shared__ int64_t s_j[kBandCap];
  __shared__ float s_c[kBandCap];
  if (threadIdx.x == 0) s_cnt = 0;
  __syncthreads();
  for (int64_t t = 0; t < ntiles; ++t) {
    if (tilemin[q * ntiles + t] > T) continue;  // uniform across the CTA
    for (int k = 0; k < EPT; ++k) {
      const int64_t j = t * kFsThreads * EPT + (int64_t)k * kFsThreads + threadIdx.x;
      if (j >= N) continue;
      const float c32 = cost32_one<CM>(grid, (int64_t)dict[j] * ch, am, eo, we, n);
      if (c32 <= T) {
        const int slot = atomicAdd(&s_cnt, 1);
        if (slot < kBandCap) {
          s_j[slot] = j;
          s_c[slot] = c32;
        }
      }
    }
  }
  __syncthreads();
  const int cnt = s_cnt;
  if (!RANGE && cnt == 1) {
    if (threadIdx.x == 0) {
      pick[q] = s_j[0];
      cost[q] = s_c[0];
    }
    return;
  }
  // pass B: exact FP64 rescore of the band (from the list, or -- if it
  // overflowed -- recomputing the in-band tiles)
  double bc = INFINITY;
  int64_t bj = INT64_MAX;
  float bc32 = 0.0f;
  if (cnt <= kBandCap) {
    for (int i = threadIdx.x; i < cnt; i += kFsThreads) {
      const int64_t j = s_j[i];
      const double c64 = exact_cost64(grid, (int64_t)dict[j] * ch, tv, tm, eo, P, ch, weights, (CM & 2) != 0);
      if (c64 < bc || (c64 == bc && j < bj)) {
        bc = c64;
        bj = j;
        bc32 = s_c[i];
      }
    }
  } else {
    for (int64_t t = 0; t < ntiles; ++t) {
      if (tilemin[q * ntiles + t] > T) continue;
      for (int k = 0; k < EPT; ++k) {
        const int64_t j = t * kFsThreads * EPT + (int64_t)k * kFsThreads + threadIdx.x;
        if (j >= N) continue;
        const int64_t sb = (int64_t)dict[j] * ch;
        const float c32 = cost32_one<CM>(grid, sb, am, eo, we, n);
        if (c32 <= T) {
          const double c64 = exact_cost64(grid, sb, tv, tm, eo, P, ch, weights, (CM & 2) != 0);
          if (c64 < bc || (c64 == bc && j < bj)) {
            bc = c64;
            bj = j;
            bc32 = c32;
          }
        }
      }
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double c2 = __shfl_xor_sync(0xffffffffu, bc, o);
    const int64_t j2 = __shfl_xor_sync(0xffffffffu, bj, o);
    const float f2 = __shfl_xor_sync(0xffffffffu, bc32, o);
    if (c2 < bc || (c2 == bc && j2 < bj)) {
      bc = c2;
      bj = j2;
      bc32 = f2;
    }
  }
  __shared__ double sd[kFsThreads / 32];
  __shared__ int64_t si[kFsThreads / 32];
  __shared__ float sf[kFsThreads / 32];
  if ((threadIdx.x & 31) == 0) {
    sd[threadIdx.x >> 5] = bc;
    si[threadIdx.x >> 5] = bj;
    sf[threadIdx.x >> 5] = bc32;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kFsThreads / 32; ++w)
      if (sd[w] < bc || (sd[w] == bc && si[w] < bj)) {
        bc = sd[w];
        bj = si[w];
        bc32 = sf[w];
      }
    if (RANGE) {
      const bool none = bj == INT64_MAX;
      pick[q] = none ? -1 : id_base + bj;
      cost[q] = none ? __int_as_float(0x7f800000) : bc32;
      cost64[q] = none ? __longlong_as_double(0x7ff0000000000000ll) : bc;
    } else if (bj == INT64_MAX) {
      pick[q] = -1;
      cost[q] = __int_as_float(0x7fc00000);
    } else {
      pick[q] = bj;
      cost[q] = bc32;
    }
  }
}

// Exact pass after the tensor-core pre-score: a group of 32 dictionary entries
// can hold the exact argmin only if its pre-score minimum lies within 2 E_q of
// the smallest one (|s_hat - s| <= E_q for every entry).  One CTA per query;
// warp w takes the selected groups of the 1024-entry chunks w, w + 8, ...; each
// lane scores one entry of a group with the FP32 cost of k_fs_band and keeps
// the entries within the FP32 band of its own running minimum (at most
// kLaneCands, pruned as the minimum falls; more sends the query through a
// second pass).  The band of the CTA's minimum is a subset of what the lanes
// kept, so the usual band / FP64 decision follows.
constexpr int kLaneCands = 4;

template <bool WEIGHTED>
__global__ void __launch_bounds__(kFsThreads) k_tc_select(const float* __restrict__ grid,
                                                          const uint8_t* __restrict__ mask, Geo g,
                                                          const uint32_t* __restrict__ dict, int64_t N,
                                                          const int* __restrict__ eoff_all,
                                                          const float* __restrict__ weights,
                                                          const int64_t* __restrict__ centre_lin,
                                                          const float* __restrict__ submin, int64_t nsub,
                                                          const double* __restrict__ bound,
                                                          int64_t* __restrict__ pick, float* __restrict__ cost,
                                                          int* __restrict__ nsel) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n = g.n, ch = g.ch, P = g.P;
  float2* am = reinterpret_cast<float2*>(smem_raw);
  float* tv = reinterpret_cast<float*>(am + n);
  int* eo = reinterpret_cast<int*>(tv + n);
  float* we = reinterpret_cast<float*>(eo + n);
  uint8_t* tm = reinterpret_cast<uint8_t*>(we + n);
  __shared__ float red[kFsThreads / 32];
  __shared__ int s_cnt, s_nsel, s_over;
  __shared__ int64_t s_j[kBandCap];
  __shared__ float s_c[kBandCap];
  const int64_t q = blockIdx.x;
  const int64_t tc = centre_lin[q];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int e = threadIdx.x; e < n; e += kFsThreads) {
    const int o = eoff_all[e];
    eo[e] = o;
    we[e] = weights[e % ch];
    const float t = grid[tc * ch + o];
    const float k = mask[tc + eoff_all[e - e % ch] / ch] ? 1.0f : 0.0f;
    tv[e] = t;
    am[e] = make_float2(k, k * t);
  }
  for (int pp = threadIdx.x; pp < P; pp += kFsThreads) tm[pp] = mask[tc + eoff_all[pp * ch] / ch];
  // smallest group minimum
  const int64_t ngrp = (N + 31) / 32;
  const float* sm = submin + q * nsub;
  float mh = INFINITY;
  for (int64_t t = threadIdx.x; t < ngrp; t += kFsThreads) mh = fminf(mh, sm[t]);
  mh = warp_min(mh);
  if (lane == 0) red[warp] = mh;
  if (threadIdx.x == 0) {
    s_cnt = 0;
    s_nsel = 0;
    s_over = 0;
  }
  __syncthreads();
  mh = red[0];
  for (int w = 1; w < kFsThreads / 32; ++w) mh = fminf(mh, red[w]);
  const double thr = (double)mh + 2.0001 * bound[q] + 1e-30;
  __syncthreads();
  // fn(j) for every entry j < N of every selected group of this warp's chunks
  auto each_selected = [&](auto&& fn) {
    for (int64_t base = (int64_t)warp * 32; base < ngrp; base += kFsThreads) {
      const int64_t gi = base + lane;
      unsigned bal = __ballot_sync(0xffffffffu, gi < ngrp && (double)sm[gi] <= thr);
      while (bal) {
        const int b = __ffs(bal) - 1;
        bal &= bal - 1;
        const int64_t j = (base + b) * 32 + lane;
        fn(j);
      }
    }
  };
  // single pass: running minimum and the entries within its band
  float mt = INFINITY;
  float cc[kLaneCands];
  int64_t cj[kLaneCands];
#pragma unroll
  for (int i = 0; i < kLaneCands; ++i) {
    cc[i] = INFINITY;
    cj[i] = -1;
  }
  bool over = false;
  int mysel = 0;
  each_selected([&](int64_t j) {
    ++mysel;
    if (j >= N) return;
    const float c = cost32_one<WEIGHTED ? 1 : 0>(grid, (int64_t)dict[j] * ch, am, eo, we, n);
    if (c < mt) {
      mt = c;
      const float T = band_limit32(mt, n);
#pragma unroll
      for (int i = 0; i < kLaneCands; ++i)
        if (cc[i] > T) cc[i] = INFINITY;
    }
    if (c <= band_limit32(mt, n)) {
      bool placed = false;
#pragma unroll
      for (int i = 0; i < kLaneCands; ++i)
        if (!placed && cc[i] == INFINITY) {
          cc[i] = c;
          cj[i] = j;
          placed = true;
        }
      over |= !placed;
    }
  });
  mt = warp_min(mt);
  if (lane == 0) {
    red[warp] = mt;
    atomicAdd(&s_nsel, mysel);
  }
  if (over) s_over = 1;
  __syncthreads();
  float m32 = red[0];
  for (int w = 1; w < kFsThreads / 32; ++w) m32 = fminf(m32, red[w]);
  if (threadIdx.x == 0 && nsel) nsel[q] = s_nsel;
  const float T = band_limit32(m32, n);
  auto push = [&](int64_t j, float c) {
    const int slot = atomicAdd(&s_cnt, 1);
    if (slot < kBandCap) {
      s_j[slot] = j;
      s_c[slot] = c;
    }
  };
  if (!s_over) {
#pragma unroll
    for (int i = 0; i < kLaneCands; ++i)
      if (cc[i] <= T) push(cj[i], cc[i]);
  } else {
    each_selected([&](int64_t j) {
      if (j >= N) return;
      const float c = cost32_one<WEIGHTED ? 1 : 0>(grid, (int64_t)dict[j] * ch, am, eo, we, n);
      if (c <= T) push(j, c);
    });
  }
  __syncthreads();
  const int cnt = s_cnt;
  if (cnt == 1) {
    if (threadIdx.x == 0) {
      pick[q] = s_j[0];
      cost[q] = s_c[0];
    }
    return;
  }
  double bc = INFINITY;
  int64_t bj = INT64_MAX;
  float bc32 = 0.0f;
  auto consider = [&](int64_t j, float c32) {
    const double c64 = exact_cost64(grid, (int64_t)dict[j] * ch, tv, tm, eo, P, ch, weights);
    if (c64 < bc || (c64 == bc && j < bj)) {
      bc = c64;
      bj = j;
      bc32 = c32;
    }
  };
  if (cnt <= kBandCap) {
    for (int i = threadIdx.x; i < cnt; i += kFsThreads) consider(s_j[i], s_c[i]);
  } else {
    each_selected([&](int64_t j) {
      if (j >= N) return;
      const float c = cost32_one<WEIGHTED ? 1 : 0>(grid, (int64_t)dict[j] * ch, am, eo, we, n);
      if (c <= T) consider(j, c);
    });
  }
  for (int o = 16; o > 0; o >>= 1) {
    const double c2 = __shfl_xor_sync(0xffffffffu, bc, o);
    const int64_t j2 = __shfl_xor_sync(0xffffffffu, bj, o);
    const float f2 = __shfl_xor_sync(0xffffffffu, bc32, o);
    if (c2 < bc || (c2 == bc && j2 < bj)) {
      bc = c2;
      bj = j2;
      bc32 = f2;
    }
  }
  __shared__ double sd[kFsThreads / 32];
  __shared__ int64_t si[kFsThreads / 32];
  __shared__ float sf[kFsThreads / 32];
  if (lane == 0) {
    sd[warp] = bc;
    si[warp] = bj;
    sf[warp] = bc32;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kFsThreads / 32; ++w)
      if (sd[w] < bc || (sd[w] == bc && si[w] < bj)) {
        bc = sd[w];
        bj = si[w];
        bc32 = sf[w];
      }
    if (bj == INT64_MAX) {
      pick[q] = -1;
      cost[q] = __int_as_float(0x7fc00000);
    } else {
      pick[q] = bj;
      cost[q] = bc32;
    }
  }
}

// centre rows -> linear pixel index; invalid centres flag the status word and
// get index -1 (their outputs become -1 / NaN).
__global__ void k_centre_lin(const int32_t* __restrict__ centres, int64_t Q, Geo g, int64_t* __restrict__ lin,
                             uint32_t* __restrict__ status) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  int64_t x = centres[q * g.ndim], y = centres[q * g.ndim + 1], z = g.ndim == 3 ? centres[q * g.ndim + 2] : 0;
  if (centre_ok(g, x, y, z)) {
    lin[q] = lin_of(g, x, y, z);
  } else {
    lin[q] = -1;
    atomicOr(status, ST_BAD_CENTRE);
  }
}

// Replace invalid centres by a valid stand-in (pixel of the first centre slot)
// for the scan and mark their outputs afterwards.
__global__ void k_centre_fix(int64_t* lin, int64_t Q, Geo g, uint8_t* bad) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q >= Q) return;
  bad[q] = lin[q] < 0;
  if (lin[q] < 0) lin[q] = lin_of(g, g.r, g.r, g.ndim == 3 ? g.r : 0);
}

__global__ void k_mark_bad(const uint8_t* bad, int64_t Q, int64_t* pick, float* cost) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < Q && bad[q]) {
    pick[q] = -1;
    cost[q] = __int_as_float(0x7fc00000);
  }
}

__global__ void k_fill_u32(unsigned int* p, int64_t n, unsigned int v) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

template <int QT, int EPT, int W>
int run_scan(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
             const int* eoff_all, const float* weights, const int64_t* lin, int64_t Q, float* tilemin,
             unsigned int* gmin, int64_t ntiles, cudaStream_t st) {
  const size_t shm = (size_t)g.n * QT * sizeof(float2) + (size_t)g.n * 8;
  if (shm > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_fs_scan<QT, EPT, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  const int64_t qtiles = (Q + QT - 1) / QT;
  for (int64_t y0 = 0; y0 < qtiles; y0 += 65535) {
    int64_t ny = qtiles - y0 < 65535 ? qtiles - y0 : 65535;
    count_launch();
    k_fs_scan<QT, EPT, W><<<dim3((unsigned)ntiles, (unsigned)ny), kFsThreads, shm, st>>>(
        grid, cur_mask, g, dict, N, eoff_all, weights, lin, Q, y0 * QT, tilemin, gmin, ntiles);
    SFC_TRY(cudaGetLastError());
  }
  return SFC_OK;
}

template <int EPT, int W>
int run_band(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
             const int* eoff_all, const float* weights, const int64_t* lin, int64_t Q, const float* tilemin,
             const unsigned int* gmin, int64_t ntiles, int64_t* pick, float* cost, cudaStream_t st) {
  const size_t shm = (size_t)g.n * 20 + (size_t)g.P + 16;
  if (shm > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_fs_band<EPT, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  count_launch();
  k_fs_band<EPT, W><<<(unsigned)Q, kFsThreads, shm, st>>>(grid, cur_mask, g, dict, N, eoff_all, weights, lin,
                                                          tilemin, gmin, ntiles, pick, cost);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

// Cost-mode dispatch (cm: bit 0 weights, bit 1 L1) of the scan and band passes.
template <int QT, int EPT>
int scan_cm(int cm, const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
            const int* eoff_all, const float* weights, const int64_t* lin, int64_t Q, float* tilemin,
            unsigned int* gmin, int64_t ntiles, cudaStream_t st) {
  switch (cm & 3) {
    case 0: return run_scan<QT, EPT, 0>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
    case 1: return run_scan<QT, EPT, 1>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
    case 2: return run_scan<QT, EPT, 2>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
    default: return run_scan<QT, EPT, 3>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
  }
}

template <int EPT>
int band_cm(int cm, const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
            const int* eoff_all, const float* weights, const int64_t* lin, int64_t Q, const float* tilemin,
            const unsigned int* gmin, int64_t ntiles, int64_t* pick, float* cost, cudaStream_t st) {
  switch (cm & 3) {
    case 0: return run_band<EPT, 0>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
    case 1: return run_band<EPT, 1>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
    case 2: return run_band<EPT, 2>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
    default: return run_band<EPT, 3>(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
  }
}

template <int EPT, int W>
int run_band_range(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                   const int* eoff_all, const float* weights, const int64_t* lin, int64_t Q, const float* tilemin,
                   const unsigned int* gmin, int64_t ntiles, int64_t id_base, int64_t* id, float* cost32,
                   double* cost64, cudaStream_t st) {
  const size_t shm = (size_t)g.n * 20 + (size_t)g.P + 16;
  if (shm > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_fs_band<EPT, W, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  count_launch();
  k_fs_band<EPT, W, true><<<(unsigned)Q, kFsThreads, shm, st>>>(grid, cur_mask, g, dict, N, eoff_all, weights, lin,
                                                                tilemin, gmin, ntiles, id, cost32, cost64, id_base);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

// shard outputs of the queries whose centre is invalid: id -1, costs NaN
__global__ void k_mark_bad_range(const uint8_t* bad, int64_t Q, int64_t* id, float* cost32, double* cost64) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < Q && bad[q]) {
    id[q] = -1;
    cost32[q] = __int_as_float(0x7fc00000);
    cost64[q] = __longlong_as_double(0x7ff8000000000000ll);
  }
}

__global__ void k_fill_range_empty(int64_t Q, int64_t* id, float* cost32, double* cost64) {
  int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (q < Q) {
    id[q] = -1;
    cost32[q] = __int_as_float(0x7f800000);
    cost64[q] = __longlong_as_double(0x7ff0000000000000ll);
  }
}

}  // namespace

constexpr int kRangeEPT = 4;
int64_t fullscan_range_tiles(int64_t n) { return (n + kFsThreads * kRangeEPT - 1) / (kFsThreads * kRangeEPT); }

// Shard scan of a dictionary split: the FP32 pass over dict[0, n) (one shard's
// entries) for Q valid centres `lin`; gmin (Q words) receives the shard's
// per-query minimum FP32 cost as float bits (+inf for an empty shard); tilemin
// (Q * fullscan_range_tiles(n) floats) keeps the tile minima for the band pass.
int fullscan_range_scan(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t n,
                        const int* eoff_all, const float* weights, int cm, const int64_t* lin, int64_t Q,
                        float* tilemin, unsigned int* gmin, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  count_launch();
  k_fill_u32<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(gmin, Q, 0x7f800000u);
  SFC_TRY(cudaGetLastError());
  if (n <= 0) return SFC_OK;
  const int64_t ntiles = fullscan_range_tiles(n);
  return Q >= 8 ? scan_cm<8, kRangeEPT>(cm, g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin,
                                        ntiles, st)
                : scan_cm<1, kRangeEPT>(cm, g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin,
                                        ntiles, st);
}

// Shard band pass: gmin = the minimum over all shards; writes the shard's
// (cost64, id, cost32) minimum over its in-band entries, ids offset by id_base.
int fullscan_range_band(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t n,
                        const int* eoff_all, const float* weights, int cm, const int64_t* lin, int64_t Q,
                        const uint8_t* bad, const float* tilemin, const unsigned int* gmin, int64_t id_base,
                        int64_t* id, float* cost32, double* cost64, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  const unsigned qb = (unsigned)((Q + 255) / 256);
  if (n <= 0) {
    count_launch();
    k_fill_range_empty<<<qb, 256, 0, st>>>(Q, id, cost32, cost64);
  } else {
    const int64_t ntiles = fullscan_range_tiles(n);
    int rc;
    switch (cm & 3) {
      case 0: rc = run_band_range<kRangeEPT, 0>(g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, id_base, id, cost32, cost64, st); break;
      case 1: rc = run_band_range<kRangeEPT, 1>(g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, id_base, id, cost32, cost64, st); break;
      case 2: rc = run_band_range<kRangeEPT, 2>(g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, id_base, id, cost32, cost64, st); break;
      default: rc = run_band_range<kRangeEPT, 3>(g, grid, cur_mask, dict, n, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, id_base, id, cost32, cost64, st); break;
    }
    SFC_CHECK(rc);
  }
  count_launch();
  k_mark_bad_range<<<qb, 256, 0, st>>>(bad, Q, id, cost32, cost64);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

// Centre rows -> linear indices for a shard (invalid centres: a stand-in index
// and bad[q] = 1; the status word is flagged as for every full scan).
int centres_to_lin(const Geo& g, const int32_t* centres, int64_t Q, int64_t* lin, uint8_t* bad, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  const unsigned qb = (unsigned)((Q + 255) / 256);
  count_launch();
  k_centre_lin<<<qb, 256, 0, st>>>(centres, Q, g, lin, status_word());
  count_launch();
  k_centre_fix<<<qb, 256, 0, st>>>(lin, Q, g, bad);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

// One query whose centre (linear index) is already on the device and valid; the
// caller owns the tile-minimum buffer (ceil(N / 1024) floats) and gmin.
int fullscan_single(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                    const int* eoff_all, const float* weights, int cm, const int64_t* centre_lin,
                    int64_t* pick, float* cost, float* tilemin, unsigned int* gmin, cudaStream_t st) {
  constexpr int EPT = 4;
  const int64_t ntiles = (N + kFsThreads * EPT - 1) / (kFsThreads * EPT);
  count_launch();
  k_fill_u32<<<1, 32, 0, st>>>(gmin, 1, 0x7f800000u);
  const int rc = scan_cm<1, EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, centre_lin, 1, tilemin, gmin,
                                 ntiles, st);
  SFC_CHECK(rc);
  return band_cm<EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, centre_lin, 1, tilemin, gmin, ntiles, pick,
                      cost, st);
}

int tc_prescore(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                const int* eoff_all, const float* weights, const int64_t* centre_lin, int64_t Q, float* submin,
                float* scores, double* bound, cudaStream_t st);
int64_t tc_subs(int64_t N);

// The full scan with the tensor-core pre-score (precision SFC_FP16): pre-score
// minima of 32-entry groups, then the exact pass over the groups that can hold
// the argmin.  nsel (optional, device, Q ints) receives the number of groups
// rescored.
int fullscan_batch_tc(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                      const int* eoff_all, const float* weights, bool weighted, const int32_t* centres, int64_t Q,
                      int64_t* pick, float* cost, int* nsel, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  Scratch scr(st);  // freed on every return
  const int64_t nsub = tc_subs(N);
  int64_t* lin = nullptr;
  uint8_t* bad = nullptr;
  float* tilemin = nullptr;
  double* bound = nullptr;
  SFC_TRY(scr.alloc(&lin, sizeof(int64_t) * Q));
  SFC_TRY(scr.alloc(&bad, Q));
  SFC_TRY(scr.alloc(&tilemin, sizeof(float) * Q * nsub));
  SFC_TRY(scr.alloc(&bound, sizeof(double) * Q));
  const unsigned qb = (unsigned)((Q + 255) / 256);
  count_launch();
  k_centre_lin<<<qb, 256, 0, st>>>(centres, Q, g, lin, status_word());
  count_launch();
  k_centre_fix<<<qb, 256, 0, st>>>(lin, Q, g, bad);
  SFC_CHECK(tc_prescore(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, nullptr, bound, st));
  const size_t shm = (size_t)g.n * 20 + (size_t)g.P + 16;
  if (weighted) {
    if (shm > kSmemOptIn)
      SFC_TRY(cudaFuncSetAttribute(k_tc_select<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    count_launch();
    k_tc_select<true><<<(unsigned)Q, kFsThreads, shm, st>>>(grid, cur_mask, g, dict, N, eoff_all, weights, lin,
                                                             tilemin, nsub, bound, pick, cost, nsel);
  } else {
    if (shm > kSmemOptIn)
      SFC_TRY(cudaFuncSetAttribute(k_tc_select<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    count_launch();
    k_tc_select<false><<<(unsigned)Q, kFsThreads, shm, st>>>(grid, cur_mask, g, dict, N, eoff_all, weights, lin,
                                                              tilemin, nsub, bound, pick, cost, nsel);
  }
  count_launch();
  k_mark_bad<<<qb, 256, 0, st>>>(bad, Q, pick, cost);
  SFC_TRY(cudaGetLastError());
  tc_trace_mark(3, st);
  tc_trace_end(2.0 * (double)Q * (double)N * 6.0 * g.n);
  return SFC_OK;
}

// All Q x N pre-scores (checking): scores (device, Q*N), bound (device, Q).
int tc_prescores_all(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                     const int* eoff_all, const float* weights, const int32_t* centres, int64_t Q, float* scores,
                     double* bound, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  Scratch scr(st);  // freed on every return
  const int64_t nsub = tc_subs(N);
  int64_t* lin = nullptr;
  uint8_t* bad = nullptr;
  float* tilemin = nullptr;
  SFC_TRY(scr.alloc(&lin, sizeof(int64_t) * Q));
  SFC_TRY(scr.alloc(&bad, Q));
  SFC_TRY(scr.alloc(&tilemin, sizeof(float) * Q * nsub));
  const unsigned qb = (unsigned)((Q + 255) / 256);
  count_launch();
  k_centre_lin<<<qb, 256, 0, st>>>(centres, Q, g, lin, status_word());
  count_launch();
  k_centre_fix<<<qb, 256, 0, st>>>(lin, Q, g, bad);
  SFC_CHECK(tc_prescore(g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, scores, bound, st));
  return SFC_OK;
}

// Tile shapes of the FP32 scan (queries per CTA tile, dictionary entries per
// thread): every shape computes the same FP32 cost of every (query, entry) pair
// (the sum over the patch elements in order) and the same band, so the picks
// and costs do not depend on it; the fastest one for a workload is found by
// measurement (sfc_tune_tiles) and kept for the process.
namespace {
struct FsShape {
  int qt, ept;
};
constexpr FsShape kFsShapes[] = {{8, 4}, {8, 2}, {16, 2}, {4, 4}, {4, 8}, {16, 4}, {32, 2}};
constexpr int kFsNShapes = sizeof(kFsShapes) / sizeof(kFsShapes[0]);
std::atomic<int> g_fs_shape{0};

template <int QT, int EPT>
int fullscan_shape(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                   const int* eoff_all, const float* weights, int cm, const int32_t* centres,
                   const int64_t* centre_lin, int64_t Q, int64_t* pick, float* cost, cudaStream_t st) {
  Scratch scr(st);  // freed on every return
  const int64_t ntiles = (N + kFsThreads * EPT - 1) / (kFsThreads * EPT);
  int64_t* lin = nullptr;
  uint8_t* bad = nullptr;
  float* tilemin = nullptr;
  unsigned int* gmin = nullptr;
  SFC_TRY(scr.alloc(&tilemin, sizeof(float) * Q * ntiles));
  SFC_TRY(scr.alloc(&gmin, sizeof(unsigned int) * Q));
  SFC_TRY(scr.alloc(&bad, Q));
  SFC_TRY(scr.alloc(&lin, sizeof(int64_t) * Q));
  if (!centre_lin) {
    count_launch();
    k_centre_lin<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(centres, Q, g, lin, status_word());
  } else {
    SFC_TRY(cudaMemcpyAsync(lin, centre_lin, sizeof(int64_t) * Q, cudaMemcpyDeviceToDevice, st));
  }
  count_launch();
  k_centre_fix<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(lin, Q, g, bad);
  count_launch();
  k_fill_u32<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(gmin, Q, 0x7f800000u);
  int rc = Q >= QT ? scan_cm<QT, EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st)
                   : scan_cm<1, EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
  SFC_CHECK(rc);
  rc = band_cm<EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
  SFC_CHECK(rc);
  count_launch();
  k_mark_bad<<<(unsigned)((Q + 255) / 256), 256, 0, st>>>(bad, Q, pick, cost);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}
}  // namespace

int fullscan_tile_shapes(int* qt, int* ept) {
  for (int i = 0; i < kFsNShapes; ++i) {
    if (qt) qt[i] = kFsShapes[i].qt;
    if (ept) ept[i] = kFsShapes[i].ept;
  }
  return kFsNShapes;
}

int fullscan_tile_shape(int shape) {
  if (shape >= 0 && shape < kFsNShapes) g_fs_shape.store(shape);
  return g_fs_shape.load();
}

int fullscan_batch(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                   const int* eoff_all, const float* weights, int cm, const int32_t* centres,
                   const int64_t* centre_lin, int64_t Q, int64_t* pick, float* cost, cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  switch (g_fs_shape.load()) {
#define SFC_SHAPE(i, qt, ept) \
  case i: return fullscan_shape<qt, ept>(g, grid, cur_mask, dict, N, eoff_all, weights, cm, centres, centre_lin, Q, pick, cost, st);
    SFC_SHAPE(1, 8, 2) SFC_SHAPE(2, 16, 2) SFC_SHAPE(3, 4, 4) SFC_SHAPE(4, 4, 8) SFC_SHAPE(5, 16, 4)
    SFC_SHAPE(6, 32, 2)
#undef SFC_SHAPE
    default:
      return fullscan_shape<8, 4>(g, grid, cur_mask, dict, N, eoff_all, weights, cm, centres, centre_lin, Q, pick,
                                  cost, st);
  }
}

// The batched full scan into caller-provided scratch (no allocation): lin: Q
// int64; bad: Q bytes; gmin: Q words; tilemin: Q * ceil(N / 1024) floats.
int fullscan_batch_into(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                        const int* eoff_all, const float* weights, int cm, const int32_t* centres, int64_t Q,
                        int64_t* pick, float* cost, int64_t* lin, uint8_t* bad, unsigned int* gmin, float* tilemin,
                        cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  constexpr int EPT = 4;
  const int64_t ntiles = (N + kFsThreads * EPT - 1) / (kFsThreads * EPT);
  const unsigned qb = (unsigned)((Q + 255) / 256);
  count_launch();
  k_centre_lin<<<qb, 256, 0, st>>>(centres, Q, g, lin, status_word());
  count_launch();
  k_centre_fix<<<qb, 256, 0, st>>>(lin, Q, g, bad);
  count_launch();
  k_fill_u32<<<qb, 256, 0, st>>>(gmin, Q, 0x7f800000u);
  int rc = Q >= 8 ? scan_cm<8, EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st)
                   : scan_cm<1, EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, st);
  SFC_CHECK(rc);
  rc = band_cm<EPT>(cm, g, grid, cur_mask, dict, N, eoff_all, weights, lin, Q, tilemin, gmin, ntiles, pick, cost, st);
  SFC_CHECK(rc);
  count_launch();
  k_mark_bad<<<qb, 256, 0, st>>>(bad, Q, pick, cost);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

}  // namespace sfc
