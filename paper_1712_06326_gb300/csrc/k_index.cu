// k_index.cu -- projection to principal space (Sec. II.A), quantisation and
// Morton / z-address keys (Sec. II.C) of every dictionary entry on every index.
//
// Projection: y_k = chain of FP32 fused multiply-adds over the index's subset
// values in subset order, acc = fma(B[i][k], x_i - mu_i, acc) starting at +0 with
// x_i - mu_i rounded to FP32 (a thread runs the D chains of 4 entries of one
// index, interleaved, two axes per fma.rn.f32x2: the same IEEE operation on
// each half).  The per-axis minimum and maximum over the dictionary are
// exact reductions (order-independent).  Quantisation: q = clamp(floor((y - lo)
// * scale), 0, 2^b - 1) with scale = (float)(2^b / ((double)hi - (double)lo)) (0
// if hi == lo), then q + shift.  Key: bits interleaved highest plane first,
// dimension 0 first inside a plane (the highest-variance axis first, Sec. II.C);
// the top 64 bits when D * b' > 64.
#include <cuda_bf16.h>

#include "internal.cuh"

namespace sfc {

namespace {

// Monotone map float -> uint32 so that unsigned min/max order like the floats;
// -0 is folded to +0 first (both are the real value zero).
__device__ inline uint32_t ord_of(float v) {
  if (v == 0.0f) v = 0.0f;
  uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ inline float float_of(uint32_t u) {
  uint32_t b = (u & 0x80000000u) ? (u & 0x7fffffffu) : ~u;
  return __uint_as_float(b);
}

constexpr int kPE = 4;  // dictionary entries per thread (they share the basis reads)

// dims paired: acc2[q][h] holds the chains of axes 2h, 2h + 1 of entry q; the
// basis row pair (B[i][2h], B[i][2h+1]) is read as one 64-bit word and the
// centred value is duplicated into both halves (the same IEEE FMA per half)
template <int D>
__global__ void __launch_bounds__(256) k_project(const float* __restrict__ grid, const uint32_t* __restrict__ dict,
                                                 int64_t N, int ch, int s, const int* __restrict__ sub_eoff,
                                                 const float* __restrict__ basis, const float* __restrict__ mean,
                                                 float* __restrict__ proj, uint32_t* __restrict__ lohi, int c0) {
  constexpr int DP = (D + 1) / 2;
  const int c = c0 + blockIdx.y;
  extern __shared__ unsigned char smem_raw[];
  unsigned long long* B2 = reinterpret_cast<unsigned long long*>(smem_raw);  // s * DP pairs
  float* mu = reinterpret_cast<float*>(B2 + s * DP);                         // s
  int* eo = reinterpret_cast<int*>(mu + s);                                  // s
  for (int t = threadIdx.x; t < s * DP; t += blockDim.x) {
    const int i = t / DP, h = t % DP;
    const float b0 = basis[(int64_t)c * s * D + i * D + 2 * h];
    const float b1 = 2 * h + 1 < D ? basis[(int64_t)c * s * D + i * D + 2 * h + 1] : 0.0f;
    B2[t] = f2_pack(b0, b1);
  }
  for (int t = threadIdx.x; t < s; t += blockDim.x) {
    mu[t] = mean[(int64_t)c * s + t];
    eo[t] = sub_eoff[(int64_t)c * s + t];
  }
  __shared__ uint32_t smin[D], smax[D];
  if (threadIdx.x < D) {
    smin[threadIdx.x] = 0xffffffffu;
    smax[threadIdx.x] = 0u;
  }
  __syncthreads();
  const int64_t j0 = (int64_t)blockIdx.x * blockDim.x * kPE + threadIdx.x;
  const float* gp[kPE];
  bool ok[kPE];
#pragma unroll
  for (int q = 0; q < kPE; ++q) {
    const int64_t j = j0 + (int64_t)q * blockDim.x;
    ok[q] = j < N;
    gp[q] = grid + (int64_t)dict[ok[q] ? j : 0] * ch;
  }
  unsigned long long acc2[kPE][DP];
#pragma unroll
  for (int q = 0; q < kPE; ++q)
#pragma unroll
    for (int h = 0; h < DP; ++h) acc2[q][h] = 0ull;
#pragma unroll 2
  for (int i = 0; i < s; ++i) {
    const int o = eo[i];
    const float m = mu[i];
    unsigned long long xc2[kPE];
#pragma unroll
    for (int q = 0; q < kPE; ++q) {
      const float x = __fsub_rn(gp[q][o], m);
      xc2[q] = f2_pack(x, x);
    }
#pragma unroll
    for (int h = 0; h < DP; ++h) {
      const unsigned long long b2 = B2[i * DP + h];
#pragma unroll
      for (int q = 0; q < kPE; ++q) acc2[q][h] = f2_fma(b2, xc2[q], acc2[q][h]);
    }
  }
  float acc[kPE][D];
#pragma unroll
  for (int q = 0; q < kPE; ++q)
#pragma unroll
    for (int h = 0; h < DP; ++h) {
      float lo, hi;
      f2_unpack(acc2[q][h], lo, hi);
      acc[q][2 * h] = lo;
      if (2 * h + 1 < D) acc[q][2 * h + 1] = hi;
    }
#pragma unroll
  for (int q = 0; q < kPE; ++q)
    if (ok[q]) {
      float* out = proj + ((int64_t)c * N + j0 + (int64_t)q * blockDim.x) * D;
#pragma unroll
      for (int k = 0; k < D; ++k) out[k] = acc[q][k];
    }
  // per-axis min / max: warp reduce, then shared, then one global atomic per axis
#pragma unroll
  for (int k = 0; k < D; ++k) {
    uint32_t u = 0xffffffffu, v = 0u;
#pragma unroll
    for (int q = 0; q < kPE; ++q)
      if (ok[q]) {
        const uint32_t w = ord_of(acc[q][k]);
        u = min(u, w);
        v = max(v, w);
      }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      u = min(u, __shfl_xor_sync(0xffffffffu, u, o));
      v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&smin[k], u);
      atomicMax(&smax[k], v);
    }
  }
  __syncthreads();
  if (threadIdx.x < D) {
    atomicMin(&lohi[(c * D + threadIdx.x) * 2 + 0], smin[threadIdx.x]);
    atomicMax(&lohi[(c * D + threadIdx.x) * 2 + 1], smax[threadIdx.x]);
  }
}

__global__ void k_lohi_init(uint32_t* lohi, int n) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    lohi[2 * t] = 0xffffffffu;
    lohi[2 * t + 1] = 0u;
  }
}

__global__ void k_scale(const uint32_t* __restrict__ lohi, int n, int bits, float* __restrict__ lo,
                        float* __restrict__ scale) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) {
    float l = float_of(lohi[2 * t]), h = float_of(lohi[2 * t + 1]);
    lo[t] = l;
    scale[t] = h > l ? (float)(ldexp(1.0, bits) / ((double)h - (double)l)) : 0.0f;
  }
}

}  // namespace

namespace {

// projections are FP32, or BF16 (the precision tier) widened exactly to FP32
__device__ inline float proj_f(float v) { return v; }
__device__ inline float proj_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <int D, typename T>
__global__ void k_keys(const T* __restrict__ proj, int64_t N, int bits, int bp, int curve,
                       const float* __restrict__ lo, const float* __restrict__ scale,
                       const int32_t* __restrict__ shifts, uint64_t* __restrict__ keys, int c0) {
  const int c = c0 + blockIdx.y;
  const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= N) return;
  uint32_t q[D];
  const T* y = proj + ((int64_t)c * N + j) * D;
#pragma unroll
  for (int k = 0; k < D; ++k)
    q[k] = quantise_one(proj_f(y[k]), lo[c * D + k], scale[c * D + k], bits) + (uint32_t)shifts[c * D + k];
  keys[(int64_t)c * N + j] = curve == SFC_CURVE_HILBERT ? hilbert_key_t<D>(q, bp) : morton_key_t<D>(q, bp);
}

// sqc[c][i][k] = quantised shifted coordinate k of the entry at sorted slot i of index c
template <typename T>
__global__ void k_sorted_coords(const T* __restrict__ proj, const uint32_t* __restrict__ sids, int64_t N, int D,
                                int bits, const float* __restrict__ lo, const float* __restrict__ scale,
                                const int32_t* __restrict__ shifts, uint32_t* __restrict__ sqc) {
  const int c = blockIdx.y;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= N * D) return;
  const int64_t i = t / D;
  const int k = (int)(t - i * D);
  const int64_t j = sids[(int64_t)c * N + i];
  const float y = proj_f(proj[((int64_t)c * N + j) * D + k]);
  sqc[(int64_t)c * N * D + t] = quantise_one(y, lo[c * D + k], scale[c * D + k], bits) + (uint32_t)shifts[c * D + k];
}

template <int D>
int launch_project(Index& ix, const float* grid, float* proj, uint32_t* lohi, int c0, int nc,
                   cudaStream_t st) {
  const size_t shm = sizeof(unsigned long long) * ix.s * ((D + 1) / 2) + sizeof(float) * ix.s + sizeof(int) * ix.s;
  if (shm > kSmemOptIn) SFC_TRY(cudaFuncSetAttribute(k_project<D>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  dim3 grd((unsigned)((ix.N + 256 * kPE - 1) / (256 * kPE)), nc);
  // traced builds: events around the projection launches (from the first
  // curve's to the last one's), and the launches' algorithmic work
  if (c0 == 0 && ix.ev_proj[0]) {
    ix.proj_flops = 2.0 * (double)ix.N * ix.C * ix.s * D;
    ix.proj_bytes = (double)ix.N * ix.C * ix.s * 4.0 + (double)ix.N * ix.C * D * 4.0;
    cudaEventRecord(ix.ev_proj[0], st);
  }
  count_launch();
  k_project<D><<<grd, 256, shm, st>>>(grid, ix.dict, ix.N, ix.g.ch, ix.s, ix.sub_eoff, ix.basis, ix.mean, proj, lohi,
                                      c0);
  SFC_TRY(cudaGetLastError());
  if (c0 + nc == ix.C && ix.ev_proj[1]) cudaEventRecord(ix.ev_proj[1], st);
  return SFC_OK;
}

template <int D>
int launch_keys(const Index& ix, const float* proj, uint64_t* keys, int c0, int nc, cudaStream_t st) {
  dim3 grd((unsigned)((ix.N + 255) / 256), nc);
  count_launch();
  if (ix.bf16)
    k_keys<D, __nv_bfloat16><<<grd, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(proj), ix.N, ix.bits,
                                                   ix.bp, ix.curve, ix.lo, ix.scale, ix.shifts, keys, c0);
  else
    k_keys<D, float><<<grd, 256, 0, st>>>(proj, ix.N, ix.bits, ix.bp, ix.curve, ix.lo, ix.scale, ix.shifts, keys,
                                          c0);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

}  // namespace

int project_curves(Index& ix, const float* grid, float* proj, uint32_t* lohi, int c0, int nc, cudaStream_t st) {
  const int n = nc * ix.D;
  uint32_t* lh = lohi + 2 * (size_t)c0 * ix.D;
  count_launch();
  k_lohi_init<<<(n + 127) / 128, 128, 0, st>>>(lh, n);
  int rc = SFC_EINVAL;
  switch (ix.D) {
#define SFC_D(d) \
  case d: rc = launch_project<d>(ix, grid, proj, lohi, c0, nc, st); break;
    SFC_D(1) SFC_D(2) SFC_D(3) SFC_D(4) SFC_D(5) SFC_D(6) SFC_D(7) SFC_D(8)
    SFC_D(9) SFC_D(10) SFC_D(11) SFC_D(12) SFC_D(13) SFC_D(14) SFC_D(15) SFC_D(16)
#undef SFC_D
    default: set_error("dims must be 1..16"); return SFC_EINVAL;
  }
  SFC_CHECK(rc);
  count_launch();
  k_scale<<<(n + 127) / 128, 128, 0, st>>>(lh, n, ix.bits, ix.lo + (size_t)c0 * ix.D, ix.scale + (size_t)c0 * ix.D);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

int lohi_init(uint32_t* lohi, int n, cudaStream_t st) {
  count_launch();
  k_lohi_init<<<(n + 127) / 128, 128, 0, st>>>(lohi, n);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

int lohi_to_scale(Index& ix, const uint32_t* lohi, cudaStream_t st) {
  const int n = ix.C * ix.D;
  count_launch();
  k_scale<<<(n + 127) / 128, 128, 0, st>>>(lohi, n, ix.bits, ix.lo, ix.scale);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

int key_curves(Index& ix, const float* proj, uint64_t* keys, int c0, int nc, cudaStream_t st) {
  int rc = SFC_EINVAL;
  switch (ix.D) {
#define SFC_D(d) \
  case d: rc = launch_keys<d>(ix, proj, keys, c0, nc, st); break;
    SFC_D(1) SFC_D(2) SFC_D(3) SFC_D(4) SFC_D(5) SFC_D(6) SFC_D(7) SFC_D(8)
    SFC_D(9) SFC_D(10) SFC_D(11) SFC_D(12) SFC_D(13) SFC_D(14) SFC_D(15) SFC_D(16)
#undef SFC_D
    default: set_error("dims must be 1..16"); return SFC_EINVAL;
  }
  return rc;
}

int sorted_coords(Index& ix, const float* proj, cudaStream_t st) {
  SFC_TRY(pmalloc(&ix.sqc, sizeof(uint32_t) * ix.C * ix.N * ix.D, st));
  dim3 grd((unsigned)((ix.N * ix.D + 255) / 256), ix.C);
  count_launch();
  if (ix.bf16)
    k_sorted_coords<__nv_bfloat16><<<grd, 256, 0, st>>>(reinterpret_cast<const __nv_bfloat16*>(proj), ix.sids, ix.N,
                                                        ix.D, ix.bits, ix.lo, ix.scale, ix.shifts, ix.sqc);
  else
    k_sorted_coords<float><<<grd, 256, 0, st>>>(proj, ix.sids, ix.N, ix.D, ix.bits, ix.lo, ix.scale, ix.shifts,
                                                ix.sqc);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

}  // namespace sfc
