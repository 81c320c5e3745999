// k_proj_tc.cu -- the BF16 precision tier of the projection (Sec. II.A: each
// dictionary patch's subset values projected onto its index's first D
// principal axes), every index at once as one tensor-core GEMM.
//
//   Y (N x C D) = Xc (N x n) Bfull (n x C D),  y = bf16_rn(Y + beta)
//
// Row j of Xc is the whole patch of dictionary entry j (n values, patch raster
// order, channel innermost), centred per element by a common value m_e (the
// element's mean, which every index shares when the means come from the PCA)
// and rounded to BF16; column c D + k of Bfull holds index c's basis column k
// at the rows of its subset's elements, zero elsewhere, in BF16; beta_{c,k}
// = sum_i B_c[i][k] (m_e(i) - mu_c[i]) corrects for means that differ from the
// common centring (exactly zero for a PCA-built basis).  FP32 accumulation in
// TMEM: tcgen05.mma kind::f16 with BF16 operands, M = 128 entries, N = C D
// rounded up to 64, K = 16.  The BF16 results are the stored projections; the
// quantiser's per-axis range comes from them, so the keys are those of the
// stored values.
//
// Producer: the A operand is a gather (patches overlap, so no tensor map can
// address it): all 8 warps load one K-block (64 elements) of 128 entries from
// the grid (L2-resident), centre, round and store it in the 128-byte-swizzled
// K-major layout the MMA reads (16-byte chunk c of row r at chunk c ^ (r & 7)),
// into a 3-stage ring.  One thread issues the block's four K = 16 MMAs and
// commits the stage's "empty" barrier.  After the last block the accumulator
// barrier hands TMEM to the epilogue: warp w reads TMEM lanes 32 (w % 4) .. and
// half of the columns (32 at a time) into shared memory, then the CTA updates
// its per-axis minima / maxima and writes the BF16 projections [C][N][D].
// Every wait is bounded: on timeout the kernel raises ST_TIMEOUT, stops
// issuing, waits (bounded) for the MMAs it issued, frees its TMEM and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace sfc {

namespace {

constexpr int kPM = 128;             // dictionary entries per tile (MMA M)
constexpr int kPK = 64;              // elements per K-block (128 bytes of BF16)
constexpr int kPStages = 3;          // A ring stages
constexpr int kPThreads = 256;
constexpr uint32_t kPStageBytes = kPM * kPK * 2;  // 16 KB
// element-offset table entry of a K position no index reads (offsets relative
// to the patch centre are negative before the centre, so -1 cannot mark it)
constexpr int kNoElem = INT32_MIN;

// D = F32, A = B = BF16, both K-major, M = 128, N = nb
__device__ inline uint32_t idesc_bf16(int nb) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(nb >> 3) << 17) | ((uint32_t)(kPM >> 4) << 24);
}

__device__ inline void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc));
}

// byte offset of element k (0..63) of row r inside a 128-byte-swizzled K-block
__device__ inline uint32_t sw128_off(int r, int k) {
  return (uint32_t)r * 128u + ((((uint32_t)k >> 3) ^ ((uint32_t)r & 7u)) << 4) + ((uint32_t)k & 7u) * 2u;
}

// Monotone float -> uint32 (as in the FP32 projection's range reduction)
__device__ inline uint32_t ord_of_f(float v) {
  if (v == 0.0f) v = 0.0f;
  const uint32_t b = __float_as_uint(v);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

struct PtArgs {
  const float* grid;
  const uint32_t* dict;
  int64_t N;
  int ch, kblocks, nb, CD, D, C;
  int64_t tiles;
  const int* eo;                // kblocks * 64 element offsets (kNoElem: padding or no subset uses it)
  const float* cm;              // kblocks * 64 centring values
  const __nv_bfloat16* Bg;      // nb x (kblocks * 64), K-major
  const float* beta;            // C D
  __nv_bfloat16* proj;          // C x N x D
  uint32_t* lohi;               // 2 C D ordered words
  uint32_t* status;
  uint32_t tmem_cols;           // power of two >= nb
  int b_streamed;               // 1: B does not fit shared memory whole; each stage carries its K-block of B
};

__global__ void __launch_bounds__(kPThreads) k_proj_tc(PtArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const int Kp = a.kblocks * kPK;
  // resident B: kblocks x (nb rows x 128 B), then the stages (A: 16 KB each);
  // streamed B: no resident copy, each stage holds A (16 KB) then its B block
  const uint32_t bblk = (uint32_t)a.nb * 128u;
  const uint32_t stage_bytes = kPStageBytes + (a.b_streamed ? bblk : 0u);
  unsigned char* sB = base;
  unsigned char* sA = sB + (a.b_streamed ? 0 : (size_t)a.kblocks * bblk);
  int* s_eo = reinterpret_cast<int*>(sA + (size_t)kPStages * stage_bytes);  // Kp
  float* s_cm = reinterpret_cast<float*>(s_eo + Kp);                        // Kp
  float* s_beta = s_cm + Kp;                                                // CD
  uint32_t* s_min = reinterpret_cast<uint32_t*>(s_beta + a.CD);             // CD
  uint32_t* s_max = s_min + a.CD;                                           // CD
  int* s_cur = reinterpret_cast<int*>(s_max + a.CD);                        // CD: curve of a column
  int* s_k = s_cur + a.CD;                                                  // CD: axis of a column
  // each row's patch centre in the grid (rows past N take entry 0's: their
  // results are never stored or ranged)
  const float** s_rowp = reinterpret_cast<const float**>(((uintptr_t)(s_k + a.CD) + 7) & ~(uintptr_t)7);  // kPM
  __shared__ uint64_t empty_bar[kPStages], acc_full[2], final_bar;
  __shared__ uint32_t tmem_base;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  // B operand (swizzled like the A blocks), element tables, column tables, ranges
  for (int t = threadIdx.x; t < (a.b_streamed ? 0 : a.kblocks * a.nb * 8); t += kPThreads) {
    const int kb = t / (a.nb * 8), rem = t % (a.nb * 8), row = rem / 8, chunk = rem % 8;
    const uint4 v = *reinterpret_cast<const uint4*>(a.Bg + (size_t)row * Kp + kb * kPK + chunk * 8);
    *reinterpret_cast<uint4*>(sB + (size_t)kb * bblk + sw128_off(row, chunk * 8)) = v;
  }
  for (int t = threadIdx.x; t < Kp; t += kPThreads) {
    s_eo[t] = a.eo[t];
    s_cm[t] = a.cm[t];
  }
  for (int t = threadIdx.x; t < a.CD; t += kPThreads) {
    s_beta[t] = a.beta[t];
    s_min[t] = 0xffffffffu;
    s_max[t] = 0u;
    s_cur[t] = t / a.D;
    s_k[t] = t % a.D;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kPStages; ++s) mbar_init(&empty_bar[s], 1);
    mbar_init(&acc_full[0], 1);
    mbar_init(&acc_full[1], 1);
    mbar_init(&final_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(a.tmem_cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  // the generic-proxy writes of B must be visible to the tensor core's reads
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16(a.nb);
  const int nchunks = (a.CD + 31) / 32;
  const bool vec = 32 % a.D == 0;  // every 32-column chunk holds whole curves
  bool ok = true;
  long long it = 0;  // A ring position over all tiles
  // Software pipeline over this CTA's tiles: iteration L gathers tile L into
  // accumulator buffer L & 1 and issues its MMAs, then drains tile L - 1 (whose
  // MMAs ran during the gather) -- so the MMA latency hides behind the gather.
  for (int L = 0;; ++L) {
    const int64_t t = blockIdx.x + (int64_t)L * gridDim.x;
    const bool have = ok && t < a.tiles;
    if (have) {
      const uint32_t tacc = tmem + (uint32_t)((L & 1) * a.nb);
      for (int r = threadIdx.x; r < kPM; r += kPThreads) {
        const int64_t j = t * kPM + r;
        s_rowp[r] = a.grid + (int64_t)a.dict[j < a.N ? j : 0] * a.ch;
      }
      __syncthreads();
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kPStages);
        bool w = true;
        if (it >= kPStages) w = mbar_wait(&empty_bar[s], (uint32_t)((it / kPStages) - 1) & 1u);
        if (!__syncthreads_and(w)) {
          ok = false;
          break;
        }
        unsigned char* stage = sA + (size_t)s * stage_bytes;
        unsigned char* bstage = a.b_streamed ? stage + kPStageBytes : sB + (size_t)kb * bblk;
        if (a.b_streamed)
          for (int t2 = threadIdx.x; t2 < a.nb * 8; t2 += kPThreads) {
            const int row = t2 / 8, chunk = t2 % 8;
            const uint4 v = *reinterpret_cast<const uint4*>(a.Bg + (size_t)row * Kp + kb * kPK + chunk * 8);
            *reinterpret_cast<uint4*>(bstage + sw128_off(row, chunk * 8)) = v;
          }
        // gather: warp -> rows warp, warp + 8, ...; lane -> elements 2 lane, 2 lane + 1
        const int e0 = kb * kPK + 2 * lane;
        const int oe0 = s_eo[e0], oe1 = s_eo[e0 + 1];
        const float m0 = s_cm[e0], m1 = s_cm[e0 + 1];
        const bool u0 = oe0 != kNoElem, u1 = oe1 != kNoElem;
        const int o0 = u0 ? oe0 : 0, o1 = u1 ? oe1 : 0;  // unused elements read the centre, then give 0
        // rows warp + 8 i share r & 7, hence the swizzled chunk: one offset per thread
        unsigned char* dst0 = stage + sw128_off(warp, 2 * lane);
        float v0[kPM / 8], v1[kPM / 8];
#pragma unroll
        for (int i = 0; i < kPM / 8; ++i) {  // every load of the block in flight at once
          const float* rp = s_rowp[warp + 8 * i];
          v0[i] = __ldg(rp + o0);
          v1[i] = __ldg(rp + o1);
        }
#pragma unroll
        for (int i = 0; i < kPM / 8; ++i) {
          const float x0 = u0 ? __fsub_rn(v0[i], m0) : 0.0f;
          const float x1 = u1 ? __fsub_rn(v1[i], m1) : 0.0f;
          *reinterpret_cast<__nv_bfloat162*>(dst0 + i * 1024) = __floats2bfloat162_rn(x0, x1);  // x0 first
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
          asm volatile("tcgen05.fence::after_thread_sync;");
          const uint32_t a0 = smem_u32(stage), b0 = smem_u32(bstage);
#pragma unroll
          for (int kk = 0; kk < kPK / 16; ++kk)
            mma_bf16(tacc, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32), idesc,
                     (kb > 0 || kk > 0) ? 1u : 0u);
          tc_commit(&empty_bar[s]);
          if (kb == a.kblocks - 1) tc_commit(&acc_full[L & 1]);
        }
      }
    }
    // drain the previous tile: TMEM -> BF16 projections, per-axis ranges
    const int P = L - 1;
    const int64_t tp = blockIdx.x + (int64_t)P * gridDim.x;
    if (ok && P >= 0 && tp < a.tiles) {
      const bool w = mbar_wait(&acc_full[P & 1], (uint32_t)(P >> 1) & 1u);
      if (!__syncthreads_and(w)) {
        ok = false;
      } else {
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int q = warp & 3;  // TMEM lanes 32 q .. 32 q + 31 = rows of the tile
        const int64_t row = tp * kPM + q * 32 + lane;
        const bool valid = row < a.N;
        const uint32_t tbuf = tmem + (uint32_t)((P & 1) * a.nb) + ((uint32_t)(q * 32) << 16);
        for (int j = warp >> 2; j < nchunks; j += 2) {  // warp-uniform
          uint32_t v[32];
          tmem_ld32(tbuf + 32 * j, v);
          asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
          const int col0 = 32 * j;
          uint32_t yb[16];  // the 32 columns' BF16 results, in pairs
#pragma unroll
          for (int i = 0; i < 32; i += 2) {
            const int c = col0 + i;
            const float f0 = c < a.CD ? __fadd_rn(__uint_as_float(v[i]), s_beta[c]) : 0.0f;
            const float f1 = c + 1 < a.CD ? __fadd_rn(__uint_as_float(v[i + 1]), s_beta[c + 1]) : 0.0f;
            const __nv_bfloat162 h = __floats2bfloat162_rn(f0, f1);
            yb[i / 2] = *reinterpret_cast<const uint32_t*>(&h);
          }
          if (valid) {
            if (vec) {
              // whole curves: vector stores of each curve's D values
#define SFC_OUT(cs) (a.proj + ((int64_t)s_cur[col0 + (cs) * a.D] * a.N + row) * a.D)
              switch (a.D) {
                case 16:
#pragma unroll
                  for (int cs = 0; cs < 2; ++cs)
                    if (col0 + cs * 16 < a.CD) {
                      uint4* o = reinterpret_cast<uint4*>(SFC_OUT(cs));
                      o[0] = make_uint4(yb[8 * cs], yb[8 * cs + 1], yb[8 * cs + 2], yb[8 * cs + 3]);
                      o[1] = make_uint4(yb[8 * cs + 4], yb[8 * cs + 5], yb[8 * cs + 6], yb[8 * cs + 7]);
                    }
                  break;
                case 8:
#pragma unroll
                  for (int cs = 0; cs < 4; ++cs)
                    if (col0 + cs * 8 < a.CD)
                      *reinterpret_cast<uint4*>(SFC_OUT(cs)) =
                          make_uint4(yb[4 * cs], yb[4 * cs + 1], yb[4 * cs + 2], yb[4 * cs + 3]);
                  break;
                case 4:
#pragma unroll
                  for (int cs = 0; cs < 8; ++cs)
                    if (col0 + cs * 4 < a.CD) *reinterpret_cast<uint2*>(SFC_OUT(cs)) = make_uint2(yb[2 * cs], yb[2 * cs + 1]);
                  break;
                case 2:
#pragma unroll
                  for (int cs = 0; cs < 16; ++cs)
                    if (col0 + cs * 2 < a.CD) *reinterpret_cast<uint32_t*>(SFC_OUT(cs)) = yb[cs];
                  break;
                default:  // D == 1
#pragma unroll
                  for (int cs = 0; cs < 32; ++cs)
                    if (col0 + cs < a.CD)
                      *reinterpret_cast<unsigned short*>(SFC_OUT(cs)) = (unsigned short)(yb[cs / 2] >> (16 * (cs & 1)));
                  break;
              }
#undef SFC_OUT
            } else {
#pragma unroll
              for (int i = 0; i < 32; ++i) {
                const int c = col0 + i;
                if (c < a.CD)
                  *reinterpret_cast<unsigned short*>(a.proj + ((int64_t)s_cur[c] * a.N + row) * a.D + s_k[c]) =
                      (unsigned short)(yb[i / 2] >> (16 * (i & 1)));
              }
            }
          }
          // the columns' ranges over the warp's 32 rows
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const int c = col0 + i;
            if (c < a.CD) {  // warp-uniform
              const float y = __uint_as_float((i & 1) ? (yb[i / 2] & 0xffff0000u) : (yb[i / 2] << 16));
              const uint32_t u = ord_of_f(y);
              uint32_t lo = valid ? u : 0xffffffffu, hi = valid ? u : 0u;
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
              }
              if (lane == 0) {
                atomicMin(&s_min[c], lo);
                atomicMax(&s_max[c], hi);
              }
            }
          }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
      }
    }
    if (!have) break;
  }
  // ranges of this CTA
  if (ok)
    for (int t = threadIdx.x; t < a.CD; t += kPThreads) {
      atomicMin(&a.lohi[2 * t], s_min[t]);
      atomicMax(&a.lohi[2 * t + 1], s_max[t]);
    }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!ok) atomicOr(a.status, ST_TIMEOUT);
    // every MMA issued above has completed before the TMEM and shared memory go
    tc_commit(&final_bar);
    if (!mbar_wait(&final_bar, 0)) atomicOr(a.status, ST_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols));
  }
}

// Operand and table preparation: Bfull (nb x Kp BF16, zero-filled by the
// caller) from every index's basis, the common centring m_e (the mean of the
// first index using element e), and beta_{c,k} = sum_i B_c[i][k] (m_e(i) -
// mu_c[i]) as an FP32 multiply-add chain in subset order.
__global__ void k_pt_prep(const float* __restrict__ basis, const float* __restrict__ mean,
                          const int* __restrict__ elem, const int* __restrict__ first, int C, int s, int D, int Kp,
                          __nv_bfloat16* __restrict__ Bg, float* __restrict__ cm, float* __restrict__ beta) {
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
  for (int t = tid; t < C * s * D; t += nth) {
    const int c = t / (s * D), i = (t / D) % s, k = t % D;
    Bg[(size_t)(c * D + k) * Kp + elem[c * s + i]] = __float2bfloat16_rn(basis[t]);
  }
  for (int e = tid; e < Kp; e += nth) cm[e] = first[e] >= 0 ? mean[first[e]] : 0.0f;
  for (int t = tid; t < C * D; t += nth) {
    const int c = t / D, k = t % D;
    float acc = 0.0f;
    for (int i = 0; i < s; ++i) {
      const float me = mean[first[elem[c * s + i]]];
      acc = __fmaf_rn(basis[((size_t)c * s + i) * D + k], __fsub_rn(me, mean[(size_t)c * s + i]), acc);
    }
    beta[t] = acc;
  }
}

}  // namespace

int project_bf16(Index& ix, const float* grid, void* proj, uint32_t* lohi, cudaStream_t st) {
  const Geo& g = ix.g;
  const int n = g.n, C = ix.C, D = ix.D, s = ix.s, m = ix.m, ch = g.ch;
  const int kblocks = (n + kPK - 1) / kPK, Kp = kblocks * kPK;
  const int CD = C * D;
  const int nb = (CD + 63) / 64 * 64;
  if (nb > 256) {
    set_error("the BF16 projection takes C * D <= 256 (curves * dims)");
    return SFC_EUNSUPPORTED;
  }
  // host tables: the patch element of every subset value, the first (index,
  // value) using each element, and the element offsets the gather reads
  // (kNoElem: padding, or an element no subset uses)
  std::vector<int> elem((size_t)C * s), first(Kp, -1), eo(Kp, kNoElem);
  for (int c = 0; c < C; ++c)
    for (int i = 0; i < s; ++i) {
      const int e = ix.subset_h[(size_t)c * m + i / ch] * ch + i % ch;
      elem[(size_t)c * s + i] = e;
      if (first[e] < 0) first[e] = c * s + i;
    }
  for (int e = 0; e < n; ++e)
    if (first[e] >= 0) eo[e] = (int)(patch_off(g, e / ch) * ch + e % ch);
  Scratch scr(st);
  int *d_elem = nullptr, *d_first = nullptr, *d_eo = nullptr;
  __nv_bfloat16* Bg = nullptr;
  float *cm = nullptr, *beta = nullptr;
  SFC_TRY(scr.alloc(&d_elem, sizeof(int) * elem.size()));
  SFC_TRY(scr.alloc(&d_first, sizeof(int) * Kp));
  SFC_TRY(scr.alloc(&d_eo, sizeof(int) * Kp));
  SFC_TRY(scr.alloc(&Bg, sizeof(__nv_bfloat16) * (size_t)nb * Kp));
  SFC_TRY(scr.alloc(&cm, sizeof(float) * Kp));
  SFC_TRY(scr.alloc(&beta, sizeof(float) * CD));
  SFC_TRY(cudaMemcpyAsync(d_elem, elem.data(), sizeof(int) * elem.size(), cudaMemcpyHostToDevice, st));
  SFC_TRY(cudaMemcpyAsync(d_first, first.data(), sizeof(int) * Kp, cudaMemcpyHostToDevice, st));
  SFC_TRY(cudaMemcpyAsync(d_eo, eo.data(), sizeof(int) * Kp, cudaMemcpyHostToDevice, st));
  SFC_TRY(cudaMemsetAsync(Bg, 0, sizeof(__nv_bfloat16) * (size_t)nb * Kp, st));
  count_launch();
  k_pt_prep<<<64, 256, 0, st>>>(ix.basis, ix.mean, d_elem, d_first, C, s, D, Kp, Bg, cm, beta);
  SFC_TRY(cudaGetLastError());
  SFC_CHECK(lohi_init(lohi, CD, st));
  // launch: one or two CTAs per SM (by shared memory), persistent over tiles
  const size_t tables = (size_t)Kp * 8 + (size_t)CD * 20 + 8 + kPM * 8;
  size_t shm = 1024 + (size_t)kblocks * nb * 128 + (size_t)kPStages * kPStageBytes + tables;
  int streamed = 0;
  if (shm > 227 * 1024) {  // B streamed through the stages with A
    streamed = 1;
    shm = 1024 + (size_t)kPStages * (kPStageBytes + (size_t)nb * 128) + tables;
  }
  if (shm > 227 * 1024) {
    set_error("the BF16 projection's operands do not fit shared memory (patch too large)");
    return SFC_EUNSUPPORTED;
  }
  SFC_TRY(cudaFuncSetAttribute(k_proj_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  SFC_TRY(cudaFuncSetAttribute(k_proj_tc, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int dev = 0, sms = 0, per_sm = 0;
  SFC_TRY(cudaGetDevice(&dev));
  SFC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // two CTAs per SM when their shared memory fits (one CTA's gather then
  // overlaps the other's waits); TMEM below
  per_sm = 2 * (shm + 2048) <= 233472 ? 2 : 1;
  PtArgs a;
  a.grid = grid;
  a.dict = ix.dict;
  a.N = ix.N;
  a.ch = ch;
  a.kblocks = kblocks;
  a.nb = nb;
  a.CD = CD;
  a.D = D;
  a.C = C;
  a.tiles = (ix.N + kPM - 1) / kPM;
  a.eo = d_eo;
  a.cm = cm;
  a.Bg = Bg;
  a.beta = beta;
  a.proj = static_cast<__nv_bfloat16*>(proj);
  a.lohi = lohi;
  a.status = status_word();
  // TMEM columns: two accumulator buffers of nb columns (the epilogue reads
  // 32-column chunks below round_up(C D, 32) <= nb of a buffer)
  uint32_t cols = 32;
  while (cols < (uint32_t)(2 * nb)) cols <<= 1;
  a.tmem_cols = cols;
  per_sm = std::min(per_sm, (int)(512 / cols));  // every CTA on an SM holds its columns at once
  a.b_streamed = streamed;
  const int64_t grid_n = std::min<int64_t>(a.tiles, (int64_t)sms * per_sm);
  // the method's work: N C s D multiply-adds; its bytes: the patch values
  // gathered (N n FP32) and the BF16 projections written
  ix.proj_flops = 2.0 * (double)ix.N * C * s * D;
  ix.proj_bytes = (double)ix.N * n * 4.0 + (double)ix.N * CD * 2.0;
  if (ix.ev_proj[0]) cudaEventRecord(ix.ev_proj[0], st);
  if (grid_n > 0) {
    count_launch();
    k_proj_tc<<<(unsigned)grid_n, kPThreads, shm, st>>>(a);
    SFC_TRY(cudaGetLastError());
  }
  if (ix.ev_proj[1]) cudaEventRecord(ix.ev_proj[1], st);
  return lohi_to_scale(ix, lohi, st);
}

}  // namespace sfc
