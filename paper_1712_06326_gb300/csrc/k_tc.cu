// k_tc.cu -- the full scan's pre-score as a tensor-core GEMM (tcgen05, sm_103a).
//
// The masked cost expands as cost(q, j) = sum m w t'^2 - 2 sum m w t' p'_j +
// sum m w p'_j^2 (values centred per channel), so the pre-score
//     s(q, j) = sum_e [ (-2 m w t')_e p'_je + (m w)_e (p'_je)^2 ]
// is a dot product of a query row a(q) = [-2 m w t' ; m w] with a dictionary row
// b(j) = [p' ; p'^2] and differs from the cost by a per-query constant: a GEMM
// when many queries share the dictionary.  FP16 operands with FP32 accumulation;
// every operand is split into a high and a low FP16 part and the three leading
// products are laid out along K as [lo*hi | hi*lo | hi*hi], six parts of n8
// (n rounded up to 8) values each: the small products are accumulated first,
// while the accumulator is still small, and the hi*hi products are shared
// between two TMEM accumulators (K-blocks before / after kb_split) that the
// epilogue adds; the certified bound charges each product for the K positions
// that follow it in its accumulator (see k_tc_prep_A).
//
// Kernel structure (one 128 x 256 output tile per CTA): warp 0 issues TMA loads
// (128-byte swizzle) of the A and B K-slices into a 4-stage shared-memory ring;
// warp 1 allocates 512 TMEM columns and issues tcgen05.mma (M = 128, N = 256,
// K = 16) from one thread, committing each stage back to its "empty" barrier;
// warps 2-5 wait for the last commit, read their 32 TMEM lanes each with
// tcgen05.ld, add the two accumulators and write the minimum pre-score of their
// row over every 32 columns (valid columns only).  Every wait is bounded: on
// timeout the CTA raises ST_TIMEOUT and a launch-wide abort flag (CTAs that
// start later skip their tile), drains what it issued (again bounded), frees its
// TMEM and returns.
#include <cuda.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.cuh"
#include "tc_ptx.cuh"

namespace sfc {

namespace {

constexpr int kBM = 128, kBN = 256, kBK = 64, kStages = 4;
constexpr int kTcThreads = 192;
constexpr uint32_t kStageA = kBM * kBK * 2, kStageB = kBN * kBK * 2;  // bytes
// Instruction descriptor: D = F32, A = B = F16, both K-major, N = 256, M = 128.
constexpr uint32_t kIdesc = (1u << 4) | (0u << 7) | (0u << 10) | ((uint32_t)(kBN >> 3) << 17) |
                            ((uint32_t)(kBM >> 4) << 24);

__device__ inline void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(acc));
}
struct TcArgs {
  int64_t Q, N;        // real rows of A / of this launch's B (a chunk of the dictionary)
  int64_t n0;          // first dictionary entry of the chunk (a multiple of 256)
  int64_t Nt;          // entries of the whole dictionary (row stride of scores)
  int kblocks;         // Kp / 64
  int kb_split;        // first K-block of the second accumulator (== kblocks: none)
  int64_t mtiles;      // 128-row query tiles
  int64_t tiles;       // mtiles * ceil(N / 256)
  int64_t nsub;        // 32-column groups per query row of submin (8 per tile)
  float* submin;       // [Q][nsub] minimum over each 32 dictionary entries
  float* scores;       // optional [Q][N] (checking only)
  uint32_t* status;
  int* abort_all;      // set by a CTA that timed out; the others stop at their next tile
};

// Persistent: CTA b takes the tiles b, b + gridDim.x, ...; tile t covers query
// rows 128 (t % mtiles) .. and dictionary entries 256 (t / mtiles) .., so CTAs
// running at the same time share dictionary tiles (read from HBM once, then
// from L2).  The stage ring and its phases run on across tiles, so the
// producer prefetches the next tile while the epilogue drains the current one;
// the MMA issuer waits for the epilogue to release the accumulators.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_gemm(const __grid_constant__ CUtensorMap mapA,
                                                           const __grid_constant__ CUtensorMap mapB, TcArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned stage buffers (the swizzle pattern repeats every 1024 B)
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = base;                      // kStages * kStageA
  unsigned char* sB = base + kStages * kStageA;  // kStages * kStageB
  __shared__ uint64_t full_bar[kStages], empty_bar[kStages], acc_full, acc_empty, final_bar;
  __shared__ uint32_t tmem_base;
  __shared__ int abort_flag;
  __shared__ long long s_issued, s_consumed;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], 1);
    }
    mbar_init(&acc_full, 1);
    mbar_init(&acc_empty, 4);  // one arrival per epilogue warp
    mbar_init(&final_bar, 1);
    abort_flag = 0;
    s_issued = 0;
    s_consumed = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_base;
  // stop_here: this CTA's flag (shared memory, checked per K-block); stop: also
  // the launch-wide flag (a global load, checked once per tile)
  auto stop_here = [&]() { return *(volatile int*)&abort_flag != 0; };
  auto stop = [&]() { return stop_here() || *(volatile int*)a.abort_all != 0; };
  auto fail = [&]() {
    atomicExch(&abort_flag, 1);
    atomicExch(a.abort_all, 1);
  };

  if (warp == 0 && lane == 0) {
    // producer: ring position it -> stage it % kStages, phase (it / kStages) & 1
    long long it = 0;
    for (int64_t t = blockIdx.x; t < a.tiles && !stop(); t += gridDim.x) {
      const int m_tile = (int)(t % a.mtiles), n_tile = (int)(t / a.mtiles);
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kStages);
        if (it >= kStages && !mbar_wait(&empty_bar[s], (uint32_t)((it / kStages) - 1) & 1)) {
          fail();
          break;
        }
        if (stop_here()) break;
        mbar_expect_tx(&full_bar[s], kStageA + kStageB);
        tma_load_2d(sA + s * kStageA, &mapA, kb * kBK, m_tile * kBM, &full_bar[s]);
        tma_load_2d(sB + s * kStageB, &mapB, kb * kBK, n_tile * kBN, &full_bar[s]);
        s_issued = it + 1;
      }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    long long it = 0;
    int local = 0;
    for (int64_t t = blockIdx.x; t < a.tiles && !stop(); t += gridDim.x, ++local) {
      if (local > 0 && !mbar_wait(&acc_empty, (uint32_t)(local - 1) & 1)) {
        fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      bool ok = true;
      for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
        const int s = (int)(it % kStages);
        if (!mbar_wait(&full_bar[s], (uint32_t)(it / kStages) & 1) || stop_here()) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        const uint32_t a0 = smem_u32(sA + s * kStageA), b0 = smem_u32(sB + s * kStageB);
        const bool second = kb >= a.kb_split;
        const uint32_t d = tmem + (second ? 256u : 0u);
        const bool first_block = kb == 0 || kb == a.kb_split;
#pragma unroll
        for (int kk = 0; kk < kBK / 16; ++kk) {
          // a K step of 16 FP16 = 32 bytes inside the 128-byte swizzled rows
          tc_mma(d, smem_desc_sw128(a0 + kk * 32), smem_desc_sw128(b0 + kk * 32),
                 (first_block && kk == 0) ? 0u : 1u);
        }
        tc_commit(&empty_bar[s]);
        s_consumed = it + 1;
      }
      if (!ok) {
        fail();
        break;
      }
      tc_commit(&acc_full);  // arrives when this tile's MMAs have completed
    }
    tc_commit(&final_bar);  // every MMA issued above has completed
    if (!mbar_wait(&final_bar, 0)) fail();
  } else if (warp >= 2) {
    // epilogue warps 2..5: TMEM lanes 32 * (warp % 4) ..
    const int quarter = warp & 3;
    const bool two = a.kb_split < a.kblocks;
    int local = 0;
    for (int64_t t = blockIdx.x; t < a.tiles; t += gridDim.x, ++local) {
      const int m_tile = (int)(t % a.mtiles), n_tile = (int)(t / a.mtiles);
      // warp-uniform outcome (tcgen05.ld below is a whole-warp instruction)
      const bool ok = __all_sync(0xffffffffu, !stop() && mbar_wait(&acc_full, (uint32_t)local & 1));
      if (!ok) {
        if (lane == 0) fail();
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;");
      const int64_t row = (int64_t)m_tile * kBM + quarter * 32 + lane;
      const int64_t col0 = (int64_t)n_tile * kBN;
      float mins[kBN / 32];
#pragma unroll
      for (int c = 0; c < kBN; c += 32) {
        uint32_t r[32], r2[32];
        const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c;
        tmem_ld32(taddr, r);
        if (two) tmem_ld32(taddr + 256u, r2);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        float mn = INFINITY;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const int64_t col = col0 + c + i;
          const float v = two ? __fadd_rn(__uint_as_float(r[i]), __uint_as_float(r2[i])) : __uint_as_float(r[i]);
          if (col < a.N) {
            mn = fminf(mn, v);
            if (a.scores && row < a.Q) a.scores[row * a.Nt + a.n0 + col] = v;
          }
        }
        mins[c / 32] = mn;
      }
      // the accumulators are free once every lane's loads are done
      asm volatile("tcgen05.fence::before_thread_sync;");
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&acc_empty)) : "memory");
      if (row < a.Q) {
        float4* dst =
            reinterpret_cast<float4*>(a.submin + row * a.nsub + (a.n0 + (int64_t)n_tile * kBN) / 32);
        dst[0] = make_float4(mins[0], mins[1], mins[2], mins[3]);
        dst[1] = make_float4(mins[4], mins[5], mins[6], mins[7]);
      }
    }
  }
  __syncwarp();
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (threadIdx.x == 0) {
    if (abort_flag) atomicOr(a.status, ST_TIMEOUT);
    // after a stop (here or in another CTA): drain the TMA loads issued but
    // not consumed (bounded) before the shared memory is released
    for (long long it = s_consumed; it < s_issued; ++it)
      mbar_wait(&full_bar[it % kStages], (uint32_t)(it / kStages) & 1);
  }
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ----------------------------------------------------------------------------
// operand rows
// ----------------------------------------------------------------------------
__device__ inline void split16(float v, __half& hi, __half& lo) {
  hi = __float2half_rn(v);
  lo = __float2half_rn(v - __half2float(hi));
}

// Layout of K (n8 = n rounded up to 8; part stride n8, zeros past n in each
// part and past 6 n8 up to Kp):
//   A row of query q:      [a1l a2l | a1h a2h | a1h a2h]   a1 = -2 m w t', a2 = m w
//   B row of entry j:      [b1h b2h | b1l b2l | b1h b2h]   b1 = p', b2 = p'^2
// so parts 0-3 hold the small cross products lo*hi and hi*lo, parts 4-5 the
// hi*hi products.  K-blocks [0, kb_split) accumulate in TMEM columns 0..255,
// the rest in columns 256..511.
struct TcLayout {
  int n8, Kp, kblocks, kb_split;
};
inline TcLayout tc_layout(int n) {
  TcLayout L;
  L.n8 = (n + 7) / 8 * 8;
  L.Kp = (6 * L.n8 + kBK - 1) / kBK * kBK;
  L.kblocks = L.Kp / kBK;
  // the two accumulators take about half of the hi*hi products each
  L.kb_split = std::min(L.kblocks, (5 * L.n8 + kBK / 2) / kBK);
  if (L.kb_split < 1) L.kb_split = L.kblocks;
  return L;
}

// bound[q] = E_q >= |s_hat(q, j) - s(q, j)| for every dictionary row j, with
// |p'| <= pmax[c], u16 = 2^-11, u32 = 2^-24:
//  * operand splitting: a = ah + al + da with |da| <= u16^2 |a| + 2^-25 (the
//    low part may be an FP16 subnormal); dropping al*bl and the da, db terms
//    costs <= 3.01 u16^2 M + 2^-24 S + 2^-47 n, where
//      M = sum_e m (|a1| pmax + |a2| pmax^2),  S = sum_e m (|a1| + |a2| + pmax + pmax^2);
//  * FP32 rounding of the centred operands (t - mu, w t', p - mu, p'^2):
//    <= 4 u32 M;
//  * accumulation: the sequential FP32 bound sum_k u32 |S_k| (S_k the partial
//    sums of one accumulator) is at most u32 sum_i mu_i rem_i, where mu_i bounds
//    the i-th product (from the actual FP16 pieces of a and pmax) and rem_i is
//    the number of K positions from i to the end of its accumulator (padding
//    included: the hardware rounds per instruction, not per nonzero product);
//    taken eight times (blocked, truncating accumulation), plus one rounding of
//    acc0 + acc1:   8 u32 T + 1.01 u32 sum_i mu_i,   T = sum_i mu_i rem_i.
__global__ void k_tc_prep_A(const float* __restrict__ grid, const uint8_t* __restrict__ mask, Geo g,
                            const int64_t* __restrict__ centre_lin, int64_t Q, const int* __restrict__ eoff,
                            const float* __restrict__ w, const float* __restrict__ mu, const float* __restrict__ pmax,
                            TcLayout L, __half* __restrict__ A, double* __restrict__ bound) {
  const int64_t q = blockIdx.x;
  const int n = g.n, ch = g.ch, n8 = L.n8, Ks = L.kb_split * kBK;
  __shared__ double red[4][8];
  double msum = 0.0, ssum = 0.0, tri = 0.0, mass = 0.0;
  __half* row = A + q * L.Kp;
  const __half z = __float2half_rn(0.0f);
  for (int e = 6 * n8 + threadIdx.x; e < L.Kp; e += blockDim.x) row[e] = z;
  const int64_t tc = q < Q ? centre_lin[q] : 0;
  // K positions from k to the end of k's accumulator
  auto rem = [&](int k) { return (double)((k < Ks ? Ks : L.Kp) - k); };
  for (int e = threadIdx.x; e < n8; e += blockDim.x) {
    __half a1h = z, a1l = z, a2h = z, a2l = z;
    if (q < Q && e < n) {
      const int c = e % ch;
      const float k = mask[tc + eoff[e - c] / ch] ? 1.0f : 0.0f;
      const float tp = grid[tc * ch + eoff[e]] - mu[c];
      const float a1 = -2.0f * k * w[c] * tp, a2 = k * w[c];
      split16(a1, a1h, a1l);
      split16(a2, a2h, a2l);
      if (k != 0.0f) {
        const double pm = pmax[c], pm2 = pm * pm;
        msum += (double)fabsf(a1) * pm + (double)fabsf(a2) * pm2;
        ssum += (double)fabsf(a1) + (double)fabsf(a2) + pm + pm2;
        // product bounds: |bh| <= b (1 + u16), |bl| <= u16 b + 2^-25 for b in {pmax, pmax^2}
        const double u16 = 0x1p-11, up = 1.0 + u16;
        const double h1 = fabs((double)__half2float(a1h)), l1 = fabs((double)__half2float(a1l));
        const double h2 = fabs((double)__half2float(a2h)), l2 = fabs((double)__half2float(a2l));
        const double m0 = l1 * pm * up, m1 = l2 * pm2 * up;
        const double m2 = h1 * (u16 * pm + 0x1p-25), m3 = h2 * (u16 * pm2 + 0x1p-25);
        const double m4 = h1 * pm * up, m5 = h2 * pm2 * up;
        tri += m0 * rem(e) + m1 * rem(n8 + e) + m2 * rem(2 * n8 + e) + m3 * rem(3 * n8 + e) +
               m4 * rem(4 * n8 + e) + m5 * rem(5 * n8 + e);
        mass += m0 + m1 + m2 + m3 + m4 + m5;
      }
    }
    row[e] = a1l;
    row[n8 + e] = a2l;
    row[2 * n8 + e] = a1h;
    row[3 * n8 + e] = a2h;
    row[4 * n8 + e] = a1h;
    row[5 * n8 + e] = a2h;
  }
  for (int o = 16; o > 0; o >>= 1) {
    msum += __shfl_xor_sync(0xffffffffu, msum, o);
    ssum += __shfl_xor_sync(0xffffffffu, ssum, o);
    tri += __shfl_xor_sync(0xffffffffu, tri, o);
    mass += __shfl_xor_sync(0xffffffffu, mass, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = msum;
    red[1][threadIdx.x >> 5] = ssum;
    red[2][threadIdx.x >> 5] = tri;
    red[3][threadIdx.x >> 5] = mass;
  }
  __syncthreads();
  if (threadIdx.x == 0 && q < Q) {
    double M = 0.0, Sa = 0.0, T = 0.0, Ms = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) {
      M += red[0][i];
      Sa += red[1][i];
      T += red[2][i];
      Ms += red[3][i];
    }
    const double u16 = 0x1p-11, u32 = 0x1p-24;
    // (the double sums above carry relative errors ~1e-16, far inside the slack)
    bound[q] = 3.01 * u16 * u16 * M + 0x1p-24 * Sa + 0x1p-47 * n + 4.0 * u32 * M + 8.0 * u32 * T + 1.01 * u32 * Ms;
  }
}

// B rows: one thread per 8 consecutive elements of one row (six 16-byte
// stores), or per 8 zeros of the tail [6 n8, Kp).
__global__ void k_tc_prep_B(const float* __restrict__ grid, const uint32_t* __restrict__ dict, int64_t N,
                            int64_t Npad, Geo g, const int* __restrict__ eoff, const float* __restrict__ mu,
                            TcLayout L, __half* __restrict__ B) {
  const int n = g.n, ch = g.ch, n8 = L.n8;
  const int G = n8 / 8, Zg = (L.Kp - 6 * n8) / 8, per = G + Zg;
  const int64_t total = Npad * per;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t j = t / per;
    const int gg = (int)(t - j * per);
    __half* row = B + j * L.Kp;
    if (gg >= G) {
      reinterpret_cast<uint4*>(row + 6 * n8)[gg - G] = make_uint4(0u, 0u, 0u, 0u);
      continue;
    }
    __align__(16) __half h1[8], l1[8], h2[8], l2[8];
    const int64_t sb = j < N ? (int64_t)dict[j] * ch : 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = gg * 8 + i;
      float p = 0.0f;
      if (j < N && e < n) p = grid[sb + eoff[e]] - mu[e % ch];
      split16(p, h1[i], l1[i]);
      split16(p * p, h2[i], l2[i]);
    }
    const uint4 vh1 = *reinterpret_cast<const uint4*>(h1), vl1 = *reinterpret_cast<const uint4*>(l1);
    const uint4 vh2 = *reinterpret_cast<const uint4*>(h2), vl2 = *reinterpret_cast<const uint4*>(l2);
    uint4* r = reinterpret_cast<uint4*>(row) + gg;
    const int ps = n8 / 8;  // part stride in 16-byte units
    r[0] = vh1;
    r[ps] = vh2;
    r[2 * ps] = vl1;
    r[3 * ps] = vl2;
    r[4 * ps] = vh1;
    r[5 * ps] = vh2;
  }
}

// per-channel minimum and maximum of the grid (order-preserving integer codes)
__device__ inline unsigned f2ord(float v) {
  const unsigned u = __float_as_uint(v);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__global__ void k_tc_range(const float* __restrict__ grid, int64_t npix, int ch, unsigned* __restrict__ lo,
                           unsigned* __restrict__ hi) {
  for (int c = 0; c < ch; ++c) {
    unsigned l = 0xFFFFFFFFu, h = 0u;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
      const unsigned o = f2ord(grid[i * ch + c]);
      l = min(l, o);
      h = max(h, o);
    }
    for (int o = 16; o > 0; o >>= 1) {
      l = min(l, __shfl_xor_sync(0xffffffffu, l, o));
      h = max(h, __shfl_xor_sync(0xffffffffu, h, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMin(&lo[c], l);
      atomicMax(&hi[c], h);
    }
  }
}

// ----------------------------------------------------------------------------
// host side: tensor maps through the driver entry point (no libcuda link)
// ----------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    cudaGetLastError();
  });
  return fn;
}

int make_map(CUtensorMap* map, const void* ptr, int64_t rows, int64_t cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return SFC_EUNSUPPORTED;
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(ptr), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
    return SFC_ECUDA;
  }
  return SFC_OK;
}

}  // namespace

// Pre-scores of Q queries against the N dictionary entries on the tensor cores.
// Outputs submin [Q][tc_subs(N)] -- the minimum over each 32 consecutive
// dictionary entries (groups past N are not written) -- bound[Q] and, when
// `scores` is non-null, all Q x N pre-scores; the per-query constant
// sum m w t'^2 is not included.
int tc_prescore(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                const int* eoff_all, const float* weights, const int64_t* centre_lin, int64_t Q, float* submin,
                float* scores, double* bound, cudaStream_t st) {
  const TcLayout L = tc_layout(g.n);
  const int Kp = L.Kp;
  const int64_t Qpad = ((Q + kBM - 1) / kBM) * kBM, Npad = ((N + kBN - 1) / kBN) * kBN;
  const int ntiles = (int)(Npad / kBN);
  const int64_t npix = g.X * g.Y * g.Z;
  __half *A = nullptr, *B = nullptr;
  unsigned* rng = nullptr;
  float* cent = nullptr;
  Scratch scr(st);  // freed on every return
  SFC_TRY(scr.alloc(&rng, sizeof(unsigned) * 2 * g.ch));
  SFC_TRY(scr.alloc(&cent, sizeof(float) * 2 * g.ch));
  SFC_TRY(cudaMemsetAsync(rng, 0xFF, sizeof(unsigned) * g.ch, st));
  SFC_TRY(cudaMemsetAsync(rng + g.ch, 0, sizeof(unsigned) * g.ch, st));
  count_launch();
  k_tc_range<<<256, 256, 0, st>>>(grid, npix, g.ch, rng, rng + g.ch);
  SFC_TRY(cudaGetLastError());
  {
    // centring at the channel mid-range (smallest max |value - mu|), and the
    // range check of the FP16 operands (largest finite 65504): |p'| < 128 so
    // p'^2 < 16384, and |2 w t'| and w below 30000
    std::vector<unsigned> rh(2 * g.ch);
    std::vector<float> wh(g.ch), ch_h(2 * g.ch);
    SFC_TRY(cudaMemcpyAsync(rh.data(), rng, sizeof(unsigned) * 2 * g.ch, cudaMemcpyDeviceToHost, st));
    SFC_TRY(cudaMemcpyAsync(wh.data(), weights, sizeof(float) * g.ch, cudaMemcpyDeviceToHost, st));
    SFC_TRY(cudaStreamSynchronize(st));
    auto ord2f = [](unsigned o) {
      const unsigned u = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
      float f;
      std::memcpy(&f, &u, sizeof(float));
      return f;
    };
    bool ok = true;
    for (int c = 0; c < g.ch; ++c) {
      const float lo = ord2f(rh[c]), hi = ord2f(rh[g.ch + c]);
      const float m = 0.5f * lo + 0.5f * hi;
      const float pm = std::fmax(std::fabs(hi - m), std::fabs(lo - m));
      ch_h[c] = m;
      ch_h[g.ch + c] = pm;
      ok = ok && std::isfinite(lo) && std::isfinite(hi) && pm < 128.0f && wh[c] < 30000.0f &&
           2.0f * wh[c] * pm < 30000.0f;
    }
    if (!ok) {
      set_error("grid values or weights out of range for the FP16 tensor-core pre-score (need finite values, "
                "max |value - mid-range| < 128, weights and 2 w |value - mid-range| < 30000; use SFC_FP32)");
      return SFC_EINVAL;
    }
    SFC_TRY(cudaMemcpyAsync(cent, ch_h.data(), sizeof(float) * 2 * g.ch, cudaMemcpyHostToDevice, st));
  }
  const float* mu = cent;
  const float* pmax = cent + g.ch;
  // the dictionary operand in chunks of at most kChunkBytes (one chunk for
  // dictionaries up to ~1.9 M entries at n = 363)
  constexpr int64_t kChunkBytes = (int64_t)8 << 30;
  int64_t Nc = kChunkBytes / ((int64_t)Kp * 2) / kBN * kBN;
  if (Nc < kBN) Nc = kBN;
  if (Nc > Npad) Nc = Npad;
  SFC_TRY(scr.alloc(&A, sizeof(__half) * Qpad * Kp));
  SFC_TRY(scr.alloc(&B, sizeof(__half) * Nc * Kp));
  count_launch();
  k_tc_prep_A<<<(unsigned)Qpad, 256, 0, st>>>(grid, cur_mask, g, centre_lin, Q, eoff_all, weights, mu, pmax, L,
                                               A, bound);
  SFC_TRY(cudaGetLastError());
  CUtensorMap mapA;
  SFC_CHECK(make_map(&mapA, A, Qpad, Kp, kBM));
  int* abort_all = nullptr;
  SFC_TRY(scr.alloc(&abort_all, sizeof(int)));
  SFC_TRY(cudaMemsetAsync(abort_all, 0, sizeof(int), st));
  const size_t shm = (size_t)kStages * (kStageA + kStageB) + 1024;
  SFC_TRY(cudaFuncSetAttribute(k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  int dev = 0, sms = 0;
  SFC_TRY(cudaGetDevice(&dev));
  SFC_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  for (int64_t j0 = 0; j0 < N; j0 += Nc) {
    const int64_t Nch = std::min(Nc, N - j0), Npch = (Nch + kBN - 1) / kBN * kBN;
    count_launch();
    k_tc_prep_B<<<152 * 32, 256, 0, st>>>(grid, dict + j0, Nch, Npch, g, eoff_all, mu, L, B);
    SFC_TRY(cudaGetLastError());
    CUtensorMap mapB;
    SFC_CHECK(make_map(&mapB, B, Npch, Kp, kBN));
    TcArgs a;
    a.abort_all = abort_all;
    a.Q = Q;
    a.N = Nch;
    a.n0 = j0;
    a.Nt = N;
    a.kblocks = L.kblocks;
    a.kb_split = L.kb_split;
    a.mtiles = Qpad / kBM;
    a.tiles = a.mtiles * (Npch / kBN);
    a.nsub = (int64_t)ntiles * (kBN / 32);
    a.submin = submin;
    a.scores = scores;
    a.status = status_word();
    const unsigned grid_x = (unsigned)std::min<int64_t>(a.tiles, std::max(sms, 1));
    if (j0 == 0) tc_trace_mark(1, st);
    count_launch();
    k_tc_gemm<<<grid_x, kTcThreads, shm, st>>>(mapA, mapB, a);
    SFC_TRY(cudaGetLastError());
  }
  tc_trace_mark(2, st);
  return SFC_OK;
}

// 32-entry groups per query row of submin (a multiple of 8)
int64_t tc_subs(int64_t N) { return (N + kBN - 1) / kBN * (kBN / 32); }

}  // namespace sfc
