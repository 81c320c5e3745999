// k_query.cu -- batched SFC queries (Fig. 1(b)-(d)): one CTA per query.
//
//  1. stage the target patch (values, known flags) in shared memory;
//  2. select the indices: all of them, or the one whose pixel subset covers the
//     most known pixels (ties: lowest index) -- "the index that best covers the
//     search area", Fig. 1(b);
//  3. per selected index (one warp each): project the known subset values with
//     the same FP32 fused multiply-add chain as the dictionary (unknown values
//     contribute exactly zero), quantise with the index's lo/scale (clamped),
//     shift, Morton key; warp-cooperative lower_bound on the sorted keys (32
//     probes per step); copy the ids of the W sorted slots around the position;
//  4. bitonic sort + de-duplication of the candidate union in shared memory;
//  5. filter-and-refine (Fig. 1(d)): FP32 masked-L2 cost of every candidate, one
//     warp per candidate, each lane holding its patch elements' known flag,
//     target value and grid offset in registers, gathered reads of the source
//     patch rows, warp-shuffle sum; block minimum; a single candidate inside
//     the FP32 error band is the exact argmin, several (near-ties) are rescored
//     with the exact FP64 sequential cost and the argmin over (cost, id) taken.
//     The reported cost is the FP32 cost of the pick.
#include "internal.cuh"

namespace sfc {

namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;

struct QArgs {
  const float* grid;
  const uint8_t* mask;
  const int32_t* centres;
  Geo g;
  int C, D, bits, bp, W, select, m, s, L, maxsel;
  int64_t N;
  const uint32_t* dict;
  const int32_t* sub_pix;
  const float* basis;
  const float* mean;
  const float* lo;
  const float* scale;
  const int32_t* shifts;
  const uint64_t* skeys;
  const uint32_t* sids;
  const int* eoff_all;
  const float* weights;
  int64_t* pick;
  float* cost;
  uint64_t* qkeys;
  int64_t* pos;
  int32_t* cand_out;
  int32_t* ncand_out;
  uint32_t* status;
};

// Number of keys < key in the sorted array (32 probes per step).
__device__ int64_t warp_lower_bound(const uint64_t* __restrict__ a, int64_t N, uint64_t key) {
  const int lane = threadIdx.x & 31;
  int64_t lo = 0, hi = N;
  while (hi - lo > 32) {
    int64_t step = (hi - lo) / 32;
    int64_t idx = lo + lane * step;
    bool lt = a[idx] < key;
    unsigned b = __ballot_sync(0xffffffffu, lt);
    int t = __popc(b);
    if (t == 0) {
      hi = lo;
    } else {
      int64_t nlo = lo + (int64_t)(t - 1) * step + 1;
      if (t < 32) hi = lo + (int64_t)t * step;
      lo = nlo;
    }
  }
  int64_t idx = lo + lane;
  bool lt = idx < hi && a[idx] < key;
  return lo + __popc(__ballot_sync(0xffffffffu, lt));
}

template <int MAXE, bool WEIGHTED>
__global__ void __launch_bounds__(kQThreads) k_query(QArgs a) {
  const int64_t q = blockIdx.x;
  const Geo& g = a.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n, P = g.P, ch = g.ch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tv = reinterpret_cast<float*>(smem_raw);          // n
  int* eo = reinterpret_cast<int*>(tv + n);                // n
  uint32_t* cand = reinterpret_cast<uint32_t*>(eo + n);    // L
  uint32_t* ucand = cand + a.L;                            // L
  float* c32 = reinterpret_cast<float*>(ucand + a.L);      // L
  uint8_t* tm = reinterpret_cast<uint8_t*>(c32 + a.L);     // P
  __shared__ int s_sel[16];
  __shared__ int s_cov[16];
  __shared__ int s_nsel, s_ncand, s_bad;
  __shared__ uint32_t s_part[kQThreads];
  __shared__ float s_redf[kQWarps];
  __shared__ double s_redd[kQWarps];
  __shared__ int64_t s_redi[kQWarps];

  // --- centre -------------------------------------------------------------
  if (tid == 0) {
    int64_t cx = a.centres[q * g.ndim + 0], cy = a.centres[q * g.ndim + 1];
    int64_t cz = g.ndim == 3 ? a.centres[q * g.ndim + 2] : 0;
    s_bad = centre_ok(g, cx, cy, cz) ? 0 : 1;
    s_part[0] = (uint32_t)0;
    if (!s_bad) {
      int64_t lin = lin_of(g, cx, cy, cz);
      s_redi[0] = lin;
    }
  }
  __syncthreads();
  if (s_bad) {
    if (tid == 0) {
      atomicOr(a.status, ST_BAD_CENTRE);
      if (a.pick) {
        a.pick[q] = -1;
        a.cost[q] = __int_as_float(0x7fc00000);
      }
      if (a.ncand_out) a.ncand_out[q] = 0;
    }
    return;
  }
  const int64_t tc = s_redi[0];
  for (int e = tid; e < n; e += kQThreads) {
    int o = a.eoff_all[e];
    eo[e] = o;
    tv[e] = a.grid[tc * ch + o];
  }
  for (int pp = tid; pp < P; pp += kQThreads) tm[pp] = a.mask[tc + a.eoff_all[pp * ch] / ch];
  __syncthreads();

  // --- index selection ------------------------------------------------------
  if (a.select == SFC_SELECT_BEST) {
    for (int c = warp; c < a.C; c += kQWarps) {
      int cov = 0;
      for (int i = lane; i < a.m; i += 32) cov += tm[a.sub_pix[c * a.m + i]] ? 1 : 0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) cov += __shfl_xor_sync(0xffffffffu, cov, o);
      if (lane == 0) s_cov[c] = cov;
    }
    __syncthreads();
    if (tid == 0) {
      int best = 0;
      for (int c = 1; c < a.C; ++c)
        if (s_cov[c] > s_cov[best]) best = c;
      s_sel[0] = best;
      s_nsel = 1;
    }
  } else if (tid == 0) {
    for (int c = 0; c < a.C; ++c) s_sel[c] = c;
    s_nsel = a.C;
  }
  __syncthreads();
  const int nsel = s_nsel;
  const int64_t len = a.W < a.N ? a.W : a.N;
  int64_t maxs = a.N - a.W;
  if (maxs < 0) maxs = 0;

  // --- per index: project, key, search, window -------------------------------
  for (int slot = warp; slot < nsel; slot += kQWarps) {
    const int c = s_sel[slot];
    float acc = 0.0f;
    if (lane < a.D) {
      const float* B = a.basis + (int64_t)c * a.s * a.D;
      const float* mu = a.mean + (int64_t)c * a.s;
      const int32_t* sp = a.sub_pix + c * a.m;
      for (int i = 0; i < a.s; ++i) {
        int pp = sp[i / ch];
        if (!tm[pp]) continue;
        float xc = __fsub_rn(tv[pp * ch + i % ch], mu[i]);
        acc = __fmaf_rn(B[(int64_t)i * a.D + lane], xc, acc);
      }
    }
    uint32_t qk = 0;
    if (lane < a.D) qk = quantise_one(acc, a.lo[c * a.D + lane], a.scale[c * a.D + lane], a.bits) +
                         (uint32_t)a.shifts[c * a.D + lane];
    uint64_t key = 0;
    int nb = 0;
    for (int p = a.bp - 1; p >= 0 && nb < 64; --p)
      for (int k = 0; k < a.D && nb < 64; ++k, ++nb) {
        uint32_t v = __shfl_sync(0xffffffffu, qk, k);
        key = (key << 1) | (uint64_t)((v >> p) & 1u);
      }
    const uint64_t* sk = a.skeys + (int64_t)c * a.N;
    int64_t pos = warp_lower_bound(sk, a.N, key);
    int64_t start = pos - a.W / 2;
    if (start > maxs) start = maxs;
    if (start < 0) start = 0;
    const uint32_t* si = a.sids + (int64_t)c * a.N + start;
    for (int64_t i = lane; i < len; i += 32) cand[slot * len + i] = si[i];
    if (a.qkeys && lane == 0) {
      a.qkeys[q * a.C + c] = key;
      a.pos[q * a.C + c] = pos;
    }
  }
  if (a.qkeys && nsel < a.C) {
    for (int c = tid; c < a.C; c += kQThreads) {
      bool used = false;
      for (int t = 0; t < nsel; ++t) used |= s_sel[t] == c;
      if (!used) {
        a.qkeys[q * a.C + c] = 0;
        a.pos[q * a.C + c] = -1;
      }
    }
  }
  const int L0 = (int)(nsel * len);
  for (int i = L0 + tid; i < a.L; i += kQThreads) cand[i] = 0xffffffffu;
  __syncthreads();

  // --- bitonic sort of the candidate union ---------------------------------
  for (int k = 2; k <= a.L; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < a.L; i += kQThreads) {
        int ixj = i ^ j;
        if (ixj > i) {
          uint32_t x = cand[i], y = cand[ixj];
          bool up = (i & k) == 0;
          if ((x > y) == up) {
            cand[i] = y;
            cand[ixj] = x;
          }
        }
      }
      __syncthreads();
    }
  }
  // --- de-duplicate (stream compaction of first occurrences) -----------------
  {
    const int per = (a.L + kQThreads - 1) / kQThreads;
    const int b0 = tid * per, b1 = min(b0 + per, a.L);
    uint32_t cnt = 0;
    for (int i = b0; i < b1; ++i) cnt += (cand[i] != 0xffffffffu && (i == 0 || cand[i] != cand[i - 1])) ? 1u : 0u;
    s_part[tid] = cnt;
    __syncthreads();
    if (warp == 0) {
      uint32_t loc[kQWarps], sum = 0;
#pragma unroll
      for (int t = 0; t < kQWarps; ++t) {
        loc[t] = s_part[lane * kQWarps + t];
        sum += loc[t];
      }
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      uint32_t run = incl - sum;
#pragma unroll
      for (int t = 0; t < kQWarps; ++t) {
        s_part[lane * kQWarps + t] = run;
        run += loc[t];
      }
      if (lane == 31) s_ncand = (int)run;
    }
    __syncthreads();
    uint32_t w = s_part[tid];
    for (int i = b0; i < b1; ++i)
      if (cand[i] != 0xffffffffu && (i == 0 || cand[i] != cand[i - 1])) ucand[w++] = cand[i];
  }
  __syncthreads();
  const int ncand = s_ncand;
  if (a.cand_out) {
    const int cap = a.C * a.W;
    for (int i = tid; i < cap; i += kQThreads) a.cand_out[q * cap + i] = i < ncand ? (int32_t)ucand[i] : -1;
    if (tid == 0) a.ncand_out[q] = ncand;
  }
  if (!a.pick) return;

  // --- FP32 rescore --------------------------------------------------------
  float am[MAXE], mt[MAXE], wv[MAXE];
  int eor[MAXE];
#pragma unroll
  for (int t = 0; t < MAXE; ++t) {
    int e = lane + 32 * t;
    if (e < n) {
      float k = tm[e / ch] ? 1.0f : 0.0f;
      am[t] = k;
      mt[t] = k * tv[e];
      eor[t] = eo[e];
      wv[t] = WEIGHTED ? a.weights[e % ch] : 1.0f;
    } else {
      am[t] = 0.0f;
      mt[t] = 0.0f;
      eor[t] = 0;
      wv[t] = 0.0f;
    }
  }
  float wmin = INFINITY;
  for (int ci = warp; ci < ncand; ci += kQWarps) {
    const int64_t sb = (int64_t)a.dict[ucand[ci]] * ch;
    float acc = 0.0f;
#pragma unroll
    for (int t = 0; t < MAXE; ++t) {
      if (lane + 32 * t < n) {
        float p = __ldg(a.grid + sb + eor[t]);
        float d = __fmaf_rn(-am[t], p, mt[t]);
        if (WEIGHTED)
          acc = __fmaf_rn(__fmul_rn(wv[t], d), d, acc);
        else
          acc = __fmaf_rn(d, d, acc);
      }
    }
    acc = warp_sum(acc);
    if (lane == 0) c32[ci] = acc;
    wmin = fminf(wmin, acc);
  }
  if (lane == 0) s_redf[warp] = wmin;
  __syncthreads();
  float m32 = s_redf[0];
  for (int w = 1; w < kQWarps; ++w) m32 = fminf(m32, s_redf[w]);
  const float T = band_limit32(m32, n);
  // --- band: a single member is the exact argmin; otherwise rescore in FP64 ---
  int nband = 0, mine = -1;
  for (int ci = tid; ci < ncand; ci += kQThreads)
    if (c32[ci] <= T) {
      ++nband;
      mine = ci;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nband += __shfl_xor_sync(0xffffffffu, nband, o);
  if (lane == 0) s_part[warp] = (uint32_t)nband;
  __syncthreads();
  int total = 0;
  for (int w = 0; w < kQWarps; ++w) total += (int)s_part[w];
  if (total == 1) {
    if (mine >= 0) {
      a.pick[q] = ucand[mine];
      a.cost[q] = c32[mine];
    }
    return;
  }
  double bc = INFINITY;
  int64_t bi = INT64_MAX;  // candidate slot; slots are in ascending id order
  for (int ci = tid; ci < ncand; ci += kQThreads) {
    if (c32[ci] <= T) {
      const uint32_t j = ucand[ci];
      const double c64 = exact_cost64(a.grid, (int64_t)a.dict[j] * ch, tv, tm, eo, P, ch, a.weights);
      if (c64 < bc || (c64 == bc && ci < bi)) {
        bc = c64;
        bi = ci;
      }
    }
  }
  warp_argmin64(bc, bi);
  __syncthreads();
  if (lane == 0) {
    s_redd[warp] = bc;
    s_redi[warp] = bi;
  }
  __syncthreads();
  if (tid == 0) {
    double c = s_redd[0];
    int64_t i = s_redi[0];
    for (int w = 1; w < kQWarps; ++w)
      if (s_redd[w] < c || (s_redd[w] == c && s_redi[w] < i)) {
        c = s_redd[w];
        i = s_redi[w];
      }
    if (ncand == 0 || i == INT64_MAX) {
      a.pick[q] = -1;
      a.cost[q] = __int_as_float(0x7fc00000);
    } else {
      a.pick[q] = ucand[i];
      a.cost[q] = c32[i];
    }
  }
}

template <int MAXE, bool W>
int launch_q(const QArgs& a, int64_t Q, size_t shm, cudaStream_t st) {
  if (shm > 48 * 1024)
    SFC_TRY(cudaFuncSetAttribute(k_query<MAXE, W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
  count_launch();
  k_query<MAXE, W><<<(unsigned)Q, kQThreads, shm, st>>>(a);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

template <bool W>
int dispatch_q(const QArgs& a, int64_t Q, size_t shm, cudaStream_t st) {
  const int need = (a.g.n + 31) / 32;
  if (need <= 4) return launch_q<4, W>(a, Q, shm, st);
  if (need <= 8) return launch_q<8, W>(a, Q, shm, st);
  if (need <= 12) return launch_q<12, W>(a, Q, shm, st);
  if (need <= 16) return launch_q<16, W>(a, Q, shm, st);
  if (need <= 24) return launch_q<24, W>(a, Q, shm, st);
  if (need <= 32) return launch_q<32, W>(a, Q, shm, st);
  set_error("patch has more than 1024 values; not supported by the query kernel");
  return SFC_EUNSUPPORTED;
}

}  // namespace

int query_batch(const Index& ix, const float* grid, const uint8_t* cur_mask, const int32_t* centres, int64_t Q,
                int64_t* pick, float* cost, uint64_t* qkeys, int64_t* pos, int32_t* cand, int32_t* ncand,
                cudaStream_t st) {
  if (Q <= 0) return SFC_OK;
  if (Q > 0x7fffffffLL) {
    set_error("too many queries in one batch");
    return SFC_EINVAL;
  }
  QArgs a;
  a.grid = grid;
  a.mask = cur_mask;
  a.centres = centres;
  a.g = ix.g;
  a.C = ix.C;
  a.D = ix.D;
  a.bits = ix.bits;
  a.bp = ix.bp;
  a.W = ix.W;
  a.select = ix.select;
  a.m = ix.m;
  a.s = ix.s;
  a.N = ix.N;
  a.maxsel = ix.select == SFC_SELECT_BEST ? 1 : ix.C;
  int64_t len = ix.W < ix.N ? ix.W : ix.N;
  int64_t need = len * a.maxsel;
  int L = 2;
  while (L < need) L <<= 1;
  if (L > 8192) {
    set_error("curves * window exceeds 8192 candidates per query");
    return SFC_EINVAL;
  }
  a.L = L;
  a.dict = ix.dict;
  a.sub_pix = ix.sub_pix;
  a.basis = ix.basis;
  a.mean = ix.mean;
  a.lo = ix.lo;
  a.scale = ix.scale;
  a.shifts = ix.shifts;
  a.skeys = ix.skeys;
  a.sids = ix.sids;
  a.eoff_all = ix.eoff_all;
  a.weights = ix.weights;
  a.pick = pick;
  a.cost = cost;
  a.qkeys = qkeys;
  a.pos = pos;
  a.cand_out = cand;
  a.ncand_out = ncand;
  a.status = status_word();
  const size_t shm = (size_t)ix.g.n * 8 + (size_t)L * 12 + (((size_t)ix.g.P + 15) & ~(size_t)15);
  bool weighted = false;
  for (float w : ix.weights_h) weighted |= (w != 1.0f);
  return weighted ? dispatch_q<true>(a, Q, shm, st) : dispatch_q<false>(a, Q, shm, st);
}

}  // namespace sfc
