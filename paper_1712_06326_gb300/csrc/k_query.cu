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
//     probes per step); copy the ids of the W sorted slots around the position,
//     or, with knn = k, find the exact k nearest entries in the quantised space
//     (Sec. II.D; warp_knn below);
//  4. bitonic sort + de-duplication of the candidate union in shared memory;
//  5. filter-and-refine (Fig. 1(d)): FP32 masked-L2 cost of every candidate
//     over the target's known elements only (compacted in patch order: the
//     unknown ones add exactly zero), one warp per candidate and two candidates
//     per pass, each lane holding its elements' target value and grid offset in
//     registers, gathered reads of the source patch, warp-shuffle sum; block
//     minimum; a single candidate inside
//     the FP32 error band is the exact argmin, several (near-ties) are rescored
//     with the exact FP64 sequential cost and the argmin over (cost, id) taken.
//     The reported cost is the FP32 cost of the pick.
#include "internal.cuh"

namespace sfc {

namespace {

constexpr int kQThreads = 256;
constexpr int kQWarps = kQThreads / 32;
// centred subset values (and the basis rows) staged per warp for the query
// projection, kXChunk subset values at a time
constexpr int kXChunk = 64;

// Everything that belongs to one image (or volume) and its index.
struct QImg {
  const float* grid;   // targets (geometry g)
  const float* dgrid;  // dictionary patches (the index's grid; = grid unless queried from another grid)
  const int* deoff;    // element offsets of a patch in dgrid
  const uint8_t* mask;
  Geo g;
  int64_t N;
  const uint32_t* sqc;
  const uint32_t* dict;
  const int32_t* sub_pix;
  const float* basis;
  const float* mean;
  const float* lo;
  const float* scale;
  const int32_t* shifts;
  const uint64_t* skeys;
  const uint32_t* sids;
  const int* eoff_all;  // element offsets of a patch in grid
};

struct QArgs {
  QImg img;            // the image of every query, or, with imgs: ignored
  const QImg* imgs;    // several images: query q belongs to imgs[img_of[q]]
  const int32_t* img_of;
  int nimg;
  const int32_t* centres;
  int C, D, bits, bp, W, select, m, s, L, maxsel, knn, capw, curve, l1;
  const float* weights;
  int64_t* pick;
  float* cost;
  uint64_t* qkeys;
  int64_t* pos;
  int32_t* cand_out;
  int32_t* ncand_out;
  float* c32_out;  // split form: FP32 cost of every candidate slot (stride C * capw)
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

// Morton key (top 64 bits; bit planes from the top, dimension 0 first) of the
// coordinates held by lanes 0..D-1.
__device__ uint64_t warp_key(uint32_t x, int D, int bp) {
  // one ballot per bit plane gives the plane's bits with lane k at bit k; bit
  // reversed and shifted, dimension 0 is the group's most significant bit
  // (lanes >= D hold 0 and fall off the shift)
  uint64_t key = 0;
  int nb = 0;
  for (int p = bp - 1; p >= 0 && nb < 64; --p) {
    const uint32_t plane = __ballot_sync(0xffffffffu, (x >> p) & 1u);
    const uint32_t grp = __brev(plane) >> (32 - D);
    const int take = 64 - nb < D ? 64 - nb : D;
    key = (key << take) | (uint64_t)(grp >> (D - take));
    nb += take;
  }
  return key;
}

// Hilbert key of the coordinates held by lanes 0..D-1 (every lane computes it
// identically).  Kept out of line: inlined, its loops over a 16-word array
// cost the query kernel's window path ~10 % even when the z-curve is used.
__device__ __noinline__ uint64_t warp_hilbert_key(uint32_t x, int D, int bp) {
  uint32_t xq[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) xq[d] = __shfl_sync(0xffffffffu, x, d);
  return hilbert_key(xq, D, bp);
}

// Bits of v at the positions set in m, the highest first (a software pext).
__device__ inline uint32_t extract_bits(uint64_t v, uint64_t m) {
  uint32_t r = 0;
  while (m) {
    const int i = 63 - __clzll((long long)m);
    r = (r << 1) | (uint32_t)((v >> i) & 1u);
    m &= ~(1ull << i);
  }
  return r;
}

// One pending region of the k-NN traversal: the key-space box [zmin, zmax] and
// the slots [a, b) of the sorted array whose keys lie in [zmin, zmax].
struct KnnRegion {
  uint64_t zmin, zmax;
  int64_t a, b;
};
constexpr int kKnnStack = 66;  // depth <= key bits + 1
constexpr int kKnnLeaf = 2048;  // mu: regions of at most this many slots are scanned (measured best of 32..8192)

// First slot in [0, n) whose key is > key.
__device__ inline int64_t warp_upper_bound(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
  return key == ~0ull ? n : warp_lower_bound(a, n, key + 1);
}

// The kk (<= 128) entries of one index nearest to the query in the quantised
// space, by (squared Euclidean distance, id) -- the paper's exact k-NN list,
// found with its outside-in search (Sec. II.D, Fig. 3): a region of the key
// space (an axis-aligned box of truncated coordinates, i.e. a z-interval) is
// split where the most significant bit of its corners differs, into the
// halves [min, litmax] and [bigmin, max]; their slot ranges come from binary
// searches inside the parent's range; the half nearer to the query is
// visited first, and a half whose box lies farther from the query than the
// current k-th entry is culled; regions of at most kKnnLeaf slots (or a single
// cell) are scanned entry by entry.  Lane d < D holds the query's shifted
// coordinate x.  The list lives in registers (entry e = 32 s + lane in slot s);
// the region stack (kKnnStack entries) in shared memory.  Writes the ids to
// out[0..kk).
__device__ void warp_knn(const uint64_t* __restrict__ sk, const uint32_t* __restrict__ sq,
                         const uint32_t* __restrict__ si, int64_t N, int D, int bp, uint32_t x, int kk,
                         uint32_t* out, KnnRegion* stk) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int KPL = 4;
  const int lane = threadIdx.x & 31;
  const int nb = D * bp < 64 ? D * bp : 64;
  uint32_t qv[16];
#pragma unroll
  for (int d = 0; d < 16; ++d) qv[d] = __shfl_sync(FULL, x, d);
  // lane d < D: the key bits of dimension d, and how many coordinate bits lie below them
  uint64_t dmask = 0;
  int kept = 0;
  if (lane < D)
    for (int t = lane; t < nb; t += D) {
      dmask |= 1ull << (nb - 1 - t);
      ++kept;
    }
  const int low = bp - kept;
  uint64_t ld[KPL];
  uint32_t li[KPL];
#pragma unroll
  for (int s = 0; s < KPL; ++s) {
    ld[s] = ~0ull;
    li[s] = ~0u;
  }
  // the list's worst entry (largest (distance, id)), its lane and slot
  uint64_t wd = ~0ull;
  uint32_t wi = ~0u;
  int wl = 0, ws = 0;
  auto find_worst = [&]() {
    uint64_t bd = 0;
    uint32_t bi = 0;
    int bs = -1;
#pragma unroll
    for (int s = 0; s < KPL; ++s)
      if (s * 32 + lane < kk && (bs < 0 || ld[s] > bd || (ld[s] == bd && li[s] > bi))) {
        bd = ld[s];
        bi = li[s];
        bs = s;
      }
    int bl = lane;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t od = __shfl_xor_sync(FULL, bd, o);
      const uint32_t oi = __shfl_xor_sync(FULL, bi, o);
      const int ol = __shfl_xor_sync(FULL, bl, o), os = __shfl_xor_sync(FULL, bs, o);
      const bool take = os >= 0 && (bs < 0 || od > bd || (od == bd && (oi > bi || (oi == bi && ol < bl))));
      if (take) {
        bd = od;
        bi = oi;
        bl = ol;
        bs = os;
      }
    }
    wd = bd;
    wi = bi;
    wl = bl;
    ws = bs;
  };
  find_worst();
  // score the slots [i, end) (one per lane) and merge the better entries
  auto score = [&](int64_t i, int64_t end) {
    const int64_t e = i + lane;
    const bool ok = e < end;
    uint64_t d2 = ~0ull;
    uint32_t id = ~0u;
    if (ok) {
      // coordinates < 2^22: 32-bit differences, 32 x 32 -> 64-bit squares
      auto sq_diff = [](uint32_t c, uint32_t q) {
        const int t = (int)(c - q);
        return (uint64_t)((long long)t * t);
      };
      const uint32_t* c = sq + e * D;
      d2 = 0;
      if ((D & 3) == 0) {
        const uint4* c4 = reinterpret_cast<const uint4*>(c);  // rows of 4 D words: 16-byte aligned
#pragma unroll
        for (int v = 0; v < 4; ++v)
          if (4 * v < D) {
            const uint4 w = __ldg(c4 + v);
            d2 += sq_diff(w.x, qv[4 * v]) + sq_diff(w.y, qv[4 * v + 1]) + sq_diff(w.z, qv[4 * v + 2]) +
                  sq_diff(w.w, qv[4 * v + 3]);
          }
      } else {
#pragma unroll
        for (int d = 0; d < 16; ++d)
          if (d < D) d2 += sq_diff(__ldg(c + d), qv[d]);
      }
      id = si[e];
    }
    unsigned bal = __ballot_sync(FULL, ok && (d2 < wd || (d2 == wd && id < wi)));
    while (bal) {
      const int b = __ffs(bal) - 1;
      bal &= bal - 1;
      const uint64_t bd = __shfl_sync(FULL, d2, b);
      const uint32_t bi = __shfl_sync(FULL, id, b);
      if (bd < wd || (bd == wd && bi < wi)) {
        if (lane == wl) {
#pragma unroll
          for (int s = 0; s < KPL; ++s)
            if (s == ws) {
              ld[s] = bd;
              li[s] = bi;
            }
        }
        find_worst();
      }
    }
  };
  // squared distance from the query to the box [zmin, zmax] (warp-uniform)
  auto box_dist = [&](uint64_t zmin, uint64_t zmax) -> uint64_t {
    uint64_t dd = 0;
    if (lane < D) {
      const int64_t lo = (int64_t)extract_bits(zmin, dmask) << low;
      const int64_t hi = ((int64_t)extract_bits(zmax, dmask) << low) | ((1ll << low) - 1);
      const int64_t xq = (int64_t)x;
      const int64_t t = xq < lo ? lo - xq : (xq > hi ? xq - hi : 0);
      dd = (uint64_t)(t * t);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dd += __shfl_xor_sync(FULL, dd, o);
    return dd;
  };
  int sp = 0;
  if (lane == 0) stk[0] = KnnRegion{0ull, nb == 64 ? ~0ull : ((1ull << nb) - 1), 0, N};
  sp = 1;
  __syncwarp();
  while (sp > 0) {
    const KnnRegion r = stk[--sp];
    __syncwarp();
    if (r.b <= r.a) continue;
    if (wd != ~0ull && box_dist(r.zmin, r.zmax) > wd) continue;  // culled
    if (r.b - r.a <= kKnnLeaf || r.zmin == r.zmax || sp + 2 > kKnnStack) {
      for (int64_t i = r.a; i < r.b; i += 32) score(i, i + 32 < r.b ? i + 32 : r.b);
      continue;
    }
    // split where the corners' most significant bit differs
    const int i = 63 - __clzll((long long)(r.zmin ^ r.zmax));
    const int d = (nb - 1 - i) % D;
    const uint64_t bit = 1ull << i;
    const uint64_t below = __shfl_sync(FULL, dmask, d) & (bit - 1);
    const uint64_t litmax = (r.zmax & ~bit) | below;
    const uint64_t bigmin = (r.zmin & ~below) | bit;
    const int64_t ml = r.a + warp_upper_bound(sk + r.a, r.b - r.a, litmax);
    const int64_t mr = ml + warp_lower_bound(sk + ml, r.b - ml, bigmin);
    const KnnRegion L{r.zmin, litmax, r.a, ml}, R{bigmin, r.zmax, mr, r.b};
    const uint64_t dl = box_dist(L.zmin, L.zmax), dr = box_dist(R.zmin, R.zmax);
    const bool left_first = dl <= dr;
    if (lane == 0) {
      // the far half below the near one on the stack
      stk[sp] = left_first ? R : L;
      stk[sp + 1] = left_first ? L : R;
    }
    sp += 2;
    __syncwarp();
  }
#pragma unroll
  for (int s = 0; s < KPL; ++s)
    if (s * 32 + lane < kk) out[s * 32 + lane] = li[s];
}

// FP32 costs of the candidates ucand[0..ncand), one warp per candidate (the
// target's nk known elements, compacted: lane holds known elements lane + 32 t
// in registers), into c32; returns this warp's minimum.
// L1 (Sec. III.K): w |d| instead of w d^2.
// The target patch of centre tc in shared memory: tv[e] its values, deo[e]
// the element offsets in the dictionary grid, tm[pp] its known flags.
__device__ __forceinline__ void stage_target(const QImg& I, int64_t tc, float* tv, int* deo, uint8_t* tm) {
  const Geo& g = I.g;
  for (int e = threadIdx.x; e < g.n; e += kQThreads) {
    deo[e] = I.deoff[e];
    tv[e] = I.grid[tc * g.ch + I.eoff_all[e]];
  }
  for (int pp = threadIdx.x; pp < g.P; pp += kQThreads) tm[pp] = I.mask[tc + I.eoff_all[pp * g.ch] / g.ch];
}

// The known elements of the staged target, compacted in patch order (unknown
// ones add exactly 0 to a cost, so only known values are gathered): ceo their
// dictionary-grid offsets, ct their values, cw their channel weights.  Returns
// their number; the whole CTA calls it.
template <bool WEIGHTED>
__device__ int compact_known(int n, int ch, const uint8_t* tm, const int* deo, const float* tv,
                             const float* __restrict__ weights, int* ceo, float* ct, float* cw, uint32_t* s_part) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int nk = 0;
  for (int r0 = 0; r0 < n; r0 += kQThreads) {
    const int e = r0 + tid;
    const bool kn = e < n && tm[e / ch] != 0;
    const unsigned bal = __ballot_sync(0xffffffffu, kn);
    if (lane == 0) s_part[warp] = (uint32_t)__popc(bal);
    __syncthreads();
    int off = nk, tot = 0;
    for (int w = 0; w < kQWarps; ++w) {
      if (w < warp) off += (int)s_part[w];
      tot += (int)s_part[w];
    }
    if (kn) {
      const int at = off + __popc(bal & ((1u << lane) - 1u));
      ceo[at] = deo[e];
      ct[at] = tv[e];
      cw[at] = WEIGHTED ? weights[e % ch] : 1.0f;
    }
    __syncthreads();
    nk += tot;
  }
  return nk;
}

// Lane registers of the compacted elements lane + 32 t.
template <int MAXE>
__device__ __forceinline__ void lane_elems(int nk, const int* ceo, const float* ct, const float* cw, float (&tr)[MAXE],
                                           int (&eor)[MAXE], float (&wv)[MAXE]) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int t = 0; t < MAXE; ++t) {
    const int e = lane + 32 * t;
    const bool in = e < nk;
    tr[t] = in ? ct[e] : 0.0f;
    eor[t] = in ? ceo[e] : 0;
    wv[t] = in ? cw[e] : 0.0f;
  }
}

template <int MAXE, bool WEIGHTED, bool L1>
__device__ __forceinline__ float rescore_all(const float* __restrict__ dgrid, const uint32_t* __restrict__ dict,
                                             const uint32_t* ucand, int ncand, int ch, int nk, const float (&tr)[MAXE],
                                             const int (&eor)[MAXE], const float (&wv)[MAXE], float* c32) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float wmin = INFINITY;
  // two candidates per pass (ci and ci + kQWarps): twice the gathers in flight;
  // each candidate's sum keeps its order (known element t per lane, then the
  // warp sum)
  for (int ci = warp; ci < ncand; ci += 2 * kQWarps) {
    const int cj = ci + kQWarps;
    const bool two = cj < ncand;
    const int64_t sb = (int64_t)dict[ucand[ci]] * ch;
    const int64_t sb2 = (int64_t)dict[ucand[two ? cj : ci]] * ch;
    float acc = 0.0f, acc2 = 0.0f;
#pragma unroll
    for (int t = 0; t < MAXE; ++t) {
      if (lane + 32 * t < nk) {
        const float p = __ldg(dgrid + sb + eor[t]);
        const float p2 = __ldg(dgrid + sb2 + eor[t]);
        const float d = __fsub_rn(tr[t], p);
        const float d2 = __fsub_rn(tr[t], p2);
        if (L1) {
          acc = WEIGHTED ? __fmaf_rn(wv[t], fabsf(d), acc) : __fadd_rn(acc, fabsf(d));
          acc2 = WEIGHTED ? __fmaf_rn(wv[t], fabsf(d2), acc2) : __fadd_rn(acc2, fabsf(d2));
        } else if (WEIGHTED) {
          acc = __fmaf_rn(__fmul_rn(wv[t], d), d, acc);
          acc2 = __fmaf_rn(__fmul_rn(wv[t], d2), d2, acc2);
        } else {
          acc = __fmaf_rn(d, d, acc);
          acc2 = __fmaf_rn(d2, d2, acc2);
        }
      }
    }
    acc = warp_sum(acc);
    acc2 = warp_sum(acc2);
    if (lane == 0) {
      c32[ci] = acc;
      if (two) c32[cj] = acc2;
    }
    wmin = fminf(wmin, acc);
    if (two) wmin = fminf(wmin, acc2);
  }
  return wmin;
}

template <int MAXE, bool WEIGHTED, bool KNN, bool MULTI>
__global__ void __launch_bounds__(kQThreads) k_query(QArgs a) {
  const int64_t q = blockIdx.x;
  // this query's image: the launch's own, or (MULTI) its entry of the image
  // table, copied to shared memory for the whole CTA
  __shared__ QImg s_img;
  __shared__ int s_badimg;
  if (MULTI) {
    if (threadIdx.x == 0) {
      const int im = a.img_of[q];
      s_badimg = im < 0 || im >= a.nimg;
      s_img = a.imgs[s_badimg ? 0 : im];
    }
    __syncthreads();
  }
  const QImg& I = MULTI ? s_img : a.img;
  const Geo& g = I.g;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int n = g.n, P = g.P, ch = g.ch;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tv = reinterpret_cast<float*>(smem_raw);          // n
  int* ceo = reinterpret_cast<int*>(tv + n);               // n: known elements' dictionary-grid offsets
  uint32_t* cand = reinterpret_cast<uint32_t*>(ceo + n);   // L
  uint32_t* ucand = cand + a.L;                            // L
  float* c32 = reinterpret_cast<float*>(ucand + a.L);      // L
  int* deo = reinterpret_cast<int*>(c32 + a.L);            // n (dictionary-grid offsets)
  float* xcb = reinterpret_cast<float*>(deo + n);          // kQWarps * kXChunk
  float* bcb = xcb + kQWarps * kXChunk;                    // kQWarps * kXChunk * D
  float* ct = bcb + kQWarps * kXChunk * a.D;               // n: known elements' target values
  float* cw = ct + n;                                      // n: their channel weights
  uint8_t* tm = reinterpret_cast<uint8_t*>(cw + n);        // P
  // k-NN region stacks, one per warp (k-NN mode only), rounded up to a 16-byte
  // boundary after tm (its offset 12 n + 12 L is only 4-aligned for odd n)
  KnnRegion* knn_stack = reinterpret_cast<KnnRegion*>(((uintptr_t)(tm + g.P) + 15) & ~(uintptr_t)15);
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
    s_bad = centre_ok(g, cx, cy, cz) && !(MULTI && s_badimg) ? 0 : 1;
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
  stage_target(I, tc, tv, deo, tm);
  __syncthreads();

  // --- index selection ------------------------------------------------------
  if (a.select == SFC_SELECT_BEST) {
    for (int c = warp; c < a.C; c += kQWarps) {
      int cov = 0;
      for (int i = lane; i < a.m; i += 32) cov += tm[I.sub_pix[c * a.m + i]] ? 1 : 0;
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
  const int64_t wk = a.knn > 0 ? a.knn : a.W;
  const int64_t len = wk < I.N ? wk : I.N;
  int64_t maxs = I.N - a.W;
  if (maxs < 0) maxs = 0;

  // --- per index: project, key, search, window -------------------------------
  for (int slot = warp; slot < nsel; slot += kQWarps) {
    const int c = s_sel[slot];
    // lane k < D runs the FMA chain of axis k over the subset values in order,
    // known values only; the warp stages the centred values kXChunk at a time
    // (with their known bits) so that the chain reads shared memory only
    float acc = 0.0f;
    {
      const float* B = I.basis + (int64_t)c * a.s * a.D;
      const float* mu = I.mean + (int64_t)c * a.s;
      const int32_t* sp = I.sub_pix + c * a.m;
      float* xw = xcb + warp * kXChunk;
      float* bw = bcb + warp * kXChunk * a.D;
      for (int i0 = 0; i0 < a.s; i0 += kXChunk) {
        const int cnt = a.s - i0 < kXChunk ? a.s - i0 : kXChunk;
        bool kn0 = false, kn1 = false;
        if (lane < cnt) {
          const int i = i0 + lane, pp = sp[i / ch];
          kn0 = tm[pp] != 0;
          xw[lane] = __fsub_rn(tv[pp * ch + i % ch], mu[i]);
        }
        if (lane + 32 < cnt) {
          const int i = i0 + lane + 32, pp = sp[i / ch];
          kn1 = tm[pp] != 0;
          xw[lane + 32] = __fsub_rn(tv[pp * ch + i % ch], mu[i]);
        }
        const uint32_t m0 = __ballot_sync(0xffffffffu, kn0), m1 = __ballot_sync(0xffffffffu, kn1);
        const float* Bc = B + (int64_t)i0 * a.D;
        for (int u = lane; u < cnt * a.D; u += 32) bw[u] = Bc[u];
        __syncwarp();
        if (lane < a.D) {
#pragma unroll 4
          for (int u = 0; u < cnt; ++u) {
            const uint32_t mw = u < 32 ? m0 : m1;
            const float r = __fmaf_rn(bw[u * a.D + lane], xw[u], acc);
            acc = ((mw >> (u & 31)) & 1u) ? r : acc;
          }
        }
        __syncwarp();
      }
    }
    uint32_t qk = 0;
    if (lane < a.D) qk = quantise_one(acc, I.lo[c * a.D + lane], I.scale[c * a.D + lane], a.bits) +
                         (uint32_t)I.shifts[c * a.D + lane];
    const uint64_t key = a.curve == SFC_CURVE_HILBERT ? warp_hilbert_key(qk, a.D, a.bp) : warp_key(qk, a.D, a.bp);
    const uint64_t* sk = I.skeys + (int64_t)c * I.N;
    int64_t pos = warp_lower_bound(sk, I.N, key);
    if (KNN) {
      warp_knn(sk, I.sqc + (int64_t)c * I.N * a.D, I.sids + (int64_t)c * I.N, I.N, a.D, a.bp, qk, (int)len,
               cand + slot * len, knn_stack + warp * kKnnStack);
    } else {
      int64_t start = pos - a.W / 2;
      if (start > maxs) start = maxs;
      if (start < 0) start = 0;
      const uint32_t* si = I.sids + (int64_t)c * I.N + start;
      for (int64_t i = lane; i < len; i += 32) cand[slot * len + i] = si[i];
    }
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
    const int cap = a.C * a.capw;
    for (int i = tid; i < cap; i += kQThreads) a.cand_out[q * cap + i] = i < ncand ? (int32_t)ucand[i] : -1;
    if (tid == 0) a.ncand_out[q] = ncand;
  }
  if (!a.pick) return;

  // --- FP32 rescore --------------------------------------------------------
  const int nk = compact_known<WEIGHTED>(n, ch, tm, deo, tv, a.weights, ceo, ct, cw, s_part);
  float tr[MAXE], wv[MAXE];
  int eor[MAXE];
  lane_elems<MAXE>(nk, ceo, ct, cw, tr, eor, wv);
  // the L2 / L1 choice is uniform: one specialised loop each, no test per element
  const float wmin = a.l1 ? rescore_all<MAXE, WEIGHTED, true>(I.dgrid, I.dict, ucand, ncand, ch, nk, tr, eor, wv, c32)
                          : rescore_all<MAXE, WEIGHTED, false>(I.dgrid, I.dict, ucand, ncand, ch, nk, tr, eor, wv, c32);
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
      const double c64 = exact_cost64(I.dgrid, (int64_t)I.dict[j] * ch, tv, tm, deo, P, ch, a.weights, a.l1 != 0);
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

// ---------------------------------------------------------------------------
// Split form for small batches (a few queries; the fill loop asks one per
// step).  One CTA per query leaves most SMs idle while it rescores its C * W
// candidates two per warp at a time; here the rescore is spread out:
//   k_query with pick == nullptr writes each query's de-duplicated candidates;
//   k_qs_rescore: CTA (b, q) rescores slots [b S, (b + 1) S) of query q with
//     rescore_all, i.e. per candidate the same FP32 operations in the same
//     order as the one-CTA kernel (the costs are bit-identical);
//   k_qs_pick: the FP32 minimum, the band and the FP64 decision over (cost,
//     slot) exactly as the one-CTA kernel takes them.
constexpr int kQsSlice = 2 * kQWarps;  // candidates per rescoring CTA: one pass of rescore_all
constexpr int64_t kQsMaxQ = 32;        // batches up to this size take the split form

template <int MAXE, bool WEIGHTED, bool L1>
__global__ void __launch_bounds__(kQThreads) k_qs_rescore(QArgs a) {
  const int64_t q = blockIdx.y;
  const int cap = a.C * a.capw;
  const int nc = a.ncand_out[q];  // 0: invalid centre
  const int c0 = blockIdx.x * kQsSlice;
  if (c0 >= nc) return;
  const QImg& I = a.imgs ? a.imgs[a.img_of[q]] : a.img;  // nc > 0: a valid image
  const Geo& g = I.g;
  const int n = g.n;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tv = reinterpret_cast<float*>(smem_raw);  // n
  int* deo = reinterpret_cast<int*>(tv + n);       // n
  int* ceo = deo + n;                              // n
  float* ct = reinterpret_cast<float*>(ceo + n);   // n
  float* cw = ct + n;                              // n
  uint8_t* tm = reinterpret_cast<uint8_t*>(cw + n);  // P
  __shared__ uint32_t s_part[kQWarps];
  const int64_t cx = a.centres[q * g.ndim + 0], cy = a.centres[q * g.ndim + 1];
  const int64_t cz = g.ndim == 3 ? a.centres[q * g.ndim + 2] : 0;
  stage_target(I, lin_of(g, cx, cy, cz), tv, deo, tm);
  __syncthreads();
  const int nk = compact_known<WEIGHTED>(n, g.ch, tm, deo, tv, a.weights, ceo, ct, cw, s_part);
  float tr[MAXE], wv[MAXE];
  int eor[MAXE];
  lane_elems<MAXE>(nk, ceo, ct, cw, tr, eor, wv);
  const int cnt = nc - c0 < kQsSlice ? nc - c0 : kQsSlice;
  rescore_all<MAXE, WEIGHTED, L1>(I.dgrid, I.dict, reinterpret_cast<const uint32_t*>(a.cand_out) + q * cap + c0, cnt,
                                  g.ch, nk, tr, eor, wv, a.c32_out + q * cap + c0);
}

__global__ void __launch_bounds__(kQThreads) k_qs_pick(QArgs a) {
  const int64_t q = blockIdx.x;
  const int cap = a.C * a.capw;
  const int nc = a.ncand_out[q];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (nc == 0) {  // invalid centre (k_query raised ST_BAD_CENTRE)
    if (tid == 0) {
      a.pick[q] = -1;
      a.cost[q] = __int_as_float(0x7fc00000);
    }
    return;
  }
  const QImg& I = a.imgs ? a.imgs[a.img_of[q]] : a.img;  // nc > 0: a valid image
  const Geo& g = I.g;
  const float* c32 = a.c32_out + q * cap;
  const uint32_t* uc = reinterpret_cast<const uint32_t*>(a.cand_out) + q * cap;
  __shared__ float s_redf[kQWarps];
  __shared__ int s_cnt[kQWarps];
  __shared__ double s_redd[kQWarps];
  __shared__ int64_t s_redi[kQWarps];
  float m = INFINITY;
  for (int ci = tid; ci < nc; ci += kQThreads) m = fminf(m, c32[ci]);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fminf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if (lane == 0) s_redf[warp] = m;
  __syncthreads();
  float m32 = s_redf[0];
  for (int w = 1; w < kQWarps; ++w) m32 = fminf(m32, s_redf[w]);
  const float T = band_limit32(m32, g.n);
  int nband = 0, mine = -1;
  for (int ci = tid; ci < nc; ci += kQThreads)
    if (c32[ci] <= T) {
      ++nband;
      mine = ci;
    }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) nband += __shfl_xor_sync(0xffffffffu, nband, o);
  if (lane == 0) s_cnt[warp] = nband;
  __syncthreads();
  int total = 0;
  for (int w = 0; w < kQWarps; ++w) total += s_cnt[w];
  if (total == 1) {
    if (mine >= 0) {
      a.pick[q] = uc[mine];
      a.cost[q] = c32[mine];
    }
    return;
  }
  // near-ties: the exact FP64 cost of every band member, (cost, slot) minimum
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* tv = reinterpret_cast<float*>(smem_raw);    // n
  int* deo = reinterpret_cast<int*>(tv + g.n);       // n
  uint8_t* tm = reinterpret_cast<uint8_t*>(deo + g.n);  // P
  const int64_t cx = a.centres[q * g.ndim + 0], cy = a.centres[q * g.ndim + 1];
  const int64_t cz = g.ndim == 3 ? a.centres[q * g.ndim + 2] : 0;
  stage_target(I, lin_of(g, cx, cy, cz), tv, deo, tm);
  __syncthreads();
  double bc = INFINITY;
  int64_t bi = INT64_MAX;
  for (int ci = tid; ci < nc; ci += kQThreads) {
    if (c32[ci] <= T) {
      const double c64 = exact_cost64(I.dgrid, (int64_t)I.dict[uc[ci]] * g.ch, tv, tm, deo, g.P, g.ch, a.weights,
                                      a.l1 != 0);
      if (c64 < bc || (c64 == bc && ci < bi)) {
        bc = c64;
        bi = ci;
      }
    }
  }
  warp_argmin64(bc, bi);
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
    if (i == INT64_MAX) {
      a.pick[q] = -1;
      a.cost[q] = __int_as_float(0x7fc00000);
    } else {
      a.pick[q] = uc[i];
      a.cost[q] = c32[i];
    }
  }
}

template <int MAXE, bool W, bool KNN, bool MULTI>
int launch_q3(const QArgs& a, int64_t Q, size_t shm, cudaStream_t st) {
  if (shm > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_query<MAXE, W, KNN, MULTI>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)shm));
  count_launch();
  k_query<MAXE, W, KNN, MULTI><<<(unsigned)Q, kQThreads, shm, st>>>(a);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

// the multi-image launch runs the window search (no k-NN variant)
template <int MAXE, bool W>
int launch_q(const QArgs& a, int64_t Q, size_t shm, cudaStream_t st) {
  if (a.imgs) return launch_q3<MAXE, W, false, true>(a, Q, shm, st);
  return a.knn > 0 ? launch_q3<MAXE, W, true, false>(a, Q, shm, st) : launch_q3<MAXE, W, false, false>(a, Q, shm, st);
}

template <bool W>
int dispatch_q(const QArgs& a, int64_t Q, size_t shm, cudaStream_t st) {
  const int need = (a.img.g.n + 31) / 32;
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

namespace {

// The image descriptor of an index with its grid(s).
QImg image_of(const Index& ix, const float* grid, const uint8_t* cur_mask, const TargetGrid* tgt) {
  QImg I;
  I.grid = grid;
  I.dgrid = tgt ? tgt->dict_grid : grid;
  I.deoff = ix.eoff_all;
  I.mask = cur_mask;
  I.g = tgt ? tgt->g : ix.g;
  I.N = ix.N;
  I.sqc = ix.sqc;
  I.dict = ix.dict;
  I.sub_pix = ix.sub_pix;
  I.basis = ix.basis;
  I.mean = ix.mean;
  I.lo = ix.lo;
  I.scale = ix.scale;
  I.shifts = ix.shifts;
  I.skeys = ix.skeys;
  I.sids = ix.sids;
  I.eoff_all = tgt ? tgt->eoff : ix.eoff_all;
  return I;
}

// The fields shared by every query of a launch; maxN: the largest dictionary.
int common_args(const Index& ix, int64_t maxN, QArgs& a) {
  a.C = ix.C;
  a.D = ix.D;
  a.bits = ix.bits;
  a.bp = ix.bp;
  a.W = ix.W;
  a.select = ix.select;
  a.m = ix.m;
  a.s = ix.s;
  a.maxsel = ix.select == SFC_SELECT_BEST ? 1 : ix.C;
  a.knn = ix.knn;
  a.curve = ix.curve;
  a.l1 = ix.l1 ? 1 : 0;
  a.capw = ix.knn > 0 ? ix.knn : ix.W;
  if (ix.knn > 0 && !ix.sqc) {
    set_error("k-NN search without the index's quantised coordinates");
    return SFC_EINVAL;
  }
  const int64_t wk = ix.knn > 0 ? ix.knn : ix.W;
  const int64_t len = wk < maxN ? wk : maxN;
  const int64_t need = len * a.maxsel;
  int L = 2;
  while (L < need) L <<= 1;
  if (L > 8192) {
    set_error("curves * window (or k) exceeds 8192 candidates per query");
    return SFC_EINVAL;
  }
  a.L = L;
  a.weights = ix.weights;
  a.imgs = nullptr;
  a.img_of = nullptr;
  a.nimg = 0;
  a.c32_out = nullptr;
  a.status = status_word();
  return SFC_OK;
}

bool index_weighted(const Index& ix) {
  bool weighted = false;
  for (float w : ix.weights_h) weighted |= (w != 1.0f);
  return weighted;
}

int launch_query(const Index& ix, const QArgs& a, int64_t Q, cudaStream_t st) {
  const size_t shm = (size_t)ix.g.n * 20 + (size_t)a.L * 12 + sizeof(float) * kQWarps * kXChunk * (1 + ix.D) +
                     (size_t)ix.g.P +
                     (ix.knn > 0 ? 16 + sizeof(KnnRegion) * kKnnStack * kQWarps : 0);
  return index_weighted(ix) ? dispatch_q<true>(a, Q, shm, st) : dispatch_q<false>(a, Q, shm, st);
}

template <int MAXE>
void launch_qs_rescore(const QArgs& a, bool weighted, dim3 grd, size_t shm, cudaStream_t st) {
  if (weighted)
    a.l1 ? k_qs_rescore<MAXE, true, true><<<grd, kQThreads, shm, st>>>(a)
         : k_qs_rescore<MAXE, true, false><<<grd, kQThreads, shm, st>>>(a);
  else
    a.l1 ? k_qs_rescore<MAXE, false, true><<<grd, kQThreads, shm, st>>>(a)
         : k_qs_rescore<MAXE, false, false><<<grd, kQThreads, shm, st>>>(a);
}

// The split form (kernels above) of a batch of Q <= kQsMaxQ queries with
// picks; cand / ncand / c32: Q * (C * capw), Q, Q * (C * capw) device words.
int launch_query_split(const Index& ix, const QArgs& a, int64_t Q, int32_t* cand, int32_t* ncand, float* c32,
                       cudaStream_t st) {
  QArgs a1 = a;
  a1.pick = nullptr;
  a1.cost = nullptr;
  a1.cand_out = cand;
  a1.ncand_out = ncand;
  SFC_CHECK(launch_query(ix, a1, Q, st));
  QArgs a2 = a;
  a2.qkeys = nullptr;
  a2.pos = nullptr;
  a2.cand_out = cand;
  a2.ncand_out = ncand;
  a2.c32_out = c32;
  const int n = ix.g.n, P = ix.g.P, need = (n + 31) / 32;
  const int cap = a.C * a.capw;
  const dim3 grd((unsigned)((cap + kQsSlice - 1) / kQsSlice), (unsigned)Q);
  const size_t shm_r = (size_t)n * 20 + (size_t)P;
  const bool w = index_weighted(ix);
  count_launch();
  if (need <= 4) launch_qs_rescore<4>(a2, w, grd, shm_r, st);
  else if (need <= 8) launch_qs_rescore<8>(a2, w, grd, shm_r, st);
  else if (need <= 12) launch_qs_rescore<12>(a2, w, grd, shm_r, st);
  else if (need <= 16) launch_qs_rescore<16>(a2, w, grd, shm_r, st);
  else if (need <= 24) launch_qs_rescore<24>(a2, w, grd, shm_r, st);
  else launch_qs_rescore<32>(a2, w, grd, shm_r, st);  // n <= 1024: checked by launch_query
  SFC_TRY(cudaGetLastError());
  count_launch();
  k_qs_pick<<<(unsigned)Q, kQThreads, (size_t)n * 8 + (size_t)P, st>>>(a2);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

}  // namespace

int64_t query_split_cap(const Index& ix) { return (int64_t)ix.C * (ix.knn > 0 ? ix.knn : ix.W); }

int query_batch(const Index& ix, const float* grid, const uint8_t* cur_mask, const int32_t* centres, int64_t Q,
                int64_t* pick, float* cost, uint64_t* qkeys, int64_t* pos, int32_t* cand, int32_t* ncand,
                cudaStream_t st, const TargetGrid* tgt, const QSplit* split) {
  if (Q <= 0) return SFC_OK;
  if (Q > 0x7fffffffLL) {
    set_error("too many queries in one batch");
    return SFC_EINVAL;
  }
  QArgs a;
  SFC_CHECK(common_args(ix, ix.N, a));
  a.img = image_of(ix, grid, cur_mask, tgt);
  a.centres = centres;
  a.pick = pick;
  a.cost = cost;
  a.qkeys = qkeys;
  a.pos = pos;
  a.cand_out = cand;
  a.ncand_out = ncand;
  a.c32_out = nullptr;
  if (pick && !cand && Q <= kQsMaxQ) {
    // a small batch: the split form, in the caller's buffers or in stream-ordered
    // scratch (not while the stream is being captured: then the one-CTA form)
    const int64_t cap = (int64_t)a.C * a.capw;
    if (split && split->cap >= cap && split->qmax >= Q)
      return launch_query_split(ix, a, Q, split->cand, split->ncand, split->c32, st);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusActive;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      Scratch scr(st);
      int32_t *sc = nullptr, *sn = nullptr;
      float* sf = nullptr;
      SFC_TRY(scr.alloc(&sc, sizeof(int32_t) * Q * cap));
      SFC_TRY(scr.alloc(&sn, sizeof(int32_t) * Q));
      SFC_TRY(scr.alloc(&sf, sizeof(float) * Q * cap));
      return launch_query_split(ix, a, Q, sc, sn, sf, st);
    }
    cudaGetLastError();
  }
  return launch_query(ix, a, Q, st);
}

// Several images, one launch: every index built with the same parameters
// (patch, curves, dimensions, bits, window / k, selection, curve, cost,
// channel weights, subsets); query q belongs to image img_of[q].
struct MultiQuery {
  const Index* first = nullptr;  // the parameters (indices outlive the object)
  QImg* imgs = nullptr;          // device, one per image
  int64_t maxN = 0;
  int n = 0;
};

int multi_query_create(const Index* const* ixs, const float* const* grids, const uint8_t* const* masks, int n,
                       cudaStream_t st, MultiQuery** out) {
  if (n < 1) {
    set_error("sfc_multi_create: no images");
    return SFC_EINVAL;
  }
  const Index& f = *ixs[0];
  if (f.knn > 0) {
    set_error("sfc_multi_create: the multi-image launch runs the window search (build with knn = 0)");
    return SFC_EUNSUPPORTED;
  }
  std::vector<QImg> h(n);
  int64_t maxN = 0;
  for (int i = 0; i < n; ++i) {
    const Index& x = *ixs[i];
    const bool same = x.g.ndim == f.g.ndim && x.g.ch == f.g.ch && x.g.K == f.g.K && x.C == f.C && x.D == f.D &&
                      x.bits == f.bits && x.bp == f.bp && x.W == f.W && x.select == f.select && x.m == f.m &&
                      x.s == f.s && x.knn == f.knn && x.curve == f.curve && x.l1 == f.l1 &&
                      x.weights_h == f.weights_h && x.subset_h == f.subset_h;
    if (!same) {
      set_error("sfc_multi_create: index " + std::to_string(i) + " was built with other parameters than index 0");
      return SFC_EINVAL;
    }
    if (!grids[i] || !masks[i]) {
      set_error("sfc_multi_create: NULL grid or mask");
      return SFC_EINVAL;
    }
    h[i] = image_of(x, grids[i], masks[i], nullptr);
    maxN = std::max(maxN, x.N);
  }
  auto* m = new MultiQuery();
  m->first = &f;
  m->n = n;
  m->maxN = maxN;
  if (pmalloc(&m->imgs, sizeof(QImg) * n, st) != cudaSuccess ||
      cudaMemcpyAsync(m->imgs, h.data(), sizeof(QImg) * n, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    if (m->imgs) cudaFree(m->imgs);
    delete m;
    set_error("sfc_multi_create: out of device memory");
    return SFC_ENOMEM;
  }
  *out = m;
  return SFC_OK;
}

void multi_query_destroy(MultiQuery* m) {
  if (!m) return;
  cudaDeviceSynchronize();
  if (m->imgs) cudaFreeAsync(m->imgs, nullptr);
  cudaStreamSynchronize(nullptr);
  delete m;
}

int multi_query_run(const MultiQuery* m, const int32_t* img_of, const int32_t* centres, int64_t Q, int64_t* pick,
                    float* cost, cudaStream_t st, const QSplit* split) {
  if (Q <= 0) return SFC_OK;
  if (Q > 0x7fffffffLL) {
    set_error("too many queries in one batch");
    return SFC_EINVAL;
  }
  QArgs a;
  SFC_CHECK(common_args(*m->first, m->maxN, a));
  a.img = image_of(*m->first, nullptr, nullptr, nullptr);  // unused: every CTA reads imgs
  a.imgs = m->imgs;
  a.img_of = img_of;
  a.nimg = m->n;
  a.centres = centres;
  a.pick = pick;
  a.cost = cost;
  a.qkeys = nullptr;
  a.pos = nullptr;
  a.cand_out = nullptr;
  a.ncand_out = nullptr;
  // the split form only in the caller's buffers (the public entry point is one
  // launch with no allocation)
  if (split && Q <= kQsMaxQ && split->cap >= (int64_t)a.C * a.capw && split->qmax >= Q)
    return launch_query_split(*m->first, a, Q, split->cand, split->ncand, split->c32, st);
  return launch_query(*m->first, a, Q, st);
}

}  // namespace sfc
