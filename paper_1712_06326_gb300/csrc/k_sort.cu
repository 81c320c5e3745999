// k_sort.cu -- stable LSD radix sort of (64-bit key, 32-bit id) pairs, one sort
// per index, all indices in the same launches (Sec. II.C: the dictionary is sorted
// by z-order; a stable sort from id order gives the order (key, id)).
//
// Scheme: "onesweep" (Adinets & Merrill, 2022).  One up-front kernel counts the
// 8-bit digits of every pass; then each pass is a single kernel in which a CTA
// takes the next tile (dynamic tile counter, so tiles start in order), ranks its
// keys stably (warp match-any ranking), publishes its per-digit count, looks back
// over the preceding tiles' published counts (decoupled look-back) to find its
// per-digit offset, and scatters through shared memory so the global writes of a
// digit run are contiguous.  Look-back spins are bounded (kSpinLimit): on
// timeout the CTA raises ST_TIMEOUT in the status word and carries on, so the
// device never hangs.  Only the passes covering the key bits in use run.
//
// Dictionaries of up to 2^20 entries per index take a sample sort instead
// (below): the same order -- the ids enter in ascending order, so the stable
// order by key is the order of the unique pairs (key, id) -- in five launches
// that read and write every pair about twice instead of eight times.
#include <atomic>

#include "internal.cuh"

namespace sfc {

namespace {

// Failure injection for tests (sfc_debug_lookback): the look-back's poll limit,
// and a switch that makes every look-back poll a word nothing ever writes.
std::atomic<long long> g_spin_limit{kSpinLimit};
std::atomic<int> g_stall{0};
__device__ uint32_t g_never_set[256];  // zero, never written

constexpr int kThreads = 256;
constexpr int kItems = 12;
constexpr int kTileKeys = kThreads * kItems;  // 3072
constexpr int kWarps = kThreads / 32;
constexpr int kLook = 4;  // look-back window: predecessor tiles read at once
constexpr uint32_t kFlagAgg = 1u << 30, kFlagPrefix = 2u << 30, kValMask = (1u << 30) - 1u;

__global__ void k_hist(const uint64_t* __restrict__ keys, int64_t N, int npass, uint32_t* __restrict__ hist) {
  const int c = blockIdx.y;
  __shared__ uint32_t h[8][256];
  for (int t = threadIdx.x; t < 8 * 256; t += blockDim.x) (&h[0][0])[t] = 0;
  __syncthreads();
  const uint64_t* k = keys + (int64_t)c * N;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x) {
    uint64_t key = k[i];
    for (int p = 0; p < npass; ++p) atomicAdd(&h[p][(key >> (8 * p)) & 255u], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < npass * 256; t += blockDim.x) {
    uint32_t v = (&h[0][0])[t];
    if (v) atomicAdd(&hist[((int64_t)c * 8 + t / 256) * 256 + t % 256], v);
  }
}

// hist[c][p][d] -> goffs[p][c][d]: the exclusive prefix over d of index c's
// digit counts of pass p, laid out as the pass reads it.
__global__ void k_hist_scan(const uint32_t* __restrict__ hist, uint32_t* __restrict__ goffs) {
  const uint32_t* h = hist + ((int64_t)blockIdx.y * 8 + blockIdx.x) * 256;
  __shared__ uint32_t s[256];
  const int d = threadIdx.x, lane = d & 31, warp = d >> 5;
  const uint32_t v = h[d];
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) s[warp] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += s[w];
  goffs[((int64_t)blockIdx.x * gridDim.y + blockIdx.y) * 256 + d] = before + incl - v;
}

// One onesweep pass over every index's keys.  in_vals == nullptr: the values are
// the ids (first pass).
__global__ void __launch_bounds__(kThreads, 3) k_onesweep(const uint64_t* __restrict__ in_keys,
                                                       const uint32_t* __restrict__ in_vals,
                                                       uint64_t* __restrict__ out_keys,
                                                       uint32_t* __restrict__ out_vals, int64_t N, int shift,
                                                       const uint32_t* __restrict__ goffs,  // [C][256] this pass
                                                       uint32_t* __restrict__ status,       // [C][ntiles][256]
                                                       uint32_t* __restrict__ tile_ctr,     // [C]
                                                       int64_t ntiles, uint32_t* __restrict__ err,
                                                       long long spin_limit, int stall) {
  const int c = blockIdx.y;
  __shared__ uint32_t s_tile;
  __shared__ uint32_t whist[kWarps][256];  // per-warp counts -> per-warp exclusive offsets
  __shared__ uint32_t tcount[256];         // tile count per digit
  __shared__ uint32_t tstart[256];         // tile-local exclusive start per digit
  __shared__ uint32_t gbase[256];          // global position of the tile's first key of digit d
  __shared__ uint64_t skey[kTileKeys];
  __shared__ uint32_t sval[kTileKeys];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(&tile_ctr[c], 1u);
  for (int t = threadIdx.x; t < kWarps * 256; t += kThreads) (&whist[0][0])[t] = 0;
  tcount[threadIdx.x] = 0;
  __syncthreads();
  const int64_t tile = s_tile;
  const int64_t base = tile * kTileKeys + (int64_t)warp * 32 * kItems;
  const uint64_t* ik = in_keys + (int64_t)c * N;
  const uint32_t* iv = in_vals ? in_vals + (int64_t)c * N : nullptr;

  // digits are recomputed from the keys where needed (fewer registers, so
  // three CTAs fit an SM); items past N get the singleton group 256 + lane
  uint64_t key[kItems];
  uint32_t val[kItems];
  uint32_t rnk[kItems];
  const int64_t nvalid = N - base;  // items k * 32 + lane < nvalid are valid
#define DIG(k) (((int64_t)(k) * 32 + lane < nvalid) ? (int)((key[k] >> shift) & 255u) : 256 + lane)
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    int64_t idx = base + k * 32 + lane;
    bool ok = idx < N;
    key[k] = ok ? ik[idx] : 0ull;
    val[k] = ok ? (iv ? iv[idx] : (uint32_t)idx) : 0u;
  }
  // the tile's digit counts first, published at once (the successors' look-
  // backs then wait on this tile's ranking no longer)
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int dg = DIG(k);
    if (dg < 256) atomicAdd(&tcount[dg], 1u);
  }
  __syncthreads();
  {
    uint32_t* st = status + ((int64_t)c * ntiles) * 256;
    const int d = threadIdx.x;
    atomicExch(&st[tile * 256 + d], (tile == 0 ? kFlagPrefix : kFlagAgg) | tcount[d]);
  }
  // stable rank inside the warp, items in order, lanes in order; the lanes
  // holding the same digit are found with one ballot per digit bit
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int dg = DIG(k);
    const bool in = dg < 256;
    unsigned peers = __ballot_sync(0xffffffffu, in);
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const bool bit = (dg >> b) & 1;
      const unsigned bal = __ballot_sync(0xffffffffu, bit);
      peers &= bit ? bal : ~bal;
    }
    if (!in) peers = 1u << lane;
    unsigned before = peers & ((1u << lane) - 1u);
    uint32_t b = dg < 256 ? whist[warp][dg] : 0u;
    rnk[k] = b + __popc(before);
    __syncwarp();
    if (dg < 256 && before == 0) whist[warp][dg] = b + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // per-digit: exclusive offsets of the warps, tile total
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
    for (int w = 0; w < kWarps; ++w) {
      uint32_t v = whist[w][d];
      whist[w][d] = run;
      run += v;
    }
    // (run == tcount[d], the count published above)  look back
    uint32_t* st = status + ((int64_t)c * ntiles) * 256;
    uint32_t excl = 0;
    if (tile != 0) {
      // the predecessors' words are read kLook at a time (independent loads),
      // then taken in order: aggregates summed until an inclusive prefix; a
      // word not yet published ends the window and is polled again
      int64_t j = tile - 1;
      long long spins = 0;
      const uint32_t before_first = kFlagPrefix;  // "tile -1": an empty inclusive prefix
      while (j >= 0) {
        uint32_t v[kLook];
#pragma unroll
        for (int u = 0; u < kLook; ++u)
          v[u] = stall ? *((volatile uint32_t*)&g_never_set[d])
                       : (j - u >= 0 ? *((volatile uint32_t*)&st[(j - u) * 256 + d]) : before_first);
        int used = 0;
        bool found = false;
#pragma unroll
        for (int u = 0; u < kLook; ++u) {
          if (found || used < u || v[u] == 0) continue;
          excl += v[u] & kValMask;
          found = (v[u] & kFlagPrefix) != 0;
          used = u + 1;
        }
        if (found) break;
        if (used == 0) {
          if (++spins > spin_limit) {
            atomicOr(err, ST_TIMEOUT);
            break;
          }
          __nanosleep(20);
          continue;
        }
        j -= used;
      }
      atomicExch(&st[tile * 256 + d], kFlagPrefix | ((excl + run) & kValMask));
    }
    gbase[d] = goffs[c * 256 + d] + excl;
  }
  __syncthreads();
  // tile-local starts: exclusive scan of tcount over digits (warp 0)
  if (warp == 0) {
    uint32_t loc[8];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      loc[i] = tcount[lane * 8 + i];
      sum += loc[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      tstart[lane * 8 + i] = run;
      run += loc[i];
    }
  }
  __syncthreads();
  // place into shared memory in tile-sorted order
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int dg = DIG(k);
    if (dg < 256) {
      uint32_t pos = tstart[dg] + whist[warp][dg] + rnk[k];
      skey[pos] = key[k];
      sval[pos] = val[k];
    }
  }
#undef DIG
  __syncthreads();
  int64_t valid = N - tile * kTileKeys;
  if (valid > kTileKeys) valid = kTileKeys;
  uint64_t* ok_ = out_keys + (int64_t)c * N;
  uint32_t* ov = out_vals + (int64_t)c * N;
  for (int i = threadIdx.x; i < valid; i += kThreads) {
    uint64_t kk = skey[i];
    int d = (int)((kk >> shift) & 255u);
    int64_t dst = (int64_t)gbase[d] + (i - (int64_t)tstart[d]);
    if (dst < 0 || dst >= N) {  // only after a timed-out look-back
      atomicOr(err, ST_TIMEOUT);
      continue;
    }
    ok_[dst] = kk;
    ov[dst] = sval[i];
  }
}

}  // namespace

namespace {
struct SortLayout {
  int npass;
  int64_t ntiles;
  size_t hist, status, ctr, tk, tv, goffs, total;  // byte offsets / size
};
SortLayout sort_layout(int64_t N, int C, int key_bits) {
  SortLayout L;
  L.npass = (key_bits + 7) / 8;
  if (L.npass < 1) L.npass = 1;
  if (L.npass > 8) L.npass = 8;
  L.ntiles = (N + kTileKeys - 1) / kTileKeys;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o = 0;
  L.hist = o;
  o += up(sizeof(uint32_t) * C * 8 * 256);
  L.status = o;
  o += up(sizeof(uint32_t) * (size_t)L.npass * C * L.ntiles * 256);
  L.ctr = o;
  o += up(sizeof(uint32_t) * L.npass * C);
  L.tk = o;
  o += up(sizeof(uint64_t) * C * N);
  L.tv = o;
  o += up(sizeof(uint32_t) * C * N);
  L.goffs = o;
  o += up(sizeof(uint32_t) * L.npass * C * 256);
  L.total = o;
  return L;
}
}  // namespace

void sort_lookback_test(long long spin_limit, int stall) {
  g_spin_limit.store(spin_limit > 0 ? spin_limit : kSpinLimit);
  g_stall.store(stall ? 1 : 0);
}

size_t radix_sort_scratch_bytes(int64_t N, int C, int key_bits) { return N > 0 ? sort_layout(N, C, key_bits).total : 0; }

int radix_sort_pairs(const uint64_t* keys, uint64_t* skeys, uint32_t* sids, int64_t N, int C, int key_bits,
                     cudaStream_t st, void* scratch) {
  if (N <= 0) return SFC_OK;
  if (N >= (int64_t)kValMask) {
    set_error("dictionary too large for the radix sort (>= 2^30 entries per index)");
    return SFC_EINVAL;
  }
  const SortLayout L = sort_layout(N, C, key_bits);
  const int npass = L.npass;
  const int64_t ntiles = L.ntiles;
  unsigned char* ws = static_cast<unsigned char*>(scratch);
  Scratch scr(st);  // frees the sort's own scratch (if it takes one) on return
  if (!ws) SFC_TRY(scr.alloc(&ws, L.total));
  uint32_t* hist = reinterpret_cast<uint32_t*>(ws + L.hist);
  uint32_t* status = reinterpret_cast<uint32_t*>(ws + L.status);
  uint32_t* ctr = reinterpret_cast<uint32_t*>(ws + L.ctr);
  uint64_t* tk = reinterpret_cast<uint64_t*>(ws + L.tk);
  uint32_t* tv = reinterpret_cast<uint32_t*>(ws + L.tv);
  uint32_t* goffs = reinterpret_cast<uint32_t*>(ws + L.goffs);
  // hist, status and the tile counters are adjacent: one clear
  SFC_TRY(cudaMemsetAsync(ws + L.hist, 0, L.tk - L.hist, st));
  int hb = (int)((N + 1023) / 1024);
  if (hb > 1024) hb = 1024;
  count_launch();
  k_hist<<<dim3(hb, C), 256, 0, st>>>(keys, N, npass, hist);
  count_launch();
  k_hist_scan<<<dim3(npass, C), 256, 0, st>>>(hist, goffs);
  SFC_TRY(cudaGetLastError());
  const uint64_t* ink = keys;
  const uint32_t* inv = nullptr;
  for (int p = 0; p < npass; ++p) {
    const bool to_out = ((npass - 1 - p) % 2) == 0;
    uint64_t* ok_ = to_out ? skeys : tk;
    uint32_t* ov = to_out ? sids : tv;
    count_launch();
    k_onesweep<<<dim3((unsigned)ntiles, C), kThreads, 0, st>>>(ink, inv, ok_, ov, N, 8 * p,
                                                               goffs + (size_t)p * C * 256,
                                                               status + (size_t)p * C * ntiles * 256, ctr + p * C,
                                                               ntiles, status_word(), g_spin_limit.load(),
                                                               g_stall.load());
    SFC_TRY(cudaGetLastError());
    ink = ok_;
    inv = ov;
  }
  return SFC_OK;
}


// ---------------------------------------------------------------------------
// Sample sort of (key, id) pairs, ids 0..N-1, for N <= kSsMaxN (2^20) per index:
//   k_ss_sample  a stratified sample of S = kSsOver * B pairs per index
//                (stratum i = positions [i N / S, (i + 1) N / S), the position
//                inside it from a hash of (index, i)), cut into runs of
//                kSsRun, each merge-sorted in shared memory by its own CTA;
//   k_ss_pick    every sampled pair's rank in the whole sample (its place in
//                its run + binary searches in the other runs); the pairs of
//                ranks kSsOver - 1, 2 kSsOver - 1, ... are the B - 1 splitters;
//   k_ss_count   each pair's bucket = the number of splitters <= the pair
//                (binary search over the splitters in shared memory); bucket
//                totals;
//   k_ss_scan    bucket starts; an index whose largest bucket holds more than
//                the bucket capacity is flagged, and its pairs are left to the
//                LSD sort (the caller reads the flags);
//   k_ss_place   every pair to its bucket (one atomic per bucket and tile
//                reserves the tile's range; the order inside a bucket is
//                arbitrary);
//   k_ss_bucket  one CTA per bucket: merge sort of its pairs by (key, id) in
//                shared memory, written to the sorted arrays.
// B = the power of two >= N / 512 (average bucket <= 512 pairs, capacity
// 2,048).  A bucket's size is about a sum of 8 sample spacings (a Gamma(8)
// variable), so one above 4x the average is rare: ~1e-7 per bucket at 2^20
// entries, ~1e-9 at 0.9 M; the index is then sorted again by the LSD sort.
namespace {

constexpr int kSsOver = 8;              // samples per bucket
constexpr int kSsRun = 1024;            // sampled pairs per sorting CTA
constexpr int kSsCap = 2048;            // pairs per bucket sorted in shared memory
constexpr int kSsBucketE = 4;           // pairs per thread and chunk in the bucket sort
constexpr int kSsBucketThreads = 256;   // threads of a bucket-sorting CTA
constexpr int kSsTile = 256 * 16;       // pairs per CTA of the count / place passes
constexpr int64_t kSsMaxN = 1ll << 20;  // larger dictionaries: the LSD sort
std::atomic<int> g_ss_force_lsd{0};
std::atomic<int> g_ss_cap{kSsCap};

int ss_buckets(int64_t N) {
  int B = 1;
  while ((int64_t)B * 512 < N) B <<= 1;
  return B;
}

__device__ __forceinline__ uint32_t ss_hash(uint32_t c, uint32_t i) {
  // a 32-bit integer mix (murmur3 finaliser) of the index and the stratum
  uint32_t h = i * 0x9e3779b9u ^ (c + 0x7f4a7c15u);
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ bool pair_gt(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib) {
  return ka > kb || (ka == kb && ia > ib);
}

__device__ __forceinline__ void ce_pair(uint64_t& ka, uint32_t& va, uint64_t& kb, uint32_t& vb) {
  if (pair_gt(ka, va, kb, vb)) {
    const uint64_t tk = ka;
    const uint32_t tv = va;
    ka = kb;
    va = vb;
    kb = tk;
    vb = tv;
  }
}

// Pairs in shared memory as three 32-bit arrays (key high word, key low word,
// id), element i stored at i + i / 32: a warp reading elements 4 apart (or 1
// apart) touches 32 different banks.
struct SPairs {
  uint32_t* hi;
  uint32_t* lo;
  uint32_t* id;
};
__device__ __forceinline__ int sw(int i) { return i + (i >> 5); }
__host__ __device__ constexpr int sw_len(int n) { return n + (n >> 5) + 1; }
__device__ __forceinline__ SPairs spairs(uint32_t* base, int n) {
  const int L = sw_len(n);
  return SPairs{base, base + L, base + 2 * L};
}
__device__ __forceinline__ void sp_get(const SPairs& a, int i, uint64_t& k, uint32_t& v) {
  const int p = sw(i);
  k = ((uint64_t)a.hi[p] << 32) | a.lo[p];
  v = a.id[p];
}
__device__ __forceinline__ void sp_put(const SPairs& a, int i, uint64_t k, uint32_t v) {
  const int p = sw(i);
  a.hi[p] = (uint32_t)(k >> 32);
  a.lo[p] = (uint32_t)k;
  a.id[p] = v;
}

// Batcher's odd-even merge network on E = 4 or 8 pairs in registers.
template <int E>
__device__ __forceinline__ void sort_net(uint64_t (&k)[E], uint32_t (&v)[E]) {
#define CE(i, j) ce_pair(k[i], v[i], k[j], v[j])
  if (E == 4) {
    CE(0, 1); CE(2, 3); CE(0, 2); CE(1, 3); CE(1, 2);
  } else {
    CE(0, 1); CE(2, 3); CE(4, 5); CE(6, 7);
    CE(0, 2); CE(1, 3); CE(4, 6); CE(5, 7);
    CE(1, 2); CE(5, 6);
    CE(0, 4); CE(1, 5); CE(2, 6); CE(3, 7);
    CE(2, 4); CE(3, 5);
    CE(1, 2); CE(3, 4); CE(5, 6);
  }
#undef CE
}

// Merge sort of n pairs by (key, id) in shared memory, by the whole CTA: runs
// of E sorted in registers, then merge passes of doubling width, each thread
// producing E outputs per chunk from its merge-path split (a binary search on
// the output diagonal).  a holds the input; b is a second buffer.  Returns true
// if the result is in b.  The pairs are distinct, so no tie rule is needed.
template <int E>
__device__ bool merge_sort_pairs(const SPairs& a, const SPairs& b, int n) {
  const int T = blockDim.x;
  for (int o0 = threadIdx.x * E; o0 < n; o0 += T * E) {
    const int r = n - o0 < E ? n - o0 : E;
    uint64_t k[E];
    uint32_t v[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
      if (e < r) sp_get(a, o0 + e, k[e], v[e]);
      else {
        k[e] = ~0ull;
        v[e] = ~0u;
      }
    }
    sort_net<E>(k, v);
#pragma unroll
    for (int e = 0; e < E; ++e)
      if (e < r) sp_put(a, o0 + e, k[e], v[e]);
  }
  __syncthreads();
  bool in_b = false;
  for (int w = E; w < n; w <<= 1) {
    const SPairs& src = in_b ? b : a;
    const SPairs& dst = in_b ? a : b;
    for (int o0 = threadIdx.x * E; o0 < n; o0 += T * E) {
      const int p0 = o0 & ~(2 * w - 1);
      const int a1 = p0 + w < n ? p0 + w : n, b1 = p0 + 2 * w < n ? p0 + 2 * w : n;
      const int la = a1 - p0, lb = b1 - a1, d = o0 - p0;
      // i = how many of the first d outputs come from the first run
      int lo = d - lb > 0 ? d - lb : 0, hi = d < la ? d : la;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        uint64_t ka, kb;
        uint32_t va, vb;
        sp_get(src, p0 + mid, ka, va);
        sp_get(src, a1 + d - mid - 1, kb, vb);
        if (pair_gt(kb, vb, ka, va)) lo = mid + 1;
        else hi = mid;
      }
      int ia = p0 + lo, ib = a1 + d - lo;
      uint64_t ka = 0, kb = 0;
      uint32_t va = 0, vb = 0;
      if (ia < a1) sp_get(src, ia, ka, va);
      if (ib < b1) sp_get(src, ib, kb, vb);
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int o = o0 + e;
        if (o >= b1) break;
        const bool take_a = ib >= b1 || (ia < a1 && !pair_gt(ka, va, kb, vb));
        if (take_a) {
          sp_put(dst, o, ka, va);
          if (++ia < a1) sp_get(src, ia, ka, va);
        } else {
          sp_put(dst, o, kb, vb);
          if (++ib < b1) sp_get(src, ib, kb, vb);
        }
      }
    }
    __syncthreads();
    in_b = !in_b;
  }
  return in_b;
}

// grid (runs, indices): run r = sample slots [r kSsRun, (r + 1) kSsRun) of S
__global__ void __launch_bounds__(256) k_ss_sample(const uint64_t* __restrict__ keys, int64_t N, int S,
                                                   uint64_t* __restrict__ samk, uint32_t* __restrict__ sami) {
  const int c = blockIdx.y;
  const int i0 = blockIdx.x * kSsRun;
  const int n = S - i0 < kSsRun ? S - i0 : kSsRun;
  __shared__ uint32_t sm[6 * sw_len(kSsRun)];
  const SPairs pa = spairs(sm, n), pb = spairs(sm + 3 * sw_len(n), n);
  const uint64_t* k = keys + (int64_t)c * N;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = i0 + t;
    const int64_t lo = (int64_t)i * N / S, hi = (int64_t)(i + 1) * N / S;  // hi > lo: N >= S
    const int64_t j = lo + (int64_t)(ss_hash((uint32_t)c, (uint32_t)i) % (uint32_t)(hi - lo));
    sp_put(pa, t, k[j], (uint32_t)j);
  }
  __syncthreads();
  const SPairs& r = merge_sort_pairs<4>(pa, pb, n) ? pb : pa;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    uint64_t kk;
    uint32_t vv;
    sp_get(r, t, kk, vv);
    samk[(int64_t)c * S + i0 + t] = kk;
    sami[(int64_t)c * S + i0 + t] = vv;
  }
}

// grid (runs, indices), 1024 threads: the ranks of run blockIdx.x's pairs
__global__ void __launch_bounds__(1024) k_ss_pick(const uint64_t* __restrict__ samk, const uint32_t* __restrict__ sami,
                                                  int S, int B, uint64_t* __restrict__ splk,
                                                  uint32_t* __restrict__ spli) {
  const int c = blockIdx.y, r = blockIdx.x;
  const int nruns = (S + kSsRun - 1) / kSsRun;
  extern __shared__ __align__(16) unsigned char ss_smem[];
  uint64_t* rk = reinterpret_cast<uint64_t*>(ss_smem);  // the whole sample, run after run
  uint32_t* ri = reinterpret_cast<uint32_t*>(rk + S);
  for (int t = threadIdx.x; t < S; t += blockDim.x) {
    rk[t] = samk[(int64_t)c * S + t];
    ri[t] = sami[(int64_t)c * S + t];
  }
  __syncthreads();
  const int i0 = r * kSsRun;
  const int n = S - i0 < kSsRun ? S - i0 : kSsRun;
  for (int t = threadIdx.x; t < n; t += blockDim.x) {
    const uint64_t x = rk[i0 + t];
    const uint32_t xi = ri[i0 + t];
    int rank = t;
    for (int q = 0; q < nruns; ++q) {
      if (q == r) continue;
      // pairs of run q below (x, xi): lower bound (the pairs are distinct)
      int lo = q * kSsRun, hi = lo + (S - lo < kSsRun ? S - lo : kSsRun);
      const int q0 = lo;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (pair_gt(x, xi, rk[mid], ri[mid])) lo = mid + 1;
        else hi = mid;
      }
      rank += lo - q0;
    }
    if ((rank + 1) % kSsOver == 0 && rank / kSsOver < B - 1) {
      splk[(int64_t)c * (B - 1) + rank / kSsOver] = x;
      spli[(int64_t)c * (B - 1) + rank / kSsOver] = xi;
    }
  }
}

// the bucket of pair (key, j): the number of splitters <= (key, j)
__device__ __forceinline__ int ss_bucket(const uint64_t* sk, const uint32_t* si, int B, uint64_t key, uint32_t j) {
  int pos = 0;
  for (int step = B >> 1; step > 0; step >>= 1) {
    const int t = pos + step - 1;
    if (!pair_gt(sk[t], si[t], key, j)) pos += step;
  }
  return pos;
}

__global__ void __launch_bounds__(256) k_ss_count(const uint64_t* __restrict__ keys, int64_t N, int B,
                                                  const uint64_t* __restrict__ splk, const uint32_t* __restrict__ spli,
                                                  uint16_t* __restrict__ bkt, uint32_t* __restrict__ counts) {
  const int c = blockIdx.y;
  extern __shared__ __align__(16) unsigned char ss_smem[];
  uint64_t* sk = reinterpret_cast<uint64_t*>(ss_smem);
  uint32_t* si = reinterpret_cast<uint32_t*>(sk + (B - 1));
  uint32_t* h = si + (B - 1);
  for (int t = threadIdx.x; t < B - 1; t += blockDim.x) {
    sk[t] = splk[(int64_t)c * (B - 1) + t];
    si[t] = spli[(int64_t)c * (B - 1) + t];
  }
  for (int t = threadIdx.x; t < B; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const uint64_t* k = keys + (int64_t)c * N;
  uint16_t* bo = bkt + (int64_t)c * N;
  const int64_t j0 = (int64_t)blockIdx.x * kSsTile;
  for (int u = threadIdx.x; u < kSsTile; u += blockDim.x) {
    const int64_t j = j0 + u;
    if (j >= N) break;
    const int b = ss_bucket(sk, si, B, k[j], (uint32_t)j);
    bo[j] = (uint16_t)b;
    atomicAdd(&h[b], 1u);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < B; t += blockDim.x)
    if (h[t]) atomicAdd(&counts[(int64_t)c * B + t], h[t]);
}

// exclusive scan of the B <= 2048 bucket totals of one index (1024 threads)
__global__ void __launch_bounds__(1024) k_ss_scan(const uint32_t* __restrict__ counts, int B, int cap,
                                                  uint32_t* __restrict__ start, uint32_t* __restrict__ fill,
                                                  int* __restrict__ ovf) {
  const int c = blockIdx.x;
  __shared__ uint32_t ws[32];
  __shared__ uint32_t wmax[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint32_t* cn = counts + (int64_t)c * B;
  const int b0 = 2 * tid;
  const uint32_t v0 = b0 < B ? cn[b0] : 0u, v1 = b0 + 1 < B ? cn[b0 + 1] : 0u;
  const uint32_t sum = v0 + v1;
  uint32_t incl = sum, mx = v0 > v1 ? v0 : v1;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
    const uint32_t m2 = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = m2 > mx ? m2 : mx;
  }
  if (lane == 31) ws[warp] = incl;
  if (lane == 0) wmax[warp] = mx;
  __syncthreads();
  uint32_t before = 0;
  for (int w = 0; w < warp; ++w) before += ws[w];
  const uint32_t ex = before + incl - sum;
  uint32_t* st = start + (int64_t)c * (B + 1);
  if (b0 < B) st[b0] = ex;
  if (b0 + 1 < B) st[b0 + 1] = ex + v0;
  if (b0 < B) fill[(int64_t)c * B + b0] = 0u;
  if (b0 + 1 < B) fill[(int64_t)c * B + b0 + 1] = 0u;
  if (tid == 0) {
    uint32_t total = 0, m = 0;
    for (int w = 0; w < 32; ++w) {
      total += ws[w];
      m = wmax[w] > m ? wmax[w] : m;
    }
    st[B] = total;
    ovf[c] = m > (uint32_t)cap ? 1 : 0;
  }
}

__global__ void __launch_bounds__(256) k_ss_place(const uint64_t* __restrict__ keys, int64_t N, int B,
                                                  const uint16_t* __restrict__ bkt, const uint32_t* __restrict__ start,
                                                  uint32_t* __restrict__ fill, const int* __restrict__ ovf,
                                                  uint64_t* __restrict__ tk, uint32_t* __restrict__ tv) {
  constexpr int kPer = kSsTile / 256;
  const int c = blockIdx.y;
  if (ovf[c]) return;
  extern __shared__ __align__(16) unsigned char ss_smem[];
  uint32_t* h = reinterpret_cast<uint32_t*>(ss_smem);  // B: tile counts, then the tile's bases
  for (int t = threadIdx.x; t < B; t += blockDim.x) h[t] = 0;
  __syncthreads();
  const uint16_t* bi = bkt + (int64_t)c * N;
  const int64_t j0 = (int64_t)blockIdx.x * kSsTile;
  int b[kPer];
  uint32_t r[kPer];
#pragma unroll
  for (int u = 0; u < kPer; ++u) {
    const int64_t j = j0 + u * 256 + threadIdx.x;
    b[u] = j < N ? (int)bi[j] : -1;
    r[u] = b[u] >= 0 ? atomicAdd(&h[b[u]], 1u) : 0u;
  }
  __syncthreads();
  const uint32_t* st = start + (int64_t)c * (B + 1);
  for (int t = threadIdx.x; t < B; t += blockDim.x) {
    const uint32_t n = h[t];
    h[t] = n ? st[t] + atomicAdd(&fill[(int64_t)c * B + t], n) : 0u;
  }
  __syncthreads();
  const uint64_t* k = keys + (int64_t)c * N;
#pragma unroll
  for (int u = 0; u < kPer; ++u)
    if (b[u] >= 0) {
      const int64_t j = j0 + u * 256 + threadIdx.x;
      const int64_t pos = (int64_t)c * N + h[b[u]] + r[u];
      tk[pos] = k[j];
      tv[pos] = (uint32_t)j;
    }
}

__global__ void __launch_bounds__(kSsBucketThreads) k_ss_bucket(const uint64_t* __restrict__ tk, const uint32_t* __restrict__ tv,
                                                   int64_t N, int B, const uint32_t* __restrict__ start,
                                                   const int* __restrict__ ovf, uint64_t* __restrict__ skeys,
                                                   uint32_t* __restrict__ sids) {
  const int c = blockIdx.y, b = blockIdx.x;
  if (ovf[c]) return;
  const uint32_t* st = start + (int64_t)c * (B + 1);
  const int64_t s0 = st[b];
  const int M = (int)(st[b + 1] - s0);  // <= kSsCap (checked by k_ss_scan)
  if (M == 0) return;
  const int64_t base = (int64_t)c * N + s0;
  if (M == 1) {
    if (threadIdx.x == 0) {
      skeys[base] = tk[base];
      sids[base] = tv[base];
    }
    return;
  }
  extern __shared__ __align__(16) unsigned char ss_smem[];
  uint32_t* sm = reinterpret_cast<uint32_t*>(ss_smem);
  const SPairs pa = spairs(sm, M), pb = spairs(sm + 3 * sw_len(M), M);  // two buffers of the bucket
  for (int t = threadIdx.x; t < M; t += blockDim.x) sp_put(pa, t, tk[base + t], tv[base + t]);
  __syncthreads();
  const SPairs& r = merge_sort_pairs<kSsBucketE>(pa, pb, M) ? pb : pa;
  for (int t = threadIdx.x; t < M; t += blockDim.x) {
    uint64_t kk;
    uint32_t vv;
    sp_get(r, t, kk, vv);
    skeys[base + t] = kk;
    sids[base + t] = vv;
  }
}

struct SsLayout {
  int B;
  int64_t ntiles;
  size_t samk, sami, splk, spli, bkt, counts, start, fill, tk, tv, total;
};
SsLayout ss_layout(int64_t N, int C) {
  SsLayout L;
  L.B = ss_buckets(N);
  L.ntiles = (N + kSsTile - 1) / kSsTile;
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o = 0;
  const size_t B = (size_t)L.B;
  L.samk = o;
  o += up(sizeof(uint64_t) * C * kSsOver * B);
  L.sami = o;
  o += up(sizeof(uint32_t) * C * kSsOver * B);
  L.splk = o;
  o += up(sizeof(uint64_t) * C * (B > 1 ? B - 1 : 1));
  L.spli = o;
  o += up(sizeof(uint32_t) * C * (B > 1 ? B - 1 : 1));
  L.counts = o;
  o += up(sizeof(uint32_t) * C * B);
  L.start = o;
  o += up(sizeof(uint32_t) * C * (B + 1));
  L.fill = o;
  o += up(sizeof(uint32_t) * C * B);
  L.bkt = o;
  o += up(sizeof(uint16_t) * C * N);
  L.tk = o;
  o += up(sizeof(uint64_t) * C * N);
  L.tv = o;
  o += up(sizeof(uint32_t) * C * N);
  L.total = o;
  return L;
}

}  // namespace

bool sample_sort_fits(int64_t N) { return N >= 1 && N <= kSsMaxN && !g_ss_force_lsd.load(); }

size_t sample_sort_scratch_bytes(int64_t N, int C) { return N > 0 ? ss_layout(N, C).total : 0; }

void sample_sort_test(int force_lsd, int cap) {
  g_ss_force_lsd.store(force_lsd ? 1 : 0);
  g_ss_cap.store(cap > 0 && cap < kSsCap ? cap : kSsCap);
}

int sample_sort_pairs(const uint64_t* keys, uint64_t* skeys, uint32_t* sids, int64_t N, int C, int* ovf,
                      cudaStream_t st, void* scratch) {
  if (N <= 0) return SFC_OK;
  if (N > kSsMaxN) {
    set_error("sample sort: more than 2^20 entries per index");
    return SFC_EINVAL;
  }
  const SsLayout L = ss_layout(N, C);
  const int B = L.B;
  unsigned char* ws = static_cast<unsigned char*>(scratch);
  Scratch scr(st);
  if (!ws) SFC_TRY(scr.alloc(&ws, L.total));
  uint64_t* splk = reinterpret_cast<uint64_t*>(ws + L.splk);
  uint32_t* spli = reinterpret_cast<uint32_t*>(ws + L.spli);
  uint32_t* counts = reinterpret_cast<uint32_t*>(ws + L.counts);
  uint32_t* start = reinterpret_cast<uint32_t*>(ws + L.start);
  uint32_t* fill = reinterpret_cast<uint32_t*>(ws + L.fill);
  uint16_t* bkt = reinterpret_cast<uint16_t*>(ws + L.bkt);
  uint64_t* tk = reinterpret_cast<uint64_t*>(ws + L.tk);
  uint32_t* tv = reinterpret_cast<uint32_t*>(ws + L.tv);
  SFC_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * C * B, st));
  if (B > 1) {
    const int S = kSsOver * B, nruns = (S + kSsRun - 1) / kSsRun;
    uint64_t* samk = reinterpret_cast<uint64_t*>(ws + L.samk);
    uint32_t* sami = reinterpret_cast<uint32_t*>(ws + L.sami);
    count_launch();
    k_ss_sample<<<dim3(nruns, C), 256, 0, st>>>(keys, N, S, samk, sami);
    const size_t shm = (size_t)S * 12;  // the whole sample (<= 196,608 bytes)
    if (shm > kSmemOptIn)
      SFC_TRY(cudaFuncSetAttribute(k_ss_pick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    count_launch();
    k_ss_pick<<<dim3(nruns, C), 1024, shm, st>>>(samk, sami, S, B, splk, spli);
  }
  const dim3 tg((unsigned)L.ntiles, C);
  count_launch();
  k_ss_count<<<tg, 256, (size_t)(B - 1) * 12 + (size_t)B * 4, st>>>(keys, N, B, splk, spli, bkt, counts);
  count_launch();
  k_ss_scan<<<C, 1024, 0, st>>>(counts, B, g_ss_cap.load(), start, fill, ovf);
  count_launch();
  k_ss_place<<<tg, 256, (size_t)B * 4, st>>>(keys, N, B, bkt, start, fill, ovf, tk, tv);
  const size_t shm_b = sizeof(uint32_t) * 6 * (size_t)sw_len(kSsCap);  // two buffers of a bucket
  if (shm_b > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_ss_bucket, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_b));
  count_launch();
  k_ss_bucket<<<dim3((unsigned)B, C), kSsBucketThreads, shm_b, st>>>(tk, tv, N, B, start, ovf, skeys, sids);
  SFC_TRY(cudaGetLastError());
  return SFC_OK;
}

}  // namespace sfc
