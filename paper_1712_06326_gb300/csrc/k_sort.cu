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

// In place: hist[c][p][d] -> exclusive prefix over d.
__global__ void k_hist_scan(uint32_t* __restrict__ hist) {
  uint32_t* h = hist + ((int64_t)blockIdx.y * 8 + blockIdx.x) * 256;
  __shared__ uint32_t s[256];
  s[threadIdx.x] = h[threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int d = 0; d < 256; ++d) {
      uint32_t v = s[d];
      s[d] = run;
      run += v;
    }
  }
  __syncthreads();
  h[threadIdx.x] = s[threadIdx.x];
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
  // stable rank inside the warp, items in order, lanes in order
#pragma unroll
  for (int k = 0; k < kItems; ++k) {
    const int dg = DIG(k);
    unsigned peers = __match_any_sync(0xffffffffu, dg);
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
    tcount[d] = run;
    // publish own aggregate, then look back
    uint32_t* st = status + ((int64_t)c * ntiles) * 256;
    uint32_t excl = 0;
    if (tile == 0) {
      atomicExch(&st[d], kFlagPrefix | run);
    } else {
      atomicExch(&st[tile * 256 + d], kFlagAgg | run);
      int64_t j = tile - 1;
      long long spins = 0;
      while (j >= 0) {
        const uint32_t v = stall ? *((volatile uint32_t*)&g_never_set[d]) : *((volatile uint32_t*)&st[j * 256 + d]);
        if (v == 0) {
          if (++spins > spin_limit) {
            atomicOr(err, ST_TIMEOUT);
            break;
          }
          __nanosleep(20);
          continue;
        }
        excl += v & kValMask;
        if (v & kFlagPrefix) break;
        --j;
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
  const size_t status_words = (size_t)npass * C * ntiles * 256;
  SFC_TRY(cudaMemsetAsync(hist, 0, sizeof(uint32_t) * C * 8 * 256, st));
  SFC_TRY(cudaMemsetAsync(status, 0, sizeof(uint32_t) * status_words, st));
  SFC_TRY(cudaMemsetAsync(ctr, 0, sizeof(uint32_t) * npass * C, st));
  int hb = (int)((N + 1023) / 1024);
  if (hb > 1024) hb = 1024;
  count_launch();
  k_hist<<<dim3(hb, C), 256, 0, st>>>(keys, N, npass, hist);
  count_launch();
  k_hist_scan<<<dim3(npass, C), 256, 0, st>>>(hist);
  SFC_TRY(cudaGetLastError());
  // hist is laid out [C][8][256]; pass p needs the [C][256] slice of every index
  for (int p = 0; p < npass; ++p)
    SFC_TRY(cudaMemcpy2DAsync(goffs + (size_t)p * C * 256, 256 * sizeof(uint32_t), hist + (size_t)p * 256,
                              8 * 256 * sizeof(uint32_t), 256 * sizeof(uint32_t), C, cudaMemcpyDeviceToDevice, st));
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

}  // namespace sfc
