// k_noalloc.cu -- fullscan_query_batch_static: the exact full scan of
// fullscan_query_batch, for callers that must not allocate device memory.
//
// Every intermediate (mask filters, compaction counts, the dictionary, element
// offsets, weights, centre indices, per-query minima, per-tile minima) lives in
// one file-scope device array of kScratchBytes.  Every GPU that loads the library
// holds that array until the process exits.  All calls share it and it keeps the
// last call's contents; everything a call reads is written by the same call
// first.  Calls that overlap on the GPU (other streams, other host threads)
// race on the array and must be serialised by the caller.
#include <cmath>
#include <mutex>
#include <vector>

#include "internal.cuh"

namespace sfc {

namespace {

constexpr size_t kScratchBytes = (size_t)16 << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_scr_mu;
unsigned char* g_scr_ptr[128] = {};

// Device address of g_scratch on the current device, looked up once per device
// (the first call on a device performs this lookup).
int scratch_base(unsigned char** out) {
  int dev = 0;
  SFC_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 128) {
    set_error("device ordinal out of range");
    return SFC_EINVAL;
  }
  std::lock_guard<std::mutex> lk(g_scr_mu);
  if (!g_scr_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error(std::string("cudaGetSymbolAddress(g_scratch): ") + cudaGetErrorString(e));
      return SFC_ECUDA;
    }
    g_scr_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scr_ptr[dev];
  return SFC_OK;
}

inline size_t up256(size_t v) { return (v + 255) & ~(size_t)255; }

__global__ void k_static_tables(Geo g, int* eoff, float* w, int have_w) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < g.n; e += gridDim.x * blockDim.x)
    eoff[e] = (int)(patch_off(g, e / g.ch) * g.ch + e % g.ch);
  if (!have_w && blockIdx.x == 0)
    for (int c = threadIdx.x; c < g.ch; c += blockDim.x) w[c] = 1.0f;
}

}  // namespace

}  // namespace sfc

using namespace sfc;

extern "C" int fullscan_query_batch_static(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask,
                                           const sfc_grid* gp, const sfc_params* p, const int32_t* centres,
                                           int64_t Q, int64_t* pick, float* cost, void* stream) {
  set_error("");
  if (!p || Q < 0) {
    set_error("fullscan_query_batch_static: NULL params or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!grid || !dict_mask || !cur_mask || !centres || !pick || !cost) {
    set_error("fullscan_query_batch_static: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  Geo g;
  SFC_CHECK(make_geo(gp, p->K, &g));
  bool weighted = false;
  if (p->ch_weights)
    for (int c = 0; c < g.ch; ++c) {
      const float v = p->ch_weights[c];
      if (!(v > 0.0f) || !std::isfinite(v)) {
        set_error("channel weights must be positive and finite");
        return SFC_EINVAL;
      }
      weighted |= v != 1.0f;
    }
  if (p->precision != SFC_FP32 && p->precision != SFC_FP16) {
    set_error("fullscan_query_batch_static: precision must be SFC_FP32 or SFC_FP16");
    return SFC_EUNSUPPORTED;
  }
  if (p->cost != SFC_COST_L2 && p->cost != SFC_COST_L1) {
    set_error("cost must be SFC_COST_L2 or SFC_COST_L1");
    return SFC_EINVAL;
  }
  if (p->precision == SFC_FP16 && p->cost != SFC_COST_L2) {
    set_error("the tensor-core pre-score (SFC_FP16) is an L2 expansion; use SFC_FP32 with SFC_COST_L1");
    return SFC_EUNSUPPORTED;
  }
  // SFC_FP16 runs the FP32 scan here: the tensor-core form's picks and costs
  // are the FP32 scan's by construction, and its operands would not fit the
  // static array.
  const int cm = (weighted ? 1 : 0) | (p->cost == SFC_COST_L1 ? 2 : 0);
  // scratch layout (every piece 256-byte aligned), sized by the largest
  // possible dictionary (every valid centre)
  const int64_t npix = g.X * g.Y * g.Z;
  const int64_t nmax = (g.X - g.K + 1) * (g.Y - g.K + 1) * (g.ndim == 3 ? g.Z - g.K + 1 : 1);
  const int64_t ntiles_max = (nmax + 1023) / 1024;
  // Each factor is bounded by the array size before any product is formed, so
  // the offsets below cannot wrap around.
  if (npix > (int64_t)kScratchBytes || nmax > (int64_t)(kScratchBytes / 4) || Q > (int64_t)(kScratchBytes / 13) ||
      g.n > (int64_t)(kScratchBytes / 4)) {
    set_error("fullscan_query_batch_static: the grid or the batch is larger than the " +
              std::to_string(kScratchBytes) + "-byte static scratch allows (use fullscan_query_batch, or fewer "
              "queries per call)");
    return SFC_EINVAL;
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += up256(bytes);
    return o;
  };
  const size_t o_a = take(npix), o_b = take(npix), o_cnt = take(sizeof(uint32_t) * ((npix + 2047) / 2048));
  const size_t o_tot = take(sizeof(int64_t)), o_dict = take(sizeof(uint32_t) * nmax);
  const size_t o_eo = take(sizeof(int) * g.n), o_w = take(sizeof(float) * g.ch);
  const size_t o_lin = take(sizeof(int64_t) * Q), o_bad = take(Q), o_gmin = take(sizeof(unsigned int) * Q);
  const size_t o_tm = take(sizeof(float) * Q * ntiles_max);
  if (off > kScratchBytes) {
    set_error("fullscan_query_batch_static: this grid and batch need " + std::to_string(off) +
              " bytes of scratch; the static scratch holds " + std::to_string(kScratchBytes) +
              " (use fullscan_query_batch, or fewer queries per call)");
    return SFC_EINVAL;
  }
  unsigned char* base = nullptr;
  SFC_CHECK(scratch_base(&base));
  cudaStream_t st = (cudaStream_t)stream;
  int* eo = reinterpret_cast<int*>(base + o_eo);
  float* w = reinterpret_cast<float*>(base + o_w);
  if (p->ch_weights) SFC_TRY(cudaMemcpyAsync(w, p->ch_weights, sizeof(float) * g.ch, cudaMemcpyHostToDevice, st));
  count_launch();
  k_static_tables<<<(g.n + 255) / 256, 256, 0, st>>>(g, eo, w, p->ch_weights ? 1 : 0);
  SFC_TRY(cudaGetLastError());
  uint32_t* dict = reinterpret_cast<uint32_t*>(base + o_dict);
  int64_t N = 0;
  SFC_CHECK(dict_extract_into(dict_mask, g, st, base + o_a, base + o_b, reinterpret_cast<uint32_t*>(base + o_cnt),
                              reinterpret_cast<int64_t*>(base + o_tot), dict, &N));
  if (N <= 0) {
    set_error("the dictionary is empty (no fully known patch)");
    return SFC_EINVAL;
  }
  return fullscan_batch_into(g, grid, cur_mask, dict, N, eo, w, cm, centres, Q, pick, cost,
                             reinterpret_cast<int64_t*>(base + o_lin), base + o_bad,
                             reinterpret_cast<unsigned int*>(base + o_gmin), reinterpret_cast<float*>(base + o_tm),
                             st);
}
