// sfc_api.cu -- the extern "C" boundary of libsfc (declared in include/sfc.h):
// argument validation, index lifecycle and the orchestration of the kernels.
#include <algorithm>
#include <atomic>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

struct sfc_index {
  sfc::Index ix;
  int device;
};

struct sfc_multi {
  sfc::MultiQuery* mq;
};

namespace sfc {

namespace {
thread_local std::string g_err;
__device__ uint32_t g_status_word;
std::mutex g_mu;
uint32_t* g_status_ptr[128] = {};
}  // namespace

void set_error(const std::string& msg) { g_err = msg; }

namespace {
struct TraceAcc {
  bool on = false;
  double ms[SFC_TRACE_PHASES] = {};
  int64_t builds = 0;
  double eig_flops = 0.0;
  double eig_flops32 = 0.0;
  double tc_ms[SFC_TRACE_TC_PHASES] = {};
  int64_t tc_calls = 0;
  double tc_flops = 0.0;
  double proj_ms = 0.0, proj_flops = 0.0, proj_bytes = 0.0;  // BF16 tensor-core projections
  int64_t proj_calls = 0;
} g_trace;
std::mutex g_trace_mu;
// events of the tensor-core full scan in flight on this host thread
thread_local cudaEvent_t g_tc_ev[SFC_TRACE_TC_PHASES + 1] = {};
thread_local bool g_tc_active = false;
}  // namespace

void tc_trace_begin(cudaStream_t st) {
  {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    g_tc_active = g_trace.on;
  }
  if (!g_tc_active) return;
  for (auto& e : g_tc_ev)
    if (!e && cudaEventCreate(&e) != cudaSuccess) {
      cudaGetLastError();
      g_tc_active = false;
      return;
    }
  cudaEventRecord(g_tc_ev[0], st);
}

void tc_trace_mark(int k, cudaStream_t st) {
  if (g_tc_active) cudaEventRecord(g_tc_ev[k], st);
}

void tc_trace_end(double gemm_flops) {
  if (!g_tc_active) return;
  g_tc_active = false;
  float t[SFC_TRACE_TC_PHASES] = {};
  bool ok = cudaEventSynchronize(g_tc_ev[SFC_TRACE_TC_PHASES]) == cudaSuccess;
  for (int k = 0; k < SFC_TRACE_TC_PHASES && ok; ++k)
    ok = cudaEventElapsedTime(&t[k], g_tc_ev[k], g_tc_ev[k + 1]) == cudaSuccess;
  cudaGetLastError();
  if (!ok) return;
  std::lock_guard<std::mutex> lk(g_trace_mu);
  for (int k = 0; k < SFC_TRACE_TC_PHASES; ++k) g_trace.tc_ms[k] += t[k];
  g_trace.tc_calls += 1;
  g_trace.tc_flops += gemm_flops;
}

void trace_mark(Index& ix, int k, cudaStream_t st) {
  if (ix.traced && ix.ev[k]) cudaEventRecord(ix.ev[k], st);
}

// Fold a finished traced build into the accumulators (device idle).
static void trace_fold(Index& ix) {
  if (!ix.traced) return;
  float t[SFC_TRACE_PHASES] = {};
  bool ok = true;
  for (int k = 0; k < SFC_TRACE_PHASES && ok; ++k) ok = cudaEventElapsedTime(&t[k], ix.ev[k], ix.ev[k + 1]) == cudaSuccess;
  std::vector<int> it(2 * ix.C, 0);
  if (ok && ix.eig_iters)
    ok = cudaMemcpy(it.data(), ix.eig_iters, sizeof(int) * 2 * ix.C, cudaMemcpyDeviceToHost) == cudaSuccess;
  cudaGetLastError();
  if (ok) {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    for (int k = 0; k < SFC_TRACE_PHASES; ++k) g_trace.ms[k] += t[k];
    g_trace.builds += 1;
    const double s = ix.s, p = ix.p_block;
    // per product A Q: 2 s^2 p (FP64 or FP32); per orthonormalisation (Gram +
    // Q = Z R^-1, FP64): 4 s p^2
    for (int c = 0; c < ix.C; ++c) {
      const int i64 = it[c], i32 = it[ix.C + c];
      g_trace.eig_flops += i64 * 2.0 * s * s * p + std::ceil((double)(i64 + i32) / ix.eig_per_orth) * 4.0 * s * p * p;
      g_trace.eig_flops32 += i32 * 2.0 * s * s * p;
    }
  }
  if (ix.ev_proj[0] && ix.ev_proj[1]) {
    float pm = 0.0f;
    if (cudaEventElapsedTime(&pm, ix.ev_proj[0], ix.ev_proj[1]) == cudaSuccess) {
      std::lock_guard<std::mutex> lk(g_trace_mu);
      g_trace.proj_ms += pm;
      g_trace.proj_calls += 1;
      g_trace.proj_flops += ix.proj_flops;
      g_trace.proj_bytes += ix.proj_bytes;
    }
    cudaGetLastError();
  }
  for (auto& e : ix.ev)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  for (auto& e : ix.ev_proj)
    if (e) {
      cudaEventDestroy(e);
      e = nullptr;
    }
  ix.traced = false;
}

namespace {
std::atomic<uint64_t> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(int64_t n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

uint32_t* status_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_status_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status_word) != cudaSuccess) return nullptr;
    g_status_ptr[dev] = static_cast<uint32_t*>(p);
  }
  return g_status_ptr[dev];
}

namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pool[128] = {};
bool g_pool_tried[128] = {};
}  // namespace

namespace {
std::atomic<int64_t> g_fail_alloc{0};  // > 0: the g_fail_alloc-th next allocation fails (tests)
std::atomic<int64_t> g_alloc_count{0};
}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st) {
  if (g_fail_alloc.load() > 0 && g_fail_alloc.fetch_sub(1) == 1) {
    *p = nullptr;
    return cudaErrorMemoryAllocation;
  }
  g_alloc_count.fetch_add(1);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  cudaMemPool_t pool = nullptr;
  if (dev >= 0 && dev < 128) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pool_tried[dev]) {
      g_pool_tried[dev] = true;
      cudaMemPoolProps props = {};
      props.allocType = cudaMemAllocationTypePinned;
      props.location.type = cudaMemLocationTypeDevice;
      props.location.id = dev;
      if (cudaMemPoolCreate(&g_pool[dev], &props) == cudaSuccess) {
        uint64_t keep = ~0ull;
        cudaMemPoolSetAttribute(g_pool[dev], cudaMemPoolAttrReleaseThreshold, &keep);
      } else {
        g_pool[dev] = nullptr;
        cudaGetLastError();
      }
    }
    pool = g_pool[dev];
  }
  const cudaError_t e2 = pool ? cudaMallocFromPoolAsync(p, bytes, pool, st) : cudaMallocAsync(p, bytes, st);
  if (e2 != cudaSuccess) *p = nullptr;
  return e2;
}

namespace {
std::mutex g_aux_mu;
cudaStream_t g_aux[128][kAuxStreams] = {};
cudaStream_t g_aux_hi[128] = {};
}  // namespace

cudaStream_t aux_stream_hi() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return nullptr;
  std::lock_guard<std::mutex> lk(g_aux_mu);
  if (!g_aux_hi[dev]) {
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess ||
        cudaStreamCreateWithPriority(&g_aux_hi[dev], cudaStreamNonBlocking, greatest) != cudaSuccess) {
      g_aux_hi[dev] = nullptr;
      cudaGetLastError();
    }
  }
  return g_aux_hi[dev];
}

cudaStream_t aux_stream(int k) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128 || k < 0 || k >= kAuxStreams) return nullptr;
  std::lock_guard<std::mutex> lk(g_aux_mu);
  if (!g_aux[dev][k] && cudaStreamCreateWithFlags(&g_aux[dev][k], cudaStreamNonBlocking) != cudaSuccess) {
    g_aux[dev][k] = nullptr;
    cudaGetLastError();
  }
  return g_aux[dev][k];
}

int fill_loop(const Geo& g, float* grid, uint8_t* mask, int prio, int mode, const Index* ix, const uint32_t* dict,
              int64_t N, const int* eoff_all, const float* weights, int cm, int64_t max_steps, int64_t* log,
              int64_t* steps_done, cudaStream_t st);

// The device must be an sm_103 part (the library carries sm_103a code only) and
// the status word must be reachable.
int check_device() {
  int dev = 0;
  SFC_TRY(cudaGetDevice(&dev));
  int maj = 0, mnr = 0;
  SFC_TRY(cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, dev));
  SFC_TRY(cudaDeviceGetAttribute(&mnr, cudaDevAttrComputeCapabilityMinor, dev));
  if (maj != 10 || mnr != 3) {
    set_error("libsfc is built for sm_103a; device " + std::to_string(dev) + " is sm_" + std::to_string(maj) +
              std::to_string(mnr));
    return SFC_EUNSUPPORTED;
  }
  if (!status_word()) {
    set_error("cannot reach the library status word on this device");
    return SFC_ECUDA;
  }
  return SFC_OK;
}

int make_geo(const sfc_grid* gp, int K, Geo* out) {
  if (!gp) {
    set_error("grid geometry is NULL");
    return SFC_EINVAL;
  }
  if (gp->ndim != 2 && gp->ndim != 3) {
    set_error("ndim must be 2 or 3");
    return SFC_EINVAL;
  }
  if (gp->ch < 1 || gp->ch > 64) {
    set_error("ch must be 1..64");
    return SFC_EINVAL;
  }
  if (K < 3 || K > 15 || (K % 2) == 0) {
    set_error("K must be odd, 3..15");
    return SFC_EINVAL;
  }
  const int64_t Z = gp->ndim == 3 ? gp->ext[2] : 1;
  if (gp->ndim == 2 && gp->ext[2] != 1 && gp->ext[2] != 0) {
    set_error("a 2-D grid needs ext[2] == 1");
    return SFC_EINVAL;
  }
  if (gp->ext[0] < K || gp->ext[1] < K || Z < (gp->ndim == 3 ? K : 1)) {
    set_error("every grid extent must be >= K");
    return SFC_EINVAL;
  }
  const int64_t npix = gp->ext[0] * gp->ext[1] * Z;
  if (npix >= (int64_t)1 << 32) {
    set_error("grids must have fewer than 2^32 pixels");
    return SFC_EINVAL;
  }
  Geo g;
  g.ndim = gp->ndim;
  g.ch = gp->ch;
  g.K = K;
  g.r = K / 2;
  g.P = gp->ndim == 3 ? K * K * K : K * K;
  g.X = gp->ext[0];
  g.Y = gp->ext[1];
  g.Z = Z;
  g.n = g.P * g.ch;
  if (g.n > 4096) {
    set_error("patches with more than 4096 values are not supported");
    return SFC_EINVAL;
  }
  *out = g;
  return SFC_OK;
}

namespace {

// Subset rule (Fig. 2): anchors at the middles of the patch edges and at its
// corners (2-D: top, right, bottom, left middles, then TL, TR, BR, BL corners;
// 3-D: the 8 corners in raster order, then the face middles z-, z+, y-, y+, x-,
// x+), in doubled coordinates where pixel p is at 2p+1 and the patch spans
// [0, 2K]; the m pixels of smallest squared distance, ties to the lower raster
// index, listed in ascending order.
std::vector<int32_t> subsets_host(int ndim, int K, int C, int m) {
  const int P = ndim == 3 ? K * K * K : K * K;
  const int E = 2 * K, H = K;
  std::vector<std::array<int, 3>> an;
  if (ndim == 2) {
    an = {{H, 0, 0}, {E, H, 0}, {H, E, 0}, {0, H, 0}, {0, 0, 0}, {E, 0, 0}, {E, E, 0}, {0, E, 0}};
  } else {
    for (int z = 0; z < 2; ++z)
      for (int y = 0; y < 2; ++y)
        for (int x = 0; x < 2; ++x) an.push_back({x * E, y * E, z * E});
    an.push_back({H, H, 0});
    an.push_back({H, H, E});
    an.push_back({H, 0, H});
    an.push_back({H, E, H});
    an.push_back({0, H, H});
    an.push_back({E, H, H});
  }
  std::vector<int32_t> out((size_t)C * m);
  std::vector<std::pair<long long, int>> d(P);
  for (int c = 0; c < C; ++c) {
    for (int pp = 0; pp < P; ++pp) {
      const long long x = 2 * (pp % K) + 1 - an[c][0];
      const long long y = 2 * ((pp / K) % K) + 1 - an[c][1];
      const long long z = ndim == 3 ? 2 * (pp / (K * K)) + 1 - an[c][2] : 0;
      d[pp] = {x * x + y * y + z * z, pp};
    }
    std::sort(d.begin(), d.end());
    std::vector<int32_t> sel(m);
    for (int i = 0; i < m; ++i) sel[i] = d[i].second;
    std::sort(sel.begin(), sel.end());
    std::copy(sel.begin(), sel.end(), out.begin() + (size_t)c * m);
  }
  return out;
}

// *dst = a new device copy of count host values (nullptr on failure: nothing
// is left allocated)
template <typename T>
int upload(T** dst, const T* src, size_t count, cudaStream_t st) {
  *dst = nullptr;
  T* d = nullptr;
  SFC_TRY(pmalloc(&d, sizeof(T) * (count ? count : 1), st));
  if (count) {
    const cudaError_t e = cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      cudaFreeAsync(d, st);
      set_error(std::string("upload: ") + cudaGetErrorString(e));
      return SFC_ECUDA;
    }
  }
  *dst = d;
  return SFC_OK;
}

void free_index(Index& ix) {
  cudaDeviceSynchronize();
  trace_fold(ix);
  void* ptrs[] = {ix.dict,  ix.eoff_all, ix.sub_eoff, ix.sub_pix, ix.weights, ix.basis, ix.mean,      ix.evals,
                  ix.lo,    ix.scale,    ix.shifts,   ix.proj,    ix.keys,    ix.skeys, ix.sids,       ix.sqc,
                  ix.eig_iters, ix.pca_done};
  cudaDeviceSynchronize();
  for (void* p : ptrs)
    if (p) cudaFreeAsync(p, nullptr);
  cudaStreamSynchronize(nullptr);
}

std::vector<float> weights_of(const sfc_params* p, int ch) {
  std::vector<float> w(ch, 1.0f);
  if (p->ch_weights)
    for (int c = 0; c < ch; ++c) w[c] = p->ch_weights[c];
  return w;
}

int check_weights(const std::vector<float>& w) {
  for (float v : w)
    if (!(v > 0.0f) || !std::isfinite(v)) {
      set_error("channel weights must be positive and finite");
      return SFC_EINVAL;
    }
  return SFC_OK;
}

}  // namespace

int upload_patch_tables(const Geo& g, int** eoff_all, cudaStream_t st) {
  std::vector<int> eo(g.n);
  for (int e = 0; e < g.n; ++e) eo[e] = (int)(patch_off(g, e / g.ch) * g.ch + e % g.ch);
  return upload(eoff_all, eo.data(), eo.size(), st);
}

// ---------------------------------------------------------------------------
// index files: a fixed header, the parameters as int64 (and the subset
// fraction as a double), then every array as (byte count, bytes); host byte
// order (little-endian on every supported machine)
// ---------------------------------------------------------------------------
namespace {
constexpr char kIndexMagic[8] = {'S', 'F', 'C', 'I', 'D', 'X', 'v', '1'};

struct FileOut {
  FILE* f;
  bool ok = true;
  void raw(const void* p, size_t n) { ok = ok && std::fwrite(p, 1, n, f) == n; }
  void i64(int64_t v) { raw(&v, sizeof v); }
};
struct FileIn {
  FILE* f;
  bool ok = true;
  void raw(void* p, size_t n) { ok = ok && std::fread(p, 1, n, f) == n; }
  int64_t i64() {
    int64_t v = 0;
    raw(&v, sizeof v);
    return v;
  }
};

template <class T>
void host_out(FileOut& o, const T* h, size_t count) {
  o.i64((int64_t)(sizeof(T) * count));
  o.raw(h, sizeof(T) * count);
}
template <class T>
int dev_out(FileOut& o, const T* d, size_t count) {
  std::vector<T> h(count);
  if (count) SFC_TRY(cudaMemcpy(h.data(), d, sizeof(T) * count, cudaMemcpyDeviceToHost));
  host_out(o, h.data(), count);
  return SFC_OK;
}
template <class T>
bool host_in(FileIn& in, std::vector<T>& h, size_t count) {
  if (in.i64() != (int64_t)(sizeof(T) * count)) return false;
  h.resize(count);
  in.raw(h.data(), sizeof(T) * count);
  return in.ok;
}
template <class T>
int dev_in(FileIn& in, T** d, size_t count, cudaStream_t st) {
  std::vector<T> h;
  if (!host_in(in, h, count)) {
    set_error("index file: truncated or inconsistent array");
    return SFC_EINVAL;
  }
  SFC_CHECK(upload(d, h.data(), count, st));
  return SFC_OK;
}
}  // namespace

// Projection, keys and sort of every curve, pipelined over groups of curves:
// the groups' projections and keys run in order on a high-priority library
// stream, and each group's sort on one of the library's default-priority
// streams as soon as its keys exist, so the sorts (latency-bound) fill the SMs
// around the projections (issue-bound) without holding them up.  With the
// sample sort (ss) there is one group: the sort follows the projections.  Phase 5 of
// the trace is marked once every group's keys exist, phase 6 (by the caller)
// once every sort is done.  st waits for all of it, also on an error, so
// nothing the caller frees next is still in use.
int project_sort_pipelined(Index& ix, const float* grid, float* proj, uint64_t* keys, uint32_t* lohi, int* ovf,
                           bool ss, cudaStream_t st) {
  const int C = ix.C;
  const int64_t N = ix.N;
  const int key_bits = std::min(64, ix.D * ix.bp);
  // the sort of curves [c0, c0 + nc): the sample sort (ss) or the LSD sort
  auto sort_group = [&](int c0, int nc, cudaStream_t s, void* ws) -> int {
    return ss ? sample_sort_pairs(keys + (size_t)c0 * N, ix.skeys + (size_t)c0 * N, ix.sids + (size_t)c0 * N, N,
                                  nc, ovf + c0, s, ws)
              : radix_sort_pairs(keys + (size_t)c0 * N, ix.skeys + (size_t)c0 * N, ix.sids + (size_t)c0 * N, N, nc,
                                 key_bits, s, ws);
  };
  cudaStream_t hi = aux_stream_hi();
  cudaStream_t lo[kAuxStreams];
  int nlo = 0;
  while (nlo < kAuxStreams && (lo[nlo] = aux_stream(nlo)) != nullptr) ++nlo;
  if (!hi || nlo == 0) {  // no library streams: everything in order on st
    if (ix.bf16)
      SFC_CHECK(project_bf16(ix, grid, proj, lohi, st));
    else
      SFC_CHECK(project_curves(ix, grid, proj, lohi, 0, C, st));
    SFC_CHECK(key_curves(ix, proj, keys, 0, C, st));
    trace_mark(ix, 5, st);
    return sort_group(0, C, st, nullptr);
  }
  // groups of curves: the sample sort gains more from sorting every curve in
  // one set of launches than from overlapping smaller sorts with the
  // projections (1,024² workload: step 3.52 ms with one group, 3.55 with two,
  // 3.57 with four); the LSD sort of larger dictionaries overlaps, in four
  constexpr int kGroups = 4;
  int G = C < kGroups ? C : kGroups;
  if (ss) G = 1;
  const int per = (C + G - 1) / G;
  G = (C + per - 1) / per;
  // every group's sort scratch is taken on st before the fork and returned
  // after the join, so no memory moves between the streams' pool queues
  const size_t ws_bytes = ss ? sample_sort_scratch_bytes(N, per) : radix_sort_scratch_bytes(N, per, key_bits);
  unsigned char* ws = nullptr;
  SFC_TRY(pmalloc(&ws, ws_bytes * G, st));
  cudaEvent_t ev_fork = nullptr, ev_hi = nullptr, ev_keys[kGroups] = {}, ev_done[kGroups] = {};
  int rc = SFC_OK;
  auto mk = [&](cudaEvent_t* e) {
    if (rc == SFC_OK && cudaEventCreateWithFlags(e, cudaEventDisableTiming) != cudaSuccess) {
      set_error("cudaEventCreateWithFlags failed");
      rc = SFC_ECUDA;
    }
  };
  mk(&ev_fork);
  mk(&ev_hi);
  for (int g = 0; g < G; ++g) {
    mk(&ev_keys[g]);
    mk(&ev_done[g]);
  }
  bool forked = false;
  if (rc == SFC_OK && cudaEventRecord(ev_fork, st) == cudaSuccess && cudaStreamWaitEvent(hi, ev_fork, 0) == cudaSuccess)
    forked = true;
  else if (rc == SFC_OK)
    rc = SFC_ECUDA;
  int sorted = 0;  // groups whose sort stream recorded ev_done
  for (int g = 0; g < G && rc == SFC_OK; ++g) {
    const int c0 = g * per, nc = std::min(per, C - c0);
    // (BF16 tier: one tensor-core launch projects every curve, before the first group's keys)
    if (!ix.bf16)
      rc = project_curves(ix, grid, proj, lohi, c0, nc, hi);
    else if (g == 0)
      rc = project_bf16(ix, grid, proj, lohi, hi);
    if (rc == SFC_OK) rc = key_curves(ix, proj, keys, c0, nc, hi);
    if (rc == SFC_OK && cudaEventRecord(ev_keys[g], hi) != cudaSuccess) rc = SFC_ECUDA;
    if (rc != SFC_OK) break;
    cudaStream_t s = lo[g % nlo];
    if (cudaStreamWaitEvent(s, ev_keys[g], 0) != cudaSuccess) {
      rc = SFC_ECUDA;
      break;
    }
    rc = sort_group(c0, nc, s, ws + ws_bytes * g);
    if (cudaEventRecord(ev_done[g], s) == cudaSuccess)
      sorted = g + 1;
    else if (rc == SFC_OK)
      rc = SFC_ECUDA;
  }
  // join: the high-priority stream's end, then every sort
  if (forked && cudaEventRecord(ev_hi, hi) == cudaSuccess) cudaStreamWaitEvent(st, ev_hi, 0);
  if (rc == SFC_OK) trace_mark(ix, 5, st);
  for (int g = 0; g < sorted; ++g) cudaStreamWaitEvent(st, ev_done[g], 0);
  cudaFreeAsync(ws, st);
  for (cudaEvent_t e : {ev_fork, ev_hi})
    if (e) cudaEventDestroy(e);
  for (int g = 0; g < G; ++g)
    for (cudaEvent_t e : {ev_keys[g], ev_done[g]})
      if (e) cudaEventDestroy(e);
  if (rc == SFC_ECUDA && sfc_last_error()[0] == 0)
    set_error(std::string("pipelined build: ") + cudaGetErrorString(cudaGetLastError()));
  return rc;
}

// Build every array of an index (shared by sfc_index_build and inpaint_run).
int build_index(const float* grid, const uint8_t* dict_mask, const sfc_grid* gp, const sfc_params* p,
                cudaStream_t st, Index& ix) {
  if (!grid || !dict_mask || !p) {
    set_error("sfc_index_build: NULL argument");
    return SFC_EINVAL;
  }
  SFC_CHECK(make_geo(gp, p->K, &ix.g));
  const Geo& g = ix.g;
  const int maxC = g.ndim == 2 ? 8 : 14;
  if (p->curves < 1 || p->curves > maxC) {
    set_error("curves must be 1.." + std::to_string(maxC));
    return SFC_EINVAL;
  }
  if (p->dims < 1 || p->dims > 16 || p->bits < 1 || p->bits > 21 || p->window < 1 ||
      !(p->subset_frac > 0.0f && p->subset_frac <= 1.0f) || (p->select != SFC_SELECT_ALL && p->select != SFC_SELECT_BEST) ||
      p->knn < 0 || p->knn > 128 || (p->curve != SFC_CURVE_MORTON && p->curve != SFC_CURVE_HILBERT)) {
    set_error("parameter out of range (dims 1..16, bits 1..21, window >= 1, subset_frac in (0, 1], select, "
              "knn 0..128, curve)");
    return SFC_EINVAL;
  }
  if (p->cost != SFC_COST_L2 && p->cost != SFC_COST_L1) {
    set_error("cost must be SFC_COST_L2 or SFC_COST_L1");
    return SFC_EINVAL;
  }
  if (p->knn > 0 && p->curve != SFC_CURVE_MORTON) {
    set_error("the k-NN search (knn > 0) runs on the z-curve (SFC_CURVE_MORTON) only");
    return SFC_EUNSUPPORTED;
  }
  if (p->precision != SFC_FP32 && p->precision != SFC_BF16) {
    set_error("the index path takes SFC_FP32 (exact FMA-chain projections) or SFC_BF16 (tensor-core projections, "
              "stored in BF16)");
    return SFC_EUNSUPPORTED;
  }
  ix.bf16 = p->precision == SFC_BF16;
  ix.C = p->curves;
  ix.D = p->dims;
  ix.bits = p->bits;
  ix.W = p->window;
  ix.knn = p->knn;
  ix.curve = p->curve;
  ix.l1 = p->cost == SFC_COST_L1;
  ix.select = p->select;
  ix.frac = p->subset_frac;
  ix.pca_sample = p->pca_sample;
  ix.keep = p->keep_intermediates != 0;
  int m = (int)std::floor((double)p->subset_frac * g.P + 0.5);
  m = std::max(1, std::min(m, g.P));
  ix.m = m;
  ix.s = m * g.ch;
  if (ix.D > ix.s) {
    set_error("dims must not exceed the subset length m * ch");
    return SFC_EINVAL;
  }
  std::vector<int32_t> sh((size_t)ix.C * ix.D, 0);
  ix.bp = ix.bits;
  if (p->shifts) {
    for (size_t i = 0; i < sh.size(); ++i) {
      sh[i] = p->shifts[i];
      if (sh[i] < 0 || sh[i] >= (1 << ix.bits)) {
        set_error("shifts must lie in [0, 2^bits)");
        return SFC_EINVAL;
      }
      if (sh[i] != 0) ix.bp = ix.bits + 1;
    }
  }
  ix.weights_h = weights_of(p, g.ch);
  SFC_CHECK(check_weights(ix.weights_h));
  if (p->basis && !p->mean) {
    set_error("a given basis needs its mean");
    return SFC_EINVAL;
  }
  ix.subset_h = subsets_host(g.ndim, g.K, ix.C, m);
  std::vector<int32_t> sub_eoff((size_t)ix.C * ix.s);
  for (int c = 0; c < ix.C; ++c)
    for (int i = 0; i < ix.s; ++i)
      sub_eoff[(size_t)c * ix.s + i] =
          (int32_t)(patch_off(g, ix.subset_h[(size_t)c * m + i / g.ch]) * g.ch + i % g.ch);
  SFC_CHECK(upload_patch_tables(g, &ix.eoff_all, st));
  SFC_CHECK(upload(&ix.sub_pix, ix.subset_h.data(), ix.subset_h.size(), st));
  SFC_CHECK(upload(&ix.sub_eoff, sub_eoff.data(), sub_eoff.size(), st));
  SFC_CHECK(upload(&ix.weights, ix.weights_h.data(), ix.weights_h.size(), st));
  SFC_CHECK(upload(&ix.shifts, sh.data(), sh.size(), st));
  {
    std::lock_guard<std::mutex> lk(g_trace_mu);
    ix.traced = g_trace.on;
  }
  if (ix.traced) {
    for (auto& e : ix.ev) SFC_TRY(cudaEventCreate(&e));
    for (auto& e : ix.ev_proj) SFC_TRY(cudaEventCreate(&e));
    trace_mark(ix, 0, st);
  }
  SFC_TRY(pmalloc(&ix.eig_iters, sizeof(int) * 2 * ix.C, st));
  SFC_TRY(cudaMemsetAsync(ix.eig_iters, 0, sizeof(int) * 2 * ix.C, st));
  SFC_CHECK(dict_extract(dict_mask, g, st, &ix.dict, &ix.N));
  trace_mark(ix, 1, st);
  if (ix.N <= 0) {
    set_error("the dictionary is empty (no fully known patch)");
    return SFC_EINVAL;
  }
  const int C = ix.C, D = ix.D, s = ix.s;
  const int64_t N = ix.N;
  SFC_TRY(pmalloc(&ix.basis, sizeof(float) * C * s * D, st));
  SFC_TRY(pmalloc(&ix.mean, sizeof(float) * C * s, st));
  SFC_TRY(pmalloc(&ix.evals, sizeof(double) * C * s, st));
  SFC_TRY(pmalloc(&ix.lo, sizeof(float) * C * D, st));
  SFC_TRY(pmalloc(&ix.scale, sizeof(float) * C * D, st));
  SFC_TRY(pmalloc(&ix.skeys, sizeof(uint64_t) * C * N, st));
  SFC_TRY(pmalloc(&ix.sids, sizeof(uint32_t) * C * N, st));
  if (p->basis) {
    SFC_TRY(cudaMemcpyAsync(ix.basis, p->basis, sizeof(float) * C * s * D, cudaMemcpyHostToDevice, st));
    SFC_TRY(cudaMemcpyAsync(ix.mean, p->mean, sizeof(float) * C * s, cudaMemcpyHostToDevice, st));
    SFC_TRY(cudaMemsetAsync(ix.evals, 0xff, sizeof(double) * C * s, st));  // NaN
    trace_mark(ix, 2, st);
    trace_mark(ix, 3, st);
  } else {
    SFC_CHECK(pca_build(ix, grid, st));
  }
  trace_mark(ix, 4, st);
  float* proj = nullptr;
  uint64_t* keys = nullptr;
  uint32_t* lohi = nullptr;
  int* ovf = nullptr;
  std::vector<int> done(C, 1);
  {
    Scratch scr(st);
    SFC_TRY(scr.alloc(&proj, (ix.bf16 ? 2 : sizeof(float)) * C * N * D));
    SFC_TRY(scr.alloc(&keys, sizeof(uint64_t) * C * N));
    SFC_TRY(scr.alloc(&lohi, sizeof(uint32_t) * 2 * C * D));
    SFC_TRY(scr.alloc(&ovf, sizeof(int) * C));
    SFC_TRY(cudaMemsetAsync(ovf, 0, sizeof(int) * C, st));
    const bool ss = sample_sort_fits(N);
    SFC_CHECK(project_sort_pipelined(ix, grid, proj, keys, lohi, ovf, ss, st));
    // one wait for the flags: the eigen-solves' convergence and the indices the
    // sample sort left to the LSD sort (sorted now, from the keys)
    if (ss || ix.pca_done) {
      std::vector<int> ov(C, 0);
      if (ss) SFC_TRY(cudaMemcpyAsync(ov.data(), ovf, sizeof(int) * C, cudaMemcpyDeviceToHost, st));
      if (ix.pca_done) SFC_TRY(cudaMemcpyAsync(done.data(), ix.pca_done, sizeof(int) * C, cudaMemcpyDeviceToHost, st));
      SFC_TRY(cudaStreamSynchronize(st));
      const int key_bits = std::min(64, ix.D * ix.bp);
      for (int c = 0; c < C; ++c)
        if (ov[c])
          SFC_CHECK(radix_sort_pairs(keys + (size_t)c * N, ix.skeys + (size_t)c * N, ix.sids + (size_t)c * N, N, 1,
                                     key_bits, st));
    }
    if (ix.knn > 0) SFC_CHECK(sorted_coords(ix, proj, st));
    trace_mark(ix, 6, st);
    if (ix.keep) {
      scr.keep(proj);
      scr.keep(keys);
      ix.proj = proj;
      ix.keys = keys;
    }
  }
  SFC_TRY(cudaGetLastError());
  if (ix.pca_done) {
    // every eigen-solve must have converged (flags read above)
    for (int c = 0; c < C; ++c)
      if (!done[c]) {
        set_error("the PCA eigen-solve of index " + std::to_string(c) + " (subset length " + std::to_string(s) +
                  ", D = " + std::to_string(D) + ") did not converge: the covariance spectrum is too flat "
                  "beyond the D-th eigenvalue for the iteration; give a basis, or fewer dimensions");
        return SFC_ENOCONV;
      }
  }
  return SFC_OK;
}

}  // namespace sfc

using namespace sfc;

extern "C" {

void sfc_params_default(sfc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->K = 9;
  p->curves = 8;
  p->dims = 10;
  p->bits = 8;
  p->window = 80;
  p->subset_frac = 0.6f;
  p->select = SFC_SELECT_ALL;
  p->precision = SFC_FP32;
  p->pca_sample = 16384;
  p->priority = SFC_PRIO_CONFIDENCE;
}

const char* sfc_last_error(void) { return g_err.c_str(); }

uint64_t sfc_launch_count(void) { return g_launches.load(); }

int sfc_trace(int on) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  g_trace = TraceAcc();
  g_trace.on = on != 0;
  return SFC_OK;
}

int sfc_trace_tc_read(double* ms, int64_t* calls, double* gemm_flops) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (ms)
    for (int k = 0; k < SFC_TRACE_TC_PHASES; ++k) ms[k] = g_trace.tc_ms[k];
  if (calls) *calls = g_trace.tc_calls;
  if (gemm_flops) *gemm_flops = g_trace.tc_flops;
  return SFC_OK;
}

int sfc_trace_eig_read(double* fp64_flops, double* fp32_flops) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (fp64_flops) *fp64_flops = g_trace.eig_flops;
  if (fp32_flops) *fp32_flops = g_trace.eig_flops32;
  return SFC_OK;
}

int sfc_trace_proj_read(double* ms, int64_t* calls, double* flops, double* bytes) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (ms) *ms = g_trace.proj_ms;
  if (calls) *calls = g_trace.proj_calls;
  if (flops) *flops = g_trace.proj_flops;
  if (bytes) *bytes = g_trace.proj_bytes;
  return SFC_OK;
}

int sfc_trace_read(double* ms, int64_t* builds, double* eig_flops) {
  std::lock_guard<std::mutex> lk(g_trace_mu);
  if (ms)
    for (int k = 0; k < SFC_TRACE_PHASES; ++k) ms[k] = g_trace.ms[k];
  if (builds) *builds = g_trace.builds;
  if (eig_flops) *eig_flops = g_trace.eig_flops;
  return SFC_OK;
}

int sfc_index_build(const float* grid, const uint8_t* dict_mask, const sfc_grid* g, const sfc_params* p,
                    void* stream, sfc_index** out) {
  g_err.clear();
  if (!out) {
    set_error("sfc_index_build: out is NULL");
    return SFC_EINVAL;
  }
  *out = nullptr;
  SFC_CHECK(check_device());
  auto* h = new sfc_index();
  cudaGetDevice(&h->device);
  int rc = build_index(grid, dict_mask, g, p, (cudaStream_t)stream, h->ix);
  if (rc != SFC_OK) {
    free_index(h->ix);
    delete h;
    return rc;
  }
  *out = h;
  return SFC_OK;
}

int sfc_index_destroy(sfc_index* ix) {
  if (!ix) return SFC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(ix->device);
  free_index(ix->ix);
  cudaSetDevice(prev);
  delete ix;
  return SFC_OK;
}

int sfc_index_info(const sfc_index* ix, int64_t* N, int32_t* m, int32_t* s) {
  if (!ix) {
    set_error("sfc_index_info: NULL index");
    return SFC_EINVAL;
  }
  if (N) *N = ix->ix.N;
  if (m) *m = ix->ix.m;
  if (s) *s = ix->ix.s;
  return SFC_OK;
}

int sfc_index_export(const sfc_index* h, int64_t* dict, int32_t* subsets, float* basis, float* mean, double* evals,
                     float* lo, float* scale, float* proj, uint64_t* keys, uint64_t* skeys, uint32_t* sids) {
  g_err.clear();
  if (!h) {
    set_error("sfc_index_export: NULL index");
    return SFC_EINVAL;
  }
  const Index& ix = h->ix;
  if ((proj || keys) && !ix.keep) {
    set_error("projections/unsorted keys are only kept with keep_intermediates = 1");
    return SFC_EINVAL;
  }
  SFC_TRY(cudaDeviceSynchronize());
  const size_t C = ix.C, D = ix.D, s = ix.s, N = ix.N;
  if (dict) {
    std::vector<uint32_t> d(N);
    SFC_TRY(cudaMemcpy(d.data(), ix.dict, sizeof(uint32_t) * N, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < N; ++i) dict[i] = d[i];
  }
  if (subsets) std::memcpy(subsets, ix.subset_h.data(), sizeof(int32_t) * ix.subset_h.size());
  if (basis) SFC_TRY(cudaMemcpy(basis, ix.basis, sizeof(float) * C * s * D, cudaMemcpyDeviceToHost));
  if (mean) SFC_TRY(cudaMemcpy(mean, ix.mean, sizeof(float) * C * s, cudaMemcpyDeviceToHost));
  if (evals) SFC_TRY(cudaMemcpy(evals, ix.evals, sizeof(double) * C * s, cudaMemcpyDeviceToHost));
  if (lo) SFC_TRY(cudaMemcpy(lo, ix.lo, sizeof(float) * C * D, cudaMemcpyDeviceToHost));
  if (scale) SFC_TRY(cudaMemcpy(scale, ix.scale, sizeof(float) * C * D, cudaMemcpyDeviceToHost));
  if (proj && !ix.bf16) SFC_TRY(cudaMemcpy(proj, ix.proj, sizeof(float) * C * N * D, cudaMemcpyDeviceToHost));
  if (proj && ix.bf16) {  // stored in BF16: widened exactly to FP32
    std::vector<uint16_t> h((size_t)C * N * D);
    SFC_TRY(cudaMemcpy(h.data(), ix.proj, sizeof(uint16_t) * h.size(), cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < h.size(); ++i) {
      const uint32_t u = (uint32_t)h[i] << 16;
      std::memcpy(&proj[i], &u, sizeof(float));
    }
  }
  if (keys) SFC_TRY(cudaMemcpy(keys, ix.keys, sizeof(uint64_t) * C * N, cudaMemcpyDeviceToHost));
  if (skeys) SFC_TRY(cudaMemcpy(skeys, ix.skeys, sizeof(uint64_t) * C * N, cudaMemcpyDeviceToHost));
  if (sids) SFC_TRY(cudaMemcpy(sids, ix.sids, sizeof(uint32_t) * C * N, cudaMemcpyDeviceToHost));
  return SFC_OK;
}

int sfc_multi_create(const sfc_index* const* ix, const float* const* grids, const uint8_t* const* masks, int32_t n,
                     void* stream, sfc_multi** out) {
  g_err.clear();
  if (!ix || !grids || !masks || !out || n < 1) {
    set_error("sfc_multi_create: NULL argument or n < 1");
    return SFC_EINVAL;
  }
  *out = nullptr;
  SFC_CHECK(check_device());
  std::vector<const Index*> v(n);
  for (int i = 0; i < n; ++i) {
    if (!ix[i]) {
      set_error("sfc_multi_create: NULL index");
      return SFC_EINVAL;
    }
    v[i] = &ix[i]->ix;
  }
  MultiQuery* mq = nullptr;
  SFC_CHECK(multi_query_create(v.data(), grids, masks, n, (cudaStream_t)stream, &mq));
  *out = new sfc_multi{mq};
  return SFC_OK;
}

int sfc_multi_query(const sfc_multi* mu, const int32_t* image, const int32_t* centres, int64_t Q, int64_t* pick,
                    float* cost, void* stream) {
  g_err.clear();
  if (!mu || Q < 0) {
    set_error("sfc_multi_query: NULL object or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!image || !centres || !pick || !cost) {
    set_error("sfc_multi_query: NULL pointer");
    return SFC_EINVAL;
  }
  return multi_query_run(mu->mq, image, centres, Q, pick, cost, (cudaStream_t)stream);
}

int sfc_multi_destroy(sfc_multi* mu) {
  if (!mu) return SFC_OK;
  multi_query_destroy(mu->mq);
  delete mu;
  return SFC_OK;
}

int sfc_index_params(const sfc_index* h, sfc_params* p, sfc_grid* g) {
  g_err.clear();
  if (!h) {
    set_error("sfc_index_params: NULL index");
    return SFC_EINVAL;
  }
  const Index& ix = h->ix;
  if (p) {
    sfc_params_default(p);
    p->K = ix.g.K;
    p->curves = ix.C;
    p->dims = ix.D;
    p->bits = ix.bits;
    p->window = ix.W;
    p->subset_frac = ix.frac;
    p->select = ix.select;
    p->pca_sample = ix.pca_sample;
    p->knn = ix.knn;
    p->curve = ix.curve;
    p->cost = ix.l1 ? SFC_COST_L1 : SFC_COST_L2;
    p->precision = ix.bf16 ? SFC_BF16 : SFC_FP32;
  }
  if (g) {
    g->ndim = ix.g.ndim;
    g->ch = ix.g.ch;
    g->ext[0] = ix.g.X;
    g->ext[1] = ix.g.Y;
    g->ext[2] = ix.g.Z;
  }
  return SFC_OK;
}

int sfc_index_save(const sfc_index* h, const char* path) {
  g_err.clear();
  if (!h || !path) {
    set_error("sfc_index_save: NULL index or path");
    return SFC_EINVAL;
  }
  const Index& ix = h->ix;
  SFC_TRY(cudaDeviceSynchronize());
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("sfc_index_save: cannot open ") + path);
    return SFC_EINVAL;
  }
  FileOut o{f};
  o.raw(kIndexMagic, sizeof kIndexMagic);
  const int64_t head[] = {ix.g.ndim, ix.g.ch,  ix.g.K,  ix.g.X, ix.g.Y, ix.g.Z,       ix.C,         ix.D,
                          ix.bits,   ix.bp,    ix.W,    ix.select, ix.m, ix.s,        ix.N,         ix.knn,
                          ix.curve,  ix.l1 ? 1 : 0, ix.p_block, ix.eig_per_orth, ix.pca_sample,
                          ix.bf16 ? SFC_BF16 : SFC_FP32};
  o.i64((int64_t)(sizeof head / sizeof head[0]));
  o.raw(head, sizeof head);
  const double frac = ix.frac;
  o.raw(&frac, sizeof frac);
  const int64_t C = ix.C, N = ix.N, D = ix.D, s = ix.s, m = ix.m;
  host_out(o, ix.subset_h.data(), ix.subset_h.size());
  host_out(o, ix.weights_h.data(), ix.weights_h.size());
  int rc = SFC_OK;
  if (rc == SFC_OK) rc = dev_out(o, ix.dict, (size_t)N);
  if (rc == SFC_OK) rc = dev_out(o, ix.eoff_all, (size_t)ix.g.n);
  if (rc == SFC_OK) rc = dev_out(o, ix.sub_eoff, (size_t)(C * s));
  if (rc == SFC_OK) rc = dev_out(o, ix.sub_pix, (size_t)(C * m));
  if (rc == SFC_OK) rc = dev_out(o, ix.weights, (size_t)ix.g.ch);
  if (rc == SFC_OK) rc = dev_out(o, ix.basis, (size_t)(C * s * D));
  if (rc == SFC_OK) rc = dev_out(o, ix.mean, (size_t)(C * s));
  if (rc == SFC_OK) rc = dev_out(o, ix.evals, (size_t)(C * s));
  if (rc == SFC_OK) rc = dev_out(o, ix.lo, (size_t)(C * D));
  if (rc == SFC_OK) rc = dev_out(o, ix.scale, (size_t)(C * D));
  if (rc == SFC_OK) rc = dev_out(o, ix.shifts, (size_t)(C * D));
  if (rc == SFC_OK) rc = dev_out(o, ix.skeys, (size_t)(C * N));
  if (rc == SFC_OK) rc = dev_out(o, ix.sids, (size_t)(C * N));
  if (rc == SFC_OK && ix.knn > 0) rc = dev_out(o, ix.sqc, (size_t)(C * N * D));
  const bool ok = o.ok && std::fclose(f) == 0;
  if (rc != SFC_OK) return rc;
  if (!ok) {
    set_error(std::string("sfc_index_save: write to ") + path + " failed");
    return SFC_EINVAL;
  }
  return SFC_OK;
}

int sfc_index_load(const char* path, void* stream, sfc_index** out) {
  g_err.clear();
  if (!path || !out) {
    set_error("sfc_index_load: NULL path or out");
    return SFC_EINVAL;
  }
  *out = nullptr;
  SFC_CHECK(check_device());
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("sfc_index_load: cannot open ") + path);
    return SFC_EINVAL;
  }
  FileIn in{f};
  char magic[8] = {};
  in.raw(magic, sizeof magic);
  const int64_t nhead = in.i64();
  int64_t head[22] = {};  // 21 entries in files written before the precision was recorded (FP32)
  if (!in.ok || std::memcmp(magic, kIndexMagic, sizeof magic) != 0 || (nhead != 21 && nhead != 22)) {
    std::fclose(f);
    set_error("sfc_index_load: not an index file of this library version");
    return SFC_EINVAL;
  }
  in.raw(head, sizeof(int64_t) * nhead);
  double frac = 0.0;
  in.raw(&frac, sizeof frac);
  cudaStream_t st = (cudaStream_t)stream;
  auto* h = new sfc_index();
  cudaGetDevice(&h->device);
  Index& ix = h->ix;
  sfc_grid gp;
  gp.ndim = (int32_t)head[0];
  gp.ch = (int32_t)head[1];
  gp.ext[0] = head[3];
  gp.ext[1] = head[4];
  gp.ext[2] = head[5];
  int rc = in.ok ? make_geo(&gp, (int)head[2], &ix.g) : SFC_EINVAL;
  ix.C = (int)head[6];
  ix.D = (int)head[7];
  ix.bits = (int)head[8];
  ix.bp = (int)head[9];
  ix.W = (int)head[10];
  ix.select = (int)head[11];
  ix.m = (int)head[12];
  ix.s = (int)head[13];
  ix.N = head[14];
  ix.knn = (int)head[15];
  ix.curve = (int)head[16];
  ix.l1 = head[17] != 0;
  ix.p_block = (int)head[18];
  ix.eig_per_orth = (int)head[19];
  ix.pca_sample = head[20];
  ix.bf16 = nhead > 21 && head[21] == SFC_BF16;
  ix.frac = (float)frac;
  ix.keep = false;
  const int64_t C = ix.C, N = ix.N, D = ix.D, s = ix.s, m = ix.m;
  if (rc == SFC_OK && (C < 1 || C > 14 || D < 1 || D > 16 || N < 1 || s != m * ix.g.ch || m < 1 || m > ix.g.P ||
                       ix.bits < 1 || ix.bits > 21 || ix.knn < 0 || ix.knn > 128)) {
    set_error("sfc_index_load: inconsistent index parameters");
    rc = SFC_EINVAL;
  }
  if (rc == SFC_OK && !(host_in(in, ix.subset_h, (size_t)(C * m)) && host_in(in, ix.weights_h, (size_t)ix.g.ch))) {
    set_error("sfc_index_load: truncated file");
    rc = SFC_EINVAL;
  }
  if (rc == SFC_OK) rc = dev_in(in, &ix.dict, (size_t)N, st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.eoff_all, (size_t)ix.g.n, st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.sub_eoff, (size_t)(C * s), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.sub_pix, (size_t)(C * m), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.weights, (size_t)ix.g.ch, st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.basis, (size_t)(C * s * D), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.mean, (size_t)(C * s), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.evals, (size_t)(C * s), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.lo, (size_t)(C * D), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.scale, (size_t)(C * D), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.shifts, (size_t)(C * D), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.skeys, (size_t)(C * N), st);
  if (rc == SFC_OK) rc = dev_in(in, &ix.sids, (size_t)(C * N), st);
  if (rc == SFC_OK && ix.knn > 0) rc = dev_in(in, &ix.sqc, (size_t)(C * N * D), st);
  if (rc == SFC_OK && (pmalloc(&ix.eig_iters, sizeof(int) * 2 * C, st) != cudaSuccess ||
                       cudaMemsetAsync(ix.eig_iters, 0, sizeof(int) * 2 * C, st) != cudaSuccess)) {
    cudaGetLastError();
    set_error("sfc_index_load: out of device memory");
    rc = SFC_ENOMEM;
  }
  std::fclose(f);
  if (rc != SFC_OK) {
    free_index(ix);
    delete h;
    return rc;
  }
  SFC_TRY(cudaStreamSynchronize(st));
  *out = h;
  return SFC_OK;
}

int sfc_query_batch_dict(const sfc_index* h, const float* dict_grid, const float* grid, const uint8_t* cur_mask,
                         const sfc_grid* gp, const int32_t* centres, int64_t Q, int64_t* pick, float* cost,
                         void* stream) {
  g_err.clear();
  if (!h || Q < 0) {
    set_error("sfc_query_batch_dict: NULL index or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!dict_grid || !grid || !cur_mask || !centres || !pick || !cost || !gp) {
    set_error("sfc_query_batch_dict: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  const Index& ix = h->ix;
  if (gp->ndim != ix.g.ndim || gp->ch != ix.g.ch) {
    set_error("sfc_query_batch_dict: the target grid needs the index's dimension and channel count");
    return SFC_EINVAL;
  }
  TargetGrid tg;
  SFC_CHECK(make_geo(gp, ix.g.K, &tg.g));
  cudaStream_t st = (cudaStream_t)stream;
  int* eo = nullptr;
  SFC_CHECK(upload_patch_tables(tg.g, &eo, st));
  tg.eoff = eo;
  tg.dict_grid = dict_grid;
  const int rc = query_batch(ix, grid, cur_mask, centres, Q, pick, cost, nullptr, nullptr, nullptr, nullptr, st, &tg);
  cudaFreeAsync(eo, st);
  return rc;
}

int sfc_query_batch(const sfc_index* h, const float* grid, const uint8_t* cur_mask, const int32_t* centres,
                    int64_t Q, int64_t* pick, float* cost, void* stream) {
  g_err.clear();
  if (!h || Q < 0) {
    set_error("sfc_query_batch: NULL index or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!grid || !cur_mask || !centres || !pick || !cost) {
    set_error("sfc_query_batch: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  return query_batch(h->ix, grid, cur_mask, centres, Q, pick, cost, nullptr, nullptr, nullptr, nullptr,
                     (cudaStream_t)stream);
}

int sfc_query_candidates(const sfc_index* h, const float* grid, const uint8_t* cur_mask, const int32_t* centres,
                         int64_t Q, uint64_t* qkeys, int64_t* pos, int32_t* cand, int32_t* ncand, void* stream) {
  g_err.clear();
  if (!h || Q < 0) {
    set_error("sfc_query_candidates: NULL index or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!grid || !cur_mask || !centres || !qkeys || !pos || !cand || !ncand) {
    set_error("sfc_query_candidates: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  return query_batch(h->ix, grid, cur_mask, centres, Q, nullptr, nullptr, qkeys, pos, cand, ncand,
                     (cudaStream_t)stream);
}

int fullscan_query_batch(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* gp,
                         const sfc_params* p, const int32_t* centres, int64_t Q, int64_t* pick, float* cost,
                         void* stream) {
  g_err.clear();
  if (!p || Q < 0) {
    set_error("fullscan_query_batch: NULL params or negative Q");
    return SFC_EINVAL;
  }
  if (Q == 0) return SFC_OK;
  if (!grid || !dict_mask || !cur_mask || !centres || !pick || !cost) {
    set_error("fullscan_query_batch: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  Geo g;
  SFC_CHECK(make_geo(gp, p->K, &g));
  std::vector<float> w = weights_of(p, g.ch);
  SFC_CHECK(check_weights(w));
  bool weighted = false;
  for (float v : w) weighted |= v != 1.0f;
  if (p->precision != SFC_FP32 && p->precision != SFC_FP16) {
    set_error("fullscan_query_batch: precision must be SFC_FP32 or SFC_FP16");
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
  const int cm = (weighted ? 1 : 0) | (p->cost == SFC_COST_L1 ? 2 : 0);
  const bool tc = p->precision == SFC_FP16;
  cudaStream_t st = (cudaStream_t)stream;
  if (tc) tc_trace_begin(st);
  uint32_t* dict = nullptr;
  int64_t N = 0;
  int* eo = nullptr;
  float* wd = nullptr;
  Scratch scr(st);  // dictionary and tables, freed on every return
  SFC_CHECK(dict_extract(dict_mask, g, st, &dict, &N));
  scr.adopt(dict);
  if (N <= 0) {
    set_error("the dictionary is empty (no fully known patch)");
    return SFC_EINVAL;
  }
  SFC_CHECK(upload_patch_tables(g, &eo, st));
  scr.adopt(eo);
  SFC_CHECK(upload(&wd, w.data(), w.size(), st));
  scr.adopt(wd);
  return tc ? fullscan_batch_tc(g, grid, cur_mask, dict, N, eo, wd, weighted, centres, Q, pick, cost, nullptr, st)
            : fullscan_batch(g, grid, cur_mask, dict, N, eo, wd, cm, centres, nullptr, Q, pick, cost, st);
}

int sfc_tc_prescores(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* gp,
                     const sfc_params* p, const int32_t* centres, int64_t Q, float* scores, double* bound,
                     int64_t* N_out, void* stream) {
  g_err.clear();
  if (!p || Q < 0 || !N_out) {
    set_error("sfc_tc_prescores: NULL params/N_out or negative Q");
    return SFC_EINVAL;
  }
  if (!grid || !dict_mask || !cur_mask || (Q > 0 && (!centres || !scores || !bound))) {
    set_error("sfc_tc_prescores: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  Geo g;
  SFC_CHECK(make_geo(gp, p->K, &g));
  std::vector<float> w = weights_of(p, g.ch);
  SFC_CHECK(check_weights(w));
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* dict = nullptr;
  int64_t N = 0;
  int* eo = nullptr;
  float* wd = nullptr;
  Scratch scr(st);
  SFC_CHECK(dict_extract(dict_mask, g, st, &dict, &N));
  scr.adopt(dict);
  *N_out = N;
  if (N <= 0) {
    set_error("the dictionary is empty (no fully known patch)");
    return SFC_EINVAL;
  }
  SFC_CHECK(upload_patch_tables(g, &eo, st));
  scr.adopt(eo);
  SFC_CHECK(upload(&wd, w.data(), w.size(), st));
  scr.adopt(wd);
  return tc_prescores_all(g, grid, cur_mask, dict, N, eo, wd, centres, Q, scores, bound, st);
}

int inpaint_run(float* grid, uint8_t* mask, const sfc_grid* gp, const sfc_params* p, int32_t mode, int64_t max_steps,
                int64_t* log, int64_t* steps_done, void* stream) {
  g_err.clear();
  if (!grid || !mask || !p || !steps_done) {
    set_error("inpaint_run: NULL pointer");
    return SFC_EINVAL;
  }
  if (mode != SFC_MODE_FULLSCAN && mode != SFC_MODE_SFC) {
    set_error("inpaint_run: mode must be SFC_MODE_FULLSCAN or SFC_MODE_SFC");
    return SFC_EINVAL;
  }
  *steps_done = 0;
  SFC_CHECK(check_device());
  Geo g;
  SFC_CHECK(make_geo(gp, p->K, &g));
  if (p->priority != SFC_PRIO_CONFIDENCE && p->priority != SFC_PRIO_CRIMINISI) {
    set_error("inpaint_run: unknown priority");
    return SFC_EINVAL;
  }
  if (p->priority == SFC_PRIO_CRIMINISI && g.ndim != 2) {
    set_error("inpaint_run: the Criminisi priority is defined for 2-D grids");
    return SFC_EINVAL;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<float> w = weights_of(p, g.ch);
  SFC_CHECK(check_weights(w));
  bool weighted = false;
  for (float v : w) weighted |= v != 1.0f;
  if (p->cost != SFC_COST_L2 && p->cost != SFC_COST_L1) {
    set_error("cost must be SFC_COST_L2 or SFC_COST_L1");
    return SFC_EINVAL;
  }
  const int cm = (weighted ? 1 : 0) | (p->cost == SFC_COST_L1 ? 2 : 0);
  Index ix;
  int rc = SFC_OK;
  uint32_t* dict = nullptr;
  int64_t N = 0;
  int* eo = nullptr;
  float* wd = nullptr;
  if (mode == SFC_MODE_SFC) {
    rc = build_index(grid, mask, gp, p, st, ix);
    if (rc != SFC_OK) {
      free_index(ix);
      return rc;
    }
    dict = ix.dict;
    N = ix.N;
    eo = ix.eoff_all;
    wd = ix.weights;
    rc = fill_loop(g, grid, mask, p->priority, mode, &ix, dict, N, eo, wd, cm, max_steps, log, steps_done, st);
    free_index(ix);
    return rc;
  }
  {
    Scratch scr(st);  // dictionary and tables of the full-scan mode
    SFC_CHECK(dict_extract(mask, g, st, &dict, &N));
    scr.adopt(dict);
    SFC_CHECK(upload_patch_tables(g, &eo, st));
    scr.adopt(eo);
    SFC_CHECK(upload(&wd, w.data(), w.size(), st));
    scr.adopt(wd);
    rc = fill_loop(g, grid, mask, p->priority, mode, nullptr, dict, N, eo, wd, cm, max_steps, log, steps_done, st);
  }
  cudaStreamSynchronize(st);
  return rc;
}

int inpaint_run_multi(float* const* grids, uint8_t* const* masks, const sfc_grid* gs, int32_t n, const sfc_params* p,
                      int64_t max_steps, int64_t* const* logs, int64_t* steps_done, void* stream) {
  g_err.clear();
  if (n < 1 || !grids || !masks || !gs || !p || !steps_done) {
    set_error("inpaint_run_multi: NULL pointer or n < 1");
    return SFC_EINVAL;
  }
  for (int i = 0; i < n; ++i) {
    steps_done[i] = 0;
    if (!grids[i] || !masks[i]) {
      set_error("inpaint_run_multi: NULL grid or mask of image " + std::to_string(i));
      return SFC_EINVAL;
    }
  }
  SFC_CHECK(check_device());
  if (p->priority != SFC_PRIO_CONFIDENCE && p->priority != SFC_PRIO_CRIMINISI) {
    set_error("inpaint_run_multi: unknown priority");
    return SFC_EINVAL;
  }
  if (p->priority == SFC_PRIO_CRIMINISI && gs[0].ndim != 2) {
    set_error("inpaint_run_multi: the Criminisi priority is defined for 2-D grids");
    return SFC_EINVAL;
  }
  if (p->knn > 0) {
    set_error("inpaint_run_multi: the multi-image search runs the window search (knn = 0)");
    return SFC_EUNSUPPORTED;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // every image's index of its initial image (released on every return)
  std::vector<Index> ixs(n);
  struct Free {
    std::vector<Index>& v;
    int built = 0;
    ~Free() {
      for (int i = 0; i < built; ++i) free_index(v[i]);
    }
  } fr{ixs};
  for (int i = 0; i < n; ++i) {
    if (gs[i].ndim != gs[0].ndim || gs[i].ch != gs[0].ch) {
      set_error("inpaint_run_multi: every image needs image 0's dimension and channel count");
      return SFC_EINVAL;
    }
    const int rc = build_index(grids[i], masks[i], &gs[i], p, st, ixs[i]);
    fr.built = i + 1;
    if (rc != SFC_OK) return rc;
  }
  std::vector<const Index*> ptr(n);
  for (int i = 0; i < n; ++i) ptr[i] = &ixs[i];
  const int rc = fill_loop_multi(ptr.data(), grids, masks, n, p->priority, max_steps, logs, steps_done, st);
  cudaStreamSynchronize(st);
  return rc;
}

int sfc_debug_fail_alloc(int64_t n) {
  g_fail_alloc.store(n > 0 ? n : 0);
  return SFC_OK;
}

int64_t sfc_debug_alloc_count(void) { return g_alloc_count.load(); }

int sfc_debug_pool_used(uint64_t* bytes) {
  g_err.clear();
  if (!bytes) {
    set_error("sfc_debug_pool_used: NULL pointer");
    return SFC_EINVAL;
  }
  *bytes = 0;
  int dev = 0;
  SFC_TRY(cudaGetDevice(&dev));
  SFC_TRY(cudaDeviceSynchronize());
  cudaMemPool_t pool = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev >= 0 && dev < 128) pool = g_pool[dev];
  }
  if (pool) SFC_TRY(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, bytes));
  return SFC_OK;
}

int sfc_debug_lookback(int64_t spin_limit, int32_t stall) {
  sort_lookback_test(spin_limit, stall);
  return SFC_OK;
}

int sfc_debug_sort(int32_t force_lsd, int32_t bucket_cap) {
  sample_sort_test(force_lsd, bucket_cap);
  return SFC_OK;
}

int sfc_status(void* stream) {
  g_err.clear();
  SFC_CHECK(check_device());
  SFC_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  uint32_t v = 0, zero = 0;
  SFC_TRY(cudaMemcpyFromSymbol(&v, g_status_word, sizeof(v)));
  SFC_TRY(cudaMemcpyToSymbol(g_status_word, &zero, sizeof(zero)));
  if (v & ST_TIMEOUT) {
    set_error("a bounded device-side wait timed out");
    return SFC_ETIMEOUT;
  }
  if (v & ST_OVERFLOW) {
    set_error("the fill loop stopped: a step filled no pixel");
    return SFC_EDEVICE;
  }
  if (v & ST_BAD_CENTRE) {
    set_error("a query centre lies outside the valid centre range");
    return SFC_EDEVICE;
  }
  return SFC_OK;
}

}  // extern "C"
