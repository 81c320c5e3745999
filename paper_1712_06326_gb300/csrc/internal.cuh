// internal.cuh -- declarations shared by the translation units of libsfc.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "common.cuh"

namespace sfc {

void set_error(const std::string& msg);

// Host-side count of kernel launches made by the library (diagnostics).
void count_launch();
void count_launches(int64_t n);  // n kernels launched at once (a graph), or -n captured but not run

// Evaluate a CUDA runtime call; on failure record the message and return SFC_ECUDA
// (SFC_ENOMEM for allocation failures) from the enclosing function.
#define SFC_TRY(call)                                                                                  \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess) {                                                                           \
      ::sfc::set_error(std::string(#call) + ": " + cudaGetErrorString(e_));                            \
      return e_ == cudaErrorMemoryAllocation ? SFC_ENOMEM : SFC_ECUDA;                                 \
    }                                                                                                  \
  } while (0)

#define SFC_CHECK(rc)                     \
  do {                                    \
    int r_ = (rc);                        \
    if (r_ != SFC_OK) return r_;          \
  } while (0)

// Dynamic shared memory above this size is opted into per kernel
// (cudaFuncAttributeMaxDynamicSharedMemorySize): without the opt-in, static +
// dynamic shared memory must stay within 48 KB, and the static part of the
// library's kernels is below 8 KB.
constexpr size_t kSmemOptIn = 40 * 1024;

// Library-owned device status word of the current device (see ST_* bits).
uint32_t* status_word();

// Stream-ordered allocation from the library's own memory pool on the current
// device (created on first use; it keeps freed memory for reuse instead of
// returning it to the driver at every synchronisation).
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t st);
template <typename T>
inline cudaError_t pmalloc(T** p, size_t bytes, cudaStream_t st) {
  return pool_malloc(reinterpret_cast<void**>(p), bytes, st);
}

// The stream-ordered allocations of one call: each is freed on the stream
// (cudaFreeAsync) when the guard goes out of scope, unless ownership was passed
// on with keep() -- so an early error return frees everything taken so far.
class Scratch {
 public:
  explicit Scratch(cudaStream_t st) : st_(st) {}
  Scratch(const Scratch&) = delete;
  Scratch& operator=(const Scratch&) = delete;
  ~Scratch() {
    for (void* p : ptrs_)
      if (p) cudaFreeAsync(p, st_);
  }
  template <typename T>
  cudaError_t alloc(T** p, size_t bytes) {
    *p = nullptr;
    cudaError_t e = pool_malloc(reinterpret_cast<void**>(p), bytes, st_);
    if (e == cudaSuccess) ptrs_.push_back(*p);
    return e;
  }
  // p, allocated elsewhere on the same stream, is freed by the guard too
  void adopt(void* p) {
    if (p) ptrs_.push_back(p);
  }
  // ownership of p moves to the caller's object (not freed by the guard)
  void keep(const void* p) {
    for (void*& q : ptrs_)
      if (q == p) q = nullptr;
  }

 private:
  cudaStream_t st_;
  std::vector<void*> ptrs_;
};

// Per-index state (host struct, device arrays).
struct Index {
  Geo g;
  int C, D, bits, bp, W, select, m, s;
  int64_t N;
  float frac;
  int64_t pca_sample;
  bool keep;
  std::vector<int32_t> subset_h;  // C*m patch pixel indices
  std::vector<float> weights_h;   // ch
  // device arrays
  uint32_t* dict = nullptr;   // N centre linear indices
  int* eoff_all = nullptr;    // n element offsets (pixel offset * ch + channel) of the whole patch
  int* sub_eoff = nullptr;    // C*s element offsets of the subset values
  int* sub_pix = nullptr;     // C*m patch pixel indices of the subsets
  float* weights = nullptr;   // ch
  float* basis = nullptr;     // C*s*D
  float* mean = nullptr;      // C*s
  double* evals = nullptr;    // C*s
  float* lo = nullptr;        // C*D
  float* scale = nullptr;     // C*D
  int32_t* shifts = nullptr;  // C*D
  float* proj = nullptr;      // C*N*D (kept only with keep_intermediates)
  uint64_t* keys = nullptr;   // C*N unsorted (kept only with keep_intermediates)
  uint64_t* skeys = nullptr;  // C*N
  uint32_t* sids = nullptr;   // C*N
  int knn = 0;                // k of the exact k-NN lists (0: window search)
  int curve = SFC_CURVE_MORTON;
  bool l1 = false;            // rescore with the L1 norm (Sec. III.K)
  uint32_t* sqc = nullptr;    // C*N*D quantised shifted coordinates in curve order (knn > 0 only)
  // tracing (sfc_trace): phase events of the build and the eigen-solve iterations
  cudaEvent_t ev[SFC_TRACE_PHASES + 1] = {};
  bool traced = false;
  int p_block = 0;             // subspace block size
  int* eig_iters = nullptr;    // 2C (device): FP64 then FP32 products A Q computed per index
  int eig_per_orth = 1;        // products per orthonormalisation (2 on the cluster path)
  int* pca_done = nullptr;     // C (device): 1 where the eigen-solve converged (PCA builds only)
  bool bf16 = false;           // precision tier: projections on tensor cores, stored as BF16 (proj holds BF16)
  cudaEvent_t ev_proj[2] = {};  // traced BF16 builds: around the tensor-core projection launch
  double proj_flops = 0.0, proj_bytes = 0.0;  // its algorithmic work (set by project_bf16)
};

// Record phase boundary k of a traced build (no-op otherwise).
void trace_mark(Index& ix, int k, cudaStream_t st);
// Tracing of one tensor-core full scan on this host thread (no-ops unless
// tracing is on): begin records boundary 0, mark boundary k (1..3), end waits
// for the last one and adds the phase times and the GEMM's flops.
void tc_trace_begin(cudaStream_t st);
void tc_trace_mark(int k, cudaStream_t st);
void tc_trace_end(double gemm_flops);

// k_dict.cu
int dict_extract(const uint8_t* mask, const Geo& g, cudaStream_t st, uint32_t** dict, int64_t* N);

int dict_extract_into(const uint8_t* mask, const Geo& g, cudaStream_t st, uint8_t* a, uint8_t* b, uint32_t* counts,
                      int64_t* dtotal, uint32_t* out, int64_t* N);

// k_pca.cu: basis/mean/evals of every index from a deterministic sample.
int pca_build(Index& ix, const float* grid, cudaStream_t st);

// k_index.cu: projection, quantisation, Morton keys.
// Curves [c0, c0 + nc): projections (with the per-axis minima / maxima in
// lohi, 2 words per axis of every curve, and lo / scale), then keys.
int project_curves(Index& ix, const float* grid, float* proj, uint32_t* lohi, int c0, int nc, cudaStream_t st);
int key_curves(Index& ix, const float* proj, uint64_t* keys, int c0, int nc, cudaStream_t st);
// lohi (2 words per axis of every curve) reset, and lo / scale of every curve from it
int lohi_init(uint32_t* lohi, int n, cudaStream_t st);
int lohi_to_scale(Index& ix, const uint32_t* lohi, cudaStream_t st);
// k_proj_tc.cu: the BF16 tier -- every curve's projections (proj as BF16
// [C][N][D]) by one tensor-core GEMM, with the per-axis minima / maxima in lohi
// (initialised here) and lo / scale; keys then come from key_curves.
int project_bf16(Index& ix, const float* grid, void* proj, uint32_t* lohi, cudaStream_t st);
// The library's auxiliary streams of the current device (k < kAuxStreams,
// default priority) and one of the highest priority, created on first use,
// non-blocking; nullptr if a stream cannot be created.
constexpr int kAuxStreams = 3;
cudaStream_t aux_stream(int k);
cudaStream_t aux_stream_hi();
// Quantised, shifted coordinates of the dictionary in each index's sorted order
// (the k-NN search reads them next to the sorted keys): ix.sqc from proj.
int sorted_coords(Index& ix, const float* proj, cudaStream_t st);

// k_sort.cu: stable LSD radix sort (onesweep) of (key, id) per index.
// scratch: radix_sort_scratch_bytes(N, C, key_bits) bytes of device memory
// usable on st, or nullptr (then allocated and freed on st).
int radix_sort_pairs(const uint64_t* keys, uint64_t* skeys, uint32_t* sids, int64_t N, int C, int key_bits,
                     cudaStream_t st, void* scratch = nullptr);
size_t radix_sort_scratch_bytes(int64_t N, int C, int key_bits);
// Failure injection (tests): the onesweep look-back's poll limit (<= 0: the
// default kSpinLimit) and, with stall = 1, look-backs that poll a word nothing
// writes, so every tile after the first gives up after spin_limit polls.
void sort_lookback_test(long long spin_limit, int stall);
// k_sort.cu: sample sort of (key, id) per index for N <= 2^20 (the same order
// as the LSD sort).  ovf: C device ints, set to 1 for an index whose pairs were
// not sorted (a bucket above the shared-memory capacity): the caller sorts
// that index with radix_sort_pairs.  scratch as for radix_sort_pairs.
bool sample_sort_fits(int64_t N);
int sample_sort_pairs(const uint64_t* keys, uint64_t* skeys, uint32_t* sids, int64_t N, int C, int* ovf,
                      cudaStream_t st, void* scratch = nullptr);
size_t sample_sort_scratch_bytes(int64_t N, int C);
// Tests: force the LSD sort (force_lsd = 1), or lower the bucket capacity
// (cap > 0) so that indices overflow and take the LSD sort after the sample
// sort; (0, 0) restores the defaults.
void sample_sort_test(int force_lsd, int cap);

// k_query.cu
// Targets on a grid other than the index's: its geometry, its patch element
// offsets (device), and the index's grid holding the dictionary patches.
struct TargetGrid {
  Geo g;
  const int* eoff;
  const float* dict_grid;
};
// Device buffers for the split form of a small batch (up to qmax queries of up
// to cap candidates each): the candidate ids, their number and their FP32 costs.
struct QSplit {
  int32_t* cand = nullptr;  // qmax * cap
  int32_t* ncand = nullptr; // qmax
  float* c32 = nullptr;     // qmax * cap
  int64_t cap = 0, qmax = 0;
};
// Candidates per query of an index (C * window, or C * k): the size of a QSplit.
int64_t query_split_cap(const Index& ix);
// Batches of up to 32 queries with picks run in the split form (the rescore
// spread over many CTAs; same picks and costs), in `split` if given and large
// enough, else in stream-ordered scratch (the one-CTA form while `st` is being
// captured).
int query_batch(const Index& ix, const float* grid, const uint8_t* cur_mask, const int32_t* centres, int64_t Q,
                int64_t* pick, float* cost, uint64_t* qkeys, int64_t* pos, int32_t* cand, int32_t* ncand,
                cudaStream_t st, const TargetGrid* tgt = nullptr, const QSplit* split = nullptr);
// Queries of several images in one launch (every index built with the same
// parameters); the object keeps a device table of the images.
struct MultiQuery;
int multi_query_create(const Index* const* ixs, const float* const* grids, const uint8_t* const* masks, int n,
                       cudaStream_t st, MultiQuery** out);
void multi_query_destroy(MultiQuery* m);
// split: buffers for the split form (used when Q <= 32 and they are large enough).
int multi_query_run(const MultiQuery* m, const int32_t* img_of, const int32_t* centres, int64_t Q, int64_t* pick,
                    float* cost, cudaStream_t st, const QSplit* split = nullptr);
// k_fill.cu: the fill loops of n images in SFC mode, every round one step of
// every image not done (ixs: each image's index of its initial image, built
// with the same parameters; grids / masks: device, updated in place; logs:
// NULL or n device logs; steps_done: host int64[n]).  Synchronises st.
int fill_loop_multi(const Index* const* ixs, float* const* grids, uint8_t* const* masks, int n, int prio,
                    int64_t max_steps, int64_t* const* logs, int64_t* steps_done, cudaStream_t st);

// k_fullscan.cu
// cm (cost mode): bit 0 = channel weights other than 1, bit 1 = L1 norm (Sec. III.K).
int fullscan_batch(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                   const int* eoff_all, const float* weights, int cm, const int32_t* centres,
                   const int64_t* centre_lin, int64_t Q, int64_t* pick, float* cost, cudaStream_t st);
// The FP32 scan's tile shapes: their number, with (queries per tile, entries
// per thread) into qt / ept (either may be NULL; arrays of at least 8).
int fullscan_tile_shapes(int* qt, int* ept);
// The shape fullscan_batch uses (process-wide): shape in range sets it; returns
// the one in use.
int fullscan_tile_shape(int shape);

int fullscan_batch_tc(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                      const int* eoff_all, const float* weights, bool weighted, const int32_t* centres, int64_t Q,
                      int64_t* pick, float* cost, int* nsel, cudaStream_t st);
int tc_prescores_all(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                     const int* eoff_all, const float* weights, const int32_t* centres, int64_t Q, float* scores,
                     double* bound, cudaStream_t st);

int fullscan_batch_into(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                        const int* eoff_all, const float* weights, int cm, const int32_t* centres, int64_t Q,
                        int64_t* pick, float* cost, int64_t* lin, uint8_t* bad, unsigned int* gmin, float* tilemin,
                        cudaStream_t st);

// Dictionary split of the full scan (one shard's part; see k_fullscan.cu).
int64_t fullscan_range_tiles(int64_t n);
int fullscan_range_scan(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t n,
                        const int* eoff_all, const float* weights, int cm, const int64_t* lin, int64_t Q,
                        float* tilemin, unsigned int* gmin, cudaStream_t st);
int fullscan_range_band(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t n,
                        const int* eoff_all, const float* weights, int cm, const int64_t* lin, int64_t Q,
                        const uint8_t* bad, const float* tilemin, const unsigned int* gmin, int64_t id_base,
                        int64_t* id, float* cost32, double* cost64, cudaStream_t st);
int centres_to_lin(const Geo& g, const int32_t* centres, int64_t Q, int64_t* lin, uint8_t* bad, cudaStream_t st);

// helpers (sfc_api.cu)
int upload_patch_tables(const Geo& g, int** eoff_all, cudaStream_t st);
int check_device();
int make_geo(const sfc_grid* gp, int K, Geo* out);

}  // namespace sfc
