/* sfc.h -- C-ABI of libsfc, the GB300 (sm_103a) patch-search library for
 * exemplar-based inpainting with space-filling-curve indices (Dahmen et al.,
 * "Space-Filling Curve Indices as Acceleration Structure for Exemplar-Based
 * Inpainting").
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Pointers.  Unless a parameter says "host", it is a DEVICE pointer on the
 * current CUDA device, owned by the caller, which keeps it alive until the work
 * enqueued on `stream` has finished.  `stream` is a cudaStream_t passed as
 * void* (NULL = the legacy default stream).
 *
 * Grid layout.  float32, C-contiguous [Z][Y][X][ch] (x fastest, channel
 * innermost); Z = 1 for 2-D.  Masks are uint8 [Z][Y][X], 1 = known value.
 * A pixel's linear index is (z*Y + y)*X + x.  Patches are K x K (x K) boxes
 * centred on a pixel, with elements in patch raster order (x fastest) and the
 * channels innermost (the paper treats RGB values separately, Sec. II intro).
 * Centres are int32 (x, y[, z]) rows; a valid centre keeps its whole patch
 * inside the grid.
 *
 * Dictionary.  The patches whose box is inside the grid and fully known under
 * the dictionary mask (Sec. I: the known parts of the image split into
 * patches).  A dictionary id is the rank of the centre in raster order.
 *
 * Cost.  Masked squared L2 (Sec. II after Fig. 1: differences at unknown
 * pixels are taken as zero), optionally weighted per channel:
 *   cost(t, j) = sum over known elements e of t: w[ch(e)] * (t_e - p_{j,e})^2.
 * Picks are the argmin over the exact value -- the FP64 sum over elements in
 * raster order with operands widened from FP32 and no fused multiply-add --
 * with ties to the lowest dictionary id.  The kernels compute FP32 costs; when
 * more than one candidate lies inside the band that the FP32 rounding error
 * bound leaves around the minimum, those candidates are rescored with that FP64
 * sum, so the picks are exactly those of the definition.  Reported costs are the
 * FP32 costs of the picks (within (n + 8) * 2^-24 relative of the exact value,
 * n = values per patch).
 *
 * Errors.  Every entry point returns SFC_OK (0) or a negative SFC_E* code and
 * records a message readable with sfc_last_error() (per host thread).  Calls
 * are asynchronous unless stated: argument errors are reported at once; faults
 * a kernel detects (an invalid centre, a timed-out wait) are written to a
 * status word and reported by sfc_status() or by the next synchronising call.
 * No entry point falls back to a CPU path.
 */
#ifndef SFC_H
#define SFC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SFC_OK = 0,
  SFC_EINVAL = -1,       /* invalid argument (sizes, null pointers, parameter ranges) */
  SFC_ENOMEM = -2,       /* device allocation failed */
  SFC_ECUDA = -3,        /* a CUDA runtime call failed */
  SFC_ETIMEOUT = -4,     /* a bounded device-side wait gave up */
  SFC_EUNSUPPORTED = -5, /* device is not sm_103 / feature not built */
  SFC_EDEVICE = -6,      /* a kernel flagged invalid data (e.g. a centre outside the grid) */
  SFC_ENOCONV = -7       /* a PCA eigen-solve of sfc_index_build did not converge */
};

enum { SFC_SELECT_ALL = 0, SFC_SELECT_BEST = 1 };
enum { SFC_FP32 = 0, SFC_BF16 = 1, SFC_FP16 = 2 };
enum { SFC_PRIO_CONFIDENCE = 0, SFC_PRIO_CRIMINISI = 1 };
enum { SFC_MODE_FULLSCAN = 0, SFC_MODE_SFC = 1 };
/* Curve of the index keys: the z-curve of the paper (Sec. II.C), or the
 * Hilbert curve (Skilling's transpose method, "Programming the Hilbert curve",
 * 2004: the coordinates are transformed to the transposed Hilbert index, then
 * interleaved like the Morton key and cut to the top 64 bits the same way). */
enum { SFC_CURVE_MORTON = 0, SFC_CURVE_HILBERT = 1 };
/* Cost of a (target, source) pair over the target's known elements: the
 * squared L2 norm sum w (t - p)^2 (Sec. II) or the L1 norm sum w |t - p|
 * (Sec. III.K).  The exact pick is the argmin of the FP64 sum (terms in patch
 * raster order, channel innermost); FP32 costs are within (n + 8) 2^-24 of it. */
enum { SFC_COST_L2 = 0, SFC_COST_L1 = 1 };

/* Grid geometry.  ext = {X, Y, Z}; ndim 2 (Z must be 1) or 3; ch >= 1. */
typedef struct sfc_grid {
  int32_t ndim;
  int32_t ch;
  int64_t ext[3];
} sfc_grid;

/* Method parameters (Table 1 of the paper: K, c, D, k; here k is a window W).
 * Host pointers inside are read during the call only. */
typedef struct sfc_params {
  int32_t K;              /* patch side, odd, 3..15, <= every extent */
  int32_t curves;         /* C: number of indices, 1..8 (2-D) or 1..14 (3-D) (Sec. II, Fig. 2) */
  int32_t dims;           /* D: principal components kept, 1..16, <= subset length (Sec. II.A) */
  int32_t bits;           /* b: bits per quantised coordinate, 1..21 (Sec. II.C) */
  int32_t window;         /* W >= 1: sorted slots read around the binary-search position */
  float subset_frac;      /* c in (0, 1]: fraction of patch pixels per index (Sec. II) */
  const int32_t* shifts;  /* host, curves*dims integer shifts in [0, 2^b), or NULL (= none) */
  const float* ch_weights;/* host, ch positive weights, or NULL (= all 1) */
  const float* basis;     /* host, curves*s*D FP32 basis (row i = subset value i), or NULL = PCA */
  const float* mean;      /* host, curves*s FP32 means (required with basis) */
  int32_t select;         /* SFC_SELECT_ALL or SFC_SELECT_BEST (Fig. 1(b)) */
  int32_t precision;      /* SFC_FP32; fullscan_query_batch also takes SFC_FP16 (tensor-core pre-score);
                             sfc_index_build also takes SFC_BF16 (the precision tier: dictionary projections
                             on tensor cores, stored in BF16) */
  int64_t pca_sample;     /* dictionary entries used for the covariance; <= 0: all */
  int32_t priority;       /* fill order: SFC_PRIO_CONFIDENCE or SFC_PRIO_CRIMINISI (2-D) */
  int32_t keep_intermediates; /* 1: keep projections and unsorted keys for sfc_index_export */
  int32_t knn;            /* k in 1..128: per selected index, the exact k nearest dictionary entries in the
                             quantised principal space (Sec. II.D) are the candidates instead of the window;
                             0: the window of W sorted slots */
  int32_t curve;          /* SFC_CURVE_MORTON (default) or SFC_CURVE_HILBERT (window search only) */
  int32_t cost;           /* SFC_COST_L2 (default) or SFC_COST_L1; full scan, queries and fill loop
                             (SFC_FP16 takes L2 only) */
} sfc_params;

typedef struct sfc_index sfc_index; /* opaque; owned by the library */

/* Fill `p` with the paper's defaults (K = 9, c = 0.6, D = 10, 8 indices; Sec.
 * III.A) and W = 80, b = 8, SELECT_ALL, FP32, pca_sample = 16384, knn = 0
 * (window search). */
void sfc_params_default(sfc_params* p);

/* Build the multi-index (Sec. II.A-C): dictionary extraction, the pixel subsets
 * of Fig. 2, a PCA per index (covariance of a deterministic sample accumulated to FP64
 * accuracy, leading eigenvectors by FP64 subspace iteration) unless p->basis is
 * given, FP32 projection, per-axis
 * quantisation to b bits, Morton keys (top 64 bits), and a sort of (key, id)
 * per index in key order, ties by id (a sample sort for up to 2^20 dictionary
 * entries, an LSD radix sort above).  grid/dict_mask: device, layout above.  On
 * success *out owns device memory until sfc_index_destroy.  Synchronises
 * `stream` once to learn the dictionary size and, when it computes the PCA or
 * takes the sample sort, once more near the end to read the eigen-solves'
 * convergence and the sort's flags (an index whose sample sort overflowed a
 * bucket is sorted again by the radix sort).  Subsets of up to 64 values
 * are solved completely by FP64 Jacobi; longer ones by subspace iteration,
 * taken over by Jacobi (up to 112 values) where the iteration stalls.
 * SFC_EINVAL if the dictionary is empty; SFC_ENOCONV (no index is returned) if
 * an eigen-solve did not converge.
 *
 * Precision tier (p->precision = SFC_BF16): the dictionary's projections are
 * one tensor-core GEMM for every index at once (tcgen05, BF16 operands, FP32
 * accumulation): the whole patch, centred per element by its mean and rounded
 * to BF16, times the indices' basis columns in BF16 (zero outside each index's
 * subset), rounded to BF16 -- the stored projections (exported widened to
 * FP32).  The quantiser's range and the keys come from these values; queries
 * still project in FP32 and every pick is rescored exactly, so only the
 * candidate windows differ from the FP32 index.  Requires curves * dims <= 256. */
int sfc_index_build(const float* grid, const uint8_t* dict_mask, const sfc_grid* g, const sfc_params* p,
                    void* stream, sfc_index** out);

/* Release an index (waits for the device first).  NULL is accepted. */
int sfc_index_destroy(sfc_index* ix);

/* Sizes of an index: dictionary size N, subset pixels m, values per subset s. */
int sfc_index_info(const sfc_index* ix, int64_t* N, int32_t* m, int32_t* s);

/* Copy the index's arrays to HOST buffers (any may be NULL); synchronises.
 * dict: N centre linear indices (int64); subsets: C*m patch pixel indices;
 * basis: C*s*D; mean: C*s; evals: C*s (descending; the leading
 * min(s, max(2D, D + 8), 24) are computed, the rest and all of them with a
 * given basis are NaN);
 * lo, scale: C*D; proj: C*N*D and keys: C*N (need keep_intermediates);
 * skeys: C*N; sids: C*N (sorted order per index). */
int sfc_index_export(const sfc_index* ix, int64_t* dict, int32_t* subsets, float* basis, float* mean, double* evals,
                     float* lo, float* scale, float* proj, uint64_t* keys, uint64_t* skeys, uint32_t* sids);

/* Answer Q queries against the index (Fig. 1(b)-(d)): for each centre, select
 * the indices (all, or the one covering most known subset pixels), project the
 * known subset values (unknown ones contribute zero), quantise with the index's
 * lo/scale (clamped), take the Morton key, binary-search each sorted key array,
 * gather the W sorted slots around the position (clamped inside [0, N)), rescore
 * the union of candidates with the exact cost in image space and return the
 * argmin.  grid/cur_mask: the current image and known-mask (same geometry as the
 * build); centres: Q x ndim int32; pick: Q int64 dictionary ids; cost: Q float
 * (FP32 cost of the pick).  Q = 0 is a no-op.  A centre outside the valid range
 * yields pick = -1, cost = NaN and SFC_EDEVICE from sfc_status(). */
int sfc_query_batch(const sfc_index* ix, const float* grid, const uint8_t* cur_mask, const int32_t* centres,
                    int64_t Q, int64_t* pick, float* cost, void* stream);

/* With knn = k > 0 in the build parameters, the window is replaced by the
 * paper's exact k-NN list (Sec. II.D) per selected index: the k dictionary
 * entries nearest to the query in the quantised principal space (squared
 * Euclidean distance of the integer coordinates, ties by id).  The index then
 * also keeps the quantised coordinates in curve order (C*N*D uint32); each
 * list is found by one warp that scans the index's sorted keys inside the
 * z-interval of the box around the query that the current k-th distance
 * spans, shrinking the box as the list improves and jumping over runs of keys
 * outside the box with Tropf and Herzog's BIGMIN.  The candidates are the union
 * of the lists, rescored as above. */

/* Stored indices (for a dictionary that is built once and queried many
 * times, or from other grids).  sfc_index_save writes every array of the index
 * and its parameters to the HOST file `path` (synchronises; projections and
 * unsorted keys are not saved); sfc_index_load reads such a file onto the
 * current device (synchronises `stream` at the end) -- the result answers
 * queries exactly like the saved index.  The index does not hold its grid: the
 * caller keeps the grid the index was built from.  Files are host byte order,
 * with a magic and version checked on load (SFC_EINVAL when they differ or the
 * file is truncated). */
int sfc_index_save(const sfc_index* ix, const char* path);
/* The scalar build parameters (pointers NULL, shifts/weights/basis not
 * returned) and the build grid's geometry of an index; either may be NULL. */
int sfc_index_params(const sfc_index* ix, sfc_params* p, sfc_grid* g);
int sfc_index_load(const char* path, void* stream, sfc_index** out);

/* sfc_query_batch for targets on another grid: the target patches are read
 * from grid / cur_mask (device, geometry g: the index's ndim and ch, any
 * extents >= K; centres in its coordinates) and the dictionary patches from
 * dict_grid (device, the grid the index was built from).  Outputs as
 * sfc_query_batch. */
int sfc_query_batch_dict(const sfc_index* ix, const float* dict_grid, const float* grid, const uint8_t* cur_mask,
                         const sfc_grid* g, const int32_t* centres, int64_t Q, int64_t* pick, float* cost,
                         void* stream);

/* Many images (or volumes) of uneven size, one launch: sfc_multi_create
 * takes n indices built with the same parameters (patch, curves, dimensions,
 * bits, window, selection, curve, cost, channel weights; shifts may differ;
 * knn = 0) and each index's grid and current mask (device, the build
 * geometry), and uploads a table of the images (synchronises `stream`).
 * sfc_multi_query answers Q targets of any of the images in ONE kernel launch
 * with no allocation and no synchronisation (so it can be captured into a
 * CUDA graph): image[q] (device int32) is the target's image, centres (device,
 * Q x ndim) its centre in that image; outputs as sfc_query_batch, picks being
 * ids of that image's dictionary.  An image number outside [0, n) is treated
 * as an invalid centre (pick -1, cost NaN, SFC_EDEVICE from sfc_status).  The
 * object refers to the indices, grids and masks: destroy it before them. */
typedef struct sfc_multi sfc_multi;
int sfc_multi_create(const sfc_index* const* ix, const float* const* grids, const uint8_t* const* masks, int32_t n,
                     void* stream, sfc_multi** out);
int sfc_multi_query(const sfc_multi* mu, const int32_t* image, const int32_t* centres, int64_t Q, int64_t* pick,
                    float* cost, void* stream);
int sfc_multi_destroy(sfc_multi* mu);

/* Intermediate results of sfc_query_batch for checking: qkeys (Q*C uint64),
 * pos (Q*C int64 lower_bound positions; -1 for unselected indices),
 * cand (Q*C*L int32 sorted unique candidate ids, padded with -1; L = W, or k
 * with knn = k), ncand (Q int32). */
int sfc_query_candidates(const sfc_index* ix, const float* grid, const uint8_t* cur_mask, const int32_t* centres,
                         int64_t Q, uint64_t* qkeys, int64_t* pos, int32_t* cand, int32_t* ncand, void* stream);

/* Exact full scan (Sec. I): the cost of every dictionary patch (dictionary =
 * fully known patches of dict_mask) for each of the Q centres, evaluated against
 * cur_mask, then the global argmin (ties to the lowest id).  p supplies K and
 * ch_weights.  Outputs as sfc_query_batch. */
int fullscan_query_batch(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                         const sfc_params* p, const int32_t* centres, int64_t Q, int64_t* pick, float* cost,
                         void* stream);

/* With p->precision == SFC_FP16, fullscan_query_batch computes the pre-score
 * s(q, j) = sum m w (p'^2 - 2 t' p') (the cost minus a per-query constant,
 * values centred per channel) as a tensor-core GEMM (tcgen05; FP16 operands
 * split into high and low parts, FP32 accumulation), keeps per query the
 * minimum of every 32-entry dictionary group, and rescores exactly (FP32 +
 * FP64 band, as above) every group whose minimum lies within twice the pre-score
 * error bound E_q of the smallest: the group of the exact argmin always
 * qualifies, so picks and costs are those of the FP32 path.  E_q bounds the
 * operand splitting (3.01 u16^2 sum|a b|) and the FP32 accumulation
 * (8 K' u32 sum|a b|, K' = 6 n), with |p'| bounded by the grid's per-channel
 * range.  Values must satisfy |value - channel mean| < 128 (else SFC_EINVAL).
 *
 * Checking entry point: all Q x N pre-scores into `scores` (device, Q*N floats,
 * row-major) and E_q into `bound` (device, Q doubles); *N_out (host) gets N. */
int sfc_tc_prescores(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                     const sfc_params* p, const int32_t* centres, int64_t Q, float* scores, double* bound,
                     int64_t* N_out, void* stream);

/* fullscan_query_batch without device allocation.  The paper has no
 * counterpart: this is an interface for callers that cannot call cudaMalloc --
 * for example a host framework whose own allocator owns the device memory and
 * forbids libraries from allocating behind its back, or a latency-critical
 * caller that cannot afford the implicit synchronisation an allocation may
 * cause.  Arguments, results and errors are those of fullscan_query_batch; the
 * caller still passes every input and output.  With SFC_FP16 this entry point
 * runs the FP32 scan, whose picks and costs the tensor-core form reproduces
 * bit for bit anyway (its operands would not fit the static array).  All scratch lives in one
 * library-owned static device array of 16 MiB (held by every GPU that loads the
 * library until the process exits); a call whose grid and batch would need more
 * -- about 2 bytes per pixel + 4 bytes per valid centre + 13 bytes per query +
 * 4 bytes per query per 1,024 valid centres -- is rejected with SFC_EINVAL
 * before any device work (so is any single size beyond the array: more pixels
 * than bytes, or more than 16 MiB / 13 queries).  The first call on a device looks up that array's
 * device address; make that first call before any stream capture.  All calls
 * share the array and it keeps the last call's contents, so calls that overlap
 * on the GPU (concurrent streams or host threads) race: serialise them.
 * Synchronises `stream` once (to learn the dictionary size). */
int fullscan_query_batch_static(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask,
                                const sfc_grid* g, const sfc_params* p, const int32_t* centres, int64_t Q,
                                int64_t* pick, float* cost, void* stream);

/* ---- The full scan split over dictionary shards (several GPUs) ------------
 * One exact full scan (Sec. I) over a dictionary shared out among S shards,
 * e.g. one per GPU: shard s owns the dictionary ids [floor(s N / S),
 * floor((s + 1) N / S)).  Per query batch:
 *   sfc_shard_scan  -- the shard's FP32 scan; min32 (device, Q uint32) gets the
 *                      shard's minimum FP32 cost as float bits (+inf bits for
 *                      an empty shard; costs are >= 0, so the bits order like
 *                      the values);
 *   (caller)        -- gmin32 = the element-wise minimum of min32 over all
 *                      shards (e.g. an all-reduce-min);
 *   sfc_shard_band  -- every shard entry inside the FP32 error band of gmin32
 *                      rescored with the exact FP64 cost; cost64 (device, Q
 *                      doubles), id (device, Q int64, ids of the whole
 *                      dictionary) and cost32 (device, Q floats) get the
 *                      shard's (cost64, id) minimum and its FP32 cost, or
 *                      (+inf, -1, +inf) if the shard holds no band entry;
 *   (caller)        -- the pick is the (cost64, id) minimum over the shards
 *                      (e.g. an all-gather of 20 bytes per query and shard),
 *                      its cost the FP32 cost reported with it.
 * The result equals fullscan_query_batch's picks and costs (SFC_FP32 only).  An
 * invalid centre gives (NaN, -1, NaN) on every shard (and SFC_EDEVICE from
 * sfc_status()).  sfc_shard_create extracts the dictionary (synchronises
 * `stream` once), keeps the centres' indices and the scan's scratch; the shard
 * refers to grid and cur_mask (device, the caller keeps them alive) and must be
 * used on the device it was created on.  sfc_shard_range reports N and the
 * shard's [j0, j1); any output may be NULL. */
typedef struct sfc_shard sfc_shard;
int sfc_shard_create(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                     const sfc_params* p, const int32_t* centres, int64_t Q, int32_t shard, int32_t nshards,
                     void* stream, sfc_shard** out);
int sfc_shard_range(const sfc_shard* s, int64_t* N, int64_t* j0, int64_t* j1);
int sfc_shard_scan(sfc_shard* s, uint32_t* min32, void* stream);
int sfc_shard_band(sfc_shard* s, const uint32_t* gmin32, double* cost64, int64_t* id, float* cost32, void* stream);
int sfc_shard_destroy(sfc_shard* s);

/* Exemplar-based inpainting loop (Sec. I; Fig. 1(a)): repeat { find the fill
 * front (known pixels with an unknown axis neighbour; centres moved inside the
 * valid range), take the centre of highest priority (ties: lowest linear
 * index), search the dictionary of the initial mask (mode: full scan, or SFC
 * query against an index built here from the initial image), copy the source
 * patch into the target's unknown pixels } until no pixel is unknown or
 * max_steps (> 0) steps.  grid, mask: device, updated in place.  log: device
 * int64 [max_steps or #unknown][ndim + 1] rows (centre coordinates, pick), or
 * NULL.  steps_done: host.  Synchronises `stream`. */
int inpaint_run(float* grid, uint8_t* mask, const sfc_grid* g, const sfc_params* p, int32_t mode, int64_t max_steps,
                int64_t* log, int64_t* steps_done, void* stream);

/* The inpainting loop of n images at once (the batched configuration; the
 * paper runs one image at a time): each image gets the index of its initial
 * image (sfc_index_build with p, SFC mode, knn = 0), then every round takes one
 * step of every image whose loop is not done -- priorities, target, one
 * multi-image query launch for all images, insert -- until every image is done
 * or has max_steps (> 0) steps.  Each image ends exactly as inpaint_run(mode =
 * SFC_MODE_SFC) leaves it: same grid, mask and log.  grids, masks, logs: HOST
 * arrays of n DEVICE pointers (logs: NULL, or each image's log as for
 * inpaint_run); gs: host array of n grids (same dimension and channels, any
 * extents); steps_done: host int64[n].  SFC_EUNSUPPORTED for knn > 0.
 * Synchronises `stream`. */
int inpaint_run_multi(float* const* grids, uint8_t* const* masks, const sfc_grid* gs, int32_t n, const sfc_params* p,
                      int64_t max_steps, int64_t* const* logs, int64_t* steps_done, void* stream);

/* Read and clear the library's device-side status flags (synchronises stream):
 * SFC_OK, SFC_ETIMEOUT (a bounded wait gave up), or SFC_EDEVICE (an invalid
 * centre was seen, or a fill step made no progress). */
int sfc_status(void* stream);

/* Number of kernels the library has launched in this process so far (all host
 * threads).  Diagnostics: the difference across a region counts its launches. */
uint64_t sfc_launch_count(void);

/* Phase tracing of sfc_index_build (diagnostics; the paper reports only wall
 * times).  sfc_trace(1) enables it and clears the accumulators, sfc_trace(0)
 * disables it.  While enabled, every build records CUDA events on its stream
 * around its phases; when that index is destroyed (the device is idle then) the
 * phase durations are added to the accumulators.  sfc_trace_read copies to HOST
 * ms[SFC_TRACE_PHASES] the summed milliseconds of the phases -- dictionary,
 * moments (mean + covariance), eigen-solve, basis finalisation,
 * projection + keys, sort -- and *builds the number of builds summed, and
 * (the projections, keys and sorts run on the library's own streams; with
 * the radix sort of dictionaries above 2^20 entries they are pipelined over
 * groups of curves, and "projection + keys" ends when every group's keys exist
 * and includes the sorts of the earlier groups that overlap it; "sort" is the
 * rest of the sorting, with the sample sort all of it) and
 * *eig_flops the summed algorithmic FP64 flops of the eigen-solves
 * (per index: 2 s^2 p per product of the covariance with the block and 4 s p^2
 * per orthonormalisation, s = subset length, p = block size).  Any output may be NULL. */
enum { SFC_TRACE_PHASES = 6 };
int sfc_trace(int on);
int sfc_trace_read(double* ms, int64_t* builds, double* eig_flops);
/* The eigen-solves' algorithmic flops split by precision: *fp64_flops as
 * eig_flops above (FP64 products and every orthonormalisation), *fp32_flops
 * 2 s^2 p per product taken in FP32 (the early iterations of the cluster
 * path).  Either output may be NULL. */
int sfc_trace_eig_read(double* fp64_flops, double* fp32_flops);

/* While tracing is enabled, every fullscan_query_batch with SFC_FP16 also
 * records events around its phases -- operands (dictionary, centring, A and B
 * rows), pre-score GEMM, exact pass -- and waits for the last one before it
 * returns.  sfc_trace_tc_read copies to HOST ms[SFC_TRACE_TC_PHASES] their
 * summed milliseconds, *calls the number of calls summed and *gemm_flops the
 * summed algorithmic GEMM flops (per call 2 Q N 6 n).  Any output may be NULL. */
enum { SFC_TRACE_TC_PHASES = 3 };
int sfc_trace_tc_read(double* ms, int64_t* calls, double* gemm_flops);

/* While tracing is enabled, every build also records events around its
 * projection launches (SFC_BF16: the tensor-core launch; SFC_FP32: from the
 * first curve's FMA-chain launch to the last one's, which with the radix sort
 * of dictionaries above 2^20 entries also spans the keys of the earlier
 * curve groups); when the index is destroyed that time is added up.
 * sfc_trace_proj_read gives the summed milliseconds, the number of builds
 * counted, and the summed algorithmic work: 2 N C s D flops and N n 4 + N C D 2
 * bytes (SFC_BF16: patch values gathered, BF16 projections written) or
 * N C s 4 + N C D 4 bytes (SFC_FP32: subset values gathered per curve, FP32
 * projections written).  Any output may be NULL. */
int sfc_trace_proj_read(double* ms, int64_t* calls, double* flops, double* bytes);

/* ---- Parameter search (the tuned index of a batch of queries) -------------
 * sfc_autotune builds an index for every combination of the listed index
 * counts C (spec->curves), principal dimensions D (spec->dims) and windows W
 * (spec->windows; with base->knn > 0 they are the list lengths k instead) on
 * (grid, mask) -- the other parameters are base's -- and answers the Q
 * queries `centres` (device, Q x ndim) with it.  Per configuration it measures
 *   - ms: the median over spec->reps timed runs (after one untimed run) of the
 *     CUDA-event time on `stream` of build + query (SFC_TUNE_STEP) or of the
 *     query alone (SFC_TUNE_QUERY);
 *   - ae: the acceleration error of Sec. III.C on a sample of the queries
 *     (every ceil(Q / spec->sample)-th one): the mean over the sample of
 *     sqrt(cost) / sqrt(exact cost) - 1, where the exact pick comes from
 *     fullscan_query_batch (SFC_FP16 for the L2 cost, else SFC_FP32) and a
 *     query counts 0 if the two costs are equal, 1 if only the exact cost is 0.
 * The chosen configuration is the fastest with ae <= spec->ae_max (ties to the
 * first in list order, C outermost, W innermost); if none qualifies, the one of
 * least ae (ties to the faster).  *best = base with that C, D and W (or k);
 * *chosen (host, may be NULL) its position; table (host, may be NULL) receives
 * 5 doubles per configuration in list order: C, D, W (or k), ms, ae.
 * base->shifts, basis and mean must be NULL (they are sized for one (C, D)).
 * Synchronises `stream`; every configuration's index is destroyed before the
 * call returns.  Errors: SFC_EINVAL for empty lists, more than 4096
 * configurations, sample < 1, reps outside 1..100, ae_max < 0, and any
 * configuration the build refuses (the message names it). */
enum { SFC_TUNE_STEP = 0, SFC_TUNE_QUERY = 1 };
typedef struct sfc_tune_spec {
  const int32_t* curves; /* host */
  int32_t n_curves;
  const int32_t* dims;   /* host */
  int32_t n_dims;
  const int32_t* windows; /* host */
  int32_t n_windows;
  int64_t sample;        /* queries whose exact picks give ae (>= 1; all Q if larger) */
  int32_t reps;          /* timed runs per configuration, 1..100 */
  int32_t objective;     /* SFC_TUNE_STEP or SFC_TUNE_QUERY */
  double ae_max;         /* acceptable mean acceleration error, e.g. 0.01 (the paper's 1 %) */
} sfc_tune_spec;
int sfc_autotune(const float* grid, const uint8_t* mask, const sfc_grid* g, const sfc_params* base,
                 const int32_t* centres, int64_t Q, const sfc_tune_spec* spec, sfc_params* best, double* table,
                 int32_t* chosen, void* stream);
/* The selection rule of sfc_autotune on given measurements (host only; no
 * device work): returns the chosen position in 0..n-1, or -1 if n <= 0 or a
 * pointer is NULL.  NaN measurements count as +infinity. */
int32_t sfc_tune_select(int32_t n, const double* ms, const double* ae, double ae_max);

/* Tile shapes of the FP32 full scan (the paper's full scan is a CPU loop; the
 * shapes are this library's): the scan has compiled variants of (queries per
 * CTA tile, dictionary entries per thread) -- (8, 4), (8, 2), (16, 2), (4, 4),
 * (4, 8), (16, 4), (32, 2) -- that compute the same FP32 cost of every (query, entry) pair and
 * so give the same picks and costs.  sfc_tune_tiles times fullscan_query_batch
 * (precision SFC_FP32; same arguments as there) with each shape (median of
 * reps timed calls after one untimed, CUDA events on `stream`), checks that
 * every shape returns shape 0's picks and cost bits (SFC_EDEVICE if not), and
 * makes the fastest the shape of every later FP32 full scan in this process.
 * table: HOST double [7][3] (queries per tile, entries per thread, ms) or NULL;
 * chosen: the shape taken, or NULL.  sfc_tile_shape(shape) sets the shape
 * (0..6; any other value only reads it) and returns the one in use.
 * fullscan_query_batch_static always takes shape 0 (its scratch is sized for
 * it). */
int sfc_tune_tiles(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                   const sfc_params* p, const int32_t* centres, int64_t Q, int32_t reps, double* table,
                   int32_t* chosen, void* stream);
int32_t sfc_tile_shape(int32_t shape);

/* ---- Failure injection for tests ------------------------------------------
 * The paper has no counterpart: these hooks let tests drive the library's
 * failure paths without faulting the GPU.
 *
 * sfc_debug_fail_alloc(n): the n-th library device allocation from now on
 * fails as if the device were out of memory (n <= 0: off); the entry point
 * that made it returns SFC_ENOMEM and releases everything it had taken.
 * sfc_debug_alloc_count(): library device allocations made so far (process).
 * sfc_debug_pool_used(bytes): synchronises the device, then *bytes (host) = the
 * bytes currently allocated from the library's memory pool on this device.
 * sfc_debug_lookback(spin_limit, stall): the radix sort's decoupled look-back
 * gives up after spin_limit polls (<= 0: the default 2^24), and with stall = 1
 * every look-back polls a word nothing writes -- so every sort tile after the
 * first gives up, the sort's output is garbage and sfc_status() reports
 * SFC_ETIMEOUT (writes stay inside the output arrays; the GPU stays usable).
 * Reset with sfc_debug_lookback(0, 0).
 * sfc_debug_sort(force_lsd, bucket_cap): index builds with up to 2^20
 * dictionary entries sort each index by a sample sort; force_lsd = 1 makes them
 * take the LSD radix sort (the one the look-back hook above acts on), and
 * bucket_cap in 1..4095 lowers the sample sort's bucket capacity so that an
 * index whose largest bucket exceeds it is sorted again by the LSD sort (its
 * fallback path).  Same sorted arrays either way.  Reset with (0, 0). */
int sfc_debug_fail_alloc(int64_t n);
int64_t sfc_debug_alloc_count(void);
int sfc_debug_pool_used(uint64_t* bytes);
int sfc_debug_lookback(int64_t spin_limit, int32_t stall);
int sfc_debug_sort(int32_t force_lsd, int32_t bucket_cap);

/* Message of the last failed call on this host thread ("" if none). */
const char* sfc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SFC_H */
