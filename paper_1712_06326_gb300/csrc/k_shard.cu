// k_shard.cu -- the full scan split over shards of the dictionary, for running
// one exact full scan (Sec. I: the cost of every dictionary patch, then the
// global minimum) on several GPUs.
//
// Shard s of S owns the dictionary ids [floor(s N / S), floor((s + 1) N / S)).
// The exact pick needs one exchange in the middle:
//   1. every shard scans its ids in FP32 and reports its per-query minimum
//      cost (float bits; costs are >= 0, so the bits order like the values);
//   2. the caller takes the minimum over the shards (an all-reduce-min);
//   3. every shard lists its entries inside the FP32 error band of that global
//      minimum and rescores them with the exact FP64 cost, reporting its own
//      (FP64 cost, id, FP32 cost) minimum;
//   4. the caller takes the (FP64 cost, id) minimum over the shards (an
//      all-gather of 20 bytes per query and shard): the pick and its FP32 cost.
// The band of step 3 is the single-GPU scan's band (same FP32 costs, same
// global minimum), so the picks and costs equal fullscan_query_batch's.
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace sfc;

struct sfc_shard {
  int device = 0;
  Geo g{};
  int cm = 0;
  const float* grid = nullptr;
  const uint8_t* cur_mask = nullptr;
  int64_t Q = 0, N = 0, j0 = 0, j1 = 0;
  uint32_t* dict = nullptr;   // the whole dictionary (N ids)
  int* eo = nullptr;          // patch element offsets
  float* w = nullptr;         // channel weights
  int64_t* lin = nullptr;     // Q centre linear indices
  uint8_t* bad = nullptr;     // Q invalid-centre flags
  float* tilemin = nullptr;   // Q * tiles of the shard
};

namespace {

void shard_free(sfc_shard* s) {
  if (!s) return;
  cudaDeviceSynchronize();
  for (void* p : {(void*)s->dict, (void*)s->eo, (void*)s->w, (void*)s->lin, (void*)s->bad, (void*)s->tilemin})
    if (p) cudaFreeAsync(p, nullptr);
  cudaStreamSynchronize(nullptr);
  delete s;
}

int shard_create(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* gp,
                 const sfc_params* p, const int32_t* centres, int64_t Q, int32_t shard, int32_t nshards,
                 cudaStream_t st, sfc_shard* s) {
  SFC_CHECK(make_geo(gp, p->K, &s->g));
  const Geo& g = s->g;
  std::vector<float> w(g.ch, 1.0f);
  bool weighted = false;
  for (int c = 0; c < g.ch; ++c) {
    if (p->ch_weights) w[c] = p->ch_weights[c];
    if (!(w[c] > 0.0f) || !std::isfinite(w[c])) {
      set_error("channel weights must be positive and finite");
      return SFC_EINVAL;
    }
    weighted |= w[c] != 1.0f;
  }
  if (p->cost != SFC_COST_L2 && p->cost != SFC_COST_L1) {
    set_error("cost must be SFC_COST_L2 or SFC_COST_L1");
    return SFC_EINVAL;
  }
  if (p->precision != SFC_FP32) {
    set_error("sfc_shard: the dictionary split runs the FP32 scan (precision must be SFC_FP32)");
    return SFC_EUNSUPPORTED;
  }
  s->cm = (weighted ? 1 : 0) | (p->cost == SFC_COST_L1 ? 2 : 0);
  s->grid = grid;
  s->cur_mask = cur_mask;
  s->Q = Q;
  SFC_CHECK(dict_extract(dict_mask, g, st, &s->dict, &s->N));
  if (s->N <= 0) {
    set_error("the dictionary is empty (no fully known patch)");
    return SFC_EINVAL;
  }
  s->j0 = s->N * shard / nshards;
  s->j1 = s->N * (shard + 1) / nshards;
  SFC_CHECK(upload_patch_tables(g, &s->eo, st));
  SFC_TRY(pmalloc(&s->w, sizeof(float) * g.ch, st));
  SFC_TRY(cudaMemcpyAsync(s->w, w.data(), sizeof(float) * g.ch, cudaMemcpyHostToDevice, st));
  const int64_t qa = Q > 0 ? Q : 1;
  SFC_TRY(pmalloc(&s->lin, sizeof(int64_t) * qa, st));
  SFC_TRY(pmalloc(&s->bad, qa, st));
  const int64_t nt = fullscan_range_tiles(s->j1 - s->j0);
  SFC_TRY(pmalloc(&s->tilemin, sizeof(float) * qa * (nt > 0 ? nt : 1), st));
  SFC_CHECK(centres_to_lin(g, centres, Q, s->lin, s->bad, st));
  return SFC_OK;
}

int shard_device(const sfc_shard* s) {
  int dev = -1;
  SFC_TRY(cudaGetDevice(&dev));
  if (dev != s->device) {
    set_error("sfc_shard: called on another device than the one it was created on");
    return SFC_EINVAL;
  }
  return SFC_OK;
}

}  // namespace

extern "C" {

int sfc_shard_create(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                     const sfc_params* p, const int32_t* centres, int64_t Q, int32_t shard, int32_t nshards,
                     void* stream, sfc_shard** out) {
  set_error("");
  if (!out) {
    set_error("sfc_shard_create: out is NULL");
    return SFC_EINVAL;
  }
  *out = nullptr;
  if (!grid || !dict_mask || !cur_mask || !p || (Q > 0 && !centres) || Q < 0) {
    set_error("sfc_shard_create: NULL pointer or negative Q");
    return SFC_EINVAL;
  }
  if (nshards < 1 || shard < 0 || shard >= nshards) {
    set_error("sfc_shard_create: need 0 <= shard < nshards");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  auto* s = new sfc_shard();
  cudaGetDevice(&s->device);
  const int rc = shard_create(grid, dict_mask, cur_mask, g, p, centres, Q, shard, nshards, (cudaStream_t)stream, s);
  if (rc != SFC_OK) {
    shard_free(s);
    return rc;
  }
  *out = s;
  return SFC_OK;
}

int sfc_shard_range(const sfc_shard* s, int64_t* N, int64_t* j0, int64_t* j1) {
  if (!s) {
    set_error("sfc_shard_range: NULL shard");
    return SFC_EINVAL;
  }
  if (N) *N = s->N;
  if (j0) *j0 = s->j0;
  if (j1) *j1 = s->j1;
  return SFC_OK;
}

int sfc_shard_scan(sfc_shard* s, uint32_t* min32, void* stream) {
  set_error("");
  if (!s || (s->Q > 0 && !min32)) {
    set_error("sfc_shard_scan: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(shard_device(s));
  return fullscan_range_scan(s->g, s->grid, s->cur_mask, s->dict + s->j0, s->j1 - s->j0, s->eo, s->w, s->cm, s->lin,
                             s->Q, s->tilemin, min32, (cudaStream_t)stream);
}

int sfc_shard_band(sfc_shard* s, const uint32_t* gmin32, double* cost64, int64_t* id, float* cost32,
                   void* stream) {
  set_error("");
  if (!s || (s->Q > 0 && (!gmin32 || !cost64 || !id || !cost32))) {
    set_error("sfc_shard_band: NULL pointer");
    return SFC_EINVAL;
  }
  SFC_CHECK(shard_device(s));
  return fullscan_range_band(s->g, s->grid, s->cur_mask, s->dict + s->j0, s->j1 - s->j0, s->eo, s->w, s->cm, s->lin,
                             s->Q, s->bad, s->tilemin, gmin32, s->j0, id, cost32, cost64, (cudaStream_t)stream);
}

int sfc_shard_destroy(sfc_shard* s) {
  if (!s) return SFC_OK;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(s->device);
  shard_free(s);
  cudaSetDevice(prev);
  return SFC_OK;
}

}  // extern "C"
