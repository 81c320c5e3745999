// sfc_tune.cu -- search over the index parameters (C, D, W) for one batch of
// queries.  Host code only: every build, query and full scan goes through the
// library's own entry points, so the search runs the same kernels as a user.
//
// The quality measure is the acceleration error of Sec. III.C: per query the L2
// norm of the SFC pick's difference over the L2 norm of the exact pick's, minus
// one, averaged over a sample of the queries.  The exact picks are those of the
// full scan (Sec. I), whose picks equal the definition's.
#include <algorithm>
#include <cstring>
#include <cmath>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace sfc;

namespace {

double finite_or_inf(double v) { return std::isnan(v) ? INFINITY : v; }

// Per-query acceleration error from FP32 costs (squared norms): 0 when the two
// costs are equal, sqrt(c) / sqrt(c_exact) - 1 when the exact cost is positive,
// and 1 when the exact cost is 0 but the SFC pick's is not.
double query_error(float c, float c_exact) {
  if (c == c_exact) return 0.0;
  if (!(c_exact > 0.0f)) return 1.0;
  return std::sqrt((double)c) / std::sqrt((double)c_exact) - 1.0;
}

struct Events {
  cudaEvent_t e[3] = {};
  ~Events() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

}  // namespace

extern "C" {

int32_t sfc_tune_select(int32_t n, const double* ms, const double* ae, double ae_max) {
  if (n <= 0 || !ms || !ae) return -1;
  int32_t best = -1;
  for (int32_t i = 0; i < n; ++i)
    if (ae[i] <= ae_max && (best < 0 || finite_or_inf(ms[i]) < finite_or_inf(ms[best]))) best = i;
  if (best >= 0) return best;
  for (int32_t i = 0; i < n; ++i) {
    if (best < 0) {
      best = i;
      continue;
    }
    const double a = finite_or_inf(ae[i]), b = finite_or_inf(ae[best]);
    if (a < b || (a == b && finite_or_inf(ms[i]) < finite_or_inf(ms[best]))) best = i;
  }
  return best;
}

int sfc_autotune(const float* grid, const uint8_t* mask, const sfc_grid* g, const sfc_params* base,
                 const int32_t* centres, int64_t Q, const sfc_tune_spec* spec, sfc_params* best, double* table,
                 int32_t* chosen, void* stream) {
  if (!grid || !mask || !g || !base || !centres || !spec || !best || Q < 1) {
    set_error("sfc_autotune: NULL argument or Q < 1");
    return SFC_EINVAL;
  }
  if (!spec->curves || !spec->dims || !spec->windows || spec->n_curves < 1 || spec->n_dims < 1 ||
      spec->n_windows < 1 || spec->sample < 1 || spec->reps < 1 || spec->reps > 100 ||
      (spec->objective != SFC_TUNE_STEP && spec->objective != SFC_TUNE_QUERY) || !(spec->ae_max >= 0.0)) {
    set_error("sfc_autotune: invalid spec (empty lists, sample < 1, reps 1..100, objective, ae_max >= 0)");
    return SFC_EINVAL;
  }
  const int64_t n_cfg = (int64_t)spec->n_curves * spec->n_dims * spec->n_windows;
  if (n_cfg > 4096) {
    set_error("sfc_autotune: more than 4096 configurations");
    return SFC_EINVAL;
  }
  if (base->shifts || base->basis || base->mean) {
    set_error("sfc_autotune: shifts and imported bases are sized for one (C, D); pass NULL");
    return SFC_EINVAL;
  }
  if (g->ndim != 2 && g->ndim != 3) {
    set_error("sfc_autotune: ndim must be 2 or 3");
    return SFC_EINVAL;
  }
  SFC_CHECK(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  const int ndim = g->ndim;

  // the sample: every step-th query
  const int64_t S0 = std::min<int64_t>(spec->sample, Q);
  const int64_t step = (Q + S0 - 1) / S0;
  std::vector<int32_t> all((size_t)Q * ndim);
  SFC_TRY(cudaMemcpyAsync(all.data(), centres, sizeof(int32_t) * all.size(), cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  std::vector<int64_t> rows;
  for (int64_t i = 0; i < Q; i += step) rows.push_back(i);
  const int64_t S = (int64_t)rows.size();
  std::vector<int32_t> samp((size_t)S * ndim);
  for (int64_t k = 0; k < S; ++k)
    for (int a = 0; a < ndim; ++a) samp[(size_t)k * ndim + a] = all[(size_t)rows[k] * ndim + a];

  DevBuf d_samp, d_spick, d_scost, d_pick, d_cost;
  SFC_TRY(cudaMalloc(&d_samp.p, sizeof(int32_t) * samp.size()));
  SFC_TRY(cudaMalloc(&d_spick.p, sizeof(int64_t) * S));
  SFC_TRY(cudaMalloc(&d_scost.p, sizeof(float) * S));
  SFC_TRY(cudaMalloc(&d_pick.p, sizeof(int64_t) * Q));
  SFC_TRY(cudaMalloc(&d_cost.p, sizeof(float) * Q));
  SFC_TRY(cudaMemcpyAsync(d_samp.p, samp.data(), sizeof(int32_t) * samp.size(), cudaMemcpyHostToDevice, st));

  // exact picks of the sample (tensor-core pre-score for the L2 cost)
  sfc_params fp = *base;
  fp.precision = base->cost == SFC_COST_L2 ? SFC_FP16 : SFC_FP32;
  SFC_CHECK(fullscan_query_batch(grid, mask, mask, g, &fp, (const int32_t*)d_samp.p, S, (int64_t*)d_spick.p,
                                 (float*)d_scost.p, stream));
  std::vector<float> exact(S), cost(Q);
  SFC_TRY(cudaMemcpyAsync(exact.data(), d_scost.p, sizeof(float) * S, cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));

  Events ev;
  for (auto& e : ev.e) SFC_TRY(cudaEventCreate(&e));
  std::vector<double> ms_all(n_cfg), ae_all(n_cfg);
  std::vector<sfc_params> cfg(n_cfg);
  int64_t c_i = 0;
  for (int32_t ic = 0; ic < spec->n_curves; ++ic)
    for (int32_t id = 0; id < spec->n_dims; ++id)
      for (int32_t iw = 0; iw < spec->n_windows; ++iw, ++c_i) {
        sfc_params p = *base;
        p.curves = spec->curves[ic];
        p.dims = spec->dims[id];
        if (base->knn > 0)
          p.knn = spec->windows[iw];
        else
          p.window = spec->windows[iw];
        cfg[c_i] = p;
        std::vector<double> t;
        for (int r = 0; r <= spec->reps; ++r) {  // r = 0 warms up, untimed
          sfc_index* ix = nullptr;
          SFC_TRY(cudaEventRecord(ev.e[0], st));
          int rc = sfc_index_build(grid, mask, g, &p, stream, &ix);
          if (rc != SFC_OK) {
            set_error("sfc_autotune: configuration (C " + std::to_string(p.curves) + ", D " +
                      std::to_string(p.dims) + ", W/k " + std::to_string(spec->windows[iw]) +
                      "): " + sfc_last_error());
            return rc;
          }
          cudaEventRecord(ev.e[1], st);
          rc = sfc_query_batch(ix, grid, mask, centres, Q, (int64_t*)d_pick.p, (float*)d_cost.p, stream);
          cudaEventRecord(ev.e[2], st);
          cudaError_t ce = cudaEventSynchronize(ev.e[2]);
          if (rc == SFC_OK && ce == cudaSuccess && r == spec->reps)
            ce = cudaMemcpy(cost.data(), d_cost.p, sizeof(float) * Q, cudaMemcpyDeviceToHost);
          sfc_index_destroy(ix);
          if (rc != SFC_OK) return rc;
          if (ce != cudaSuccess) {
            set_error(std::string("sfc_autotune: ") + cudaGetErrorString(ce));
            return SFC_ECUDA;
          }
          if (r > 0) {
            float v = 0.0f;
            cudaEventElapsedTime(&v, ev.e[spec->objective == SFC_TUNE_STEP ? 0 : 1], ev.e[2]);
            t.push_back(v);
          }
        }
        std::sort(t.begin(), t.end());
        ms_all[c_i] = t[t.size() / 2];
        double acc = 0.0;
        for (int64_t k = 0; k < S; ++k) acc += query_error(cost[rows[k]], exact[k]);
        ae_all[c_i] = acc / (double)S;
        if (table) {
          double* row = table + 5 * c_i;
          row[0] = p.curves;
          row[1] = p.dims;
          row[2] = spec->windows[iw];
          row[3] = ms_all[c_i];
          row[4] = ae_all[c_i];
        }
      }
  const int32_t k = sfc_tune_select((int32_t)n_cfg, ms_all.data(), ae_all.data(), spec->ae_max);
  *best = cfg[k];
  if (chosen) *chosen = k;
  return SFC_OK;
}

int32_t sfc_tile_shape(int32_t shape) { return fullscan_tile_shape(shape); }

int sfc_tune_tiles(const float* grid, const uint8_t* dict_mask, const uint8_t* cur_mask, const sfc_grid* g,
                   const sfc_params* p, const int32_t* centres, int64_t Q, int32_t reps, double* table,
                   int32_t* chosen, void* stream) {
  if (!grid || !dict_mask || !cur_mask || !g || !p || !centres || Q < 1 || reps < 1 || reps > 100) {
    set_error("sfc_tune_tiles: NULL argument, Q < 1 or reps outside 1..100");
    return SFC_EINVAL;
  }
  if (p->precision != SFC_FP32) {
    set_error("sfc_tune_tiles: the tile shapes are the FP32 full scan's (precision SFC_FP32)");
    return SFC_EUNSUPPORTED;
  }
  SFC_CHECK(check_device());
  cudaStream_t st = (cudaStream_t)stream;
  int qt[8], ept[8];
  const int ns = fullscan_tile_shapes(qt, ept);
  const int prev = fullscan_tile_shape(-1);
  DevBuf d_pick, d_cost;
  SFC_TRY(cudaMalloc(&d_pick.p, sizeof(int64_t) * Q));
  SFC_TRY(cudaMalloc(&d_cost.p, sizeof(float) * Q));
  std::vector<int64_t> pick0(Q), pk(Q);
  std::vector<float> cost0(Q), cs(Q);
  Events ev;
  for (auto& e : ev.e) SFC_TRY(cudaEventCreate(&e));
  std::vector<double> ms(ns);
  int rc = SFC_OK;
  for (int k = 0; k < ns && rc == SFC_OK; ++k) {
    fullscan_tile_shape(k);
    std::vector<double> t;
    for (int r = 0; r <= reps && rc == SFC_OK; ++r) {  // r = 0 warms up, untimed
      cudaEventRecord(ev.e[0], st);
      rc = fullscan_query_batch(grid, dict_mask, cur_mask, g, p, centres, Q, (int64_t*)d_pick.p, (float*)d_cost.p,
                                stream);
      cudaEventRecord(ev.e[1], st);
      if (rc == SFC_OK && cudaEventSynchronize(ev.e[1]) != cudaSuccess) rc = SFC_ECUDA;
      float v = 0.0f;
      if (rc == SFC_OK && r > 0 && cudaEventElapsedTime(&v, ev.e[0], ev.e[1]) == cudaSuccess) t.push_back(v);
    }
    if (rc != SFC_OK) break;
    std::sort(t.begin(), t.end());
    ms[k] = t[t.size() / 2];
    // every shape must give the same picks and cost bits
    if (cudaMemcpy(k == 0 ? pick0.data() : pk.data(), d_pick.p, sizeof(int64_t) * Q, cudaMemcpyDeviceToHost) !=
            cudaSuccess ||
        cudaMemcpy(k == 0 ? cost0.data() : cs.data(), d_cost.p, sizeof(float) * Q, cudaMemcpyDeviceToHost) !=
            cudaSuccess) {
      rc = SFC_ECUDA;
      break;
    }
    if (k > 0 && (pk != pick0 || std::memcmp(cs.data(), cost0.data(), sizeof(float) * Q) != 0)) {
      set_error("sfc_tune_tiles: tile shape " + std::to_string(k) + " gave other picks or costs than shape 0");
      rc = SFC_EDEVICE;
    }
  }
  if (rc != SFC_OK) {
    fullscan_tile_shape(prev);
    return rc;
  }
  int best = 0;
  for (int k = 1; k < ns; ++k)
    if (ms[k] < ms[best]) best = k;
  fullscan_tile_shape(best);
  if (table)
    for (int k = 0; k < ns; ++k) {
      table[3 * k + 0] = qt[k];
      table[3 * k + 1] = ept[k];
      table[3 * k + 2] = ms[k];
    }
  if (chosen) *chosen = best;
  return SFC_OK;
}

}  // extern "C"
