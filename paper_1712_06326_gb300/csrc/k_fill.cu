// k_fill.cu -- the exemplar-based inpainting loop (Sec. I; Fig. 1(a)) on the
// device.  Per step, without a host round trip:
//   k_prio    priorities of the candidate centres whose value can have changed
//             (the whole grid at the start, then the box of radius 2r+1 around the
//             last target: the patch changed mask/values/confidence within r,
//             which reaches front flags within r+1 and confidence sums within 2r);
//   k_argmax  packed max over (valid, priority bits, ~linear index): the highest
//             priority, ties to the lowest linear index;
//   k_select  decode the target (or mark the loop done);
//   search    full scan (k_fs_scan + k_fs_band, Q = 1) or SFC query (Q = 1);
//   k_insert  copy the source patch into the target's unknown pixels, mark them
//             known, give them the target's confidence term, log the step.
// Candidate centres: a known pixel with an unknown axis neighbour (4-/6-
// connected) is a front pixel; its centre is the pixel moved into the valid
// range [r, ext-1-r] per axis.  Priority (Criminisi et al.'s order, written out
// since the paper defers to it): confidence term Cterm = (sum of confidence over
// the patch, FP32 in raster order) / K^dim; CONFIDENCE: P = Cterm; CRIMINISI
// (2-D): P = Cterm * (|(-gy) nx + gx ny| + 0.001), grey-value gradient by central
// differences over known neighbours (one-sided if one side is unknown), n the
// normalised central-difference gradient of the known-mask (outside = known).
// Every product and sum is rounded separately (explicit _rn intrinsics).
#include "internal.cuh"

namespace sfc {

int fullscan_single(const Geo& g, const float* grid, const uint8_t* cur_mask, const uint32_t* dict, int64_t N,
                    const int* eoff_all, const float* weights, int cm, const int64_t* centre_lin,
                    int64_t* pick, float* cost, float* tilemin, unsigned int* gmin, cudaStream_t st);

namespace {

struct FillState {
  unsigned long long* key;  // npix packed priorities
  float* conf;              // npix confidence
  float* cterm;             // npix confidence term of candidate centres
  unsigned long long* best;
  int64_t* sel_lin;         // chosen centre (linear)
  int32_t* sel_xyz;         // chosen centre (x, y, z)
  float* sel_cterm;
  int64_t* pick;
  float* cost;
  int* done;
  int64_t* steps;
};

__device__ inline bool in_grid(const Geo& g, int64_t x, int64_t y, int64_t z) {
  return x >= 0 && y >= 0 && z >= 0 && x < g.X && y < g.Y && z < g.Z;
}

__device__ inline bool is_front(const Geo& g, const uint8_t* mask, int64_t x, int64_t y, int64_t z) {
  if (!mask[lin_of(g, x, y, z)]) return false;
  const int64_t nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z}, {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
  for (int a = 0; a < 2 * g.ndim; ++a)
    if (in_grid(g, nb[a][0], nb[a][1], nb[a][2]) && !mask[lin_of(g, nb[a][0], nb[a][1], nb[a][2])]) return true;
  return false;
}

__device__ inline float gray_at(const Geo& g, const float* grid, int64_t q) {
  if (g.ch == 1) return grid[q];
  float acc = grid[q * g.ch];
  for (int c = 1; c < g.ch; ++c) acc = __fadd_rn(acc, grid[q * g.ch + c]);
  return __fdiv_rn(acc, (float)g.ch);
}

// Priority of centre (x, y, z); writes key (0 = not a candidate) and cterm.
__device__ void prio_one(const Geo& g, const float* __restrict__ grid, const uint8_t* __restrict__ mask,
                         const float* __restrict__ conf, int prio, int64_t x, int64_t y, int64_t z,
                         unsigned long long* key, float* cterm) {
  const int64_t c = lin_of(g, x, y, z);
  if (!centre_ok(g, x, y, z)) {
    key[c] = 0ull;
    return;
  }
  // preimage of the clamping
  int64_t lo[3], hi[3];
  const int64_t cc[3] = {x, y, z}, ext[3] = {g.X, g.Y, g.Z};
  for (int a = 0; a < 3; ++a) {
    if (a >= g.ndim) {
      lo[a] = hi[a] = 0;
      continue;
    }
    lo[a] = cc[a] == g.r ? 0 : cc[a];
    hi[a] = cc[a] == ext[a] - 1 - g.r ? ext[a] - 1 : cc[a];
  }
  bool cand = false;
  for (int64_t pz = lo[2]; pz <= hi[2] && !cand; ++pz)
    for (int64_t py = lo[1]; py <= hi[1] && !cand; ++py)
      for (int64_t px = lo[0]; px <= hi[0] && !cand; ++px) cand = is_front(g, mask, px, py, pz);
  if (!cand) {
    key[c] = 0ull;
    return;
  }
  // the confidence sum in raster order, a patch row at a time (the row's loads
  // are independent of the running sum, so they are issued ahead of it)
  float sum = 0.0f;
  const int K = g.K, nz = g.ndim == 3 ? K : 1;
  for (int dz = 0; dz < nz; ++dz)
    for (int dy = 0; dy < K; ++dy) {
      const float* row = conf + c + ((int64_t)(g.ndim == 3 ? dz - g.r : 0) * g.Y + (dy - g.r)) * g.X - g.r;
      int dx = 0;
      for (; dx + 4 <= K; dx += 4) {
        const float a0 = row[dx], a1 = row[dx + 1], a2 = row[dx + 2], a3 = row[dx + 3];
        sum = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(sum, a0), a1), a2), a3);
      }
      for (; dx < K; ++dx) sum = __fadd_rn(sum, row[dx]);
    }
  const float Ct = __fdiv_rn(sum, (float)g.P);
  float P = Ct;
  if (prio == SFC_PRIO_CRIMINISI) {
    const bool kc = mask[c] != 0;
    float gxy[2];
    for (int a = 0; a < 2; ++a) {
      int64_t x0 = x - (a == 0), y0 = y - (a == 1), x1 = x + (a == 0), y1 = y + (a == 1);
      bool k0 = in_grid(g, x0, y0, 0) && mask[lin_of(g, x0, y0, 0)];
      bool k1 = in_grid(g, x1, y1, 0) && mask[lin_of(g, x1, y1, 0)];
      float gv = 0.0f;
      if (k0 && k1)
        gv = __fmul_rn(0.5f, __fsub_rn(gray_at(g, grid, lin_of(g, x1, y1, 0)), gray_at(g, grid, lin_of(g, x0, y0, 0))));
      else if (kc && k1)
        gv = __fsub_rn(gray_at(g, grid, lin_of(g, x1, y1, 0)), gray_at(g, grid, c));
      else if (kc && k0)
        gv = __fsub_rn(gray_at(g, grid, c), gray_at(g, grid, lin_of(g, x0, y0, 0)));
      gxy[a] = gv;
    }
    auto mval = [&](int64_t xx, int64_t yy) -> float {
      if (!in_grid(g, xx, yy, 0)) return 1.0f;
      return mask[lin_of(g, xx, yy, 0)] ? 1.0f : 0.0f;
    };
    float mx = __fmul_rn(0.5f, __fsub_rn(mval(x + 1, y), mval(x - 1, y)));
    float my = __fmul_rn(0.5f, __fsub_rn(mval(x, y + 1), mval(x, y - 1)));
    float nrm = __fsqrt_rn(__fadd_rn(__fmul_rn(mx, mx), __fmul_rn(my, my)));
    float nx = 0.0f, ny = 0.0f;
    if (nrm > 0.0f) {
      nx = __fdiv_rn(mx, nrm);
      ny = __fdiv_rn(my, nrm);
    }
    float t1 = __fmul_rn(-gxy[1], nx);
    float t2 = __fmul_rn(gxy[0], ny);
    float Dt = fabsf(__fadd_rn(t1, t2));
    P = __fmul_rn(Ct, __fadd_rn(Dt, 0.001f));
  }
  key[c] = (1ull << 63) | ((unsigned long long)__float_as_uint(P) << 32) | (unsigned long long)(0xffffffffu - (uint32_t)c);
  cterm[c] = Ct;
}

// Priorities of the whole grid (whole = 1) or of the box around the last
// target, by CTA bx of nbx (grid-stride).
__device__ void prio_body(const float* __restrict__ grid, const uint8_t* __restrict__ mask, const Geo& g, int prio,
                          const FillState& s, int whole, int bx, int nbx) {
  if (!whole && *s.done) return;
  int64_t bx0 = 0, by0 = 0, bz0 = 0, bnx = g.X, bny = g.Y, bnz = g.Z;
  if (!whole) {
    const int R = 2 * g.r + 1;
    const int64_t t = *s.sel_lin;
    const int64_t tx = t % g.X, ty = (t / g.X) % g.Y, tz = t / (g.X * g.Y);
    bx0 = tx - R;
    by0 = ty - R;
    bz0 = g.ndim == 3 ? tz - R : 0;
    bnx = 2 * R + 1;
    bny = 2 * R + 1;
    bnz = g.ndim == 3 ? 2 * R + 1 : 1;
  }
  const int64_t total = bnx * bny * bnz;
  for (int64_t i = bx * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)nbx * blockDim.x) {
    int64_t x = bx0 + i % bnx, y = by0 + (i / bnx) % bny, z = bz0 + i / (bnx * bny);
    if (!in_grid(g, x, y, z)) continue;
    prio_one(g, grid, mask, s.conf, prio, x, y, z, s.key, s.cterm);
  }
}

__global__ void k_prio(const float* __restrict__ grid, const uint8_t* __restrict__ mask, Geo g, int prio,
                       FillState s, int whole) {
  prio_body(grid, mask, g, prio, s, whole, blockIdx.x, gridDim.x);
}

__global__ void k_argmax(const unsigned long long* __restrict__ key, int64_t npix, FillState s) {
  if (*s.done) return;
  unsigned long long m = 0ull;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long v = key[i];
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
    m = w > m ? w : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(s.best, m);
}

// The target of the highest packed priority b (0: no candidate left): marks
// the loop done, or decodes the centre.  Returns true if a target was taken.
__device__ bool select_apply(const Geo& g, const FillState& s, int64_t max_steps, unsigned long long b) {
  if (b == 0ull || (max_steps > 0 && *s.steps >= max_steps)) {
    *s.done = 1;
    return false;
  }
  const int64_t c = (int64_t)(0xffffffffu - (uint32_t)(b & 0xffffffffull));
  *s.sel_lin = c;
  s.sel_xyz[0] = (int32_t)(c % g.X);
  s.sel_xyz[1] = (int32_t)((c / g.X) % g.Y);
  s.sel_xyz[2] = (int32_t)(c / (g.X * g.Y));
  *s.sel_cterm = s.cterm[c];
  return true;
}

__global__ void k_select(Geo g, FillState s, int64_t max_steps) {
  if (*s.done) return;
  const unsigned long long b = *s.best;
  *s.best = 0ull;
  select_apply(g, s, max_steps, b);
}

__device__ void insert_body(float* __restrict__ grid, uint8_t* __restrict__ mask, const Geo& g,
                            const uint32_t* __restrict__ dict, const FillState& s, int64_t* __restrict__ log,
                            int64_t log_cap, int64_t* __restrict__ unknown_left, uint32_t* __restrict__ status) {
  if (*s.done) return;
  const int64_t t = *s.sel_lin;
  const int64_t j = *s.pick;
  if (j < 0) {
    if (threadIdx.x == 0) *s.done = 1;
    return;
  }
  const int64_t src = dict[j];
  const float ct = *s.sel_cterm;
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  int mine = 0;
  for (int pp = threadIdx.x; pp < g.P; pp += blockDim.x) {
    const int64_t off = patch_off(g, pp);
    const int64_t qt = t + off;
    if (mask[qt]) continue;
    const int64_t qs = src + off;
    for (int c = 0; c < g.ch; ++c) grid[qt * g.ch + c] = grid[qs * g.ch + c];
    mask[qt] = 1;
    s.conf[qt] = ct;
    ++mine;
  }
  atomicAdd(&cnt, mine);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int64_t k = *s.steps;
    if (cnt == 0) {  // every step fills at least one pixel; stop rather than spin
      atomicOr(status, ST_OVERFLOW);
      *s.done = 1;
      return;
    }
    if (log && k < log_cap) {
      log[k * (g.ndim + 1) + 0] = s.sel_xyz[0];
      log[k * (g.ndim + 1) + 1] = s.sel_xyz[1];
      if (g.ndim == 3) log[k * (g.ndim + 1) + 2] = s.sel_xyz[2];
      log[k * (g.ndim + 1) + g.ndim] = j;
    }
    *s.steps = k + 1;
    *unknown_left -= cnt;
  }
}

__global__ void k_insert(float* __restrict__ grid, uint8_t* __restrict__ mask, Geo g, const uint32_t* __restrict__ dict,
                         FillState s, int64_t* __restrict__ log, int64_t log_cap, int64_t* __restrict__ unknown_left,
                         uint32_t* __restrict__ status) {
  insert_body(grid, mask, g, dict, s, log, log_cap, unknown_left, status);
}

__global__ void k_conf_init(const uint8_t* __restrict__ mask, int64_t npix, float* __restrict__ conf,
                            int64_t* __restrict__ unknown) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < npix) {
    conf[i] = mask[i] ? 1.0f : 0.0f;
    if (!mask[i]) atomicAdd((unsigned long long*)unknown, 1ull);
  }
}

__global__ void k_state_init(FillState s, Geo g) {
  *s.best = 0ull;
  *s.done = 0;
  *s.steps = 0;
  *s.sel_lin = lin_of(g, g.r, g.r, g.ndim == 3 ? g.r : 0);
  s.sel_xyz[0] = g.r;
  s.sel_xyz[1] = g.r;
  s.sel_xyz[2] = g.ndim == 3 ? g.r : 0;
  *s.sel_cterm = 0.0f;
  *s.pick = -1;
}

}  // namespace

// Runs the loop; `ix` is null in full-scan mode.  dict/N: the dictionary of the
// initial mask.  Synchronises `st` every chunk of steps to test for completion.
int fill_loop(const Geo& g, float* grid, uint8_t* mask, int prio, int mode, const Index* ix, const uint32_t* dict,
              int64_t N, const int* eoff_all, const float* weights, int cm, int64_t max_steps, int64_t* log,
              int64_t* steps_done, cudaStream_t st) {
  const int64_t npix = g.X * g.Y * g.Z;
  FillState s;
  int64_t* unknown = nullptr;
  float* tilemin = nullptr;
  unsigned int* gmin = nullptr;
  const int64_t ntiles = (N + 1023) / 1024;
  Scratch scr(st);  // the loop's state, freed on every return
  SFC_TRY(scr.alloc(&s.key, sizeof(unsigned long long) * npix));
  SFC_TRY(scr.alloc(&s.conf, sizeof(float) * npix));
  SFC_TRY(scr.alloc(&s.cterm, sizeof(float) * npix));
  SFC_TRY(scr.alloc(&s.best, sizeof(unsigned long long)));
  SFC_TRY(scr.alloc(&s.sel_lin, sizeof(int64_t)));
  SFC_TRY(scr.alloc(&s.sel_xyz, sizeof(int32_t) * 4));
  SFC_TRY(scr.alloc(&s.sel_cterm, sizeof(float)));
  SFC_TRY(scr.alloc(&s.pick, sizeof(int64_t)));
  SFC_TRY(scr.alloc(&s.cost, sizeof(float)));
  SFC_TRY(scr.alloc(&s.done, sizeof(int)));
  SFC_TRY(scr.alloc(&s.steps, sizeof(int64_t)));
  SFC_TRY(scr.alloc(&unknown, sizeof(int64_t)));
  SFC_TRY(scr.alloc(&tilemin, sizeof(float) * (ntiles > 0 ? ntiles : 1)));
  SFC_TRY(scr.alloc(&gmin, sizeof(unsigned int)));
  QSplit qs;  // the search's buffers (SFC mode): the split form of one query
  if (mode == SFC_MODE_SFC && ix) {
    qs.cap = query_split_cap(*ix);
    qs.qmax = 1;
    SFC_TRY(scr.alloc(&qs.cand, sizeof(int32_t) * qs.cap));
    SFC_TRY(scr.alloc(&qs.ncand, sizeof(int32_t)));
    SFC_TRY(scr.alloc(&qs.c32, sizeof(float) * qs.cap));
  }
  SFC_TRY(cudaMemsetAsync(unknown, 0, sizeof(int64_t), st));
  SFC_TRY(cudaMemsetAsync(s.key, 0, sizeof(unsigned long long) * npix, st));
  SFC_TRY(cudaMemsetAsync(s.cterm, 0, sizeof(float) * npix, st));
  count_launch();
  k_state_init<<<1, 1, 0, st>>>(s, g);
  count_launch();
  k_conf_init<<<(unsigned)((npix + 255) / 256), 256, 0, st>>>(mask, npix, s.conf, unknown);
  int pg = (int)((npix + 255) / 256 < 152 * 16 ? (npix + 255) / 256 : 152 * 16);
  count_launch();
  k_prio<<<pg, 256, 0, st>>>(grid, mask, g, prio, s, 1);
  SFC_TRY(cudaGetLastError());
  const int R = 2 * g.r + 1;
  const int64_t box = (int64_t)(2 * R + 1) * (2 * R + 1) * (g.ndim == 3 ? 2 * R + 1 : 1);
  const int bg = (int)((box + 255) / 256);
  const int ag = (int)((npix + 255) / 256 < 152 * 8 ? (npix + 255) / 256 : 152 * 8);
  int64_t left = 0;
  SFC_TRY(cudaMemcpyAsync(&left, unknown, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  if (left > 0 && N <= 0) {
    set_error("inpaint_run: the dictionary is empty but pixels are unknown");
    return SFC_EINVAL;
  }
  // every step fills >= 1 unknown pixel, so `left` steps always suffice
  const int64_t log_cap = max_steps > 0 ? (max_steps < left ? max_steps : left) : left;
  // One step: the priorities around the last insert (the first step has the
  // whole map just computed), the target, the search, the insert.
  auto step = [&](bool update) -> int {
    if (update) {
      count_launch();
      k_prio<<<bg, 256, 0, st>>>(grid, mask, g, prio, s, 0);
    }
    count_launch();
    k_argmax<<<ag, 256, 0, st>>>(s.key, npix, s);
    count_launch();
    k_select<<<1, 1, 0, st>>>(g, s, max_steps);
    const int r = mode == SFC_MODE_SFC
                      ? query_batch(*ix, grid, mask, s.sel_xyz, 1, s.pick, s.cost, nullptr, nullptr, nullptr, nullptr,
                                    st, nullptr, &qs)
                      : fullscan_single(g, grid, mask, dict, N, eoff_all, weights, cm, s.sel_lin, s.pick, s.cost,
                                        tilemin, gmin, st);
    if (r != SFC_OK) return r;
    count_launch();
    k_insert<<<1, 256, 0, st>>>(grid, mask, g, dict, s, log, log_cap, unknown, status_word());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("inpaint_run: ") + cudaGetErrorString(e));
      return SFC_ECUDA;
    }
    return SFC_OK;
  };
  // After the first step (eager), the loop runs as a CUDA graph of kGraphSteps
  // steps replayed between completion checks: every kernel of a step reads its
  // inputs from device state and returns at once after the last step, so a
  // replay past the end does nothing but a search on the last target.  If the
  // capture cannot be made, the same steps are enqueued one by one.
  constexpr int kGraphSteps = 8;
  struct GraphHold {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    ~GraphHold() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
    }
  } gh;
  int64_t enqueued = 0;
  int done = 0;
  int rc = step(false);
  ++enqueued;
  bool graph_ok = false;
  uint64_t per_graph = 0;
  // The steps run on the library's own stream (a capture needs a stream other
  // than the legacy default one), ordered after `st` by an event and joined
  // back into it at the end.
  // (joined on every return, before the scratch guard frees on `st`)
  struct Join {
    cudaStream_t caller = nullptr, own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ~Join() {
      if (own && ev_out && cudaEventRecord(ev_out, own) == cudaSuccess) cudaStreamWaitEvent(caller, ev_out, 0);
      if (ev_in) cudaEventDestroy(ev_in);
      if (ev_out) cudaEventDestroy(ev_out);
    }
  } jn;
  const cudaStream_t caller = st;
  jn.caller = st;
  if (cudaStream_t own = aux_stream(0)) {
    if (cudaEventCreateWithFlags(&jn.ev_in, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&jn.ev_out, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(jn.ev_in, caller) == cudaSuccess && cudaStreamWaitEvent(own, jn.ev_in, 0) == cudaSuccess) {
      jn.own = own;
      st = own;
    }
  }
  cudaGetLastError();
  if (rc == SFC_OK && st != caller) {
    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) cudaGetLastError();
    else {
    const uint64_t l0 = sfc_launch_count();
    int r = SFC_OK;
    for (int k = 0; k < kGraphSteps && r == SFC_OK; ++k) r = step(true);
    const cudaError_t e = cudaStreamEndCapture(st, &gh.g);
    per_graph = sfc_launch_count() - l0;
    count_launches(-(int64_t)per_graph);  // captured, not run yet
    graph_ok = r == SFC_OK && e == cudaSuccess && gh.g && cudaGraphInstantiate(&gh.x, gh.g, 0) == cudaSuccess;
    if (!graph_ok) {
      cudaGetLastError();
      set_error("");
    }
    }
  }
  int reps = 1;
  while (!done && rc == SFC_OK) {
    for (int k = 0; k < reps && rc == SFC_OK; ++k) {
      if (graph_ok) {
        SFC_TRY(cudaGraphLaunch(gh.x, st));
        count_launches((int64_t)per_graph);
        enqueued += kGraphSteps;
      } else {
        for (int u = 0; u < kGraphSteps && rc == SFC_OK; ++u, ++enqueued) rc = step(true);
      }
    }
    if (rc != SFC_OK) break;
    SFC_TRY(cudaMemcpyAsync(&done, s.done, sizeof(int), cudaMemcpyDeviceToHost, st));
    SFC_TRY(cudaStreamSynchronize(st));
    if (reps < 32) reps *= 2;
    if (!done && enqueued > left + kGraphSteps) {
      set_error("inpaint_run: the loop did not finish within one step per unknown pixel");
      rc = SFC_EDEVICE;
    }
  }
  if (jn.own) {  // join the caller's stream now (the rest runs on it)
    if (cudaEventRecord(jn.ev_out, jn.own) == cudaSuccess) cudaStreamWaitEvent(caller, jn.ev_out, 0);
    jn.own = nullptr;
    st = caller;
  }
  int64_t steps = 0;
  SFC_TRY(cudaMemcpyAsync(&steps, s.steps, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  *steps_done = steps;
  return rc;
}


// ---------------------------------------------------------------------------
// Many images at once (SFC mode): every round takes one step of every image
// whose loop is not done, in five launches for all images -- priorities of
// the boxes around the last targets, the maxima of the 1,024-pixel tiles those
// boxes touch, each image's target from its tile maxima (one CTA per image),
// one multi-image query launch, the inserts.  Per image the steps are those
// of fill_loop (same priorities, same packed-key maximum, same search and
// decision), so each image ends as its own inpaint_run would leave it.
namespace {

constexpr int kTileShift = 10;  // pixels per priority tile: 1,024

struct FillImg {
  Geo g;
  float* grid;
  uint8_t* mask;
  FillState s;
  unsigned long long* tmax;  // max packed key per tile
  int64_t ntiles;
  const uint32_t* dict;
  int64_t* log;
  int64_t log_cap;
  int64_t* unknown;
  int32_t* cen;  // this image's query centre (ndim ints)
};

__global__ void k_m_init(const FillImg* __restrict__ im) {
  const FillImg& f = im[blockIdx.x];
  if (threadIdx.x == 0) {
    const Geo& g = f.g;
    *f.s.best = 0ull;
    *f.s.done = 0;
    *f.s.steps = 0;
    *f.s.sel_lin = lin_of(g, g.r, g.r, g.ndim == 3 ? g.r : 0);
    f.s.sel_xyz[0] = g.r;
    f.s.sel_xyz[1] = g.r;
    f.s.sel_xyz[2] = g.ndim == 3 ? g.r : 0;
    *f.s.sel_cterm = 0.0f;
    *f.s.pick = -1;
    *f.unknown = 0;
    for (int a = 0; a < g.ndim; ++a) f.cen[a] = g.r;  // a valid centre until the first target
  }
}

__global__ void k_m_conf(const FillImg* __restrict__ im) {
  const FillImg& f = im[blockIdx.y];
  const int64_t npix = f.g.X * f.g.Y * f.g.Z;
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const bool kn = f.mask[i] != 0;
    f.s.conf[i] = kn ? 1.0f : 0.0f;
    f.s.key[i] = 0ull;
    f.s.cterm[i] = 0.0f;
    cnt += kn ? 0 : 1;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if ((threadIdx.x & 31) == 0 && cnt) atomicAdd((unsigned long long*)f.unknown, cnt);
}

__global__ void k_m_prio(const FillImg* __restrict__ im, int prio, int whole) {
  const FillImg& f = im[blockIdx.y];
  prio_body(f.grid, f.mask, f.g, prio, f.s, whole, blockIdx.x, gridDim.x);
}

// Tile maxima: every tile (whole = 1), or the tiles of the rows of the box
// k_m_prio just updated; one warp per (row, first / last tile of its span).
__global__ void k_m_tiles(const FillImg* __restrict__ im, int whole) {
  const FillImg& f = im[blockIdx.y];
  const Geo& g = f.g;
  if (!whole && *f.s.done) return;
  const int lane = threadIdx.x & 31;
  const int64_t item = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int64_t npix = g.X * g.Y * g.Z;
  int64_t tile;
  if (whole) {
    if (item >= f.ntiles) return;
    tile = item;
  } else {
    const int R = 2 * g.r + 1;
    const int64_t t = *f.s.sel_lin;
    const int64_t tx = t % g.X, ty = (t / g.X) % g.Y, tz = t / (g.X * g.Y);
    const int64_t rows_y = 2 * R + 1, rows = g.ndim == 3 ? rows_y * rows_y : rows_y;
    const int64_t row = item >> 1;
    if (row >= rows) return;
    const int64_t y = ty - R + row % rows_y, z = g.ndim == 3 ? tz - R + row / rows_y : 0;
    if (y < 0 || y >= g.Y || z < 0 || z >= g.Z) return;
    const int64_t x0 = tx - R < 0 ? 0 : tx - R, x1 = tx + R > g.X - 1 ? g.X - 1 : tx + R;
    const int64_t t0 = lin_of(g, x0, y, z) >> kTileShift, t1 = lin_of(g, x1, y, z) >> kTileShift;
    if ((item & 1) && t1 == t0) return;
    tile = (item & 1) ? t1 : t0;
  }
  const int64_t p0 = tile << kTileShift;
  const int64_t p1 = p0 + (1 << kTileShift) < npix ? p0 + (1 << kTileShift) : npix;
  unsigned long long m = 0ull;
  for (int64_t i = p0 + lane; i < p1; i += 32) {
    const unsigned long long v = f.s.key[i];
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
    m = w > m ? w : m;
  }
  if (lane == 0) f.tmax[tile] = m;
}

// One CTA per image: the maximum over the tile maxima, then the target.
__global__ void k_m_select(const FillImg* __restrict__ im, int64_t max_steps) {
  const FillImg& f = im[blockIdx.x];
  if (*f.s.done) return;
  __shared__ unsigned long long red[32];
  unsigned long long m = 0ull;
  for (int64_t t = threadIdx.x; t < f.ntiles; t += blockDim.x) {
    const unsigned long long v = f.tmax[t];
    m = v > m ? v : m;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_xor_sync(0xffffffffu, m, o);
    m = w > m ? w : m;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = red[w] > m ? red[w] : m;
    m = red[0] > m ? red[0] : m;
    if (select_apply(f.g, f.s, max_steps, m))
      for (int a = 0; a < f.g.ndim; ++a) f.cen[a] = f.s.sel_xyz[a];
  }
}

__global__ void k_m_insert(const FillImg* __restrict__ im, uint32_t* __restrict__ status) {
  const FillImg& f = im[blockIdx.x];
  insert_body(f.grid, f.mask, f.g, f.dict, f.s, f.log, f.log_cap, f.unknown, status);
}

}  // namespace

int fill_loop_multi(const Index* const* ixs, float* const* grids, uint8_t* const* masks, int n, int prio,
                    int64_t max_steps, int64_t* const* logs, int64_t* steps_done, cudaStream_t st) {
  if (n < 1) return SFC_OK;
  MultiQuery* mq = nullptr;
  {
    std::vector<const float*> gr(grids, grids + n);
    std::vector<const uint8_t*> mk(masks, masks + n);
    SFC_CHECK(multi_query_create(ixs, gr.data(), mk.data(), n, st, &mq));
  }
  struct MqHold {
    MultiQuery* m;
    ~MqHold() { multi_query_destroy(m); }
  } mqh{mq};
  const int ndim = ixs[0]->g.ndim;
  // one allocation for every image's state
  std::vector<FillImg> h(n);
  std::vector<size_t> off_key(n), off_conf(n), off_ct(n), off_tm(n);
  auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
  size_t o = 0;
  int64_t max_ntiles = 0, max_npix = 0;
  for (int i = 0; i < n; ++i) {
    const Geo& g = ixs[i]->g;
    const int64_t npix = g.X * g.Y * g.Z;
    if (npix >= ((int64_t)1 << 32)) {
      set_error("inpaint_run_multi: an image of 2^32 or more pixels");
      return SFC_EINVAL;
    }
    const int64_t nt = (npix + (1 << kTileShift) - 1) >> kTileShift;
    max_ntiles = std::max(max_ntiles, nt);
    max_npix = std::max(max_npix, npix);
    off_key[i] = o;
    o += up(sizeof(unsigned long long) * npix);
    off_conf[i] = o;
    o += up(sizeof(float) * npix);
    off_ct[i] = o;
    o += up(sizeof(float) * npix);
    off_tm[i] = o;
    o += up(sizeof(unsigned long long) * nt);
  }
  // per image scalars: best, sel_lin, pick, steps, unknown (8 B); sel_xyz (4 x 4 B);
  // sel_cterm, cost (4 B); done (4 B); query centre (ndim x 4 B)
  const size_t o_best = o, o_sel = o_best + up(8 * n), o_pick = o_sel + up(8 * n), o_steps = o_pick + up(8 * n),
               o_unk = o_steps + up(8 * n), o_xyz = o_unk + up(8 * n), o_ct = o_xyz + up(16 * n),
               o_cost = o_ct + up(4 * n), o_done = o_cost + up(4 * n), o_cen = o_done + up(4 * n),
               o_img = o_cen + up(4 * (size_t)ndim * n), total = o_img + up(sizeof(FillImg) * n);
  Scratch scr(st);
  unsigned char* ws = nullptr;
  SFC_TRY(scr.alloc(&ws, total));
  for (int i = 0; i < n; ++i) {
    FillImg& f = h[i];
    f.g = ixs[i]->g;
    f.grid = grids[i];
    f.mask = masks[i];
    f.s.key = reinterpret_cast<unsigned long long*>(ws + off_key[i]);
    f.s.conf = reinterpret_cast<float*>(ws + off_conf[i]);
    f.s.cterm = reinterpret_cast<float*>(ws + off_ct[i]);
    f.tmax = reinterpret_cast<unsigned long long*>(ws + off_tm[i]);
    f.ntiles = (f.g.X * f.g.Y * f.g.Z + (1 << kTileShift) - 1) >> kTileShift;
    f.s.best = reinterpret_cast<unsigned long long*>(ws + o_best) + i;
    f.s.sel_lin = reinterpret_cast<int64_t*>(ws + o_sel) + i;
    f.s.pick = reinterpret_cast<int64_t*>(ws + o_pick) + i;
    f.s.steps = reinterpret_cast<int64_t*>(ws + o_steps) + i;
    f.unknown = reinterpret_cast<int64_t*>(ws + o_unk) + i;
    f.s.sel_xyz = reinterpret_cast<int32_t*>(ws + o_xyz) + 4 * i;
    f.s.sel_cterm = reinterpret_cast<float*>(ws + o_ct) + i;
    f.s.cost = reinterpret_cast<float*>(ws + o_cost) + i;
    f.s.done = reinterpret_cast<int*>(ws + o_done) + i;
    f.cen = reinterpret_cast<int32_t*>(ws + o_cen) + (size_t)ndim * i;
    f.dict = ixs[i]->dict;
    f.log = logs ? logs[i] : nullptr;
    f.log_cap = 0;
  }
  FillImg* d_img = reinterpret_cast<FillImg*>(ws + o_img);
  int32_t* img_of = nullptr;
  std::vector<int32_t> iota(n);
  for (int i = 0; i < n; ++i) iota[i] = i;
  SFC_TRY(scr.alloc(&img_of, sizeof(int32_t) * n));
  SFC_TRY(cudaMemcpyAsync(img_of, iota.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, st));
  SFC_TRY(cudaMemcpyAsync(d_img, h.data(), sizeof(FillImg) * n, cudaMemcpyHostToDevice, st));
  const unsigned pgx = (unsigned)std::min<int64_t>((max_npix + 255) / 256, 152 * 4);
  count_launch();
  k_m_init<<<n, 32, 0, st>>>(d_img);
  count_launch();
  k_m_conf<<<dim3(pgx, n), 256, 0, st>>>(d_img);
  count_launch();
  k_m_prio<<<dim3(pgx, n), 256, 0, st>>>(d_img, prio, 1);
  count_launch();
  k_m_tiles<<<dim3((unsigned)((max_ntiles + 7) / 8), n), 256, 0, st>>>(d_img, 1);
  SFC_TRY(cudaGetLastError());
  // unknown pixels per image: the log capacities and the bound on the rounds
  std::vector<int64_t> left(n);
  {
    std::vector<int64_t> u(n);
    SFC_TRY(cudaMemcpyAsync(u.data(), ws + o_unk, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
    SFC_TRY(cudaStreamSynchronize(st));
    left = u;
  }
  int64_t max_left = 0;
  for (int i = 0; i < n; ++i) {
    if (left[i] > 0 && ixs[i]->N <= 0) {
      set_error("inpaint_run_multi: image " + std::to_string(i) + " has unknown pixels but an empty dictionary");
      return SFC_EINVAL;
    }
    h[i].log_cap = max_steps > 0 ? std::min(max_steps, left[i]) : left[i];
    max_left = std::max(max_left, left[i]);
  }
  SFC_TRY(cudaMemcpyAsync(d_img, h.data(), sizeof(FillImg) * n, cudaMemcpyHostToDevice, st));
  const int R = 2 * ixs[0]->g.r + 1;
  const int64_t box = (int64_t)(2 * R + 1) * (2 * R + 1) * (ndim == 3 ? 2 * R + 1 : 1);
  const unsigned bg = (unsigned)((box + 255) / 256);
  const int64_t rows = (int64_t)(2 * R + 1) * (ndim == 3 ? 2 * R + 1 : 1);
  const unsigned tg = (unsigned)((2 * rows + 7) / 8);
  int64_t* pick_tab = reinterpret_cast<int64_t*>(ws + o_pick);
  float* cost_tab = reinterpret_cast<float*>(ws + o_cost);
  int32_t* cen = reinterpret_cast<int32_t*>(ws + o_cen);
  QSplit qs;  // a round's search in the split form when there are at most 32 images
  qs.cap = query_split_cap(*ixs[0]);
  qs.qmax = n;
  SFC_TRY(scr.alloc(&qs.cand, sizeof(int32_t) * qs.cap * n));
  SFC_TRY(scr.alloc(&qs.ncand, sizeof(int32_t) * n));
  SFC_TRY(scr.alloc(&qs.c32, sizeof(float) * qs.cap * n));
  auto round = [&](bool update) -> int {
    if (update) {
      count_launch();
      k_m_prio<<<dim3(bg, n), 256, 0, st>>>(d_img, prio, 0);
      count_launch();
      k_m_tiles<<<dim3(tg, n), 256, 0, st>>>(d_img, 0);
    }
    count_launch();
    k_m_select<<<n, 256, 0, st>>>(d_img, max_steps);
    SFC_CHECK(multi_query_run(mq, img_of, cen, n, pick_tab, cost_tab, st, &qs));
    count_launch();
    k_m_insert<<<n, 256, 0, st>>>(d_img, status_word());
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      set_error(std::string("inpaint_run_multi: ") + cudaGetErrorString(e));
      return SFC_ECUDA;
    }
    return SFC_OK;
  };
  // the rounds as in fill_loop: the first eager, then a graph of kGraphRounds
  // rounds on the library's stream, replayed between completion checks
  constexpr int kGraphRounds = 8;
  struct GraphHold {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    ~GraphHold() {
      if (x) cudaGraphExecDestroy(x);
      if (g) cudaGraphDestroy(g);
    }
  } gh;
  struct Join {
    cudaStream_t caller = nullptr, own = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    ~Join() {
      if (own && ev_out && cudaEventRecord(ev_out, own) == cudaSuccess) cudaStreamWaitEvent(caller, ev_out, 0);
      if (ev_in) cudaEventDestroy(ev_in);
      if (ev_out) cudaEventDestroy(ev_out);
    }
  } jn;
  int rc = round(false);
  int64_t enqueued = 1;
  const cudaStream_t caller = st;
  jn.caller = st;
  if (cudaStream_t own = aux_stream(0)) {
    if (cudaEventCreateWithFlags(&jn.ev_in, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&jn.ev_out, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventRecord(jn.ev_in, caller) == cudaSuccess && cudaStreamWaitEvent(own, jn.ev_in, 0) == cudaSuccess) {
      jn.own = own;
      st = own;
    }
  }
  cudaGetLastError();
  bool graph_ok = false;
  uint64_t per_graph = 0;
  if (rc == SFC_OK && st != caller && cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    const uint64_t l0 = sfc_launch_count();
    int r = SFC_OK;
    for (int k = 0; k < kGraphRounds && r == SFC_OK; ++k) r = round(true);
    const cudaError_t e = cudaStreamEndCapture(st, &gh.g);
    per_graph = sfc_launch_count() - l0;
    count_launches(-(int64_t)per_graph);
    graph_ok = r == SFC_OK && e == cudaSuccess && gh.g && cudaGraphInstantiate(&gh.x, gh.g, 0) == cudaSuccess;
    if (!graph_ok) {
      cudaGetLastError();
      set_error("");
    }
  } else {
    cudaGetLastError();
  }
  // completion: every image's done flag (an image also stops if a step fills nothing)
  std::vector<int> dflags(n, 0);
  int done = 0, reps = 1;
  while (done < n && rc == SFC_OK) {
    for (int k = 0; k < reps && rc == SFC_OK; ++k) {
      if (graph_ok) {
        SFC_TRY(cudaGraphLaunch(gh.x, st));
        count_launches((int64_t)per_graph);
        enqueued += kGraphRounds;
      } else {
        for (int u = 0; u < kGraphRounds && rc == SFC_OK; ++u, ++enqueued) rc = round(true);
      }
    }
    if (rc != SFC_OK) break;
    SFC_TRY(cudaMemcpyAsync(dflags.data(), ws + o_done, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
    SFC_TRY(cudaStreamSynchronize(st));
    done = 0;
    for (int v : dflags) done += v != 0;
    if (reps < 32) reps *= 2;
    if (done < n && enqueued > max_left + kGraphRounds) {
      set_error("inpaint_run_multi: the loops did not finish within one round per unknown pixel");
      rc = SFC_EDEVICE;
    }
  }
  if (jn.own) {
    if (cudaEventRecord(jn.ev_out, jn.own) == cudaSuccess) cudaStreamWaitEvent(caller, jn.ev_out, 0);
    jn.own = nullptr;
    st = caller;
  }
  SFC_TRY(cudaMemcpyAsync(steps_done, ws + o_steps, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  return rc;
}

}  // namespace sfc
