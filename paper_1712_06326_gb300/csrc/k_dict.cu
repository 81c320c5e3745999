// k_dict.cu -- dictionary extraction (Sec. I: the dictionary is the set of fully
// known patches).  A centre qualifies when its K^dim box lies inside the grid and
// every pixel of the box is known.  The test is a separable minimum filter of the
// mask (one pass per axis, each pixel reads 2r+1 bytes), followed by a stream
// compaction that keeps raster order, so dictionary ids are ranks in raster order.
#include "internal.cuh"

namespace sfc {

// ok[p] = all(in[p + t*stride_axis] for t in [-r, r]) and the whole window lies
// inside the axis extent.  `coord` extracts the coordinate along the axis.
__global__ void k_window_all(const uint8_t* __restrict__ in, uint8_t* __restrict__ out, int64_t npix, int64_t X,
                             int64_t Y, int axis, int64_t ext, int r) {
  int64_t stride = axis == 0 ? 1 : (axis == 1 ? X : X * Y);
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < npix; p += (int64_t)gridDim.x * blockDim.x) {
    int64_t c = axis == 0 ? p % X : (axis == 1 ? (p / X) % Y : p / (X * Y));
    uint8_t ok = 0;
    if (c >= r && c <= ext - 1 - r) {
      ok = 1;
      for (int t = -r; t <= r; ++t)
        if (!in[p + t * stride]) {
          ok = 0;
          break;
        }
    }
    out[p] = ok;
  }
}

// Stream compaction in raster order: 3 phases over tiles of kTile pixels.
constexpr int kTile = 2048;

__global__ void k_tile_count(const uint8_t* __restrict__ flag, int64_t npix, uint32_t* __restrict__ counts) {
  __shared__ uint32_t wsum[32];
  int64_t base = (int64_t)blockIdx.x * kTile;
  uint32_t c = 0;
  for (int i = threadIdx.x; i < kTile; i += blockDim.x) {
    int64_t p = base + i;
    c += (p < npix && flag[p]) ? 1u : 0u;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += wsum[w];
    counts[blockIdx.x] = t;
  }
}

// Single-block exclusive scan of the tile counts (in place) + total.
__global__ void k_scan_counts(uint32_t* __restrict__ counts, int64_t ntiles, int64_t* __restrict__ total) {
  __shared__ uint32_t part[1024];
  // each thread scans a contiguous chunk sequentially, then the chunk sums are scanned
  int64_t chunk = (ntiles + blockDim.x - 1) / blockDim.x;
  int64_t b = threadIdx.x * chunk, e = b + chunk < ntiles ? b + chunk : ntiles;
  uint32_t s = 0;
  for (int64_t i = b; i < e; ++i) s += counts[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t run = 0;
    for (int i = 0; i < (int)blockDim.x; ++i) {
      uint32_t v = part[i];
      part[i] = run;
      run += v;
    }
    *total = run;
  }
  __syncthreads();
  uint32_t run = part[threadIdx.x];
  for (int64_t i = b; i < e; ++i) {
    uint32_t v = counts[i];
    counts[i] = run;
    run += v;
  }
}

// Write the linear indices of flagged pixels at their raster rank.
__global__ void k_tile_emit(const uint8_t* __restrict__ flag, int64_t npix, const uint32_t* __restrict__ offs,
                            uint32_t* __restrict__ out) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t run;
  int64_t base = (int64_t)blockIdx.x * kTile;
  if (threadIdx.x == 0) run = offs[blockIdx.x];
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < kTile; i0 += blockDim.x) {
    int64_t p = base + i0 + threadIdx.x;
    bool f = p < npix && flag[p];
    unsigned bal = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[warp] = __popc(bal);
    __syncthreads();
    uint32_t before = 0, tot = 0;
    for (int w = 0; w < nw; ++w) {
      uint32_t v = wsum[w];
      if (w < warp) before += v;
      tot += v;
    }
    if (f) out[run + before + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)p;
    __syncthreads();
    if (threadIdx.x == 0) run += tot;
    __syncthreads();
  }
}

// Returns N (synchronises the stream once to read it); *dict is allocated here
// with cudaMallocAsync on `st` (caller frees).  Pixels must number < 2^32.
int dict_extract(const uint8_t* mask, const Geo& g, cudaStream_t st, uint32_t** dict, int64_t* N) {
  const int64_t npix = g.X * g.Y * g.Z;
  uint8_t *a = nullptr, *b = nullptr;
  uint32_t* counts = nullptr;
  int64_t* dtotal = nullptr;
  const int64_t ntiles = (npix + kTile - 1) / kTile;
  *dict = nullptr;
  Scratch scr(st);
  SFC_TRY(scr.alloc(&a, npix));
  SFC_TRY(scr.alloc(&b, npix));
  SFC_TRY(scr.alloc(&counts, ntiles * sizeof(uint32_t)));
  SFC_TRY(scr.alloc(&dtotal, sizeof(int64_t)));
  int grid = (int)((npix + 255) / 256 < 152 * 64 ? (npix + 255) / 256 : 152 * 64);
  count_launch();
  k_window_all<<<grid, 256, 0, st>>>(mask, a, npix, g.X, g.Y, 0, g.X, g.r);
  count_launch();
  k_window_all<<<grid, 256, 0, st>>>(a, b, npix, g.X, g.Y, 1, g.Y, g.r);
  const uint8_t* flag = b;
  if (g.ndim == 3) {
    count_launch();
    k_window_all<<<grid, 256, 0, st>>>(b, a, npix, g.X, g.Y, 2, g.Z, g.r);
    flag = a;
  }
  count_launch();
  k_tile_count<<<(unsigned)ntiles, 256, 0, st>>>(flag, npix, counts);
  count_launch();
  k_scan_counts<<<1, 1024, 0, st>>>(counts, ntiles, dtotal);
  int64_t total = 0;
  SFC_TRY(cudaMemcpyAsync(&total, dtotal, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  uint32_t* out = nullptr;
  if (total > 0) {
    SFC_TRY(scr.alloc(&out, total * sizeof(uint32_t)));
    count_launch();
    k_tile_emit<<<(unsigned)ntiles, 256, 0, st>>>(flag, npix, counts, out);
  }
  SFC_TRY(cudaGetLastError());
  scr.keep(out);
  *dict = out;
  *N = total;
  return SFC_OK;
}

// The same extraction into caller-provided buffers (no allocation): a, b: npix
// bytes each; counts: ceil(npix / 2048) words; dtotal: one int64; out: room for
// every valid centre.  Synchronises `st` once to read N.
int dict_extract_into(const uint8_t* mask, const Geo& g, cudaStream_t st, uint8_t* a, uint8_t* b, uint32_t* counts,
                      int64_t* dtotal, uint32_t* out, int64_t* N) {
  const int64_t npix = g.X * g.Y * g.Z;
  const int64_t ntiles = (npix + kTile - 1) / kTile;
  int grid = (int)((npix + 255) / 256 < 152 * 64 ? (npix + 255) / 256 : 152 * 64);
  count_launch();
  k_window_all<<<grid, 256, 0, st>>>(mask, a, npix, g.X, g.Y, 0, g.X, g.r);
  count_launch();
  k_window_all<<<grid, 256, 0, st>>>(a, b, npix, g.X, g.Y, 1, g.Y, g.r);
  const uint8_t* flag = b;
  if (g.ndim == 3) {
    count_launch();
    k_window_all<<<grid, 256, 0, st>>>(b, a, npix, g.X, g.Y, 2, g.Z, g.r);
    flag = a;
  }
  count_launch();
  k_tile_count<<<(unsigned)ntiles, 256, 0, st>>>(flag, npix, counts);
  count_launch();
  k_scan_counts<<<1, 1024, 0, st>>>(counts, ntiles, dtotal);
  int64_t total = 0;
  SFC_TRY(cudaMemcpyAsync(&total, dtotal, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  SFC_TRY(cudaStreamSynchronize(st));
  if (total > 0) {
    count_launch();
    k_tile_emit<<<(unsigned)ntiles, 256, 0, st>>>(flag, npix, counts, out);
  }
  SFC_TRY(cudaGetLastError());
  *N = total;
  return SFC_OK;
}

}  // namespace sfc
