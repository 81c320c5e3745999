// k_pca.cu -- one PCA per index (Sec. II.A: a conventional PCA, the first D
// principal components are kept).
//
// Data of index c: the subset values (Fig. 2) of dictionary patches, s = m*ch per
// patch.  The covariance is accumulated in FP64 over a deterministic sample (ids
// 0, step, 2 step, ... with step = ceil(N / S)), the eigen-decomposition is the
// cyclic Jacobi method in FP64 with a parallel (round-robin) ordering: in every
// round the s/2 disjoint index pairs are rotated at once, A <- J^T A J and
// V <- V J, one launch per round, the matrix double-buffered so every launch
// reads the previous round's matrix only.  Sweeps stop when the off-diagonal
// norm falls below 1e-15 of the whole norm (checked after every sweep on the
// device; later launches then return at once).  Eigenvectors are ordered by
// descending eigenvalue (ties: lower column), signed so that the component of
// largest magnitude is positive (ties: lowest index), and rounded to FP32.
#include <cmath>

#include "internal.cuh"

namespace sfc {

namespace {

constexpr int kTile = 32;    // covariance tile (kTile x kTile outputs per CTA)
constexpr int kChunk = 32;   // samples staged per shared-memory step
constexpr int kMaxSweeps = 16;

// mean[c][i] = (1/S') sum_a x_{ids[a]}[i], FP64, fixed summation order.
__global__ void k_mean(const float* __restrict__ grid, const uint32_t* __restrict__ dict, int64_t step, int64_t cnt,
                       const int* __restrict__ sub_eoff, int s, int ch, double* __restrict__ mean) {
  const int c = blockIdx.y;
  const int i = blockIdx.x * 32 + (threadIdx.x & 31);
  const int lane_s = threadIdx.x >> 5;  // 8 sample lanes
  __shared__ double part[8][32];
  double acc = 0.0;
  if (i < s) {
    const int eo = sub_eoff[c * s + i];
    for (int64_t a = lane_s; a < cnt; a += 8) acc += (double)grid[(int64_t)dict[a * step] * ch + eo];
  }
  part[lane_s][threadIdx.x & 31] = acc;
  __syncthreads();
  if (lane_s == 0 && i < s) {
    double t = 0.0;
    for (int l = 0; l < 8; ++l) t += part[l][threadIdx.x];
    mean[c * s + i] = t / (double)cnt;
  }
}

// Partial covariance tile: rows [ti*32, +32) x cols [tj*32, +32) (tj >= ti) over
// the samples of one split.  partial layout [c][split][pair][32][32].
__global__ void k_cov_partial(const float* __restrict__ grid, const uint32_t* __restrict__ dict, int64_t step,
                              int64_t cnt, const int* __restrict__ sub_eoff, const double* __restrict__ mean, int s,
                              int ch, int nsplit, const int2* __restrict__ pairs, int npairs,
                              double* __restrict__ partial) {
  const int c = blockIdx.z, split = blockIdx.y, pr = blockIdx.x;
  const int2 tp = pairs[pr];
  const int i0 = tp.x * kTile, j0 = tp.y * kTile;
  __shared__ double xi[kChunk][kTile + 1];
  __shared__ double xj[kChunk][kTile + 1];
  __shared__ int eoi[kTile], eoj[kTile];
  __shared__ double mi[kTile], mj[kTile];
  if (threadIdx.x < kTile) {
    int i = i0 + threadIdx.x, j = j0 + threadIdx.x;
    eoi[threadIdx.x] = i < s ? sub_eoff[c * s + i] : 0;
    eoj[threadIdx.x] = j < s ? sub_eoff[c * s + j] : 0;
    mi[threadIdx.x] = i < s ? mean[c * s + i] : 0.0;
    mj[threadIdx.x] = j < s ? mean[c * s + j] : 0.0;
  }
  __syncthreads();
  const int64_t per = (cnt + nsplit - 1) / nsplit;
  const int64_t a0 = split * per, a1 = a0 + per < cnt ? a0 + per : cnt;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // 16x16 threads, 2x2 outputs each
  double acc[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (int64_t ab = a0; ab < a1; ab += kChunk) {
    for (int t = threadIdx.x; t < kChunk * kTile; t += blockDim.x) {
      int k = t / kTile, e = t % kTile;
      int64_t a = ab + k;
      double vi = 0.0, vj = 0.0;
      if (a < a1) {
        int64_t base = (int64_t)dict[a * step] * ch;
        if (i0 + e < s) vi = (double)grid[base + eoi[e]] - mi[e];
        if (j0 + e < s) vj = (double)grid[base + eoj[e]] - mj[e];
      }
      xi[k][e] = vi;
      xj[k][e] = vj;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < kChunk; ++k) {
      double a0v = xi[k][ty * 2], a1v = xi[k][ty * 2 + 1];
      double b0v = xj[k][tx * 2], b1v = xj[k][tx * 2 + 1];
      acc[0][0] = fma(a0v, b0v, acc[0][0]);
      acc[0][1] = fma(a0v, b1v, acc[0][1]);
      acc[1][0] = fma(a1v, b0v, acc[1][0]);
      acc[1][1] = fma(a1v, b1v, acc[1][1]);
    }
    __syncthreads();
  }
  double* out = partial + (((int64_t)c * nsplit + split) * npairs + pr) * kTile * kTile;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) out[(ty * 2 + a) * kTile + tx * 2 + b] = acc[a][b];
}

// A[c] (ns x ns, ns = s rounded up to even) = sum over splits / cnt, symmetric;
// padding rows/cols are zero.  V[c] = identity.
__global__ void k_cov_reduce(const double* __restrict__ partial, int nsplit, const int2* __restrict__ pairs,
                             int npairs, int64_t cnt, int s, int ns, double* __restrict__ A, double* __restrict__ V) {
  const int c = blockIdx.y;
  double* Ac = A + (int64_t)c * ns * ns;
  double* Vc = V + (int64_t)c * ns * ns;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)ns * ns;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / ns), j = (int)(t % ns);
    Vc[t] = i == j ? 1.0 : 0.0;
    double v = 0.0;
    if (i < s && j < s) {
      int a = i <= j ? i : j, b = i <= j ? j : i;
      int ti = a / kTile, tj = b / kTile;
      // pair index of (ti, tj) in the row-major upper-triangle enumeration
      int T = (s + kTile - 1) / kTile;
      int pr = ti * T - ti * (ti - 1) / 2 + (tj - ti);
      for (int sp = 0; sp < nsplit; ++sp)
        v += partial[(((int64_t)c * nsplit + sp) * npairs + pr) * kTile * kTile + (a - ti * kTile) * kTile +
                     (b - tj * kTile)];
      v = v / (double)cnt;
    }
    Ac[t] = v;
  }
}

// Round-robin pairing of round k over n (even) indices: pair 0 = (k, n-1),
// pair i >= 1 = ((k + i) mod (n-1), (k - i) mod (n-1)); every pair of indices
// meets exactly once in n-1 rounds.
__device__ inline void rr_pair(int k, int i, int n, int& p, int& q) {
  int a, b;
  if (i == 0) {
    a = k;
    b = n - 1;
  } else {
    a = (k + i) % (n - 1);
    b = ((k - i) % (n - 1) + (n - 1)) % (n - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// One parallel Jacobi round on every index: Anew = J^T Aold J, V <- V J.
__global__ void k_jacobi_round(const double* __restrict__ Aold, double* __restrict__ Anew, double* __restrict__ V,
                               int ns, int round, const int* __restrict__ done) {
  const int c = blockIdx.y;
  if (done[c]) {
    // keep the buffers in step: copy so the next round reads the same matrix
    const double* a = Aold + (int64_t)c * ns * ns;
    double* b = Anew + (int64_t)c * ns * ns;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)ns * ns;
         t += (int64_t)gridDim.x * blockDim.x)
      b[t] = a[t];
    return;
  }
  extern __shared__ unsigned char smem_raw[];
  double* al = reinterpret_cast<double*>(smem_raw);  // alpha[i] = J[i][i]
  double* be = al + ns;                               // beta[i]  = J[partner][i]
  int* pa = reinterpret_cast<int*>(be + ns);          // partner[i]
  const double* A = Aold + (int64_t)c * ns * ns;
  const int half = ns / 2;
  for (int i = threadIdx.x; i < half; i += blockDim.x) {
    int p, q;
    rr_pair(round, i, ns, p, q);
    double apq = A[(int64_t)p * ns + q];
    double cs = 1.0, sn = 0.0;
    if (apq != 0.0) {
      double app = A[(int64_t)p * ns + p], aqq = A[(int64_t)q * ns + q];
      double tau = (aqq - app) / (2.0 * apq);
      double t = tau >= 0.0 ? 1.0 / (tau + sqrt(1.0 + tau * tau)) : -1.0 / (-tau + sqrt(1.0 + tau * tau));
      cs = 1.0 / sqrt(1.0 + t * t);
      sn = t * cs;
    }
    // J[p][p] = c, J[p][q] = s, J[q][p] = -s, J[q][q] = c
    al[p] = cs;
    be[p] = -sn;
    pa[p] = q;
    al[q] = cs;
    be[q] = sn;
    pa[q] = p;
  }
  __syncthreads();
  double* An = Anew + (int64_t)c * ns * ns;
  double* Vc = V + (int64_t)c * ns * ns;
  const int64_t nblk = (int64_t)half * (half + 1) / 2;
  const int64_t nv = (int64_t)ns * half;
  const int64_t total = nblk + nv;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    if (t < nblk) {
      // block (u, v), u <= v, of the pairing
      int u = (int)((sqrtf((float)(8 * t + 1)) - 1.0f) * 0.5f);
      while ((int64_t)(u + 1) * (u + 2) / 2 <= t) ++u;
      while ((int64_t)u * (u + 1) / 2 > t) --u;
      int v = (int)(t - (int64_t)u * (u + 1) / 2);  // v <= u
      int pu, qu, pv, qv;
      rr_pair(round, u, ns, pu, qu);
      rr_pair(round, v, ns, pv, qv);
      const int I[2] = {pu, qu}, Jx[2] = {pv, qv};
      double a[2][2], rr[2][2];
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) a[x][y] = A[(int64_t)I[x] * ns + Jx[y]];
      // rows: (J^T A)_{ij} = alpha_i A_ij + beta_i A_i'j
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) rr[x][y] = fma(al[I[x]], a[x][y], be[I[x]] * a[1 - x][y]);
      // columns: (R J)_{ij} = alpha_j R_ij + beta_j R_ij'
      for (int x = 0; x < 2; ++x)
        for (int y = 0; y < 2; ++y) {
          int i = I[x], j = Jx[y];
          double r = fma(al[j], rr[x][y], be[j] * rr[x][1 - y]);
          An[(int64_t)i * ns + j] = r;
          An[(int64_t)j * ns + i] = r;
        }
    } else {
      int64_t w = t - nblk;
      int row = (int)(w / half), v = (int)(w % half);
      int pv, qv;
      rr_pair(round, v, ns, pv, qv);
      double x0 = Vc[(int64_t)row * ns + pv], x1 = Vc[(int64_t)row * ns + qv];
      Vc[(int64_t)row * ns + pv] = fma(al[pv], x0, be[pv] * x1);
      Vc[(int64_t)row * ns + qv] = fma(al[qv], x1, be[qv] * x0);
    }
  }
}

// After a sweep: done[c] = off(A) <= 1e-30 * |A|^2 (squared norms).
__global__ void k_jacobi_check(const double* __restrict__ A, int ns, int* __restrict__ done) {
  const int c = blockIdx.x;
  const double* a = A + (int64_t)c * ns * ns;
  double off = 0.0, all = 0.0;
  for (int64_t t = threadIdx.x; t < (int64_t)ns * ns; t += blockDim.x) {
    double v = a[t] * a[t];
    all += v;
    if (t / ns != t % ns) off += v;
  }
  __shared__ double so[32], sa[32];
  for (int o = 16; o > 0; o >>= 1) {
    off += __shfl_xor_sync(0xffffffffu, off, o);
    all += __shfl_xor_sync(0xffffffffu, all, o);
  }
  if ((threadIdx.x & 31) == 0) {
    so[threadIdx.x >> 5] = off;
    sa[threadIdx.x >> 5] = all;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double o2 = 0.0, a2 = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      o2 += so[w];
      a2 += sa[w];
    }
    if (o2 <= 1e-30 * a2 || o2 == 0.0) done[c] = 1;
  }
}

// Order, sign and round the top-D eigenvectors of every index.
__global__ void k_pca_finalize(const double* __restrict__ A, const double* __restrict__ V,
                               const double* __restrict__ mean, int s, int ns, int D, float* __restrict__ basis,
                               float* __restrict__ mean32, double* __restrict__ evals) {
  const int c = blockIdx.x;
  const double* a = A + (int64_t)c * ns * ns;
  const double* v = V + (int64_t)c * ns * ns;
  extern __shared__ int rank_of_col[];  // rank -> column
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double ei = a[(int64_t)i * ns + i];
    int rk = 0;
    for (int j = 0; j < s; ++j) {
      double ej = a[(int64_t)j * ns + j];
      if (ej > ei || (ej == ei && j < i)) ++rk;
    }
    rank_of_col[rk] = i;
    evals[(int64_t)c * s + rk] = ei;
    mean32[(int64_t)c * s + i] = (float)mean[(int64_t)c * s + i];
  }
  __syncthreads();
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    int col = rank_of_col[k];
    int imax = 0;
    double vmax = -1.0;
    for (int i = 0; i < s; ++i) {
      double x = fabs(v[(int64_t)i * ns + col]);
      if (x > vmax) {
        vmax = x;
        imax = i;
      }
    }
    double sg = v[(int64_t)imax * ns + col] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < s; ++i) basis[((int64_t)c * s + i) * D + k] = (float)(sg * v[(int64_t)i * ns + col]);
  }
}

}  // namespace

int pca_build(Index& ix, const float* grid, cudaStream_t st) {
  const int C = ix.C, s = ix.s, D = ix.D;
  const int64_t N = ix.N;
  const int64_t S = (ix.pca_sample <= 0 || ix.pca_sample >= N) ? N : ix.pca_sample;
  const int64_t step = (N + S - 1) / S;
  const int64_t cnt = (N + step - 1) / step;
  const int ns = (s + 1) & ~1;
  const int T = (s + kTile - 1) / kTile;
  std::vector<int2> pairs_h;
  for (int i = 0; i < T; ++i)
    for (int j = i; j < T; ++j) pairs_h.push_back(make_int2(i, j));
  const int npairs = (int)pairs_h.size();
  int nsplit = (int)((cnt + 1023) / 1024);
  if (nsplit > 64) nsplit = 64;
  if (nsplit < 1) nsplit = 1;

  double *mean = nullptr, *partial = nullptr, *A0 = nullptr, *A1 = nullptr, *V = nullptr;
  int2* pairs = nullptr;
  int* done = nullptr;
  SFC_TRY(cudaMallocAsync(&mean, sizeof(double) * C * s, st));
  SFC_TRY(cudaMallocAsync(&partial, sizeof(double) * C * nsplit * npairs * kTile * kTile, st));
  SFC_TRY(cudaMallocAsync(&A0, sizeof(double) * C * ns * ns, st));
  SFC_TRY(cudaMallocAsync(&A1, sizeof(double) * C * ns * ns, st));
  SFC_TRY(cudaMallocAsync(&V, sizeof(double) * C * ns * ns, st));
  SFC_TRY(cudaMallocAsync(&pairs, sizeof(int2) * npairs, st));
  SFC_TRY(cudaMallocAsync(&done, sizeof(int) * C, st));
  SFC_TRY(cudaMemcpyAsync(pairs, pairs_h.data(), sizeof(int2) * npairs, cudaMemcpyHostToDevice, st));
  SFC_TRY(cudaMemsetAsync(done, 0, sizeof(int) * C, st));

  count_launch();
  k_mean<<<dim3((s + 31) / 32, C), 256, 0, st>>>(grid, ix.dict, step, cnt, ix.sub_eoff, s, ix.g.ch, mean);
  count_launch();
  k_cov_partial<<<dim3(npairs, nsplit, C), 256, 0, st>>>(grid, ix.dict, step, cnt, ix.sub_eoff, mean, s, ix.g.ch,
                                                          nsplit, pairs, npairs, partial);
  count_launch();
  k_cov_reduce<<<dim3(64, C), 256, 0, st>>>(partial, nsplit, pairs, npairs, cnt, s, ns, A0, V);
  SFC_TRY(cudaGetLastError());

  const size_t shm = sizeof(double) * 2 * ns + sizeof(int) * ns;
  int ctas = 152 / C;
  if (ctas < 4) ctas = 4;
  double *Ain = A0, *Aout = A1;
  for (int sweep = 0; sweep < kMaxSweeps; ++sweep) {
    for (int r = 0; r < ns - 1; ++r) {
      count_launch();
      k_jacobi_round<<<dim3(ctas, C), 256, shm, st>>>(Ain, Aout, V, ns, r, done);
      double* t = Ain;
      Ain = Aout;
      Aout = t;
    }
    count_launch();
    k_jacobi_check<<<C, 256, 0, st>>>(Ain, ns, done);
  }
  SFC_TRY(cudaGetLastError());
  count_launch();
  k_pca_finalize<<<C, 256, sizeof(int) * s, st>>>(Ain, V, mean, s, ns, D, ix.basis, ix.mean, ix.evals);
  SFC_TRY(cudaGetLastError());
  cudaFreeAsync(mean, st);
  cudaFreeAsync(partial, st);
  cudaFreeAsync(A0, st);
  cudaFreeAsync(A1, st);
  cudaFreeAsync(V, st);
  cudaFreeAsync(pairs, st);
  cudaFreeAsync(done, st);
  return SFC_OK;
}

}  // namespace sfc
