// k_pca.cu -- one PCA per index (Sec. II.A: a conventional PCA, the first D
// principal components are kept).
//
// Data of index c: the subset values (Fig. 2) of dictionary patches, s = m*ch per
// patch, over a deterministic sample (ids 0, step, 2 step, ... with
// step = ceil(N / S)).
//
// Covariance.  Every index's subset is part of the same patch and all indices
// use the same sample, so the mean and the raw second moments are computed once
// for all n patch values and each index's covariance is cut out of them.
// FP64-accurate, computed on the FP32 pipe (this part's FP64 pipe is 1/64 of
// its FP32 rate): the raw second moments sum_a x_i x_j of the FP32 values, each product formed exactly as a pair (p, e) with p = x_i x_j and
// e = fma(x_i, x_j, -p) (Dekker's two-product), accumulated in double-float
// (Knuth's two-sum on the high word, the rounding errors and e added to a low
// word); per sample split the pair is folded to FP64, the splits are summed in
// FP64 in a fixed order and cov = M2 / S - mu mu^T is formed in FP64.  The mean
// is accumulated the same way.  Fixed orders throughout: the result is the same
// on every run.
//
// Eigenvectors.  Only the leading D are needed, so the eigen-solve is block
// subspace iteration with Rayleigh-Ritz projection (Rutishauser's simultaneous
// iteration; e.g. Saad, "Numerical Methods for Large Eigenvalue Problems",
// Ch. 5), in FP64, on p = min(s, max(2D, D + 8), 24) vectors:
//     Y = A Q;  H = Q^T Y;  H = W diag(e) W^T (parallel-order Jacobi, p x p);
//     X = Q W;  Z = Y W (= A X);  stop when |Z_k - e_k X_k| <= 1e-11 e_0 for
//     every k < D;  else Q = orthonormal basis of Z (Cholesky QR, twice; on
//     the cluster path, once the block is close to orthogonal, a Cholesky
//     factor in FP32 of the equilibrated Gram matrix followed by the FP64
//     second-order correction (I + E)^(-1/2) ~ I - E/2 + 3/8 E^2).
// The start block holds the unit vectors of the p largest diagonal entries of A
// plus a small deterministic perturbation.  When A's row slices fit in shared
// memory, the whole iteration runs in one launch on a cluster of 16 CTAs per
// curve (8 where 16-CTA clusters cannot be scheduled; see k_si_cluster); there
// the products are taken in FP32 (A and Q rounded, FP32 accumulation) until a
// Rayleigh-Ritz residual reaches 3.2e-6 of e_0 -- the iteration is
// self-correcting, so this only changes the start of the FP64 iterations, and
// convergence is tested on FP64 products only; otherwise one launch per iteration
// computes Y = A Q with every curve's rows spread over the GPU and a second (one
// CTA per curve) does the p-sized work, a device-side flag ending the iteration
// early.  For s <= kSJacobi the whole s x s problem is solved by Jacobi
// instead (k_eig_full), and for s <= kSFull Jacobi also takes over every curve
// the iteration left unconverged; a curve that is still unconverged is
// reported by the build (SFC_ENOCONV).  Jacobi rotation angles are taken in FP32 and the
// rotation made orthogonal to FP64 precision by a Newton step for
// 1/sqrt(1 + t^2) (no FP64 division or square root in the loop).  Eigenvectors
// are ordered by descending eigenvalue and signed so that the component of
// largest magnitude is positive (ties: lowest index), then rounded to FP32.
#include <cooperative_groups.h>

#include <cmath>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace sfc {

namespace {

constexpr int kTile = 32;    // covariance tile (kTile x kTile outputs per CTA)
constexpr int kChunk = 32;   // samples staged per shared-memory step
constexpr int kMaxIter = 48; // subspace iterations enqueued at most
constexpr int kPMax = 24;    // largest block size p

// (hi, lo) += v in double-float (two-sum on hi, the error into lo)
__device__ inline void df_add(float v, float& hi, float& lo) {
  float t = __fadd_rn(hi, v);
  float bp = __fsub_rn(t, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(v, bp));
  lo = __fadd_rn(lo, err);
  hi = t;
}

// (hi, lo) += a * b, the product formed exactly (two-product)
__device__ inline void df_acc_prod(float a, float b, float& hi, float& lo) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  float t = __fadd_rn(hi, p);
  float bp = __fsub_rn(t, hi);
  float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  lo = __fadd_rn(lo, __fadd_rn(err, e));
  hi = t;
}

// (hi, lo) += a * b for hi >= 0 and a, b >= 0: the product p >= 0, so the
// larger of hi and p is also the one of larger magnitude and Fast2Sum on the
// ordered pair gives the same rounded sum and the same exact error as the
// two-sum above (both are error-free transformations): three additions and
// two max/min instead of six additions.
__device__ inline void df_acc_prod_nonneg(float a, float b, float& hi, float& lo) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  float big = fmaxf(hi, p), small = fminf(hi, p);
  float t = __fadd_rn(big, small);
  float err = __fsub_rn(small, __fsub_rn(t, big));
  lo = __fadd_rn(lo, __fadd_rn(err, e));
  hi = t;
}

// (hi, lo) += a * b when a * b <= hi is known beforehand (hi >= 0): Fast2Sum
// in the given order, the same rounded sum and exact error as the two-sum
__device__ inline void df_acc_prod_dominated(float a, float b, float& hi, float& lo) {
  float p = __fmul_rn(a, b);
  float e = __fmaf_rn(a, b, -p);
  float t = __fadd_rn(hi, p);
  float err = __fsub_rn(p, __fsub_rn(t, hi));
  lo = __fadd_rn(lo, __fadd_rn(err, e));
  hi = t;
}

// Partial raw second moments sum_a x_i x_j of the whole patch (n values), tile
// (ti, tj), ti <= tj, over one split of the sample: partial layout
// [split][pair][32][32] (FP64, folded from double-float).  The CTAs of the
// diagonal tiles (ti == tj) also sum the values themselves, sample by sample
// in order (double-float): msum[split][e], the mean's partial sums.
__global__ void __launch_bounds__(256) k_cov_partial(const float* __restrict__ grid, const uint32_t* __restrict__ dict,
                                                     int64_t step, int64_t cnt, const int* __restrict__ eoff, int n,
                                                     int ch, int nsplit, const int2* __restrict__ pairs, int npairs,
                                                     double* __restrict__ partial, double* __restrict__ msum) {
  const int split = blockIdx.y, pr = blockIdx.x;
  const int2 tp = pairs[pr];
  const int i0 = tp.x * kTile, j0 = tp.y * kTile;
  __shared__ float xi[kChunk][kTile + 1];
  __shared__ float xj[kChunk][kTile + 1];
  __shared__ int eoi[kTile], eoj[kTile];
  if (threadIdx.x < kTile) {
    int i = i0 + threadIdx.x, j = j0 + threadIdx.x;
    eoi[threadIdx.x] = i < n ? eoff[i] : 0;
    eoj[threadIdx.x] = j < n ? eoff[j] : 0;
  }
  __syncthreads();
  const int64_t per = (cnt + nsplit - 1) / nsplit;
  const int64_t a0 = split * per, a1 = a0 + per < cnt ? a0 + per : cnt;
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;  // 16x16 threads, 2x2 outputs each
  float hi[2][2] = {{0.f, 0.f}, {0.f, 0.f}}, lo[2][2] = {{0.f, 0.f}, {0.f, 0.f}};
  const bool msums = tp.x == tp.y && tx == 0;  // this thread also sums rows ty*2, ty*2+1
  float mh[2] = {0.f, 0.f}, ml[2] = {0.f, 0.f};
  // the next chunk's values are loaded into registers while the current one
  // is accumulated (each thread stages kPer (sample, value) pairs)
  constexpr int kPer = kChunk * kTile / 256;
  float pi[kPer], pj[kPer];
  auto load_chunk = [&](int64_t ab) {
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int t = threadIdx.x + u * 256;
      const int k = t / kTile, e = t % kTile;
      const int64_t a = ab + k;
      float vi = 0.0f, vj = 0.0f;
      if (a < a1) {
        const int64_t base = (int64_t)dict[a * step] * ch;
        if (i0 + e < n) vi = grid[base + eoi[e]];
        if (j0 + e < n) vj = grid[base + eoj[e]];
      }
      pi[u] = vi;
      pj[u] = vj;
    }
  };
  // while every staged value so far is >= 0 (pixel data), the sums take the
  // shorter non-negative form; the first negative or NaN value in any chunk
  // switches this block to the general two-sum for good (same results either
  // way).  In the non-negative form, a warp whose every accumulator is already
  // at least the square of the chunk's largest value skips the ordering: no
  // product of the chunk can exceed an accumulator, which only grows.
  __shared__ uint32_t s_wmax[8];
  bool general = false;
  if (a0 < a1) load_chunk(a0);
  for (int64_t ab = a0; ab < a1; ab += kChunk) {
    bool neg = false;
    float vmax = 0.0f;
#pragma unroll
    for (int u = 0; u < kPer; ++u) {
      const int t = threadIdx.x + u * 256;
      xi[t / kTile][t % kTile] = pi[u];
      xj[t / kTile][t % kTile] = pj[u];
      neg |= !(pi[u] >= 0.0f) | !(pj[u] >= 0.0f);
      vmax = fmaxf(vmax, fmaxf(pi[u], pj[u]));
    }
    // non-negative floats order like their bit patterns
    const uint32_t wmax = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
    if ((threadIdx.x & 31) == 0) s_wmax[threadIdx.x >> 5] = wmax;
    general |= __syncthreads_or(neg) != 0;
    if (ab + kChunk < a1) load_chunk(ab + kChunk);
    bool dominated = false;
    if (!general) {
      uint32_t bm = s_wmax[0];
#pragma unroll
      for (int w = 1; w < 8; ++w) bm = max(bm, s_wmax[w]);
      const float m = __uint_as_float(bm);
      const float m2 = __fmul_rn(m, m);  // >= every rounded product of the chunk
      const float hmin = fminf(fminf(hi[0][0], hi[0][1]), fminf(hi[1][0], hi[1][1]));
      dominated = __all_sync(0xffffffffu, hmin >= m2);
    }
    if (dominated) {
#pragma unroll 4
      for (int k = 0; k < kChunk; ++k) {
        float a0v = xi[k][ty * 2], a1v = xi[k][ty * 2 + 1];
        float b0v = xj[k][tx * 2], b1v = xj[k][tx * 2 + 1];
        df_acc_prod_dominated(a0v, b0v, hi[0][0], lo[0][0]);
        df_acc_prod_dominated(a0v, b1v, hi[0][1], lo[0][1]);
        df_acc_prod_dominated(a1v, b0v, hi[1][0], lo[1][0]);
        df_acc_prod_dominated(a1v, b1v, hi[1][1], lo[1][1]);
        if (msums) {
          df_add(a0v, mh[0], ml[0]);
          df_add(a1v, mh[1], ml[1]);
        }
      }
    } else if (general) {
#pragma unroll 4
      for (int k = 0; k < kChunk; ++k) {
        float a0v = xi[k][ty * 2], a1v = xi[k][ty * 2 + 1];
        float b0v = xj[k][tx * 2], b1v = xj[k][tx * 2 + 1];
        df_acc_prod(a0v, b0v, hi[0][0], lo[0][0]);
        df_acc_prod(a0v, b1v, hi[0][1], lo[0][1]);
        df_acc_prod(a1v, b0v, hi[1][0], lo[1][0]);
        df_acc_prod(a1v, b1v, hi[1][1], lo[1][1]);
        if (msums) {
          df_add(a0v, mh[0], ml[0]);
          df_add(a1v, mh[1], ml[1]);
        }
      }
    } else {
#pragma unroll 4
      for (int k = 0; k < kChunk; ++k) {
        float a0v = xi[k][ty * 2], a1v = xi[k][ty * 2 + 1];
        float b0v = xj[k][tx * 2], b1v = xj[k][tx * 2 + 1];
        df_acc_prod_nonneg(a0v, b0v, hi[0][0], lo[0][0]);
        df_acc_prod_nonneg(a0v, b1v, hi[0][1], lo[0][1]);
        df_acc_prod_nonneg(a1v, b0v, hi[1][0], lo[1][0]);
        df_acc_prod_nonneg(a1v, b1v, hi[1][1], lo[1][1]);
        if (msums) {
          df_add(a0v, mh[0], ml[0]);
          df_add(a1v, mh[1], ml[1]);
        }
      }
    }
    __syncthreads();
  }
  if (msums)
    for (int a = 0; a < 2; ++a)
      if (i0 + ty * 2 + a < n) msum[(int64_t)split * n + i0 + ty * 2 + a] = (double)mh[a] + (double)ml[a];
  double* out = partial + ((int64_t)split * npairs + pr) * kTile * kTile;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) out[(ty * 2 + a) * kTile + tx * 2 + b] = (double)hi[a][b] + (double)lo[a][b];
}

// Full-patch second moments M[e][f] (n x n, both triangles) = sum over splits;
// mean[e] = (the splits' sums of value e, in order) / cnt.
__global__ void k_cov_reduce(const double* __restrict__ partial, int nsplit, int npairs, int n,
                             double* __restrict__ M, const double* __restrict__ msum, int64_t cnt,
                             double* __restrict__ mean) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int sp = 0; sp < nsplit; ++sp) t += msum[(int64_t)sp * n + e];
    mean[e] = t / (double)cnt;
  }
  const int T = (n + kTile - 1) / kTile;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)n * n;
       t += (int64_t)gridDim.x * blockDim.x) {
    int i = (int)(t / n), j = (int)(t % n);
    int a = i <= j ? i : j, b = i <= j ? j : i;
    int ti = a / kTile, tj = b / kTile;
    int pr = ti * T - ti * (ti - 1) / 2 + (tj - ti);
    double v = 0.0;
    for (int sp = 0; sp < nsplit; ++sp)
      v += partial[((int64_t)sp * npairs + pr) * kTile * kTile + (a - ti * kTile) * kTile + (b - tj * kTile)];
    M[t] = v;
  }
}

// Covariance of index c from the full-patch moments: the subset's value i is
// patch value e_i = sub_pix[c][i / ch] * ch + i % ch;
// A[c][i][j] = M[e_i][e_j] / cnt - mean[e_i] mean[e_j]; mean_c[i] = mean[e_i].
__global__ void k_cov_extract(const double* __restrict__ M, const double* __restrict__ mean, int n, int ch, int64_t cnt,
                              const int32_t* __restrict__ sub_pix, int m, int s, double* __restrict__ A,
                              double* __restrict__ mean_c) {
  const int c = blockIdx.y;
  const int32_t* sp = sub_pix + (int64_t)c * m;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < (int64_t)s * s;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(t / s), j = (int)(t % s);
    const int ei = sp[i / ch] * ch + i % ch, ej = sp[j / ch] * ch + j % ch;
    A[(int64_t)c * s * s + t] = M[(int64_t)ei * n + ej] / (double)cnt - mean[ei] * mean[ej];
    if (j == 0) mean_c[(int64_t)c * s + i] = mean[ei];
  }
}

// ----------------------------------------------------------------------------
// subspace iteration
// ----------------------------------------------------------------------------
struct SiBufs {
  double* A;   // C*s*s
  double* Q;   // C*s*p
  double* Y;   // C*s*p
  double* X;   // C*s*p
  double* e;   // C*p
  int* done;   // C
  int* iters;  // C: FP64 products with A (tracing)
  int* iters32;  // C: FP32 products with A (tracing; cluster path)
};

// Y = A Q for every curve; blockIdx.y = curve, the s*p outputs spread over
// blockIdx.x.
__global__ void __launch_bounds__(256) k_si_gemm(SiBufs b, int s, int p) {
  const int c = blockIdx.y;
  if (b.done[c]) return;
  extern __shared__ double qs[];  // s*p
  const double* Q = b.Q + (int64_t)c * s * p;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) qs[t] = Q[t];
  __syncthreads();
  const double* A = b.A + (int64_t)c * s * s;
  double* Y = b.Y + (int64_t)c * s * p;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < s * p; t += gridDim.x * blockDim.x) {
    const int i = t / p, k = t % p;
    const double* ar = A + (int64_t)i * s;
    double acc = 0.0;
    for (int j = 0; j < s; ++j) acc = fma(ar[j], qs[j * p + k], acc);
    Y[t] = acc;
  }
}

// Sum of one double per thread over the CTA (result in every thread).
__device__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
  __syncthreads();
  return t;
}

// Orthonormalise the s x p block Z (shared, in place) by Cholesky QR: G = Z^T Z,
// G = R^T R, Z <- Z R^{-1}.  G (p x p, shared) holds R afterwards.
__device__ void chol_qr(double* Z, int s, int p, double* G) {
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    int a = t / p, b = t % p;
    double acc = 0.0;
    if (a <= b)
      for (int i = 0; i < s; ++i) acc = fma(Z[i * p + a], Z[i * p + b], acc);
    G[t] = acc;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    for (int k = 0; k < p; ++k) {
      if (threadIdx.x == 0) G[k * p + k] = sqrt(fmax(G[k * p + k], 1e-300));
      __syncwarp();
      const double rkk = G[k * p + k];
      for (int j = k + 1 + threadIdx.x; j < p; j += 32) G[k * p + j] /= rkk;
      __syncwarp();
      for (int t = threadIdx.x; t < p * p; t += 32) {
        int i = t / p, j = t % p;
        if (i > k && j >= i) G[i * p + j] -= G[k * p + i] * G[k * p + j];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double z[kPMax];
    for (int k = 0; k < p; ++k) z[k] = Z[i * p + k];
    for (int k = 0; k < p; ++k) {
      double v = z[k];
      for (int j = 0; j < k; ++j) v -= z[j] * G[j * p + k];
      z[k] = v / G[k * p + k];
    }
    for (int k = 0; k < p; ++k) Z[i * p + k] = z[k];
  }
  __syncthreads();
}

// Round-robin pairing of round r over n (even) indices: pair 0 = (r, n-1), pair
// i >= 1 = ((r + i) mod (n-1), (r - i) mod (n-1)); every pair meets once per
// n-1 rounds.
__device__ inline void rr_pair(int r, int i, int n, int& p, int& q) {
  int a, b;
  if (i == 0) {
    a = r;
    b = n - 1;
  } else {
    a = (r + i) % (n - 1);
    b = ((r - i) % (n - 1) + (n - 1)) % (n - 1);
  }
  p = a < b ? a : b;
  q = a < b ? b : a;
}

// Parallel-order Jacobi on the small symmetric H (np x np, np even, shared;
// padding rows/columns zero), eigenvectors accumulated into W.  Each round
// rotates np/2 disjoint pairs; every thread updates whole 2x2 blocks in place.
__device__ void small_jacobi(double* H, double* W, int np, double* al, double* be, double* red) {
  for (int t = threadIdx.x; t < np * np; t += blockDim.x) W[t] = (t / np == t % np) ? 1.0 : 0.0;
  __syncthreads();
  const int half = np / 2;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
      double v = H[t] * H[t];
      all += v;
      if (t / np != t % np) off += v;
    }
    off = block_sum(off, red);
    all = block_sum(all, red);
    if (off <= 1e-28 * all || off == 0.0) break;
    for (int r = 0; r < np - 1; ++r) {
      for (int i = threadIdx.x; i < half; i += blockDim.x) {
        int pp, qq;
        rr_pair(r, i, np, pp, qq);
        const double apq = H[pp * np + qq];
        double cs = 1.0, sn = 0.0;
        const float apq32 = (float)apq;
        if (apq32 != 0.0f) {
          // angle in FP32, rotation orthogonal to FP64 precision
          const float tau = __fdiv_rn((float)(H[qq * np + qq] - H[pp * np + pp]), 2.0f * apq32);
          const float t32 = tau >= 0.0f ? 1.0f / (tau + sqrtf(1.0f + tau * tau))
                                        : -1.0f / (-tau + sqrtf(1.0f + tau * tau));
          const double t = (double)t32;
          const double u = fma(t, t, 1.0);
          double y = (double)rsqrtf((float)u);
          y = y * fma(-0.5 * u, y * y, 1.5);
          y = y * fma(-0.5 * u, y * y, 1.5);
          cs = y;
          sn = t * y;
        }
        // J[p][p] = c, J[p][q] = s, J[q][p] = -s, J[q][q] = c
        al[pp] = cs;
        be[pp] = -sn;
        al[qq] = cs;
        be[qq] = sn;
      }
      __syncthreads();
      const int nblk = half * (half + 1) / 2;
      for (int t = threadIdx.x; t < nblk + np * half; t += blockDim.x) {
        if (t < nblk) {
          int u = 0;
          while ((u + 1) * (u + 2) / 2 <= t) ++u;
          const int v = t - u * (u + 1) / 2;
          int pu, qu, pv, qv;
          rr_pair(r, u, np, pu, qu);
          rr_pair(r, v, np, pv, qv);
          const int I[2] = {pu, qu}, J[2] = {pv, qv};
          double a[2][2], rw[2][2];
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) a[x][y] = H[I[x] * np + J[y]];
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) rw[x][y] = fma(al[I[x]], a[x][y], be[I[x]] * a[1 - x][y]);
          for (int x = 0; x < 2; ++x)
            for (int y = 0; y < 2; ++y) {
              const double v2 = fma(al[J[y]], rw[x][y], be[J[y]] * rw[x][1 - y]);
              H[I[x] * np + J[y]] = v2;
              H[J[y] * np + I[x]] = v2;
            }
        } else {
          const int w = t - nblk;
          const int row = w / half, v = w % half;
          int pv, qv;
          rr_pair(r, v, np, pv, qv);
          const double x0 = W[row * np + pv], x1 = W[row * np + qv];
          W[row * np + pv] = fma(al[pv], x0, be[pv] * x1);
          W[row * np + qv] = fma(al[qv], x1, be[qv] * x0);
        }
      }
      __syncthreads();
    }
  }
}

// The p-sized part of one iteration (one CTA per curve, all in shared memory):
// H = Q^T Y, eig(H), X = Q W, Z = Y W, convergence test, Q = orth(Z).
__global__ void __launch_bounds__(256) k_si_small(SiBufs b, int s, int p, int D) {
  const int c = blockIdx.x;
  if (b.done[c]) return;
  if (threadIdx.x == 0) b.iters[c] += 1;
  const int np = p + (p & 1);
  extern __shared__ double sm[];
  double* Q = sm;               // s*p
  double* Y = Q + s * p;        // s*p
  double* H = Y + s * p;        // np*np
  double* W = H + np * np;      // np*np
  double* ev = W + np * np;     // np
  double* al = ev + np;         // np
  double* be = al + np;         // np
  int* ord = reinterpret_cast<int*>(be + np);  // np
  __shared__ double red[8];
  const double* Qg = b.Q + (int64_t)c * s * p;
  const double* Yg = b.Y + (int64_t)c * s * p;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) {
    Q[t] = Qg[t];
    Y[t] = Yg[t];
  }
  __syncthreads();
  for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
    const int a = t / np, bb = t % np;
    double acc = 0.0;
    if (a < p && bb < p && a <= bb) {
      for (int i = 0; i < s; ++i) acc = fma(Q[i * p + a], Y[i * p + bb], acc);
      // Q^T A Q is symmetric up to rounding: average the two triangles
      double acc2 = 0.0;
      for (int i = 0; i < s; ++i) acc2 = fma(Q[i * p + bb], Y[i * p + a], acc2);
      acc = 0.5 * (acc + acc2);
    }
    if (a <= bb) {
      H[a * np + bb] = acc;
      H[bb * np + a] = acc;
    }
  }
  __syncthreads();
  small_jacobi(H, W, np, al, be, red);
  // order the p real Ritz values descending (ties: lower column)
  for (int k = threadIdx.x; k < p; k += blockDim.x) {
    const double ek = H[k * np + k];
    int r = 0;
    for (int j = 0; j < p; ++j) {
      const double ej = H[j * np + j];
      if (ej > ek || (ej == ek && j < k)) ++r;
    }
    ord[r] = k;
    ev[r] = ek;
  }
  __syncthreads();
  double* Xg = b.X + (int64_t)c * s * p;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    double x[kPMax], z[kPMax];
    for (int k = 0; k < p; ++k) {
      const int col = ord[k];
      double ax = 0.0, az = 0.0;
      for (int j = 0; j < p; ++j) {
        ax = fma(Q[i * p + j], W[j * np + col], ax);
        az = fma(Y[i * p + j], W[j * np + col], az);
      }
      x[k] = ax;
      z[k] = az;
    }
    for (int k = 0; k < p; ++k) {
      Xg[(int64_t)i * p + k] = x[k];
      Q[i * p + k] = x[k];
      Y[i * p + k] = z[k];
    }
  }
  __syncthreads();
  double worst = 0.0;
  for (int k = 0; k < D; ++k) {
    double r2 = 0.0;
    for (int i = threadIdx.x; i < s; i += blockDim.x) {
      const double r = Y[i * p + k] - ev[k] * Q[i * p + k];
      r2 = fma(r, r, r2);
    }
    worst = fmax(worst, block_sum(r2, red));
  }
  if (threadIdx.x < p) b.e[(int64_t)c * p + threadIdx.x] = ev[threadIdx.x];
  const bool conv = sqrt(worst) <= 1e-11 * fabs(ev[0]);
  __syncthreads();
  if (conv) {
    if (threadIdx.x == 0) b.done[c] = 1;
    return;
  }
  chol_qr(Y, s, p, H);
  chol_qr(Y, s, p, H);
  double* Qw = b.Q + (int64_t)c * s * p;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) Qw[t] = Y[t];
}

// Start block: unit vectors of the p largest diagonal entries (ties: lower
// index) + a deterministic perturbation, orthonormalised.
__global__ void __launch_bounds__(256) k_si_init(SiBufs b, int s, int p) {
  const int c = blockIdx.x;
  extern __shared__ double sm[];
  double* Z = sm;          // s*p
  double* G = Z + s * p;   // p*p
  const double* A = b.A + (int64_t)c * s * s;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    Z[t] = 1e-3 * (double)(((i * 7 + k * 13) % 17) - 8) / 8.0;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    const double di = A[(int64_t)i * s + i];
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double dj = A[(int64_t)j * s + j];
      if (dj > di || (dj == di && j < i)) ++r;
    }
    if (r < p) Z[i * p + r] += 1.0;
  }
  __syncthreads();
  chol_qr(Z, s, p, G);
  chol_qr(Z, s, p, G);
  double* Qg = b.Q + (int64_t)c * s * p;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) Qg[t] = Z[t];
  if (threadIdx.x == 0) {
    b.done[c] = 0;
    b.iters[c] = 0;
  }
}

// Top-D Ritz vectors -> FP32 basis with the sign convention; evals: the p Ritz
// values then NaN; mean rounded to FP32.
__global__ void k_pca_finalize(SiBufs b, const double* __restrict__ mean, int s, int p, int D,
                               float* __restrict__ basis, float* __restrict__ mean32, double* __restrict__ evals,
                               uint32_t* __restrict__ status) {
  const int c = blockIdx.x;
  const double* X = b.X + (int64_t)c * s * p;
  for (int i = threadIdx.x; i < s; i += blockDim.x) {
    mean32[(int64_t)c * s + i] = (float)mean[(int64_t)c * s + i];
    evals[(int64_t)c * s + i] = i < p ? b.e[(int64_t)c * p + i] : __longlong_as_double(0x7ff8000000000000ll);
  }
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    int imax = 0;
    double vmax = -1.0;
    for (int i = 0; i < s; ++i) {
      const double x = fabs(X[(int64_t)i * p + k]);
      if (x > vmax) {
        vmax = x;
        imax = i;
      }
    }
    const double sg = X[(int64_t)imax * p + k] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < s; ++i) basis[((int64_t)c * s + i) * D + k] = (float)(sg * X[(int64_t)i * p + k]);
  }
}

// Full eigen-decomposition of each index's s x s covariance (s <= kSFull) by
// the parallel-order Jacobi method above, one CTA per curve, everything in
// shared memory.  Used instead of the subspace iteration when s <= kSJacobi
// (the cost, ~s^3 per sweep, is then below the iteration's), and after it for
// kSJacobi < s <= kSFull on the curves the iteration left unconverged
// (only_unconverged = 1): a flat tail of the spectrum (a noise floor, where
// l_{p+1} / l_D is close to 1) stalls the iteration but not Jacobi.  Writes the
// leading p eigenpairs (descending; ties to the lower column) into X and e and
// done[c] = 1 when the off-diagonal norm fell below 1e-14 of the whole.
constexpr int kSJacobi = 64;
constexpr int kSFull = 112;

__global__ void __launch_bounds__(256) k_eig_full(SiBufs b, int s, int p, int only_unconverged) {
  const int c = blockIdx.x;
  if (only_unconverged && b.done[c]) return;
  const int np = s + (s & 1);
  extern __shared__ double sm[];
  double* H = sm;            // np*np
  double* W = H + np * np;   // np*np
  double* al = W + np * np;  // np
  double* be = al + np;      // np
  int* ord = reinterpret_cast<int*>(be + np);  // np
  __shared__ double red[8];
  const double* A = b.A + (int64_t)c * s * s;
  for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
    const int i = t / np, j = t % np;
    H[t] = (i < s && j < s) ? A[(int64_t)i * s + j] : 0.0;
  }
  __syncthreads();
  small_jacobi(H, W, np, al, be, red);
  double off = 0.0, all = 0.0;
  for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
    const double v = H[t] * H[t];
    all += v;
    if (t / np != t % np) off += v;
  }
  off = block_sum(off, red);
  all = block_sum(all, red);
  // order the s eigenvalues descending (the zero padding column excluded)
  for (int k = threadIdx.x; k < s; k += blockDim.x) {
    const double ek = H[k * np + k];
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double ej = H[j * np + j];
      if (ej > ek || (ej == ek && j < k)) ++r;
    }
    ord[r] = k;
  }
  __syncthreads();
  double* X = b.X + (int64_t)c * s * p;
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    X[t] = W[i * np + ord[k]];
  }
  if (threadIdx.x < p) b.e[(int64_t)c * p + threadIdx.x] = H[ord[threadIdx.x] * np + ord[threadIdx.x]];
  if (threadIdx.x == 0) b.done[c] = (off <= 1e-28 * all || off == 0.0) ? 1 : 0;
}

// ----------------------------------------------------------------------------
// the same iteration in one launch per build: a thread-block cluster of CS CTAs
// per curve, A's rows split over the CTAs (in shared memory), partial p x p
// products reduced through distributed shared memory in rank order (every CTA
// ends with the same sums), the Q slices all-gathered the same way, hardware
// cluster barriers between phases.  Rayleigh-Ritz and the convergence test run
// every kRR-th iteration (the subspace converges at the same rate without it).
// ----------------------------------------------------------------------------
constexpr int kRR = 3;  // Rayleigh-Ritz every kRR iterations (of two products each)
constexpr int kMaxIterCl = 64;
constexpr int kLowpIters = 16;  // iterations with FP32 products at most

// 1/sqrt(x) to FP64 accuracy from an FP32 seed: each Newton step
// y (1.5 - x y^2 / 2) doubles the correct bits, 23 -> 46 -> 92 (FMAs only)
__device__ inline double rsqrt64(double x) {
  double y = (double)rsqrtf((float)x);
  y = y * fma(-0.5 * x, y * y, 1.5);
  return y * fma(-0.5 * x, y * y, 1.5);
}

// Eigen-decomposition of the small symmetric H (np x np, shared, FP64) for the
// cluster path: parallel Jacobi in FP32 (cheap on this part), then two steps of
// Ogita & Aishima's iterative refinement in FP64 ("Iterative refinement for
// symmetric eigenvalue decomposition", 2018): with X the current eigenvector
// matrix, R = I - X^T X, S = X^T H X, l_i = S_ii / (1 - R_ii),
// E_ij = (S_ij + l_j R_ij) / (l_j - l_i) (i != j; R_ij / 2 when l_i, l_j are too
// close), E_ii = R_ii / 2, X <- X + X E.  Each step squares the error, so two
// steps take the FP32 result to FP64 accuracy; all FP64 work is dense
// np x np products spread over the CTA.  On exit W holds X and ev the l_i.
__device__ void small_eig_refined(const double* H, double* W, double* ev, int np, float* H32, float* W32,
                                  double* T1, double* T2, double* red) {
  // Index walks avoid run-time integer division: an element t = i * np + j is
  // visited with (i, j) advanced incrementally.
  const int nn = np * np;
  const int di = blockDim.x / np, dj = blockDim.x % np;  // step of (i, j) per blockDim.x
  // FP32 cyclic Jacobi (one warp; np <= 24)
  {
    int i = threadIdx.x / np, j = threadIdx.x % np;
    for (int t = threadIdx.x; t < nn; t += blockDim.x) {
      H32[t] = (float)H[t];
      W32[t] = i == j ? 1.0f : 0.0f;
      i += di;
      j += dj;
      if (j >= np) {
        j -= np;
        ++i;
      }
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // parallel Jacobi (round-robin ordering): each round rotates np / 2
    // disjoint pairs at once -- the angles from the matrix at the start of the
    // round, then all column rotations, then all row rotations (J^T H J with J
    // the product of the pairs' rotations); np - 1 rounds make a sweep
    const int lane = threadIdx.x;
    const int half = np / 2;
    const int m1 = np - 1;
    // this lane's walks: columns step (element l = t % half, row k = t / half),
    // rows step (pair l = t / np, column k = t % np), diagonal test (t / np, t % np)
    const int cl0 = lane % half, ck0 = lane / half, cdl = 32 % half, cdk = 32 / half;
    const int rl0 = lane / np, rk0 = lane % np, rdl = 32 / np, rdk = 32 % np;
    __shared__ int jp[12], jq[12];
    __shared__ float jc[12], js[12];
    for (int sweep = 0; sweep < 12; ++sweep) {
      float off = 0.0f, all = 0.0f;
      {
        int i = rl0, j = rk0;
        for (int t = lane; t < nn; t += 32) {
          const float v = H32[t] * H32[t];
          all += v;
          if (i != j) off += v;
          i += rdl;
          j += rdk;
          if (j >= np) {
            j -= np;
            ++i;
          }
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
      }
      // off-diagonal norm 1e-5 of the whole: the FP64 refinement below squares
      // the error twice, well past FP64 accuracy
      if (off <= 1e-10f * all) break;
      for (int r = 0; r < m1; ++r) {
        if (lane < half) {
          // pair lane of round r: (0, 1 + r) for lane 0, else two players
          // rotating around the fixed player 0
          int a, b;
          if (lane == 0) {
            a = 0;
            b = 1 + r;
          } else {
            int u = r + lane;  // < 2 (np - 1)
            if (u >= m1) u -= m1;
            int v = r - lane + m1;  // in [0, 2 (np - 1))
            if (v >= m1) v -= m1;
            a = 1 + u;
            b = 1 + v;
          }
          const int pp = a < b ? a : b, q = a < b ? b : a;
          const float apq = H32[pp * np + q];
          float cs = 1.0f, sn = 0.0f;
          if (apq != 0.0f) {
            // the angle needs no more than FP32 accuracy (the FP64 steps below
            // refine the eigenvectors), so it uses the hardware approximations;
            // |tau| > 1e18 takes t = 1 / (2 tau), which keeps tau^2 finite
            const float tau = __fdividef(H32[q * np + q] - H32[pp * np + pp], 2.0f * apq);
            const float at = fabsf(tau);
            float tt;
            if (at > 1e18f) {
              tt = __fdividef(0.5f, at);
            } else {
              const float w = __fmaf_rn(at, at, 1.0f);
              tt = __fdividef(1.0f, at + w * rsqrtf(w));
            }
            tt = copysignf(tt, tau);
            cs = rsqrtf(__fmaf_rn(tt, tt, 1.0f));
            sn = tt * cs;
          }
          jp[lane] = pp;
          jq[lane] = q;
          jc[lane] = cs;
          js[lane] = sn;
        }
        __syncwarp();
        // columns pp, q of every row k (and of W); consecutive lanes take
        // different pairs of one row, so their words sit in different banks
        {
          int l = cl0, k = ck0;
          for (int t = lane; t < half * np; t += 32) {
            const int pp = jp[l], q = jq[l];
            const float cs = jc[l], sn = js[l];
            const float hkp = H32[k * np + pp], hkq = H32[k * np + q];
            H32[k * np + pp] = cs * hkp - sn * hkq;
            H32[k * np + q] = sn * hkp + cs * hkq;
            const float wkp = W32[k * np + pp], wkq = W32[k * np + q];
            W32[k * np + pp] = cs * wkp - sn * wkq;
            W32[k * np + q] = sn * wkp + cs * wkq;
            l += cdl;
            k += cdk;
            if (l >= half) {
              l -= half;
              ++k;
            }
          }
        }
        __syncwarp();
        // rows pp, q
        {
          int l = rl0, k = rk0;
          for (int t = lane; t < half * np; t += 32) {
            const int pp = jp[l], q = jq[l];
            const float cs = jc[l], sn = js[l];
            const float hpk = H32[pp * np + k], hqk = H32[q * np + k];
            H32[pp * np + k] = cs * hpk - sn * hqk;
            H32[q * np + k] = sn * hpk + cs * hqk;
            l += rdl;
            k += rdk;
            if (k >= np) {
              k -= np;
              ++l;
            }
          }
        }
        __syncwarp();
      }
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nn; t += blockDim.x) W[t] = (double)W32[t];
  __syncthreads();
  const int i0 = threadIdx.x / np, j0 = threadIdx.x % np;
  for (int step = 0; step < 2; ++step) {
    // T1 = H X
    {
      int i = i0, j = j0;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        double a0 = 0.0, a1 = 0.0;
        for (int k = 0; k < np; k += 2) {
          a0 = fma(H[i * np + k], W[k * np + j], a0);
          if (k + 1 < np) a1 = fma(H[i * np + k + 1], W[(k + 1) * np + j], a1);
        }
        T1[t] = a0 + a1;
        i += di;
        j += dj;
        if (j >= np) {
          j -= np;
          ++i;
        }
      }
    }
    __syncthreads();
    // T2 = S = X^T H X; R = I - X^T X (kept as doubles in the float scratch)
    double* R = reinterpret_cast<double*>(H32);
    {
      int i = i0, j = j0;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        double sv = 0.0, rv = 0.0;
        for (int k = 0; k < np; ++k) {
          sv = fma(W[k * np + i], T1[k * np + j], sv);
          rv = fma(W[k * np + i], W[k * np + j], rv);
        }
        T2[t] = sv;
        R[t] = (i == j ? 1.0 : 0.0) - rv;
        i += di;
        j += dj;
        if (j >= np) {
          j -= np;
          ++i;
        }
      }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < np; i += blockDim.x) ev[i] = T2[i * np + i] / (1.0 - R[i * np + i]);
    __syncthreads();
    // E into T1, then W <- W + W E.  The off-diagonal E_ij are corrections of
    // the size of the current error, so 1 / (l_j - l_i) is taken from the FP32
    // reciprocal with one FP64 Newton step (relative error ~1e-14).
    double smax = 0.0;
    for (int i = 0; i < np; ++i) smax = fmax(smax, fabs(ev[i]));
    {
      int i = i0, j = j0;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        double e;
        if (i == j) {
          e = 0.5 * R[t];
        } else {
          const double d = ev[j] - ev[i];
          const double ad = fabs(d);
          if (ad > 1e-13 * smax) {
            if (ad > 1e-30 && ad < 1e30) {  // inside FP32's normal range
              double rcp = (double)__frcp_rn((float)d);
              rcp = rcp * fma(-d, rcp, 2.0);
              e = (T2[t] + ev[j] * R[t]) * rcp;
            } else {
              e = (T2[t] + ev[j] * R[t]) / d;
            }
          } else {
            e = 0.5 * R[t];
          }
        }
        T1[t] = e;
        i += di;
        j += dj;
        if (j >= np) {
          j -= np;
          ++i;
        }
      }
    }
    __syncthreads();
    {
      int i = i0, j = j0;
      for (int t = threadIdx.x; t < nn; t += blockDim.x) {
        double a = W[t];
        for (int k = 0; k < np; ++k) a = fma(W[i * np + k], T1[k * np + j], a);
        T2[t] = a;
        i += di;
        j += dj;
        if (j >= np) {
          j -= np;
          ++i;
        }
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < nn; t += blockDim.x) W[t] = T2[t];
    __syncthreads();
  }
}

struct ClShm {
  double* As;   // rp x s  (this CTA's rows of A)
  double* Qf;   // s x p   (full Q)
  double* Ys;   // rp x p
  double* Zs;   // rp x p
  double* Xs;   // rp x p
  double* part; // np x np (partial sums exchanged through DSMEM)
  double* Hf;   // np x np
  double* Wf;   // np x np
  double* T1;   // np x np
  double* T2;   // np x np
  double* Rv;   // np x np (as doubles; float scratch of the FP32 Jacobi aliases it)
  float* W32;   // np x np
  double* ev;   // np
  double* al;   // np
  double* be;   // np
  int* ord;     // np
  // upper-triangle pairs (i, j), i <= j < p, ordered by i descending: the pairs
  // with i > k are the first (p - 1 - k)(p - k) / 2 (the trailing part of a
  // Cholesky step k)
  const unsigned char* tri_i;
  const unsigned char* tri_j;
  float* As32;  // rp x s  (this CTA's rows of A rounded to FP32)
  float* Qf32;  // s x p   (Qf rounded to FP32, for the FP32 products)
};

// every CTA: the rows of Qf held by the other CTAs of the cluster (row i by
// rank i / rp), read through distributed shared memory; 16-byte reads where
// the rows pair up and the array is aligned
template <int CS>
__device__ void cl_gather_qf(cg::cluster_group& cl, ClShm& m, int s, int p, int rp) {
  const int me = (int)cl.block_rank();
  if ((p & 1) == 0 && (((uintptr_t)m.Qf) & 15) == 0) {
    const int half = p / 2;
    double2* q2 = reinterpret_cast<double2*>(m.Qf);
#pragma unroll 8
    for (int t = threadIdx.x; t < s * half; t += blockDim.x) {
      const int rk = (t / half) / rp;
      if (rk != me) q2[t] = cl.map_shared_rank(q2, rk)[t];
    }
  } else {
#pragma unroll 4
    for (int t = threadIdx.x; t < s * p; t += blockDim.x) {
      const int rk = (t / p) / rp;
      if (rk != me) m.Qf[t] = cl.map_shared_rank(m.Qf, rk)[t];
    }
  }
}

// every CTA: out[t] = sum over ranks (in order) of part[t], t < len
template <int CS>
__device__ void cl_allreduce(cg::cluster_group& cl, double* part, double* out, int len) {
  cl.sync();
  for (int t = threadIdx.x; t < len; t += blockDim.x) {
    double v[CS];
#pragma unroll
    for (int rk = 0; rk < CS; ++rk) v[rk] = cl.map_shared_rank(part, rk)[t];
    double acc = 0.0;
#pragma unroll
    for (int rk = 0; rk < CS; ++rk) acc += v[rk];
    out[t] = acc;
  }
  cl.sync();
}

// Q rows [r0, r1) := orthonormal basis rows of the distributed block Z (rows
// [r0, r1) here): Cholesky QR, the Gram matrix reduced over the cluster, the
// factor computed redundantly (identically) in every CTA; then all-gather Q.
template <int CS>
__device__ void cl_cholqr(cg::cluster_group& cl, ClShm& m, int nr, int r0, int s, int p, int rp) {
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    double acc = 0.0;
    if (a <= b)
      for (int i = 0; i < nr; ++i) acc = fma(m.Zs[i * p + a], m.Zs[i * p + b], acc);
    m.part[t] = acc;
  }
  cl_allreduce<CS>(cl, m.part, m.Hf, p * p);
  double* G = m.Hf;
  if (threadIdx.x < 32) {
    for (int k = 0; k < p; ++k) {
      const double gkk = G[k * p + k];
      const double y = gkk > 1e-30 ? rsqrt64(gkk) : 0.0;  // a null direction stays a zero column
      __syncwarp();
      if (threadIdx.x == 0) {
        G[k * p + k] = y;  // store 1 / R_kk on the diagonal
      }
      for (int j = k + 1 + threadIdx.x; j < p; j += 32) G[k * p + j] *= y;
      __syncwarp();
      const int nt = (p - 1 - k) * (p - k) / 2;
      for (int u = threadIdx.x; u < nt; u += 32) {
        const int i = m.tri_i[u], j = m.tri_j[u];
        G[i * p + j] = fma(-G[k * p + i], G[k * p + j], G[i * p + j]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // Rinv (upper) in Hf's lower triangle region is in use: build it in part[]
  double* Ri = m.part;
  if (threadIdx.x < p) {
    const int j = threadIdx.x;  // column j of R^{-1}, back substitution
    for (int i = p - 1; i >= 0; --i) {
      double v = 0.0;
      if (i == j) v = 1.0;
      if (i < j)
        for (int k = i + 1; k <= j; ++k) v = fma(-G[i * p + k], Ri[k * p + j], v);
      Ri[i * p + j] = i <= j ? v * G[i * p + i] : 0.0;  // G[i][i] holds 1 / R_ii
    }
  }
  __syncthreads();
  // Q rows = Z rows R^{-1}, one (row, column) per thread
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0; j <= k; j += 2) {
      a0 = fma(m.Zs[i * p + j], Ri[j * p + k], a0);
      if (j + 1 <= k) a1 = fma(m.Zs[i * p + j + 1], Ri[(j + 1) * p + k], a1);
    }
    m.Qf[(r0 + i) * p + k] = a0 + a1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) m.Zs[t] = m.Qf[(r0 + t / p) * p + t % p];
  cl.sync();
  cl_gather_qf<CS>(cl, m, s, p, rp);
  cl.sync();
}

// every CTA: Qf (s x p) := the block whose rows [r0, r0 + nr) are Zs here
template <int CS>
__device__ void cl_allgather_rows(cg::cluster_group& cl, ClShm& m, int nr, int r0, int s, int p, int rp) {
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) m.Qf[(r0 + t / p) * p + t % p] = m.Zs[t];
  cl.sync();
  cl_gather_qf<CS>(cl, m, s, p, rp);
  cl.sync();
}

// Orthonormal basis of a distributed block Z whose columns are already nearly
// orthogonal (the later iterations), with the serial p x p work in FP32:
//   G = Z^T Z (FP64, reduced over the cluster), d_i = G_ii^(-1/2);
//   R = Cholesky factor of D G D in FP32, Q1 = Z D R^{-1} (FP64 products);
//   E = Q1^T Q1 - I (FP64, reduced), Q = Q1 (I - E/2 + 3/8 E^2),
// the last factor being the series of (I + E)^(-1/2) to second order, so that
// Q^T Q = I + O(|E|^3).  Both factors only recombine the columns of Z, so the
// span is Z's.  Returns false, leaving Zs untouched, when the FP32 factor
// fails or max |E| > 1e-5 (then the orthogonality after the series would not
// reach FP64 rounding); every CTA of the cluster takes the same decision, as
// its inputs are the cluster-reduced matrices.
template <int CS>
__device__ bool cl_orth_fast(cg::cluster_group& cl, ClShm& m, int nr, int r0, int s, int p, int rp) {
  __shared__ int s_fail;
  __shared__ double s_emax;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    double acc = 0.0;
    if (a <= b)
      for (int i = 0; i < nr; ++i) acc = fma(m.Zs[i * p + a], m.Zs[i * p + b], acc);
    m.part[t] = acc;
  }
  cl_allreduce<CS>(cl, m.part, m.Hf, p * p);
  double* dsc = m.be;
  float* G32 = reinterpret_cast<float*>(m.Rv);  // p x p factor, then p x p inverse (Rv holds 2 np^2 floats)
  if (threadIdx.x == 0) s_fail = 0;
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double g = m.Hf[i * p + i];
    dsc[i] = g > 1e-300 ? rsqrt64(g) : 0.0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    G32[t] = a <= b ? (float)(m.Hf[t] * dsc[a] * dsc[b]) : 0.0f;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // upper Cholesky factor in place, 1 / R_kk kept on the diagonal
    for (int k = 0; k < p; ++k) {
      const float gkk = G32[k * p + k];
      const bool bad = !(gkk > 1e-6f);
      const float y = bad ? 0.0f : rsqrtf(gkk);
      __syncwarp();
      if (threadIdx.x == 0) {
        G32[k * p + k] = y;
        if (bad) s_fail = 1;
      }
      for (int j = k + 1 + threadIdx.x; j < p; j += 32) G32[k * p + j] *= y;
      __syncwarp();
      const int nt = (p - 1 - k) * (p - k) / 2;
      for (int u = threadIdx.x; u < nt; u += 32) {
        const int i = m.tri_i[u], j = m.tri_j[u];
        G32[i * p + j] = __fmaf_rn(-G32[k * p + i], G32[k * p + j], G32[i * p + j]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (s_fail) return false;
  // M = D R^{-1} (R^{-1} by back substitution in FP32, one column per thread)
  float* Ri32 = G32 + p * p;
  if (threadIdx.x < p) {
    const int j = threadIdx.x;
    for (int i = p - 1; i >= 0; --i) {
      float v = i == j ? 1.0f : 0.0f;
      if (i < j)
        for (int k = i + 1; k <= j; ++k) v = __fmaf_rn(-G32[i * p + k], Ri32[k * p + j], v);
      Ri32[i * p + j] = i <= j ? v * G32[i * p + i] : 0.0f;
    }
  }
  __syncthreads();
  double* M = m.T1;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) M[t] = dsc[t / p] * (double)Ri32[t];
  __syncthreads();
  // Q1 rows = Z rows M (into Ys, free here)
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0; j <= k; j += 2) {
      a0 = fma(m.Zs[i * p + j], M[j * p + k], a0);
      if (j + 1 <= k) a1 = fma(m.Zs[i * p + j + 1], M[(j + 1) * p + k], a1);
    }
    m.Ys[t] = a0 + a1;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    double acc = 0.0;
    if (a <= b)
      for (int i = 0; i < nr; ++i) acc = fma(m.Ys[i * p + a], m.Ys[i * p + b], acc);
    m.part[t] = acc;
  }
  cl_allreduce<CS>(cl, m.part, m.Hf, p * p);
  // E (symmetric, from the upper triangle) into T1; max |E_ij|
  double* E = m.T1;
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    const double g = a <= b ? m.Hf[t] : m.Hf[b * p + a];
    E[t] = a == b ? g - 1.0 : g;
  }
  if (threadIdx.x == 0) s_emax = 0.0;
  __syncthreads();
  if (threadIdx.x < 32) {
    double e = 0.0;
    for (int t = threadIdx.x; t < p * p; t += 32) e = fmax(e, fabs(E[t]));
    for (int o = 16; o > 0; o >>= 1) e = fmax(e, __shfl_xor_sync(0xffffffffu, e, o));
    if (threadIdx.x == 0) s_emax = e;
  }
  __syncthreads();
  if (!(s_emax <= 1e-5)) return false;
  // T = I - E/2 + 3/8 E^2 into T2
  for (int t = threadIdx.x; t < p * p; t += blockDim.x) {
    const int a = t / p, b = t % p;
    double e2 = 0.0;
    for (int k = 0; k < p; ++k) e2 = fma(E[a * p + k], E[k * p + b], e2);
    m.T2[t] = (a == b ? 1.0 : 0.0) - 0.5 * E[t] + 0.375 * e2;
  }
  __syncthreads();
  // Q rows = Q1 rows T, into Qf (own rows) and Zs; then gather every row
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0; j < p; j += 2) {
      a0 = fma(m.Ys[i * p + j], m.T2[j * p + k], a0);
      if (j + 1 < p) a1 = fma(m.Ys[i * p + j + 1], m.T2[(j + 1) * p + k], a1);
    }
    m.Zs[t] = a0 + a1;
  }
  __syncthreads();
  cl_allgather_rows<CS>(cl, m, nr, r0, s, p, rp);
  return true;
}

// out := rows [r0, r0 + nr) of A Qf in FP32 (A and Q rounded to FP32, FP32
// accumulation), widened to FP64: the early iterations only need the span
// to move towards the eigenvectors, which this does at the FP32 pipe's rate
__device__ inline void local_rows_times32(const ClShm& m, int nr, int s, int p, double* out) {
  for (int t = threadIdx.x; t < s * p; t += blockDim.x) m.Qf32[t] = (float)m.Qf[t];
  __syncthreads();
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    const float* ar = m.As32 + i * s;
    float a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, a3 = 0.0f;
    int j = 0;
    for (; j + 3 < s; j += 4) {
      a0 = __fmaf_rn(ar[j], m.Qf32[j * p + k], a0);
      a1 = __fmaf_rn(ar[j + 1], m.Qf32[(j + 1) * p + k], a1);
      a2 = __fmaf_rn(ar[j + 2], m.Qf32[(j + 2) * p + k], a2);
      a3 = __fmaf_rn(ar[j + 3], m.Qf32[(j + 3) * p + k], a3);
    }
    for (; j < s; ++j) a0 = __fmaf_rn(ar[j], m.Qf32[j * p + k], a0);
    out[t] = (double)((a0 + a1) + (a2 + a3));
  }
}

// Zs := rows [r0, r0 + nr) of A Qf
__device__ inline void local_rows_times(const ClShm& m, int nr, int s, int p, double* out) {
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = t / p, k = t % p;
    const double* ar = m.As + i * s;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int j = 0;
    for (; j + 3 < s; j += 4) {
      a0 = fma(ar[j], m.Qf[j * p + k], a0);
      a1 = fma(ar[j + 1], m.Qf[(j + 1) * p + k], a1);
      a2 = fma(ar[j + 2], m.Qf[(j + 2) * p + k], a2);
      a3 = fma(ar[j + 3], m.Qf[(j + 3) * p + k], a3);
    }
    for (; j < s; ++j) a0 = fma(ar[j], m.Qf[j * p + k], a0);
    out[t] = (a0 + a1) + (a2 + a3);
  }
}

template <int CS>
__global__ void __launch_bounds__(256) k_si_cluster(SiBufs b, int s, int p, int D, int use32) {
  cg::cluster_group cl = cg::this_cluster();
  const int c = blockIdx.x / CS;
  const int me = (int)cl.block_rank();
  const int rp = (s + CS - 1) / CS;
  const int r0 = me * rp < s ? me * rp : s;
  const int r1 = r0 + rp < s ? r0 + rp : s;
  const int nr = r1 - r0;
  const int np = p + (p & 1);
  extern __shared__ double sm[];
  ClShm m;
  m.As = sm;
  m.Qf = m.As + rp * s;
  m.Ys = m.Qf + s * p;
  m.Zs = m.Ys + rp * p;
  m.Xs = m.Zs + rp * p;
  m.part = m.Xs + rp * p;
  m.Hf = m.part + np * np;
  m.Wf = m.Hf + np * np;
  m.T1 = m.Wf + np * np;
  m.T2 = m.T1 + np * np;
  m.Rv = m.T2 + np * np;
  m.W32 = reinterpret_cast<float*>(m.Rv + np * np);
  m.ev = reinterpret_cast<double*>(m.W32 + np * np + 2);
  m.al = m.ev + np;
  m.be = m.al + np;
  m.ord = reinterpret_cast<int*>(m.be + np);
  // FP32 copies for the early products (only when shared memory allows)
  m.As32 = use32 ? reinterpret_cast<float*>(((uintptr_t)(m.ord + np) + 15) & ~(uintptr_t)15) : nullptr;
  m.Qf32 = use32 ? m.As32 + rp * s : nullptr;
  __shared__ unsigned char tri_i[kPMax * (kPMax + 1) / 2], tri_j[kPMax * (kPMax + 1) / 2];
  if (threadIdx.x < p) {  // row i = p - 1 - threadIdx.x starts at pair (p - 1 - i)(p - i) / 2
    const int i = p - 1 - threadIdx.x;
    int u = (p - 1 - i) * (p - i) / 2;
    for (int j = i; j < p; ++j, ++u) {
      tri_i[u] = (unsigned char)i;
      tri_j[u] = (unsigned char)j;
    }
  }
  m.tri_i = tri_i;
  m.tri_j = tri_j;
  __shared__ double red[8];
  const double* A = b.A + (int64_t)c * s * s;
  for (int t = threadIdx.x; t < nr * s; t += blockDim.x) {
    const double v = A[(int64_t)r0 * s + t];
    m.As[t] = v;
    if (use32) m.As32[t] = (float)v;
  }
  // start block rows: unit vectors of the p largest diagonal entries + perturbation
  for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
    const int i = r0 + t / p, k = t % p;
    m.Zs[t] = 1e-3 * (double)(((i * 7 + k * 13) % 17) - 8) / 8.0;
  }
  __syncthreads();
  for (int i = r0 + threadIdx.x; i < r1; i += blockDim.x) {
    const double di = A[(int64_t)i * s + i];
    int r = 0;
    for (int j = 0; j < s; ++j) {
      const double dj = A[(int64_t)j * s + j];
      if (dj > di || (dj == di && j < i)) ++r;
    }
    if (r < p) m.Zs[(i - r0) * p + r] += 1.0;
  }
  __syncthreads();
  // the start block is close to orthonormal: the fast form usually suffices
  if (!cl_orth_fast<CS>(cl, m, nr, r0, s, p, rp)) {
    cl_cholqr<CS>(cl, m, nr, r0, s, p, rp);
    if (!cl_orth_fast<CS>(cl, m, nr, r0, s, p, rp)) cl_cholqr<CS>(cl, m, nr, r0, s, p, rp);
  }
  bool conv = false;
  // products in FP32 until a Rayleigh-Ritz residual reaches 3.2e-6 of l_1 (or
  // kLowpIters iterations have passed), in FP64 from then on; convergence is
  // only accepted on FP64 products.  Every CTA of the cluster takes the same
  // decisions (they depend on cluster-reduced values only).
  bool lowp = use32 != 0;
  int prod64 = 0, prod32 = 0;
  for (int it = 0; it < kMaxIterCl && !conv; ++it) {
    // Y = A Q (this CTA's rows)
    const bool lp1 = lowp;
    if (lp1) {
      local_rows_times32(m, nr, s, p, m.Ys);
      ++prod32;
    } else {
      local_rows_times(m, nr, s, p, m.Ys);
      ++prod64;
    }
    __syncthreads();
    const bool rr = (it % kRR) == kRR - 1 || it == kMaxIterCl - 1;
    if (rr) {
      // H = Q^T A Q (upper triangle, mirrored), reduced over the cluster
      for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
        const int a = t / np, bb = t % np;
        double acc = 0.0;
        if (a < p && bb < p && a <= bb)
          for (int i = 0; i < nr; ++i) acc = fma(m.Qf[(r0 + i) * p + a], m.Ys[i * p + bb], acc);
        m.part[t] = acc;
      }
      cl_allreduce<CS>(cl, m.part, m.Hf, np * np);
      for (int t = threadIdx.x; t < np * np; t += blockDim.x) {
        const int a = t / np, bb = t % np;
        if (a > bb) m.Hf[t] = m.Hf[bb * np + a];
      }
      __syncthreads();
      small_eig_refined(m.Hf, m.Wf, m.ev, np, reinterpret_cast<float*>(m.Rv), m.W32, m.T1, m.T2, red);
      // order the p Ritz values descending (ties: lower column); padding column excluded
      for (int k = threadIdx.x; k < p; k += blockDim.x) {
        const double ek = m.ev[k];
        int r = 0;
        for (int j = 0; j < p; ++j) {
          const double ej = m.ev[j];
          if (ej > ek || (ej == ek && j < k)) ++r;
        }
        m.ord[r] = k;
        m.al[r] = ek;
      }
      __syncthreads();
      for (int k = threadIdx.x; k < p; k += blockDim.x) m.ev[k] = m.al[k];
      __syncthreads();
      // X = Q W, Z = Y W (this CTA's rows), one (row, column) per thread
      double* Xg = b.X + (int64_t)c * s * p;
      for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
        const int i = t / p, k = t % p, col = m.ord[k];
        double ax = 0.0, az = 0.0;
        for (int j = 0; j < p; ++j) {
          ax = fma(m.Qf[(r0 + i) * p + j], m.Wf[j * np + col], ax);
          az = fma(m.Ys[i * p + j], m.Wf[j * np + col], az);
        }
        m.Xs[t] = ax;
        m.Zs[t] = az;
        Xg[(int64_t)(r0 + i) * p + k] = ax;
      }
      __syncthreads();
      // residual partial sums |Z_k - e_k X_k|^2 of this CTA's rows, k < D
      for (int t = threadIdx.x; t < np * np; t += blockDim.x) m.part[t] = 0.0;
      for (int t = threadIdx.x; t < nr * p; t += blockDim.x) {
        const int k = t % p;
        const double r = fma(-m.ev[k], m.Xs[t], m.Zs[t]);
        m.Ys[t] = r * r;  // Y is not needed after Z = Y W
      }
      __syncthreads();
      if (threadIdx.x < D) {
        double acc = 0.0;
        for (int i = 0; i < nr; ++i) acc += m.Ys[i * p + threadIdx.x];
        m.part[threadIdx.x] = acc;
      }
      cl_allreduce<CS>(cl, m.part, m.Hf, D);
      double worst = 0.0;
      for (int k = 0; k < D; ++k) worst = fmax(worst, m.Hf[k]);
      conv = !lp1 && worst <= 1e-22 * m.ev[0] * m.ev[0];
      if (lowp && (worst <= 1e-11 * m.ev[0] * m.ev[0] || it >= kLowpIters)) lowp = false;
      if (conv || it == kMaxIterCl - 1) {
        if (me == 0 && threadIdx.x < p) b.e[(int64_t)c * p + threadIdx.x] = m.ev[threadIdx.x];
        if (me == 0 && threadIdx.x == 0) {
          b.done[c] = conv ? 1 : 0;
          b.iters[c] = prod64;  // FP64 products with A
          b.iters32[c] = prod32;
        }
        break;
      }
    } else {
      for (int t = threadIdx.x; t < nr * p; t += blockDim.x) m.Zs[t] = m.Ys[t];
      __syncthreads();
    }
    // a second product before orthonormalising: Z = A^2 Q (A^2 X after a
    // Rayleigh-Ritz step), which squares the convergence factor per Cholesky QR;
    // the block's condition stays near (l_1 / l_p)^2, inside CholeskyQR2's reach
    __syncthreads();
    cl_allgather_rows<CS>(cl, m, nr, r0, s, p, rp);
    if (lowp) {
      local_rows_times32(m, nr, s, p, m.Zs);
      ++prod32;
    } else {
      local_rows_times(m, nr, s, p, m.Zs);
      ++prod64;
    }
    __syncthreads();
    // two passes while the block is far from the eigen-directions; afterwards
    // Z has nearly orthogonal columns and one pass is accurate to rounding
    // the FP32 factor with the FP64 second-order correction when the block is
    // close enough to orthogonal, else two FP64 Cholesky QR passes
    // (after one FP64 pass the block is close to orthonormal, so the second
    // pass is the fast form whenever its FP32 factor succeeds)
    if (!cl_orth_fast<CS>(cl, m, nr, r0, s, p, rp)) {
      cl_cholqr<CS>(cl, m, nr, r0, s, p, rp);
      if (!cl_orth_fast<CS>(cl, m, nr, r0, s, p, rp)) cl_cholqr<CS>(cl, m, nr, r0, s, p, rp);
    }
  }
  cl.sync();  // no CTA leaves while others may still read its shared memory
}

size_t cluster_shm_bytes(int s, int p, int CS, bool use32) {
  const int rp = (s + CS - 1) / CS;
  const int np = p + (p & 1);
  // As, Qf, Ys, Zs, Xs, part, Hf, Wf, T1, T2, Rv (doubles); W32 (floats) + pad;
  // ev, al, be (doubles); ord (ints); 16-byte alignment; As32, Qf32 (floats)
  return sizeof(double) * ((size_t)rp * s + (size_t)s * p + 3 * (size_t)rp * p + 6 * (size_t)np * np + 3 * np) +
         sizeof(float) * ((size_t)np * np + 2) + sizeof(int) * np +
         (use32 ? 16 + sizeof(float) * ((size_t)rp * s + (size_t)s * p) : 0);
}

}  // namespace

int pca_build(Index& ix, const float* grid, cudaStream_t st) {
  const int C = ix.C, s = ix.s, D = ix.D;
  const int64_t N = ix.N;
  const int64_t S = (ix.pca_sample <= 0 || ix.pca_sample >= N) ? N : ix.pca_sample;
  const int64_t step = (N + S - 1) / S;
  const int64_t cnt = (N + step - 1) / step;
  int p = 2 * D > D + 8 ? 2 * D : D + 8;
  if (p > kPMax) p = kPMax;
  if (p > s) p = s;
  const int np = p + (p & 1);
  const int n = ix.g.n;
  const int T = (n + kTile - 1) / kTile;
  std::vector<int2> pairs_h;
  for (int i = 0; i < T; ++i)
    for (int j = i; j < T; ++j) pairs_h.push_back(make_int2(i, j));
  const int npairs = (int)pairs_h.size();
  int nsplit = (int)((cnt + 511) / 512);
  if (nsplit > 64) nsplit = 64;
  if (nsplit < 1) nsplit = 1;

  double *mean = nullptr, *mean_c = nullptr, *msum = nullptr, *partial = nullptr, *M = nullptr;
  int2* pairs = nullptr;
  SiBufs b;
  Scratch scr(st);
  SFC_TRY(scr.alloc(&mean, sizeof(double) * n));
  SFC_TRY(scr.alloc(&mean_c, sizeof(double) * C * s));
  SFC_TRY(scr.alloc(&msum, sizeof(double) * nsplit * n));
  SFC_TRY(scr.alloc(&partial, sizeof(double) * nsplit * npairs * kTile * kTile));
  SFC_TRY(scr.alloc(&M, sizeof(double) * n * n));
  SFC_TRY(scr.alloc(&pairs, sizeof(int2) * npairs));
  SFC_TRY(scr.alloc(&b.A, sizeof(double) * C * s * s));
  SFC_TRY(scr.alloc(&b.Q, sizeof(double) * C * s * p));
  SFC_TRY(scr.alloc(&b.Y, sizeof(double) * C * s * p));
  SFC_TRY(scr.alloc(&b.X, sizeof(double) * C * s * p));
  SFC_TRY(scr.alloc(&b.e, sizeof(double) * C * p));
  SFC_TRY(scr.alloc(&b.done, sizeof(int) * C));
  b.iters = ix.eig_iters;
  b.iters32 = ix.eig_iters + C;
  SFC_TRY(cudaMemsetAsync(b.iters, 0, sizeof(int) * C, st));
  SFC_TRY(cudaMemcpyAsync(pairs, pairs_h.data(), sizeof(int2) * npairs, cudaMemcpyHostToDevice, st));

  count_launch();
  k_cov_partial<<<dim3(npairs, nsplit), 256, 0, st>>>(grid, ix.dict, step, cnt, ix.eoff_all, n, ix.g.ch, nsplit,
                                                      pairs, npairs, partial, msum);
  count_launch();
  k_cov_reduce<<<128, 256, 0, st>>>(partial, nsplit, npairs, n, M, msum, cnt, mean);
  count_launch();
  k_cov_extract<<<dim3(64, C), 256, 0, st>>>(M, mean, n, ix.g.ch, cnt, ix.sub_pix, ix.m, s, b.A, mean_c);
  SFC_TRY(cudaGetLastError());
  trace_mark(ix, 2, st);
  ix.p_block = p;

  const size_t shm_init = sizeof(double) * ((size_t)s * p + (size_t)p * p);
  const size_t shm_small = sizeof(double) * (2 * (size_t)s * p + 2 * (size_t)np * np + 3 * np) + sizeof(int) * np;
  const size_t shm_gemm = sizeof(double) * (size_t)s * p;
  if (shm_init > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_si_init, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_init));
  if (shm_small > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_si_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_small));
  if (shm_gemm > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_si_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_gemm));
  const int npf = s + (s & 1);
  const size_t shm_full = sizeof(double) * (2 * (size_t)npf * npf + 2 * npf) + sizeof(int) * npf;
  if (s <= kSFull && shm_full > kSmemOptIn)
    SFC_TRY(cudaFuncSetAttribute(k_eig_full, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_full));
  // cluster path: the first of (16 CTAs, FP32 copies), (8, FP32 copies),
  // (16, none), (8, none) whose clusters for every curve can all run at once
  // (a second wave of clusters costs about as much as the first: 16-CTA
  // clusters at one CTA per SM measured 1.27 against 0.80 ms); if none can,
  // the schedulable one with the most clusters at once
  int cs = 0, use32 = 0, best_n = 0;
  size_t shm_cl = 0;
  for (int opt = 0; opt < 4 && s > kSJacobi; ++opt) {
    const int cand = (opt & 1) == 0 ? 16 : 8;
    const bool w32 = opt < 2;
    const size_t need = cluster_shm_bytes(s, p, cand, w32);
    if (need > 200 * 1024) continue;
    const void* fn = cand == 16 ? (const void*)k_si_cluster<16> : (const void*)k_si_cluster<8>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)need) != cudaSuccess) continue;
    if (cand == 16 && cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    cudaLaunchConfig_t q = {};
    q.gridDim = dim3(C * cand);
    q.blockDim = dim3(256);
    q.dynamicSmemBytes = need;
    cudaLaunchAttribute qa[1];
    qa[0].id = cudaLaunchAttributeClusterDimension;
    qa[0].val.clusterDim.x = cand;
    qa[0].val.clusterDim.y = 1;
    qa[0].val.clusterDim.z = 1;
    q.attrs = qa;
    q.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &q) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      continue;
    }
    if (nclusters > best_n) {
      best_n = nclusters;
      cs = cand;
      use32 = w32 ? 1 : 0;
      shm_cl = need;
    }
    if (nclusters >= C) break;  // one wave
  }
  if (cs) {  // the chosen kernel's shared-memory size (a later candidate may have set another)
    const void* fn = cs == 16 ? (const void*)k_si_cluster<16> : (const void*)k_si_cluster<8>;
    SFC_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_cl));
  }
  if (s <= kSJacobi) {
    count_launch();
    k_eig_full<<<C, 256, shm_full, st>>>(b, s, p, 0);
  } else if (cs) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(C * cs);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = shm_cl;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = cs;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    ix.eig_per_orth = 2;
    count_launch();
    if (cs == 16)
      SFC_TRY(cudaLaunchKernelEx(&cfg, k_si_cluster<16>, b, s, p, D, use32));
    else
      SFC_TRY(cudaLaunchKernelEx(&cfg, k_si_cluster<8>, b, s, p, D, use32));
  } else {
    count_launch();
    k_si_init<<<C, 256, shm_init, st>>>(b, s, p);
  int gx = (s * p + 255) / 256;
  const int per_curve = 152 / C > 0 ? 152 / C : 1;
  if (gx > per_curve) gx = per_curve;
    for (int it = 0; it < kMaxIter; ++it) {
      count_launch();
      k_si_gemm<<<dim3(gx, C), 256, shm_gemm, st>>>(b, s, p);
      count_launch();
      k_si_small<<<C, 256, shm_small, st>>>(b, s, p, D);
    }
  }
  if (s > kSJacobi && s <= kSFull) {
    // the curves the iteration left unconverged (returns at once for the others)
    count_launch();
    k_eig_full<<<C, 256, shm_full, st>>>(b, s, p, 1);
  }
  SFC_TRY(cudaGetLastError());
  trace_mark(ix, 3, st);
  count_launch();
  k_pca_finalize<<<C, 256, 0, st>>>(b, mean_c, s, p, D, ix.basis, ix.mean, ix.evals, status_word());
  SFC_TRY(cudaGetLastError());
  scr.keep(b.done);
  ix.pca_done = b.done;  // read by the build once the device is done with it
  return SFC_OK;  // the guard frees the rest on the stream
}

}  // namespace sfc
