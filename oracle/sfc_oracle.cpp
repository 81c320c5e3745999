// sfc_oracle.cpp -- plain, slow, single-threaded CPU oracle for the patch search
// of "Space-Filling Curve Indices as Acceleration Structure for Exemplar-Based
// Inpainting" (Dahmen et al.).
//
// TEST INFRASTRUCTURE ONLY.  This file is the checker the CUDA path is compared
// against; only the tests, the smoke entry and the benchmark's CPU-baseline leg
// load it.  It shares no code, header, table or constant with the CUDA library,
// and the CUDA library never calls it.
//
// Build: g++ -O2 -ffp-contract=off -fPIC -shared (no fast-math), so every float
// and double operation below is one IEEE-754 round-to-nearest operation in the
// order written.
//
// Every function follows the definition it cites, written out directly, with no
// blocking, fusion or reordering:
//   * patches, patch space, RGB channels treated separately  -- Sec. II (intro)
//   * masked L2 cost, unknown differences count as zero      -- Sec. II, after Fig. 1
//   * full scan = cost for every dictionary patch + global min -- Sec. I
//   * dictionary = the fully known patches                   -- Sec. I, Sec. IV
//   * one index per pixel subset (edge middles, corners), c  -- Sec. II, Fig. 2
//   * PCA per index, first D components                      -- Sec. II.A
//   * quantised coordinates, Morton/z-address, MSB first,
//     dimension 0 first, highest-variance dimension first   -- Sec. II.C
//   * z-order comparison: the axis with the highest differing bit -- Sec. II.C
//   * sort by z-order, binary search on the sorted array     -- Sec. II.B, II.C
//   * filter-and-refine: candidates rescored in image space  -- Fig. 1(d)
//   * fill front, search area, target area, best index       -- Fig. 1(a)-(c)
//   * brute-force k-NN in the quantised principal space       -- Sec. II.D (result definition)
// Readings where the paper is silent (tie rules, subset anchors, quantiser,
// candidate window, priority formula) are stated beside each function.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <numeric>
#include <vector>

namespace {

struct Geo {
  int ndim;
  int64_t X, Y, Z;
  int ch;
  int K;
  int r;
  int P;  // pixels per patch, K^ndim
};

Geo make_geo(int ndim, const int64_t* ext, int ch, int K) {
  Geo g;
  g.ndim = ndim;
  g.X = ext[0];
  g.Y = ext[1];
  g.Z = ndim == 3 ? ext[2] : 1;
  g.ch = ch;
  g.K = K;
  g.r = K / 2;
  g.P = ndim == 3 ? K * K * K : K * K;
  return g;
}

inline void coords_of(const Geo& g, int64_t lin, int64_t* c) {
  c[0] = lin % g.X;
  int64_t t = lin / g.X;
  c[1] = t % g.Y;
  c[2] = t / g.Y;
}

inline int64_t lin_of(const Geo& g, int64_t x, int64_t y, int64_t z) { return (z * g.Y + y) * g.X + x; }

// Patch pixel pp (raster order inside the patch, x fastest) -> (dx, dy, dz).
inline void patch_delta(const Geo& g, int pp, int* d) {
  d[0] = pp % g.K - g.r;
  d[1] = (pp / g.K) % g.K - g.r;
  d[2] = g.ndim == 3 ? pp / (g.K * g.K) - g.r : 0;
}

inline int64_t patch_pixel(const Geo& g, int64_t centre, int pp) {
  int d[3];
  patch_delta(g, pp, d);
  int64_t c[3];
  coords_of(g, centre, c);
  return lin_of(g, c[0] + d[0], c[1] + d[1], c[2] + d[2]);
}

inline bool centre_valid(const Geo& g, int64_t x, int64_t y, int64_t z) {
  if (x < g.r || x > g.X - 1 - g.r) return false;
  if (y < g.r || y > g.Y - 1 - g.r) return false;
  if (g.ndim == 3 && (z < g.r || z > g.Z - 1 - g.r)) return false;
  return true;
}

// Masked L2 cost in FP64 (Sec. II after Fig. 1: differences at unknown pixels are
// taken as zero).  Reading: the squared form (same argmin as the norm); elements
// summed one by one in patch raster order, channel innermost; operands widened
// from FP32; term = w_ch * (d * d); no fused multiply-add.  norm == 1: the L1
// norm of Sec. III.K instead, term = w_ch * |d|, same order.
double cost64(const Geo& g, const float* grid, const uint8_t* cur_mask, int64_t t, int64_t s, const float* w,
              int norm) {
  double acc = 0.0;
  for (int pp = 0; pp < g.P; ++pp) {
    int64_t qt = patch_pixel(g, t, pp);
    if (!cur_mask[qt]) continue;
    int64_t qs = patch_pixel(g, s, pp);
    for (int c = 0; c < g.ch; ++c) {
      double d = (double)grid[qt * g.ch + c] - (double)grid[qs * g.ch + c];
      double term = norm == 1 ? std::fabs(d) : d * d;
      double wc = w ? (double)w[c] : 1.0;
      acc = acc + wc * term;
    }
  }
  return acc;
}

inline void sort_unique(std::vector<int64_t>& v) {
  std::sort(v.begin(), v.end());
  v.erase(std::unique(v.begin(), v.end()), v.end());
}

}  // namespace

extern "C" {

// ----------------------------------------------------------------------------
// Dictionary (Sec. I: "the known parts of the image ... split into patches";
// Sec. IV: undamaged parts are the dictionary).  Reading: every patch whose box
// lies inside the grid and whose pixels are all known under the build-time mask;
// dictionary id = rank of its centre in raster order (x fastest, then y, z).
// Returns N; writes min(N, cap) centre linear indices when out != NULL.
// ----------------------------------------------------------------------------
int64_t or_dict_extract(const uint8_t* mask, int ndim, const int64_t* ext, int K, int64_t* out, int64_t cap) {
  Geo g = make_geo(ndim, ext, 1, K);
  int64_t n = 0;
  for (int64_t z = 0; z < g.Z; ++z)
    for (int64_t y = 0; y < g.Y; ++y)
      for (int64_t x = 0; x < g.X; ++x) {
        if (!centre_valid(g, x, y, z)) continue;
        int64_t centre = lin_of(g, x, y, z);
        bool ok = true;
        for (int pp = 0; pp < g.P && ok; ++pp) ok = mask[patch_pixel(g, centre, pp)] != 0;
        if (!ok) continue;
        if (out && n < cap) out[n] = centre;
        ++n;
      }
  return n;
}

// Exact cost of one (target, source) pair, exposed for tests (norm: 0 = L2, 1 = L1).
double or_cost64(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K,
                 int64_t target, int64_t source, const float* w, int norm) {
  Geo g = make_geo(ndim, ext, ch, K);
  return cost64(g, grid, cur_mask, target, source, w, norm);
}

// ----------------------------------------------------------------------------
// Full scan (Sec. I): the cost for every dictionary patch, then the global
// minimum.  Reading: ties go to the lowest dictionary id (strict "<" in id order).
// ----------------------------------------------------------------------------
void or_fullscan(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K,
                 const int64_t* dict, int64_t N, const int64_t* targets, int64_t Q, const float* w, int64_t* pick,
                 double* cost, int norm) {
  Geo g = make_geo(ndim, ext, ch, K);
  for (int64_t q = 0; q < Q; ++q) {
    double best = INFINITY;
    int64_t bj = -1;
    for (int64_t j = 0; j < N; ++j) {
      double c = cost64(g, grid, cur_mask, targets[q], dict[j], w, norm);
      if (c < best) {
        best = c;
        bj = j;
      }
    }
    pick[q] = bj;
    cost[q] = best;
  }
}

// ----------------------------------------------------------------------------
// Pixel subsets of the indices (Sec. II, Fig. 2): each index uses the fraction c
// of the patch pixels nearest to the middle of one patch edge or one corner.
// Reading: the patch is the square/cube [-1/2, K-1/2]^dim around the pixel
// centres; anchors in 2-D, in this order: middles of the top, right, bottom,
// left edges, then the corners top-left, top-right, bottom-right, bottom-left;
// in 3-D: the 8 corners (x fastest), then the middles of the faces z-, z+, y-,
// y+, x-, x+.  m = floor(c * K^dim + 1/2) pixels with the smallest squared
// distance to the anchor, ties to the lower raster index; every channel of a
// chosen pixel is used.  Output: out[cv * m + i] = patch pixel index, ascending.
// Returns 0, or -1 if C exceeds the number of anchors.
// ----------------------------------------------------------------------------
int or_subsets(int ndim, int K, double frac, int C, int32_t* out, int32_t* m_out) {
  int P = ndim == 3 ? K * K * K : K * K;
  int m = (int)std::floor(frac * P + 0.5);
  if (m < 1) m = 1;
  if (m > P) m = P;
  *m_out = m;
  // anchors in doubled coordinates: pixel centre p sits at 2p+1, the patch
  // spans [0, 2K] per axis.
  std::vector<std::array<int, 3>> anchors;
  const int E = 2 * K, H = K;
  if (ndim == 2) {
    anchors = {{H, 0, 0}, {E, H, 0}, {H, E, 0}, {0, H, 0}, {0, 0, 0}, {E, 0, 0}, {E, E, 0}, {0, E, 0}};
  } else {
    for (int cz = 0; cz < 2; ++cz)
      for (int cy = 0; cy < 2; ++cy)
        for (int cx = 0; cx < 2; ++cx) anchors.push_back({cx * E, cy * E, cz * E});
    anchors.push_back({H, H, 0});
    anchors.push_back({H, H, E});
    anchors.push_back({H, 0, H});
    anchors.push_back({H, E, H});
    anchors.push_back({0, H, H});
    anchors.push_back({E, H, H});
  }
  if (C > (int)anchors.size() || C < 1) return -1;
  for (int cv = 0; cv < C; ++cv) {
    std::vector<std::pair<int64_t, int>> d(P);
    for (int pp = 0; pp < P; ++pp) {
      int px = pp % K, py = (pp / K) % K, pz = ndim == 3 ? pp / (K * K) : 0;
      int64_t dx = 2 * px + 1 - anchors[cv][0];
      int64_t dy = 2 * py + 1 - anchors[cv][1];
      int64_t dz = ndim == 3 ? 2 * pz + 1 - anchors[cv][2] : 0;
      d[pp] = {dx * dx + dy * dy + dz * dz, pp};
    }
    std::sort(d.begin(), d.end());
    std::vector<int> sel(m);
    for (int i = 0; i < m; ++i) sel[i] = d[i].second;
    std::sort(sel.begin(), sel.end());
    for (int i = 0; i < m; ++i) out[(int64_t)cv * m + i] = sel[i];
  }
  return 0;
}

// ----------------------------------------------------------------------------
// Symmetric eigen-decomposition by the cyclic (row-by-row) Jacobi method, the
// textbook algorithm (Golub & Van Loan, "Matrix Computations", Sec. 8.5): for
// each pair p < q choose the plane rotation that zeroes A[p][q], apply it on both
// sides of A and on the right of V.  Sweeps repeat until the off-diagonal
// Frobenius norm is <= 1e-15 of the whole norm, or max_sweeps.
// A (n x n, row-major) is overwritten; evals[i] = final A[i][i]; V columns are the
// eigenvectors.  Returns the number of sweeps used.
// ----------------------------------------------------------------------------
int or_jacobi(double* A, int n, double* evals, double* V, int max_sweeps) {
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) V[(int64_t)i * n + j] = i == j ? 1.0 : 0.0;
  int sweep = 0;
  for (; sweep < max_sweeps; ++sweep) {
    double off = 0.0, all = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double a = A[(int64_t)i * n + j];
        all += a * a;
        if (i != j) off += a * a;
      }
    if (off <= 1e-30 * all || off == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        double apq = A[(int64_t)p * n + q];
        if (apq == 0.0) continue;
        double app = A[(int64_t)p * n + p], aqq = A[(int64_t)q * n + q];
        double tau = (aqq - app) / (2.0 * apq);
        double t = tau >= 0.0 ? 1.0 / (tau + std::sqrt(1.0 + tau * tau)) : -1.0 / (-tau + std::sqrt(1.0 + tau * tau));
        double c = 1.0 / std::sqrt(1.0 + t * t);
        double s = t * c;
        // A <- A J   (columns p, q)
        for (int k = 0; k < n; ++k) {
          double akp = A[(int64_t)k * n + p], akq = A[(int64_t)k * n + q];
          A[(int64_t)k * n + p] = c * akp - s * akq;
          A[(int64_t)k * n + q] = s * akp + c * akq;
        }
        // A <- J^T A (rows p, q)
        for (int k = 0; k < n; ++k) {
          double apk = A[(int64_t)p * n + k], aqk = A[(int64_t)q * n + k];
          A[(int64_t)p * n + k] = c * apk - s * aqk;
          A[(int64_t)q * n + k] = s * apk + c * aqk;
        }
        // V <- V J
        for (int k = 0; k < n; ++k) {
          double vkp = V[(int64_t)k * n + p], vkq = V[(int64_t)k * n + q];
          V[(int64_t)k * n + p] = c * vkp - s * vkq;
          V[(int64_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) evals[i] = A[(int64_t)i * n + i];
  return sweep;
}

// ----------------------------------------------------------------------------
// PCA of one index (Sec. II.A: conventional PCA, keep the first D components).
// Readings: data = the index's subset values of dictionary patches (subset pixel
// order, channel innermost), s = m * ch values each; deterministic sample = ids
// 0, step, 2*step, ... < N with step = ceil(N / S), S = min(N, sample) (all of N
// when sample <= 0); mean and covariance in FP64 summed in sample order,
// normalised by the sample count; eigenpairs by cyclic Jacobi, ordered by
// descending eigenvalue (ties: lower original column); each eigenvector's
// largest-magnitude component made positive (ties: lowest index); rounded to
// FP32.  basis is s x D row-major (basis[i*D + k]); mean32 has s entries;
// evals_out gets all s eigenvalues in the chosen order.  Returns Jacobi sweeps.
// ----------------------------------------------------------------------------
int or_pca(const float* grid, int ndim, const int64_t* ext, int ch, int K, const int64_t* dict, int64_t N,
           const int32_t* subset, int m, int64_t sample, int D, float* basis, float* mean32, double* evals_out,
           double* cov_out) {
  Geo g = make_geo(ndim, ext, ch, K);
  const int s = m * ch;
  int64_t S = (sample <= 0 || sample >= N) ? N : sample;
  int64_t step = (N + S - 1) / S;
  std::vector<int64_t> ids;
  for (int64_t j = 0; j < N; j += step) ids.push_back(j);
  const int64_t cnt = (int64_t)ids.size();
  auto value = [&](int64_t j, int i) -> double {
    int pp = subset[i / ch];
    int c = i % ch;
    return (double)grid[patch_pixel(g, dict[j], pp) * ch + c];
  };
  std::vector<double> mu(s, 0.0);
  for (int64_t a = 0; a < cnt; ++a)
    for (int i = 0; i < s; ++i) mu[i] += value(ids[a], i);
  for (int i = 0; i < s; ++i) mu[i] = mu[i] / (double)cnt;
  std::vector<double> A((size_t)s * s, 0.0);
  std::vector<double> x(s);
  for (int64_t a = 0; a < cnt; ++a) {
    for (int i = 0; i < s; ++i) x[i] = value(ids[a], i) - mu[i];
    for (int i = 0; i < s; ++i)
      for (int j = i; j < s; ++j) A[(size_t)i * s + j] += x[i] * x[j];
  }
  for (int i = 0; i < s; ++i)
    for (int j = i; j < s; ++j) {
      double v = A[(size_t)i * s + j] / (double)cnt;
      A[(size_t)i * s + j] = v;
      A[(size_t)j * s + i] = v;
    }
  if (cov_out) std::memcpy(cov_out, A.data(), sizeof(double) * s * s);
  std::vector<double> ev(s), V((size_t)s * s);
  int sweeps = or_jacobi(A.data(), s, ev.data(), V.data(), 100);
  std::vector<int> order(s);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ev[a] > ev[b]; });
  for (int k = 0; k < s; ++k) evals_out[k] = ev[order[k]];
  for (int k = 0; k < D; ++k) {
    int col = order[k];
    int imax = 0;
    double vmax = -1.0;
    for (int i = 0; i < s; ++i) {
      double a = std::fabs(V[(size_t)i * s + col]);
      if (a > vmax) {
        vmax = a;
        imax = i;
      }
    }
    double sign = V[(size_t)imax * s + col] < 0.0 ? -1.0 : 1.0;
    for (int i = 0; i < s; ++i) basis[(size_t)i * D + k] = (float)(sign * V[(size_t)i * s + col]);
  }
  for (int i = 0; i < s; ++i) mean32[i] = (float)mu[i];
  return sweeps;
}

// ----------------------------------------------------------------------------
// Projection to principal space (Sec. II.A).  Reading: y_k = sum over subset
// values i, in subset order, of B[i][k] * (x_i - mu_i), with x_i - mu_i rounded
// to FP32 and the sum a chain of FP32 fused multiply-adds starting at +0.
// When mask != NULL (a query), values at unknown pixels are skipped: they
// contribute exactly zero (the principal-space analogue of the zero difference
// at unknown pixels, Sec. II after Fig. 1).
// ----------------------------------------------------------------------------
void or_project_one(const float* grid, const uint8_t* mask, int ndim, const int64_t* ext, int ch, int K,
                    int64_t centre, const int32_t* subset, int m, const float* basis, const float* mean32, int D,
                    float* y) {
  Geo g = make_geo(ndim, ext, ch, K);
  for (int k = 0; k < D; ++k) {
    float acc = 0.0f;
    for (int i = 0; i < m * ch; ++i) {
      int64_t q = patch_pixel(g, centre, subset[i / ch]);
      if (mask && !mask[q]) continue;
      float xc = grid[q * ch + i % ch] - mean32[i];
      acc = std::fma(basis[(size_t)i * D + k], xc, acc);
    }
    y[k] = acc;
  }
}

void or_project(const float* grid, int ndim, const int64_t* ext, int ch, int K, const int64_t* dict, int64_t N,
                const int32_t* subset, int m, const float* basis, const float* mean32, int D, float* y) {
  for (int64_t j = 0; j < N; ++j)
    or_project_one(grid, nullptr, ndim, ext, ch, K, dict[j], subset, m, basis, mean32, D, y + (size_t)j * D);
}

// ----------------------------------------------------------------------------
// Quantisation of principal coordinates (Sec. II.C: the listings compare byte
// coordinates).  Reading: per dimension lo = min, hi = max over the N dictionary
// projections (as real values: a zero is stored as +0); scale = (float)(2^b / ((double)hi - (double)lo)), or 0 when
// hi == lo; q = clamp(floor((y - lo) * scale), 0, 2^b - 1) with the subtraction
// and the product each rounded to FP32.  Queries reuse lo/scale and the clamp.
// ----------------------------------------------------------------------------
void or_quant_params(const float* y, int64_t N, int D, int bits, float* lo, float* scale) {
  for (int k = 0; k < D; ++k) {
    float mn = INFINITY, mx = -INFINITY;
    for (int64_t j = 0; j < N; ++j) {
      float v = y[(size_t)j * D + k];
      if (v < mn) mn = v;
      if (v > mx) mx = v;
    }
    if (mn == 0.0f) mn = 0.0f;  // the real value zero: stored as +0
    if (mx == 0.0f) mx = 0.0f;
    lo[k] = mn;
    scale[k] = mx > mn ? (float)(std::ldexp(1.0, bits) / ((double)mx - (double)mn)) : 0.0f;
  }
}

uint32_t or_quantise_one(float y, float lo, float scale, int bits) {
  float t = y - lo;
  float u = t * scale;
  double f = std::floor((double)u);
  double top = std::ldexp(1.0, bits) - 1.0;
  if (!(f >= 0.0)) f = 0.0;  // also catches NaN
  if (f > top) f = top;
  return (uint32_t)f;
}

void or_quantise(const float* y, int64_t N, int D, int bits, const float* lo, const float* scale, uint32_t* q) {
  for (int64_t j = 0; j < N; ++j)
    for (int k = 0; k < D; ++k) q[(size_t)j * D + k] = or_quantise_one(y[(size_t)j * D + k], lo[k], scale[k], bits);
}

// ----------------------------------------------------------------------------
// Morton / z-address (Sec. II.C): interleave the coordinate bits, highest bit
// plane first, dimension 0 first inside a plane.  Reading: with D * bp <= 64 the
// key is that D*bp-bit number; otherwise it is its top 64 bits (the first 64
// bits emitted).  Shifted curves (optional, default none): q' = q + shift[k] and
// one more bit per coordinate (bp = b + 1) whenever any shift is non-zero.
// ----------------------------------------------------------------------------
uint64_t or_morton(const uint32_t* q, int D, int bp) {
  uint64_t key = 0;
  int n = 0;
  for (int p = bp - 1; p >= 0; --p)
    for (int k = 0; k < D; ++k) {
      if (n == 64) return key;
      key = (key << 1) | (uint64_t)((q[k] >> p) & 1u);
      ++n;
    }
  return key;
}

// ----------------------------------------------------------------------------
// Hilbert keys (the alternative curve of the 3-D configuration; not in the
// paper, which uses the z-curve): Skilling's transpose method ("Programming the
// Hilbert curve", AIP Conf. Proc. 707, 2004).  The D coordinates of bp bits are
// turned in place into the "transposed" Hilbert index -- the index whose bits,
// read plane by plane from the top with dimension 0 first, are the Hilbert
// position -- by (1) walking the bit planes from the top: below the current
// plane, either invert the low bits of coordinate 0 (the current bit of
// coordinate i is set) or swap the low bits of coordinates 0 and i (it is
// clear), which undoes the rotations and reflections of the sub-cubes; (2) a
// Gray code across the dimensions (each coordinate xor the previous one); (3)
// xor every coordinate with the mask collecting, per plane, whether the last
// coordinate's bit there is set (as the low-bit mask of that plane).  The key is
// then interleaved exactly like the Morton key (or_morton).
// ----------------------------------------------------------------------------
uint64_t or_hilbert(const uint32_t* q, int D, int bp) {
  std::vector<uint32_t> x(q, q + D);
  const uint32_t top = 1u << (bp - 1);
  for (uint32_t plane = top; plane > 1; plane >>= 1) {
    const uint32_t low = plane - 1;
    for (int i = 0; i < D; ++i) {
      if (x[i] & plane) {
        x[0] ^= low;
      } else {
        const uint32_t diff = (x[0] ^ x[i]) & low;
        x[0] ^= diff;
        x[i] ^= diff;
      }
    }
  }
  for (int i = 1; i < D; ++i) x[i] ^= x[i - 1];
  uint32_t flip = 0;
  for (uint32_t plane = top; plane > 1; plane >>= 1)
    if (x[D - 1] & plane) flip ^= plane - 1;
  for (int i = 0; i < D; ++i) x[i] ^= flip;
  return or_morton(x.data(), D, bp);
}

int or_key_bits(int D, int bits, const int32_t* shift) {
  int bp = bits;
  if (shift)
    for (int k = 0; k < D; ++k)
      if (shift[k] != 0) bp = bits + 1;
  return bp;
}

// curve: 0 = Morton (z-curve, Sec. II.C), 1 = Hilbert (or_hilbert)
uint64_t or_curve_key(const uint32_t* q, int D, int bp, int curve) {
  return curve == 1 ? or_hilbert(q, D, bp) : or_morton(q, D, bp);
}

void or_keys_curve(const uint32_t* q, int64_t N, int D, int bits, const int32_t* shift, int curve, uint64_t* keys) {
  int bp = or_key_bits(D, bits, shift);
  std::vector<uint32_t> t(D);
  for (int64_t j = 0; j < N; ++j) {
    for (int k = 0; k < D; ++k) t[k] = q[(size_t)j * D + k] + (uint32_t)(shift ? shift[k] : 0);
    keys[j] = or_curve_key(t.data(), D, bp, curve);
  }
}

void or_keys(const uint32_t* q, int64_t N, int D, int bits, const int32_t* shift, uint64_t* keys) {
  or_keys_curve(q, N, D, bits, shift, 0, keys);
}

// z-order comparison of two quantised points without forming their keys
// (Sec. II.C).  The curve reads bit planes from the top and, inside a plane,
// dimension 0 first, so the first bit at which the two interleaved keys differ
// is owned by the dimension whose coordinate difference reaches the highest
// bit position; among dimensions that reach the same position the lowest one
// is read first.  That dimension's coordinates decide the order.
int or_zless(const uint32_t* a, const uint32_t* b, int D) {
  int owner = -1, top = -1;
  for (int d = 0; d < D; ++d) {
    const uint32_t x = a[d] ^ b[d];
    if (x == 0) continue;
    const int h = 31 - __builtin_clz(x);  // highest differing bit of this axis
    if (h > top) {                        // strictly higher: ties keep the lower axis
      top = h;
      owner = d;
    }
  }
  if (owner < 0) return 0;  // equal points
  return a[owner] < b[owner] ? 1 : 0;
}

// Sort of the dictionary by z-order (Sec. II.C).  Reading: a stable sort of the
// (key, id) pairs starting from id order, i.e. by key, then by id.
void or_sort(const uint64_t* keys, int64_t N, uint64_t* skeys, uint32_t* sids) {
  std::vector<uint32_t> id(N);
  std::iota(id.begin(), id.end(), 0u);
  std::stable_sort(id.begin(), id.end(), [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
  for (int64_t i = 0; i < N; ++i) {
    sids[i] = id[i];
    skeys[i] = keys[id[i]];
  }
}

// Binary search on the sorted z-array (Sec. II.B): number of keys < key.
int64_t or_lower_bound(const uint64_t* skeys, int64_t N, uint64_t key) {
  int64_t lo = 0, hi = N;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (skeys[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// ----------------------------------------------------------------------------
// One SFC query (Fig. 1(b)-(d)).  Readings:
//  * index selection: select == 1 ("best"): the single index covering the most
//    known subset pixels, ties to the lowest index; select == 0 ("all"): every
//    index;
//  * query key: projection with unknown values skipped, the dictionary's lo/scale
//    with clamping, shift, Morton;
//  * the paper's k-NN list is replaced by a window of W sorted slots around the
//    lower_bound position: start = clamp(pos - W/2, 0, max(0, N - W)), length
//    min(W, N);
//  * candidates = sorted union of the windows' ids; every candidate is rescored
//    with the exact image-space cost, argmin with ties to the lowest id.
// Arrays are per index, concatenated: subset[C*m], basis[C*s*D], mean[C*s],
// lo/scale[C*D], shift[C*D] (or NULL), skeys/sids[C*N].
// Outputs: qkeys[C], pos[C] (0 / -1 for unselected indices), cand (<= C*W ids),
// *ncand, *pick (-1 if there is no candidate), *cost.
// ----------------------------------------------------------------------------
void or_query_curve(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K, int C,
                    int D, int bits, int W, int select, const float* w, const int32_t* subset, int m,
                    const float* basis, const float* mean32, const float* lo, const float* scale,
                    const int32_t* shift, int curve, const uint64_t* skeys, const uint32_t* sids, const int64_t* dict,
                    int64_t N, int64_t target, uint64_t* qkeys, int64_t* pos, int64_t* cand, int64_t* ncand,
                    int64_t* pick, double* cost, int norm);

void or_query(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K, int C,
              int D, int bits, int W, int select, const float* w, const int32_t* subset, int m, const float* basis,
              const float* mean32, const float* lo, const float* scale, const int32_t* shift, const uint64_t* skeys,
              const uint32_t* sids, const int64_t* dict, int64_t N, int64_t target, uint64_t* qkeys, int64_t* pos,
              int64_t* cand, int64_t* ncand, int64_t* pick, double* cost) {
  or_query_curve(grid, cur_mask, ndim, ext, ch, K, C, D, bits, W, select, w, subset, m, basis, mean32, lo, scale,
                 shift, 0, skeys, sids, dict, N, target, qkeys, pos, cand, ncand, pick, cost, 0);
}

// The same query on indices keyed by `curve` (0 Morton, 1 Hilbert), with the
// cost norm `norm` (0 L2, 1 L1).
void or_query_curve(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K, int C,
                    int D, int bits, int W, int select, const float* w, const int32_t* subset, int m,
                    const float* basis, const float* mean32, const float* lo, const float* scale,
                    const int32_t* shift, int curve, const uint64_t* skeys, const uint32_t* sids, const int64_t* dict,
                    int64_t N, int64_t target, uint64_t* qkeys, int64_t* pos, int64_t* cand, int64_t* ncand,
                    int64_t* pick, double* cost, int norm) {
  Geo g = make_geo(ndim, ext, ch, K);
  const int s = m * ch;
  std::vector<int> use;
  if (select == 1) {
    int best = 0, bestcov = -1;
    for (int cv = 0; cv < C; ++cv) {
      int cov = 0;
      for (int i = 0; i < m; ++i) cov += cur_mask[patch_pixel(g, target, subset[cv * m + i])] ? 1 : 0;
      if (cov > bestcov) {
        bestcov = cov;
        best = cv;
      }
    }
    use.push_back(best);
  } else {
    for (int cv = 0; cv < C; ++cv) use.push_back(cv);
  }
  std::vector<int64_t> ids;
  for (int cv = 0; cv < C; ++cv) {
    qkeys[cv] = 0;
    pos[cv] = -1;
  }
  std::vector<float> y(D);
  std::vector<uint32_t> qq(D);
  for (int cv : use) {
    or_project_one(grid, cur_mask, ndim, ext, ch, K, target, subset + (size_t)cv * m, m,
                   basis + (size_t)cv * s * D, mean32 + (size_t)cv * s, D, y.data());
    const int32_t* sh = shift ? shift + (size_t)cv * D : nullptr;
    for (int k = 0; k < D; ++k)
      qq[k] = or_quantise_one(y[k], lo[cv * D + k], scale[cv * D + k], bits) + (uint32_t)(sh ? sh[k] : 0);
    uint64_t key = or_curve_key(qq.data(), D, or_key_bits(D, bits, sh), curve);
    qkeys[cv] = key;
    int64_t p = or_lower_bound(skeys + (size_t)cv * N, N, key);
    pos[cv] = p;
    int64_t len = W < N ? W : N;
    int64_t start = p - W / 2;
    int64_t maxs = N - W > 0 ? N - W : 0;
    if (start > maxs) start = maxs;
    if (start < 0) start = 0;
    for (int64_t i = start; i < start + len; ++i) ids.push_back(sids[(size_t)cv * N + i]);
  }
  sort_unique(ids);
  for (size_t i = 0; i < ids.size(); ++i) cand[i] = ids[i];
  *ncand = (int64_t)ids.size();
  double best = INFINITY;
  int64_t bj = -1;
  for (int64_t j : ids) {
    double c = cost64(g, grid, cur_mask, target, dict[j], w, norm);
    if (c < best) {
      best = c;
      bj = j;
    }
  }
  *pick = bj;
  *cost = best;
}

// ----------------------------------------------------------------------------
// Exact k-NN in the quantised principal space by brute force: the result the
// paper's outside-in search (Sec. II.D) returns exactly.  Squared Euclidean
// distance between integer coordinates (exact in int64), ties by id; out[k].
// ----------------------------------------------------------------------------
void or_knn_bruteforce(const uint32_t* qcoords, int64_t N, int D, const uint32_t* query, int k, int64_t* out,
                       int64_t* dist) {
  std::vector<std::pair<int64_t, int64_t>> d(N);
  for (int64_t j = 0; j < N; ++j) {
    int64_t acc = 0;
    for (int a = 0; a < D; ++a) {
      int64_t t = (int64_t)qcoords[(size_t)j * D + a] - (int64_t)query[a];
      acc += t * t;
    }
    d[j] = {acc, j};
  }
  int kk = (int)std::min<int64_t>(k, N);
  std::partial_sort(d.begin(), d.begin() + kk, d.end());
  for (int i = 0; i < kk; ++i) {
    out[i] = d[i].second;
    dist[i] = d[i].first;
  }
}

// ----------------------------------------------------------------------------
// One SFC query with the paper's exact k-NN lists (Sec. II.D) in place of the
// window: per selected index, the k dictionary entries nearest to the query in
// the quantised principal space (squared Euclidean distance between the
// integer coordinates, ties by id -- the set or_knn_bruteforce returns); the
// candidates are the sorted union of those lists, rescored with the exact
// image-space cost as in or_query.  Index selection, projection and
// quantisation (clamped) as in or_query; distances use unshifted coordinates
// (a common shift leaves them unchanged).
// qc[C*N*D]: quantised, unshifted coordinates of every dictionary entry.
// Outputs: cand (<= C*k ids), *ncand, *pick (-1 if no candidate), *cost.
// ----------------------------------------------------------------------------
void or_query_knn(const float* grid, const uint8_t* cur_mask, int ndim, const int64_t* ext, int ch, int K, int C,
                  int D, int bits, int k, int select, const float* w, const int32_t* subset, int m,
                  const float* basis, const float* mean32, const float* lo, const float* scale, const uint32_t* qc,
                  const int64_t* dict, int64_t N, int64_t target, int64_t* cand, int64_t* ncand, int64_t* pick,
                  double* cost, int norm) {
  Geo g = make_geo(ndim, ext, ch, K);
  const int s = m * ch;
  std::vector<int> use;
  if (select == 1) {
    int best = 0, bestcov = -1;
    for (int cv = 0; cv < C; ++cv) {
      int cov = 0;
      for (int i = 0; i < m; ++i) cov += cur_mask[patch_pixel(g, target, subset[cv * m + i])] ? 1 : 0;
      if (cov > bestcov) {
        bestcov = cov;
        best = cv;
      }
    }
    use.push_back(best);
  } else {
    for (int cv = 0; cv < C; ++cv) use.push_back(cv);
  }
  std::vector<int64_t> ids;
  std::vector<float> y(D);
  std::vector<uint32_t> qq(D);
  const int kk = (int)std::min<int64_t>(k, N);
  std::vector<int64_t> nn(kk), dd(kk);
  for (int cv : use) {
    or_project_one(grid, cur_mask, ndim, ext, ch, K, target, subset + (size_t)cv * m, m,
                   basis + (size_t)cv * s * D, mean32 + (size_t)cv * s, D, y.data());
    for (int a = 0; a < D; ++a) qq[a] = or_quantise_one(y[a], lo[cv * D + a], scale[cv * D + a], bits);
    or_knn_bruteforce(qc + (size_t)cv * N * D, N, D, qq.data(), k, nn.data(), dd.data());
    for (int i = 0; i < kk; ++i) ids.push_back(nn[i]);
  }
  sort_unique(ids);
  for (size_t i = 0; i < ids.size(); ++i) cand[i] = ids[i];
  *ncand = (int64_t)ids.size();
  double best = INFINITY;
  int64_t bj = -1;
  for (int64_t j : ids) {
    double c = cost64(g, grid, cur_mask, target, dict[j], w, norm);
    if (c < best) {
      best = c;
      bj = j;
    }
  }
  *pick = bj;
  *cost = best;
}

// ----------------------------------------------------------------------------
// Queries against an index built on another grid (a stored dictionary, Sec.
// II.H: the index is built once and reused): the target patch lives in tgrid /
// tmask (geometry gt), the dictionary patches in dgrid (geometry gd, the
// index's); same channels and patch size.  cost64_2 is cost64 with the two
// patches taken from different grids (same element order and arithmetic).
// ----------------------------------------------------------------------------
double cost64_2(const Geo& gt, const float* tgrid, const uint8_t* tmask, int64_t t, const Geo& gd,
                const float* dgrid, int64_t s, const float* w, int norm) {
  double acc = 0.0;
  for (int pp = 0; pp < gt.P; ++pp) {
    int64_t qt = patch_pixel(gt, t, pp);
    if (!tmask[qt]) continue;
    int64_t qs = patch_pixel(gd, s, pp);
    for (int c = 0; c < gt.ch; ++c) {
      double d = (double)tgrid[qt * gt.ch + c] - (double)dgrid[qs * gd.ch + c];
      double term = norm == 1 ? std::fabs(d) : d * d;
      double wc = w ? (double)w[c] : 1.0;
      acc = acc + wc * term;
    }
  }
  return acc;
}

double or_cost64_2(const float* tgrid, const uint8_t* tmask, int tndim, const int64_t* text, const float* dgrid,
                   const int64_t* dext, int ch, int K, int64_t target, int64_t source, const float* w, int norm) {
  Geo gt = make_geo(tndim, text, ch, K), gd = make_geo(tndim, dext, ch, K);
  return cost64_2(gt, tgrid, tmask, target, gd, dgrid, source, w, norm);
}

// or_query_curve with the target in (tgrid, tmask, text) and the dictionary
// patches in (dgrid, dext); `target` is a linear pixel index of the target grid.
void or_query_dict(const float* dgrid, const int64_t* dext, const float* tgrid, const uint8_t* tmask,
                   const int64_t* text, int ndim, int ch, int K, int C, int D, int bits, int W, int select,
                   const float* w, const int32_t* subset, int m, const float* basis, const float* mean32,
                   const float* lo, const float* scale, const int32_t* shift, int curve, const uint64_t* skeys,
                   const uint32_t* sids, const int64_t* dict, int64_t N, int64_t target, int64_t* cand,
                   int64_t* ncand, int64_t* pick, double* cost, int norm) {
  Geo gt = make_geo(ndim, text, ch, K), gd = make_geo(ndim, dext, ch, K);
  const int s = m * ch;
  std::vector<int> use;
  if (select == 1) {
    int best = 0, bestcov = -1;
    for (int cv = 0; cv < C; ++cv) {
      int cov = 0;
      for (int i = 0; i < m; ++i) cov += tmask[patch_pixel(gt, target, subset[cv * m + i])] ? 1 : 0;
      if (cov > bestcov) {
        bestcov = cov;
        best = cv;
      }
    }
    use.push_back(best);
  } else {
    for (int cv = 0; cv < C; ++cv) use.push_back(cv);
  }
  std::vector<int64_t> ids;
  std::vector<float> y(D);
  std::vector<uint32_t> qq(D);
  for (int cv : use) {
    // the projection of the target's known subset values (or_project_one on the target grid)
    or_project_one(tgrid, tmask, ndim, text, ch, K, target, subset + (size_t)cv * m, m, basis + (size_t)cv * s * D,
                   mean32 + (size_t)cv * s, D, y.data());
    const int32_t* sh = shift ? shift + (size_t)cv * D : nullptr;
    for (int k = 0; k < D; ++k)
      qq[k] = or_quantise_one(y[k], lo[cv * D + k], scale[cv * D + k], bits) + (uint32_t)(sh ? sh[k] : 0);
    const uint64_t key = or_curve_key(qq.data(), D, or_key_bits(D, bits, sh), curve);
    const int64_t p = or_lower_bound(skeys + (size_t)cv * N, N, key);
    const int64_t len = W < N ? W : N;
    int64_t start = p - W / 2;
    const int64_t maxs = N - W > 0 ? N - W : 0;
    if (start > maxs) start = maxs;
    if (start < 0) start = 0;
    for (int64_t i = start; i < start + len; ++i) ids.push_back(sids[(size_t)cv * N + i]);
  }
  sort_unique(ids);
  for (size_t i = 0; i < ids.size(); ++i) cand[i] = ids[i];
  *ncand = (int64_t)ids.size();
  double best = INFINITY;
  int64_t bj = -1;
  for (int64_t j : ids) {
    double c = cost64_2(gt, tgrid, tmask, target, gd, dgrid, dict[j], w, norm);
    if (c < best) {
      best = c;
      bj = j;
    }
  }
  *pick = bj;
  *cost = best;
}

// Priority of a candidate centre c (reading of the fill order that the paper
// takes from Criminisi et al., Sec. I and Sec. II.G).  terms[0] = confidence
// C(p): the patch's confidence values summed one by one in patch raster order
// (FP32), divided by K^dim.  With prio == 1 (2-D only) the data term follows:
// terms[1], terms[2] = the grey gradient (g_x, g_y), grey = channel mean (summed
// left to right, divided by ch); each component is the central difference
// 0.5 (I(+1) - I(-1)) when both axis neighbours are known, the one-sided
// difference towards the known neighbour when only one is known and the centre
// itself is known, else 0 (out of the grid counts as unknown).  terms[3],
// terms[4] = the unit normal n of the fill front: the central-difference
// gradient of the mask as 0/1 (out of the grid counts as 1 = known), divided by
// its IEEE sqrtf norm, or (0, 0) when the norm is 0.  terms[5] = the data term
// D(p) = |(-g_y) n_x + g_x n_y| (the isophote, the gradient turned by 90
// degrees, against the normal; alpha = 1).  terms[6] = the priority: C(p) for
// prio == 0, C(p) (D(p) + 0.001) for prio == 1.  Every product and sum is
// rounded separately (no fused multiply-add).
static void prio_terms(const Geo& g, const float* grid, const uint8_t* mask, const float* conf, int64_t c, int prio,
                       float* terms) {
  float sum = 0.0f;
  for (int pp = 0; pp < g.P; ++pp) sum = sum + conf[patch_pixel(g, c, pp)];
  const float Ct = sum / (float)g.P;
  for (int i = 0; i < 7; ++i) terms[i] = 0.0f;
  terms[0] = Ct;
  terms[6] = Ct;
  if (prio != 1) return;
  auto known_at = [&](int64_t x, int64_t y) -> bool {
    if (x < 0 || y < 0 || x >= g.X || y >= g.Y) return false;
    return mask[lin_of(g, x, y, 0)] != 0;
  };
  auto gray = [&](int64_t q) -> float {
    if (g.ch == 1) return grid[q];
    float acc = grid[q * g.ch];
    for (int k = 1; k < g.ch; ++k) acc = acc + grid[q * g.ch + k];
    return acc / (float)g.ch;
  };
  auto mval = [&](int64_t x, int64_t y) -> float {
    if (x < 0 || y < 0 || x >= g.X || y >= g.Y) return 1.0f;
    return mask[lin_of(g, x, y, 0)] ? 1.0f : 0.0f;
  };
  int64_t cc[3];
  coords_of(g, c, cc);
  const int64_t x = cc[0], y = cc[1];
  const bool kc = mask[c] != 0;
  float gxy[2];
  for (int a = 0; a < 2; ++a) {
    const int64_t x0 = x - (a == 0), y0 = y - (a == 1), x1 = x + (a == 0), y1 = y + (a == 1);
    const bool k0 = known_at(x0, y0), k1 = known_at(x1, y1);
    float gv = 0.0f;
    if (k0 && k1)
      gv = 0.5f * (gray(lin_of(g, x1, y1, 0)) - gray(lin_of(g, x0, y0, 0)));
    else if (kc && k1)
      gv = gray(lin_of(g, x1, y1, 0)) - gray(c);
    else if (kc && k0)
      gv = gray(c) - gray(lin_of(g, x0, y0, 0));
    gxy[a] = gv;
  }
  const float mx = 0.5f * (mval(x + 1, y) - mval(x - 1, y));
  const float my = 0.5f * (mval(x, y + 1) - mval(x, y - 1));
  const float mx2 = mx * mx;
  const float my2 = my * my;
  const float nrm = std::sqrt(mx2 + my2);
  float nx = 0.0f, ny = 0.0f;
  if (nrm > 0.0f) {
    nx = mx / nrm;
    ny = my / nrm;
  }
  const float t1 = (-gxy[1]) * nx;
  const float t2 = gxy[0] * ny;
  const float Dt = std::fabs(t1 + t2);
  terms[1] = gxy[0];
  terms[2] = gxy[1];
  terms[3] = nx;
  terms[4] = ny;
  terms[5] = Dt;
  terms[6] = Ct * (Dt + 0.001f);
}

// The priority terms of one centre, exposed for tests (conf: npix floats, or
// NULL = 1 on known pixels and 0 on unknown ones).  Returns -1 for an invalid
// centre and -2 for prio == 1 outside 2-D.
int or_priority(const float* grid, const uint8_t* mask, const float* conf, int ndim, const int64_t* ext, int ch,
                int K, int64_t centre, int prio, float* terms) {
  Geo g = make_geo(ndim, ext, ch, K);
  if (prio == 1 && ndim != 2) return -2;
  if (centre < 0 || centre >= g.X * g.Y * g.Z) return -1;
  int64_t cc[3];
  coords_of(g, centre, cc);
  if (!centre_valid(g, cc[0], cc[1], cc[2])) return -1;
  std::vector<float> own;
  if (!conf) {
    own.resize(g.X * g.Y * g.Z);
    for (size_t i = 0; i < own.size(); ++i) own[i] = mask[i] ? 1.0f : 0.0f;
    conf = own.data();
  }
  prio_terms(g, grid, mask, conf, centre, prio, terms);
  return 0;
}

// ----------------------------------------------------------------------------
// Inpainting loop (Sec. I; Fig. 1(a)).  Readings:
//  * fill front: known pixels with an unknown axis-neighbour (4-/6-connected);
//    a target centre is a front pixel moved into [r, ext-1-r] per axis (the
//    adjacent unknown pixel stays inside the patch); equal centres merge;
//  * priority (the paper defers to Criminisi et al.):
//      prio == 0 (confidence / onion peel): P = Cterm = (sum of confidence over
//        the patch, FP32, raster order) / K^dim;
//      prio == 1 (Criminisi, 2-D): P = Cterm * (Dterm + 0.001), Dterm =
//        |(-gy) nx + gx ny| with (gx, gy) the gradient of the grey value (mean
//        of channels) by central differences over known neighbours (one-sided
//        when one side is unknown, 0 when both are), n the normalised
//        central-difference gradient of the known-mask (outside the grid counts
//        as known); every product and sum rounded separately;
//    argmax, ties to the lowest linear centre index;
//  * search: mode 0 = full scan, mode 1 = SFC query (arrays as in or_query);
//  * insert: copy the source patch into the target's unknown pixels only, mark
//    them known, give them confidence Cterm of the target;
//  * stop when no pixel is unknown, or after max_steps (> 0).
// log (may be NULL) receives per step ndim centre coordinates then the pick id.
// confidence (optional in/out, npix floats): NULL = start from the mask.
// norm: the cost of the search (0 L2, 1 L1, as cost64).
// Returns the number of steps; -1 when the dictionary is empty and pixels are
// unknown; -2 for an unsupported priority.
// ----------------------------------------------------------------------------
int64_t or_inpaint(float* grid, uint8_t* mask, int ndim, const int64_t* ext, int ch, int K, int mode, int prio,
                   const float* w, const int64_t* dict, int64_t N, int C, int D, int bits, int W, int select,
                   const int32_t* subset, int m, const float* basis, const float* mean32, const float* lo,
                   const float* scale, const int32_t* shift, const uint64_t* skeys, const uint32_t* sids,
                   int64_t max_steps, int64_t* log, int norm, int knn, const uint32_t* qc) {
  Geo g = make_geo(ndim, ext, ch, K);
  const int64_t npix = g.X * g.Y * g.Z;
  if (prio == 1 && ndim != 2) return -2;
  if (mode == 1 && knn > 0 && !qc) return -3;
  std::vector<float> conf(npix);
  for (int64_t i = 0; i < npix; ++i) conf[i] = mask[i] ? 1.0f : 0.0f;
  int64_t steps = 0;
  std::vector<uint8_t> is_centre(npix);
  std::vector<int64_t> cands;
  std::vector<uint64_t> qkeys(C > 0 ? C : 1);
  std::vector<int64_t> pos(C > 0 ? C : 1), cand((size_t)(C > 0 ? C : 1) * std::max(W > 0 ? W : 1, knn > 0 ? knn : 1));
  while (max_steps <= 0 || steps < max_steps) {
    // front and candidate centres
    std::fill(is_centre.begin(), is_centre.end(), 0);
    bool any_unknown = false;
    for (int64_t z = 0; z < g.Z; ++z)
      for (int64_t y = 0; y < g.Y; ++y)
        for (int64_t x = 0; x < g.X; ++x) {
          int64_t q = lin_of(g, x, y, z);
          if (!mask[q]) {
            any_unknown = true;
            continue;
          }
          bool front = false;
          const int64_t nb[6][3] = {{x - 1, y, z}, {x + 1, y, z}, {x, y - 1, z},
                                    {x, y + 1, z}, {x, y, z - 1}, {x, y, z + 1}};
          for (int a = 0; a < 2 * ndim; ++a) {
            int64_t nx = nb[a][0], ny = nb[a][1], nz = nb[a][2];
            if (nx < 0 || ny < 0 || nz < 0 || nx >= g.X || ny >= g.Y || nz >= g.Z) continue;
            if (!mask[lin_of(g, nx, ny, nz)]) front = true;
          }
          if (!front) continue;
          int64_t cx = std::min(std::max<int64_t>(x, g.r), g.X - 1 - g.r);
          int64_t cy = std::min(std::max<int64_t>(y, g.r), g.Y - 1 - g.r);
          int64_t cz = ndim == 3 ? std::min(std::max<int64_t>(z, g.r), g.Z - 1 - g.r) : 0;
          is_centre[lin_of(g, cx, cy, cz)] = 1;
        }
    if (!any_unknown) break;
    if (N <= 0) return -1;
    float bestP = -1.0f;
    int64_t bestc = -1;
    float bestC = 0.0f;
    for (int64_t c = 0; c < npix; ++c) {
      if (!is_centre[c]) continue;
      float terms[7];
      prio_terms(g, grid, mask, conf.data(), c, prio, terms);
      const float P = terms[6];
      if (P > bestP) {
        bestP = P;
        bestc = c;
        bestC = terms[0];
      }
    }
    int64_t j;
    double cst;
    if (mode == 0) {
      or_fullscan(grid, mask, ndim, ext, ch, K, dict, N, &bestc, 1, w, &j, &cst, norm);
    } else {
      int64_t nc;
      if (knn > 0)  // candidates = the exact k-NN lists of the query (Sec. II.D)
        or_query_knn(grid, mask, ndim, ext, ch, K, C, D, bits, knn, select, w, subset, m, basis, mean32, lo, scale,
                     qc, dict, N, bestc, cand.data(), &nc, &j, &cst, norm);
      else
        or_query_curve(grid, mask, ndim, ext, ch, K, C, D, bits, W, select, w, subset, m, basis, mean32, lo, scale,
                       shift, 0, skeys, sids, dict, N, bestc, qkeys.data(), pos.data(), cand.data(), &nc, &j, &cst,
                       norm);
    }
    int64_t src = dict[j];
    for (int pp = 0; pp < g.P; ++pp) {
      int64_t qt = patch_pixel(g, bestc, pp);
      if (mask[qt]) continue;
      int64_t qs = patch_pixel(g, src, pp);
      for (int c = 0; c < ch; ++c) grid[qt * ch + c] = grid[qs * ch + c];
      mask[qt] = 1;
      conf[qt] = bestC;
    }
    if (log) {
      int64_t cc[3];
      coords_of(g, bestc, cc);
      for (int a = 0; a < ndim; ++a) log[steps * (ndim + 1) + a] = cc[a];
      log[steps * (ndim + 1) + ndim] = j;
    }
    ++steps;
  }
  return steps;
}

}  // extern "C"
