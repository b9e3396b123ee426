// Index construction on the GPU (Algorithm 1 of the paper).
//
//  1. PCA (Algorithm 1, PCA training and residual variances):
//     float64 column mean and covariance (1/N) of the base, then a float64
//     parallel cyclic Jacobi eigendecomposition (round-robin pairing, one
//     launch computes all n/2 rotation angles of a round, one launch applies
//     them to A and to the eigenvector matrix).  Eigenvalues are sorted in
//     descending order; each eigenvector's largest-magnitude entry is made
//     positive.
//  2. Random orthogonal P_r: float64 modified Gram-Schmidt (two passes) on a
//     d x d Gaussian draw, i.e. the Q of G = QR with diag(R) > 0.
//  3. W = [P_r^T P_p[:d]; P_p[d:]] (float64 product, stored float32): one GEMM
//     gives a centred vector's rotated lead part x_d' and its tail x_r.
//  4. Base projection, k-means (Lloyd, float32 distances, float64 sums) on
//     x_d' (IVF on the projected vectors, Exp-6), list-major reordering (stable
//     radix sort by list), quantization of o' = (x_d' - c')/|x_d' - c'| and the
//     per-vector factors of Eq. 4 / Eq. 5.
//  5. Device layout: every list padded to a multiple of 32 vectors; codes stored
//     as bit planes, 32-vector blocks interleaved so that one warp reads the
//     same word of 32 consecutive vectors in one coalesced transaction.
#include <cub/cub.cuh>

#include <algorithm>
#include <cmath>
#include <numeric>
#include <unordered_map>

#include "common.cuh"

namespace mrq {
namespace {

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// SplitMix64 (Steele, Lea, Flood 2014): the library's own counter-based draws.
struct SplitMix64 {
  uint64_t s;
  uint64_t next() {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }  // (0,1)
  double gauss() {  // Box-Muller
    double u1 = uniform(), u2 = uniform();
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
  }
};

// ------------------------------------------------------------ mean / covariance

// rows[i] of X (n x D) into row i of out (one CTA per row)
__global__ void k_gather_rows(const float* __restrict__ X, int D, const int64_t* __restrict__ rows,
                              int64_t nrows, float* __restrict__ out) {
  const int64_t i = blockIdx.x;
  if (i >= nrows) return;
  const float* src = X + rows[i] * (int64_t)D;
  for (int c = threadIdx.x; c < D; c += blockDim.x) out[i * D + c] = src[c];
}

__global__ void k_colsum(const float* __restrict__ X, int64_t n, int D, int64_t rows_per,
                         double* __restrict__ sum) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= D) return;
  int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = min(n, r0 + rows_per);
  double s = 0.0;
  for (int64_t r = r0; r < r1; ++r) s += (double)X[r * D + c];
  atomicAdd(&sum[c], s);
}

__global__ void k_scale_d(double* a, int64_t n, double f) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] *= f;
}

// Upper-triangular 64x64 tiles of (X - mu)^T (X - mu), float64, one row chunk
// per blockIdx.y, partial tiles accumulated with float64 atomics.
constexpr int CT = 64, CR = 16;
__global__ void __launch_bounds__(256) k_cov(const float* __restrict__ X, int64_t n, int D,
                                             const double* __restrict__ mu,
                                             const int2* __restrict__ tiles, int64_t rows_per,
                                             double* __restrict__ C) {
  __shared__ double Ai[CR][CT + 1], Aj[CR][CT + 1];
  const int2 t = tiles[blockIdx.x];
  const int i0 = t.x * CT, j0 = t.y * CT;
  const int tid = threadIdx.x, ti = tid >> 4, tj = tid & 15;
  int64_t r0 = (int64_t)blockIdx.y * rows_per, r1 = min(n, r0 + rows_per);
  double acc[4][4] = {};
  for (int64_t rb = r0; rb < r1; rb += CR) {
    for (int e = tid; e < CR * CT; e += 256) {
      int rr = e / CT, cc = e % CT;
      int64_t r = rb + rr;
      double vi = 0.0, vj = 0.0;
      if (r < r1) {
        if (i0 + cc < D) vi = (double)X[r * D + i0 + cc] - mu[i0 + cc];
        if (j0 + cc < D) vj = (double)X[r * D + j0 + cc] - mu[j0 + cc];
      }
      Ai[rr][cc] = vi;
      Aj[rr][cc] = vj;
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < CR; ++rr) {
      double a[4], b[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) { a[u] = Ai[rr][ti + 16 * u]; b[u] = Aj[rr][tj + 16 * u]; }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      int i = i0 + ti + 16 * u, j = j0 + tj + 16 * v;
      if (i < D && j < D) atomicAdd(&C[(int64_t)i * D + j], acc[u][v]);
    }
}

// Copy cov (D x D, upper tiles filled) into the padded m x m Jacobi matrix,
// mirroring the upper triangle into the lower one and scaling by 1/n.
__global__ void k_cov_to_jacobi(const double* __restrict__ C, int D, int m, double inv_n,
                                double* __restrict__ A, double* __restrict__ V) {
  int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= m) return;
  double v = 0.0;
  if (i < D && j < D) v = C[(int64_t)min(i, j) * D + max(i, j)] * inv_n;  // exactly symmetric
  A[(int64_t)i * m + j] = v;
  V[(int64_t)i * m + j] = (i == j) ? 1.0 : 0.0;
}

// ------------------------------------------------------------------ Jacobi

// Round-robin (circle method) pairing: position 0 is fixed, the others rotate.
__device__ __forceinline__ int rr_player(int pos, int round, int m) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (m - 1);
}

__global__ void k_jacobi_angles(const double* __restrict__ A, int m, int round,
                                int* __restrict__ partner, double* __restrict__ cself,
                                double* __restrict__ cpart) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m / 2) return;
  int a = rr_player(i, round, m), b = rr_player(m - 1 - i, round, m);
  int p = min(a, b), q = max(a, b);
  double app = A[(int64_t)p * m + p], aqq = A[(int64_t)q * m + q], apq = A[(int64_t)p * m + q];
  double c = 1.0, s = 0.0;
  if (fabs(apq) > 1e-300 && fabs(apq) > 1e-18 * (fabs(app) + fabs(aqq))) {
    // rotation zeroing A[p][q]: t = tan(theta) is the smaller root of t^2 + 2 tau t - 1 = 0
    double tau = (aqq - app) / (2.0 * apq);
    double t;
    if (fabs(tau) > 1e150)
      t = 0.5 / tau;
    else
      t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    c = 1.0 / sqrt(1.0 + t * t);
    s = t * c;
  }
  partner[p] = q;
  partner[q] = p;
  cself[p] = c; cpart[p] = -s;  // new_p = c old_p - s old_q
  cself[q] = c; cpart[q] = s;   // new_q = s old_p + c old_q
}

// A' = R A R^T and V' = V R^T for the disjoint rotations of one round.
__global__ void k_jacobi_apply(const double* __restrict__ A, double* __restrict__ A2,
                               const double* __restrict__ V, double* __restrict__ V2, int m,
                               const int* __restrict__ partner, const double* __restrict__ cself,
                               const double* __restrict__ cpart) {
  int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= m) return;
  int pi = partner[i], pj = partner[j];
  double ci = cself[i], si = cpart[i], cj = cself[j], sj = cpart[j];
  const int64_t ri = (int64_t)i * m, rpi = (int64_t)pi * m;
  double v = ci * (cj * A[ri + j] + sj * A[ri + pj]) + si * (cj * A[rpi + j] + sj * A[rpi + pj]);
  if (pj == i) v = 0.0;
  A2[ri + j] = v;
  V2[ri + j] = cj * V[ri + j] + sj * V[ri + pj];
}

__global__ void k_offdiag(const double* __restrict__ A, int m, double* __restrict__ out) {
  int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  double off = 0.0, tot = 0.0;
  if (j < m) {
    double v = A[(int64_t)i * m + j];
    tot = v * v;
    off = (i != j) ? v * v : 0.0;
  }
  off = warp_sum_d(off);
  tot = warp_sum_d(tot);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&out[0], off);
    atomicAdd(&out[1], tot);
  }
}

__global__ void k_diag(const double* A, int m, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = A[(int64_t)i * m + i];
}

// sign of each eigenvector column: + if its largest-magnitude entry (lowest index) is positive
__global__ void k_eig_sign(const double* __restrict__ V, int m, int D, double* __restrict__ sgn) {
  int c = blockIdx.x;
  __shared__ double sv[256];
  __shared__ int si[256];
  double best = -1.0;
  int bi = 0x7fffffff;
  for (int k = threadIdx.x; k < D; k += blockDim.x) {
    double a = fabs(V[(int64_t)k * m + c]);
    if (a > best || (a == best && k < bi)) { best = a; bi = k; }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = blockDim.x / 2; s; s >>= 1) {
    if (threadIdx.x < s) {
      double a = sv[threadIdx.x + s];
      int k = si[threadIdx.x + s];
      if (a > sv[threadIdx.x] || (a == sv[threadIdx.x] && k < si[threadIdx.x])) {
        sv[threadIdx.x] = a;
        si[threadIdx.x] = k;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sgn[c] = V[(int64_t)si[0] * m + c] < 0 ? -1.0 : 1.0;
}

// Pp[r][k] = sgn * V[k][order[r]]
__global__ void k_make_pp(const double* __restrict__ V, int m, int D, const int* __restrict__ order,
                          const double* __restrict__ sgn, double* __restrict__ Pp) {
  int k = blockIdx.x * blockDim.x + threadIdx.x, r = blockIdx.y;
  if (k >= D) return;
  int c = order[r];
  Pp[(int64_t)r * D + k] = sgn[c] * V[(int64_t)k * m + c];
}

// ------------------------------------------------------------ random rotation

// Modified Gram-Schmidt on the columns of Q (d x d, row-major), in place.
__global__ void k_mgs(double* Q, int d) {
  __shared__ double red[32];
  __shared__ double nrm;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  for (int j = 0; j < d; ++j) {
    double s = 0.0;
    for (int i = tid; i < d; i += blockDim.x) s += Q[(int64_t)i * d + j] * Q[(int64_t)i * d + j];
    s = warp_sum_d(s);
    if (lane == 0) red[wid] = s;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < nw; ++w) t += red[w];
      nrm = sqrt(t);
    }
    __syncthreads();
    for (int i = tid; i < d; i += blockDim.x) Q[(int64_t)i * d + j] /= nrm;
    __syncthreads();
    for (int k = j + 1 + wid; k < d; k += nw) {
      double dot = 0.0;
      for (int i = lane; i < d; i += 32) dot += Q[(int64_t)i * d + j] * Q[(int64_t)i * d + k];
      dot = warp_sum_d(dot);
      for (int i = lane; i < d; i += 32) Q[(int64_t)i * d + k] -= dot * Q[(int64_t)i * d + j];
    }
    __syncthreads();
  }
}

// W[i][k] = sum_j Pr[j][i] Pp[j][k] for i < d; W[i][k] = Pp[i][k] for i >= d.
__global__ void k_make_w(const double* __restrict__ Pr, const double* __restrict__ Pp, int d,
                         int D, float* __restrict__ W) {
  int k = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (k >= D) return;
  double v;
  if (i < d) {
    v = 0.0;
    for (int j = 0; j < d; ++j) v = fma(Pr[(int64_t)j * d + i], Pp[(int64_t)j * D + k], v);
  } else {
    v = Pp[(int64_t)i * D + k];
  }
  W[(int64_t)i * D + k] = (float)v;
}

__global__ void k_d2f(const double* a, float* b, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// ------------------------------------------------------------------ k-means

__global__ void k_gather_rows(const float* __restrict__ src, int ld, const int64_t* __restrict__ rows,
                              int64_t nrows, int width, float* __restrict__ dst) {
  int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= nrows) return;
  int64_t s = rows[r];
  for (int c = threadIdx.x & 31; c < width; c += 32) dst[r * width + c] = src[s * ld + c];
}

__global__ void k_kmeans_accum(const float* __restrict__ X, int64_t n, int d,
                               const int32_t* __restrict__ a, double* __restrict__ sums,
                               unsigned int* __restrict__ cnt) {
  int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (r >= n) return;
  int lane = threadIdx.x & 31;
  int j = a[r];
  for (int c = lane; c < d; c += 32) atomicAdd(&sums[(int64_t)j * d + c], (double)X[r * d + c]);
  if (lane == 0) atomicAdd(&cnt[j], 1u);
}

__global__ void k_kmeans_update(const double* __restrict__ sums, const unsigned int* __restrict__ cnt,
                                int nlist, int d, float* __restrict__ C) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)nlist * d) return;
  int j = (int)(e / d);
  if (cnt[j] > 0) C[e] = (float)(sums[e] / (double)cnt[j]);
}

__global__ void k_iota(int32_t* a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int32_t)i;
}

__global__ void k_hist(const int32_t* a, int64_t n, unsigned int* h) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) atomicAdd(&h[a[i]], 1u);
}

// list-major gather of x_d', x_r; ids
__global__ void k_reorder(const float* __restrict__ xd_t, const float* __restrict__ xr_t, int d,
                          int r, const int32_t* __restrict__ perm, int64_t n,
                          float* __restrict__ xd, float* __restrict__ xr, int64_t* __restrict__ ids) {
  int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= n) return;
  int lane = threadIdx.x & 31;
  int64_t s = perm[p];
  for (int c = lane; c < d; c += 32) xd[p * d + c] = xd_t[s * d + c];
  for (int c = lane; c < r; c += 32) xr[p * r + c] = xr_t[s * r + c];
  if (lane == 0) ids[p] = s;
}

__global__ void k_rownorm2(const float* __restrict__ X, int64_t n, int w, float* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= n) return;
  float s = 0.f;
  for (int c = threadIdx.x & 31; c < w; c += 32) {
    float v = X[p * w + c];
    s = fmaf(v, v, s);
  }
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) out[p] = s;
}

// Eq. 4 / Eq. 5 factors of a code v with <v, o'> = ip and |v|^2 = vn2
__device__ __forceinline__ void code_factors(double rn, double ip, double vn2, int d, float& fr,
                                             float& fe) {
  if (rn > 0.0 && ip > 0.0) {
    const double a = ip / sqrt(vn2);
    fr = (float)(-2.0 * rn / ip);
    fe = (float)(2.0 * rn * sqrt(fmax(1.0 - a * a, 0.0) / (a * a)) / sqrt((double)(d - 1)));
  } else {
    fr = 0.f;
    fe = 0.f;
  }
}

// Quantization (Algorithm 1, quantize step) and factors (Eq. 4, Eq. 5), one warp per vector.
// With bits > 1 and fres1 != NULL it also writes the factors of the sign plane, the 1-bit
// code v1_i = sign(o'_i) (the top bit of the level), for the 1 bit + refinement scan.
__global__ void k_quantize(const float* __restrict__ xd, const float* __restrict__ xr2,
                           const float* __restrict__ cent, const int32_t* __restrict__ assign,
                           const int64_t* __restrict__ ids, int64_t n, int d, int bits,
                           uint8_t* __restrict__ levels, float* __restrict__ fadd,
                           float* __restrict__ fres, float* __restrict__ ferr,
                           float* __restrict__ xn2, float* __restrict__ fres1,
                           float* __restrict__ ferr1) {
  int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= n) return;
  const int lane = threadIdx.x & 31;
  const int j = assign[ids[p]];
  const int top = (1 << bits) - 1;
  const int nc = d / 32;
  float r[MRQ_MAX_D / 32];
  float ss = 0.f, xx = 0.f;
  for (int c = 0; c < nc; ++c) {
    float x = xd[p * d + c * 32 + lane];
    r[c] = x - cent[(int64_t)j * d + c * 32 + lane];
    ss = fmaf(r[c], r[c], ss);
    xx = fmaf(x, x, xx);
  }
  ss = warp_sum(ss);
  xx = warp_sum(xx);
  const float nr = sqrtf(ss);
  float mx = 0.f;
  for (int c = 0; c < nc; ++c) {
    r[c] = nr > 0.f ? r[c] / nr : 0.f;  // o'
    mx = fmaxf(mx, fabsf(r[c]));
  }
  mx = warp_max(mx);
  const float t = mx > 0.f ? (float)top / mx : 0.f;
  double ip = 0.0, vn2 = 0.0, ip1 = 0.0;
  for (int c = 0; c < nc; ++c) {
    const float o = r[c];
    float lev = 1.f;
    if (bits > 1) {
      float y = fabsf(o) * t;
      lev = fminf(fmaxf(2.f * floorf(y * 0.5f) + 1.f, 1.f), (float)top);
    }
    float v = (o > 0.f) ? lev : -lev;
    if (mx == 0.f) v = -(float)top;
    levels[p * d + c * 32 + lane] = (uint8_t)((int)(v + top) / 2);
    ip += (double)v * (double)o;
    vn2 += (double)v * (double)v;
    ip1 += v > 0.f ? (double)o : -(double)o;
  }
  ip = warp_sum_d(ip);
  vn2 = warp_sum_d(vn2);
  if (fres1) ip1 = warp_sum_d(ip1);
  if (lane == 0) {
    const double rn = (double)nr;
    const double tail = (double)xr2[p];
    fadd[p] = (float)(rn * rn + tail);
    xn2[p] = (float)((double)xx + tail);
    code_factors(rn, ip, vn2, d, fres[p], ferr[p]);
    if (fres1) code_factors(rn, ip1, (double)d, d, fres1[p], ferr1[p]);
  }
}

// ------------------------------------------------------------------ layout

__device__ __forceinline__ int64_t list_of(const int64_t* __restrict__ off, int nlist, int64_t p) {
  int lo = 0, hi = nlist - 1;  // last j with off[j] <= p
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int64_t code_word(int64_t pp, int w, int words, int vw) {
  int64_t blk = pp >> 5;
  int lane = (int)(pp & 31);
  return ((blk * (words / vw) + w / vw) * 32 + lane) * vw + (w % vw);
}

__global__ void k_pack(const uint8_t* __restrict__ levels, const float* __restrict__ fa,
                       const float* __restrict__ fr, const float* __restrict__ fe,
                       const float* __restrict__ fr1, const float* __restrict__ fe1,
                       const int64_t* __restrict__ loff, const int64_t* __restrict__ ploff,
                       int nlist, int64_t n, int d, int bits, int words, int vw,
                       uint32_t* __restrict__ codes, float* __restrict__ pa,
                       float* __restrict__ pr, float* __restrict__ pe, float* __restrict__ pr1,
                       float* __restrict__ pe1) {
  int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= n) return;
  const int lane = threadIdx.x & 31;
  int j = (int)list_of(loff, nlist, p);
  int64_t pp = ploff[j] + (p - loff[j]);
  const int nc = d / 32;
  for (int c = 0; c < nc; ++c) {
    int u = levels[p * d + c * 32 + lane];
    for (int a = 0; a < bits; ++a) {
      uint32_t word = __ballot_sync(0xffffffffu, (u >> a) & 1);
      if (lane == 0) codes[code_word(pp, a * nc + c, words, vw)] = word;
    }
  }
  if (lane == 0) {
    pa[pp] = fa[p];
    pr[pp] = fr[p];
    pe[pp] = fe[p];
    if (pr1) {
      pr1[pp] = fr1[p];
      pe1[pp] = fe1[p];
    }
  }
}

__global__ void k_unpack(const uint32_t* __restrict__ codes, const int64_t* __restrict__ loff,
                         const int64_t* __restrict__ ploff, int nlist, int64_t n, int d, int bits,
                         int words, int vw, uint8_t* __restrict__ levels) {
  int64_t p = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (p >= n) return;
  const int lane = threadIdx.x & 31;
  int j = (int)list_of(loff, nlist, p);
  int64_t pp = ploff[j] + (p - loff[j]);
  const int nc = d / 32;
  for (int c = 0; c < nc; ++c) {
    int u = 0;
    for (int a = 0; a < bits; ++a) u |= ((codes[code_word(pp, a * nc + c, words, vw)] >> lane) & 1) << a;
    levels[p * d + c * 32 + lane] = (uint8_t)u;
  }
}

__global__ void k_unpad(const float* __restrict__ padded, const int64_t* __restrict__ loff,
                        const int64_t* __restrict__ ploff, int nlist, int64_t n,
                        float* __restrict__ out) {
  int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  int j = (int)list_of(loff, nlist, p);
  out[p] = padded[ploff[j] + (p - loff[j])];
}

// hi = bf16(x), lo = bf16(x - hi): rows [0, n) and [n, 2n) of out
__global__ void k_bf16_split(const float* __restrict__ X, int64_t n, __nv_bfloat16* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float w = X[i];
  __nv_bfloat16 h = __float2bfloat16_rn(w);
  out[i] = h;
  out[n + i] = __float2bfloat16_rn(w - __bfloat162float(h));
}

__global__ void k_cent_norm(const float* __restrict__ C, int nlist, int d, float* __restrict__ out) {
  int64_t j = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (j >= nlist) return;
  float s = 0.f;
  for (int c = threadIdx.x & 31; c < d; c += 32) s = fmaf(C[j * d + c], C[j * d + c], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) out[j] = s;
}

inline int warps_grid(int64_t n, int wpb = 8) { return ceil_div(n, wpb); }

}  // namespace

// ================================================================== host side

void finalize_layout(mrq_index* idx, const uint8_t* levels, const float* fa, const float* fr,
                     const float* fe, cudaStream_t st, const float* fr1, const float* fe1) {
  const int nlist = idx->nlist;
  idx->words = idx->bits * idx->d / 32;
  idx->vw = (idx->words % 4 == 0) ? 4 : (idx->words % 2 == 0) ? 2 : 1;
  idx->h_ploff.assign(nlist + 1, 0);
  idx->max_list = 0;
  std::vector<int64_t> sizes(nlist);
  for (int j = 0; j < nlist; ++j) {
    int64_t s = idx->h_loff[j + 1] - idx->h_loff[j];
    sizes[j] = s;
    idx->max_list = std::max(idx->max_list, s);
    idx->h_ploff[j + 1] = idx->h_ploff[j] + ((s + 31) / 32) * 32;
  }
  idx->np = idx->h_ploff[nlist];
  std::sort(sizes.begin(), sizes.end(), std::greater<int64_t>());
  idx->cap_by_nprobe.assign(nlist + 1, 0);
  for (int r = 0; r < nlist; ++r) idx->cap_by_nprobe[r + 1] = idx->cap_by_nprobe[r] + sizes[r];

  idx->loff.alloc(nlist + 1);
  idx->ploff.alloc(nlist + 1);
  MRQ_CUDA(cudaMemcpyAsync(idx->loff.p, idx->h_loff.data(), 8 * (nlist + 1), cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(idx->ploff.p, idx->h_ploff.data(), 8 * (nlist + 1), cudaMemcpyHostToDevice, st));
  const int64_t np = std::max<int64_t>(idx->np, 32);
  idx->codes.alloc((size_t)np * idx->words);
  idx->fadd.alloc(np);
  idx->fres.alloc(np);
  idx->ferr.alloc(np);
  MRQ_CUDA(cudaMemsetAsync(idx->codes.p, 0, idx->codes.bytes(), st));
  MRQ_CUDA(cudaMemsetAsync(idx->fadd.p, 0, idx->fadd.bytes(), st));
  MRQ_CUDA(cudaMemsetAsync(idx->fres.p, 0, idx->fres.bytes(), st));
  MRQ_CUDA(cudaMemsetAsync(idx->ferr.p, 0, idx->ferr.bytes(), st));
  const bool sign_factors = idx->bits > 1 && fr1 && fe1;
  if (sign_factors) {
    idx->fres1.alloc(np);
    idx->ferr1.alloc(np);
    MRQ_CUDA(cudaMemsetAsync(idx->fres1.p, 0, idx->fres1.bytes(), st));
    MRQ_CUDA(cudaMemsetAsync(idx->ferr1.p, 0, idx->ferr1.bytes(), st));
  } else {
    idx->fres1.release();
    idx->ferr1.release();
  }
  if (idx->n > 0) {
    k_pack<<<warps_grid(idx->n), 256, 0, st>>>(
        levels, fa, fr, fe, sign_factors ? fr1 : nullptr, sign_factors ? fe1 : nullptr,
        idx->loff.p, idx->ploff.p, nlist, idx->n, idx->d, idx->bits, idx->words, idx->vw,
        idx->codes.p, idx->fadd.p, idx->fres.p, idx->ferr.p, idx->fres1.p, idx->ferr1.p);
    MRQ_CHECK_LAUNCH();
  }
  make_bf16_split(idx, st);
  compute_centroid_norms(idx, st);
}

void export_levels(const mrq_index* idx, uint8_t* levels, cudaStream_t st) {
  if (idx->n == 0) return;
  k_unpack<<<warps_grid(idx->n), 256, 0, st>>>(idx->codes.p, idx->loff.p, idx->ploff.p, idx->nlist,
                                               idx->n, idx->d, idx->bits, idx->words, idx->vw, levels);
  MRQ_CHECK_LAUNCH();
}

void export_padded(const mrq_index* idx, const float* padded, float* out, cudaStream_t st) {
  if (idx->n == 0) return;
  k_unpad<<<ceil_div(idx->n, 256), 256, 0, st>>>(padded, idx->loff.p, idx->ploff.p, idx->nlist,
                                                 idx->n, out);
  MRQ_CHECK_LAUNCH();
}

void make_bf16_split(mrq_index* idx, cudaStream_t st) {
  int64_t nn = (int64_t)idx->D * idx->D;
  idx->W2.alloc(2 * nn);
  k_bf16_split<<<ceil_div(nn, 256), 256, 0, st>>>(idx->W.p, nn, idx->W2.p);
  MRQ_CHECK_LAUNCH();
  if (idx->D % 16 == 0) {  // the FP8 projection's operand: 16-byte e4m3 rows
    idx->W8.alloc((size_t)nn);
    idx->W8s.alloc(idx->D);
    quantize_rows_fp8(idx->W.p, idx->D, idx->D, idx->D, nullptr, idx->W8.p, idx->W8s.p, st);
  }
  int64_t nc = (int64_t)idx->nlist * idx->d;
  idx->cent2.alloc(2 * nc);
  k_bf16_split<<<ceil_div(nc, 256), 256, 0, st>>>(idx->cent.p, nc, idx->cent2.p);
  MRQ_CHECK_LAUNCH();
}

void compute_centroid_norms(mrq_index* idx, cudaStream_t st) {
  idx->cent_n2.alloc(idx->nlist);
  k_cent_norm<<<warps_grid(idx->nlist), 256, 0, st>>>(idx->cent.p, idx->nlist, idx->d, idx->cent_n2.p);
  MRQ_CHECK_LAUNCH();
}

// Symmetric eigendecomposition of the D x D covariance held in Cdev (upper
// tiles, unscaled).  Returns eigenvalues (descending) in lam_host and P_p
// (rows = eigenvectors) in Pp_dev (float64, D x D).
static void eigen_pca(const double* Cdev, int D, double inv_n, std::vector<double>& lam_host,
                      DevBuf<double>& Pp_dev, cudaStream_t st) {
  const int m = D + (D & 1);
  DevBuf<double> A((size_t)m * m), A2((size_t)m * m), V((size_t)m * m), V2((size_t)m * m);
  DevBuf<int> partner(m);
  DevBuf<double> cself(m), cpart(m), red(2), diag(m);
  dim3 g2(ceil_div(m, 128), m);
  k_cov_to_jacobi<<<g2, 128, 0, st>>>(Cdev, D, m, inv_n, A.p, V.p);
  MRQ_CHECK_LAUNCH();
  double h_red[2];
  for (int sweep = 0; sweep < 40; ++sweep) {
    MRQ_CUDA(cudaMemsetAsync(red.p, 0, 16, st));
    k_offdiag<<<g2, 128, 0, st>>>(A.p, m, red.p);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaMemcpyAsync(h_red, red.p, 16, cudaMemcpyDeviceToHost, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
    if (!(h_red[0] > 1e-30 * h_red[1])) break;  // relative off-diagonal norm below 1e-15
    for (int round = 0; round < m - 1; ++round) {
      k_jacobi_angles<<<ceil_div(m / 2, 128), 128, 0, st>>>(A.p, m, round, partner.p, cself.p, cpart.p);
      k_jacobi_apply<<<g2, 128, 0, st>>>(A.p, A2.p, V.p, V2.p, m, partner.p, cself.p, cpart.p);
      std::swap(A.p, A2.p);
      std::swap(V.p, V2.p);
    }
    MRQ_CHECK_LAUNCH();
  }
  k_diag<<<ceil_div(m, 128), 128, 0, st>>>(A.p, m, diag.p);
  std::vector<double> dg(m);
  MRQ_CUDA(cudaMemcpyAsync(dg.data(), diag.p, 8 * m, cudaMemcpyDeviceToHost, st));
  MRQ_CUDA(cudaStreamSynchronize(st));
  std::vector<int> order(D);
  std::iota(order.begin(), order.end(), 0);  // the padding index (D) is never selected
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return dg[a] > dg[b]; });
  lam_host.resize(D);
  for (int r = 0; r < D; ++r) lam_host[r] = std::max(dg[order[r]], 0.0);
  DevBuf<int> dorder(D);
  DevBuf<double> sgn(m);
  MRQ_CUDA(cudaMemcpyAsync(dorder.p, order.data(), 4 * D, cudaMemcpyHostToDevice, st));
  k_eig_sign<<<m, 256, 0, st>>>(V.p, m, D, sgn.p);
  Pp_dev.alloc((size_t)D * D);
  k_make_pp<<<dim3(ceil_div(D, 128), D), 128, 0, st>>>(V.p, m, D, dorder.p, sgn.p, Pp_dev.p);
  MRQ_CHECK_LAUNCH();
  MRQ_CUDA(cudaStreamSynchronize(st));
}

void eigen_sym(const double* Cdev, int D, std::vector<double>& lam_host, DevBuf<double>& V_dev,
               cudaStream_t st) {
  eigen_pca(Cdev, D, 1.0, lam_host, V_dev, st);
}

// Eq. 8: the smallest power of two p >= 128 whose leading p eigenvalues hold `target` of
// their total (all D), capped at the largest multiple of 32 not above min(D, MRQ_MAX_D)
static int choose_d(const std::vector<double>& lam, int D, double target) {
  double total = 0.0;
  for (int i = 0; i < D; ++i) total += std::max(lam[i], 0.0);
  const int cap = std::min((D / 32) * 32, MRQ_MAX_D);
  double lead = 0.0;
  int i = 0;
  for (int p = 128; p < cap; p *= 2) {
    for (; i < p; ++i) lead += std::max(lam[i], 0.0);
    if (lead >= target * total) return p;
  }
  return cap;
}

void build_index(mrq_index* idx, const float* X, const mrq_build_opts& o, cudaStream_t st) {
  const int64_t n = idx->n;
  const int D = idx->D, nlist = idx->nlist;
  const uint64_t seed = o.seed ? o.seed : 1;

  // ---- PCA: float64 mean and covariance, over all rows or over the sampled rows
  DevBuf<float> Xs;
  const float* XP = X;
  int64_t npca = n;
  if (o.pca_rows) {
    npca = o.pca_n;
    DevBuf<int64_t> rows(npca);
    MRQ_CUDA(cudaMemcpyAsync(rows.p, o.pca_rows, 8 * npca, cudaMemcpyHostToDevice, st));
    Xs.alloc((size_t)npca * D);
    k_gather_rows<<<(unsigned)npca, 128, 0, st>>>(X, D, rows.p, npca, Xs.p);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaStreamSynchronize(st));
    XP = Xs.p;
  }
  DevBuf<double> mu_d(D), C((size_t)D * D);
  MRQ_CUDA(cudaMemsetAsync(mu_d.p, 0, 8 * D, st));
  {
    int64_t rows_per = 4096;
    dim3 g(ceil_div(D, 128), ceil_div(npca, rows_per));
    k_colsum<<<g, 128, 0, st>>>(XP, npca, D, rows_per, mu_d.p);
    MRQ_CHECK_LAUNCH();
    k_scale_d<<<ceil_div(D, 256), 256, 0, st>>>(mu_d.p, D, 1.0 / (double)npca);
    MRQ_CHECK_LAUNCH();
  }
  MRQ_CUDA(cudaMemsetAsync(C.p, 0, C.bytes(), st));
  {
    int T = ceil_div(D, CT);
    std::vector<int2> tl;
    for (int i = 0; i < T; ++i)
      for (int j = i; j < T; ++j) tl.push_back(make_int2(i, j));
    DevBuf<int2> tiles(tl.size());
    MRQ_CUDA(cudaMemcpyAsync(tiles.p, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice, st));
    int64_t rows_per = std::max<int64_t>(CR, ((npca + 255) / 256 + CR - 1) / CR * CR);
    rows_per = std::max<int64_t>(rows_per, 2048);
    dim3 g((unsigned)tl.size(), ceil_div(npca, rows_per));
    k_cov<<<g, 256, 0, st>>>(XP, npca, D, mu_d.p, tiles.p, rows_per, C.p);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaStreamSynchronize(st));
  }
  Xs.release();
  std::vector<double> lam_h;
  DevBuf<double> Pp;
  eigen_pca(C.p, D, 1.0 / (double)npca, lam_h, Pp, st);
  C.release();
  if (idx->d == 0) idx->d = choose_d(lam_h, D, o.auto_d_variance);  // Eq. 8
  const int d = idx->d, r = D - d;

  // ---- random rotation P_r (d x d): Q of the Gaussian draw
  std::vector<double> G((size_t)d * d);
  if (o.rotation_gauss) {
    std::copy(o.rotation_gauss, o.rotation_gauss + (size_t)d * d, G.begin());
  } else {
    SplitMix64 rng{seed * 0x632BE59BD9B4E019ull + 1};
    for (auto& g : G) g = rng.gauss();
  }
  DevBuf<double> Pr((size_t)d * d);
  MRQ_CUDA(cudaMemcpyAsync(Pr.p, G.data(), 8 * G.size(), cudaMemcpyHostToDevice, st));
  k_mgs<<<1, 256, 0, st>>>(Pr.p, d);
  k_mgs<<<1, 256, 0, st>>>(Pr.p, d);  // second pass restores orthogonality to rounding level
  MRQ_CHECK_LAUNCH();

  // ---- W, mu, lam on the index
  idx->W.alloc((size_t)D * D);
  k_make_w<<<dim3(ceil_div(D, 128), D), 128, 0, st>>>(Pr.p, Pp.p, d, D, idx->W.p);
  MRQ_CHECK_LAUNCH();
  idx->mu.alloc(D);
  k_d2f<<<ceil_div(D, 256), 256, 0, st>>>(mu_d.p, idx->mu.p, D);
  MRQ_CHECK_LAUNCH();
  idx->lam.alloc(D);
  {
    std::vector<float> lf(D);
    for (int i = 0; i < D; ++i) lf[i] = (float)lam_h[i];
    MRQ_CUDA(cudaMemcpyAsync(idx->lam.p, lf.data(), 4 * D, cudaMemcpyHostToDevice, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
  }

  // ---- projection of the base: [x_d' | x_r] = W (x - mu)
  DevBuf<float> xd_t((size_t)n * d), xr_t((size_t)n * std::max(r, 1));
  gemm_nt_f32(X, D, idx->mu.p, idx->W.p, D, (int)n, D, D, xd_t.p, d, xr_t.p, r, d, st);

  // ---- k-means on x_d' (rotated frame; Lloyd iterations commute with P_r)
  idx->cent.alloc((size_t)nlist * d);
  if (o.init_centroids) {
    // project the raw-space centroids with the first d rows of W
    DevBuf<float> ic((size_t)nlist * D);
    MRQ_CUDA(cudaMemcpyAsync(ic.p, o.init_centroids, 4 * ic.n, cudaMemcpyDefault, st));
    gemm_nt_f32(ic.p, D, idx->mu.p, idx->W.p, D, nlist, d, D, idx->cent.p, d, nullptr, 0, d, st);
  } else {
    std::vector<int64_t> pick(nlist);
    if (o.init_ids) {
      std::copy(o.init_ids, o.init_ids + nlist, pick.begin());
      for (auto v : pick) MRQ_REQUIRE(v >= 0 && v < n, "init_ids out of range");
    } else {
      // first nlist entries of a seeded Fisher-Yates permutation of 0..n-1
      SplitMix64 rng{seed * 0x9E3779B97F4A7C15ull + 7};
      std::unordered_map<int64_t, int64_t> moved;
      auto at = [&](int64_t i) { auto it = moved.find(i); return it == moved.end() ? i : it->second; };
      for (int i = 0; i < nlist; ++i) {
        int64_t j = i + (int64_t)(rng.next() % (uint64_t)(n - i));
        int64_t vi = at(i), vj = at(j);
        moved[i] = vj;
        moved[j] = vi;
        pick[i] = vj;
      }
    }
    DevBuf<int64_t> dp(nlist);
    MRQ_CUDA(cudaMemcpyAsync(dp.p, pick.data(), 8 * nlist, cudaMemcpyHostToDevice, st));
    k_gather_rows<<<warps_grid(nlist), 256, 0, st>>>(xd_t.p, d, dp.p, nlist, d, idx->cent.p);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaStreamSynchronize(st));
  }
  DevBuf<int32_t> assign(n);
  DevBuf<unsigned long long> amin(n);
  {
    DevBuf<double> sums((size_t)nlist * d);
    DevBuf<unsigned int> cnt(nlist);
    for (int it = 0; it < o.kmeans_iters; ++it) {
      nearest_f32(xd_t.p, d, idx->cent.p, d, (int)n, nlist, d, amin.p, assign.p, st);
      MRQ_CUDA(cudaMemsetAsync(sums.p, 0, sums.bytes(), st));
      MRQ_CUDA(cudaMemsetAsync(cnt.p, 0, cnt.bytes(), st));
      k_kmeans_accum<<<warps_grid(n), 256, 0, st>>>(xd_t.p, n, d, assign.p, sums.p, cnt.p);
      MRQ_CHECK_LAUNCH();
      k_kmeans_update<<<ceil_div((int64_t)nlist * d, 256), 256, 0, st>>>(sums.p, cnt.p, nlist, d, idx->cent.p);
      MRQ_CHECK_LAUNCH();
    }
  }
  nearest_f32(xd_t.p, d, idx->cent.p, d, (int)n, nlist, d, amin.p, assign.p, st);
  amin.release();

  // ---- list-major order: stable radix sort of (list, id)
  DevBuf<int32_t> keys_out(n), ids_in(n), perm(n);
  k_iota<<<ceil_div(n, 256), 256, 0, st>>>(ids_in.p, n);
  MRQ_CHECK_LAUNCH();
  {
    int end_bit = 1;
    while ((1 << end_bit) < nlist) ++end_bit;
    size_t tmp_bytes = 0;
    cub::DeviceRadixSort::SortPairs(nullptr, tmp_bytes, assign.p, keys_out.p, ids_in.p, perm.p,
                                    (int)n, 0, end_bit, st);
    DevBuf<uint8_t> tmp(tmp_bytes + 16);
    MRQ_CUDA(cub::DeviceRadixSort::SortPairs(tmp.p, tmp_bytes, assign.p, keys_out.p, ids_in.p,
                                             perm.p, (int)n, 0, end_bit, st));
  }
  keys_out.release();
  ids_in.release();
  {
    DevBuf<unsigned int> h(nlist);
    MRQ_CUDA(cudaMemsetAsync(h.p, 0, 4 * nlist, st));
    k_hist<<<ceil_div(n, 256), 256, 0, st>>>(assign.p, n, h.p);
    MRQ_CHECK_LAUNCH();
    std::vector<unsigned int> hh(nlist);
    MRQ_CUDA(cudaMemcpyAsync(hh.data(), h.p, 4 * nlist, cudaMemcpyDeviceToHost, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
    idx->h_loff.assign(nlist + 1, 0);
    for (int j = 0; j < nlist; ++j) idx->h_loff[j + 1] = idx->h_loff[j] + hh[j];
  }
  idx->xd.alloc((size_t)n * d);
  idx->xr.alloc((size_t)n * std::max(r, 1));
  idx->ids.alloc(n);
  k_reorder<<<warps_grid(n), 256, 0, st>>>(xd_t.p, xr_t.p, d, r, perm.p, n, idx->xd.p, idx->xr.p,
                                           idx->ids.p);
  MRQ_CHECK_LAUNCH();
  xd_t.release();
  xr_t.release();
  perm.release();

  // ---- quantization and factors
  DevBuf<float> xr2(n), fa(n), fr(n), fe(n), fr1, fe1;
  DevBuf<uint8_t> levels((size_t)n * d);
  if (idx->bits > 1) {
    fr1.alloc(n);
    fe1.alloc(n);
  }
  idx->xn2.alloc(n);
  if (r > 0) {
    k_rownorm2<<<warps_grid(n), 256, 0, st>>>(idx->xr.p, n, r, xr2.p);
    MRQ_CHECK_LAUNCH();
  } else {
    MRQ_CUDA(cudaMemsetAsync(xr2.p, 0, 4 * n, st));
  }
  k_quantize<<<warps_grid(n), 256, 0, st>>>(idx->xd.p, xr2.p, idx->cent.p, assign.p, idx->ids.p, n,
                                            d, idx->bits, levels.p, fa.p, fr.p, fe.p, idx->xn2.p,
                                            fr1.p, fe1.p);
  MRQ_CHECK_LAUNCH();
  finalize_layout(idx, levels.p, fa.p, fr.p, fe.p, st, fr1.p, fe1.p);
  MRQ_CUDA(cudaStreamSynchronize(st));
}

}  // namespace mrq
