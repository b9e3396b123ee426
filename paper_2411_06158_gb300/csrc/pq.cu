// MR-PQ (Appendix A.2, Exp-5): optimized product quantization of the projected lead
// coordinates x_d', trained on the GPU.  Non-parametric OPQ: with the rotation R fixed,
// Lloyd k-means of each of the M subspaces of d/M consecutive coordinates of x_d' R; with
// the codebooks fixed, R = the orthogonal factor closest to A = X^T Y (Y the decoded
// rows), i.e. R = U V^T for A = U S V^T, computed as A (A^T A)^(-1/2) with A^T A
// diagonalised by the library's float64 Jacobi eigensolver.  Distances, sums and A are
// accumulated in float64; the rotated rows and the codebooks are stored in float32.
#include <algorithm>
#include <cmath>
#include <numeric>

#include "common.cuh"

namespace mrq {
namespace {

// codes[i * M + m] = argmin_c |Xr[i, m*ds : (m+1)*ds] - C[m][c]|^2 (ties: lower c),
// distances in float64; one thread per (row, subspace)
__global__ void k_pq_assign(const float* __restrict__ Xr, int64_t n, int d, int M, int K,
                            const float* __restrict__ C, uint8_t* __restrict__ codes) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * M) return;
  const int64_t i = t / M;
  const int m = (int)(t % M), ds = d / M;
  const float* x = Xr + i * d + (int64_t)m * ds;
  const float* cb = C + (int64_t)m * K * ds;
  double best = 0.0;
  int arg = 0;
  for (int c = 0; c < K; ++c) {
    double s = 0.0;
    for (int e = 0; e < ds; ++e) {
      const double v = (double)x[e] - (double)cb[c * ds + e];
      s = fma(v, v, s);
    }
    if (c == 0 || s < best) { best = s; arg = c; }
  }
  codes[t] = (uint8_t)arg;
}

// per (subspace, centroid): float64 sums of its members' sub-rows and their count
__global__ void k_pq_accum(const float* __restrict__ Xr, int64_t n, int d, int M, int K,
                           const uint8_t* __restrict__ codes, double* __restrict__ sums,
                           unsigned long long* __restrict__ cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * M) return;
  const int64_t i = t / M;
  const int m = (int)(t % M), ds = d / M;
  const int c = codes[t];
  const float* x = Xr + i * d + (int64_t)m * ds;
  double* s = sums + ((int64_t)m * K + c) * ds;
  for (int e = 0; e < ds; ++e) atomicAdd(s + e, (double)x[e]);
  atomicAdd(cnt + (int64_t)m * K + c, 1ull);
}

// centroid = mean of its members; an empty one keeps its value
__global__ void k_pq_update(const double* __restrict__ sums,
                            const unsigned long long* __restrict__ cnt, int MK, int ds,
                            float* __restrict__ C) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= MK * ds) return;
  const unsigned long long c = cnt[t / ds];
  if (c) C[t] = (float)(sums[t] / (double)c);
}

// A = X^T Y (d x d, float64): X the rows of x_d', Y their decoded rows (codebook entries
// of their codes, in the rotated frame).  A 32 x 32 output tile per CTA and a slice of
// the rows; partial sums added with float64 atomics.
__global__ void __launch_bounds__(256) k_pq_xty(const float* __restrict__ X, int64_t n, int d,
                                                int M, int K, const float* __restrict__ C,
                                                const uint8_t* __restrict__ codes,
                                                int64_t rows_per, double* __restrict__ A) {
  __shared__ float sx[64][33], sy[64][33];
  const int i0 = blockIdx.x * 32, j0 = blockIdx.y * 32;
  const int64_t r0 = (int64_t)blockIdx.z * rows_per;
  const int64_t r1 = min(n, r0 + rows_per);
  const int ds = d / M;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 8 row groups of 4 outputs
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int64_t rb = r0; rb < r1; rb += 64) {
    for (int e = threadIdx.x; e < 64 * 32; e += 256) {
      const int rr = e >> 5, cc = e & 31;
      const int64_t row = rb + rr;
      float xv = 0.f, yv = 0.f;
      if (row < r1) {
        if (i0 + cc < d) xv = X[row * d + i0 + cc];
        const int j = j0 + cc;
        if (j < d) {
          const int m = j / ds;
          yv = C[((int64_t)m * K + codes[row * M + m]) * ds + (j - m * ds)];
        }
      }
      sx[rr][cc] = xv;
      sy[rr][cc] = yv;
    }
    __syncthreads();
    for (int rr = 0; rr < 64; ++rr) {
      const double yv = (double)sy[rr][tx];
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] = fma((double)sx[rr][ty * 4 + u], yv, acc[u]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int i = i0 + ty * 4 + u, j = j0 + tx;
    if (i < d && j < d) atomicAdd(A + (int64_t)i * d + j, acc[u]);
  }
}

// out = op(A) * B for small float64 d x d matrices (op: transpose when ta)
__global__ void k_dgemm_small(const double* __restrict__ A, const double* __restrict__ B, int d,
                              bool ta, double* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= d) return;
  double s = 0.0;
  for (int t = 0; t < d; ++t) s = fma(ta ? A[(int64_t)t * d + i] : A[(int64_t)i * d + t],
                                     B[(int64_t)t * d + j], s);
  out[(int64_t)i * d + j] = s;
}

// S = V^T diag(w) V for V holding eigenvectors as rows
__global__ void k_eig_recombine(const double* __restrict__ V, const double* __restrict__ w, int d,
                                double* __restrict__ S) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= d) return;
  double s = 0.0;
  for (int r = 0; r < d; ++r) s = fma(V[(int64_t)r * d + i] * w[r], V[(int64_t)r * d + j], s);
  S[(int64_t)i * d + j] = s;
}

__global__ void k_d2f_t(const double* __restrict__ R, int d, float* __restrict__ Rf,
                        float* __restrict__ Rt) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x, i = blockIdx.y;
  if (j >= d) return;
  const float v = (float)R[(int64_t)i * d + j];
  Rf[(int64_t)i * d + j] = v;
  Rt[(int64_t)j * d + i] = v;
}

__global__ void k_gather_sub(const float* __restrict__ Xr, int d, int M, int K,
                             const int64_t* __restrict__ rows, float* __restrict__ C) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= K * d) return;
  const int ds = d / M;
  const int c = t / d, j = t % d, m = j / ds;        // C is subspace-major: [m][c][e]
  C[((int64_t)m * K + c) * ds + (j - m * ds)] = Xr[rows[c] * d + j];
}

__global__ void k_rownorm2(const float* __restrict__ X, int64_t n, int r, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (i >= n) return;
  float s = 0.f;
  for (int c = threadIdx.x & 31; c < r; c += 32) {
    const float v = X[i * r + c];
    s = fmaf(v, v, s);
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) out[i] = s;
}

}  // namespace

// Lloyd rounds of every subspace at once (assign, then float64 means; an empty centroid
// keeps its value), then the final assignment: the codes of the current codebooks
static void pq_kmeans(const float* Xr, int64_t n, int d, int M, int K, int iters, float* C,
                      uint8_t* codes, double* sums, unsigned long long* cnt, cudaStream_t st) {
  const int ds = d / M;
  const unsigned g = (unsigned)ceil_div(n * M, 256);
  for (int it = 0; it < iters; ++it) {
    k_pq_assign<<<g, 256, 0, st>>>(Xr, n, d, M, K, C, codes);
    MRQ_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * (size_t)M * K * ds, st));
    MRQ_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * (size_t)M * K, st));
    k_pq_accum<<<g, 256, 0, st>>>(Xr, n, d, M, K, codes, sums, cnt);
    k_pq_update<<<ceil_div(M * K * ds, 256), 256, 0, st>>>(sums, cnt, M * K, ds, C);
    MRQ_CHECK_LAUNCH();
  }
  k_pq_assign<<<g, 256, 0, st>>>(Xr, n, d, M, K, C, codes);
  MRQ_CHECK_LAUNCH();
}

void pq_train(mrq_index* idx, int M, int K, int opq_iters, int km_iters, const int64_t* init_rows,
              cudaStream_t st) {
  const int64_t n = idx->n;
  const int d = idx->d, ds = d / M, r = idx->D - idx->d;
  DevBuf<float> Xr((size_t)n * d), C((size_t)M * K * ds), Rf((size_t)d * d), Rt((size_t)d * d);
  DevBuf<uint8_t> codes((size_t)n * M);
  DevBuf<double> sums((size_t)M * K * ds), A((size_t)d * d), AtA((size_t)d * d),
      Sinv((size_t)d * d), Rd((size_t)d * d), w(d);
  DevBuf<unsigned long long> cnt((size_t)M * K);
  DevBuf<int64_t> rows(K);
  std::vector<float> eye((size_t)d * d, 0.f);
  for (int i = 0; i < d; ++i) eye[(size_t)i * d + i] = 1.f;
  MRQ_CUDA(cudaMemcpyAsync(Rf.p, eye.data(), 4 * eye.size(), cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(Rt.p, eye.data(), 4 * eye.size(), cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(rows.p, init_rows, 8 * (size_t)K, cudaMemcpyHostToDevice, st));
  // x_d' R (R = Rt^T, so each output row is X times the rows of Rt)
  auto rotate = [&]() { gemm_nt_f32(idx->xd.p, d, nullptr, Rt.p, d, (int)n, d, d, Xr.p, d,
                                    Xr.p, d, d, st); };
  rotate();
  k_gather_sub<<<ceil_div(K * d, 256), 256, 0, st>>>(Xr.p, d, M, K, rows.p, C.p);
  MRQ_CHECK_LAUNCH();
  const dim3 gsq(ceil_div(d, 128), d);
  for (int it = 0; it < opq_iters; ++it) {
    rotate();
    pq_kmeans(Xr.p, n, d, M, K, km_iters, C.p, codes.p, sums.p, cnt.p, st);
    // Procrustes: R = A (A^T A)^(-1/2), A = X^T Y
    MRQ_CUDA(cudaMemsetAsync(A.p, 0, A.bytes(), st));
    const int64_t rows_per = std::max<int64_t>(4096, (n + 127) / 128);
    k_pq_xty<<<dim3(ceil_div(d, 32), ceil_div(d, 32), (unsigned)ceil_div(n, rows_per)), 256, 0,
               st>>>(idx->xd.p, n, d, M, K, C.p, codes.p, rows_per, A.p);
    k_dgemm_small<<<gsq, 128, 0, st>>>(A.p, A.p, d, true, AtA.p);
    MRQ_CHECK_LAUNCH();
    std::vector<double> lam;
    DevBuf<double> V;
    eigen_sym(AtA.p, d, lam, V, st);
    std::vector<double> wh(d);
    const double floor_ = std::max(lam[0], 1e-300) * 1e-24;
    for (int i = 0; i < d; ++i) wh[i] = 1.0 / std::sqrt(std::max(lam[i], floor_));
    MRQ_CUDA(cudaMemcpyAsync(w.p, wh.data(), 8 * (size_t)d, cudaMemcpyHostToDevice, st));
    k_eig_recombine<<<gsq, 128, 0, st>>>(V.p, w.p, d, Sinv.p);
    k_dgemm_small<<<gsq, 128, 0, st>>>(A.p, Sinv.p, d, false, Rd.p);
    k_d2f_t<<<gsq, 128, 0, st>>>(Rd.p, d, Rf.p, Rt.p);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaStreamSynchronize(st));
  }
  rotate();
  pq_kmeans(Xr.p, n, d, M, K, km_iters, C.p, codes.p, sums.p, cnt.p, st);
  DevBuf<float> xr2((size_t)std::max<int64_t>(n, 1));
  if (r > 0) {
    k_rownorm2<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(idx->xr.p, n, r, xr2.p);
    MRQ_CHECK_LAUNCH();
  } else {
    MRQ_CUDA(cudaMemsetAsync(xr2.p, 0, 4 * (size_t)n, st));
  }
  MRQ_CUDA(cudaStreamSynchronize(st));
  idx->pq_M = M;
  idx->pq_K = K;
  idx->pq_R = std::move(Rf);
  idx->pq_Rt = std::move(Rt);
  idx->pq_C = std::move(C);
  idx->pq_codes = std::move(codes);
  idx->pq_xr2 = std::move(xr2);
}

// an OPQ given from outside (the index file): R, codebooks and codes in host memory
void pq_install(mrq_index* idx, int M, int K, const float* R, const float* C,
                const uint8_t* codes, cudaStream_t st) {
  const int64_t n = idx->n;
  const int d = idx->d, ds = d / M, r = idx->D - idx->d;
  DevBuf<float> Rf((size_t)d * d), Rt((size_t)d * d), Cd((size_t)M * K * ds);
  DevBuf<uint8_t> cd((size_t)n * M);
  std::vector<float> rt((size_t)d * d);
  for (int i = 0; i < d; ++i)
    for (int j = 0; j < d; ++j) rt[(size_t)j * d + i] = R[(size_t)i * d + j];
  MRQ_CUDA(cudaMemcpyAsync(Rf.p, R, 4 * (size_t)d * d, cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(Rt.p, rt.data(), 4 * rt.size(), cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(Cd.p, C, 4 * (size_t)M * K * ds, cudaMemcpyHostToDevice, st));
  MRQ_CUDA(cudaMemcpyAsync(cd.p, codes, (size_t)n * M, cudaMemcpyHostToDevice, st));
  DevBuf<float> xr2((size_t)std::max<int64_t>(n, 1));
  if (r > 0) {
    k_rownorm2<<<(unsigned)ceil_div(n, 8), 256, 0, st>>>(idx->xr.p, n, r, xr2.p);
    MRQ_CHECK_LAUNCH();
  } else {
    MRQ_CUDA(cudaMemsetAsync(xr2.p, 0, 4 * (size_t)n, st));
  }
  MRQ_CUDA(cudaStreamSynchronize(st));
  idx->pq_M = M;
  idx->pq_K = K;
  idx->pq_R = std::move(Rf);
  idx->pq_Rt = std::move(Rt);
  idx->pq_C = std::move(Cd);
  idx->pq_codes = std::move(cd);
  idx->pq_xr2 = std::move(xr2);
}

}  // namespace mrq
