// Float32 CUDA-core tile kernels: the plain-precision query/base projection
// (x_p = P_p (x - mu), Algorithm 1 and Algorithm 2, first step), the probe
// distances |q_d - c|^2 (Algorithm 2, IVF probing) and the nearest-centroid
// assignment of k-means (Algorithm 1, IVF step).
//
// One kernel template computes a 128 x 128 output tile per CTA (256 threads,
// 8 x 8 outputs per thread in two 4-wide strips per axis so that shared-memory
// float4 reads are conflict-free), K streamed in 16-wide slices through
// shared memory.  OP selects <a, b> (dot) or |a - b|^2 (direct squared
// distance, no norm expansion, so no cancellation).
#include "common.cuh"

namespace mrq {
namespace {

constexpr int BM = 128, BN = 128, BK = 16, NT = 256;

enum { OP_DOT = 0, OP_SQD = 1 };
enum { EPI_STORE = 0, EPI_ARGMIN = 1 };

struct EpiArgs {
  float* out0;
  int ld0;
  float* out1;
  int ld1;
  int split;
  unsigned long long* amin;  // packed (key << 32 | col) per row
};

template <int OP, int EPI>
__global__ void __launch_bounds__(NT) k_tile(const float* __restrict__ A, int lda,
                                             const float* __restrict__ a_shift,
                                             const float* __restrict__ B, int ldb, int M, int N,
                                             int K, EpiArgs ea) {
  __shared__ __align__(16) float As[BK][BM + 4];
  __shared__ __align__(16) float Bs[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int64_t n0 = (int64_t)blockIdx.y * BN;

  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  // loader mapping: row lr = tid / 2 (0..127), k-offset lk = (tid & 1) * 8
  const int lr = tid >> 1, lk = (tid & 1) * 8;
  for (int k0 = 0; k0 < K; k0 += BK) {
    {
      const int64_t gm = m0 + lr;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        int gk = k0 + lk + e;
        float v = 0.f;
        if (gm < M && gk < K) {
          v = A[gm * lda + gk];
          if (a_shift) v -= a_shift[gk];
        }
        As[lk + e][lr] = v;
      }
      const int64_t gn = n0 + lr;
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        int gk = k0 + lk + e;
        float v = 0.f;
        if (gn < N && gk < K) v = B[gn * ldb + gk];
        Bs[lk + e][lr] = v;
      }
    }
    __syncthreads();
    const int kmax = min(BK, K - k0);
    for (int kk = 0; kk < kmax; ++kk) {
      float a[8], b[8];
      float4 t;
      t = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      a[0] = t.x; a[1] = t.y; a[2] = t.z; a[3] = t.w;
      t = *reinterpret_cast<const float4*>(&As[kk][64 + ty * 4]);
      a[4] = t.x; a[5] = t.y; a[6] = t.z; a[7] = t.w;
      t = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      b[0] = t.x; b[1] = t.y; b[2] = t.z; b[3] = t.w;
      t = *reinterpret_cast<const float4*>(&Bs[kk][64 + tx * 4]);
      b[4] = t.x; b[5] = t.y; b[6] = t.z; b[7] = t.w;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (OP == OP_DOT) {
            acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
          } else {
            float df = a[i] - b[j];
            acc[i][j] = fmaf(df, df, acc[i][j]);
          }
        }
    }
    __syncthreads();
  }

  if (EPI == EPI_STORE) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      if (gm >= M) continue;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (gn >= N) continue;
        if (gn < ea.split)
          ea.out0[gm * ea.ld0 + gn] = acc[i][j];
        else
          ea.out1[gm * ea.ld1 + (gn - ea.split)] = acc[i][j];
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      int64_t gm = m0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4));
      unsigned long long best = ~0ull;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int64_t gn = n0 + (j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4));
        if (gn < N) {
          unsigned long long key = ((unsigned long long)fkey(acc[i][j]) << 32) | (uint32_t)gn;
          best = key < best ? key : best;
        }
      }
      // the 16 threads sharing ty sit in one half-warp
#pragma unroll
      for (int off = 8; off >= 1; off >>= 1) {
        unsigned long long o = __shfl_xor_sync(0xffffffffu, best, off);
        best = o < best ? o : best;
      }
      if (tx == 0 && gm < M && best != ~0ull) atomicMin(&ea.amin[gm], best);
    }
  }
}

__global__ void k_unpack_argmin(const unsigned long long* amin, int64_t M, int32_t* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < M) out[i] = (int32_t)(amin[i] & 0xffffffffu);
}

dim3 tile_grid(int M, int N) { return dim3(ceil_div(M, BM), ceil_div(N, BN)); }

}  // namespace

void gemm_nt_f32(const float* A, int lda, const float* a_shift, const float* B, int ldb, int M,
                 int N, int K, float* out0, int ld0, float* out1, int ld1, int split,
                 cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  EpiArgs ea{out0, ld0, out1, ld1, split, nullptr};
  k_tile<OP_DOT, EPI_STORE><<<tile_grid(M, N), NT, 0, st>>>(A, lda, a_shift, B, ldb, M, N, K, ea);
  MRQ_CHECK_LAUNCH();
}

void sqdist_f32(const float* A, int lda, const float* B, int ldb, int M, int N, int K,
                float* Dout, int ldd, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  EpiArgs ea{Dout, ldd, nullptr, 0, N, nullptr};
  k_tile<OP_SQD, EPI_STORE><<<tile_grid(M, N), NT, 0, st>>>(A, lda, nullptr, B, ldb, M, N, K, ea);
  MRQ_CHECK_LAUNCH();
}

void nearest_f32(const float* A, int lda, const float* B, int ldb, int M, int N, int K,
                 unsigned long long* scratch, int32_t* out, cudaStream_t st) {
  if (M <= 0 || N <= 0) return;
  MRQ_CUDA(cudaMemsetAsync(scratch, 0xff, sizeof(unsigned long long) * (size_t)M, st));
  EpiArgs ea{nullptr, 0, nullptr, 0, 0, scratch};
  k_tile<OP_SQD, EPI_ARGMIN><<<tile_grid(M, N), NT, 0, st>>>(A, lda, nullptr, B, ldb, M, N, K, ea);
  MRQ_CHECK_LAUNCH();
  k_unpack_argmin<<<ceil_div(M, 256), 256, 0, st>>>(scratch, M, out);
  MRQ_CHECK_LAUNCH();
}

}  // namespace mrq
