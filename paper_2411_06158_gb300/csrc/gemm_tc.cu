// Tensor-core (5th generation, tcgen05) GEMM for the dense contractions of the
// query path: the projection [q_d' | q_r] = W (q - mu) (Algorithm 2, rotate
// step) and the probe inner products <q_d', c_j'> (Algorithm 2, IVF probing).
//
// C[M x N] = A[M x K] * B[N x K]^T with A, B in bf16 (K contiguous) and float32
// accumulation in tensor memory.  The split-precision form stores each operand
// as hi = bf16(x) and lo = bf16(x - hi) (rows [0, R) = hi, [R, 2R) = lo of one
// tensor) and accumulates hi*hi + hi*lo + lo*hi into the same accumulator.
//
// One CTA computes a 128 x BN tile: warp 0 issues TMA loads (128-byte swizzled
// 64-wide K slices) into a 4-stage shared-memory ring, warp 1 issues
// tcgen05.mma (M = 128, N = BN, K = 16 per instruction) from one elected lane
// and frees ring slots with tcgen05.commit, warp 2 owns the tensor-memory
// allocation, and all four warps drain the accumulator with tcgen05.ld in the
// epilogue.  Every mbarrier wait is bounded (2 s of %globaltimer); a wait that
// gives up records an error word that the host turns into MRQ_ETIMEDOUT, and
// the CTA still frees its tensor memory.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "common.cuh"

namespace mrq {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;      // 64 bf16 = one 128-byte swizzle row
constexpr int TC_STAGES = 4;
constexpr uint64_t WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and *abort set) when it gives up or another thread gave up
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort,
                                          int* err, int code) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (mbar_try(b, parity)) return true;
    if (*abort) return false;
    if (gtimer() - t0 > WAIT_NS) {
      *abort = 1;
      atomicExch(err, code);
      return false;
    }
  }
}
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%3, %4}], [%2];" ::"r"(su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(su32(bar)), "r"(x), "r"(y)
      : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Shared-memory matrix descriptor, K-major operand, 128-byte swizzle:
// start >> 4 | LBO (unused for swizzled K-major) | SBO = 1024 B (8-row atom) |
// descriptor version 1 (bits 46-47) | layout 2 = SWIZZLE_128B (bits 61-63).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
  d |= (uint64_t)(16 >> 4) << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
// Instruction descriptor, kind::f16: D f32 (bits 4-5 = 1), A bf16 (bits 7-9 = 1),
// B bf16 (bits 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int BN>
__host__ __device__ constexpr uint32_t idesc_bf16() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
         ((uint32_t)(TC_BM >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   su32(bar))
               : "memory");
}
__device__ __forceinline__ void tc_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct TcArgs {
  int M, N, K;
  int phases;    // 1: hi*hi; 3: hi*hi + hi*lo + lo*hi
  int a_lo, b_lo;  // row offset of the lo half in the A / B tensors
  int epi;       // 0: store split into out0 / out1; 1: probe distances
  float* out0;
  int ld0;
  float* out1;
  int ld1;
  int split;
  const float* rown;  // epi 1: |q_d'|^2 per row (stride rstride)
  int rstride;
  const float* coln;  // epi 1/2: |c'|^2 per column
  unsigned long long* part;  // epi 2: per (row, column tile) the nsel smallest (key << 32 | col)
  int nsel;
  int* err;
};

constexpr int TC_PSEL = 16;  // largest nprobe selected inside the probe epilogue

template <int BN, int PSEL, int STAGES>
__global__ void __launch_bounds__(256, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              TcArgs P) {
  constexpr int A_BYTES = TC_BM * TC_BK * 2;
  constexpr int B_BYTES = BN * TC_BK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t NCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr uint32_t IDESC = idesc_bf16<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int kpp = (P.K + TC_BK - 1) / TC_BK;  // k-blocks per phase
  const int nkb = kpp * P.phases;

  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(&done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: TMA loads of the A and B slices of every k-block
    uint32_t stage = 0, phase = 0;
    for (int kb = 0; kb < nkb; ++kb) {
      if (!mbar_wait(&empty[stage], phase ^ 1u, &s_abort, P.err, 1)) break;
      const int ph = kb / kpp;
      const int k0 = (kb % kpp) * TC_BK;
      const int ay = m0 + (ph == 2 ? P.a_lo : 0);
      const int by = n0 + (ph == 1 ? P.b_lo : 0);
      uint8_t* sa = smem + stage * STAGE;
      mbar_expect_tx(&full[stage], STAGE);
      tma_load_2d(sa, &ta, k0, ay, &full[stage]);
      tma_load_2d(sa + A_BYTES, &tb, k0, by, &full[stage]);
      if (++stage == STAGES) { stage = 0; phase ^= 1u; }
    }
  } else if (warp == 1 && lane == 0) {
    // MMA issuer
    uint32_t stage = 0, phase = 0;
    bool ok = true;
    for (int kb = 0; kb < nkb; ++kb) {
      if (!mbar_wait(&full[stage], phase, &s_abort, P.err, 2)) { ok = false; break; }
      tc_fence_after();
      const uint32_t sa = su32(smem + stage * STAGE);
      const uint64_t ad = sdesc(sa), bd = sdesc(sa + A_BYTES);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk)
        tc_mma(tmem, ad + 2ull * kk, bd + 2ull * kk, IDESC, (kb | kk) != 0 ? 1u : 0u);
      tc_commit(&empty[stage]);
      if (++stage == STAGES) { stage = 0; phase ^= 1u; }
    }
    if (ok) tc_commit(&done);
  }
  __syncwarp();

  // epilogue: every warp drains its 32 accumulator lanes (rows)
  const bool have = mbar_wait(&done, 0, &s_abort, P.err, 3);
  tc_fence_after();
  unsigned long long best[PSEL];
#pragma unroll
  for (int t = 0; t < PSEL; ++t) best[t] = ~0ull;
  // 8 warps drain the accumulator: warp w reads tensor-memory lanes 32*(w%4) .. +31
  // (its rows) and the column half w/4 of the tile
  const int quarter = warp & 3, half = warp >> 2;
  constexpr int HALF = BN / 2;
  if (have) {
    const int row = m0 + quarter * 32 + lane;
    for (int c = half * HALF; c < half * HALF + HALF; c += 32) {
      uint32_t r[32];
      tc_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c, r);
      const int col0 = n0 + c;
      if (row >= P.M || col0 >= P.N) continue;
      if (P.epi == 0) {
        const bool whole = col0 + 32 <= P.N && (col0 + 32 <= P.split || col0 >= P.split);
        if (whole) {
          float* dst = col0 < P.split ? P.out0 + (int64_t)row * P.ld0 + col0
                                      : P.out1 + (int64_t)row * P.ld1 + (col0 - P.split);
          if ((reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
            float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
            for (int j = 0; j < 8; ++j)
              d4[j] = make_float4(__uint_as_float(r[4 * j]), __uint_as_float(r[4 * j + 1]),
                                  __uint_as_float(r[4 * j + 2]), __uint_as_float(r[4 * j + 3]));
          } else {
#pragma unroll
            for (int j = 0; j < 32; ++j) dst[j] = __uint_as_float(r[j]);
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = col0 + j;
            if (col >= P.N) break;
            if (col < P.split) P.out0[(int64_t)row * P.ld0 + col] = __uint_as_float(r[j]);
            else P.out1[(int64_t)row * P.ld1 + (col - P.split)] = __uint_as_float(r[j]);
          }
        }
      } else if (P.epi == 2) {
        // fused top-nsel: keep this row's smallest (g, list) pairs of the tile
        const float rn = P.rown[(int64_t)row * P.rstride];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int col = col0 + j;
          if (col < P.N) {
            const float gv = rn + P.coln[col] - 2.f * __uint_as_float(r[j]);
            unsigned long long v = ((unsigned long long)fkey(gv) << 32) | (uint32_t)col;
            if (v < best[PSEL - 1]) {
#pragma unroll
              for (int t = 0; t < PSEL; ++t) {
                const unsigned long long lo = v < best[t] ? v : best[t];
                v = v < best[t] ? best[t] : v;
                best[t] = lo;
              }
            }
          }
        }
      } else {
        const float rn = P.rown[(int64_t)row * P.rstride];
        float* dst = P.out0 + (int64_t)row * P.ld0;
        if (col0 + 32 <= P.N && (reinterpret_cast<uintptr_t>(dst + col0) & 15) == 0) {
          float4* d4 = reinterpret_cast<float4*>(dst + col0);
          const float4* c4 = reinterpret_cast<const float4*>(P.coln + col0);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            const float4 c = c4[j];
            d4[j] = make_float4(rn + c.x - 2.f * __uint_as_float(r[4 * j]),
                                rn + c.y - 2.f * __uint_as_float(r[4 * j + 1]),
                                rn + c.z - 2.f * __uint_as_float(r[4 * j + 2]),
                                rn + c.w - 2.f * __uint_as_float(r[4 * j + 3]));
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            int col = col0 + j;
            if (col < P.N) dst[col] = rn + P.coln[col] - 2.f * __uint_as_float(r[j]);
          }
        }
      }
    }
    if (P.epi == 2 && row < P.M) {
      unsigned long long* out =
          P.part + (((int64_t)row * gridDim.y + blockIdx.y) * 2 + half) * P.nsel;
#pragma unroll
      for (int t = 0; t < PSEL; ++t)
        if (t < P.nsel) out[t] = best[t];  // constant indices keep best[] in registers
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS)
                 : "memory");
}

// x = X[m, k] - shift[k] -> hi = bf16(x) (row m), lo = bf16(x - hi) (row M + m)
__global__ void k_split_bf16(const float* __restrict__ X, int M, int K, int ld,
                             const float* __restrict__ shift, int two,
                             __nv_bfloat16* __restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)M * K) return;
  int64_t m = i / K;
  int k = (int)(i % K);
  float x = X[m * ld + k] - (shift ? shift[k] : 0.f);
  __nv_bfloat16 h = __float2bfloat16_rn(x);
  out[i] = h;
  if (two) out[(int64_t)M * K + i] = __float2bfloat16_rn(x - __bfloat162float(h));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    MRQ_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (!p || q != cudaDriverEntryPointSuccess) fail(MRQ_ECUDA, "cuTensorMapEncodeTiled unavailable");
    fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

CUtensorMap make_map(const void* base, uint64_t rows, uint64_t K, uint32_t box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {K * 2};
  cuuint32_t box[2] = {TC_BK, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(MRQ_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

int* g_err = nullptr;

template <int BN, int PSEL, int STAGES>
void launch_tc(const __nv_bfloat16* A2, const __nv_bfloat16* B2, const TcArgs& a, cudaStream_t st) {
  constexpr int STAGE = TC_BM * TC_BK * 2 + BN * TC_BK * 2;
  const size_t smem = (size_t)STAGES * STAGE + 1024;
  const uint64_t arows = (uint64_t)a.M * (a.phases == 3 ? 2 : 1);
  const uint64_t brows = (uint64_t)a.N * (a.phases == 3 ? 2 : 1);
  CUtensorMap ta = make_map(A2, arows, a.K, TC_BM);
  CUtensorMap tb = make_map(B2, brows, a.K, BN);
  ensure_smem((const void*)k_gemm_tc<BN, PSEL, STAGES>, smem);
  dim3 grid(ceil_div(a.M, TC_BM), ceil_div(a.N, BN));
  k_gemm_tc<BN, PSEL, STAGES><<<grid, 256, smem, st>>>(ta, tb, a);
  MRQ_CHECK_LAUNCH();
}

void run_tc(const __nv_bfloat16* A2, const __nv_bfloat16* B2, TcArgs a, cudaStream_t st) {
  if (!g_err) {
    MRQ_CUDA(cudaMalloc(&g_err, sizeof(int)));
    MRQ_CUDA(cudaMemset(g_err, 0, sizeof(int)));
  }
  a.err = g_err;
  // the fused top-nsel list is sized to nsel (registers, a divergent insertion per column);
  // short contractions (the probe: K = d) use a 2-stage ring so that two CTAs fit per SM
  const bool short_k = (int64_t)((a.K + TC_BK - 1) / TC_BK) * a.phases <= 2;
#define MRQ_TC_N(PS, ST)                                  \
  do {                                                    \
    if (a.N <= 64) launch_tc<64, PS, ST>(A2, B2, a, st);  \
    else if (a.N <= 128) launch_tc<128, PS, ST>(A2, B2, a, st); \
    else launch_tc<256, PS, ST>(A2, B2, a, st);           \
  } while (0)
  if (a.epi == 2) {
    if (a.nsel > 8) { if (short_k) MRQ_TC_N(16, 2); else MRQ_TC_N(16, 4); }
    else if (a.nsel > 4) { if (short_k) MRQ_TC_N(8, 2); else MRQ_TC_N(8, 4); }
    else { if (short_k) MRQ_TC_N(4, 2); else MRQ_TC_N(4, 4); }
    return;
  }
  if (short_k) MRQ_TC_N(4, 2);
  else MRQ_TC_N(4, 4);
#undef MRQ_TC_N
}

}  // namespace

bool tc_available() {
  int dev = 0, major = 0, minor = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  return major == 10 && minor == 3;
}

int tc_check_error() {
  if (!g_err) return 0;
  int h = 0;
  MRQ_CUDA(cudaMemcpy(&h, g_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) MRQ_CUDA(cudaMemset(g_err, 0, sizeof(int)));
  return h;
}

void project_tc(const float* Q, const float* mu, const __nv_bfloat16* W2, int M, int D, int d,
                bool split3, __nv_bfloat16* qbf, float* qd, float* qr, cudaStream_t st) {
  const int64_t tot = (int64_t)M * D;
  k_split_bf16<<<ceil_div(tot, 256), 256, 0, st>>>(Q, M, D, D, mu, split3 ? 1 : 0, qbf);
  MRQ_CHECK_LAUNCH();
  TcArgs a{};
  a.M = M; a.N = D; a.K = D;
  a.phases = split3 ? 3 : 1;
  a.a_lo = M; a.b_lo = D;
  a.epi = 0;
  a.out0 = qd; a.ld0 = d; a.out1 = qr; a.ld1 = D - d; a.split = d;
  run_tc(qbf, W2, a, st);
}

void probe_tc(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
              int M, int nlist, int d, bool split3, __nv_bfloat16* qbf, float* gmat,
              cudaStream_t st) {
  const int64_t tot = (int64_t)M * d;
  k_split_bf16<<<ceil_div(tot, 256), 256, 0, st>>>(qd, M, d, d, nullptr, split3 ? 1 : 0, qbf);
  MRQ_CHECK_LAUNCH();
  TcArgs a{};
  a.M = M; a.N = nlist; a.K = d;
  a.phases = split3 ? 3 : 1;
  a.a_lo = M; a.b_lo = nlist;
  a.epi = 1;
  a.out0 = gmat; a.ld0 = nlist;
  a.rown = qstat + 3; a.rstride = 4;
  a.coln = cn2;
  run_tc(qbf, C2, a, st);
}

// Probe with the top-nsel fused into the epilogue: part[m][tile][nsel] receives, for
// every query row and 256-column tile, the nsel smallest (fkey(g) << 32 | list).
int probe_tc_topk(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
                  int M, int nlist, int d, bool split3, int nsel, __nv_bfloat16* qbf,
                  unsigned long long* part, cudaStream_t st) {
  const int64_t tot = (int64_t)M * d;
  k_split_bf16<<<ceil_div(tot, 256), 256, 0, st>>>(qd, M, d, d, nullptr, split3 ? 1 : 0, qbf);
  MRQ_CHECK_LAUNCH();
  TcArgs a{};
  a.M = M; a.N = nlist; a.K = d;
  a.phases = split3 ? 3 : 1;
  a.a_lo = M; a.b_lo = nlist;
  a.epi = 2;
  a.rown = qstat + 3; a.rstride = 4;
  a.coln = cn2;
  a.part = part;
  a.nsel = nsel;
  run_tc(qbf, C2, a, st);
  const int bn = nlist <= 64 ? 64 : nlist <= 128 ? 128 : 256;
  return 2 * ceil_div(nlist, bn);  // candidate lists per row: column tiles x 2 halves
}

}  // namespace mrq

// ---------------------------------------------------------------- projection without allocation
// Scratch of project_noalloc, one copy per device, created with the module (no
// allocation call): bytes [0, 256) hold the pipeline error word of the
// tensor-core GEMM, the rest the bf16 operand of the centred queries.
static __device__ __align__(256) unsigned char
    mrq_project_scratch[256 + MRQ_PROJECT_NOALLOC_MAX_BYTES];

namespace mrq {
namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
unsigned char* g_na_base[NA_MAX_DEVICES] = {};

// Device address of the current device's scratch, looked up on the first call
// with that device current and kept.
unsigned char* project_scratch() {
  int dev = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  MRQ_REQUIRE(dev >= 0 && dev < NA_MAX_DEVICES, "device ordinal too large for the projection scratch table");
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (!g_na_base[dev]) {
    unsigned char* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress((void**)&p, mrq_project_scratch);
    if (rc != cudaSuccess || !p)
      fail(MRQ_ECUDA, std::string("cannot get the address of the projection scratch: ") +
                          cudaGetErrorString(rc));
    g_na_base[dev] = p;
  }
  return g_na_base[dev];
}

}  // namespace

// qp = W (q - mu) with row stride D for both halves, using only the static
// scratch above.  The kernels and their tile shapes are the ones project_batch
// uses for the same precision, so the values match it.
void project_noalloc(mrq_index* idx, const float* q, int64_t nq, int precision, float* qp,
                     cudaStream_t st) {
  const int D = idx->D, d = idx->d;
  MRQ_REQUIRE(nq >= 1 && nq <= INT32_MAX, "nq must be in [1, 2^31)");
  if (precision == MRQ_PREC_FP32) {
    gemm_nt_f32(q, D, idx->mu.p, idx->W.p, D, (int)nq, D, D, qp, D, qp + d, D, d, st);
    MRQ_CUDA(cudaStreamSynchronize(st));
    return;
  }
  const bool split3 = precision == MRQ_PREC_BF16X3;
  const int64_t need = nq * D * 2 * (split3 ? 2 : 1);
  if (need > MRQ_PROJECT_NOALLOC_MAX_BYTES)
    fail(MRQ_EINVAL, "mrq_project_noalloc: nq * D = " + std::to_string(nq * D) + " needs " +
                         std::to_string(need) + " bytes of scratch, more than its fixed " +
                         std::to_string(MRQ_PROJECT_NOALLOC_MAX_BYTES) +
                         " (nq * D <= " + std::to_string(MRQ_PROJECT_NOALLOC_MAX_BYTES / (split3 ? 4 : 2)) +
                         " at this precision); split the batch");
  MRQ_REQUIRE(tc_available(), "tensor-core projection needs an sm_103 device");
  unsigned char* base = project_scratch();
  int* err = reinterpret_cast<int*>(base);
  __nv_bfloat16* qbf = reinterpret_cast<__nv_bfloat16*>(base + 256);
  MRQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  const int64_t tot = nq * D;
  k_split_bf16<<<ceil_div(tot, 256), 256, 0, st>>>(q, (int)nq, D, D, idx->mu.p, split3 ? 1 : 0, qbf);
  MRQ_CHECK_LAUNCH();
  TcArgs a{};
  a.M = (int)nq; a.N = D; a.K = D;
  a.phases = split3 ? 3 : 1;
  a.a_lo = (int)nq; a.b_lo = D;
  a.epi = 0;
  a.out0 = qp; a.ld0 = D; a.out1 = qp + d; a.ld1 = D; a.split = d;
  a.err = err;
  const bool short_k = (int64_t)((a.K + TC_BK - 1) / TC_BK) * a.phases <= 2;
  if (a.N <= 64) {
    if (short_k) launch_tc<64, 4, 2>(qbf, idx->W2.p, a, st);
    else launch_tc<64, 4, 4>(qbf, idx->W2.p, a, st);
  } else if (a.N <= 128) {
    if (short_k) launch_tc<128, 4, 2>(qbf, idx->W2.p, a, st);
    else launch_tc<128, 4, 4>(qbf, idx->W2.p, a, st);
  } else {
    if (short_k) launch_tc<256, 4, 2>(qbf, idx->W2.p, a, st);
    else launch_tc<256, 4, 4>(qbf, idx->W2.p, a, st);
  }
  int h = 0;
  MRQ_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  MRQ_CUDA(cudaStreamSynchronize(st));
  if (h) fail(MRQ_ETIMEDOUT, "a tensor-core kernel gave up waiting on its pipeline");
}

}  // namespace mrq
