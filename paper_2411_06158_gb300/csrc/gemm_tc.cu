// Tensor-core (5th generation, tcgen05) GEMM for the dense contractions of the
// query path: the projection [q_d' | q_r] = W (q - mu) (Algorithm 2, rotate
// step) and the probe inner products <q_d', c_j'> (Algorithm 2, IVF probing).
//
// C[M x N] = A[M x K] * B[N x K]^T with A, B in bf16 (K contiguous) and float32
// accumulation in tensor memory.  The split-precision form stores each operand
// as hi = bf16(x) and lo = bf16(x - hi) (rows [0, R) = hi, [R, 2R) = lo of one
// tensor) and accumulates hi*hi + hi*lo + lo*hi into the same accumulator.  The
// row-scaled FP8 form stores both operands as e4m3 with one float32 scale per row
// (|row|_max -> 448) and runs kind::f8f6f4 MMAs (K = 32 per instruction, the same 32
// bytes per step), the epilogue multiplying each accumulator by its two row scales.
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

#include <cuda_fp8.h>

#include "common.cuh"

namespace mrq {
namespace {

constexpr int TC_BM = 128;
constexpr int TC_BK = 64;      // 64 bf16 = one 128-byte swizzle row
constexpr uint64_t WAIT_NS = 2000000000ull;
#define FLT_MAX_F __int_as_float(0x7f7fffff)
#define FLT_INF_F __int_as_float(0x7f800000)

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
// try_wait that may suspend the thread for up to ns nanoseconds until the phase completes
__device__ __forceinline__ bool mbar_try_sleep(uint64_t* b, uint32_t parity, uint32_t ns) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity), "r"(ns)
      : "memory");
  return ok != 0;
}
// bounded wait; false (and *abort set) when it gives up or another thread gave up.
// sleep_ns > 0 lets the waiting threads sleep between tries (warps that only wait
// for the accumulator then leave the issue slots to the co-resident CTA).
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort,
                                          int* err, int code, uint32_t sleep_ns = 0) {
  if (mbar_try(b, parity)) return true;
  const uint64_t t0 = gtimer();
  while (true) {
    if (sleep_ns ? mbar_try_sleep(b, parity, sleep_ns) : mbar_try(b, parity)) return true;
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
// Instruction descriptor, kind::f8f6f4: D f32 (bits 4-5 = 1), A and B e4m3 (format 0 in
// bits 7-9 and 10-12), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
template <int N>
__host__ __device__ constexpr uint32_t idesc_e4m3() {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
}
__device__ __forceinline__ void tc_mma_f8(uint32_t dtmem, uint64_t a, uint64_t b, uint32_t idesc,
                                          uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(dtmem),
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
  __nv_bfloat16* pbf;  // epi 0, optional: the first `split` columns again, split into bf16
  int pbf_two;         // hi (rows 0..M-1) and, when set, lo (rows M..2M-1) for the probe
  const float* rscale;  // FP8 form, epi 0: per-row scale of A (M) and of B (N)
  const float* cscale;
};


template <int BN, int PSEL, int STAGES, bool F8 = false>
__global__ void __launch_bounds__(256, 1)
    k_gemm_tc(const __grid_constant__ CUtensorMap ta, const __grid_constant__ CUtensorMap tb,
              TcArgs P) {
  constexpr int A_BYTES = TC_BM * TC_BK * 2;  // 128-byte K slices: 64 bf16 or 128 e4m3
  constexpr int B_BYTES = BN * TC_BK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr int KBE = F8 ? 2 * TC_BK : TC_BK;  // elements per K slice
  constexpr uint32_t NCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr uint32_t IDESC = F8 ? idesc_e4m3<BN>() : idesc_bf16<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~static_cast<uintptr_t>(1023));
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES], done;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  __shared__ __align__(16) float s_coln[BN];  // epi 2: |c'|^2 of this tile's columns

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * TC_BM, n0 = blockIdx.y * BN;
  const int kpp = (P.K + KBE - 1) / KBE;  // k-blocks per phase
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
      const int k0 = (kb % kpp) * KBE;
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
      // four MMAs of 32 bytes of K each (16 bf16 or 32 e4m3)
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk) {
        if constexpr (F8)
          tc_mma_f8(tmem, ad + 2ull * kk, bd + 2ull * kk, IDESC, (kb | kk) != 0 ? 1u : 0u);
        else
          tc_mma(tmem, ad + 2ull * kk, bd + 2ull * kk, IDESC, (kb | kk) != 0 ? 1u : 0u);
      }
      tc_commit(&empty[stage]);
      if (++stage == STAGES) { stage = 0; phase ^= 1u; }
    }
    if (ok) tc_commit(&done);
  }
  __syncwarp();

  // epilogue: every warp drains its 32 accumulator lanes (rows)
  if (P.epi == 2) {
    for (int t = threadIdx.x; t < BN; t += blockDim.x)
      s_coln[t] = n0 + t < P.N ? P.coln[n0 + t] : 0.f;
    __syncthreads();
  }
  const bool have = mbar_wait(&done, 0, &s_abort, P.err, 3, 20000);
  tc_fence_after();
  // 8 warps drain the accumulator: warp w reads tensor-memory lanes 32*(w%4) .. +31
  // (its rows) and the column half w/4 of the tile
  const int quarter = warp & 3, half = warp >> 2;
  constexpr int HALF = BN / 2;
  const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16);
  if (have && P.epi != 2) {
    const int row = m0 + quarter * 32 + lane;
    for (int c = half * HALF; c < half * HALF + HALF; c += 32) {
      uint32_t r[32];
      tc_ld32(trow + (uint32_t)c, r);
      const int col0 = n0 + c;
      if (row >= P.M || col0 >= P.N) continue;
      if constexpr (F8) {  // the two row scales of the e4m3 operands
        const float rs = P.rscale[row];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const float cs = col0 + j < P.N ? P.cscale[col0 + j] : 0.f;
          r[j] = __float_as_uint(__uint_as_float(r[j]) * rs * cs);
        }
      }
      if (P.epi == 0) {
        if (P.pbf && col0 + 32 <= P.split) {
          // the probe's bf16 operand (hi, and lo = x - hi) of these 32 q_d' coordinates,
          // as the bf16 split kernel would compute it from the stored values
          uint32_t hw[16], lw[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) {
            const float x0 = __uint_as_float(r[2 * t]), x1 = __uint_as_float(r[2 * t + 1]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            hw[t] = *reinterpret_cast<const uint32_t*>(&h);
            lw[t] = *reinterpret_cast<const uint32_t*>(&l);
          }
          uint4* dh = reinterpret_cast<uint4*>(P.pbf + (int64_t)row * P.split + col0);
#pragma unroll
          for (int t = 0; t < 4; ++t) dh[t] = make_uint4(hw[4 * t], hw[4 * t + 1], hw[4 * t + 2], hw[4 * t + 3]);
          if (P.pbf_two) {
            uint4* dl = reinterpret_cast<uint4*>(P.pbf + ((int64_t)P.M + row) * P.split + col0);
#pragma unroll
            for (int t = 0; t < 4; ++t)
              dl[t] = make_uint4(lw[4 * t], lw[4 * t + 1], lw[4 * t + 2], lw[4 * t + 3]);
          }
        }
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
  } else if (have) {
    // fused top-nsel of g = |q_d'|^2 + |c'|^2 - 2 <q_d', c'> over this row's half
    // tile.  Pass 1 keeps the PSEL smallest g in a branch-free min/max insertion
    // network; pass 2 recomputes g, marks the columns at or below the nsel-th
    // smallest in a bit mask, and emits those below it plus ties at it in column
    // order (lower list ids first).  g is never -0 (its terms are sums of squares
    // and an exact cancellation rounds to +0), so float and key order agree.
    const int row = m0 + quarter * 32 + lane;
    const bool rv = row < P.M;
    const float rn = rv ? P.rown[(int64_t)row * P.rstride] : 0.f;
    // four independent networks (one per column residue mod 4) keep four dependency
    // chains in flight; they are merged below (the PSEL smallest of the union are the
    // same values whatever the order of insertion)
    float b[PSEL], b4[4][PSEL];
#pragma unroll
    for (int t = 0; t < PSEL; ++t) {
      b[t] = FLT_MAX_F;
#pragma unroll
      for (int u = 0; u < 4; ++u) b4[u][t] = FLT_MAX_F;
    }
    for (int c = half * HALF; c < half * HALF + HALF; c += 32) {
      uint32_t r[32];
      tc_ld32(trow + (uint32_t)c, r);
      const int col0 = n0 + c;
      if (col0 + 32 <= P.N) {
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const float4 cn = *reinterpret_cast<const float4*>(s_coln + c + j);
          const float g4[4] = {fmaf(-2.f, __uint_as_float(r[j]), rn + cn.x),
                               fmaf(-2.f, __uint_as_float(r[j + 1]), rn + cn.y),
                               fmaf(-2.f, __uint_as_float(r[j + 2]), rn + cn.z),
                               fmaf(-2.f, __uint_as_float(r[j + 3]), rn + cn.w)};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int t = PSEL - 1; t >= 1; --t)
              b4[u][t] = fminf(b4[u][t], fmaxf(b4[u][t - 1], g4[u]));
            b4[u][0] = fminf(b4[u][0], g4[u]);
          }
        }
      } else {
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          if (col0 + j < P.N) {
            const float g = fmaf(-2.f, __uint_as_float(r[j]), rn + s_coln[c + j]);
#pragma unroll
            for (int t = PSEL - 1; t >= 1; --t) b[t] = fminf(b[t], fmaxf(b[t - 1], g));
            b[0] = fminf(b[0], g);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
#pragma unroll
      for (int v = 0; v < PSEL; ++v) {
        const float g = b4[u][v];
#pragma unroll
        for (int t = PSEL - 1; t >= 1; --t) b[t] = fminf(b[t], fmaxf(b[t - 1], g));
        b[0] = fminf(b[0], g);
      }
    }
    float thr = b[0];  // b[] is ascending: b[nsel - 1] is the largest of the first nsel
#pragma unroll
    for (int t = 1; t < PSEL; ++t) thr = t < P.nsel ? fmaxf(thr, b[t]) : thr;
    int ns = 0;  // values strictly below the threshold (all of them are among b[])
#pragma unroll
    for (int t = 0; t < PSEL; ++t) ns += (t < P.nsel && b[t] < thr) ? 1 : 0;
    unsigned long long* out =
        P.part + (((int64_t)row * gridDim.y + blockIdx.y) * 2 + half) * P.nsel;
    int si = 0, ti = 0;
    const int tcap = P.nsel - ns;
    // this lane's g values of one chunk, in the operand ring (idle once the MMAs are done)
    float* gs = reinterpret_cast<float*>(smem) + (warp * 32 + lane) * 36;
    for (int c = half * HALF; c < half * HALF + HALF; c += 32) {
      uint32_t r[32];
      tc_ld32(trow + (uint32_t)c, r);
      const int col0 = n0 + c;
      uint32_t mask = 0;
#pragma unroll
      for (int j = 0; j < 32; j += 4) {
        const float4 cn = *reinterpret_cast<const float4*>(s_coln + c + j);
        const float4 g4 = make_float4(fmaf(-2.f, __uint_as_float(r[j]), rn + cn.x),
                                      fmaf(-2.f, __uint_as_float(r[j + 1]), rn + cn.y),
                                      fmaf(-2.f, __uint_as_float(r[j + 2]), rn + cn.z),
                                      fmaf(-2.f, __uint_as_float(r[j + 3]), rn + cn.w));
        mask |= (g4.x <= thr ? 1u : 0u) << j;
        mask |= (g4.y <= thr ? 1u : 0u) << (j + 1);
        mask |= (g4.z <= thr ? 1u : 0u) << (j + 2);
        mask |= (g4.w <= thr ? 1u : 0u) << (j + 3);
        *reinterpret_cast<float4*>(gs + j) = g4;
      }
      if (!rv) mask = 0;
      if (col0 + 32 > P.N) mask &= P.N > col0 ? (0xffffffffu >> (32 - (P.N - col0))) : 0u;
      while (mask) {
        const int jj = __ffs(mask) - 1;
        mask &= mask - 1;
        const float g = gs[jj];
        const unsigned long long key =
            ((unsigned long long)fkey(g) << 32) | (uint32_t)(col0 + jj);
        if (g < thr) out[si++] = key;
        else if (ti < tcap) out[ns + ti++] = key;
      }
    }
    if (rv)
      for (int t = ns + ti; t < P.nsel; ++t) out[t] = ~0ull;  // fewer than nsel columns
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS)
                 : "memory");
}

// ------------------------------------------------------------------ fused projection
// [q_d' | q_r] = W (q - mu) straight from the float32 queries (Algorithm 2, rotate step):
// the centring and the bf16 split of the query operand happen inside the GEMM, so no
// split kernel and no bf16 copy of the queries in global memory.
//
// Persistent CTAs (one per SM) walk the 128 x BN output tiles in row-major tile order
// (consecutive CTAs share a block of query rows, which then comes from L2).  Warp roles:
//   warp 0 (one lane)  TMA producer: float32 query slices (two 32-float, 128-byte
//                      swizzled boxes per 64-wide K slice) into the staging ring, and
//                      W's bf16 slices (hi, and lo in the split form) into the operand ring;
//   warp 1 (one lane)  tcgen05.mma issuer (hi*hi, plus hi*lo + lo*hi in the split form),
//                      into one of two tensor-memory accumulators;
//   warp 2             tensor-memory allocation;
//   warps 4-7          converters: thread t reads row t of a staged slice, subtracts mu,
//                      rounds to bf16 hi (and lo = bf16(x - hi)), and writes the 128-byte
//                      swizzled K-major operand rows the MMA reads;
//   warps 8-11         epilogue: tcgen05.ld of their 32 accumulator lanes, float32 rows of
//                      q_d' and q_r, and the probe's bf16 operand of q_d'.
// The two accumulators let the epilogue of one tile run under the MMAs of the next.
struct ProjArgs {
  int M, N, K;        // queries, output columns (D), reduction length (D)
  int b_lo;           // row offset of W's lo half in its tensor (split form)
  const float* mu;    // centre, K floats
  float* out0;        // columns [0, split), row stride ld0
  int ld0;
  float* out1;        // columns [split, N), row stride ld1
  int ld1;
  int split;
  __nv_bfloat16* pbf;  // optional: the first `split` columns again as bf16 hi (rows 0..M-1)
  int pbf_two;         // and lo (rows M..2M-1)
  int* err;
  int tiles_n;        // ceil(N / BN)
  int tiles;          // ceil(M / 128) * tiles_n
};

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ void fence_async_shared() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr int PJ_THREADS = 384;
constexpr int PJ_F32_STAGE = TC_BM * 64 * 4;  // 128 rows x 64 float32 = two 16 KB boxes

template <int BN, int SA, int SB, int S32, bool THREE>
__global__ void __launch_bounds__(PJ_THREADS, 1)
    k_proj_tc(const __grid_constant__ CUtensorMap tq, const __grid_constant__ CUtensorMap tw,
              ProjArgs P) {
  constexpr int A_BYTES = TC_BM * TC_BK * 2;
  constexpr int B_BYTES = BN * TC_BK * 2;
  constexpr int AST = A_BYTES * (THREE ? 2 : 1);  // one A stage: hi (and lo)
  constexpr int BST = B_BYTES * (THREE ? 2 : 1);  // one B stage: hi (and lo)
  // the two accumulators start at column 0 and at BSTR (BN rounded up to a power of two)
  constexpr uint32_t BSTR = BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
  constexpr uint32_t NCOLS = 2 * BSTR;
  constexpr uint32_t IDESC = idesc_bf16<BN>();
  extern __shared__ uint8_t smem_raw[];
  uint8_t* ar = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                           ~static_cast<uintptr_t>(1023));
  uint8_t* br = ar + SA * AST;
  uint8_t* f32r = br + SB * BST;
  __shared__ __align__(8) uint64_t f_full[S32], f_empty[S32], a_full[SA], a_empty[SA];
  __shared__ __align__(8) uint64_t b_full[SB], b_empty[SB], c_full[2], c_empty[2];
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nkb = (P.K + TC_BK - 1) / TC_BK;
  if (threadIdx.x == 0) {
    s_abort = 0;
    for (int s = 0; s < S32; ++s) { mbar_init(&f_full[s], 1); mbar_init(&f_empty[s], 4); }
    for (int s = 0; s < SA; ++s) { mbar_init(&a_full[s], 4); mbar_init(&a_empty[s], 1); }
    for (int s = 0; s < SB; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
    for (int s = 0; s < 2; ++s) { mbar_init(&c_full[s], 1); mbar_init(&c_empty[s], 4); }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_shared();
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

  if (warp == 0) {
    if (lane == 0) {  // query producer: float32 slices into the staging ring
      uint32_t fs = 0, fph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
        const int m0 = (tile / P.tiles_n) * TC_BM;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&f_empty[fs], fph ^ 1u, &s_abort, P.err, 11)) { ok = false; break; }
          uint8_t* f = f32r + fs * PJ_F32_STAGE;
          mbar_expect_tx(&f_full[fs], PJ_F32_STAGE);
          tma_load_2d(f, &tq, kb * TC_BK, m0, &f_full[fs]);
          tma_load_2d(f + PJ_F32_STAGE / 2, &tq, kb * TC_BK + 32, m0, &f_full[fs]);
          if (++fs == S32) { fs = 0; fph ^= 1u; }
        }
      }
    }
  } else if (warp == 3) {
    if (lane == 0) {  // W producer: bf16 slices (hi, and lo) into the B ring
      uint32_t bs = 0, bph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
        const int n0 = (tile % P.tiles_n) * BN;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&b_empty[bs], bph ^ 1u, &s_abort, P.err, 12)) { ok = false; break; }
          uint8_t* b = br + bs * BST;
          mbar_expect_tx(&b_full[bs], BST);
          tma_load_2d(b, &tw, kb * TC_BK, n0, &b_full[bs]);
          if constexpr (THREE) tma_load_2d(b + B_BYTES, &tw, kb * TC_BK, n0 + P.b_lo, &b_full[bs]);
          if (++bs == SB) { bs = 0; bph ^= 1u; }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {  // MMA issuer
      uint32_t as = 0, aph = 0, bs = 0, bph = 0, cs = 0, cph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
        if (!mbar_wait(&c_empty[cs], cph ^ 1u, &s_abort, P.err, 13)) break;
        tc_fence_after();
        const uint32_t dt = tmem + cs * BSTR;
        for (int kb = 0; kb < nkb; ++kb) {
          if (!mbar_wait(&a_full[as], aph, &s_abort, P.err, 14) ||
              !mbar_wait(&b_full[bs], bph, &s_abort, P.err, 18)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(ar + as * AST), sb = su32(br + bs * BST);
          const uint64_t ah = sdesc(sa), bh = sdesc(sb);
#pragma unroll
          for (int kk = 0; kk < TC_BK / 16; ++kk)
            tc_mma(dt, ah + 2ull * kk, bh + 2ull * kk, IDESC, (kb | kk) != 0 ? 1u : 0u);
          if constexpr (THREE) {
            const uint64_t al = sdesc(sa + A_BYTES), bl = sdesc(sb + B_BYTES);
#pragma unroll
            for (int kk = 0; kk < TC_BK / 16; ++kk) {
              tc_mma(dt, ah + 2ull * kk, bl + 2ull * kk, IDESC, 1u);
              tc_mma(dt, al + 2ull * kk, bh + 2ull * kk, IDESC, 1u);
            }
          }
          tc_commit(&a_empty[as]);
          tc_commit(&b_empty[bs]);
          if (++as == SA) { as = 0; aph ^= 1u; }
          if (++bs == SB) { bs = 0; bph ^= 1u; }
        }
        if (!ok) break;
        tc_commit(&c_full[cs]);
        cs ^= 1u;
        if (cs == 0) cph ^= 1u;
      }
    }
  } else if (warp >= 4 && warp < 8) {  // converters: thread t owns row t of each slice
    const int t = threadIdx.x - 128;
    const int sw = t & 7;
    uint32_t fs = 0, fph = 0, as = 0, aph = 0;
    bool ok = true;
    for (int tile = blockIdx.x; ok && tile < P.tiles; tile += gridDim.x) {
      for (int kb = 0; kb < nkb; ++kb) {
        // the centre of this slice's 64 coordinates, read while the slice lands
        const int kc = kb * TC_BK;
        float4 mu4[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          mu4[j] = kc + 4 * j < P.K ? __ldg(reinterpret_cast<const float4*>(P.mu + kc) + j)
                                    : make_float4(0.f, 0.f, 0.f, 0.f);
        if (!mbar_wait(&f_full[fs], fph, &s_abort, P.err, 15) ||
            !mbar_wait(&a_empty[as], aph ^ 1u, &s_abort, P.err, 16)) {
          ok = false;
          break;
        }
        const uint8_t* f = f32r + fs * PJ_F32_STAGE + t * 128;
        uint8_t* ah = ar + as * AST + t * 128;
#pragma unroll
        for (int c = 0; c < 8; ++c) {  // 8 consecutive k per 16-byte bf16 chunk
          const uint8_t* fb = f + (c >> 2) * (PJ_F32_STAGE / 2);
          const int u0 = 2 * (c & 3);
          const float4 v0 = *reinterpret_cast<const float4*>(fb + ((u0 ^ sw) << 4));
          const float4 v1 = *reinterpret_cast<const float4*>(fb + (((u0 + 1) ^ sw) << 4));
          // K is a multiple of 8: a chunk is all inside or all outside (zero there)
          const bool in = kc + 8 * c < P.K;
          const float4 m0 = mu4[2 * c], m1 = mu4[2 * c + 1];
          float x[8] = {v0.x - m0.x, v0.y - m0.y, v0.z - m0.z, v0.w - m0.w,
                        v1.x - m1.x, v1.y - m1.y, v1.z - m1.z, v1.w - m1.w};
          if (!in) {
#pragma unroll
            for (int j = 0; j < 8; ++j) x[j] = 0.f;
          }
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * j], x[2 * j + 1]);
            hw[j] = *reinterpret_cast<const uint32_t*>(&h);
            if constexpr (THREE) {
              const float2 hf = __bfloat1622float2(h);
              const __nv_bfloat162 l = __floats2bfloat162_rn(x[2 * j] - hf.x, x[2 * j + 1] - hf.y);
              lw[j] = *reinterpret_cast<const uint32_t*>(&l);
            }
          }
          const int du = (c ^ sw) << 4;
          *reinterpret_cast<uint4*>(ah + du) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          if constexpr (THREE)
            *reinterpret_cast<uint4*>(ah + A_BYTES + du) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        fence_async_shared();  // the operand rows are read by the tensor cores (async proxy)
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&f_empty[fs]);
          mbar_arrive(&a_full[as]);
        }
        if (++fs == S32) { fs = 0; fph ^= 1u; }
        if (++as == SA) { as = 0; aph ^= 1u; }
      }
    }
  } else if (warp >= 8) {  // epilogue: warp 8 + q drains accumulator lanes 32q .. 32q + 31
    const int quarter = warp & 3;
    uint32_t cs = 0, cph = 0;
    for (int tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
      const int m0 = (tile / P.tiles_n) * TC_BM, n0 = (tile % P.tiles_n) * BN;
      if (!mbar_wait(&c_full[cs], cph, &s_abort, P.err, 17, 2000)) break;
      tc_fence_after();
      const uint32_t trow = tmem + ((uint32_t)(quarter * 32) << 16) + cs * BSTR;
      const int row = m0 + quarter * 32 + lane;
      for (int c = 0; c < BN; c += 32) {
        uint32_t r[32];
        tc_ld32(trow + (uint32_t)c, r);
        const int col0 = n0 + c;
        if (row >= P.M || col0 >= P.N) continue;
        if (P.pbf && col0 + 32 <= P.split) {
          uint32_t hw[16], lw[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const float x0 = __uint_as_float(r[2 * j]), x1 = __uint_as_float(r[2 * j + 1]);
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            const float2 hf = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(x0 - hf.x, x1 - hf.y);
            hw[j] = *reinterpret_cast<const uint32_t*>(&h);
            lw[j] = *reinterpret_cast<const uint32_t*>(&l);
          }
          uint4* dh = reinterpret_cast<uint4*>(P.pbf + (int64_t)row * P.split + col0);
#pragma unroll
          for (int j = 0; j < 4; ++j) dh[j] = make_uint4(hw[4 * j], hw[4 * j + 1], hw[4 * j + 2], hw[4 * j + 3]);
          if (P.pbf_two) {
            uint4* dl = reinterpret_cast<uint4*>(P.pbf + ((int64_t)P.M + row) * P.split + col0);
#pragma unroll
            for (int j = 0; j < 4; ++j)
              dl[j] = make_uint4(lw[4 * j], lw[4 * j + 1], lw[4 * j + 2], lw[4 * j + 3]);
          }
        }
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
            const int col = col0 + j;
            if (col >= P.N) break;
            if (col < P.split) P.out0[(int64_t)row * P.ld0 + col] = __uint_as_float(r[j]);
            else P.out1[(int64_t)row * P.ld1 + (col - P.split)] = __uint_as_float(r[j]);
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&c_empty[cs]);
      cs ^= 1u;
      if (cs == 0) cph ^= 1u;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 2)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(NCOLS)
                 : "memory");
}

// x = X[m, k] - shift[k] -> hi = bf16(x) (row m), lo = bf16(x - hi) (row M + m).
// One warp per row (8 rows per block); with vec (K, ld multiples of 4 and X, shift,
// out 16-byte aligned) each lane converts 4 consecutive k per step.
__global__ void k_split_bf16(const float* __restrict__ X, int M, int K, int ld,
                             const float* __restrict__ shift, int two, int vec,
                             __nv_bfloat16* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t m = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (m >= M) return;
  const float* x = X + m * ld;
  __nv_bfloat16* hi = out + m * K;
  __nv_bfloat16* lo = out + ((int64_t)M + m) * K;
  if (vec) {
    const int k4 = K >> 2;
#pragma unroll 8
    for (int c = lane; c < k4; c += 32) {
      float4 v = __ldg(reinterpret_cast<const float4*>(x) + c);
      if (shift) {
        const float4 sh = __ldg(reinterpret_cast<const float4*>(shift) + c);
        v.x -= sh.x; v.y -= sh.y; v.z -= sh.z; v.w -= sh.w;
      }
      const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y);
      const __nv_bfloat162 h1 = __floats2bfloat162_rn(v.z, v.w);
      uint2 hv;
      hv.x = *reinterpret_cast<const uint32_t*>(&h0);
      hv.y = *reinterpret_cast<const uint32_t*>(&h1);
      reinterpret_cast<uint2*>(hi)[c] = hv;
      if (two) {
        const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
        const __nv_bfloat162 l0 = __floats2bfloat162_rn(v.x - f0.x, v.y - f0.y);
        const __nv_bfloat162 l1 = __floats2bfloat162_rn(v.z - f1.x, v.w - f1.y);
        uint2 lv;
        lv.x = *reinterpret_cast<const uint32_t*>(&l0);
        lv.y = *reinterpret_cast<const uint32_t*>(&l1);
        reinterpret_cast<uint2*>(lo)[c] = lv;
      }
    }
  } else {
    for (int k = lane; k < K; k += 32) {
      const float v = x[k] - (shift ? shift[k] : 0.f);
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      hi[k] = h;
      if (two) lo[k] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
  }
}

// launch of k_split_bf16 for an M x K block of X (row stride ld)
void split_bf16(const float* X, int M, int K, int ld, const float* shift, bool two,
                __nv_bfloat16* out, cudaStream_t st) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  const int vec = (K % 4 == 0 && ld % 4 == 0 && al16(X) && (!shift || al16(shift)) &&
                   (reinterpret_cast<uintptr_t>(out) & 7) == 0)
                      ? 1
                      : 0;
  k_split_bf16<<<ceil_div(M, 8), 256, 0, st>>>(X, M, K, ld, shift, two ? 1 : 0, vec, out);
  MRQ_CHECK_LAUNCH();
}

// Row-scaled e4m3 of an M x K block of X (row stride ld), centred by `shift` when given
// (one warp per row): scale[m] = max_k |x_mk - shift_k| / 448 (1 for a zero row) and
// out[m * K + k] = e4m3((x_mk - shift_k) / scale[m]), rounded to nearest, saturating.
__global__ void k_quant_fp8(const float* __restrict__ X, int M, int K, int ld,
                            const float* __restrict__ shift, uint8_t* __restrict__ out,
                            float* __restrict__ scale) {
  const int64_t m = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (m >= M) return;
  const int lane = threadIdx.x & 31;
  const float* x = X + m * (int64_t)ld;
  float amax = 0.f;
  for (int k = lane; k < K; k += 32) amax = fmaxf(amax, fabsf(x[k] - (shift ? shift[k] : 0.f)));
#pragma unroll
  for (int o = 16; o; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(0xffffffffu, amax, o));
  const float sc = amax > 0.f ? amax / 448.f : 1.f;
  uint8_t* o8 = out + m * (int64_t)K;
  for (int k = lane; k < K; k += 32)
    o8[k] = (uint8_t)__nv_cvt_float_to_fp8((x[k] - (shift ? shift[k] : 0.f)) / sc, __NV_SATFINITE,
                                           __NV_E4M3);
  if (lane == 0) scale[m] = sc;
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

// K-major operand of `rows` rows, 128-byte swizzled slices of K (bf16, or e4m3 bytes)
CUtensorMap make_map(const void* base, uint64_t rows, uint64_t K, uint32_t box_rows, bool f8 = false) {
  CUtensorMap m;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {K * (f8 ? 1 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)(f8 ? 2 * TC_BK : TC_BK), box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, f8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                           2, const_cast<void*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(MRQ_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// float32 rows (K contiguous) read as 128-byte swizzled boxes of 32 floats x box_rows
CUtensorMap make_map_f32(const float* base, uint64_t rows, uint64_t K, uint32_t box_rows) {
  CUtensorMap m;
  cuuint64_t dims[2] = {K, rows};
  cuuint64_t strides[1] = {K * 4};
  cuuint32_t box[2] = {32, box_rows};
  cuuint32_t es[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims,
                           strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) fail(MRQ_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

// The pipeline error word (and a page-locked host copy for asynchronous readback) of
// each device, made on first use with that device current: a kernel only ever writes
// the word of the device it runs on.
constexpr int TC_MAX_DEVICES = 64;
std::mutex g_err_mu;
int* g_err_dev[TC_MAX_DEVICES] = {};
int* g_err_host[TC_MAX_DEVICES] = {};

int current_device_slot() {
  int dev = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  MRQ_REQUIRE(dev >= 0 && dev < TC_MAX_DEVICES, "device ordinal too large for the error-word table");
  return dev;
}

template <int BN, int PSEL, int STAGES, bool F8 = false>
void launch_tc(const void* A2, const void* B2, const TcArgs& a, cudaStream_t st) {
  constexpr int STAGE = TC_BM * TC_BK * 2 + BN * TC_BK * 2;
  const size_t smem = (size_t)STAGES * STAGE + 1024;
  const uint64_t arows = (uint64_t)a.M * (a.phases == 3 ? 2 : 1);
  const uint64_t brows = (uint64_t)a.N * (a.phases == 3 ? 2 : 1);
  CUtensorMap ta = make_map(A2, arows, a.K, TC_BM, F8);
  CUtensorMap tb = make_map(B2, brows, a.K, BN, F8);
  ensure_smem((const void*)k_gemm_tc<BN, PSEL, STAGES, F8>, smem);
  dim3 grid(ceil_div(a.M, TC_BM), ceil_div(a.N, BN));
  k_gemm_tc<BN, PSEL, STAGES, F8><<<grid, 256, smem, st>>>(ta, tb, a);
  MRQ_CHECK_LAUNCH();
}

int sm_count() {
  int dev = 0, n = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  MRQ_CUDA(cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev));
  return n;
}

template <int BN, int SA, int SB, int S32, bool THREE>
void launch_proj(const float* Q, const __nv_bfloat16* W2, ProjArgs a, cudaStream_t st) {
  constexpr int AST = TC_BM * TC_BK * 2 * (THREE ? 2 : 1);
  constexpr int BST = BN * TC_BK * 2 * (THREE ? 2 : 1);
  const size_t smem = (size_t)SA * AST + (size_t)SB * BST + (size_t)S32 * PJ_F32_STAGE + 1024;
  CUtensorMap tq = make_map_f32(Q, (uint64_t)a.M, (uint64_t)a.K, TC_BM);
  CUtensorMap tw = make_map(W2, (uint64_t)a.N * (THREE ? 2 : 1), a.K, BN);
  a.tiles_n = ceil_div(a.N, BN);
  a.tiles = ceil_div(a.M, TC_BM) * a.tiles_n;
  ensure_smem((const void*)k_proj_tc<BN, SA, SB, S32, THREE>, smem);
  const int grid = std::min(a.tiles, sm_count());
  k_proj_tc<BN, SA, SB, S32, THREE><<<grid, PJ_THREADS, smem, st>>>(tq, tw, a);
  MRQ_CHECK_LAUNCH();
}

// the row-scaled FP8 projection (epi 0, one phase): e4m3 A (M x K) and B (N x K)
void run_tc_f8(const uint8_t* A8, const uint8_t* B8, TcArgs a, cudaStream_t st) {
  if (!a.err) a.err = tc_error_word();
  if (a.N <= 64) launch_tc<64, 4, 4, true>(A8, B8, a, st);
  else if (a.N <= 128) launch_tc<128, 4, 4, true>(A8, B8, a, st);
  else launch_tc<256, 4, 4, true>(A8, B8, a, st);
}

void run_tc(const __nv_bfloat16* A2, const __nv_bfloat16* B2, TcArgs a, cudaStream_t st) {
  a.err = tc_error_word();
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

int* tc_error_word() {
  const int dev = current_device_slot();
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_dev[dev]) {
    int* p = nullptr;
    MRQ_CUDA(cudaMalloc(&p, sizeof(int)));
    MRQ_CUDA(cudaMemset(p, 0, sizeof(int)));
    g_err_dev[dev] = p;
  }
  return g_err_dev[dev];
}

int* tc_error_mirror() {
  const int dev = current_device_slot();
  std::lock_guard<std::mutex> lk(g_err_mu);
  if (!g_err_host[dev]) {
    int* h = nullptr;
    MRQ_CUDA(cudaHostAlloc(reinterpret_cast<void**>(&h), sizeof(int), cudaHostAllocDefault));
    g_err_host[dev] = h;
  }
  return g_err_host[dev];
}

int tc_check_error() {
  const int dev = current_device_slot();
  int* w = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_err_mu);
    w = g_err_dev[dev];
  }
  if (!w) return 0;
  int h = 0;
  MRQ_CUDA(cudaMemcpy(&h, w, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) MRQ_CUDA(cudaMemset(w, 0, sizeof(int)));
  return h;
}

// The fused projection when its operands allow it (float32 query rows in device memory,
// which its TMA loads read; rows and centre 16-byte aligned; D a multiple
// of 8); false leaves the work to the split + GEMM path.
bool project_fused(const float* Q, const float* mu, const __nv_bfloat16* W2, int M, int D, int d,
                   bool split3, float* qd, int ldd, float* qr, int ldr, __nv_bfloat16* probe_bf,
                   int* err, cudaStream_t st) {
  auto al16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (M <= 0 || D % 8 != 0 || !al16(Q) || !al16(mu)) return false;
  cudaPointerAttributes pa{};
  if (cudaPointerGetAttributes(&pa, Q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (pa.type != cudaMemoryTypeDevice) return false;
  ProjArgs a{};
  a.M = M; a.N = D; a.K = D;
  a.b_lo = D;
  a.mu = mu;
  a.out0 = qd; a.ld0 = ldd; a.out1 = qr; a.ld1 = ldr; a.split = d;
  a.pbf = (d % 32 == 0) ? probe_bf : nullptr;
  a.pbf_two = split3 ? 1 : 0;
  a.err = err;
  // the operand traffic of a CTA (float32 query rows, bf16 rows of W) grows with the
  // tiles it runs: pick the tile width whose busiest SM moves the fewest bytes
  const int sms = sm_count();
  auto busiest = [&](int bn) {
    const int64_t tiles = (int64_t)ceil_div(M, TC_BM) * ceil_div(D, bn);
    const int64_t per_tile = (int64_t)D * (TC_BM * 4 + (int64_t)bn * 2 * (split3 ? 2 : 1));
    return ((tiles + sms - 1) / sms) * per_tile;
  };
  // rings (A stages, B stages, float32 stages) within 227 KB of shared memory
  if (split3) {
    if (D <= 64) launch_proj<64, 2, 3, 2, true>(Q, W2, a, st);
    else launch_proj<128, 2, 2, 2, true>(Q, W2, a, st);
  } else if (D <= 64) {
    launch_proj<64, 2, 4, 4, false>(Q, W2, a, st);
  } else if (D <= 128) {
    launch_proj<128, 2, 4, 3, false>(Q, W2, a, st);
  } else {
    const int64_t c128 = busiest(128), c192 = busiest(192), c256 = busiest(256);
    if (c256 <= c192 && c256 <= c128) launch_proj<256, 2, 3, 3, false>(Q, W2, a, st);
    else if (c192 <= c128) launch_proj<192, 2, 4, 3, false>(Q, W2, a, st);
    else launch_proj<128, 2, 4, 3, false>(Q, W2, a, st);
  }
  return true;
}

int project_tc(const float* Q, const float* mu, const __nv_bfloat16* W2, int M, int D, int d,
               bool split3, __nv_bfloat16* qbf, float* qd, float* qr, cudaStream_t st,
               __nv_bfloat16* probe_bf) {
  if (project_fused(Q, mu, W2, M, D, d, split3, qd, d, qr, D - d, probe_bf, tc_error_word(), st))
    return 1;
  split_bf16(Q, M, D, D, mu, split3, qbf, st);
  TcArgs a{};
  a.M = M; a.N = D; a.K = D;
  a.phases = split3 ? 3 : 1;
  a.a_lo = M; a.b_lo = D;
  a.epi = 0;
  a.out0 = qd; a.ld0 = d; a.out1 = qr; a.ld1 = D - d; a.split = d;
  a.pbf = (d % 32 == 0) ? probe_bf : nullptr;
  a.pbf_two = split3 ? 1 : 0;
  run_tc(qbf, W2, a, st);
  return 2;
}

void quantize_rows_fp8(const float* X, int M, int K, int ld, const float* shift, uint8_t* out,
                       float* scale, cudaStream_t st) {
  if (M <= 0) return;
  k_quant_fp8<<<ceil_div(M, 8), 256, 0, st>>>(X, M, K, ld, shift, out, scale);
  MRQ_CHECK_LAUNCH();
}

void project_fp8(const float* Q, const float* mu, const uint8_t* W8, const float* W8s, int M,
                 int D, int d, uint8_t* q8, float* q8s, float* qd, int ldd, float* qr, int ldr,
                 cudaStream_t st, __nv_bfloat16* probe_bf, int* err) {
  quantize_rows_fp8(Q, M, D, D, mu, q8, q8s, st);
  TcArgs a{};
  a.M = M; a.N = D; a.K = D;
  a.phases = 1;
  a.epi = 0;
  a.out0 = qd; a.ld0 = ldd; a.out1 = qr; a.ld1 = ldr; a.split = d;
  a.pbf = (d % 32 == 0) ? probe_bf : nullptr;
  a.pbf_two = 0;
  a.rscale = q8s; a.cscale = W8s;
  a.err = err;
  run_tc_f8(q8, W8, a, st);
}

void probe_tc(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
              int M, int nlist, int d, bool split3, __nv_bfloat16* qbf, float* gmat,
              cudaStream_t st, bool presplit) {
  if (!presplit) split_bf16(qd, M, d, d, nullptr, split3, qbf, st);
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
int probe_tc_parts(int nlist) {
  const int bn = nlist <= 64 ? 64 : nlist <= 128 ? 128 : 256;
  return 2 * ceil_div(nlist, bn);  // column tiles x two halves
}

int probe_tc_topk(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
                  int M, int nlist, int d, bool split3, int nsel, __nv_bfloat16* qbf,
                  unsigned long long* part, cudaStream_t st, bool presplit) {
  if (!presplit) split_bf16(qd, M, d, d, nullptr, split3, qbf, st);
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
  if (precision == MRQ_PREC_FP8) {
    // scratch: [0, 256) error word, then the e4m3 queries (nq x D bytes, rounded up to
    // 256), then their row scales
    const int64_t qbytes = (nq * D + 255) / 256 * 256;
    const int64_t need = qbytes + 4 * nq;
    if (need > MRQ_PROJECT_NOALLOC_MAX_BYTES)
      fail(MRQ_EINVAL, "mrq_project_noalloc: nq * D = " + std::to_string(nq * D) + " needs " +
                           std::to_string(need) + " bytes of scratch at FP8, more than its fixed " +
                           std::to_string(MRQ_PROJECT_NOALLOC_MAX_BYTES) + "; split the batch");
    MRQ_REQUIRE(tc_available(), "tensor-core projection needs an sm_103 device");
    MRQ_REQUIRE(idx->W8.p != nullptr, "FP8 projection needs D to be a multiple of 16");
    unsigned char* base = project_scratch();
    int* err = reinterpret_cast<int*>(base);
    uint8_t* q8 = base + 256;
    float* q8s = reinterpret_cast<float*>(base + 256 + qbytes);
    MRQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
    project_fp8(q, idx->mu.p, idx->W8.p, idx->W8s.p, (int)nq, D, d, q8, q8s, qp, D, qp + d, D,
                st, nullptr, err);
    int h = 0;
    MRQ_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
    if (h) fail(MRQ_ETIMEDOUT, "a tensor-core kernel gave up waiting on its pipeline");
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
  MRQ_REQUIRE(D % 8 == 0, "tensor-core precisions need D to be a multiple of 8 (16-byte bf16 rows)");
  unsigned char* base = project_scratch();
  int* err = reinterpret_cast<int*>(base);
  __nv_bfloat16* qbf = reinterpret_cast<__nv_bfloat16*>(base + 256);
  MRQ_CUDA(cudaMemsetAsync(err, 0, sizeof(int), st));
  if (!project_fused(q, idx->mu.p, idx->W2.p, (int)nq, D, d, split3, qp, D, qp + d, D, nullptr,
                     err, st)) {
    split_bf16(q, (int)nq, D, D, idx->mu.p, split3, qbf, st);
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
  }
  int h = 0;
  MRQ_CUDA(cudaMemcpyAsync(&h, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  MRQ_CUDA(cudaStreamSynchronize(st));
  if (h) fail(MRQ_ETIMEDOUT, "a tensor-core kernel gave up waiting on its pipeline");
}

}  // namespace mrq

// ---------------------------------------------------------------- tensor-core batched scan
namespace mrq {
namespace {

// byte offset of element (row, k) of a K-major one-byte (e4m3) tile of `rows` rows stored
// as 128-byte swizzled K slices (128 elements per row per slice; 16-byte chunk c of row r
// at c ^ (r % 8)), the layout TMA writes with CU_TENSOR_MAP_SWIZZLE_128B and the MMA
// descriptor reads
__device__ __forceinline__ uint32_t sw128_off8(int rows, int row, int k) {
  const int slice = k >> 7, kin = k & 127;
  return (uint32_t)(slice * rows * 128 + (row >> 3) * 1024 + (row & 7) * 128 +
                    ((((kin >> 4) ^ (row & 7)) << 4) | (kin & 15)));
}


// e4m3 bytes of two small non-negative integers (exact up to 16)
__device__ __forceinline__ uint32_t e4m3x2(int v0, int v1) {
  return (uint32_t)__nv_cvt_float2_to_fp8x2(make_float2((float)v0, (float)v1), __NV_SATFINITE,
                                            __NV_E4M3);
}

// Stage 1 (Eq. 4, Eq. 5, the bound test of Algorithm 2) for a work item (list j, tile
// of 128 candidates, group of up to 128 pairs probing j).  The candidates' B-bit levels
// u and the pairs' quantized query codes qbar (integers 0..15, exact in e4m3) are written
// to shared memory as e4m3 bytes and one tcgen05 MMA chain (kind::f8f6f4) gives every
// integer dot <u, qbar> in fp32 (exact below 2^24).  The epilogue applies the same
// arithmetic, bound updates and survivor compaction as the popcount batched scan, per
// (pair, 32 candidates).  256 threads: two per candidate row for the expansion; the
// eight warps drain the accumulator (warp w: rows 32*(w%4).., columns 64*(w/4)..).
// Persistent over items.
template <int NCH, int BITS>
__global__ void __launch_bounds__(256) k_scan_tc(TcScanParams P) {
  constexpr int DQ = NCH * 32;
  constexpr int W = BITS * NCH;
  constexpr int VW = (W % 4 == 0) ? 4 : (W % 2 == 0) ? 2 : 1;
  constexpr int NQ = TC_SCAN_GROUP;
  constexpr int TR = TC_SCAN_TILE;
  constexpr int KS = DQ / 128;  // 128-byte K slices
  constexpr int HC = NCH / 2;   // 32-dim chunks expanded by each of a row's two threads
  constexpr int topc = (1 << BITS) - 1;
  constexpr uint32_t IDESC = idesc_e4m3<NQ>();
  constexpr int A_BYTES = TR * DQ;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* sA = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                           ~static_cast<uintptr_t>(1023));
  uint8_t* sB = sA + A_BYTES;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int s_abort;
  __shared__ int s_item;
  __shared__ int s_pair[NQ];
  __shared__ PairQ s_pq[NQ];

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    s_abort = 0;
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_slot)),
                 "r"((uint32_t)NQ)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const int n_items = *P.nitems;
  uint32_t phase = 0;
  const int row = tid & (TR - 1), hh = tid >> 7;  // candidate row, which half of its chunks
  const int quarter = warp & 3, half = warp >> 2;

  while (true) {
    if (tid == 0) s_item = (int)atomicAdd(P.work, 1u);
    __syncthreads();
    const int it = s_item;
    if (it >= n_items || s_abort) break;
    const int4 item = P.items[it];
    const int j = item.x;
    const int64_t lb0 = P.loff[j];
    const int64_t size = P.loff[j + 1] - lb0;
    const int g0 = P.loffq[j] + item.z * NQ;
    const int ng = min(P.loffq[j] + P.lcount[j], g0 + NQ) - g0;
    if (tid < NQ) {
      const int w = tid < ng ? P.lqueue[g0 + tid] : -1;
      s_pair[tid] = w;
      if (w >= 0) s_pq[tid] = P.pq[w];
    }
    // A: levels of this row's candidate (two threads per row, HC chunks each), e4m3
    {
      const int64_t idx = (int64_t)item.y * TR + row;
      const bool valid = idx < size;
      const int64_t pp = P.ploff[j] + idx;
      const uint32_t* cbase = P.codes + (pp >> 5) * (int64_t)(W * 32) + (pp & 31) * VW;
#pragma unroll
      for (int cc = 0; cc < HC; ++cc) {
        const int c = hh * HC + cc;
        uint32_t pw[BITS];
#pragma unroll
        for (int a = 0; a < BITS; ++a) {
          const int wi = a * NCH + c;
          pw[a] = valid ? __ldg(cbase + (wi / VW) * 32 * VW + (wi % VW)) : 0u;
        }
#pragma unroll
        for (int hx = 0; hx < 2; ++hx) {  // 16 dims (one 16-byte chunk) at a time
          uint32_t packed[4];
#pragma unroll
          for (int t4 = 0; t4 < 4; ++t4) {
            int v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const int bit = hx * 16 + t4 * 4 + u;
              int val = 0;
#pragma unroll
              for (int a = 0; a < BITS; ++a) val |= (int)((pw[a] >> bit) & 1u) << a;
              v[u] = val;
            }
            packed[t4] = e4m3x2(v[0], v[1]) | (e4m3x2(v[2], v[3]) << 16);
          }
          *reinterpret_cast<uint4*>(sA + sw128_off8(TR, row, c * 32 + hx * 16)) =
              make_uint4(packed[0], packed[1], packed[2], packed[3]);
        }
      }
    }
    __syncthreads();  // s_pair / s_pq visible
    // B: the group's query codes, zero rows past the group
    for (int e = tid; e < NQ * (DQ / 16); e += 256) {
      const int n = e / (DQ / 16), kc = e % (DQ / 16);
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      const int w = s_pair[n];
      if (w >= 0) v = __ldg(reinterpret_cast<const uint4*>(P.qrow + (int64_t)w * DQ) + kc);
      *reinterpret_cast<uint4*>(sB + sw128_off8(NQ, n, kc * 16)) = v;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // visible to the MMA
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < KS; ++s) {
        const uint64_t ad = sdesc(su32(sA + s * TR * 128)), bd = sdesc(su32(sB + s * NQ * 128));
#pragma unroll
        for (int kk = 0; kk < 4; ++kk)
          tc_mma_f8(tmem, ad + 2ull * kk, bd + 2ull * kk, IDESC, (s | kk) != 0 ? 1u : 0u);
      }
      tc_commit(&mbar);
    }
    mbar_wait(&mbar, phase, &s_abort, P.err, 4, 20000);
    phase ^= 1u;
    tc_fence_after();
    __syncthreads();  // every thread past the wait (or all of them told to stop)
    if (s_abort) break;
    // epilogue: warp (quarter, half) scores rows 32*quarter.. against columns 64*half..,
    // 32 columns at a time, staging each 32 x 32 block of dots in the idle operand area
    {
      const int r = quarter * 32 + lane;
      const int64_t idx = (int64_t)item.y * TR + r;
      const bool valid = idx < size;
      const int64_t pp = P.ploff[j] + idx;
      float* stg = reinterpret_cast<float*>(sA) + warp * (32 * 33);
      float fa = 0.f, fr = 0.f, fe = 0.f;
      int su = 0;
      if (valid) {
        fa = __ldg(P.fadd + pp);
        fr = __ldg(P.fres + pp);
        fe = __ldg(P.ferr + pp);
        const uint32_t* cbase = P.codes + (pp >> 5) * (int64_t)(W * 32) + (pp & 31) * VW;
#pragma unroll
        for (int wi = 0; wi < W; ++wi)
          su += __popc(__ldg(cbase + (wi / VW) * 32 * VW + (wi % VW))) << (wi / NCH);
      }
      for (int cb = 0; cb < 2; ++cb) {
        const int c0 = half * 64 + cb * 32;
        if (c0 >= ng) break;  // warp-uniform
        uint32_t acc[32];
        tc_ld32(tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)c0, acc);
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 32; ++t) stg[lane * 33 + t] = __uint_as_float(acc[t]);
        __syncwarp();
        const int ncol = min(32, ng - c0);
        // the running bounds of the columns' queries, one lane each
        const float my_tau = lane < ncol ? fkey_inv(__ldcg(P.gtau + s_pq[c0 + lane].q)) : FLT_INF_F;
        for (int t = 0; t < ncol; ++t) {
          const PairQ pr = s_pq[c0 + t];
          const int64_t q = pr.q;
          const int dot = (int)stg[lane * 33 + t];
          const float ip = pr.qdelta * (float)(2 * dot - topc * pr.qsum) +
                           pr.ql * (float)(2 * su - DQ * topc);
          const float dis = fa + pr.a0 + fr * pr.sg * ip;  // Eq. 4
          const float eps = pr.e0 * fe + pr.em;            // Eq. 5 + Chebyshev
          const float lb = valid ? dis - eps : FLT_INF_F;
          const float ub = valid ? dis + eps : FLT_INF_F;
          // the bound as read at the start of these columns (a valid upper bound of tau_A;
          // tightening by other warps since only means more survivors, filtered later)
          float tau = __shfl_sync(0xffffffffu, my_tau, t);
          if (P.k <= 32) {
            const unsigned below = __ballot_sync(0xffffffffu, ub < tau);
            if (__popc(below) >= P.k) {
              float v = ub < tau ? ub : FLT_INF_F;
#pragma unroll
              for (int size2 = 2; size2 <= 32; size2 <<= 1) {
#pragma unroll
                for (int stride = size2 >> 1; stride > 0; stride >>= 1) {
                  const float o = __shfl_xor_sync(0xffffffffu, v, stride);
                  const bool up = ((lane & size2) == 0);
                  const bool lower = (lane & stride) == 0;
                  v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
                }
              }
              const float kth = __shfl_sync(0xffffffffu, v, P.k - 1);
              if (kth < tau) {
                tau = kth;
                if (lane == 0) atomicMin(P.gtau + q, fkey(kth));
              }
            }
          }
          const bool surv = lb <= tau;
          const unsigned sm = __ballot_sync(0xffffffffu, surv);
          if (sm) {
            unsigned base = 0;
            if (lane == 0) base = atomicAdd(P.qcnt + q, (unsigned)__popc(sm));
            base = __shfl_sync(0xffffffffu, base, 0);
            const int64_t rel = (int64_t)base + __popc(sm & ((1u << lane) - 1));
            if (surv && rel < P.cap) {  // past the region: counted only (the query is redone)
              const int64_t at = q * P.cap + rel;
              P.spos[at] = (int32_t)(lb0 + idx);
              P.slb[at] = lb;
              P.sub[at] = ub;
            }
          }
        }
        __syncwarp();
      }
    }
    tc_fence_before();
    __syncthreads();  // staging and accumulator reads done before the next item
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)NQ)
                 : "memory");
}

template <int NCH, int BITS>
void launch_scan_tc(const TcScanParams& p, cudaStream_t st) {
  constexpr int DQ = NCH * 32;
  const size_t ab = (size_t)TC_SCAN_TILE * DQ + (size_t)TC_SCAN_GROUP * DQ;
  const size_t smem = std::max(ab, (size_t)8 * 32 * 33 * 4) + 1024;
  auto kern = k_scan_tc<NCH, BITS>;
  ensure_smem((const void*)kern, smem);
  // prefer the largest shared-memory carveout
  MRQ_CUDA(cudaFuncSetAttribute((const void*)kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  // The occupancy calculator reports one CTA per SM for kernels that allocate tensor
  // memory; with 128 columns and ~65 KB of shared memory each, three fit per SM (the
  // register file allows three at 80 registers), so launch three per SM.  CTAs that are
  // not resident start later and find the item queue drained.
  int dev = 0, nsm = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  MRQ_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int per_sm = smem <= 70 * 1024 ? 3 : smem <= 110 * 1024 ? 2 : 1;
  kern<<<nsm * per_sm, 256, smem, st>>>(p);
  MRQ_CHECK_LAUNCH();
}

}  // namespace

bool scan_tc_supported(int d, int bits, int qbits) {
  if (d % 128 != 0 || d < 128 || d > 512) return false;  // whole 128-byte e4m3 slices
  if (!(bits == 1 || bits == 2 || bits == 4) || qbits < 1 || qbits > 4) return false;
  const int64_t top = (int64_t)d * ((1 << bits) - 1) * ((1 << qbits) - 1);
  return top < (1 << 24);
}

void scan_tc(const TcScanParams& p, int d, int bits, cudaStream_t st) {
  const int nch = d / 32;
#define MRQ_STC(N, B)                      \
  if (nch == N && bits == B) {             \
    launch_scan_tc<N, B>(p, st);           \
    return;                                \
  }
  MRQ_STC(4, 1) MRQ_STC(4, 2) MRQ_STC(4, 4) MRQ_STC(8, 1) MRQ_STC(8, 2) MRQ_STC(8, 4)
  MRQ_STC(12, 1) MRQ_STC(12, 2) MRQ_STC(12, 4) MRQ_STC(16, 1) MRQ_STC(16, 2) MRQ_STC(16, 4)
#undef MRQ_STC
  fail(MRQ_EINVAL, "tensor-core scan: unsupported code shape");
}

}  // namespace mrq
