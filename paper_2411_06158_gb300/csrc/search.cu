// Query path of MRQ (Algorithm 2) on the GPU.
//
// Per batch of queries:
//  1. projection  [q_d' | q_r] = W (q - mu)          (gemm_f32.cu / gemm_tc.cu)
//  2. k_qstats    |q_r|^2, sigma (Eq. 6), |q_p|^2
//  3. probe       g_j = |q_d' - c_j'|^2 (direct float32 sums), then k_probe_select
//                 keeps the nprobe smallest, ties to the lower list id
//  4. k_scan      stage 1 for every (query, probed list) pair, one warp per pair
//                 from a device work queue: q' = (q_d' - c')/sqrt(g) (Alg. 2 normalise
//                 and rotate step), the code inner product <v, q'> (float32 nibble
//                 lookup table, or the quantized query with popcounts), Eq. 4
//                 estimate, Eq. 5 + Chebyshev bounds, a running upper bound of
//                 the k-th smallest upper bound, and compaction of the candidates
//                 whose lower bound does not exceed it
//  5. k_finalize  one CTA per query: tau_A, stage-1 survivors, stage 2 (Eq. 7),
//                 tau_B, stage-2 survivors, exact distances, top-k by (dist, id)
#include <cub/cub.cuh>

#include <algorithm>
#include <cfloat>
#include <map>
#include <mutex>
#include <tuple>
#include <unordered_map>

#include <cuda_fp8.h>

#include "common.cuh"

namespace mrq {
namespace {

#define FINF __int_as_float(0x7f800000)

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_min(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_sum_i(int v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------- query stats

__global__ void k_qstats(const float* __restrict__ qd, const float* __restrict__ qr,
                         const float* __restrict__ lam, int64_t nq, int d, int r,
                         float* __restrict__ qstat, unsigned int* __restrict__ qcnt,
                         unsigned int* __restrict__ gtau, unsigned int* __restrict__ work) {
  int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  // the scan's per-query survivor count and running bound, and its work counters,
  // start from zero / +inf (when given)
  if (work && blockIdx.x == 0 && threadIdx.x < 4) work[threadIdx.x] = 0u;
  if (q >= nq) return;
  const int lane = threadIdx.x & 31;
  if (qcnt && lane == 0) {
    qcnt[q] = 0u;
    gtau[q] = fkey(__int_as_float(0x7f800000));
  }
  float qr2 = 0.f, s2 = 0.f, qd2 = 0.f;
  if ((r & 3) == 0) {  // rows and lam + d are 16-byte aligned (d is a multiple of 32)
    const float4* x = reinterpret_cast<const float4*>(qr + q * r);
    const float4* l = reinterpret_cast<const float4*>(lam + d);
#pragma unroll 4
    for (int i = lane; i < (r >> 2); i += 32) {
      const float4 v = __ldg(x + i), w = __ldg(l + i);
      qr2 = fmaf(v.x, v.x, qr2); qr2 = fmaf(v.y, v.y, qr2);
      qr2 = fmaf(v.z, v.z, qr2); qr2 = fmaf(v.w, v.w, qr2);
      s2 = fmaf(v.x * v.x, w.x, s2); s2 = fmaf(v.y * v.y, w.y, s2);
      s2 = fmaf(v.z * v.z, w.z, s2); s2 = fmaf(v.w * v.w, w.w, s2);
    }
  } else {
    for (int i = lane; i < r; i += 32) {
      float v = qr[q * r + i];
      qr2 = fmaf(v, v, qr2);
      s2 = fmaf(v * v, lam[d + i], s2);
    }
  }
  {
    const float4* x = reinterpret_cast<const float4*>(qd + q * d);
#pragma unroll 4
    for (int i = lane; i < (d >> 2); i += 32) {
      const float4 v = __ldg(x + i);
      qd2 = fmaf(v.x, v.x, qd2); qd2 = fmaf(v.y, v.y, qd2);
      qd2 = fmaf(v.z, v.z, qd2); qd2 = fmaf(v.w, v.w, qd2);
    }
  }
  qr2 = warp_sum(qr2);
  s2 = warp_sum(s2);
  qd2 = warp_sum(qd2);
  if (lane == 0) {
    qstat[q * 4 + 0] = qr2;
    qstat[q * 4 + 1] = sqrtf(fmaxf(s2, 0.f));
    qstat[q * 4 + 2] = qd2 + qr2;
    qstat[q * 4 + 3] = qd2;
  }
}

// ---------------------------------------------------- block-level primitives

template <int NT>
__device__ __forceinline__ int block_sum_i(int v, int* red) {
  v = warp_sum_i(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  int t = 0;
#pragma unroll
  for (int w = 0; w < NT / 32; ++w) t += red[w];
  return t;
}

// Smallest orderable key T with #{i : key(vals[i]) <= T} >= k (bisection over the
// 32-bit key space: exact, 32 rounds).  Requires M >= k.
template <int NT>
__device__ uint32_t block_kth_key(const float* vals, int M, int k, int* red) {
  uint32_t lo = 0u, hi = 0xffffffffu;
  while (lo < hi) {
    uint32_t mid = lo + ((hi - lo) >> 1);
    int c = 0;
    for (int i = threadIdx.x; i < M; i += NT) c += fkey(vals[i]) <= mid;
    c = block_sum_i<NT>(c, red);
    if (c >= k) hi = mid; else lo = mid + 1;
  }
  return lo;
}

// Smallest orderable key T with #{i : key_i <= T} >= k, by a 4-pass radix select
// (8 bits per pass, most significant first).  key_i = fkey(vals[i]) (vals may be
// in shared or global memory).  Histogram updates are aggregated per warp with
// __match_any_sync, so equal high bytes do not serialise.  Requires M >= k.
template <int NT>
__device__ uint32_t block_radix_kth(const float* vals, int M, int k, int* hist, int* sh) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0u, mask = 0u;
  int kk = k;
  for (int shift = 24; shift >= 0; shift -= 8) {
    for (int i = threadIdx.x; i < 256; i += NT) hist[i] = 0;
    __syncthreads();
    for (int base = 0; base < M; base += NT) {
      const int i = base + threadIdx.x;
      const uint32_t key = i < M ? fkey(vals[i]) : 0u;
      const bool in = i < M && (key & mask) == prefix;
      const unsigned act = __ballot_sync(0xffffffffu, in);
      if (in) {
        const uint32_t bin = (key >> shift) & 255u;
        const unsigned peers = __match_any_sync(act, bin);
        if (lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
      }
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      int c[8], tot = 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) { c[j] = hist[lane * 8 + j]; tot += c[j]; }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      int acc = incl - tot;
      if (acc < kk && kk <= incl) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          if (acc + c[j] >= kk) { sh[0] = lane * 8 + j; sh[1] = acc; break; }
          acc += c[j];
        }
      }
    }
    __syncthreads();
    prefix |= (uint32_t)sh[0] << shift;
    mask |= 255u << shift;
    kk -= sh[1];
    __syncthreads();
  }
  return prefix;
}

// In-shared-memory ascending bitonic sort of n (power of two) 64-bit keys.
template <int NT>
__device__ void block_bitonic(unsigned long long* a, int n) {
  for (int size = 2; size <= n; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int t = threadIdx.x; t < n / 2; t += NT) {
        int i = 2 * t - (t & (stride - 1));
        int j = i + stride;
        bool up = ((i & size) == 0);
        unsigned long long x = a[i], y = a[j];
        if ((x > y) == up) { a[i] = y; a[j] = x; }
      }
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------- probe select

constexpr int PS_NT = 256;

// Top-nprobe (nprobe <= 32) of one row of the probe-distance matrix, one warp per
// query: the nprobe smallest keys (fkey(g) << 32 | list), which orders ties by the lower
// list id, are kept sorted across the lanes; the row streams through 32 values at a time
// and only keys below the current nprobe-th are inserted.  Writes plist and pg (the
// matrix value; the refine step recomputes g exactly afterwards).
__global__ void __launch_bounds__(256) k_probe_select_warp(const float* __restrict__ gmat,
                                                           int64_t nq, int nlist, int nprobe,
                                                           int32_t* __restrict__ plist,
                                                           float* __restrict__ pg) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (q >= nq) return;
  const float* row = gmat + q * nlist;
  unsigned long long lst = ~0ull, kth = ~0ull;
  for (int b = 0; b < nlist; b += 128) {  // four chunks of loads in flight
    unsigned long long x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int c = b + 32 * u + lane;
      x[u] = c < nlist ? (((unsigned long long)fkey(row[c]) << 32) | (uint32_t)c) : ~0ull;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      unsigned cand = __ballot_sync(0xffffffffu, x[u] < kth);
      while (cand) {
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const unsigned long long y = __shfl_sync(0xffffffffu, x[u], src);
        if (y < kth) {
          const int pos = __popc(__ballot_sync(0xffffffffu, lst < y));
          const unsigned long long up = __shfl_up_sync(0xffffffffu, lst, 1);
          lst = lane > pos ? up : (lane == pos ? y : lst);
          kth = __shfl_sync(0xffffffffu, lst, nprobe - 1);
        }
      }
    }
  }
  if (lane < nprobe) {
    plist[q * nprobe + lane] = (int32_t)(lst & 0xffffffffu);
    pg[q * nprobe + lane] = fkey_inv((uint32_t)(lst >> 32));
  }
}

// The nprobe smallest (g_j, j) of one query, ascending (Algorithm 2, probing).
// Shared memory: sel[cap] (64-bit (key, list) pairs) followed by the staged row
// when it fits.  Every key <= T (the nprobe-th smallest) is gathered and sorted by
// (key, list id), so ties go to the lower list id; if ties overflow sel, an
// ordered pass keeps the lowest ids among the ties instead.
__global__ void __launch_bounds__(PS_NT) k_probe_select(const float* __restrict__ gmat, int nlist,
                                                        int nprobe, int cap, int row_in_smem,
                                                        int32_t* __restrict__ plist,
                                                        float* __restrict__ pg) {
  extern __shared__ unsigned long long sel[];
  __shared__ int hist[256], shv[2];
  __shared__ unsigned int s_cnt;
  __shared__ int s_eq;
  const int64_t q = blockIdx.x;
  const float* g = gmat + q * nlist;
  if (row_in_smem) {
    float* gs = reinterpret_cast<float*>(sel + cap);
    for (int i = threadIdx.x; i < nlist; i += PS_NT) gs[i] = g[i];
    __syncthreads();
    g = gs;
  }
  // linear buckets over [min, max]: bin(g) = floor((g - min) * 1024 / (max - min)) is
  // monotone in g, so the buckets up to the one where the running count reaches nprobe
  // hold the nprobe smallest g (equal values share a bucket); those few are sorted
  // exactly below.  Too many in them (or a constant row): the radix select.
  {
    __shared__ float s_mm[2][PS_NT / 32];
    __shared__ int lhist[1024];
    __shared__ int s_b;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float mn = FINF, mx = -FINF;
    for (int i = threadIdx.x; i < nlist; i += PS_NT) {
      const float v = g[i];
      mn = fminf(mn, v);
      mx = fmaxf(mx, v);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
      mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if (lane == 0) { s_mm[0][wid] = mn; s_mm[1][wid] = mx; }
    for (int i = threadIdx.x; i < 1024; i += PS_NT) lhist[i] = 0;
    __syncthreads();
    mn = s_mm[0][0];
    mx = s_mm[1][0];
#pragma unroll
    for (int w = 1; w < PS_NT / 32; ++w) { mn = fminf(mn, s_mm[0][w]); mx = fmaxf(mx, s_mm[1][w]); }
    const float scale = 1024.f / (mx - mn);
    const bool spread = mx > mn && scale < FINF;
    if (spread) {
      for (int i = threadIdx.x; i < nlist; i += PS_NT)
        atomicAdd(&lhist[min(1023, (int)((g[i] - mn) * scale))], 1);
    }
    __syncthreads();
    if (threadIdx.x < 32) {
      int c[32], tot = 0;
#pragma unroll
      for (int j = 0; j < 32; ++j) { c[j] = lhist[lane * 32 + j]; tot += c[j]; }
      int incl = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      int acc = incl - tot;
      if (lane == 0) s_b = -1;
      __syncwarp();
      if (acc < nprobe && nprobe <= incl) {
        int bsel = lane * 32 + 31;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          acc += c[j];
          if (acc >= nprobe) { bsel = lane * 32 + j; s_cnt = (unsigned)acc; break; }
        }
        s_b = bsel;
      }
    }
    __syncthreads();
    const int bsel = s_b;
    if (spread && bsel >= 0 && (int)s_cnt <= cap) {
      __syncthreads();
      if (threadIdx.x == 0) s_cnt = 0u;
      __syncthreads();
      for (int i = threadIdx.x; i < nlist; i += PS_NT) {
        const float v = g[i];
        if (min(1023, (int)((v - mn) * scale)) <= bsel) {
          const unsigned at = atomicAdd(&s_cnt, 1u);
          sel[at] = ((unsigned long long)fkey(v) << 32) | (uint32_t)i;
        }
      }
      __syncthreads();
      const int n = (int)s_cnt;
      int n2 = 1;
      while (n2 < n) n2 <<= 1;
      for (int i = n + threadIdx.x; i < n2; i += PS_NT) sel[i] = ~0ull;
      block_bitonic<PS_NT>(sel, n2);
      for (int r = threadIdx.x; r < nprobe; r += PS_NT) {
        const unsigned long long v = sel[r];
        plist[q * nprobe + r] = (int32_t)(v & 0xffffffffu);
        pg[q * nprobe + r] = fkey_inv((uint32_t)(v >> 32));
      }
      return;
    }
    __syncthreads();
  }
  const uint32_t T = block_radix_kth<PS_NT>(g, nlist, nprobe, hist, shv);
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < nlist; i += PS_NT) {
    const uint32_t kk = fkey(g[i]);
    if (kk <= T) {
      const unsigned at = atomicAdd(&s_cnt, 1u);
      if (at < (unsigned)cap) sel[at] = ((unsigned long long)kk << 32) | (uint32_t)i;
    }
  }
  __syncthreads();
  int n = (int)s_cnt;
  if (n > cap) {
    // overflow by ties: keys < T (fewer than nprobe), then ties in list-id order
    if (threadIdx.x == 0) { s_cnt = 0u; s_eq = 0; }
    __syncthreads();
    for (int i = threadIdx.x; i < nlist; i += PS_NT) {
      const uint32_t kk = fkey(g[i]);
      if (kk < T) sel[atomicAdd(&s_cnt, 1u)] = ((unsigned long long)kk << 32) | (uint32_t)i;
    }
    __syncthreads();
    const int n_lt = (int)s_cnt;
    const int need = nprobe - n_lt;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __shared__ int wcnt[PS_NT / 32];
    for (int b0 = 0; b0 < nlist; b0 += PS_NT) {
      const int i = b0 + threadIdx.x;
      const bool eq = i < nlist && fkey(g[i]) == T;
      const unsigned m = __ballot_sync(0xffffffffu, eq);
      if (lane == 0) wcnt[wid] = __popc(m);
      __syncthreads();
      int before = 0;
      for (int w = 0; w < wid; ++w) before += wcnt[w];
      const int rank = s_eq + before + __popc(m & ((1u << lane) - 1));
      if (eq && rank < need) sel[n_lt + rank] = ((unsigned long long)T << 32) | (uint32_t)i;
      __syncthreads();
      if (threadIdx.x == 0) {
        int t = 0;
        for (int w = 0; w < PS_NT / 32; ++w) t += wcnt[w];
        s_eq += t;
      }
      __syncthreads();
      if (s_eq >= need) break;
    }
    n = nprobe;
  }
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = n + threadIdx.x; i < n2; i += PS_NT) sel[i] = ~0ull;
  block_bitonic<PS_NT>(sel, n2);
  for (int r = threadIdx.x; r < nprobe; r += PS_NT) {
    const unsigned long long v = sel[r];
    plist[q * nprobe + r] = (int32_t)(v & 0xffffffffu);
    pg[q * nprobe + r] = fkey_inv((uint32_t)(v >> 32));
  }
}

// Merge of the fused probe candidates, then the refine step of the selected lists in the
// same warp.  Per query (one warp): the nprobe smallest of the n = tiles x nprobe
// (key, list) pairs, ascending; the n <= 32 * SL keys sit in registers (SL per lane) and
// each of nprobe rounds takes a warp-wide minimum and retires it (the keys are distinct:
// every list appears in one tile).  Then g_j = |q_d' - c_j'|^2 as a direct float32 sum
// (lane-strided, then the warp tree, as k_probe_refine computes it).
template <int SL>
__global__ void k_probe_merge_refine(const unsigned long long* __restrict__ part, int64_t nq,
                                     int tiles, int nprobe, const float* __restrict__ qd,
                                     const float* __restrict__ cent, int d,
                                     int32_t* __restrict__ plist, float* __restrict__ pg) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * 8 + wid;
  if (q >= nq) return;
  const int n = tiles * nprobe;
  unsigned long long v[SL];
#pragma unroll
  for (int s = 0; s < SL; ++s) {
    const int i = s * 32 + lane;
    v[s] = i < n ? part[q * n + i] : ~0ull;
  }
  for (int r = 0; r < nprobe; ++r) {
    unsigned long long m = v[0];
#pragma unroll
    for (int s = 1; s < SL; ++s) m = v[s] < m ? v[s] : m;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long y = __shfl_xor_sync(0xffffffffu, m, o);
      m = y < m ? y : m;
    }
#pragma unroll
    for (int s = 0; s < SL; ++s)
      if (v[s] == m) v[s] = ~0ull;
    const int j = (int)(m & 0xffffffffu);
    float g = 0.f;
    for (int i = lane; i < d; i += 32) {
      const float t = qd[q * d + i] - cent[(int64_t)j * d + i];
      g = fmaf(t, t, g);
    }
    g = warp_sum(g);
    if (lane == 0) {
      plist[q * nprobe + r] = j;
      pg[q * nprobe + r] = g;
    }
  }
}

// g_j = |q_d' - c_j'|^2 of every probed list, as a direct float32 sum (one warp per
// pair); the scan's estimates use this value whatever precision chose the lists.
__global__ void k_probe_refine(const float* __restrict__ qd, const float* __restrict__ cent,
                               const int32_t* __restrict__ plist, int64_t npairs, int nprobe, int d,
                               float* __restrict__ pg) {
  int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (w >= npairs) return;
  const int lane = threadIdx.x & 31;
  const int64_t q = w / nprobe;
  const int j = plist[w];
  float s = 0.f;
  for (int i = lane; i < d; i += 32) {
    float t = qd[q * d + i] - cent[(int64_t)j * d + i];
    s = fmaf(t, t, s);
  }
  s = warp_sum(s);
  if (lane == 0) pg[w] = s;
}

// ------------------------------------------------------------------ scan

struct ScanParams {
  const float* qd;      // nq x d
  const float* qstat;   // nq x 4
  const int32_t* plist; // nq x nprobe
  const float* pg;      // nq x nprobe
  const float* cent;    // nlist x d
  const int64_t* loff;
  const int64_t* ploff;
  const uint32_t* codes;
  const float* fadd;
  const float* fres;
  const float* ferr;
  int d, bits, words, vw, nprobe, k, qbits;
  int plane0;             // first code plane scanned: 0 = the full code, bits - 1 = the sign
                          // plane alone (stage 1a of 1 bit + refinement, 1-bit factors)
  float eps0, m;
  int64_t npairs;
  int64_t cap;
  const int64_t* items;   // (pair << 32 | chunk) work items, or NULL: one item per pair
  const int* nitems;      // device count of items
  int chunk;              // candidates per chunk when items != NULL
  int seed;               // 1: publish the running bound only, write no survivor (the
                          // seed pass over the start of each query's nearest list)
  unsigned int* work;
  unsigned int* qcnt;
  unsigned int* gtau;
  int32_t* spos;
  float* slb;
  float* sub;
  // diagnostics (single pair): per-candidate outputs
  float* dbg_ip;
  float* dbg_dis;
  float* dbg_lb;
  float* dbg_ub;
  int32_t* dbg_idot;
};

constexpr int SCAN_WARPS = 8;
constexpr int SCAN_CHUNK = 4096;  // candidates per scan work item for long lists
constexpr int SEED_CHUNK = 1024;  // candidates of each query's nearest list in the seed pass

// KM: 0 = warp-sorted top-k list (k <= 32); 1 = per-lane top-m (m = ceil(k/32) <= 4);
//     2 = no running threshold (k > 128).  QUANT: query quantized to qbits.
// DBG: diagnostics (one pair, outputs per candidate, no survivors).
template <int KM, bool QUANT, bool DBG>
__global__ void __launch_bounds__(SCAN_WARPS * 32) k_scan(ScanParams P) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int d = P.d;
  const int nch = d >> 5;  // 32-dim chunks
  // per warp: q' (d) then 4d floats of nibble tables (float32 mode) or the query's
  // qbits x d/32 plane words (quantized mode, at most d/4 words)
  float* qp = smem + wid * ((QUANT ? 2 : 5) * d);
  float* lut = qp + d;               // 4d: nibble tables (float32 mode)
  uint32_t* qw = reinterpret_cast<uint32_t*>(lut);  // qbits x nch words (quantized mode)
  const int topc = (1 << (P.bits - P.plane0)) - 1;  // of the planes scanned
  const int topq = (1 << P.qbits) - 1;

  const int lvw = P.vw == 4 ? 2 : P.vw == 2 ? 1 : 0;
  const int64_t n_items = P.items ? (int64_t)*P.nitems : P.npairs;
  while (true) {
    unsigned int it = 0;
    if (lane == 0) it = DBG ? (unsigned)(blockIdx.x * SCAN_WARPS + wid) : atomicAdd(P.work, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((int64_t)it >= n_items) break;
    int64_t w = it, c_lo = 0, c_hi = -1;  // pair index, candidate range of this item
    if (P.items) {
      const int64_t v = P.items[it];
      w = v >> 32;
      c_lo = (v & 0xffffffffll) * P.chunk;
      c_hi = c_lo + P.chunk;
    }
    const int64_t q = (int64_t)w / P.nprobe;
    const int j = P.plist[w];
    const float g = P.pg[w];
    const float sg = sqrtf(g);
    const float qr2 = P.qstat[q * 4 + 0];
    const float sigma = P.qstat[q * 4 + 1];
    const float a0 = g + qr2;
    const float em = P.m * sigma;
    const float e0 = P.eps0 * sg;

    // q' = (q_d' - c_j')/sqrt(g_j)
    for (int c = 0; c < nch; ++c) {
      int i = c * 32 + lane;
      float v = P.qd[q * d + i] - P.cent[(int64_t)j * d + i];
      qp[i] = g > 0.f ? v / sg : 0.f;
    }
    __syncwarp();
    float ql = 0.f, qdelta = 0.f;
    int qsum = 0;
    if (!QUANT) {
      // lut[(c*8 + s)*16 + nib] = sum_{e<4} (bit e of nib ? +q'_i : -q'_i), i = c*32 + s*4 + e
      for (int e = lane; e < 4 * d; e += 32) {
        int gi = e >> 4, nib = e & 15;
        const float* qq = qp + gi * 4;
        float v = ((nib & 1) ? qq[0] : -qq[0]) + ((nib & 2) ? qq[1] : -qq[1]);
        v += ((nib & 4) ? qq[2] : -qq[2]) + ((nib & 8) ? qq[3] : -qq[3]);
        lut[e] = v;
      }
    } else {
      float lo = FINF, hi = -FINF;
      for (int c = 0; c < nch; ++c) {
        float v = qp[c * 32 + lane];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
      }
      lo = warp_min(lo);
      hi = warp_max(hi);
      const float delta = (hi - lo) / (float)topq;
      int s = 0;
      for (int c = 0; c < nch; ++c) {
        int qb = 0;
        if (delta > 0.f) {
          float t = (qp[c * 32 + lane] - lo) / delta;
          qb = min((int)floorf(t + 0.5f), topq);
          qb = max(qb, 0);
        }
        s += qb;
        for (int b = 0; b < P.qbits; ++b) {
          unsigned word = __ballot_sync(0xffffffffu, (qb >> b) & 1);
          if (lane == 0) qw[b * nch + c] = word;
        }
      }
      qsum = warp_sum_i(s);
      ql = lo;
      qdelta = delta;
    }
    __syncwarp();

    const int64_t lb0 = P.loff[j];
    const int64_t lsize = P.loff[j + 1] - lb0;
    const int64_t size = c_hi < 0 ? lsize : min(lsize, c_hi);
    const int64_t pb0 = P.ploff[j];
    float lst = FINF;         // KM 0: lane i holds the i-th smallest upper bound seen
    float top4[4] = {FINF, FINF, FINF, FINF};  // KM 1: this lane's smallest upper bounds
    const int mper = (P.k + 31) >> 5;
    float tau = FINF;
    float gt = FINF;
    if (!DBG && KM != 2) gt = fkey_inv(__ldcg(P.gtau + q));

    for (int64_t b0 = c_lo; b0 < size; b0 += 32) {
      const int64_t idx = b0 + lane;
      const bool valid = idx < size;
      const int64_t pp = pb0 + idx;  // padded position (always allocated)
      // word w of this candidate: cbase + (w / vw) * 32 * vw + w % vw (vw = 1 << lvw)
      const uint32_t* cbase = P.codes + (pp >> 5) * (int64_t)P.words * 32 + (pp & 31) * P.vw;
      float ip;
      int idot = 0;
      if (!QUANT) {
        float acc = 0.f;
        for (int a = P.plane0; a < P.bits; ++a) {
          float pacc = 0.f;
          for (int c = 0; c < nch; ++c) {
            const int w = a * nch + c;
            const uint32_t word = __ldg(cbase + ((w >> lvw) << (5 + lvw)) + (w & (P.vw - 1)));
            const float* L = lut + c * 128;
#pragma unroll
            for (int s = 0; s < 8; ++s) pacc += L[s * 16 + ((word >> (4 * s)) & 15)];
          }
          acc = fmaf((float)(1 << (a - P.plane0)), pacc, acc);
        }
        ip = acc;
      } else {
        int dot = 0, su = 0;
        for (int a = P.plane0; a < P.bits; ++a) {
          int pd = 0, ps = 0;
          for (int c = 0; c < nch; ++c) {
            const int w = a * nch + c;
            const uint32_t word = __ldg(cbase + ((w >> lvw) << (5 + lvw)) + (w & (P.vw - 1)));
            ps += __popc(word);
            for (int bq = 0; bq < P.qbits; ++bq) pd += __popc(word & qw[bq * nch + c]) << bq;
          }
          dot += pd << (a - P.plane0);
          su += ps << (a - P.plane0);
        }
        idot = dot;
        ip = qdelta * (float)(2 * dot - topc * qsum) + ql * (float)(2 * su - d * topc);
      }
      const float fa = __ldg(P.fadd + pp), fr = __ldg(P.fres + pp), fe = __ldg(P.ferr + pp);
      const float dis = fa + a0 + fr * sg * ip;  // Eq. 4
      const float eps = e0 * fe + em;             // Eq. 5 + Chebyshev
      float lb = dis - eps, ub = dis + eps;
      if (DBG) {
        if (valid) {
          P.dbg_ip[idx] = ip;
          P.dbg_dis[idx] = dis;
          P.dbg_lb[idx] = lb;
          P.dbg_ub[idx] = ub;
          if (QUANT && P.dbg_idot) P.dbg_idot[idx] = idot;
        }
        continue;
      }
      if (!valid) { lb = FINF; ub = FINF; }
      // running upper bound of the k-th smallest upper bound: this warp's own bound,
      // tightened by what the query's other work items have published so far
      if (KM != 2 && b0 > c_lo) {
        float g2 = 0.f;
        if (lane == 0) g2 = fkey_inv(__ldcg(P.gtau + q));
        gt = fminf(gt, __shfl_sync(0xffffffffu, g2, 0));
      }
      if (KM == 0) {
        float kth = __shfl_sync(0xffffffffu, lst, P.k - 1);
        unsigned mask = __ballot_sync(0xffffffffu, ub < kth);
        while (mask) {
          int src = __ffs(mask) - 1;
          mask &= mask - 1;
          float v = __shfl_sync(0xffffffffu, ub, src);
          float cur = __shfl_sync(0xffffffffu, lst, P.k - 1);
          if (v < cur) {
            float prev = __shfl_up_sync(0xffffffffu, lst, 1);
            float nl = (lst <= v) ? lst : ((lane == 0 || prev <= v) ? v : prev);
            lst = lane < P.k ? nl : FINF;
          }
        }
        tau = fminf(gt, __shfl_sync(0xffffffffu, lst, P.k - 1));
      } else if (KM == 1) {
        // keep this lane's mper smallest upper bounds (sorted, fixed registers)
        float v = ub;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (t < mper && v < top4[t]) { float x = top4[t]; top4[t] = v; v = x; }
        }
        float mine = mper == 1 ? top4[0] : mper == 2 ? top4[1] : mper == 3 ? top4[2] : top4[3];
        // every lane holds >= mper values <= mine, 32 * mper >= k of them in all
        tau = fminf(gt, warp_max(mine));
      }
      // publish an improved bound (once per 32 candidates at most)
      if (KM != 2 && lane == 0 && tau < gt) {
        atomicMin(P.gtau + q, fkey(tau));
      }
      if (KM != 2) gt = fminf(gt, tau);
      const bool surv = valid && lb <= tau && !P.seed;
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
    if (DBG) break;
  }
}

// Quantized-query scan with the code shape fixed at compile time: NCH 32-dim chunks,
// BITS code planes, QB query planes.  The same arithmetic, in the same order, as
// k_scan<KM, true, false>, with the query planes in registers (warp-uniform ballot
// words), the candidate's code words fetched with VW-wide loads and every loop
// unrolled.  The insertion into the warp's top-k list (KM 0) skips upper bounds not
// below the query's published bound, which cannot lower tau.
// LB: code planes stored (LB > BITS: only the top BITS planes are read, so LB = bits,
// BITS = 1 scans the sign plane of a multi-bit code: stage 1a of 1 bit + refinement).
// Per 32-candidate block the loop keeps only what each block needs: the next block's
// loads are issued before this one is scored (short codes), the query's published bound
// is read one block ahead, survivors go to a per-warp staging buffer in shared memory
// that is appended to the query's survivor list with one atomic per SCAN_STAGE entries,
// and the next work item is claimed while the current one is scanned.
constexpr int SCAN_STAGE = 64;

// resident CTAs per SM the register budget is cut for, from the registers a lane needs:
// the query planes (qb x nch words), the code words (twice for the software pipeline of
// short codes) and about 30 for the rest
constexpr int scan_q_min_ctas(int nch, int words, int qb) {
  return (qb * nch + (words <= 16 ? 2 * words : words) + 30) <= 64 ? 4
         : (qb * nch + (words <= 16 ? 2 * words : words) + 30) <= 80 ? 3
         : (qb * nch + (words <= 16 ? 2 * words : words) + 30) <= 128 ? 2 : 1;
}

template <int KM, int NCH, int BITS, int QB, int LB = BITS>
__global__ void __launch_bounds__(SCAN_WARPS * 32, scan_q_min_ctas(NCH, BITS * NCH, QB))
    k_scan_q(ScanParams P) {
  constexpr int W = BITS * NCH;                                 // words read per candidate
  constexpr int WL = LB * NCH;                                  // words stored per candidate
  constexpr int VW = (WL % 4 == 0) ? 4 : (WL % 2 == 0) ? 2 : 1; // the layout's vector width
  constexpr int OFF = (LB - BITS) * NCH;                        // first word read
  constexpr int topc = (1 << BITS) - 1;
  constexpr int topq = (1 << QB) - 1;
  constexpr int d = NCH * 32;
  __shared__ int32_t stg_pos[SCAN_WARPS][SCAN_STAGE];
  __shared__ float stg_lb[SCAN_WARPS][SCAN_STAGE];
  __shared__ float stg_ub[SCAN_WARPS][SCAN_STAGE];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int32_t* s_pos = stg_pos[wid];
  float* s_lb = stg_lb[wid];
  float* s_ub = stg_ub[wid];
  const int64_t n_items = P.items ? (int64_t)*P.nitems : P.npairs;
  unsigned int it_next = 0;
  if (lane == 0) it_next = atomicAdd(P.work, 1u);
  while (true) {
    const unsigned int it = __shfl_sync(0xffffffffu, it_next, 0);
    if ((int64_t)it >= n_items) break;
    if (lane == 0) it_next = atomicAdd(P.work, 1u);   // claimed now, used next round
    int64_t w, c_lo = 0, c_hi = -1;
    if (P.items) {
      const int64_t v = P.items[it];
      w = v >> 32;
      c_lo = (v & 0xffffffffll) * P.chunk;
      c_hi = c_lo + P.chunk;
    } else {
      // probe-rank-major order: every query's nearest list first, then every query's
      // second list, ...; a query's later lists then start from the bound its nearest
      // list published instead of an empty top-k list
      const uint32_t nqr = (uint32_t)(P.npairs / P.nprobe);
      const uint32_t r = it / nqr;
      w = (int64_t)(it - r * nqr) * P.nprobe + r;
    }
    const int64_t q = (int64_t)((uint32_t)w / (uint32_t)P.nprobe);  // pairs < 2^31
    const int j = P.plist[w];
    const float g = P.pg[w];
    const float sg = sqrtf(g);
    const float qr2 = P.qstat[q * 4 + 0];
    const float sigma = P.qstat[q * 4 + 1];
    const float a0 = g + qr2;
    const float em = P.m * sigma;
    const float e0 = P.eps0 * sg;

    // q' = (q_d' - c_j')/sqrt(g_j), quantized to QB bits on the [min, max] grid
    float qv[NCH];
    float lo = FINF, hi = -FINF;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      const int i = c * 32 + lane;
      const float v = P.qd[q * d + i] - P.cent[(int64_t)j * d + i];
      qv[c] = g > 0.f ? v / sg : 0.f;
      lo = fminf(lo, qv[c]);
      hi = fmaxf(hi, qv[c]);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    const float delta = (hi - lo) / (float)topq;
    uint32_t qw[QB][NCH];
    int s = 0;
#pragma unroll
    for (int c = 0; c < NCH; ++c) {
      int qb = 0;
      if (delta > 0.f) {
        const float t = (qv[c] - lo) / delta;
        qb = min((int)floorf(t + 0.5f), topq);
        qb = max(qb, 0);
      }
      s += qb;
#pragma unroll
      for (int b = 0; b < QB; ++b) qw[b][c] = __ballot_sync(0xffffffffu, (qb >> b) & 1);
    }
    const int qsum = warp_sum_i(s);
    const float ql = lo, qdelta = delta;

    const int64_t lb0 = P.loff[j];
    const int64_t lsize = P.loff[j + 1] - lb0;
    const int64_t size = c_hi < 0 ? lsize : min(lsize, c_hi);
    const int64_t pb0 = P.ploff[j];
    float lst = FINF, kth = FINF;
    float top4[4] = {FINF, FINF, FINF, FINF};
    const int mper = (P.k + 31) >> 5;
    float tau = FINF;
    float gt = KM != 2 ? fkey_inv(__ldcg(P.gtau + q)) : FINF;
    uint32_t gnext = 0;           // lane 0: the published bound, read one block ahead
    if (KM != 2 && lane == 0) gnext = __ldcg(P.gtau + q);
    int fill = 0;                 // staged survivors of this warp
    // one append of the staged survivors to the query's list
    auto flush = [&]() {
      __syncwarp();
      unsigned base = 0;
      if (lane == 0) base = atomicAdd(P.qcnt + q, (unsigned)fill);
      base = __shfl_sync(0xffffffffu, base, 0);
      const int64_t at = q * P.cap + base;
      const int64_t room = P.cap - (int64_t)base;   // past the region: counted only
      for (int i = lane; i < fill && i < room; i += 32) {
        P.spos[at + i] = s_pos[i];
        P.slb[at + i] = s_lb[i];
        P.sub[at + i] = s_ub[i];
      }
      __syncwarp();
      fill = 0;
    };

    // the lane's codes and factors of the 32-candidate block starting at candidate b
    // (blocks start at multiples of 32: list starts are padded, chunks are multiples of 64)
    auto fetch = [&](int64_t b, uint32_t (&cw)[W], float& fa, float& fr, float& fe) {
      const int64_t pp = pb0 + b + lane;
      const uint32_t* cptr = P.codes + (pp >> 5) * (int64_t)(WL * 32) + lane * VW;
      if constexpr (OFF % VW != 0 || W % VW != 0) {
        // the planes read do not fill whole vector groups: one word at a time
#pragma unroll
        for (int t = 0; t < W; ++t) {
          const int wl = OFF + t;
          cw[t] = __ldg(cptr + (wl / VW) * 32 * VW + wl % VW);
        }
      } else {
#pragma unroll
        for (int gq = 0; gq < W / VW; ++gq) {
          const uint32_t* src = cptr + (OFF / VW + gq) * 32 * VW;
          if (VW == 4) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(src));
            cw[gq * 4] = v.x; cw[gq * 4 + 1] = v.y; cw[gq * 4 + 2] = v.z; cw[gq * 4 + 3] = v.w;
          } else if (VW == 2) {
            const uint2 v = __ldg(reinterpret_cast<const uint2*>(src));
            cw[gq * 2] = v.x; cw[gq * 2 + 1] = v.y;
          } else {
            cw[gq] = __ldg(src);
          }
        }
      }
      fa = __ldg(P.fadd + pp);
      fr = __ldg(P.fres + pp);
      fe = __ldg(P.ferr + pp);
    };
    // software pipeline (short codes): the next U blocks' loads are in flight while these
    // are scored; long codes (W > 16) are popcount-bound and keep the registers.  Short
    // codes (W <= 4) score two blocks per iteration: two independent dots to overlap, and
    // the bound refresh, threshold and survivor bookkeeping once per 64 candidates.
    constexpr bool PF = W <= 16;
    constexpr int U = W <= 4 ? 2 : 1;
    uint32_t nw[U][W];
    float nfa[U], nfr[U], nfe[U];
    if constexpr (PF) {
#pragma unroll
      for (int u = 0; u < U; ++u)
        if (c_lo + 32 * u < size) fetch(c_lo + 32 * u, nw[u], nfa[u], nfr[u], nfe[u]);
    }
    for (int64_t b0 = c_lo; b0 < size; b0 += 32 * U) {
      uint32_t cw[U][W];
      float fa[U], fr[U], fe[U];
      if constexpr (PF) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
#pragma unroll
          for (int t = 0; t < W; ++t) cw[u][t] = nw[u][t];
          fa[u] = nfa[u]; fr[u] = nfr[u]; fe[u] = nfe[u];
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (b0 + 32 * (U + u) < size) fetch(b0 + 32 * (U + u), nw[u], nfa[u], nfr[u], nfe[u]);
      } else {
#pragma unroll
        for (int u = 0; u < U; ++u)
          if (b0 + 32 * u < size) fetch(b0 + 32 * u, cw[u], fa[u], fr[u], fe[u]);
      }
      float lb[U], ub[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        // <u, qbar> = sum_a 2^a sum_bq 2^bq popc(plane_a & qplane_bq): per query plane
        // the popcounts of all chunks are summed first, the planes weighted after
        int dot = 0, su = 0;
#pragma unroll
        for (int a = 0; a < BITS; ++a) {
          int pl[QB];
          int ps = 0;
#pragma unroll
          for (int bq = 0; bq < QB; ++bq) pl[bq] = 0;
#pragma unroll
          for (int c = 0; c < NCH; ++c) {
            const uint32_t word = cw[u][a * NCH + c];
            ps += __popc(word);
#pragma unroll
            for (int bq = 0; bq < QB; ++bq) pl[bq] += __popc(word & qw[bq][c]);
          }
          int pd = pl[QB - 1];
#pragma unroll
          for (int bq = QB - 2; bq >= 0; --bq) pd = 2 * pd + pl[bq];
          dot += pd << a;
          su += ps << a;
        }
        const float ip =
            qdelta * (float)(2 * dot - topc * qsum) + ql * (float)(2 * su - d * topc);
        const float dis = fa[u] + a0 + fr[u] * sg * ip;  // Eq. 4
        const float eps = e0 * fe[u] + em;                // Eq. 5 + Chebyshev
        const bool valid = b0 + 32 * u + lane < size;
        lb[u] = valid ? dis - eps : FINF;
        ub[u] = valid ? dis + eps : FINF;
      }
      if (KM != 2 && b0 > c_lo) {
        gt = fminf(gt, fkey_inv(__shfl_sync(0xffffffffu, gnext, 0)));
        if (lane == 0) gnext = __ldcg(P.gtau + q);
      }
      if (KM == 0) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = ub[u] < kth && ub[u] < gt;
          unsigned mask = __ballot_sync(0xffffffffu, in);
          if (mask) {
            if (__popc(mask) > 6) {
              // many: sort this block's bounds across the lanes and merge the two ascending
              // lists (the k smallest of the union are the same values in any order)
              float v = in ? ub[u] : FINF;
#pragma unroll
              for (int size2 = 2; size2 <= 32; size2 <<= 1) {
#pragma unroll
                for (int stride = size2 >> 1; stride > 0; stride >>= 1) {
                  const float o = __shfl_xor_sync(0xffffffffu, v, stride);
                  const bool up = (lane & size2) == 0, lower = (lane & stride) == 0;
                  v = (lower == up) ? fminf(v, o) : fmaxf(v, o);
                }
              }
              // min(lst[i], v[31 - i]) are the 32 smallest of both, a bitonic sequence
              float mg = fminf(lst, __shfl_sync(0xffffffffu, v, 31 - lane));
#pragma unroll
              for (int stride = 16; stride > 0; stride >>= 1) {
                const float o = __shfl_xor_sync(0xffffffffu, mg, stride);
                mg = (lane & stride) == 0 ? fminf(mg, o) : fmaxf(mg, o);
              }
              lst = lane < P.k ? mg : FINF;
              mask = 0;
            }
            while (mask) {
              int src = __ffs(mask) - 1;
              mask &= mask - 1;
              float v = __shfl_sync(0xffffffffu, ub[u], src);
              float cur = __shfl_sync(0xffffffffu, lst, P.k - 1);
              if (v < cur) {
                float prev = __shfl_up_sync(0xffffffffu, lst, 1);
                float nl = (lst <= v) ? lst : ((lane == 0 || prev <= v) ? v : prev);
                lst = lane < P.k ? nl : FINF;
              }
            }
            kth = __shfl_sync(0xffffffffu, lst, P.k - 1);
          }
        }
        tau = fminf(gt, kth);
      } else if (KM == 1) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          float v = ub[u];
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            if (t < mper && v < top4[t]) { float x = top4[t]; top4[t] = v; v = x; }
          }
        }
        float mine = mper == 1 ? top4[0] : mper == 2 ? top4[1] : mper == 3 ? top4[2] : top4[3];
        tau = fminf(gt, warp_max(mine));
      }
      if (KM != 2 && lane == 0 && tau < gt) atomicMin(P.gtau + q, fkey(tau));
      if (KM != 2) gt = fminf(gt, tau);
      unsigned sm[U], any = 0;
#pragma unroll
      for (int u = 0; u < U; ++u) {
        sm[u] = __ballot_sync(0xffffffffu, lb[u] <= tau);   // invalid lanes hold +inf
        any |= sm[u];
      }
      if (any && !P.seed) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int cnt = __popc(sm[u]);
          if (fill + cnt > SCAN_STAGE) flush();
          if ((sm[u] >> lane) & 1u) {
            const int at = fill + __popc(sm[u] & ((1u << lane) - 1));
            s_pos[at] = (int32_t)(lb0 + b0 + 32 * u + lane);
            s_lb[at] = lb[u];
            s_ub[at] = ub[u];
          }
          fill += cnt;
        }
      }
    }
    if (fill) flush();
    __syncwarp();
  }
}

// seed items: the first chunk of every query's nearest list (pair q * nprobe, chunk 0)
__global__ void k_seed_items(int64_t nq, int nprobe, int64_t* __restrict__ items,
                             int* __restrict__ nitems) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  items[q] = (q * nprobe) << 32;
  if (q == 0) *nitems = (int)nq;
}

// work items: the pairs w = i * stride (i < n) contribute max(1, ceil(size/chunk))
// items each, (w << 32 | chunk index)
// the pair of item slot i: w = i * stride, or, with rm_nq > 0 (rm_nq queries, n / rm_nq
// probes each), probe-rank-major: every query's nearest list first, then the second, ...
__device__ __forceinline__ int64_t chunk_pair(int64_t i, int64_t n, int stride, int64_t rm_nq) {
  return rm_nq > 0 ? (i % rm_nq) * (n / rm_nq) + i / rm_nq : i * stride;
}

__global__ void k_chunk_count(const int32_t* __restrict__ plist, const int64_t* __restrict__ loff,
                              int64_t n, int stride, int chunk, int* __restrict__ cnt,
                              int64_t rm_nq) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = plist[chunk_pair(i, n, stride, rm_nq)];
  const int64_t sz = loff[j + 1] - loff[j];
  const int64_t c = (sz + chunk - 1) / chunk;
  cnt[i] = c > 0 ? (int)c : 1;
}
__global__ void k_chunk_scatter(const int* __restrict__ cnt, const int* __restrict__ off,
                                int64_t n, int stride, int64_t* __restrict__ items,
                                int* __restrict__ nitems, int64_t rm_nq) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int o = off[i], c = cnt[i];
  const int64_t w = chunk_pair(i, n, stride, rm_nq);
  for (int t = 0; t < c; ++t) items[o + t] = (w << 32) | (int64_t)t;
  if (i == n - 1) *nitems = o + c;
}


// ------------------------------------------------------- batched (list-major) scan
//
// The pairs (query, probed list) are bucketed by list; k_pair_prep quantizes each
// pair's query once (Algorithm 2: normalise, rotate, quantize); a work item is
// (list j, block of 32 candidates, group of up to `group` pairs probing j).  One
// warp loads its 32 candidates' code words and factors once (registers) and scores
// them against every query of the group, so a list's codes are read once per
// group instead of once per query.

constexpr int BATCH_G = 16;     // largest number of queries per work item
constexpr int BATCH_MAXW = 16;  // code words per vector kept in registers (bits*d/32)


// pairs with w % nprobe < first are left out (scanned by the seed pass)
__global__ void k_bucket_count(const int32_t* __restrict__ plist, int64_t npairs, int nprobe,
                               int first, int* __restrict__ cnt) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w < npairs && (int)(w % nprobe) >= first) atomicAdd(&cnt[plist[w]], 1);
}
__global__ void k_bucket_fill(const int32_t* __restrict__ plist, int64_t npairs, int nprobe,
                              int first, const int* __restrict__ off, int* __restrict__ fill,
                              int* __restrict__ queue) {
  int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= npairs || (int)(w % nprobe) < first) return;
  const int j = plist[w];
  queue[off[j] + atomicAdd(&fill[j], 1)] = (int)w;
}
// items of list j: (#32-blocks) x (#groups of BATCH_G pairs)
__global__ void k_batch_count(const int* __restrict__ cnt, const int64_t* __restrict__ loff,
                              int nlist, int blk, int group, int* __restrict__ icnt) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlist) return;
  const int64_t sz = loff[j + 1] - loff[j];
  const int c = cnt[j];
  icnt[j] = (c > 0 && sz > 0) ? (int)(((sz + blk - 1) / blk) * ((c + group - 1) / group)) : 0;
}
__global__ void k_batch_scatter(const int* __restrict__ cnt, const int* __restrict__ icnt,
                                const int* __restrict__ ioff, const int64_t* __restrict__ loff,
                                int nlist, int group, int4* __restrict__ items, int* __restrict__ nitems) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nlist) return;
  const int n = icnt[j];
  const int ng = (cnt[j] + group - 1) / group;
  for (int i = 0; i < n; ++i) items[ioff[j] + i] = make_int4(j, i / ng, i % ng, 0);
  if (j == nlist - 1) *nitems = ioff[j] + n;
}

// per-pair query preparation (one warp per pair): q' and its B_q-bit planes
__global__ void k_pair_prep(const float* __restrict__ qd, const float* __restrict__ qstat,
                            const int32_t* __restrict__ plist, const float* __restrict__ pg,
                            const float* __restrict__ cent, int64_t npairs, int nprobe, int d,
                            int qbits, float eps0, float m, PairQ* __restrict__ pq,
                            uint32_t* __restrict__ qplanes, uint8_t* __restrict__ qcode) {
  const int64_t w = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (w >= npairs) return;
  const int lane = threadIdx.x & 31;
  const int64_t q = w / nprobe;
  const int j = plist[w];
  const float g = pg[w];
  const float sg = sqrtf(g);
  const int nch = d >> 5;
  const int topq = (1 << qbits) - 1;
  // q'_i = (q_d'_i - c'_i) / sqrt(g); computed twice (range, then codes) so that no
  // per-lane array is indexed at run time
  const float* qrow = qd + q * d;
  const float* crow = cent + (int64_t)j * d;
  float lo = FINF, hi = -FINF;
#pragma unroll 4
  for (int c = 0; c < nch; ++c) {
    const int i = c * 32 + lane;
    const float v = g > 0.f ? (qrow[i] - crow[i]) / sg : 0.f;
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
  }
  lo = warp_min(lo);
  hi = warp_max(hi);
  const float delta = (hi - lo) / (float)topq;
  int ssum = 0;
  uint32_t* out = qplanes + w * (int64_t)(qbits * nch);
  for (int c = 0; c < nch; ++c) {
    const int i = c * 32 + lane;
    const float v = g > 0.f ? (qrow[i] - crow[i]) / sg : 0.f;
    int qb = 0;
    if (delta > 0.f) {
      qb = min((int)floorf((v - lo) / delta + 0.5f), topq);
      qb = max(qb, 0);
    }
    ssum += qb;
    if (qcode) qcode[w * d + i] = (uint8_t)__nv_cvt_float_to_fp8((float)qb, __NV_SATFINITE, __NV_E4M3);  // exact: qb <= 15
    for (int b = 0; b < qbits; ++b) {
      const unsigned word = __ballot_sync(0xffffffffu, (qb >> b) & 1);
      if (lane == 0) out[b * nch + c] = word;
    }
  }
  ssum = warp_sum_i(ssum);
  if (lane == 0) {
    PairQ r;
    r.sg = sg;
    r.a0 = g + qstat[q * 4 + 0];
    r.e0 = eps0 * sg;
    r.em = m * qstat[q * 4 + 1];
    r.ql = lo;
    r.qdelta = delta;
    r.qsum = ssum;
    r.q = (int)q;
    pq[w] = r;
  }
}

struct BatchParams {
  const int4* items;
  const int* nitems;
  const int* lqueue;     // pairs bucketed by list
  const int* loffq;      // bucket offsets
  const int* lcount;
  const PairQ* pq;
  const uint32_t* qplanes;
  const int64_t* loff;
  const int64_t* ploff;
  const uint32_t* codes;
  const float* fadd;
  const float* fres;
  const float* ferr;
  int d, bits, words, vw, nprobe, k, qbits;
  int group;             // queries per work item (<= BATCH_G)
  int64_t cap;
  unsigned int* work;
  unsigned int* qcnt;
  unsigned int* gtau;
  int32_t* spos;
  float* slb;
  float* sub;
};

template <int W, int NCH>
__global__ void __launch_bounds__(256) k_scan_batched(BatchParams P) {
  constexpr int BITS = W / NCH;
  const int lane = threadIdx.x & 31;
  const int topc = (1 << BITS) - 1;
  const int QW = P.qbits * NCH;
  const int n_items = *P.nitems;
  while (true) {
    unsigned it = 0;
    if (lane == 0) it = atomicAdd(P.work, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((int)it >= n_items) break;
    const int4 item = P.items[it];
    const int j = item.x, blk = item.y, grp = item.z;
    const int64_t lb0 = P.loff[j];
    const int64_t size = P.loff[j + 1] - lb0;
    const int64_t idx = (int64_t)blk * 32 + lane;
    const bool valid = idx < size;
    const int64_t pp = P.ploff[j] + idx;
    // this lane's candidate: all W code words in registers, plane popcounts, factors
    const uint32_t* cbase = P.codes + (pp >> 5) * (int64_t)W * 32 + (pp & 31) * P.vw;
    const int lvw = P.vw == 4 ? 2 : P.vw == 2 ? 1 : 0;
    uint32_t cw[W];
#pragma unroll
    for (int w = 0; w < W; ++w) cw[w] = __ldg(cbase + ((w >> lvw) << (5 + lvw)) + (w & (P.vw - 1)));
    int su = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) su += __popc(cw[w]) << (w / NCH);
    const float fa = __ldg(P.fadd + pp), fr = __ldg(P.fres + pp), fe = __ldg(P.ferr + pp);
    const int g0 = P.loffq[j] + grp * P.group;
    const int ng = min(P.loffq[j] + P.lcount[j], g0 + P.group) - g0;
    const int my_pair = lane < ng ? P.lqueue[g0 + lane] : 0;  // the group's pairs, one per lane
    for (int t = 0; t < ng; ++t) {
      const int w_pair = __shfl_sync(0xffffffffu, my_pair, t);
      const PairQ pr = P.pq[w_pair];
      const int64_t q = pr.q;
      const uint32_t* qp = P.qplanes + (int64_t)w_pair * QW;
      int dot = 0;
      for (int b = 0; b < P.qbits; ++b) {
        int pd = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          const uint32_t qwd = __ldg(qp + b * NCH + c);
#pragma unroll
          for (int a = 0; a < BITS; ++a) pd += __popc(cw[a * NCH + c] & qwd) << a;
        }
        dot += pd << b;
      }
      const float ip = pr.qdelta * (float)(2 * dot - topc * pr.qsum) +
                       pr.ql * (float)(2 * su - P.d * topc);
      const float dis = fa + pr.a0 + fr * pr.sg * ip;  // Eq. 4
      const float eps = pr.e0 * fe + pr.em;            // Eq. 5 + Chebyshev
      const float lb = valid ? dis - eps : FINF;
      const float ub = valid ? dis + eps : FINF;
      float tau = fkey_inv(__ldcg(P.gtau + q));
      if (P.k <= 32) {
        // this warp's k-th smallest upper bound bounds tau_A from above
        const unsigned below = __ballot_sync(0xffffffffu, ub < tau);
        if (__popc(below) >= P.k) {
          float v = ub < tau ? ub : FINF;
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
  }
}

// ------------------------------------------------------------------ finalize

constexpr int FN_NT = 256;
constexpr int FN_SORT = 2048;  // capacity of the final (dist, id) sort

struct FinParams {
  const float* qd;
  const float* qr;
  const float* qstat;
  const int32_t* plist;
  const int64_t* loff;
  const float* xd;
  const float* xr;
  const float* xn2;
  const int64_t* ids;
  int d, r, nprobe, k, mode;
  float m;
  int64_t cap;
  const unsigned int* qcnt;
  int32_t* spos;
  float* slb;
  float* sub;
  int32_t* s2pos;
  float* s2a;
  float* s2b;
  int64_t* out_ids;
  float* out_d;
  int64_t* stats;
  // phased finalize: per-query threshold and survivor counts
  const unsigned int* gtau;  // the scan's running bound of tau_A per query (orderable key)
  float* qtau;
  int* qm1;
  int* qm2;
  int64_t nq;
};

// <row, sq> over n floats with float4 loads (row and sq 16-byte aligned, n % 4 == 0)
// or scalar loads; per-lane partial sums (the caller reduces across the warp).
template <bool DOT>
__device__ __forceinline__ void row_accum2(const float* __restrict__ r0, const float* __restrict__ r1,
                                           const float* sq, int n, bool vec, int lane, float& s0,
                                           float& s1) {
  if (vec) {
    const float4* a = reinterpret_cast<const float4*>(r0);
    const float4* b = reinterpret_cast<const float4*>(r1);
    const float4* qv = reinterpret_cast<const float4*>(sq);
    const int n4 = n >> 2;
#pragma unroll 4
    for (int c = lane; c < n4; c += 32) {
      const float4 x = __ldg(a + c), y = __ldg(b + c), qq = qv[c];
      if (DOT) {
        s0 = fmaf(x.x, qq.x, s0); s0 = fmaf(x.y, qq.y, s0); s0 = fmaf(x.z, qq.z, s0); s0 = fmaf(x.w, qq.w, s0);
        s1 = fmaf(y.x, qq.x, s1); s1 = fmaf(y.y, qq.y, s1); s1 = fmaf(y.z, qq.z, s1); s1 = fmaf(y.w, qq.w, s1);
      } else {
        float t;
        t = x.x - qq.x; s0 = fmaf(t, t, s0); t = x.y - qq.y; s0 = fmaf(t, t, s0);
        t = x.z - qq.z; s0 = fmaf(t, t, s0); t = x.w - qq.w; s0 = fmaf(t, t, s0);
        t = y.x - qq.x; s1 = fmaf(t, t, s1); t = y.y - qq.y; s1 = fmaf(t, t, s1);
        t = y.z - qq.z; s1 = fmaf(t, t, s1); t = y.w - qq.w; s1 = fmaf(t, t, s1);
      }
    }
  } else {
#pragma unroll 4
    for (int c = lane; c < n; c += 32) {
      const float x = __ldg(r0 + c), y = __ldg(r1 + c), qq = sq[c];
      if (DOT) { s0 = fmaf(x, qq, s0); s1 = fmaf(y, qq, s1); }
      else { float t = x - qq; s0 = fmaf(t, t, s0); t = y - qq; s1 = fmaf(t, t, s1); }
    }
  }
}

// Per-lane partial <x_u, q> and |x_u - q|^2 of up to R rows x_u = X[p[u]] (rows
// u >= nrow are skipped): all R loads of a column step are issued before any
// arithmetic, so R loads per lane are in flight.  The caller reduces across the warp.
template <int R>
__device__ __forceinline__ void rows_dot_dist2(const float* __restrict__ X, const int (&p)[R],
                                               int nrow, const float* sq, int n, bool vec, int lane,
                                               float (&dot)[R], float (&e)[R]) {
  if (vec) {
    const float4* qv = reinterpret_cast<const float4*>(sq);
    const int n4 = n >> 2;
    for (int c = lane; c < n4; c += 32) {
      float4 x[R];
#pragma unroll
      for (int u = 0; u < R; ++u)
        x[u] = u < nrow ? __ldg(reinterpret_cast<const float4*>(X + (int64_t)p[u] * n) + c)
                        : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 qq = qv[c];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        float t;
        dot[u] = fmaf(x[u].x, qq.x, dot[u]); dot[u] = fmaf(x[u].y, qq.y, dot[u]);
        dot[u] = fmaf(x[u].z, qq.z, dot[u]); dot[u] = fmaf(x[u].w, qq.w, dot[u]);
        t = x[u].x - qq.x; e[u] = fmaf(t, t, e[u]); t = x[u].y - qq.y; e[u] = fmaf(t, t, e[u]);
        t = x[u].z - qq.z; e[u] = fmaf(t, t, e[u]); t = x[u].w - qq.w; e[u] = fmaf(t, t, e[u]);
      }
    }
  } else {
    for (int c = lane; c < n; c += 32) {
      float x[R];
#pragma unroll
      for (int u = 0; u < R; ++u) x[u] = u < nrow ? __ldg(X + (int64_t)p[u] * n + c) : 0.f;
      const float qq = sq[c];
#pragma unroll
      for (int u = 0; u < R; ++u) {
        dot[u] = fmaf(x[u], qq, dot[u]);
        const float t = x[u] - qq;
        e[u] = fmaf(t, t, e[u]);
      }
    }
  }
}

constexpr int S2_ROWS = 4;  // rows of x_d' in flight per warp in stage 2

__global__ void __launch_bounds__(FN_NT) k_finalize(FinParams P) {
  extern __shared__ __align__(16) float fsm[];
  float* sq = fsm;  // query coordinates [q_d' | q_r], 16-byte aligned blocks
  const int dpad = (P.d + 3) & ~3;
  unsigned long long* srt =
      reinterpret_cast<unsigned long long*>(fsm + ((dpad + P.r + 3) & ~3));
  __shared__ int hist[256], shv[2];
  __shared__ unsigned int s_cnt;
  __shared__ unsigned long long s_ncand;
  const int64_t q = blockIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = FN_NT / 32;
  for (int i = threadIdx.x; i < P.d; i += FN_NT) sq[i] = P.qd[q * P.d + i];
  for (int i = threadIdx.x; i < P.r; i += FN_NT) sq[dpad + i] = P.qr[q * P.r + i];
  const bool vd = (P.d & 3) == 0;
  const bool vr = (P.r & 3) == 0;
  const float sigma = P.qstat[q * 4 + 1];
  const float qp2 = P.qstat[q * 4 + 2];
  const int64_t base = q * P.cap;
  const int M = (int)min((int64_t)P.qcnt[q], P.cap);
  if (threadIdx.x == 0) s_ncand = 0ull;
  __syncthreads();
  {
    int64_t nc = 0;
    for (int r = threadIdx.x; r < P.nprobe; r += FN_NT) {
      int j = P.plist[q * P.nprobe + r];
      nc += P.loff[j + 1] - P.loff[j];
    }
    if (nc) atomicAdd(&s_ncand, (unsigned long long)nc);
  }

  // tau_A: k-th smallest stage-1 upper bound; S1 = {LB1 <= tau_A}
  const float tauA =
      (M >= P.k) ? fkey_inv(block_radix_kth<FN_NT>(P.sub + base, M, P.k, hist, shv)) : FINF;
  if (threadIdx.x == 0) s_cnt = 0u;
  __syncthreads();
  for (int i = threadIdx.x; i < M; i += FN_NT) {
    if (P.slb[base + i] <= tauA) {
      unsigned at = atomicAdd(&s_cnt, 1u);
      P.s2pos[base + at] = P.spos[base + i];
    }
  }
  __syncthreads();
  const int M1 = (int)s_cnt;
  int M2;
  if (P.mode == MRQ_MODE_MRQ_PLUS) {
    // stage 2 (Eq. 7): dis_o' = |x_p|^2 + |q_p|^2 - 2 <x_d', q_d'>, bounds -+ m sigma
    const float em = P.m * sigma;
    for (int i = 2 * wid; i < M1; i += 2 * NW) {
      const bool two = i + 1 < M1;
      const int64_t p0 = P.s2pos[base + i], p1 = two ? P.s2pos[base + i + 1] : p0;
      float s0 = 0.f, s1 = 0.f;
      row_accum2<true>(P.xd + p0 * P.d, P.xd + p1 * P.d, sq, P.d, vd, lane, s0, s1);
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      if (lane == 0) {
        float diso = P.xn2[p0] + qp2 - 2.f * s0;
        P.s2a[base + i] = diso + em;
        P.s2b[base + i] = diso - em;
        if (two) {
          diso = P.xn2[p1] + qp2 - 2.f * s1;
          P.s2a[base + i + 1] = diso + em;
          P.s2b[base + i + 1] = diso - em;
        }
      }
    }
    __syncthreads();
    float tauB = tauA;
    if (M1 >= P.k)
      tauB = fminf(tauA, fkey_inv(block_radix_kth<FN_NT>(P.s2a + base, M1, P.k, hist, shv)));
    if (threadIdx.x == 0) s_cnt = 0u;
    __syncthreads();
    for (int i = threadIdx.x; i < M1; i += FN_NT) {
      if (P.s2b[base + i] <= tauB) {
        unsigned at = atomicAdd(&s_cnt, 1u);
        P.spos[base + at] = P.s2pos[base + i];
      }
    }
    __syncthreads();
    M2 = (int)s_cnt;
  } else {
    for (int i = threadIdx.x; i < M1; i += FN_NT) P.spos[base + i] = P.s2pos[base + i];
    M2 = M1;
  }
  __syncthreads();
  // exact distances |x_d' - q_d'|^2 + |x_r - q_r|^2 (direct sums, two candidates per warp)
  for (int i = 2 * wid; i < M2; i += 2 * NW) {
    const bool two = i + 1 < M2;
    const int64_t p0 = P.spos[base + i], p1 = two ? P.spos[base + i + 1] : p0;
    float s0 = 0.f, s1 = 0.f;
    row_accum2<false>(P.xd + p0 * P.d, P.xd + p1 * P.d, sq, P.d, vd, lane, s0, s1);
    row_accum2<false>(P.xr + p0 * P.r, P.xr + p1 * P.r, sq + dpad, P.r, vr, lane, s0, s1);
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (lane == 0) {
      P.slb[base + i] = s0;
      if (two) P.slb[base + i + 1] = s1;
    }
  }
  __syncthreads();
  // top-k by (distance, id)
  const int kk = min(P.k, M2);
  uint32_t T = 0xffffffffu;
  if (M2 > P.k) T = block_radix_kth<FN_NT>(P.slb + base, M2, P.k, hist, shv);
  if (threadIdx.x == 0) s_cnt = 0u;
  for (int i = threadIdx.x; i < FN_SORT; i += FN_NT) srt[i] = ~0ull;
  __syncthreads();
  for (int i = threadIdx.x; i < M2; i += FN_NT) {
    uint32_t key = fkey(P.slb[base + i]);
    if (key <= T) {
      unsigned at = atomicAdd(&s_cnt, 1u);
      if (at < FN_SORT) srt[at] = ((unsigned long long)key << 32) | (uint32_t)P.ids[P.spos[base + i]];
    }
  }
  __syncthreads();
  int ns = min((int)s_cnt, FN_SORT);
  int n2 = 1;
  while (n2 < ns) n2 <<= 1;
  block_bitonic<FN_NT>(srt, n2);
  for (int i = threadIdx.x; i < P.k; i += FN_NT) {
    if (i < kk && i < ns) {
      P.out_ids[q * P.k + i] = (int64_t)(uint32_t)(srt[i] & 0xffffffffu);
      P.out_d[q * P.k + i] = fkey_inv((uint32_t)(srt[i] >> 32));
    } else {
      P.out_ids[q * P.k + i] = -1;
      P.out_d[q * P.k + i] = FINF;
    }
  }
  if (threadIdx.x == 0 && P.stats) {
    P.stats[q * 3 + 0] = (int64_t)s_ncand;
    P.stats[q * 3 + 1] = M1;
    P.stats[q * 3 + 2] = M2;
  }
}

// ---------------------------------------------------- warp-per-query finalize

// Warp-local radix select: smallest key T with #{i : fkey(vals[i]) <= T} >= k.
// hist: 256 ints of this warp's shared memory.  Requires M >= k.
// chunks of 32 values a warp loop keeps in flight (one load round trip each)
constexpr int WU = 4;

__device__ uint32_t warp_radix_kth(const float* vals, int M, int k, int* hist) {
  const int lane = threadIdx.x & 31;
  uint32_t prefix = 0u, mask = 0u;
  int kk = k;
  for (int shift = 24; shift >= 0; shift -= 8) {
#pragma unroll
    for (int i = 0; i < 8; ++i) hist[lane * 8 + i] = 0;
    __syncwarp();
    for (int b = 0; b < M; b += 32 * WU) {  // WU independent loads in flight per lane
      uint32_t key[WU];
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        const int i = b + 32 * u + lane;
        key[u] = i < M ? fkey(vals[i]) : 0u;
      }
#pragma unroll
      for (int u = 0; u < WU; ++u) {
        const bool in = b + 32 * u + lane < M && (key[u] & mask) == prefix;
        const unsigned act = __ballot_sync(0xffffffffu, in);
        if (in) {
          const uint32_t bin = (key[u] >> shift) & 255u;
          const unsigned peers = __match_any_sync(act, bin);
          if (lane == __ffs(peers) - 1) atomicAdd(&hist[bin], __popc(peers));
        }
      }
    }
    __syncwarp();
    int c[8], tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) { c[j] = hist[lane * 8 + j]; tot += c[j]; }
    int incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    int acc = incl - tot;
    const unsigned who = __ballot_sync(0xffffffffu, acc < kk && kk <= incl);
    int bin = 0, before = 0;
    if (lane == __ffs(who) - 1) {
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (acc + c[j] >= kk) { bin = lane * 8 + j; before = acc; break; }
        acc += c[j];
      }
    }
    const int src = __ffs(who) - 1;
    bin = __shfl_sync(0xffffffffu, bin, src);
    before = __shfl_sync(0xffffffffu, before, src);
    prefix |= (uint32_t)bin << shift;
    mask |= 255u << shift;
    kk -= before;
    __syncwarp();
  }
  return prefix;
}

// k-th smallest key (k <= 32) of vals[0..M), M >= k.  The k smallest seen so far are
// kept sorted across the lanes (lane i holds the i-th smallest); values arrive 32 at
// a time and only those below the current k-th (and not above `hint`, an upper bound
// of the answer, or +inf) are inserted, one at a time.
// The k (<= 32) smallest keys of vals[0..M) that are <= hk, sorted across the lanes (lane
// i holds the i-th, 0xffffffff past the end): the streaming insertions of warp_kth_small.
__device__ uint32_t warp_topk_list(const float* vals, int M, int k, uint32_t hk) {
  const int lane = threadIdx.x & 31;
  uint32_t lst = 0xffffffffu, kth = 0xffffffffu;
  for (int b = 0; b < M; b += 32 * WU) {
    uint32_t x[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      x[u] = i < M ? fkey(vals[i]) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      unsigned cand = __ballot_sync(0xffffffffu, x[u] < kth && x[u] <= hk);
      while (cand) {
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const uint32_t y = __shfl_sync(0xffffffffu, x[u], src);
        if (y < kth) {
          const int pos = __popc(__ballot_sync(0xffffffffu, lst < y));
          const uint32_t up = __shfl_up_sync(0xffffffffu, lst, 1);
          lst = lane > pos ? up : (lane == pos ? y : lst);
          lst = lane < k ? lst : 0xffffffffu;
          kth = __shfl_sync(0xffffffffu, lst, k - 1);
        }
      }
    }
  }
  return lst;
}

__device__ uint32_t warp_kth_small(const float* vals, int M, int k, float hint) {
  const int lane = threadIdx.x & 31;
  const uint32_t hk = fkey(hint);
  uint32_t lst = 0xffffffffu;
  uint32_t kth = 0xffffffffu;
  for (int b = 0; b < M; b += 32 * WU) {  // WU chunks of loads in flight
    uint32_t x[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      x[u] = i < M ? fkey(vals[i]) : 0xffffffffu;
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      unsigned cand = __ballot_sync(0xffffffffu, x[u] < kth && x[u] <= hk);
      while (cand) {
        const int src = __ffs(cand) - 1;
        cand &= cand - 1;
        const uint32_t y = __shfl_sync(0xffffffffu, x[u], src);
        if (y < kth) {
          const int pos = __popc(__ballot_sync(0xffffffffu, lst < y));
          const uint32_t up = __shfl_up_sync(0xffffffffu, lst, 1);
          lst = lane > pos ? up : (lane == pos ? y : lst);
          kth = __shfl_sync(0xffffffffu, lst, k - 1);
        }
      }
    }
  }
  return kth;
}

// count of vals[0..M) that are <= h, gathering up to cap of them into buf
__device__ __forceinline__ int warp_filter_le(const float* vals, int M, float h, float* buf, int cap) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1;
  int c = 0;
  for (int b = 0; b < M; b += 32 * WU) {  // WU independent loads in flight per lane
    float v[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      v[u] = i < M ? vals[i] : FINF;
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const bool keep = v[u] <= h && b + 32 * u + lane < M;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      const int at = c + __popc(m & below);
      if (keep && at < cap) buf[at] = v[u];
      c += __popc(m);
    }
  }
  __syncwarp();
  return c;
}

// Exact k-th smallest key of vals[0..M) (M >= k).  `hint` is an upper bound of it
// (or +inf).  The values <= a pivot are gathered into the warp's buffer and
// selected there whenever their count lies in [k, cap]; the pivot is the hint or,
// failing that, a rank of a strided sample of 256 values chosen so that about
// cap/2 values are expected below it (rank adjusted and retried); a pivot is used
// only after counting confirms that at least k values lie below it, so the
// answer is exact whatever the sample.  Last resort: a radix select over vals.
__device__ uint32_t warp_kth_filtered(const float* vals, int M, int k, float hint, float* buf,
                                      int cap, int* hist) {
  const int lane = threadIdx.x & 31;
  if (M <= cap) {
    for (int i = lane; i < M; i += 32) buf[i] = vals[i];
    __syncwarp();
    return warp_radix_kth(buf, M, k, hist);
  }
  if (hint < FINF) {
    const int c = warp_filter_le(vals, M, hint, buf, cap);
    if (c >= k && c <= cap) return warp_radix_kth(buf, c, k, hist);
  }
  constexpr int S = 256;
  const int64_t r0 = ((int64_t)S * (cap / 2)) / M;
  int r = r0 < 1 ? 1 : (r0 > S ? S : (int)r0);
  const int64_t rk = ((int64_t)k * S + M - 1) / M;   // at least k values expected below
  r = max(r, rk > S ? S : (int)rk);
  for (int attempt = 0; attempt < 4 && cap >= S; ++attempt) {
    for (int i = lane; i < S; i += 32) buf[i] = vals[(int64_t)i * M / S];
    __syncwarp();
    const float h = fkey_inv(warp_radix_kth(buf, S, r, hist));
    const int c = warp_filter_le(vals, M, h, buf, cap);
    if (c >= k && c <= cap) return warp_radix_kth(buf, c, k, hist);
    if (c < k) r = min(S, r * 4);
    else r = max(1, r / 4);
    if (c > cap && r == 1) break;
  }
  return warp_radix_kth(vals, M, k, hist);
}

// ordered warp compaction: out[n..] = src[i] for every i < M with keep(i); returns new n
template <class Keep>
__device__ __forceinline__ int warp_compact(const int32_t* src, int M, int32_t* out, Keep keep) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1;
  int n = 0;
  for (int b = 0; b < M; b += 32 * WU) {  // WU independent tests in flight per lane
    bool k[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      k[u] = i < M && keep(i);
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, k[u]);
      if (k[u]) out[n + __popc(m & below)] = src[b + 32 * u + lane];
      n += __popc(m);
    }
  }
  __syncwarp();
  return n;
}

// ordered warp compaction that also moves one float per kept entry (val -> vout)
template <class Keep>
__device__ __forceinline__ int warp_compact_val(const int32_t* src, const float* val, int M,
                                                int32_t* out, float* vout, Keep keep) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1;
  int n = 0;
  for (int b = 0; b < M; b += 32 * WU) {
    bool k[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      k[u] = i < M && keep(i);
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const unsigned m = __ballot_sync(0xffffffffu, k[u]);
      if (k[u]) {
        const int at = n + __popc(m & below);
        out[at] = src[b + 32 * u + lane];
        vout[at] = val[b + 32 * u + lane];
      }
      n += __popc(m);
    }
  }
  __syncwarp();
  return n;
}

// Register-resident selection for short survivor lists: entry lane + 32 t of a query's
// list sits in register t of the lane (FR registers: up to 256 entries), all of them
// loaded in one memory round trip.  k-th smallest key (k <= 32) among the M entries whose
// key is <= hk, 0xffffffff when fewer than k are -- the insertions of warp_kth_small,
// without its loads.
constexpr int FR = 8;
__device__ uint32_t warp_kth_regs(const uint32_t (&x)[FR], int M, int k, uint32_t hk) {
  const int lane = threadIdx.x & 31;
  uint32_t lst = 0xffffffffu, kth = 0xffffffffu;
#pragma unroll
  for (int t = 0; t < FR; ++t) {
    if (32 * t >= M) break;
    unsigned cand = __ballot_sync(0xffffffffu, x[t] < kth && x[t] <= hk);
    while (cand) {
      const int src = __ffs(cand) - 1;
      cand &= cand - 1;
      const uint32_t y = __shfl_sync(0xffffffffu, x[t], src);
      if (y < kth) {
        const int pos = __popc(__ballot_sync(0xffffffffu, lst < y));
        const uint32_t up = __shfl_up_sync(0xffffffffu, lst, 1);
        lst = lane > pos ? up : (lane == pos ? y : lst);
        kth = __shfl_sync(0xffffffffu, lst, k - 1);
      }
    }
  }
  return kth;
}

constexpr int FW_WARPS = 8;   // queries per CTA in the per-query warp phases
constexpr int FW_BUF = 128;   // per-warp (distance, id) sort buffer: up to k = 128 entries

// Phased finalize (k <= 128).  Selection/compaction phases run one warp per query
// and never synchronise a block; gather phases run one CTA (8 independent warps)
// per query, each lane prefetching one candidate's position per batch of 32.

constexpr int FW_FILT = 768;  // per-warp buffer of a filtered selection

// phase 1: tau_A = k-th smallest UB1, S1 = {LB1 <= tau_A} (ordered compaction).
// The scan's final per-query bound (>= tau_A) filters the upper bounds first.
__global__ void __launch_bounds__(FW_WARPS * 32) k_fin_s1(FinParams P) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ float filt_all[FW_WARPS][FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq) return;
  int* hist = hist_all[wid];
  const int64_t base = q * P.cap;
  // the first 32 FR entries of the query's region, loaded before its survivor count
  // arrives (one round trip less for the short lists that most queries have)
  const int lim = (int)min((int64_t)(32 * FR), P.cap);
  uint32_t x[FR];
  float lb[FR];
  int32_t ps[FR];
#pragma unroll
  for (int t = 0; t < FR; ++t) {
    const int i = 32 * t + lane;
    const bool in = i < lim;
    x[t] = in ? fkey(P.sub[base + i]) : 0xffffffffu;
    lb[t] = in ? P.slb[base + i] : FINF;
    ps[t] = in ? P.spos[base + i] : 0;
  }
  const int M = (int)min((int64_t)P.qcnt[q], P.cap);
  int64_t nc = 0;
  for (int r = lane; r < P.nprobe; r += 32) {
    const int j = P.plist[q * P.nprobe + r];
    nc += P.loff[j + 1] - P.loff[j];
  }
#pragma unroll
  for (int o = 16; o; o >>= 1) nc += __shfl_xor_sync(0xffffffffu, nc, o);
  float tauA = FINF;
  int M1 = 0;
  if (M <= 32 * FR && P.k <= 32) {
    // short list: its UB1, LB1 and positions are in registers (entries past M masked)
#pragma unroll
    for (int t = 0; t < FR; ++t)
      if (32 * t + lane >= M) { x[t] = 0xffffffffu; lb[t] = FINF; }
    if (M >= P.k) {
      const uint32_t hk = P.gtau ? __ldcg(P.gtau + q) : 0xffffffffu;
      uint32_t kt = warp_kth_regs(x, M, P.k, hk);
      if (kt == 0xffffffffu) kt = warp_kth_regs(x, M, P.k, 0xffffffffu);  // hint too low
      tauA = fkey_inv(kt);
    }
    const unsigned below = (1u << lane) - 1;
#pragma unroll
    for (int t = 0; t < FR; ++t) {  // ordered compaction of S1 = {LB1 <= tau_A}
      const bool keep = 32 * t + lane < M && lb[t] <= tauA;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) P.s2pos[base + M1 + __popc(m & below)] = ps[t];
      M1 += __popc(m);
    }
    __syncwarp();
  } else {
  if (M >= P.k) {
    const float hint = P.gtau ? fkey_inv(__ldcg(P.gtau + q)) : FINF;
    if (P.k <= 32) {
      uint32_t kt = warp_kth_small(P.sub + base, M, P.k, hint);
      if (kt == 0xffffffffu) kt = warp_kth_small(P.sub + base, M, P.k, FINF);  // hint too low
      tauA = fkey_inv(kt);
    } else {
      tauA = fkey_inv(warp_kth_filtered(P.sub + base, M, P.k, hint, filt_all[wid], FW_FILT, hist));
    }
  }
  const float* slb = P.slb + base;
  M1 = warp_compact(P.spos + base, M, P.s2pos + base, [&](int i) { return slb[i] <= tauA; });
  }
  if (lane == 0) {
    P.qtau[q] = tauA;
    P.qm1[q] = M1;
    if (P.stats) { P.stats[q * 3 + 0] = nc; P.stats[q * 3 + 1] = M1; }
  }
}

// A query whose stage-1 region overflowed is searched again; its bound for that search
// is the k-th smallest UB1 over the survivors its region holds.  They are a subset of its
// candidates, so the bound is never below tau_A, and they came from its nearest lists
// first, so it is close to tau_A -- much tighter than the per-list bounds that its scan
// published.  Queries that did not overflow are left alone.
__global__ void __launch_bounds__(FW_WARPS * 32) k_ovf_seed(FinParams P, float* __restrict__ seed,
                                                           int64_t base) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ float filt_all[FW_WARPS][FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq || (int64_t)P.qcnt[q] <= P.cap) return;
  const float* ub = P.sub + q * P.cap;
  const int M = (int)P.cap;
  float t = FINF;
  if (M >= P.k) {
    const float hint = fkey_inv(__ldcg(P.gtau + q));
    if (P.k <= 32) {
      uint32_t kt = warp_kth_small(ub, M, P.k, hint);
      if (kt == 0xffffffffu) kt = warp_kth_small(ub, M, P.k, FINF);
      t = fkey_inv(kt);
    } else {
      t = fkey_inv(warp_kth_filtered(ub, M, P.k, hint, filt_all[wid], FW_FILT, hist_all[wid]));
    }
  }
  if (lane == 0) seed[base + q] = t;
}

// the running bound of a query searched again starts from its recorded seed (by row)
__global__ void k_seed_gtau(unsigned int* __restrict__ gtau, int64_t nq,
                            const float* __restrict__ seed, const int* __restrict__ rows) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const float t = seed[rows[q]];
  if (t < FINF) gtau[q] = fkey(t);
}

// tau_A / tau_B and the S1 / S2 compactions for a few queries with long survivor lists
// (a search again of overflowed queries; k <= 32): one CTA per query, its eight warps each
// taking an eighth of the list -- each warp's k smallest upper bounds (streamed, one round
// trip per WU chunks), the k-th smallest of those 8k in one warp (the k smallest of the
// union are among them), then an ordered compaction (per-warp counts, their prefix, the
// warps' writes at their offsets).  The same values as k_fin_s1 / k_fin_s2.
__device__ uint32_t cta_kth_of_slices(const float* vals, int M, int k, uint32_t hk,
                                      uint32_t (*s_l)[32], volatile uint32_t* s_out) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int per = (M + 7) / 8, lo = min(M, wid * per), hi = min(M, lo + per);
  s_l[wid][lane] = warp_topk_list(vals + lo, hi - lo, k, hk);
  __syncthreads();
  if (wid == 0) {
    uint32_t x[FR];
#pragma unroll
    for (int t = 0; t < FR; ++t) x[t] = s_l[t][lane];
    const uint32_t kt = warp_kth_regs(x, 32 * FR, k, 0xffffffffu);
    if (lane == 0) *s_out = kt;
  }
  __syncthreads();
  return *s_out;
}

// k-th smallest key of vals[0..M) among the keys <= hk over a whole CTA (k <= 128): the
// values <= the hint are gathered into the shared buffer (warp-aggregated appends), and
// when k to C of them are, warp 0 selects in the buffer (radix select); fewer than k:
// 0xffffffff; more than C: warp 0 runs the warp's filtered selection over all M values.
constexpr int WIDE_BUF = 4096;
__device__ uint32_t cta_kth_filtered(const float* vals, int M, int k, uint32_t hk, float* buf,
                                     int* hist, float* filt, volatile int* s_n,
                                     volatile uint32_t* s_out) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1;
  if (threadIdx.x == 0) *s_n = 0;
  __syncthreads();
  for (int b = 0; b < M; b += 256 * WU) {
    float v[WU];
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 256 * u + (int)threadIdx.x;
      v[u] = i < M ? vals[i] : FINF;
    }
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 256 * u + (int)threadIdx.x;
      const bool keep = i < M && fkey(v[u]) <= hk;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (m) {
        int at = 0;
        if (lane == __ffs(m) - 1) at = atomicAdd((int*)s_n, __popc(m));
        at = __shfl_sync(0xffffffffu, at, __ffs(m) - 1) + __popc(m & below);
        if (keep && at < WIDE_BUF) buf[at] = v[u];
      }
    }
  }
  __syncthreads();
  const int n = *s_n;
  if (threadIdx.x < 32) {
    uint32_t kt = 0xffffffffu;
    if (n >= k && n <= WIDE_BUF) kt = warp_radix_kth(buf, n, k, hist);
    else if (n > WIDE_BUF)
      kt = warp_kth_filtered(vals, M, k, hk == 0xffffffffu ? FINF : fkey_inv(hk), filt, FW_FILT,
                             hist);
    if (lane == 0) *s_out = kt;
  }
  __syncthreads();
  return *s_out;
}

__global__ void __launch_bounds__(256) k_fin_s1_wide(FinParams P) {
  __shared__ uint32_t s_l[8][32];
  __shared__ int s_cnt[8];
  __shared__ uint32_t s_kt;
  __shared__ int s_n;
  __shared__ float s_buf[WIDE_BUF];
  __shared__ int s_hist[256];
  __shared__ float s_filt[FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  const int64_t base = q * P.cap;
  const int M = (int)min((int64_t)P.qcnt[q], P.cap);
  float tauA = FINF;
  if (M >= P.k) {
    auto kth = [&](uint32_t hk) {
      return P.k <= 32 ? cta_kth_of_slices(P.sub + base, M, P.k, hk, s_l, &s_kt)
                       : cta_kth_filtered(P.sub + base, M, P.k, hk, s_buf, s_hist, s_filt, &s_n,
                                          &s_kt);
    };
    uint32_t kt = kth(__ldcg(P.gtau + q));
    if (kt == 0xffffffffu) kt = kth(0xffffffffu);  // the hint too low: without it
    tauA = fkey_inv(kt);
  }
  const int per = (M + 7) / 8, lo = min(M, wid * per), hi = min(M, lo + per);
  const float* slb = P.slb + base + lo;
  int c = 0;
  for (int b = 0; b < hi - lo; b += 32 * WU) {
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      c += __popc(__ballot_sync(0xffffffffu, i < hi - lo && slb[i] <= tauA));
    }
  }
  if (lane == 0) s_cnt[wid] = c;
  __syncthreads();
  int off = 0, M1 = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    off += w < wid ? s_cnt[w] : 0;
    M1 += s_cnt[w];
  }
  warp_compact(P.spos + base + lo, hi - lo, P.s2pos + base + off,
               [&](int i) { return slb[i] <= tauA; });
  if (threadIdx.x == 0) {
    int64_t nc = 0;
    for (int r = 0; r < P.nprobe; ++r) {
      const int j = P.plist[q * P.nprobe + r];
      nc += P.loff[j + 1] - P.loff[j];
    }
    P.qtau[q] = tauA;
    P.qm1[q] = M1;
    if (P.stats) { P.stats[q * 3 + 0] = nc; P.stats[q * 3 + 1] = M1; }
  }
}

__global__ void __launch_bounds__(256) k_fin_s2_wide(FinParams P) {
  __shared__ uint32_t s_l[8][32];
  __shared__ int s_cnt[8];
  __shared__ uint32_t s_kt;
  __shared__ int s_n;
  __shared__ float s_buf[WIDE_BUF];
  __shared__ int s_hist[256];
  __shared__ float s_filt[FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  const int64_t base = q * P.cap;
  const int M1 = P.qm1[q];
  const float tauA = P.qtau[q];
  // only upper bounds <= tau_A can lower tau_B = min(tau_A, k-th smallest UB2)
  float tauB = tauA;
  if (M1 >= P.k) {
    const uint32_t kt =
        P.k <= 32 ? cta_kth_of_slices(P.s2a + base, M1, P.k, fkey(tauA), s_l, &s_kt)
                  : cta_kth_filtered(P.s2a + base, M1, P.k, fkey(tauA), s_buf, s_hist, s_filt,
                                     &s_n, &s_kt);
    if (kt != 0xffffffffu) tauB = fminf(tauA, fkey_inv(kt));
  }
  const int per = (M1 + 7) / 8, lo = min(M1, wid * per), hi = min(M1, lo + per);
  const float* lb2 = P.s2b + base + lo;
  int c = 0;
  for (int b = 0; b < hi - lo; b += 32 * WU) {
#pragma unroll
    for (int u = 0; u < WU; ++u) {
      const int i = b + 32 * u + lane;
      c += __popc(__ballot_sync(0xffffffffu, i < hi - lo && lb2[i] <= tauB));
    }
  }
  if (lane == 0) s_cnt[wid] = c;
  __syncthreads();
  int off = 0, M2 = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    off += w < wid ? s_cnt[w] : 0;
    M2 += s_cnt[w];
  }
  // positions to spos, their |x_d' - q_d'|^2 (stage 2, in sub) to slb
  warp_compact_val(P.s2pos + base + lo, P.sub + base + lo, hi - lo, P.spos + base + off,
                   P.slb + base + off, [&](int i) { return lb2[i] <= tauB; });
  if (threadIdx.x == 0) {
    P.qm2[q] = M2;
    if (P.stats) P.stats[q * 3 + 2] = M2;
  }
}

// 1 bit + refinement, stage 1b: the full B-bit estimate (Eq. 4) and bounds (Eq. 5 plus
// the Chebyshev term) of every stage-1a survivor (S1a, in s2pos), UB1b -> s2a,
// LB1b -> s2b.  One CTA per query.  A survivor's pair (its probed list) is found by a
// binary search over the query's probed lists sorted by list id (list starts ascend with
// the id, and an empty list never holds a candidate, so the last probed list starting
// at or before the position holds it); its quantized query (the same grid as the scan
// of stage 1a) comes from k_pair_prep.
struct RefineParams {
  const int32_t* plist;
  const int64_t* loff;
  const int64_t* ploff;
  const uint32_t* codes;
  const float* fadd;
  const float* fres;
  const float* ferr;
  const PairQ* pq;
  const uint32_t* qplanes;
  const int* qm1;
  const int32_t* s2pos;
  float* s2a;
  float* s2b;
  int d, bits, words, vw, nprobe, qbits;
  int64_t cap;
};

__global__ void __launch_bounds__(256) k_refine1b(RefineParams P) {
  extern __shared__ int rsm[];
  int* jraw = rsm;                     // the query's probed lists in probe order
  int* jsort = rsm + P.nprobe;         // ascending list ids
  int* start = rsm + 2 * P.nprobe;     // their first positions
  const int64_t q = blockIdx.x;
  const int np = P.nprobe;
  for (int r = threadIdx.x; r < np; r += 256) jraw[r] = P.plist[q * np + r];
  __syncthreads();
  for (int r = threadIdx.x; r < np; r += 256) {  // rank of a distinct id = its sorted slot
    const int j = jraw[r];
    int rank = 0;
    for (int t = 0; t < np; ++t) rank += jraw[t] < j;
    jsort[rank] = r;
    start[rank] = (int)P.loff[j];
  }
  __syncthreads();
  const int M = P.qm1[q];
  const int64_t base = q * P.cap;
  const int nch = P.d >> 5;
  const int topc = (1 << P.bits) - 1;
  const int lvw = P.vw == 4 ? 2 : P.vw == 2 ? 1 : 0;
  for (int i = threadIdx.x; i < M; i += 256) {
    const int p = P.s2pos[base + i];
    int lo = 0, hi = np - 1;  // last t with start[t] <= p
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (start[mid] <= p) lo = mid; else hi = mid - 1;
    }
    const int r = jsort[lo];
    const int j = jraw[r];
    const int64_t w = q * np + r;
    const int64_t pp = P.ploff[j] + (p - P.loff[j]);
    const float4 pa = __ldg(reinterpret_cast<const float4*>(P.pq + w));      // sg, a0, e0, em
    const float4 pb = __ldg(reinterpret_cast<const float4*>(P.pq + w) + 1);  // ql, qdelta, qsum
    const int qsum = __float_as_int(pb.z);
    const uint32_t* qw = P.qplanes + w * (int64_t)(P.qbits * nch);
    const uint32_t* cbase = P.codes + (pp >> 5) * (int64_t)P.words * 32 + (pp & 31) * P.vw;
    int dot = 0, su = 0;
    for (int a = 0; a < P.bits; ++a) {
      int pd = 0, ps = 0;
      for (int c = 0; c < nch; ++c) {
        const int wd = a * nch + c;
        const uint32_t word = __ldg(cbase + ((wd >> lvw) << (5 + lvw)) + (wd & (P.vw - 1)));
        ps += __popc(word);
        for (int bq = 0; bq < P.qbits; ++bq) pd += __popc(word & __ldg(qw + bq * nch + c)) << bq;
      }
      dot += pd << a;
      su += ps << a;
    }
    const float ip = pb.y * (float)(2 * dot - topc * qsum) + pb.x * (float)(2 * su - P.d * topc);
    const float fa = __ldg(P.fadd + pp), fr = __ldg(P.fres + pp), fe = __ldg(P.ferr + pp);
    const float dis = fa + pa.y + fr * pa.x * ip;  // Eq. 4
    const float eps = pa.z * fe + pa.w;            // Eq. 5 + Chebyshev
    P.s2a[base + i] = dis + eps;
    P.s2b[base + i] = dis - eps;
  }
}

// phase 2 (MRQ+): dis_o' = |x_p|^2 + |q_p|^2 - 2 <x_d', q_d'> (Eq. 7), UB2/LB2 = dis_o' -+ m sigma.
// The same pass over x_d' also sums |x_d' - q_d'|^2 directly, the leading part of the
// exact distance, into sub (free once tau_A is known), so that the exact rerank
// reads only x_r.
__global__ void __launch_bounds__(256) k_fin_stage2(FinParams P) {
  extern __shared__ __align__(16) float sq[];  // q_d'
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  for (int i = threadIdx.x; i < P.d; i += 256) sq[i] = P.qd[q * P.d + i];
  __syncthreads();
  const int M1 = P.qm1[q];
  const int64_t base = q * P.cap;
  const float em = P.m * P.qstat[q * 4 + 1];
  const float qp2 = P.qstat[q * 4 + 2];
  const bool vd = (P.d & 3) == 0;
  // warp wid owns candidates [lo, hi): an even split over the 8 warps
  const int per = (M1 + 7) / 8, lo = min(M1, wid * per), hi = min(M1, lo + per);
  for (int b = lo; b < hi; b += 32) {
    const int cnt = min(32, hi - b);
    const int myp = lane < cnt ? P.s2pos[base + b + lane] : 0;
    const float myx = lane < cnt ? P.xn2[myp] : 0.f;
    float mydot = 0.f, myd2 = 0.f;
    for (int t = 0; t < cnt; t += S2_ROWS) {
      int pr[S2_ROWS];
      float sd[S2_ROWS], se[S2_ROWS];
#pragma unroll
      for (int u = 0; u < S2_ROWS; ++u) {
        pr[u] = __shfl_sync(0xffffffffu, myp, min(t + u, cnt - 1));
        sd[u] = 0.f;
        se[u] = 0.f;
      }
      rows_dot_dist2<S2_ROWS>(P.xd, pr, cnt - t, sq, P.d, vd, lane, sd, se);
#pragma unroll
      for (int u = 0; u < S2_ROWS; ++u) {
        const float a = warp_sum(sd[u]), e = warp_sum(se[u]);
        if (lane == t + u) { mydot = a; myd2 = e; }
      }
    }
    if (lane < cnt) {
      const float diso = myx + qp2 - 2.f * mydot;
      P.s2a[base + b + lane] = diso + em;
      P.s2b[base + b + lane] = diso - em;
      P.sub[base + b + lane] = myd2;
    }
  }
}

// Stage 2 for d = 32 * NC (NC = 1, 2, 4, 8): one CTA per query, each 8-lane group of a
// warp owns a row of x_d' at a time (lane j of the group reads the row's float4 chunks
// j, j + 8, ...; the query's matching chunks stay in registers), two rows per group in
// flight; the dot and |x_d' - q_d'|^2 of a row are summed over its 8 lanes in 3 steps.
template <int NC, bool SPLIT>
__global__ void __launch_bounds__(256) k_fin_stage2_g(FinParams P) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int j = lane & 7, grp = wid * 4 + (lane >> 3);   // 32 groups of 8 lanes
  const int64_t q = blockIdx.x;
  const int M1 = P.qm1[q];
  if (M1 == 0) return;
  // SPLIT: the query's rows split over gridDim.y CTAs (a few queries with long lists)
  int c0 = 0, c1 = M1;
  if constexpr (SPLIT) {
    const int share = (M1 + (int)gridDim.y - 1) / (int)gridDim.y;
    c0 = min(M1, (int)blockIdx.y * share);
    c1 = min(M1, c0 + share);
  }
  constexpr int d = NC * 32;
  const float4* qv = reinterpret_cast<const float4*>(P.qd + q * d);
  float4 qc[NC];
#pragma unroll
  for (int t = 0; t < NC; ++t) qc[t] = __ldg(qv + j + 8 * t);
  const int64_t base = q * P.cap;
  const float em = P.m * P.qstat[q * 4 + 1];
  const float qp2 = P.qstat[q * 4 + 2];
  for (int r0 = c0 + grp; r0 < c1; r0 += 64) {
    const int r1 = r0 + 32;
    const bool has1 = r1 < c1;
    const int p0 = P.s2pos[base + r0];
    const int p1 = has1 ? P.s2pos[base + r1] : p0;
    const float4* x0 = reinterpret_cast<const float4*>(P.xd + (int64_t)p0 * d);
    const float4* x1 = reinterpret_cast<const float4*>(P.xd + (int64_t)p1 * d);
    float4 a[NC], b[NC];
#pragma unroll
    for (int t = 0; t < NC; ++t) a[t] = __ldg(x0 + j + 8 * t);
#pragma unroll
    for (int t = 0; t < NC; ++t) b[t] = __ldg(x1 + j + 8 * t);
    float da = 0.f, ea = 0.f, db = 0.f, eb = 0.f;
#pragma unroll
    for (int t = 0; t < NC; ++t) {
      const float4 c = qc[t];
      float u;
      da = fmaf(a[t].x, c.x, da); da = fmaf(a[t].y, c.y, da);
      da = fmaf(a[t].z, c.z, da); da = fmaf(a[t].w, c.w, da);
      u = a[t].x - c.x; ea = fmaf(u, u, ea); u = a[t].y - c.y; ea = fmaf(u, u, ea);
      u = a[t].z - c.z; ea = fmaf(u, u, ea); u = a[t].w - c.w; ea = fmaf(u, u, ea);
      db = fmaf(b[t].x, c.x, db); db = fmaf(b[t].y, c.y, db);
      db = fmaf(b[t].z, c.z, db); db = fmaf(b[t].w, c.w, db);
      u = b[t].x - c.x; eb = fmaf(u, u, eb); u = b[t].y - c.y; eb = fmaf(u, u, eb);
      u = b[t].z - c.z; eb = fmaf(u, u, eb); u = b[t].w - c.w; eb = fmaf(u, u, eb);
    }
    // the groups of a warp may run different numbers of rows: the reduction names only
    // this group's 8 lanes (offsets 4, 2, 1 stay inside the group)
    const unsigned gmask = 0xffu << (lane & 24);
#pragma unroll
    for (int o = 4; o; o >>= 1) {
      da += __shfl_xor_sync(gmask, da, o);
      ea += __shfl_xor_sync(gmask, ea, o);
      db += __shfl_xor_sync(gmask, db, o);
      eb += __shfl_xor_sync(gmask, eb, o);
    }
    if (j == 0) {
      const float diso = __ldg(P.xn2 + p0) + qp2 - 2.f * da;
      P.s2a[base + r0] = diso + em;
      P.s2b[base + r0] = diso - em;
      P.sub[base + r0] = ea;
    } else if (j == 1 && has1) {
      const float diso = __ldg(P.xn2 + p1) + qp2 - 2.f * db;
      P.s2a[base + r1] = diso + em;
      P.s2b[base + r1] = diso - em;
      P.sub[base + r1] = eb;
    }
  }
}

// 1 bit + refinement, end of stage 1: tau_A = min(tau_A', k-th smallest UB1b over S1a),
// S1 = {i in S1a : LB1b <= tau_A} (ordered compaction, s2pos -> spos); qtau and qm1 then
// hold tau_A and |S1|
__global__ void __launch_bounds__(FW_WARPS * 32) k_fin_s1b(FinParams P) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ float filt_all[FW_WARPS][FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq) return;
  const int64_t base = q * P.cap;
  const int M = P.qm1[q];
  const float tauA1 = P.qtau[q];
  float tauA = tauA1;
  if (M >= P.k) {
    if (P.k <= 32) {
      // fewer than k upper bounds <= tau_A': the k-th exceeds it, tau_A = tau_A'
      const uint32_t kt = warp_kth_small(P.s2a + base, M, P.k, tauA1);
      if (kt != 0xffffffffu) tauA = fminf(tauA1, fkey_inv(kt));
    } else {
      tauA = fminf(tauA1, fkey_inv(warp_kth_filtered(P.s2a + base, M, P.k, tauA1, filt_all[wid],
                                                     FW_FILT, hist_all[wid])));
    }
  }
  const float* lb = P.s2b + base;
  const int M1 = warp_compact(P.s2pos + base, M, P.spos + base,
                              [&](int i) { return lb[i] <= tauA; });
  if (lane == 0) {
    P.qtau[q] = tauA;
    P.qm1[q] = M1;
    if (P.stats) P.stats[q * 3 + 1] = M1;
  }
}

// phase 3: tau_B = min(tau_A, k-th smallest UB2 over S1), S2 = {LB2 <= tau_B}
// (MRQ mode: S2 = S1)
__global__ void __launch_bounds__(FW_WARPS * 32) k_fin_s2(FinParams P) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ float filt_all[FW_WARPS][FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq) return;
  const int64_t base = q * P.cap;
  const int M1 = P.qm1[q];
  int M2;
  if (P.mode == MRQ_MODE_MRQ_PLUS && M1 <= 32 * FR && P.k <= 32) {
    // short list: UB2, LB2, positions and stage-2 terms in registers, one round trip
    const float tauA = P.qtau[q];
    uint32_t x[FR];
    float lb[FR], e2[FR];
    int32_t ps[FR];
#pragma unroll
    for (int t = 0; t < FR; ++t) {
      const int i = 32 * t + lane;
      const bool in = i < M1;
      x[t] = in ? fkey(P.s2a[base + i]) : 0xffffffffu;
      lb[t] = in ? P.s2b[base + i] : FINF;
      ps[t] = in ? P.s2pos[base + i] : 0;
      e2[t] = in ? P.sub[base + i] : 0.f;
    }
    // only upper bounds <= tau_A can lower tau_B = min(tau_A, k-th smallest UB2)
    float tauB = tauA;
    if (M1 >= P.k) {
      const uint32_t kt = warp_kth_regs(x, M1, P.k, fkey(tauA));
      if (kt != 0xffffffffu) tauB = fminf(tauA, fkey_inv(kt));
    }
    const unsigned below = (1u << lane) - 1;
    M2 = 0;
#pragma unroll
    for (int t = 0; t < FR; ++t) {  // ordered compaction of S2 = {LB2 <= tau_B}
      const bool keep = 32 * t + lane < M1 && lb[t] <= tauB;
      const unsigned m = __ballot_sync(0xffffffffu, keep);
      if (keep) {
        const int at = M2 + __popc(m & below);
        P.spos[base + at] = ps[t];
        P.slb[base + at] = e2[t];
      }
      M2 += __popc(m);
    }
    __syncwarp();
  } else if (P.mode == MRQ_MODE_MRQ_PLUS) {
    const float tauA = P.qtau[q];
    // only upper bounds <= tau_A can lower tau_B = min(tau_A, k-th smallest UB2)
    float tauB = tauA;
    if (M1 >= P.k) {
      if (P.k <= 32) {
        // fewer than k upper bounds <= tau_A: the k-th exceeds tau_A, tau_B = tau_A
        const uint32_t kt = warp_kth_small(P.s2a + base, M1, P.k, tauA);
        if (kt != 0xffffffffu) tauB = fminf(tauA, fkey_inv(kt));
      } else {
        tauB = fminf(tauA, fkey_inv(warp_kth_filtered(P.s2a + base, M1, P.k, tauA, filt_all[wid],
                                                      FW_FILT, hist_all[wid])));
      }
    }
    const float* lb2 = P.s2b + base;
    // positions to spos, their |x_d' - q_d'|^2 (stage 2, in sub) to slb
    M2 = warp_compact_val(P.s2pos + base, P.sub + base, M1, P.spos + base, P.slb + base,
                          [&](int i) { return lb2[i] <= tauB; });
  } else {
    M2 = warp_compact(P.s2pos + base, M1, P.spos + base, [&](int) { return true; });
  }
  if (lane == 0) {
    P.qm2[q] = M2;
    if (P.stats) P.stats[q * 3 + 2] = M2;
  }
}

// phase 4: exact distances |x_d' - q_d'|^2 + |x_r - q_r|^2 (direct sums)
__global__ void __launch_bounds__(256) k_fin_exact(FinParams P) {
  extern __shared__ __align__(16) float sq[];  // [q_d' | pad | q_r]
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  const int dpad = (P.d + 3) & ~3;
  for (int i = threadIdx.x; i < P.d; i += 256) sq[i] = P.qd[q * P.d + i];
  for (int i = threadIdx.x; i < P.r; i += 256) sq[dpad + i] = P.qr[q * P.r + i];
  __syncthreads();
  const int M2 = P.qm2[q];
  const int64_t base = q * P.cap;
  const bool vd = (P.d & 3) == 0, vr = (P.r & 3) == 0;
  const int per = (M2 + 7) / 8, lo = min(M2, wid * per), hi = min(M2, lo + per);
  for (int b = lo; b < hi; b += 32) {
    const int cnt = min(32, hi - b);
    const int myp = lane < cnt ? P.spos[base + b + lane] : 0;
    float mine = 0.f;
    for (int t = 0; t < cnt; t += 2) {
      const int p0 = __shfl_sync(0xffffffffu, myp, t);
      const int p1 = __shfl_sync(0xffffffffu, myp, min(t + 1, cnt - 1));
      float s0 = 0.f, s1 = 0.f;
      row_accum2<false>(P.xd + (int64_t)p0 * P.d, P.xd + (int64_t)p1 * P.d, sq, P.d, vd, lane, s0, s1);
      row_accum2<false>(P.xr + (int64_t)p0 * P.r, P.xr + (int64_t)p1 * P.r, sq + dpad, P.r, vr, lane, s0, s1);
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      if (lane == t) mine = s0;
      if (lane == t + 1) mine = s1;
    }
    if (lane < cnt) P.slb[base + b + lane] = mine;
  }
}

// phase 4, MRQ+ with r % 4 == 0: |x_d' - q_d'|^2 is already in slb (stage 2), so only
// the x_r rows are read.  A warp takes two rows at a time and keeps EX_U float4 of
// each in flight per lane.
constexpr int EX_U = 4;
__global__ void __launch_bounds__(256) k_fin_exact_r(FinParams P) {
  extern __shared__ __align__(16) float sq[];  // q_r
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = blockIdx.x;
  const int r4 = P.r >> 2;
  for (int i = threadIdx.x; i < P.r; i += 256) sq[i] = P.qr[q * P.r + i];
  __syncthreads();
  const float4* qv = reinterpret_cast<const float4*>(sq);
  const int M2 = P.qm2[q];
  const int64_t base = q * P.cap;
  // the query's rows split over gridDim.y CTAs (one unless a few queries hold long lists),
  // each CTA's share split evenly over its 8 warps
  const int share = (M2 + (int)gridDim.y - 1) / (int)gridDim.y;
  const int r0 = min(M2, (int)blockIdx.y * share), r1 = min(M2, r0 + share);
  const int per = (r1 - r0 + 7) / 8, lo = min(r1, r0 + wid * per), hi = min(r1, lo + per);
  for (int b = lo; b < hi; b += 32) {
    const int cnt = min(32, hi - b);
    const int myp = lane < cnt ? P.spos[base + b + lane] : 0;
    float mine = lane < cnt ? P.slb[base + b + lane] : 0.f;
    for (int t = 0; t < cnt; t += 2) {
      const int p0 = __shfl_sync(0xffffffffu, myp, t);
      const int p1 = __shfl_sync(0xffffffffu, myp, min(t + 1, cnt - 1));
      const float4* x0 = reinterpret_cast<const float4*>(P.xr + (int64_t)p0 * P.r);
      const float4* x1 = reinterpret_cast<const float4*>(P.xr + (int64_t)p1 * P.r);
      float s0 = 0.f, s1 = 0.f;
      for (int c0 = lane; c0 < r4; c0 += 32 * EX_U) {
        float4 a[EX_U], bb[EX_U];
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const int c = c0 + 32 * u;
          a[u] = c < r4 ? __ldg(x0 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
          bb[u] = c < r4 ? __ldg(x1 + c) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < EX_U; ++u) {
          const int c = c0 + 32 * u;
          if (c < r4) {
            const float4 qq = qv[c];
            float e;
            e = a[u].x - qq.x; s0 = fmaf(e, e, s0); e = a[u].y - qq.y; s0 = fmaf(e, e, s0);
            e = a[u].z - qq.z; s0 = fmaf(e, e, s0); e = a[u].w - qq.w; s0 = fmaf(e, e, s0);
            e = bb[u].x - qq.x; s1 = fmaf(e, e, s1); e = bb[u].y - qq.y; s1 = fmaf(e, e, s1);
            e = bb[u].z - qq.z; s1 = fmaf(e, e, s1); e = bb[u].w - qq.w; s1 = fmaf(e, e, s1);
          }
        }
      }
      s0 = warp_sum(s0);
      s1 = warp_sum(s1);
      if (lane == t) mine += s0;
      if (lane == t + 1) mine += s1;
    }
    if (lane < cnt) P.slb[base + b + lane] = mine;
  }
}

// phase 5: the k smallest (distance, id), ties at the k-th distance to the lower ids
__global__ void __launch_bounds__(FW_WARPS * 32) k_fin_topk(FinParams P) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ unsigned long long buf_all[FW_WARPS][FW_BUF];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq) return;
  unsigned long long* buf = buf_all[wid];
  const int64_t base = q * P.cap;
  const float* dist = P.slb + base;
  // the first 64 entries' distances and positions, loaded before the count arrives
  float dv[2];
  int32_t pv[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = 32 * h + lane;
    const bool in = i < P.cap;
    dv[h] = in ? dist[i] : FINF;
    pv[h] = in ? P.spos[base + i] : 0;
  }
  const int M2 = P.qm2[q];
  if (M2 <= 64 && P.k <= 32) {
    // short list: the (distance, id) keys of all M2 entries in two registers a lane
    // (entry lane and lane + 32), sorted by a bitonic network over the warp; the k
    // smallest are the answer (ties at the k-th distance: smallest ids first)
    unsigned long long v[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = 32 * h + lane;
      v[h] = i < M2 ? ((unsigned long long)fkey(dv[h]) << 32) | (uint32_t)P.ids[pv[h]] : ~0ull;
    }
    for (int size = 2; size <= 64; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int e = 32 * h + lane;
          const bool up = (e & size) == 0;
          if (stride == 32) {  // partner in this lane's other register
            if (h == 0) {
              const bool swap = (v[0] > v[1]) == up;
              const unsigned long long lo = swap ? v[1] : v[0], hi = swap ? v[0] : v[1];
              v[0] = lo;
              v[1] = hi;
            }
          } else {
            const unsigned long long o = __shfl_xor_sync(0xffffffffu, v[h], stride);
            const bool lower = (e & stride) == 0;  // this entry is the pair's first
            const bool take_min = lower == up;
            v[h] = take_min ? (o < v[h] ? o : v[h]) : (o > v[h] ? o : v[h]);
          }
        }
      }
    }
    if (lane < P.k) {
      const bool has = v[0] != ~0ull;
      P.out_ids[q * P.k + lane] = has ? (int64_t)(uint32_t)(v[0] & 0xffffffffu) : -1;
      P.out_d[q * P.k + lane] = has ? fkey_inv((uint32_t)(v[0] >> 32)) : FINF;
    }
    return;
  }
  const uint32_t T = M2 > P.k ? (P.k <= 32 ? warp_kth_small(dist, M2, P.k, FINF)
                                           : warp_radix_kth(dist, M2, P.k, hist_all[wid]))
                              : 0xffffffffu;
  int n = 0;
  for (int b = 0; b < M2; b += 32) {  // entries strictly below T (fewer than k)
    const int i = b + lane;
    const bool lt = i < M2 && fkey(dist[i]) < T;
    const unsigned m = __ballot_sync(0xffffffffu, lt);
    if (lt) buf[n + __popc(m & ((1u << lane) - 1))] =
        ((unsigned long long)fkey(dist[i]) << 32) | (uint32_t)P.ids[P.spos[base + i]];
    n += __popc(m);
  }
  if (T != 0xffffffffu) {  // ties at T, smallest ids first
    uint32_t last = 0u;
    bool first = true;
    while (n < P.k) {
      uint32_t best = 0xffffffffu;
      for (int i = lane; i < M2; i += 32) {
        if (fkey(dist[i]) == T) {
          const uint32_t id = (uint32_t)P.ids[P.spos[base + i]];
          if ((first || id > last) && id < best) best = id;
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
      if (best == 0xffffffffu) break;
      if (lane == 0) buf[n] = ((unsigned long long)T << 32) | best;
      ++n;
      last = best;
      first = false;
    }
  }
  __syncwarp();
  int n2 = 1;
  while (n2 < n) n2 <<= 1;
  for (int i = n + lane; i < n2; i += 32) buf[i] = ~0ull;
  __syncwarp();
  for (int size = 2; size <= n2; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int t = lane; t < n2 / 2; t += 32) {
        const int i = 2 * t - (t & (stride - 1));
        const int j = i + stride;
        const bool up = ((i & size) == 0);
        const unsigned long long x = buf[i], y = buf[j];
        if ((x > y) == up) { buf[i] = y; buf[j] = x; }
      }
      __syncwarp();
    }
  }
  for (int i = lane; i < P.k; i += 32) {
    if (i < n) {
      P.out_ids[q * P.k + i] = (int64_t)(uint32_t)(buf[i] & 0xffffffffu);
      P.out_d[q * P.k + i] = fkey_inv((uint32_t)(buf[i] >> 32));
    } else {
      P.out_ids[q * P.k + i] = -1;
      P.out_d[q * P.k + i] = FINF;
    }
  }
}

// ------------------------------------------------------------------ MR-SQ (Exp-5)
//
// 8-bit scalar quantization of x_d' (per dimension: 256 levels from the base's min to
// max, round to nearest, decided in float32), the estimate
// |q_d' - x_hat|^2 + |x_r|^2 + |q_r|^2, a fixed rerank range instead of error bounds.

// column min / max of X (n x d) as order-preserving keys: mm[c] = min, mm[d + c] = max
__global__ void k_sq8_minmax(const float* __restrict__ X, int64_t n, int d, int64_t rows_per,
                             unsigned int* __restrict__ mm) {
  const int c = blockIdx.x * 32 + (threadIdx.x & 31);
  const int64_t r0 = (int64_t)blockIdx.y * rows_per + (threadIdx.x >> 5);
  const int64_t r1 = min(n, (int64_t)(blockIdx.y + 1) * rows_per);
  if (c >= d) return;
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (int64_t r = r0; r < r1; r += blockDim.x >> 5) {
    const uint32_t k = fkey(X[r * d + c]);
    lo = min(lo, k);
    hi = max(hi, k);
  }
  atomicMin(mm + c, lo);
  atomicMax(mm + d + c, hi);
}

__global__ void k_sq8_grid(const unsigned int* __restrict__ mm, int d, float* __restrict__ lo,
                           float* __restrict__ delta) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= d) return;
  const float a = fkey_inv(mm[c]), b = fkey_inv(mm[d + c]);
  lo[c] = a;
  delta[c] = (b - a) / 255.f;
}

__global__ void k_sq8_encode(const float* __restrict__ X, int64_t n, int d,
                             const float* __restrict__ lo, const float* __restrict__ delta,
                             uint8_t* __restrict__ codes) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * d) return;
  const int c = (int)(i % d);
  const float dl = delta[c];
  int v = 0;
  if (dl > 0.f) {
    const float t = (X[i] - lo[c]) / dl;
    v = (int)floorf(t + 0.5f);
    v = min(max(v, 0), 255);
  }
  codes[i] = (uint8_t)v;
}

__global__ void k_sq8_rownorm(const float* __restrict__ X, int64_t n, int r, float* __restrict__ out) {
  const int64_t p = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (p >= n) return;
  float s = 0.f;
  for (int c = threadIdx.x & 31; c < r; c += 32) s = fmaf(X[p * r + c], X[p * r + c], s);
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) out[p] = s;
}

struct Sq8Params {
  const float* qd;       // nq x d
  const float* qstat;    // nq x 4 (|q_r|^2 first)
  const int32_t* plist;  // nq x nprobe
  const int64_t* loff;
  const uint8_t* codes;  // n x d, list-major
  const float* lo;
  const float* delta;
  const float* xr2;
  int d, nprobe;
  int64_t npairs, cap;
  const int64_t* items;  // (pair << 32 | chunk) work items, or NULL: one per pair
  const int* nitems;
  int chunk;
  unsigned int* work;
  unsigned int* qcnt;
  int32_t* spos;
  float* slb;
};

// one warp per (query, list) work item, one lane per candidate: the candidate's d code
// bytes in 16-byte loads, (q_d'_i - lo_i) and delta_i from shared memory; every
// candidate's (position, estimate) is appended to the query's region
__global__ void __launch_bounds__(SCAN_WARPS * 32) k_scan_sq8(Sq8Params P) {
  extern __shared__ float2 sqa[];  // per warp: d x (q_d'_i - lo_i, delta_i)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int d = P.d;
  float2* a = sqa + (int64_t)wid * d;
  const int64_t n_items = P.items ? (int64_t)*P.nitems : P.npairs;
  while (true) {
    unsigned int it = 0;
    if (lane == 0) it = atomicAdd(P.work, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((int64_t)it >= n_items) break;
    int64_t w = it, c_lo = 0, c_hi = -1;
    if (P.items) {
      const int64_t v = P.items[it];
      w = v >> 32;
      c_lo = (v & 0xffffffffll) * P.chunk;
      c_hi = c_lo + P.chunk;
    }
    const int64_t q = w / P.nprobe;
    const int j = P.plist[w];
    __syncwarp();
    for (int i = lane; i < d; i += 32) a[i] = make_float2(P.qd[q * d + i] - P.lo[i], P.delta[i]);
    __syncwarp();
    const float qr2 = P.qstat[q * 4 + 0];
    const int64_t lb0 = P.loff[j];
    const int64_t lsize = P.loff[j + 1] - lb0;
    const int64_t size = c_hi < 0 ? lsize : min(lsize, c_hi);
    for (int64_t b0 = c_lo; b0 < size; b0 += 32) {
      const int64_t idx = b0 + lane;
      const bool valid = idx < size;
      float est = 0.f;
      int64_t p = lb0 + idx;
      if (valid) {
        const uint4* row = reinterpret_cast<const uint4*>(P.codes + p * d);
        float s = 0.f;
        for (int g = 0; g < d / 16; ++g) {
          const uint4 v = __ldg(row + g);
          const uint32_t wds[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              const float2 av = a[g * 16 + e * 4 + t];
              const float x = av.x - (float)((wds[e] >> (8 * t)) & 255u) * av.y;
              s = fmaf(x, x, s);
            }
          }
        }
        est = s + __ldg(P.xr2 + p) + qr2;
      }
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      unsigned base = 0;
      if (lane == 0 && vm) base = atomicAdd(P.qcnt + q, (unsigned)__popc(vm));
      base = __shfl_sync(0xffffffffu, base, 0);
      const int64_t rel = (int64_t)base + __popc(vm & ((1u << lane) - 1));
      if (valid && rel < P.cap) {
        const int64_t at = q * P.cap + rel;
        P.spos[at] = (int32_t)p;
        P.slb[at] = est;
      }
    }
  }
}

struct PqParams {
  const float* qrot;     // nq x d: q_d' R
  const float* qstat;    // nq x 4 (|q_r|^2 first)
  const int32_t* plist;  // nq x nprobe
  const int64_t* loff;
  const uint8_t* codes;  // n x M, list-major
  const float* C;        // M x K x ds
  const float* xr2;
  int d, M, K, nprobe;
  int64_t npairs, cap;
  const int64_t* items;  // (pair << 32 | chunk) work items, or NULL: one per pair
  const int* nitems;
  int chunk;
  unsigned int* work;
  unsigned int* qcnt;
  int32_t* spos;
  float* slb;
};

// MR-PQ estimate (Exp-5): one warp per (query, list) work item builds the query's lookup
// table T[m][c] = |q'_m - C[m][c]|^2 in shared memory (q' = q_d' R, subvectors of d/M
// coordinates), then one lane per candidate sums T[m][code_m] over the M subspaces and
// adds |x_r|^2 + |q_r|^2 (the residual cross term dropped, as in Eq. 4); every
// candidate's (position, estimate) is appended to the query's region
__global__ void __launch_bounds__(SCAN_WARPS * 32) k_scan_pq(PqParams P) {
  extern __shared__ float pqt[];  // per warp: M x K table
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int M = P.M, K = P.K, ds = P.d / P.M;
  float* T = pqt + (int64_t)wid * M * K;
  const int64_t n_items = P.items ? (int64_t)*P.nitems : P.npairs;
  int64_t last_q = -1;
  while (true) {
    unsigned int it = 0;
    if (lane == 0) it = atomicAdd(P.work, 1u);
    it = __shfl_sync(0xffffffffu, it, 0);
    if ((int64_t)it >= n_items) break;
    int64_t w = it, c_lo = 0, c_hi = -1;
    if (P.items) {
      const int64_t v = P.items[it];
      w = v >> 32;
      c_lo = (v & 0xffffffffll) * P.chunk;
      c_hi = c_lo + P.chunk;
    }
    const int64_t q = w / P.nprobe;
    const int j = P.plist[w];
    if (q != last_q) {  // the table depends on the query only
      __syncwarp();
      const float* qv = P.qrot + q * P.d;
      for (int e = lane; e < M * K; e += 32) {
        const int m = e / K, c = e - m * K;
        const float* cb = P.C + ((int64_t)m * K + c) * ds;
        float s = 0.f;
        for (int t = 0; t < ds; ++t) {
          const float x = qv[m * ds + t] - cb[t];
          s = fmaf(x, x, s);
        }
        T[e] = s;
      }
      __syncwarp();
      last_q = q;
    }
    const float qr2 = P.qstat[q * 4 + 0];
    const int64_t lb0 = P.loff[j];
    const int64_t lsize = P.loff[j + 1] - lb0;
    const int64_t size = c_hi < 0 ? lsize : min(lsize, c_hi);
    for (int64_t b0 = c_lo; b0 < size; b0 += 32) {
      const int64_t idx = b0 + lane;
      const bool valid = idx < size;
      float est = 0.f;
      const int64_t p = lb0 + idx;
      if (valid) {
        const uint8_t* row = P.codes + p * M;
        float s = 0.f;
        if ((M & 3) == 0) {
          for (int m = 0; m < M; m += 4) {
            const uint32_t v4 = __ldg(reinterpret_cast<const uint32_t*>(row + m));
#pragma unroll
            for (int t = 0; t < 4; ++t) s += T[(m + t) * K + ((v4 >> (8 * t)) & 255u)];
          }
        } else {
          for (int m = 0; m < M; ++m) s += T[m * K + __ldg(row + m)];
        }
        est = s + __ldg(P.xr2 + p) + qr2;
      }
      const unsigned vm = __ballot_sync(0xffffffffu, valid);
      unsigned base = 0;
      if (lane == 0 && vm) base = atomicAdd(P.qcnt + q, (unsigned)__popc(vm));
      base = __shfl_sync(0xffffffffu, base, 0);
      const int64_t rel = (int64_t)base + __popc(vm & ((1u << lane) - 1));
      if (valid && rel < P.cap) {
        const int64_t at = q * P.cap + rel;
        P.spos[at] = (int32_t)p;
        P.slb[at] = est;
      }
    }
  }
}

// the rerank range: the R smallest estimates of each query by (estimate, id), compacted
// (positions) into s2pos; qm2 = their number
__global__ void __launch_bounds__(FW_WARPS * 32) k_sq8_select(FinParams P, int R) {
  __shared__ int hist_all[FW_WARPS][256];
  __shared__ float filt_all[FW_WARPS][FW_FILT];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t q = (int64_t)blockIdx.x * FW_WARPS + wid;
  if (q >= P.nq) return;
  const int64_t base = q * P.cap;
  const int M = (int)min((int64_t)P.qcnt[q], P.cap);
  const float* est = P.slb + base;
  const int32_t* pos = P.spos + base;
  int32_t* out = P.s2pos + base;
  int n;
  if (M <= R) {
    n = warp_compact(pos, M, out, [&](int) { return true; });
  } else {
    const uint32_t T = warp_kth_filtered(est, M, R, FINF, filt_all[wid], FW_FILT, hist_all[wid]);
    n = warp_compact(pos, M, out, [&](int i) { return fkey(est[i]) < T; });
    // estimates equal to the R-th: the lowest ids first
    uint32_t last = 0u;
    bool first = true;
    while (n < R) {
      uint32_t best = 0xffffffffu;
      int bpos = -1;
      for (int i = lane; i < M; i += 32) {
        if (fkey(est[i]) == T) {
          const uint32_t id = (uint32_t)P.ids[pos[i]];
          if ((first || id > last) && id < best) { best = id; bpos = pos[i]; }
        }
      }
#pragma unroll
      for (int o = 16; o; o >>= 1) {
        const uint32_t ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int op = __shfl_xor_sync(0xffffffffu, bpos, o);
        if (ob < best) { best = ob; bpos = op; }
      }
      if (best == 0xffffffffu) break;
      if (lane == 0) out[n] = bpos;
      ++n;
      last = best;
      first = false;
    }
    __syncwarp();
  }
  if (lane == 0) {
    P.qm2[q] = n;
    if (P.stats) {
      P.stats[q * 3 + 0] = (int64_t)M;
      P.stats[q * 3 + 1] = n;
      P.stats[q * 3 + 2] = n;
    }
  }
}

int g_num_sms = 0;
int num_sms() {
  if (!g_num_sms) {
    int dev = 0;
    MRQ_CUDA(cudaGetDevice(&dev));
    MRQ_CUDA(cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return g_num_sms;
}

template <int KM, bool QUANT, bool DBG>
void launch_scan_t(const ScanParams& p, int64_t grid_warps, size_t smem, cudaStream_t st) {
  auto kern = k_scan<KM, QUANT, DBG>;
  ensure_smem((const void*)kern, smem);
  int blocks;
  if (DBG) {
    blocks = 1;
  } else {
    const int per_sm = occupancy((const void*)kern, SCAN_WARPS * 32, smem);
    int64_t want = (grid_warps + SCAN_WARPS - 1) / SCAN_WARPS;
    blocks = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
    blocks = std::max(blocks, 1);
  }
  kern<<<blocks, SCAN_WARPS * 32, smem, st>>>(p);
  MRQ_CHECK_LAUNCH();
}

template <int KM, int NCH, int BITS, int QB, int LB = BITS>
void launch_scan_q(const ScanParams& p, int64_t grid_warps, cudaStream_t st) {
  auto kern = k_scan_q<KM, NCH, BITS, QB, LB>;
  const int per_sm = occupancy((const void*)kern, SCAN_WARPS * 32, 0);
  int64_t want = (grid_warps + SCAN_WARPS - 1) / SCAN_WARPS;
  int blocks = (int)std::min<int64_t>(want, (int64_t)num_sms() * per_sm);
  kern<<<std::max(blocks, 1), SCAN_WARPS * 32, 0, st>>>(p);
  MRQ_CHECK_LAUNCH();
}

// the specialised quantized scan for the common code shapes (k <= 128, 4-bit queries)
bool launch_scan_fixed(const ScanParams& p, int64_t npairs, cudaStream_t st) {
  if (p.qbits != 4 || p.k > 128) return false;
  const int nch = p.d >> 5;
  if (p.plane0 > 0) {  // the sign plane of a multi-bit code
    if (p.plane0 != p.bits - 1) return false;
#define MRQ_SQ1(B, N)                                                       \
    if (p.bits == B && nch == N) {                                           \
      if (p.k <= 32) launch_scan_q<0, N, 1, 4, B>(p, npairs, st);            \
      else launch_scan_q<1, N, 1, 4, B>(p, npairs, st);                      \
      return true;                                                           \
    }
    MRQ_SQ1(2, 2) MRQ_SQ1(2, 4) MRQ_SQ1(2, 8) MRQ_SQ1(4, 1) MRQ_SQ1(4, 4) MRQ_SQ1(4, 8)
#undef MRQ_SQ1
    return false;
  }
#define MRQ_SQ(B, N)                                                        \
  if (p.bits == B && nch == N) {                                             \
    if (p.k <= 32) launch_scan_q<0, N, B, 4>(p, npairs, st);                 \
    else launch_scan_q<1, N, B, 4>(p, npairs, st);                           \
    return true;                                                             \
  }
  MRQ_SQ(1, 1) MRQ_SQ(1, 2) MRQ_SQ(1, 4) MRQ_SQ(1, 8)
  MRQ_SQ(2, 2) MRQ_SQ(2, 4) MRQ_SQ(2, 8) MRQ_SQ(4, 1) MRQ_SQ(4, 4) MRQ_SQ(4, 8)
  MRQ_SQ(1, 30) MRQ_SQ(1, 32)  // d = D = 960, 1024 (no tail: IVF-RaBitQ)
#undef MRQ_SQ
  return false;
}

void launch_scan(const ScanParams& p, int64_t npairs, cudaStream_t st, bool dbg) {
  const bool quant = p.qbits > 0;
  const int km = p.k <= 32 ? 0 : (p.k <= 128 ? 1 : 2);
  if (!dbg && quant && launch_scan_fixed(p, npairs, st)) return;
  size_t smem = (size_t)SCAN_WARPS * (quant ? 2 : 5) * p.d * sizeof(float);
  if (dbg) {
    if (quant) launch_scan_t<2, true, true>(p, 1, smem, st);
    else launch_scan_t<2, false, true>(p, 1, smem, st);
    return;
  }
#define MRQ_SCAN_CASE(K)                                           \
  if (km == K) {                                                   \
    if (quant) launch_scan_t<K, true, false>(p, npairs, smem, st); \
    else launch_scan_t<K, false, false>(p, npairs, smem, st);      \
    return;                                                        \
  }
  MRQ_SCAN_CASE(0)
  MRQ_SCAN_CASE(1)
  MRQ_SCAN_CASE(2)
#undef MRQ_SCAN_CASE
}

}  // namespace

// ---------------------------------------------------------------- host side

void ensure_smem(const void* kernel, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> granted;
  int dev = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  size_t& g = granted[std::make_pair(dev, kernel)];
  if (bytes > g) {
    MRQ_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    g = bytes;
  }
}

int occupancy(const void* kernel, int threads, size_t smem) {
  static std::mutex mu;
  static std::map<std::tuple<int, const void*, int, size_t>, int> cache;
  int dev = 0;
  MRQ_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  auto key = std::make_tuple(dev, kernel, threads, smem);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int per_sm = 0;
  MRQ_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  cache[key] = std::max(per_sm, 1);
  return cache[key];
}

// CUDA event at a stage boundary of the current batch (profiled searches only)
static void mark(mrq_index* idx, int s, cudaStream_t st) {
  if (!idx->prof_on) return;
  size_t i = (size_t)idx->prof_batches * (MRQ_NSTAGES + 1) + s;
  while (idx->prof_ev.size() <= i) {
    cudaEvent_t e;
    MRQ_CUDA(cudaEventCreate(&e));
    idx->prof_ev.push_back(e);
  }
  MRQ_CUDA(cudaEventRecord(idx->prof_ev[i], st));
}

int project_batch(mrq_index* idx, Workspace& ws, const float* q, int64_t nq, int precision,
                  float* qd, float* qr, cudaStream_t st, __nv_bfloat16* probe_bf) {
  const int D = idx->D, d = idx->d, r = D - d;
  if (precision == MRQ_PREC_FP32) {
    gemm_nt_f32(q, D, idx->mu.p, idx->W.p, D, (int)nq, D, D, qd, d, qr, r, d, st);
    return 1;
  } else if (precision == MRQ_PREC_FP8) {
    MRQ_REQUIRE(tc_available(), "tensor-core projection needs an sm_103 device");
    MRQ_REQUIRE(idx->W8.p != nullptr, "FP8 projection needs D to be a multiple of 16 (16-byte e4m3 rows)");
    ws.q8.reserve((size_t)nq * D);
    ws.q8s.reserve((size_t)nq);
    project_fp8(q, idx->mu.p, idx->W8.p, idx->W8s.p, (int)nq, D, d, ws.q8.p, ws.q8s.p, qd, d, qr, r,
                st, probe_bf, nullptr);
    return 2;
  } else {
    MRQ_REQUIRE(tc_available(), "tensor-core projection needs an sm_103 device");
    MRQ_REQUIRE(D % 8 == 0, "tensor-core precisions need D to be a multiple of 8 (16-byte bf16 rows)");
    const bool s3 = precision == MRQ_PREC_BF16X3;
    if (project_fused(q, idx->mu.p, idx->W2.p, (int)nq, D, d, s3, qd, d, qr, r, probe_bf,
                      tc_error_word(), st))
      return 1;
    ws.qbf.reserve((size_t)nq * D * 2);  // the split path's bf16 queries
    return project_tc(q, idx->mu.p, idx->W2.p, (int)nq, D, d, precision == MRQ_PREC_BF16X3,
                      ws.qbf.p, qd, qr, st, probe_bf);
  }
}

static void qstats(mrq_index* idx, const float* qd, const float* qr, int64_t nq, float* qstat,
                   cudaStream_t st, unsigned int* qcnt = nullptr, unsigned int* gtau = nullptr,
                   unsigned int* work = nullptr) {
  k_qstats<<<ceil_div(nq, 8), 256, 0, st>>>(qd, qr, idx->lam.p, nq, idx->d, idx->D - idx->d, qstat,
                                            qcnt, gtau, work);
  MRQ_CHECK_LAUNCH();
}

// ---------------------------------------------------------------- scan configuration

thread_local const ScanConfig* g_force_cfg = nullptr;

ScopedScanConfig::ScopedScanConfig(const ScanConfig* c) : prev(g_force_cfg) { g_force_cfg = c; }
ScopedScanConfig::~ScopedScanConfig() { g_force_cfg = prev; }

int scan_kclass(int k) { return k <= 32 ? 0 : k <= 128 ? 1 : 2; }

ScanConfig scan_config(mrq_index* idx, const mrq_search_opts& o, int64_t nq, int k, int nprobe) {
  if (g_force_cfg) return *g_force_cfg;
  ScanConfig c{o.batched == MRQ_SCAN_AUTO ? MRQ_SCAN_PAIRS : o.batched, SCAN_CHUNK, BATCH_G};
  if (o.batched != MRQ_SCAN_AUTO) return c;
  {
    std::lock_guard<std::mutex> lk(idx->tune_mu);
    auto it = idx->tuned.find(std::make_tuple(scan_kclass(k), nprobe, o.query_bits,
                                              scan_variant(idx, o)));
    if (it != idx->tuned.end()) return it->second;
  }
  // untuned rule: batch when each probed list is shared by many queries of the batch
  const double share = (double)nq * nprobe / std::max(1, idx->nlist);
  c.scan = share >= 16.0 ? MRQ_SCAN_BATCHED : MRQ_SCAN_PAIRS;
  return c;
}

// rows[i] of src (n x D) into row i of dst
__global__ void k_gather_qrows(const float* __restrict__ src, int D, const int* __restrict__ rows,
                               int64_t n, float* __restrict__ dst) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const float* s = src + (int64_t)rows[i] * D;
  for (int c = threadIdx.x; c < D; c += blockDim.x) dst[i * D + c] = s[c];
}

// row i of the redone answers (and counters) to row rows[i] of the caller's outputs
__global__ void k_scatter_answers(const int64_t* __restrict__ ids, const float* __restrict__ d,
                                  const int64_t* __restrict__ st, int k, const int* __restrict__ rows,
                                  int64_t n, int64_t* __restrict__ out_ids, float* __restrict__ out_d,
                                  int64_t* __restrict__ out_st) {
  const int64_t i = blockIdx.x;
  if (i >= n) return;
  const int64_t row = rows[i];
  for (int t = threadIdx.x; t < k; t += blockDim.x) {
    if (out_ids) {
      out_ids[row * k + t] = ids[i * k + t];
      out_d[row * k + t] = d[i * k + t];
    }
  }
  if (threadIdx.x < 3) out_st[row * 3 + threadIdx.x] = st[i * 3 + threadIdx.x];
}

// queries whose stage-1 survivors overflowed their region: listed for a second search
__global__ void k_overflow(const unsigned int* __restrict__ qcnt, int64_t nq, int64_t cap,
                           int64_t base, int* __restrict__ ovf) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq || (int64_t)qcnt[q] <= cap) return;
  const int slot = atomicAdd(ovf, 1);
  ovf[1 + slot] = (int)(base + q);
}

void gather_query_rows(const float* src, int D, const int* rows, int64_t n, float* dst,
                       cudaStream_t st) {
  if (n <= 0) return;
  k_gather_qrows<<<(unsigned)n, 128, 0, st>>>(src, D, rows, n, dst);
  MRQ_CHECK_LAUNCH();
}

void scatter_answers(const int64_t* ids, const float* d, const int64_t* stats, int k, const int* rows,
                     int64_t n, int64_t* out_ids, float* out_d, int64_t* out_stats, cudaStream_t st) {
  if (n <= 0) return;
  k_scatter_answers<<<(unsigned)n, 128, 0, st>>>(ids, d, stats, k, rows, n, out_ids, out_d,
                                                  out_stats);
  MRQ_CHECK_LAUNCH();
}

void search_batch(mrq_index* idx, Workspace& ws, const float* q, int64_t nq, int k, int nprobe,
                  const mrq_search_opts& o, int64_t* out_ids, float* out_d, int64_t* stats,
                  cudaStream_t st) {
  const int D = idx->D, d = idx->d, r = D - d, nlist = idx->nlist;
  const int64_t cap_full = std::max<int64_t>(idx->cap_by_nprobe[nprobe], 1);
  // the bounded modes keep only stage-1 survivors, so the region may be smaller than the
  // worst case (every candidate); MR-SQ and MR-PQ append every candidate
  const bool limited = (o.mode == MRQ_MODE_MRQ || o.mode == MRQ_MODE_MRQ_PLUS) &&
                       ws.cap_limit > 0 && ws.cap_limit < cap_full && ws.ovf.p != nullptr;
  const int64_t cap = limited ? ws.cap_limit : cap_full;
  ws.qd.reserve((size_t)nq * d);
  ws.qr.reserve((size_t)nq * std::max(r, 1));
  ws.qstat.reserve((size_t)nq * 4);
  ws.gmat.reserve((size_t)nq * nlist);
  ws.plist.reserve((size_t)nq * nprobe);
  ws.pg.reserve((size_t)nq * nprobe);
  ws.qcnt.reserve(nq);
  ws.gtau.reserve(nq);
  ws.work.reserve(4);
  const size_t sc = (size_t)nq * cap;
  ws.spos.reserve(sc);
  ws.slb.reserve(sc);
  ws.sub.reserve(sc);
  ws.s2pos.reserve(sc);
  ws.s2a.reserve(sc);
  ws.s2b.reserve(sc);

  // 1-2. projection and query statistics; a tensor-core probe takes its bf16 operand
  // of q_d' straight from the projection's epilogue
  const bool tc_probe = o.precision != MRQ_PREC_FP32 && d >= 64;
  if (tc_probe) ws.qbf2.reserve((size_t)nq * d * 2);
  mark(idx, MRQ_STAGE_PROJECT, st);
  idx->launches +=
      project_batch(idx, ws, q, nq, o.precision, ws.qd.p, ws.qr.p, st, tc_probe ? ws.qbf2.p : nullptr);
  mark(idx, MRQ_STAGE_QSTATS, st);
  qstats(idx, ws.qd.p, ws.qr.p, nq, ws.qstat.p, st, ws.qcnt.p, ws.gtau.p, ws.work.p);
  if (ws.seed_tau) {  // a search again of overflowed queries: their recorded bounds
    k_seed_gtau<<<ceil_div(nq, 256), 256, 0, st>>>(ws.gtau.p, nq, ws.seed_tau, ws.seed_rows);
    MRQ_CHECK_LAUNCH();
    idx->launches += 1;
  }
  // 3. probe
  mark(idx, MRQ_STAGE_PROBE, st);
  // the fused probe emits nprobe candidates per (column tile, half tile) of each row
  const int tiles_ = probe_tc_parts(nlist);
  const bool fused = o.precision != MRQ_PREC_FP32 && d >= 64 && nprobe <= 16 &&
                     (int64_t)tiles_ * nprobe <= 512;
  if (fused) {
    ws.ppart.reserve((size_t)nq * tiles_ * nprobe);
    probe_tc_topk(ws.qd.p, ws.qstat.p, idx->cent2.p, idx->cent_n2.p, (int)nq, nlist, d,
                  o.precision == MRQ_PREC_BF16X3, nprobe, ws.qbf2.p, ws.ppart.p, st, true);
    idx->launches += 1;
  } else if (o.precision != MRQ_PREC_FP32 && d >= 64) {
    probe_tc(ws.qd.p, ws.qstat.p, idx->cent2.p, idx->cent_n2.p, (int)nq, nlist, d,
             o.precision == MRQ_PREC_BF16X3, ws.qbf2.p, ws.gmat.p, st, true);
    idx->launches += 1;
  } else {
    sqdist_f32(ws.qd.p, d, idx->cent.p, d, (int)nq, nlist, d, ws.gmat.p, nlist, st);
  }
  mark(idx, MRQ_STAGE_SELECT, st);
  if (fused) {
    const int nsl = ceil_div(tiles_ * nprobe, 32);
    const unsigned mg = ceil_div(nq, 8);
#define MRQ_MR(SLv)                                                                          \
    k_probe_merge_refine<SLv><<<mg, 256, 0, st>>>(ws.ppart.p, nq, tiles_, nprobe, ws.qd.p, \
                                                  idx->cent.p, d, ws.plist.p, ws.pg.p)
    if (nsl <= 1) MRQ_MR(1);
    else if (nsl <= 2) MRQ_MR(2);
    else if (nsl <= 4) MRQ_MR(4);
    else if (nsl <= 8) MRQ_MR(8);
    else MRQ_MR(16);
#undef MRQ_MR
    MRQ_CHECK_LAUNCH();
  } else {
    int P2 = 1;
    while (P2 < nprobe) P2 <<= 1;
    // gather capacity: room for the nprobe keys plus ties, a power of two >= nprobe
    int cap = std::min(nlist, std::max(2 * P2, 256));
    int c2 = 1;
    while (c2 < cap) c2 <<= 1;
    cap = c2;
    const int in_smem = (size_t)cap * 8 + (size_t)nlist * 4 <= 160 * 1024 ? 1 : 0;
    size_t sm = (size_t)cap * 8 + (in_smem ? (size_t)nlist * 4 : 0);
    if (nprobe <= 32) {
      k_probe_select_warp<<<ceil_div(nq, 8), 256, 0, st>>>(ws.gmat.p, nq, nlist, nprobe,
                                                          ws.plist.p, ws.pg.p);
    } else {
      ensure_smem((const void*)k_probe_select, sm);
      k_probe_select<<<(unsigned)nq, PS_NT, sm, st>>>(ws.gmat.p, nlist, nprobe, cap, in_smem,
                                                      ws.plist.p, ws.pg.p);
    }
    MRQ_CHECK_LAUNCH();
    k_probe_refine<<<ceil_div(nq * nprobe, 8), 256, 0, st>>>(ws.qd.p, idx->cent.p, ws.plist.p,
                                                            nq * nprobe, nprobe, d, ws.pg.p);
    MRQ_CHECK_LAUNCH();
  }
  // 4. scan
  mark(idx, MRQ_STAGE_SCAN, st);
  // (the survivor counts, running bounds and work counters were reset by k_qstats)
  ScanParams sp{};
  sp.qd = ws.qd.p; sp.qstat = ws.qstat.p; sp.plist = ws.plist.p; sp.pg = ws.pg.p;
  sp.cent = idx->cent.p; sp.loff = idx->loff.p; sp.ploff = idx->ploff.p; sp.codes = idx->codes.p;
  sp.fadd = idx->fadd.p; sp.fres = idx->fres.p; sp.ferr = idx->ferr.p;
  sp.d = d; sp.bits = idx->bits; sp.words = idx->words; sp.vw = idx->vw;
  sp.nprobe = nprobe; sp.k = k; sp.qbits = o.query_bits;
  sp.eps0 = o.eps0; sp.m = o.m;
  sp.npairs = nq * nprobe; sp.cap = cap;
  sp.work = ws.work.p; sp.qcnt = ws.qcnt.p; sp.gtau = ws.gtau.p;
  sp.spos = ws.spos.p; sp.slb = ws.slb.p; sp.sub = ws.sub.p;
  // scan configuration: forced (autotuner), tuned for this (k, nprobe), or the rule
  const ScanConfig cfg = scan_config(idx, o, nq, k, nprobe);
  // 1 bit + refinement: stage 1a scans the sign plane pair by pair with the 1-bit factors
  const bool refine = refine_active(idx, o);
  if (refine) {
    sp.plane0 = idx->bits - 1;
    sp.fres = idx->fres1.p;
    sp.ferr = idx->ferr1.p;
  }
  // per-pair work items (w = i * stride, i < n), long lists split into cfg.chunk chunks
  auto build_items = [&](int64_t n, int stride, int64_t rm_nq = 0) {
    const int64_t max_items = n + (nq * idx->cap_by_nprobe[nprobe]) / cfg.chunk + 1;
    ws.ccnt.reserve(n);
    ws.coff.reserve(n);
    ws.items.reserve(max_items);
    ws.nitems.reserve(1);
    k_chunk_count<<<ceil_div(n, 256), 256, 0, st>>>(ws.plist.p, idx->loff.p, n, stride,
                                                   cfg.chunk, ws.ccnt.p, rm_nq);
    MRQ_CHECK_LAUNCH();
    size_t tb = 0;
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, ws.ccnt.p, ws.coff.p, (int)n, st));
    ws.cubtmp.reserve(tb + 16);
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(ws.cubtmp.p, tb, ws.ccnt.p, ws.coff.p, (int)n, st));
    k_chunk_scatter<<<ceil_div(n, 256), 256, 0, st>>>(ws.ccnt.p, ws.coff.p, n, stride, ws.items.p,
                                                     ws.nitems.p, rm_nq);
    MRQ_CHECK_LAUNCH();
    sp.items = ws.items.p;
    sp.nitems = ws.nitems.p;
    sp.chunk = cfg.chunk;
    idx->launches += 3;
    return max_items;
  };
  if (o.mode == MRQ_MODE_SQ8 || o.mode == MRQ_MODE_PQ) {
    // MR-SQ / MR-PQ: the scan appends every probed candidate's estimate, the rerank range
    // is selected, reranked exactly and the top-k taken
    const int64_t np_ = nq * nprobe;
    if (o.mode == MRQ_MODE_PQ) {
      ws.pqq.reserve(nq * d);
      gemm_nt_f32(ws.qd.p, d, nullptr, idx->pq_Rt.p, d, (int)nq, d, d, ws.pqq.p, d, ws.pqq.p, d,
                  d, st);  // q' = q_d' R
      PqParams pp{};
      pp.qrot = ws.pqq.p; pp.qstat = ws.qstat.p; pp.plist = ws.plist.p; pp.loff = idx->loff.p;
      pp.codes = idx->pq_codes.p; pp.C = idx->pq_C.p; pp.xr2 = idx->pq_xr2.p; pp.d = d;
      pp.M = idx->pq_M; pp.K = idx->pq_K; pp.nprobe = nprobe; pp.npairs = np_; pp.cap = cap;
      pp.work = ws.work.p; pp.qcnt = ws.qcnt.p; pp.spos = ws.spos.p; pp.slb = ws.slb.p;
      int64_t grid_items = np_;
      if (idx->max_list > cfg.chunk) {
        grid_items = build_items(np_, 1);
        pp.items = sp.items; pp.nitems = sp.nitems; pp.chunk = sp.chunk;
      }
      const size_t tsm = (size_t)SCAN_WARPS * pp.M * pp.K * sizeof(float);
      ensure_smem((const void*)k_scan_pq, tsm);
      const int per_sm = occupancy((const void*)k_scan_pq, SCAN_WARPS * 32, tsm);
      const int blocks = (int)std::max<int64_t>(
          1, std::min<int64_t>((grid_items + SCAN_WARPS - 1) / SCAN_WARPS,
                               (int64_t)num_sms() * std::max(per_sm, 1)));
      k_scan_pq<<<blocks, SCAN_WARPS * 32, tsm, st>>>(pp);
      MRQ_CHECK_LAUNCH();
      idx->launches += 1;  // the query rotation (the scan is counted below)
    } else {
    Sq8Params qp{};
    qp.qd = ws.qd.p; qp.qstat = ws.qstat.p; qp.plist = ws.plist.p; qp.loff = idx->loff.p;
    qp.codes = idx->sq_codes.p; qp.lo = idx->sq_lo.p; qp.delta = idx->sq_delta.p;
    qp.xr2 = idx->sq_xr2.p; qp.d = d; qp.nprobe = nprobe; qp.npairs = np_; qp.cap = cap;
    qp.work = ws.work.p; qp.qcnt = ws.qcnt.p; qp.spos = ws.spos.p; qp.slb = ws.slb.p;
    int64_t grid_items = np_;
    if (idx->max_list > cfg.chunk) {
      grid_items = build_items(np_, 1);
      qp.items = sp.items; qp.nitems = sp.nitems; qp.chunk = sp.chunk;
    }
    const size_t qsm = (size_t)SCAN_WARPS * d * sizeof(float2);
    ensure_smem((const void*)k_scan_sq8, qsm);
    const int per_sm = occupancy((const void*)k_scan_sq8, SCAN_WARPS * 32, qsm);
    const int blocks = (int)std::max<int64_t>(
        1, std::min<int64_t>((grid_items + SCAN_WARPS - 1) / SCAN_WARPS, (int64_t)num_sms() * per_sm));
    k_scan_sq8<<<blocks, SCAN_WARPS * 32, qsm, st>>>(qp);
    MRQ_CHECK_LAUNCH();
    }
    mark(idx, MRQ_STAGE_TAU_A, st);
    FinParams fp{};
    fp.qd = ws.qd.p; fp.qr = ws.qr.p; fp.qstat = ws.qstat.p; fp.plist = ws.plist.p;
    fp.loff = idx->loff.p; fp.xd = idx->xd.p; fp.xr = idx->xr.p; fp.xn2 = idx->xn2.p;
    fp.ids = idx->ids.p; fp.d = d; fp.r = r; fp.nprobe = nprobe; fp.k = k; fp.mode = o.mode;
    fp.m = o.m; fp.cap = cap; fp.qcnt = ws.qcnt.p; fp.spos = ws.spos.p; fp.slb = ws.slb.p;
    fp.sub = ws.sub.p; fp.s2pos = ws.s2pos.p; fp.s2a = ws.s2a.p; fp.s2b = ws.s2b.p;
    fp.out_ids = out_ids; fp.out_d = out_d; fp.stats = stats;
    ws.qm2.reserve(nq);
    fp.qm2 = ws.qm2.p; fp.nq = nq;
    const unsigned gw = ceil_div(nq, FW_WARPS);
    k_sq8_select<<<gw, FW_WARPS * 32, 0, st>>>(fp, o.rerank);
    MRQ_CHECK_LAUNCH();
    for (int sidx = MRQ_STAGE_STAGE2; sidx <= MRQ_STAGE_EXACT; ++sidx) mark(idx, sidx, st);
    fp.spos = ws.s2pos.p;  // the rerank range
    const size_t esm = (size_t)(((d + 3) & ~3) + r) * 4;
    ensure_smem((const void*)k_fin_exact, esm);
    k_fin_exact<<<(unsigned)nq, 256, esm, st>>>(fp);
    MRQ_CHECK_LAUNCH();
    mark(idx, MRQ_STAGE_TOPK, st);
    k_fin_topk<<<gw, FW_WARPS * 32, 0, st>>>(fp);
    MRQ_CHECK_LAUNCH();
    mark(idx, MRQ_NSTAGES, st);
    if (idx->prof_on) idx->prof_batches++;
    // qstats, the probe (as below), the scan, select, exact, top-k
    idx->launches += (fused ? 4 : tc_probe ? 5 : 6) - 2 + 4;
    return;
  }
  // batched forms: quantized query; the popcount kernel needs code words a power of two
  // (bits in {1,2,4,8}) up to 16, the tensor-core kernel bits <= 4 and query_bits <= 4
  const int wds = idx->words;
  const bool pop_ok = o.query_bits > 0 && wds <= BATCH_MAXW && (wds & (wds - 1)) == 0 &&
                      (idx->bits & (idx->bits - 1)) == 0 && ((d / 32) & (d / 32 - 1)) == 0 &&
                      !(wds == 16 && d == 32);
  const bool use_tc = !refine && cfg.scan == MRQ_SCAN_BATCHED_TC && tc_available() &&
                      scan_tc_supported(d, idx->bits, o.query_bits);
  // the batched scan's work items are sized for the worst case (every probed list's
  // blocks for every query): beyond the budget the pairs are scanned one by one
  const bool items_fit = ws.items_budget <= 0 ||
      (int64_t)(2 * (nq * nprobe + (nq * idx->cap_by_nprobe[nprobe]) / 32 + 1)) * 8 <=
          ws.items_budget;
  const bool batched = !refine && items_fit &&
                       (use_tc || ((cfg.scan == MRQ_SCAN_BATCHED ||
                                    cfg.scan == MRQ_SCAN_BATCHED_TC) && pop_ok));
  if (batched) {
    const int64_t np_ = nq * nprobe;
    const int nch = d / 32;
    // seed pass: each query's nearest list by the per-pair scan, whose warp top-k gives a
    // tight bound of tau_A early; the batched kernel then scans the remaining pairs
    const int first = nprobe >= 4 ? 1 : 0;
    if (first) launch_scan(sp, build_items(nq, nprobe), st, false);
    ws.lcount.reserve(nlist);
    ws.loffq.reserve(nlist);
    ws.lfill.reserve(nlist);
    ws.lqueue.reserve(np_);
    ws.icnt.reserve(nlist);
    ws.ioff.reserve(nlist);
    ws.nitems.reserve(1);
    const int64_t max_items = np_ + (nq * idx->cap_by_nprobe[nprobe]) / 32 + 1;
    ws.bitems.reserve(2 * max_items);  // int4 items, two int64 slots each
    ws.pq.reserve(np_ * sizeof(PairQ));
    ws.qplanes.reserve(np_ * o.query_bits * nch);
    if (use_tc) ws.qrow.reserve(np_ * d);
    const int blk = use_tc ? TC_SCAN_TILE : 32;
    const int group = use_tc ? TC_SCAN_GROUP : cfg.group;
    MRQ_CUDA(cudaMemsetAsync(ws.lcount.p, 0, 4 * nlist, st));
    MRQ_CUDA(cudaMemsetAsync(ws.lfill.p, 0, 4 * nlist, st));
    k_bucket_count<<<ceil_div(np_, 256), 256, 0, st>>>(ws.plist.p, np_, nprobe, first, ws.lcount.p);
    size_t tb = 0;
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, ws.lcount.p, ws.loffq.p, nlist, st));
    ws.cubtmp.reserve(tb + 16);
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(ws.cubtmp.p, tb, ws.lcount.p, ws.loffq.p, nlist, st));
    k_bucket_fill<<<ceil_div(np_, 256), 256, 0, st>>>(ws.plist.p, np_, nprobe, first, ws.loffq.p,
                                                      ws.lfill.p, ws.lqueue.p);
    k_batch_count<<<ceil_div(nlist, 256), 256, 0, st>>>(ws.lcount.p, idx->loff.p, nlist, blk, group,
                                                        ws.icnt.p);
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(nullptr, tb, ws.icnt.p, ws.ioff.p, nlist, st));
    ws.cubtmp.reserve(tb + 16);
    MRQ_CUDA(cub::DeviceScan::ExclusiveSum(ws.cubtmp.p, tb, ws.icnt.p, ws.ioff.p, nlist, st));
    k_batch_scatter<<<ceil_div(nlist, 256), 256, 0, st>>>(ws.lcount.p, ws.icnt.p, ws.ioff.p,
                                                          idx->loff.p, nlist, group,
                                                          reinterpret_cast<int4*>(ws.bitems.p),
                                                          ws.nitems.p);
    k_pair_prep<<<ceil_div(np_, 8), 256, 0, st>>>(ws.qd.p, ws.qstat.p, ws.plist.p, ws.pg.p,
                                                  idx->cent.p, np_, nprobe, d, o.query_bits,
                                                  o.eps0, o.m, reinterpret_cast<PairQ*>(ws.pq.p),
                                                  ws.qplanes.p, use_tc ? ws.qrow.p : nullptr);
    MRQ_CHECK_LAUNCH();
    if (use_tc) {
      TcScanParams tp{};
      tp.items = reinterpret_cast<const int4*>(ws.bitems.p); tp.nitems = ws.nitems.p;
      tp.lqueue = ws.lqueue.p; tp.loffq = ws.loffq.p; tp.lcount = ws.lcount.p;
      tp.pq = reinterpret_cast<const PairQ*>(ws.pq.p); tp.qrow = ws.qrow.p;
      tp.loff = idx->loff.p; tp.ploff = idx->ploff.p; tp.codes = idx->codes.p;
      tp.fadd = idx->fadd.p; tp.fres = idx->fres.p; tp.ferr = idx->ferr.p;
      tp.nprobe = nprobe; tp.k = k; tp.cap = cap;
      tp.work = ws.work.p + 2; tp.qcnt = ws.qcnt.p; tp.gtau = ws.gtau.p;
      tp.spos = ws.spos.p; tp.slb = ws.slb.p; tp.sub = ws.sub.p;
      tp.err = tc_error_word();
      // items, per list: ceil(size / 128) tiles x ceil(pairs / 64) groups, fewer than the
      // popcount form's items that bitems is sized for
      scan_tc(tp, d, idx->bits, st);
      idx->launches += 8;
    } else {
    BatchParams bp{};
    bp.items = reinterpret_cast<const int4*>(ws.bitems.p); bp.nitems = ws.nitems.p;
    bp.lqueue = ws.lqueue.p; bp.loffq = ws.loffq.p; bp.lcount = ws.lcount.p;
    bp.pq = reinterpret_cast<const PairQ*>(ws.pq.p); bp.qplanes = ws.qplanes.p;
    bp.loff = idx->loff.p; bp.ploff = idx->ploff.p; bp.codes = idx->codes.p;
    bp.fadd = idx->fadd.p; bp.fres = idx->fres.p; bp.ferr = idx->ferr.p;
    bp.d = d; bp.bits = idx->bits; bp.words = idx->words; bp.vw = idx->vw;
    bp.nprobe = nprobe; bp.k = k; bp.qbits = o.query_bits; bp.cap = cap; bp.group = cfg.group;
    bp.work = ws.work.p + 1; bp.qcnt = ws.qcnt.p; bp.gtau = ws.gtau.p;
    bp.spos = ws.spos.p; bp.slb = ws.slb.p; bp.sub = ws.sub.p;
    auto launch = [&](auto kern) {
      kern<<<num_sms() * occupancy((const void*)kern, 256, 0), 256, 0, st>>>(bp);
    };
    const int nch_ = d / 32, bits_ = idx->bits;
#define MRQ_BATCH(Wv, Nv) \
    else if (idx->words == Wv && nch_ == Nv) launch(k_scan_batched<Wv, Nv>);
    if (false) {}
    MRQ_BATCH(1, 1) MRQ_BATCH(2, 1) MRQ_BATCH(2, 2) MRQ_BATCH(4, 1) MRQ_BATCH(4, 2)
    MRQ_BATCH(4, 4) MRQ_BATCH(8, 1) MRQ_BATCH(8, 2) MRQ_BATCH(8, 4) MRQ_BATCH(8, 8)
    MRQ_BATCH(16, 2) MRQ_BATCH(16, 4) MRQ_BATCH(16, 8) MRQ_BATCH(16, 16)
    else fail(MRQ_EINVAL, "batched scan: unsupported code shape");
#undef MRQ_BATCH
    (void)bits_;
    MRQ_CHECK_LAUNCH();
    idx->launches += 8;
    }
  }
  int64_t grid_items = nq * nprobe;
  if (!batched && idx->max_list > cfg.chunk) {
    // long (Zipf-sized) lists: before their chunks start together, a seed pass over the
    // first SEED_CHUNK candidates of each query's nearest list publishes a running bound
    // (the same kernel and arithmetic, so it is a k-th smallest of true UB1 values and
    // never below tau_A); it writes no survivors -- the main scan revisits those candidates
    if (o.query_bits > 0 && !refine && k <= 128) {
      ws.sitems.reserve(nq);
      ws.nitems.reserve(2);
      k_seed_items<<<ceil_div(nq, 256), 256, 0, st>>>(nq, nprobe, ws.sitems.p, ws.nitems.p + 1);
      MRQ_CHECK_LAUNCH();
      ScanParams ss = sp;
      ss.items = ws.sitems.p;
      ss.nitems = ws.nitems.p + 1;
      ss.chunk = SEED_CHUNK;
      ss.seed = 1;
      ss.work = ws.work.p + 3;
      launch_scan(ss, nq, st, false);
      idx->launches += 2;
    }
    grid_items = build_items(nq * nprobe, 1, nq);
  }
  if (refine) {  // the pairs' quantized queries, for stage 1b
    const int64_t np_ = nq * nprobe;
    ws.pq.reserve(np_ * sizeof(PairQ));
    ws.qplanes.reserve(np_ * o.query_bits * (d / 32));
    k_pair_prep<<<ceil_div(np_, 8), 256, 0, st>>>(ws.qd.p, ws.qstat.p, ws.plist.p, ws.pg.p,
                                                  idx->cent.p, np_, nprobe, d, o.query_bits,
                                                  o.eps0, o.m, reinterpret_cast<PairQ*>(ws.pq.p),
                                                  ws.qplanes.p, nullptr);
    MRQ_CHECK_LAUNCH();
  }
  if (!batched) launch_scan(sp, grid_items, st, false);
  if (limited) {
    k_overflow<<<ceil_div(nq, 256), 256, 0, st>>>(ws.qcnt.p, nq, cap, ws.ovf_base, ws.ovf.p);
    MRQ_CHECK_LAUNCH();
    idx->launches += 1;
  }
  // 5. finalize
  mark(idx, MRQ_STAGE_TAU_A, st);
  FinParams fp{};
  fp.qd = ws.qd.p; fp.qr = ws.qr.p; fp.qstat = ws.qstat.p; fp.plist = ws.plist.p;
  fp.loff = idx->loff.p; fp.xd = idx->xd.p; fp.xr = idx->xr.p; fp.xn2 = idx->xn2.p;
  fp.ids = idx->ids.p; fp.d = d; fp.r = r; fp.nprobe = nprobe; fp.k = k; fp.mode = o.mode;
  fp.m = o.m; fp.cap = cap; fp.qcnt = ws.qcnt.p; fp.spos = ws.spos.p; fp.slb = ws.slb.p;
  fp.sub = ws.sub.p; fp.s2pos = ws.s2pos.p; fp.s2a = ws.s2a.p; fp.s2b = ws.s2b.p;
  fp.out_ids = out_ids; fp.out_d = out_d; fp.stats = stats;
  if (k <= FW_BUF) {  // phased finalize: the per-warp sort buffer holds next_pow2(k) entries
    ws.qtau.reserve(nq);
    ws.qm1.reserve(nq);
    ws.qm2.reserve(nq);
    fp.qtau = ws.qtau.p; fp.qm1 = ws.qm1.p; fp.qm2 = ws.qm2.p; fp.nq = nq;
    fp.gtau = ws.gtau.p;
    const unsigned gw = ceil_div(nq, FW_WARPS);
    // a few queries with long survivor lists (a search again of overflowed queries): each
    // query's selections run on a whole CTA and its gathers are split over several CTAs
    const unsigned fsplit =
        (nq <= 8192 && cap > 4096)
            ? (unsigned)std::min<int64_t>({ceil_div(cap, 4096), std::max<int64_t>(1, 65536 / nq),
                                           65535})
            : 1u;
    const dim3 fgrid((unsigned)nq, fsplit);
    const bool wide = fsplit > 1 && !refine;
    if (limited && ws.seed_out) {
      k_ovf_seed<<<gw, FW_WARPS * 32, 0, st>>>(fp, ws.seed_out, ws.ovf_base);
      MRQ_CHECK_LAUNCH();
      idx->launches += 1;
    }
    if (wide) k_fin_s1_wide<<<(unsigned)nq, 256, 0, st>>>(fp);
    else k_fin_s1<<<gw, FW_WARPS * 32, 0, st>>>(fp);
    MRQ_CHECK_LAUNCH();
    if (refine) {
      RefineParams rp{};
      rp.plist = ws.plist.p; rp.loff = idx->loff.p; rp.ploff = idx->ploff.p;
      rp.codes = idx->codes.p; rp.fadd = idx->fadd.p; rp.fres = idx->fres.p; rp.ferr = idx->ferr.p;
      rp.pq = reinterpret_cast<const PairQ*>(ws.pq.p); rp.qplanes = ws.qplanes.p;
      rp.qm1 = ws.qm1.p; rp.s2pos = ws.s2pos.p; rp.s2a = ws.s2a.p; rp.s2b = ws.s2b.p;
      rp.d = d; rp.bits = idx->bits; rp.words = idx->words; rp.vw = idx->vw;
      rp.nprobe = nprobe; rp.qbits = o.query_bits; rp.cap = cap;
      k_refine1b<<<(unsigned)nq, 256, (size_t)12 * nprobe, st>>>(rp);
      MRQ_CHECK_LAUNCH();
      k_fin_s1b<<<gw, FW_WARPS * 32, 0, st>>>(fp);
      MRQ_CHECK_LAUNCH();
      // S1 now sits in spos: the later phases read it from there and compact into s2pos
      std::swap(fp.spos, fp.s2pos);
      idx->launches += 3;
    }
    mark(idx, MRQ_STAGE_STAGE2, st);
    if (o.mode == MRQ_MODE_MRQ_PLUS) {
#define MRQ_S2G(NCv)                                                                   \
      (fsplit > 1 ? k_fin_stage2_g<NCv, true><<<fgrid, 256, 0, st>>>(fp)               \
                  : k_fin_stage2_g<NCv, false><<<fgrid, 256, 0, st>>>(fp))
      if (d == 32) MRQ_S2G(1);
      else if (d == 64) MRQ_S2G(2);
      else if (d == 128) MRQ_S2G(4);
      else if (d == 256) MRQ_S2G(8);
#undef MRQ_S2G
      else k_fin_stage2<<<(unsigned)nq, 256, (size_t)((d + 3) & ~3) * 4, st>>>(fp);
      MRQ_CHECK_LAUNCH();
    }
    mark(idx, MRQ_STAGE_TAU_B, st);
    if (wide && o.mode == MRQ_MODE_MRQ_PLUS) k_fin_s2_wide<<<(unsigned)nq, 256, 0, st>>>(fp);
    else k_fin_s2<<<gw, FW_WARPS * 32, 0, st>>>(fp);
    MRQ_CHECK_LAUNCH();
    idx->launches += o.mode == MRQ_MODE_MRQ_PLUS ? 2 : 1;
    mark(idx, MRQ_STAGE_EXACT, st);
    if (o.mode == MRQ_MODE_MRQ_PLUS && (r & 3) == 0) {
      // the d-part of every exact distance came out of stage 2
      const size_t esm = (size_t)std::max(r, 4) * 4;
      ensure_smem((const void*)k_fin_exact_r, esm);
      k_fin_exact_r<<<fgrid, 256, esm, st>>>(fp);
    } else {
      const size_t esm = (size_t)(((d + 3) & ~3) + r) * 4;
      ensure_smem((const void*)k_fin_exact, esm);
      k_fin_exact<<<(unsigned)nq, 256, esm, st>>>(fp);
    }
    MRQ_CHECK_LAUNCH();
    mark(idx, MRQ_STAGE_TOPK, st);
    k_fin_topk<<<gw, FW_WARPS * 32, 0, st>>>(fp);
    idx->launches += 2;  // exact, top-k (the first finalize launch is counted below)
  } else {
    size_t fsm = (size_t)((((d + 3) & ~3) + r + 3) & ~3) * sizeof(float) + FN_SORT * 8;
    ensure_smem((const void*)k_finalize, fsm);
    k_finalize<<<(unsigned)nq, FN_NT, fsm, st>>>(fp);
    for (int sidx = MRQ_STAGE_STAGE2; sidx <= MRQ_STAGE_TOPK; ++sidx) mark(idx, sidx, st);
  }
  MRQ_CHECK_LAUNCH();
  mark(idx, MRQ_NSTAGES, st);
  if (idx->prof_on) idx->prof_batches++;
  // qstats, fp32 probe distances (the tensor-core probe's operand comes from the
  // projection), select + refine (one kernel in the fused probe), scan, the first
  // finalize phase
  idx->launches += fused ? 4 : tc_probe ? 5 : 6;
}

void ensure_sq8(const mrq_index* idx, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(idx->sq_mu);
  if (idx->sq_codes.p) return;
  const int64_t n = idx->n;
  const int d = idx->d, r = idx->D - idx->d;
  DevBuf<unsigned int> mm(2 * (size_t)d);
  MRQ_CUDA(cudaMemsetAsync(mm.p, 0xff, 4 * (size_t)d, st));
  MRQ_CUDA(cudaMemsetAsync(mm.p + d, 0, 4 * (size_t)d, st));
  const int64_t rows_per = 8192;
  k_sq8_minmax<<<dim3(ceil_div(d, 32), ceil_div(n, rows_per)), 256, 0, st>>>(idx->xd.p, n, d,
                                                                            rows_per, mm.p);
  MRQ_CHECK_LAUNCH();
  DevBuf<float> lo(d), delta(d), xr2(std::max<int64_t>(n, 1));
  DevBuf<uint8_t> codes((size_t)n * d);
  k_sq8_grid<<<ceil_div(d, 256), 256, 0, st>>>(mm.p, d, lo.p, delta.p);
  MRQ_CHECK_LAUNCH();
  k_sq8_encode<<<ceil_div(n * d, 256), 256, 0, st>>>(idx->xd.p, n, d, lo.p, delta.p, codes.p);
  MRQ_CHECK_LAUNCH();
  if (r > 0) {
    k_sq8_rownorm<<<ceil_div(n, 8), 256, 0, st>>>(idx->xr.p, n, r, xr2.p);
    MRQ_CHECK_LAUNCH();
  } else {
    MRQ_CUDA(cudaMemsetAsync(xr2.p, 0, 4 * (size_t)n, st));
  }
  MRQ_CUDA(cudaStreamSynchronize(st));
  idx->sq_lo = std::move(lo);
  idx->sq_delta = std::move(delta);
  idx->sq_xr2 = std::move(xr2);
  idx->sq_codes = std::move(codes);
}

size_t batch_scratch_bytes(const mrq_index* idx, int64_t nq, int k, int nprobe) {
  const int64_t D = idx->D, d = idx->d;
  const int64_t cap = std::max<int64_t>(idx->cap_by_nprobe[nprobe], 1);
  const int64_t per_q = D * 4 * 2 + D * 4 /* bf16 hi+lo */ + 16 + (int64_t)idx->nlist * 4 +
                        nprobe * (8 + 32 + 8 * (d / 32) * 4 + 16 * 8) + 16 + cap * 24 + k * 12 + 24;
  return (size_t)(nq * per_q) + (size_t)idx->nlist * 16 + (1 << 20);
}

void estimate_one(mrq_index* idx, const float* qp, int list, const mrq_search_opts& o, float* ip,
                  float* dis, float* lb, float* ub, int32_t* idot, cudaStream_t st) {
  auto& ws = idx->ws;
  const int D = idx->D, d = idx->d, r = D - d;
  ws.qd.reserve(d);
  ws.qr.reserve(std::max(r, 1));
  ws.qstat.reserve(4);
  ws.plist.reserve(1);
  ws.pg.reserve(1);
  MRQ_CUDA(cudaMemcpyAsync(ws.qd.p, qp, 4 * d, cudaMemcpyDefault, st));
  if (r > 0) MRQ_CUDA(cudaMemcpyAsync(ws.qr.p, qp + d, 4 * r, cudaMemcpyDefault, st));
  qstats(idx, ws.qd.p, ws.qr.p, 1, ws.qstat.p, st);
  MRQ_CUDA(cudaMemcpyAsync(ws.plist.p, &list, 4, cudaMemcpyHostToDevice, st));
  k_probe_refine<<<1, 256, 0, st>>>(ws.qd.p, idx->cent.p, ws.plist.p, 1, 1, d, ws.pg.p);
  MRQ_CHECK_LAUNCH();
  ScanParams sp{};
  sp.qd = ws.qd.p; sp.qstat = ws.qstat.p; sp.plist = ws.plist.p; sp.pg = ws.pg.p;
  sp.cent = idx->cent.p; sp.loff = idx->loff.p; sp.ploff = idx->ploff.p; sp.codes = idx->codes.p;
  sp.fadd = idx->fadd.p; sp.fres = idx->fres.p; sp.ferr = idx->ferr.p;
  sp.d = d; sp.bits = idx->bits; sp.words = idx->words; sp.vw = idx->vw;
  sp.nprobe = 1; sp.k = 1; sp.qbits = o.query_bits; sp.eps0 = o.eps0; sp.m = o.m;
  sp.npairs = 1;
  sp.dbg_ip = ip; sp.dbg_dis = dis; sp.dbg_lb = lb; sp.dbg_ub = ub; sp.dbg_idot = idot;
  launch_scan(sp, 1, st, true);
  MRQ_CUDA(cudaStreamSynchronize(st));
}

}  // namespace mrq
