// List-sharded search (Section 5, distributed deployment): the partition plan of the
// IVF lists over shards and the merge of the shards' answers.  The shard index itself
// is made in api.cu (it reuses the index file's canonical arrays).
#include <algorithm>
#include <limits>
#include <numeric>

#include "common.cuh"

namespace mrq {

namespace {
// device (or managed) memory; host memory, and every pointer when no GPU is present, is not
bool device_memory(const void* p) {
  cudaPointerAttributes a{};
  if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

// Lists in decreasing size (ties: lower id first), each to the shard holding the fewest
// vectors so far (ties: lower shard): a longest-processing-time split, which keeps the
// shards' vector counts within one list size of each other.
void shard_plan(const int64_t* sizes, int nlist, int nshards, int32_t* owner) {
  MRQ_REQUIRE(sizes && owner, "NULL argument");
  MRQ_REQUIRE(nlist >= 1 && nshards >= 1 && nshards <= nlist, "need 1 <= nshards <= nlist");
  std::vector<int> order(nlist);
  std::iota(order.begin(), order.end(), 0);
  for (int j = 0; j < nlist; ++j) MRQ_REQUIRE(sizes[j] >= 0, "negative list size");
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return sizes[a] > sizes[b]; });
  std::vector<int64_t> load(nshards, 0);
  for (int j : order) {
    int best = 0;
    for (int s = 1; s < nshards; ++s)
      if (load[s] < load[best]) best = s;
    owner[j] = best;
    load[best] += sizes[j];
  }
}

namespace {

// (dist, id) order of the answers; an id < 0 (padding) sorts after every real entry
__device__ __forceinline__ bool merge_less(float da, long long ia, float db, long long ib) {
  const bool pa = ia < 0, pb = ib < 0;
  if (pa != pb) return pb;
  if (pa) return false;
  if (da != db) return da < db;
  return ia < ib;
}

// one warp per query: a k-way merge of the parts' sorted rows; lane l owns parts l and
// l + 32, and each step moves the smallest head to the output
__global__ void k_merge_topk(const int64_t* __restrict__ ids, const float* __restrict__ dists,
                             int nparts, int64_t nq, int k, int64_t* __restrict__ out_ids,
                             float* __restrict__ out_d) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (q >= nq) return;
  int cur[2] = {0, 0};
  auto head = [&](int s, float& dv, long long& iv) {
    const int part = lane + 32 * s;
    if (part < nparts && cur[s] < k) {
      const int64_t at = ((int64_t)part * nq + q) * k + cur[s];
      dv = dists[at];
      iv = (long long)ids[at];
    } else {
      dv = __int_as_float(0x7f800000);
      iv = -1;
    }
  };
  for (int o = 0; o < k; ++o) {
    float bd;
    long long bi;
    int bs = 0;
    head(0, bd, bi);
    {
      float d1;
      long long i1;
      head(1, d1, i1);
      if (merge_less(d1, i1, bd, bi)) { bd = d1; bi = i1; bs = 1; }
    }
    int bl = lane;
#pragma unroll
    for (int off = 16; off; off >>= 1) {
      const float od = __shfl_xor_sync(0xffffffffu, bd, off);
      const long long oi = __shfl_xor_sync(0xffffffffu, bi, off);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
      const int os = __shfl_xor_sync(0xffffffffu, bs, off);
      if (merge_less(od, oi, bd, bi) || (!merge_less(bd, bi, od, oi) && ol < bl)) {
        bd = od; bi = oi; bl = ol; bs = os;
      }
    }
    if (lane == 0) {
      out_ids[q * k + o] = bi < 0 ? -1 : (int64_t)bi;
      out_d[q * k + o] = bi < 0 ? __int_as_float(0x7f800000) : bd;
    }
    if (bi >= 0 && lane == bl) cur[bs] += 1;
  }
}

}  // namespace

void merge_topk(const int64_t* ids, const float* dists, int nparts, int64_t nq, int k,
                cudaStream_t st, int64_t* out_ids, float* out_dists) {
  MRQ_REQUIRE(ids && dists && out_ids && out_dists, "NULL argument");
  MRQ_REQUIRE(nparts >= 1 && nparts <= 64, "nparts must be in [1, 64]");
  MRQ_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
  MRQ_REQUIRE(nq >= 0, "nq must be >= 0");
  const int dev = (int)device_memory(ids) + (int)device_memory(dists) +
                  (int)device_memory(out_ids) + (int)device_memory(out_dists);
  MRQ_REQUIRE(dev == 0 || dev == 4, "ids, dists and the outputs must all be host or all device memory");
  if (nq == 0) return;
  if (dev == 4) {
    const unsigned blocks = (unsigned)((nq + 7) / 8);
    k_merge_topk<<<blocks, 256, 0, st>>>(ids, dists, nparts, nq, k, out_ids, out_dists);
    MRQ_CHECK_LAUNCH();
    MRQ_CUDA(cudaStreamSynchronize(st));
    return;
  }
  // host: every valid entry of the query, ordered by (dist, id), the k first kept
  std::vector<std::pair<float, int64_t>> all;
  for (int64_t q = 0; q < nq; ++q) {
    all.clear();
    for (int p = 0; p < nparts; ++p)
      for (int t = 0; t < k; ++t) {
        const int64_t at = ((int64_t)p * nq + q) * k + t;
        if (ids[at] >= 0) all.emplace_back(dists[at], ids[at]);
      }
    const size_t keep = std::min<size_t>(all.size(), (size_t)k);
    std::partial_sort(all.begin(), all.begin() + keep, all.end());
    for (int t = 0; t < k; ++t) {
      const bool ok = (size_t)t < keep;
      out_ids[q * k + t] = ok ? all[t].second : -1;
      out_dists[q * k + t] = ok ? all[t].first : std::numeric_limits<float>::infinity();
    }
  }
}

}  // namespace mrq
