// Internal declarations of libmrq (GB300 / sm_103a implementation of MRQ).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <atomic>
#include <vector>

#include "../../include/mrq.h"

namespace mrq {

struct Error {
  int code;
  std::string msg;
};

[[noreturn]] inline void fail(int code, const std::string& msg) { throw Error{code, msg}; }
void set_last_error(const std::string& msg);  // message returned by mrq_last_error

#define MRQ_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      ::mrq::fail(e_ == cudaErrorMemoryAllocation ? MRQ_ENOMEM : MRQ_ECUDA,              \
                  std::string(#call) + " -> " + cudaGetErrorString(e_) + " (" __FILE__ ")"); \
  } while (0)

#define MRQ_CHECK_LAUNCH() MRQ_CUDA(cudaGetLastError())

#define MRQ_REQUIRE(cond, msg)                      \
  do {                                              \
    if (!(cond)) ::mrq::fail(MRQ_EINVAL, (msg));    \
  } while (0)

// Owning device buffer (cudaMalloc / cudaFree).
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  void alloc(size_t count) {
    release();
    if (count == 0) return;
    MRQ_CUDA(cudaMalloc(&p, count * sizeof(T)));
    n = count;
  }
  // grow-only reallocation (contents are not preserved)
  void reserve(size_t count) {
    if (count > n) alloc(count);
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  T* get() const { return p; }
};

// Process-wide count of search-scratch reallocations: a captured search graph holds the
// addresses of the scratch it was captured with, so it is captured again once this moves.
inline std::atomic<uint64_t> g_ws_epoch{0};

// a DevBuf of the search scratch: its growth moves g_ws_epoch
template <class T>
struct WsBuf : DevBuf<T> {
  void reserve(size_t count) {
    if (count > this->n) {
      this->alloc(count);
      g_ws_epoch.fetch_add(1);
    }
  }
};

// Per-index search scratch, grown on demand and reused across calls.
struct Workspace {
  WsBuf<float> q;         // nq x D staged queries (host inputs)
  WsBuf<float> qd, qr;    // projected queries
  WsBuf<float> qstat;     // nq x 4: |q_r|^2, sigma, |q_p|^2, unused
  WsBuf<float> pqq;       // nq x d: q_d' R, the OPQ-rotated query (MR-PQ)
  // optimistic survivor region: with cap_limit > 0 every query's stage-1 region holds at
  // most cap_limit entries; a query whose survivors overflow it is listed in ovf
  // ([0] = count, then query indices offset by ovf_base) and searched again in full
  int64_t cap_limit = 0;
  int64_t ovf_base = 0;
  WsBuf<int> ovf;
  int64_t items_budget = 0;  // bytes the batched scan's work items may take (0 = any)
  // per row of the call: the bound an overflowed query's search again starts from
  // (written through seed_out while the call's batches run; read through seed_tau and
  // seed_rows, the batch's rows, by the searches again)
  WsBuf<float> ovf_tau;
  float* seed_out = nullptr;
  const float* seed_tau = nullptr;
  const int* seed_rows = nullptr;
  WsBuf<__nv_bfloat16> qbf;  // nq x D bf16 hi/lo split queries (tensor-core projection)
  WsBuf<uint8_t> q8;          // nq x D row-scaled e4m3 queries (FP8 projection)
  WsBuf<float> q8s;           // their row scales
  WsBuf<__nv_bfloat16> qbf2;  // nq x d bf16 hi/lo split q_d' (tensor-core probe operand)
  WsBuf<float> gmat;      // nq x nlist probe distances
  WsBuf<unsigned long long> ppart;  // nq x tiles x nprobe fused probe candidates
  WsBuf<int32_t> plist;   // nq x nprobe probed list ids
  WsBuf<float> pg;        // nq x nprobe |q_d - c|^2 of the probed lists
  WsBuf<uint32_t> qcnt;   // nq survivor counters
  WsBuf<uint32_t> gtau;   // nq running stage-1 thresholds (orderable keys)
  WsBuf<int32_t> spos;    // nq x cap survivor positions
  WsBuf<float> slb, sub;  // nq x cap stage-1 bounds of the survivors
  WsBuf<float> s2a, s2b;  // nq x cap stage-2 scratch
  WsBuf<int32_t> s2pos;   // nq x cap
  WsBuf<int64_t> oids;    // nq x k staged results
  WsBuf<float> odist;
  WsBuf<int64_t> stats;   // nq x 3
  WsBuf<uint32_t> work;   // work-queue counters
  WsBuf<float> qtau;      // nq: tau_A per query (phased finalize)
  WsBuf<int> qm1, qm2;    // nq: stage-1 / stage-2 survivor counts
  WsBuf<int> ccnt, coff, nitems;  // long-list chunking: per-pair chunk counts, offsets
  WsBuf<int64_t> items;   // (pair << 32 | chunk) scan work items
  WsBuf<int64_t> sitems;  // the seed pass's items (each query's nearest list, chunk 0)
  WsBuf<uint8_t> cubtmp;  // CUB scan scratch
  // list-major batched scan
  WsBuf<int32_t> lcount, loffq, lfill, lqueue;  // per-list buckets of (query, list) pairs
  WsBuf<int32_t> icnt, ioff;              // work items per list and their offsets
  WsBuf<int64_t> bitems;                  // int4 work items (list, block, group)
  WsBuf<uint8_t> pq;                      // per-pair query scalars
  WsBuf<uint8_t> qrow;                    // per-pair query codes as e4m3 bytes (tensor-core scan)
  WsBuf<uint32_t> qplanes;                // per-pair quantized query bit planes
};

}  // namespace mrq

namespace mrq {
// scan configuration the autotuner chooses between
struct ScanConfig {
  int scan;   // MRQ_SCAN_PAIRS, MRQ_SCAN_BATCHED or MRQ_SCAN_BATCHED_TC
  int chunk;  // candidates per work item of a long list (per-pair scan)
  int group;  // queries per work item (batched scan), <= 16
};

// per-(query, list) scalars of the batched scans (Algorithm 2: normalise, quantize)
struct __align__(16) PairQ {
  float sg, a0, e0, em;  // sqrt(g), g + |q_r|^2, eps0*sqrt(g), m*sigma
  float ql, qdelta;      // q' ~ ql + qdelta * qbar
  int qsum, q;           // q: the pair's query
};

// the tensor-core batched scan: a work item is (list j, tile of 128 candidates, group
// of up to 128 pairs probing j); the integer code dots of the tile against the group's
// quantized queries are one e4m3 MMA chain (levels and query codes 0..15 are exact)
struct TcScanParams {
  const int4* items;     // (j, tile, group)
  const int* nitems;
  const int* lqueue;     // pairs bucketed by list
  const int* loffq;      // bucket offsets
  const int* lcount;
  const PairQ* pq;
  const uint8_t* qrow;   // per pair: d query codes as e4m3 bytes
  const int64_t* loff;
  const int64_t* ploff;
  const uint32_t* codes;
  const float* fadd;
  const float* fres;
  const float* ferr;
  int nprobe, k;
  int64_t cap;
  unsigned int* work;    // item counter (zero before the launch)
  unsigned int* qcnt;
  unsigned int* gtau;
  int32_t* spos;
  float* slb;
  float* sub;
  int* err;
};
constexpr int TC_SCAN_TILE = 128;  // candidates per item
constexpr int TC_SCAN_GROUP = 128;  // queries per item (MMA N)
// whether the tensor-core scan has a kernel for this code shape (exact fp32 sums too)
bool scan_tc_supported(int d, int bits, int qbits);
// persistent launch; the kernel pulls items from p.work until *p.nitems
void scan_tc(const TcScanParams& p, int d, int bits, cudaStream_t st);
}  // namespace mrq

struct mrq_index {
  int64_t n = 0;
  int D = 0, d = 0, bits = 1, nlist = 0;
  int device = 0;
  int words = 0;   // 32-bit code words per vector = bits * d / 32
  int vw = 1;      // words per vectorised load (1, 2 or 4)
  int64_t np = 0;  // padded vector count (every list rounded up to 32)
  int64_t max_list = 0;
  std::vector<int64_t> h_loff, h_ploff;
  std::vector<int64_t> cap_by_nprobe;  // sum of the nprobe largest list sizes

  mrq::DevBuf<float> mu, lam, W;  // D, D, D x D
  mrq::DevBuf<__nv_bfloat16> W2;          // bf16 split of W: rows [0,D) hi, [D,2D) lo
  mrq::DevBuf<uint8_t> W8;                // row-scaled e4m3 W (D x D; D % 16 == 0 only)
  mrq::DevBuf<float> W8s;                 // its row scales
  mrq::DevBuf<__nv_bfloat16> cent2;       // bf16 split of the centroids: [0,nlist) hi, then lo
  mrq::DevBuf<float> cent, cent_n2;       // nlist x d (rotated frame), nlist
  mrq::DevBuf<int64_t> loff, ploff;       // nlist + 1
  mrq::DevBuf<int64_t> ids;               // n, list-major
  mrq::DevBuf<uint32_t> codes;            // padded bit-plane layout
  mrq::DevBuf<float> fadd, fres, ferr;    // padded
  // padded factors of the sign plane (the 1-bit code of o'), held when bits > 1: the
  // first level of the 1 bit + refinement scan
  mrq::DevBuf<float> fres1, ferr1;
  // MR-SQ (MRQ_MODE_SQ8), made on first use from xd / xr: 8-bit codes of x_d' (n x d,
  // list-major), the per-dimension grid (lo, delta) and |x_r|^2 (n)
  mutable std::mutex sq_mu;
  mutable mrq::DevBuf<uint8_t> sq_codes;
  mutable mrq::DevBuf<float> sq_lo, sq_delta, sq_xr2;
  // MR-PQ (MRQ_MODE_PQ), from mrq_pq_train or the index file: the OPQ rotation R and its
  // transpose (d x d), codebooks (pq_M x pq_K x d/pq_M, subspace-major), codes (n x pq_M,
  // list-major) and |x_r|^2 (n)
  int pq_M = 0, pq_K = 0;
  mrq::DevBuf<float> pq_R, pq_Rt, pq_C, pq_xr2;
  mrq::DevBuf<uint8_t> pq_codes;
  mrq::DevBuf<float> xd, xr, xn2;         // list-major, unpadded
  mrq::Workspace ws;
  mrq::Workspace ws_redo;  // searches again the queries whose survivors overflowed
  int64_t last_redo = 0;   // queries the last search searched again
  int64_t last_nq = 0;
  mutable bool last_stats_dev = false;
  // autotuned scan configurations, keyed by (k class, nprobe, query bits, scan_variant)
  std::mutex tune_mu;
  std::map<std::tuple<int, int, int, int>, mrq::ScanConfig> tuned;  // last search's counters still in ws.stats (device)
  mutable std::vector<int64_t> last_stats;        // nq x 3 host copy of the last search's counters
  // profiling of the last search: MRQ_NSTAGES + 1 events per batch
  std::vector<cudaEvent_t> prof_ev;
  int prof_batches = 0;
  bool prof_on = false;
  double prof_ms[MRQ_NSTAGES] = {0};
  int64_t launches = 0;
  // captured search graph (device-resident calls with identical arguments)
  struct GraphKey {
    const void* q;
    void* ids;
    void* dists;
    int64_t nq;
    int k, nprobe, mode, precision, query_bits, batched, refine, rerank;
    float eps0, m;
    int64_t region;
    bool operator==(const GraphKey& o) const {
      return q == o.q && ids == o.ids && dists == o.dists && nq == o.nq && k == o.k &&
             region == o.region &&
             nprobe == o.nprobe && mode == o.mode && precision == o.precision &&
             query_bits == o.query_bits && batched == o.batched && refine == o.refine &&
             rerank == o.rerank &&
             eps0 == o.eps0 && m == o.m;
    }
  };
  bool graph_valid = false;
  GraphKey graph_key{};
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t graph_stream = nullptr;
  cudaEvent_t graph_ev[2] = {nullptr, nullptr};
  int64_t graph_launches = 0;
  uint64_t graph_epoch = 0;  // g_ws_epoch when the graph was captured
  ~mrq_index() {
    for (auto e : prof_ev) cudaEventDestroy(e);
    if (graph_exec) cudaGraphExecDestroy(graph_exec);
    if (graph_stream) cudaStreamDestroy(graph_stream);
    for (auto e : graph_ev)
      if (e) cudaEventDestroy(e);
  }
};

namespace mrq {

// ---- build-side launchers (build.cu) ----
void build_index(mrq_index* idx, const float* base_dev, const mrq_build_opts& o, cudaStream_t st);
// code levels (n x d, u8, list-major) + unpadded factors -> padded device layout
// fres1_dev / ferr1_dev: the sign plane's factors (bits > 1), or NULL
void finalize_layout(mrq_index* idx, const uint8_t* levels_dev, const float* fadd_dev,
                     const float* fres_dev, const float* ferr_dev, cudaStream_t st,
                     const float* fres1_dev = nullptr, const float* ferr1_dev = nullptr);
void export_levels(const mrq_index* idx, uint8_t* levels_dev, cudaStream_t st);
void export_padded(const mrq_index* idx, const float* padded_dev, float* out_dev, cudaStream_t st);
void make_bf16_split(mrq_index* idx, cudaStream_t st);
void compute_centroid_norms(mrq_index* idx, cudaStream_t st);

// ---- generic float32 tile kernels (gemm_f32.cu) ----
// C[M x N] = (A - a_shift) * B^T with A (M x K, lda), B (N x K, ldb).
// Columns [0, split) go to out0 (ld0), [split, N) to out1 (ld1).
void gemm_nt_f32(const float* A, int lda, const float* a_shift, const float* B, int ldb,
                 int M, int N, int K, float* out0, int ld0, float* out1, int ld1, int split,
                 cudaStream_t st);
// D[M x N] = sum_k (A[m,k] - B[n,k])^2 stored row-major (ldd).
void sqdist_f32(const float* A, int lda, const float* B, int ldb, int M, int N, int K,
                float* Dout, int ldd, cudaStream_t st);
// argmin_n sum_k (A[m,k]-B[n,k])^2 -> out[m] (ties to the lower n).
void nearest_f32(const float* A, int lda, const float* B, int ldb, int M, int N, int K,
                 unsigned long long* scratch, int32_t* out, cudaStream_t st);

// ---- tensor-core GEMMs (gemm_tc.cu) ----
bool tc_available();
void project_noalloc(mrq_index* idx, const float* q, int64_t nq, int precision, float* qp,
                     cudaStream_t st);  // static scratch only, no allocation
// MR-PQ (pq.cu): OPQ training on the GPU, or an OPQ given in host memory
void pq_train(mrq_index* idx, int M, int K, int opq_iters, int km_iters, const int64_t* init_rows,
              cudaStream_t st);
void pq_install(mrq_index* idx, int M, int K, const float* R, const float* C,
                const uint8_t* codes, cudaStream_t st);
// eigenvalues (descending) and eigenvectors (rows of V) of a symmetric D x D float64 matrix
void eigen_sym(const double* Cdev, int D, std::vector<double>& lam_host, DevBuf<double>& V_dev,
               cudaStream_t st);
// list-sharded search (shard.cu): the partition plan and the merge of per-shard answers
void shard_plan(const int64_t* sizes, int nlist, int nshards, int32_t* owner);
void merge_topk(const int64_t* ids, const float* dists, int nparts, int64_t nq, int k,
                cudaStream_t st, int64_t* out_ids, float* out_dists);
int* tc_error_word();    // device word the tensor-core kernels set when a wait gives up
int* tc_error_mirror();  // page-locked host int for reading it back asynchronously
int tc_check_error();  // nonzero if a bounded wait in a tensor-core kernel gave up
// probe_bf (optional, M x d bf16, twice with split3): the projection's epilogue also
// writes the probe's split operand of q_d', so the probe can skip its split (presplit)
// row-scaled e4m3 rows of X (centred by shift when given) and their scales
void quantize_rows_fp8(const float* X, int M, int K, int ld, const float* shift, uint8_t* out,
                       float* scale, cudaStream_t st);
// [q_d' | q_r] = W (q - mu) from e4m3 operands (MRQ_PREC_FP8); err: the pipeline error word
// (NULL: the library's)
void project_fp8(const float* Q, const float* mu, const uint8_t* W8, const float* W8s, int M,
                 int D, int d, uint8_t* q8, float* q8s, float* qd, int ldd, float* qr, int ldr,
                 cudaStream_t st, __nv_bfloat16* probe_bf, int* err);
// returns the kernels launched: 1 (the fused projection, which centres and splits the
// float32 queries itself) or 2 (split kernel + GEMM, for unaligned rows)
int project_tc(const float* Q, const float* mu, const __nv_bfloat16* W2, int M, int D, int d,
               bool split3, __nv_bfloat16* qbf, float* qd, float* qr, cudaStream_t st,
               __nv_bfloat16* probe_bf = nullptr);
// the fused projection alone (false: operands it cannot take, nothing launched)
bool project_fused(const float* Q, const float* mu, const __nv_bfloat16* W2, int M, int D, int d,
                   bool split3, float* qd, int ldd, float* qr, int ldr, __nv_bfloat16* probe_bf,
                   int* err, cudaStream_t st);
void probe_tc(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
              int M, int nlist, int d, bool split3, __nv_bfloat16* qbf, float* gmat,
              cudaStream_t st, bool presplit = false);
// candidate lists per row that probe_tc_topk writes (its part array holds M x parts x nsel
// keys)
int probe_tc_parts(int nlist);
int probe_tc_topk(const float* qd, const float* qstat, const __nv_bfloat16* C2, const float* cn2,
                  int M, int nlist, int d, bool split3, int nsel, __nv_bfloat16* qbf,
                  unsigned long long* part, cudaStream_t st, bool presplit = false);

// ---- search (search.cu) ----
// One batch of the query path on stream st with scratch ws (one Workspace per
// concurrently running batch); marks/launch counts go to idx.
void search_batch(mrq_index* idx, Workspace& ws, const float* q_dev, int64_t nq, int k,
                  int nprobe, const mrq_search_opts& o, int64_t* ids_dev, float* dists_dev,
                  int64_t* stats_dev, cudaStream_t st);
// the optimistic survivor region's second search: rows of the queries gathered, and the
// answers and counters scattered back to their rows (device buffers; out_ids NULL: counters only)
void gather_query_rows(const float* src, int D, const int* rows, int64_t n, float* dst,
                       cudaStream_t st);
void scatter_answers(const int64_t* ids, const float* d, const int64_t* stats, int k, const int* rows,
                     int64_t n, int64_t* out_ids, float* out_d, int64_t* out_stats, cudaStream_t st);
// the projection of nq device queries at a precision; returns the kernels launched
int project_batch(mrq_index* idx, Workspace& ws, const float* q_dev, int64_t nq, int precision,
                  float* qd, float* qr, cudaStream_t st, __nv_bfloat16* probe_bf = nullptr);
// MR-SQ arrays of the index (made once, on the given stream, then synchronised)
void ensure_sq8(const mrq_index* idx, cudaStream_t st);

// the search runs the 1 bit + refinement stage 1 (bits > 1 and refine = 1)
constexpr int REFINE_MAX_NPROBE = 4096;  // stage 1b's probe table: 12 B of shared memory each
inline bool refine_active(const mrq_index* idx, const mrq_search_opts& o) {
  return o.refine != 0 && idx->bits > 1 && o.mode != MRQ_MODE_SQ8 && o.mode != MRQ_MODE_PQ;
}

// which scan a search runs, for the autotuner's key: 0 one-stage, 1 refinement, 2 MR-SQ
inline int scan_variant(const mrq_index* idx, const mrq_search_opts& o) {
  return o.mode == MRQ_MODE_SQ8 ? 2 : o.mode == MRQ_MODE_PQ ? 3 : refine_active(idx, o) ? 1 : 0;
}

// the scan configuration a search uses; a ScopedScanConfig forces one on this thread
ScanConfig scan_config(mrq_index* idx, const mrq_search_opts& o, int64_t nq, int k, int nprobe);
int scan_kclass(int k);
struct ScopedScanConfig {
  explicit ScopedScanConfig(const ScanConfig* c);
  ~ScopedScanConfig();
  const ScanConfig* prev;
};
// device bytes of scratch one batch of nq queries needs (for admission control)
size_t batch_scratch_bytes(const mrq_index* idx, int64_t nq, int k, int nprobe);
void estimate_one(mrq_index* idx, const float* qp_dev, int list, const mrq_search_opts& o,
                  float* ip, float* dis, float* lb, float* ub, int32_t* idot, cudaStream_t st);

// orderable 32-bit key of a float (monotone: a < b  <=>  key(a) < key(b))
__host__ __device__ inline uint32_t fkey(float f) {
#ifdef __CUDA_ARCH__
  uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__host__ __device__ inline float fkey_inv(uint32_t k) {
  uint32_t u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
#ifdef __CUDA_ARCH__
  return __uint_as_float(u);
#else
  float f;
  memcpy(&f, &u, 4);
  return f;
#endif
}

inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

// Raise a kernel's dynamic shared-memory limit only when a launch needs more than
// already granted (host-side cache per kernel; avoids one driver call per launch).
void ensure_smem(const void* kernel, size_t bytes);
// Resident CTAs per SM of a kernel at a block size / shared-memory size (cached).
int occupancy(const void* kernel, int threads, size_t smem);

}  // namespace mrq
