/*
 * mrq.h — C ABI of the GB300 (sm_103a) implementation of MRQ, the
 * projection-plus-quantization approximate k-NN method of arXiv 2411.06158
 * ("Quantization Meets Projection").
 *
 * Problem (Section 2.1): given n base vectors in R^D and a query q, return the
 * k base vectors closest to q under squared Euclidean distance.  MRQ (Sections
 * 4-5) rotates every vector into its PCA basis, quantizes only the leading d
 * coordinates (RaBitQ-style codes, B bits per coordinate), summarises the
 * remaining D-d coordinates by their norm and variance, and searches an IVF
 * index in three stages: a code-based estimate with error bounds (Eq. 4, Eq. 5,
 * Eq. 6), a projected-distance check (Eq. 7), and an exact rerank.
 *
 * Conventions for every call:
 *  - Return value: 0 on success, a negative MRQ_E* code on error; then
 *    mrq_last_error() returns a message for the calling thread.  No call throws.
 *  - Real arrays are row-major float32; ids are int64.  Distances are squared L2.
 *  - A pointer argument may be host or device memory (CUDA unified addressing
 *    tells them apart); the caller owns it and it is only read/written during
 *    the call (the call synchronises its stream before returning).
 *  - All device work runs on the current CUDA device, on the stream given in
 *    the options (NULL = the legacy default stream).
 *  - An index is not thread-safe: serialise calls that share one index.
 */
#ifndef MRQ_H
#define MRQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define MRQ_OK 0
#define MRQ_EINVAL (-1)    /* an argument is out of range (message says which) */
#define MRQ_ENOMEM (-2)    /* device or host allocation failed */
#define MRQ_ECUDA (-3)     /* a CUDA runtime/driver call failed */
#define MRQ_EFORMAT (-4)   /* an index file is malformed or has another version */
#define MRQ_EIO (-5)       /* a file could not be opened, read or written */
#define MRQ_ETIMEDOUT (-6) /* a bounded device-side wait gave up */

/* search modes (Section 6.1, algorithm list) */
#define MRQ_MODE_MRQ 0      /* IVF-MRQ: stage 1 then exact rerank (no stage 2) */
#define MRQ_MODE_MRQ_PLUS 1 /* IVF-MRQ+: stage 1, stage 2 (Eq. 7), exact rerank */
#define MRQ_MODE_SQ8 2      /* MR-SQ (Appendix A.2, Exp-5): 8-bit scalar quantization of
                               the projected lead coordinates x_d' (per dimension, 256 levels
                               from the base's min to max, round to nearest) instead of the
                               RaBitQ code; estimate |q_d' - x_hat|^2 + |x_r|^2 + |q_r|^2; the
                               `rerank` smallest estimates (ties by id) are reranked exactly.
                               No error bound: eps0, m, query_bits, batched and refine are
                               ignored.  The codes are made from the index's x_d' on first use
                               (n * d bytes, not saved).  k <= 128. */
#define MRQ_MODE_PQ 3       /* MR-PQ (Appendix A.2, Exp-5): optimized product quantization
                               of x_d' (an orthogonal R, M subspaces of d/M coordinates of
                               x_d' R, K centroids each) instead of the RaBitQ code; estimate
                               sum_m |(q_d' R)_m - C[m][code_m]|^2 + |x_r|^2 + |q_r|^2 from a
                               per-query lookup table; the `rerank` smallest estimates (ties
                               by id) are reranked exactly.  No error bound (as MRQ_MODE_SQ8).
                               Needs an OPQ: mrq_pq_train, or the PQR_/PQC_/PQK_ sections of
                               an index file.  k <= 128. */

/* query-projection precision (the first step of Algorithm 2) */
#define MRQ_PREC_FP32 0   /* float32 CUDA-core GEMM */
#define MRQ_PREC_BF16 1   /* one bf16 tensor-core product, fp32 accumulate */
#define MRQ_PREC_BF16X3 2 /* split hi+lo bf16: hi*hi + hi*lo + lo*hi, fp32 accumulate */
#define MRQ_PREC_FP8 3    /* row-scaled e4m3: each centred query row and each row of W scaled
                             so that its largest magnitude is 448, one kind::f8f6f4 product,
                             fp32 accumulate, the two row scales applied in the epilogue (the
                             probe then runs in bf16 on the projected q_d').  Needs D % 16 == 0 */

typedef struct mrq_index mrq_index; /* opaque; owned by the library */

typedef struct {
  uint64_t seed;                /* seed of the library's own draws (0 = 1) */
  int kmeans_iters;             /* Lloyd iterations (Algorithm 1, IVF step); default 20 */
  const float* init_centroids;  /* nlist x D raw-space initial centroids, or NULL */
  const int64_t* init_ids;      /* nlist base rows used as initial centroids, or NULL */
  const double* rotation_gauss; /* d x d Gaussian draw behind P_r (Algorithm 1), or NULL */
  double auto_d_variance;       /* with d = 0: the fraction of the total PCA variance the
                                   chosen d must hold (Eq. 8); default 0.8 */
  const int64_t* pca_rows;      /* host array of pca_n base rows (each in [0, n)) whose mean
                                   and 1/pca_n covariance define the PCA and the residual
                                   variances instead of the whole base: the sampled global
                                   statistics Section 5 suggests when the data is spread over
                                   many machines; every row is still projected, clustered and
                                   encoded.  NULL (default) = all rows */
  int64_t pca_n;                /* rows in pca_rows, >= 2 when pca_rows is given */
} mrq_build_opts;

typedef struct {
  float eps0;       /* Eq. 5 confidence parameter; default 1.9 */
  float m;          /* Chebyshev multiplier of the residual bound (Eq. 6); default 4 */
  int mode;         /* MRQ_MODE_*; default MRQ_MODE_MRQ_PLUS */
  int precision;    /* MRQ_PREC_*; default MRQ_PREC_FP32 */
  int query_bits;   /* 0 = float32 query in the scan; 1..8 = scalar-quantized query */
  int batched;      /* MRQ_SCAN_PAIRS (0): one work item per (query, list);
                       MRQ_SCAN_BATCHED (1): list-major batched scan;
                       MRQ_SCAN_BATCHED_TC (3): list-major batched scan whose code dots
                       are tensor-core MMAs (bits <= 4, query_bits 1..4; others fall
                       back to MRQ_SCAN_BATCHED);
                       MRQ_SCAN_AUTO (2): the configuration mrq_autotune chose for this
                       (k, nprobe, query_bits), else batched when nq * nprobe / nlist >= 16 */
  int profile;      /* 1 = record CUDA events around each stage (see mrq_last_search_profile) */
  int graph;        /* 1 = replay a captured CUDA graph when queries, ids and dists are device
                       memory or page-locked host memory (the copies become graph nodes) and
                       every argument equals the previous graph call's (the first such call
                       runs normally, then captures; a call after the library's search
                       scratch has grown captures again); ignored with profile = 1 */
  int refine;       /* 1 = "1 bit + refinement" stage 1 for codes of bits > 1: the sign plane
                       of every code (the 1-bit code of o', with its own Eq. 4 / Eq. 5
                       factors) is scanned first, tau_A' = k-th smallest of its upper bounds,
                       S1a = {LB1a <= tau_A'}; the full B-bit estimate is then computed for
                       S1a only, tau_A = min(tau_A', k-th smallest UB1b over S1a),
                       S1 = {i in S1a : LB1b <= tau_A}.  Needs query_bits >= 1, k <= 128 and
                       an index holding the sign-plane factors (built by this library, or a
                       file with FRE1/FER1 sections); the scan then runs pair by pair
                       (batched is ignored).  With bits = 1 it changes nothing.  Default 0 */
  int rerank;       /* MRQ_MODE_SQ8 / MRQ_MODE_PQ: the rerank range R, k <= R <= 65536;
                       default 500 */
  void* cuda_stream;/* cudaStream_t, or NULL */
  int64_t survivor_region; /* MRQ / MRQ+ modes: entries of each query's stage-1 survivor
                       region.  0 (default) = every candidate of the nprobe largest lists
                       when that fits the memory budget for the batch, else the largest
                       region that does (at least 8192).  A query whose survivors overflow
                       its region is searched again with the full region after the batch,
                       so the answer does not depend on it; mrq_last_search_stats still
                       reports its counters */
} mrq_search_opts;

#define MRQ_SCAN_PAIRS 0
#define MRQ_SCAN_BATCHED 1
#define MRQ_SCAN_AUTO 2
#define MRQ_SCAN_BATCHED_TC 3

/* stages reported by mrq_last_search_profile */
#define MRQ_STAGE_PROJECT 0  /* query projection GEMM (Algorithm 2, rotate step) */
#define MRQ_STAGE_QSTATS 1   /* |q_r|^2, sigma (Eq. 6), |q_p|^2 */
#define MRQ_STAGE_PROBE 2    /* centroid distances */
#define MRQ_STAGE_SELECT 3   /* top-nprobe selection */
#define MRQ_STAGE_SCAN 4     /* stage-1 code scan, bounds and survivor compaction */
#define MRQ_STAGE_TAU_A 5    /* tau_A and stage-1 survivors (the whole finalize when k > 64) */
#define MRQ_STAGE_STAGE2 6   /* stage 2 (Eq. 7) gathers */
#define MRQ_STAGE_TAU_B 7    /* tau_B and stage-2 survivors */
#define MRQ_STAGE_EXACT 8    /* exact-distance gathers */
#define MRQ_STAGE_TOPK 9     /* top-k by (distance, id) */
#define MRQ_NSTAGES 10

typedef struct {
  int64_t n;
  int D, d, bits, nlist;
  int64_t max_list;     /* largest list size */
  int64_t device_bytes; /* device memory held by the index (its arrays, including the
                           MR-SQ codes once made and the OPQ; not the search workspace) */
  int pq_M, pq_K;       /* OPQ subspaces and centroids per subspace (0, 0: none) */
} mrq_index_info_t;

#define MRQ_MAX_D 1024 /* largest quantized dimension d */

/* Fill *opt with the defaults listed above. */
void mrq_build_opts_default(mrq_build_opts* opt);
void mrq_search_opts_default(mrq_search_opts* opt);

/*
 * Build an IVF-MRQ index on the GPU (Algorithm 1).
 *  base: n x D float32 (host or device).  d: number of leading PCA coordinates
 *  that are quantized, 32 <= d <= min(D, MRQ_MAX_D), d % 32 == 0; d = D leaves no
 *  residual tail (sigma = 0, Eq. 6), i.e. IVF-RaBitQ (Section 6.1).  d = 0 chooses d
 *  by the rule of Eq. 8 once the PCA spectrum is known: the smallest power of two
 *  >= 128 whose leading coordinates hold opt->auto_d_variance of the total variance
 *  (eigenvalues; denominator over all D), capped at the largest multiple of 32 not
 *  above min(D, MRQ_MAX_D); mrq_index_info reports it.  d = 0 with rotation_gauss is
 *  MRQ_EINVAL (the draw's size depends on d).  bits: code bits per
 *  quantized coordinate, 1..8 (1 = the paper's sign code).  nlist: IVF lists,
 *  1 <= nlist <= n.  n must be < 2^31.  opt may be NULL (defaults).
 * Steps: float64 mean/covariance and float64 Jacobi eigendecomposition (PCA,
 * residual variances), projection of the base, k-means on the leading d
 * coordinates, quantization with the random rotation P_r, precomputed factors.
 * On success *out owns device memory; release it with mrq_free.
 */
int mrq_build(const float* base, int64_t n, int D, int d, int bits, int nlist,
              const mrq_build_opts* opt, mrq_index** out);

/*
 * Search (Algorithm 2) nq queries for their k nearest neighbours among the
 * vectors of the nprobe IVF lists nearest to each query.
 *  queries: nq x D float32 (host or device).  ids: nq x k int64, dists: nq x k
 *  float32 (host or device, both the same kind).  1 <= k <= 1024,
 *  1 <= nprobe <= nlist.  Results are sorted by (distance, id); when fewer than
 *  k vectors reach the exact stage the tail is id -1, distance +inf.
 * Thresholds follow an order-independent contract (tau_A = k-th smallest stage-1
 * upper bound, tau_B = min(tau_A, k-th smallest stage-2 upper bound), survivors
 * are the candidates whose lower bound does not exceed the threshold), so the
 * answer of a query does not depend on the batch it is searched in.  Host queries
 * are copied to device memory once per batch before the projection.
 */
int mrq_search(mrq_index* index, const float* queries, int64_t nq, int k, int nprobe,
               const mrq_search_opts* opt, int64_t* ids, float* dists);

/*
 * Per-candidate stage-1 values of one query against one list (diagnostics and
 * parity tests).  The query is given already projected: qp is the D-vector
 * [q_d' | q_r] in the index's rotated PCA frame (host or device).  Outputs (host
 * or device, length = size of list `list`): ip (the inner product <v, q'> the
 * scan uses), dis (Eq. 4), lb, ub (stage-1 bounds), and, when query_bits > 0,
 * int_dot (the integer code dot <u, qbar>) else untouched (may be NULL).
 */
int mrq_estimate(mrq_index* index, const float* qp, int list, const mrq_search_opts* opt,
                 float* ip, float* dis, float* lb, float* ub, int32_t* int_dot);

/* Project queries into the index frame: qp = W (q - mu), nq x D (host or device). */
int mrq_project(mrq_index* index, const float* queries, int64_t nq,
                const mrq_search_opts* opt, float* qp);

/* Largest scratch, in bytes, that mrq_project_noalloc may use: its bf16 copy
 * of the centred queries takes 2 * nq * D bytes at MRQ_PREC_BF16 and
 * 4 * nq * D bytes at MRQ_PREC_BF16X3 (hi and lo halves); its e4m3 copy at
 * MRQ_PREC_FP8 takes nq * D bytes (rounded up to 256) plus 4 * nq of row scales. */
#define MRQ_PROJECT_NOALLOC_MAX_BYTES 8388608

/*
 * mrq_project without any allocation.  The paper has no counterpart: this is
 * an interface for callers that must not allocate device memory during a
 * call, such as an application that has given all of the GPU's memory to its
 * own pool allocator (a new cudaMalloc would fail or fragment that pool), or a
 * latency-critical serving loop that cannot take the device-wide
 * synchronisation that cudaMalloc/cudaFree can cause.
 *
 * Computes qp = W (q - mu) exactly as mrq_project does with the same opt (same
 * kernels and tile shapes), but queries (nq x D, row-major float32) and qp
 * (nq x D) must both be device memory on the index's device, and the work runs
 * on opt->cuda_stream (NULL opt or stream: the legacy default stream).  The
 * call returns once qp is written (it synchronises that stream).
 *
 * Scratch: MRQ_PREC_FP32 needs none.  The tensor-core precisions use a fixed
 * static device array of MRQ_PROJECT_NOALLOC_MAX_BYTES bytes that the library
 * owns: its pipeline error word, and, when the query rows are not 16-byte
 * aligned (the fused kernel then cannot take them) or at MRQ_PREC_FP8, the
 * bf16 or e4m3 copy of the centred queries.  The size limit below holds
 * whichever kernel runs; a request that
 * needs more (nq * D > 4194304 at MRQ_PREC_BF16, > 2097152 at MRQ_PREC_BF16X3; at
 * MRQ_PREC_FP8 whenever 256 * ceil(nq * D / 256) + 4 * nq > 8388608, e.g.
 * nq > 63550 at D = 128) returns MRQ_EINVAL without launching anything: split
 * the batch.  The
 * pipeline error word in that array is cleared at the start of every call;
 * nothing else in it has to start at zero.
 *
 * The first call on each device does one-time set-up (it looks up the scratch
 * array's address and sets kernel attributes), so make that first call before
 * any stream capture begins.  There is one scratch array per device: calls
 * that overlap in time on the same device (from two threads, or on two streams)
 * race on it and may return wrong values.  Errors: MRQ_EINVAL for NULL or host
 * pointers, nq < 1 or a too-large request; MRQ_ETIMEDOUT if a tensor-core
 * pipeline wait gave up; MRQ_ECUDA for a CUDA failure.
 */
int mrq_project_noalloc(mrq_index* index, const float* queries, int64_t nq,
                        const mrq_search_opts* opt, float* qp);

/* Result of mrq_autotune: the chosen scan configuration and what it cost. */
typedef struct {
  int scan;        /* MRQ_SCAN_PAIRS, MRQ_SCAN_BATCHED or MRQ_SCAN_BATCHED_TC */
  int chunk;       /* candidates per work item of a long list (per-pair scan) */
  int group;       /* queries per work item of the batched scan (1..16) */
  double ms;       /* median device time of one search of the tuning batch with it */
  double ms_default; /* the same for the untuned configuration of opt->batched */
  int n_tried;     /* configurations timed */
  int consistent;  /* 1 when every configuration returned identical ids and distances */
} mrq_tune_result_t;

/*
 * Autotuner of the scan's work decomposition (not a step of the paper, which scans
 * one list per query on a CPU): times, on the given queries, the per-pair scan with
 * long lists cut into work items of 1024, 4096 or 16384 candidates and the batched
 * scan with 4, 8 or 16 queries per work item and the tensor-core batched scan (where
 * the code shape allows them), each
 * as a median of 3 CUDA-event timed searches after one warm-up, and records the
 * fastest for (k, nprobe, opt->query_bits) in the index; searches with
 * opt->batched = MRQ_SCAN_AUTO then use it.  All configurations compute the same
 * answer (the threshold contract does not depend on the decomposition), which the
 * call checks.  queries: nq x D row-major float32, host or device.  Not to be called
 * while other searches on the index are running.  Errors as mrq_search.
 */
int mrq_autotune(mrq_index* index, const float* queries, int64_t nq, int k, int nprobe,
                 const mrq_search_opts* opt, mrq_tune_result_t* result);

/* Per-query counters of the last mrq_search on this index (host arrays of nq):
 * candidates scanned, stage-1 survivors, exact distances computed. */
int mrq_last_search_stats(const mrq_index* index, int64_t nq, int64_t* n_cand,
                          int64_t* n_s1, int64_t* n_exact);

/* Device time per stage of the last mrq_search run with opts.profile = 1, in
 * milliseconds summed over its internal batches (CUDA events on the search
 * stream), and the number of kernels it launched.  stage_ms: MRQ_NSTAGES doubles. */
int mrq_last_search_profile(const mrq_index* index, double* stage_ms, int64_t* launches);

/* ---------------------------------------------------------------- serving
 * Continuous batching: requests (one query each, with its own k and nprobe) are
 * queued by mrq_submit; a scheduler thread groups pending requests with equal
 * (k, nprobe), oldest first, and launches a group as one batch when one of
 * max_inflight stream slots is free and the batch's scratch fits mem_budget
 * (device bytes; one batch is always admitted); a group smaller than max_batch
 * waits at most max_wait_us for more requests.  Batches run concurrently on
 * their own streams.  The answer of every request equals a standalone mrq_search
 * of that query with the same options.  The index must not be used by other
 * calls while a server runs on it. */
typedef struct mrq_server mrq_server;
typedef struct {
  size_t mem_budget;       /* device bytes for in-flight batches; default 8 GiB */
  int max_batch;           /* queries per batch; default 4096 */
  int max_inflight;        /* concurrently running batches (streams); default 4 */
  int max_wait_us;         /* longest wait of a partial batch; default 300 */
  int max_k;               /* largest k accepted; default 128 */
  mrq_search_opts search;  /* eps0, m, mode, precision, query_bits, batched (stream ignored) */
} mrq_server_opts;
typedef struct {
  int64_t completed, batches, pending;
  double p50_us, p99_us, max_us;  /* submit-to-completion latency of completed requests */
  double qps;                     /* completed requests per second since start / reset */
} mrq_server_stats_t;

void mrq_server_opts_default(mrq_server_opts* opt);
int mrq_server_start(mrq_index* index, const mrq_server_opts* opt, mrq_server** out);
/* Queue one query (D floats, host memory, copied); *ticket identifies the request. */
int mrq_submit(mrq_server* server, const float* query, int k, int nprobe, uint64_t* ticket);
/* Results of a ticket (k ids and dists, host memory).  Returns 0 and releases the
 * ticket when done; 1 if still pending after waiting up to wait_ms milliseconds;
 * a negative MRQ_E* code if its batch failed or the ticket is unknown. */
int mrq_poll(mrq_server* server, uint64_t ticket, int64_t* ids, float* dists, int wait_ms);
/* Bulk forms: n queries (n x D, host) with per-request k and nprobe; results of n
 * tickets into n x kmax arrays (padded with -1 / +inf), status[i] = 0 done (ticket
 * released), 1 pending, or a negative MRQ_E* code. */
int mrq_submit_many(mrq_server* server, int64_t n, const float* queries, const int* k,
                    const int* nprobe, uint64_t* tickets);
int mrq_poll_many(mrq_server* server, int64_t n, const uint64_t* tickets, int kmax, int64_t* ids,
                  float* dists, int32_t* status);
/* Up to max_n completed requests in completion order (their tickets, results into
 * max_n x kmax arrays, status 0 or a negative MRQ_E* code), released; returns how
 * many (>= 0) or a negative MRQ_E* code. */
int64_t mrq_poll_completed(mrq_server* server, int64_t max_n, int kmax, uint64_t* tickets,
                           int64_t* ids, float* dists, int32_t* status);
int mrq_server_stats(mrq_server* server, mrq_server_stats_t* stats);
int mrq_server_reset_stats(mrq_server* server);
/* Finish queued and running batches, stop the scheduler, free the server. */
int mrq_server_stop(mrq_server* server);

/* Save / load the index file: magic "MRQINDEX", version 1, header (n, D, d, bits,
 * nlist), then tagged sections MU__, LAM_, W___, CENT, LOFF, IDS_, CODE (one u8 level
 * per dimension), FADD, FRES, FERR, XD__, XR__, XN2_ (list-major, unpadded), and, for
 * bits > 1, the optional FRE1, FER1 (f32[n]: Eq. 4 / Eq. 5 factors of the sign plane,
 * used by refine = 1; written when the index holds them, both or neither), and the optional
 * MR-PQ sections PQR_ (f32[d*d], R), PQC_ (f32[K*d], codebooks M x K x d/M) and PQK_
 * (u8[n*M], codes, list-major), all three or none.  Unknown
 * sections are skipped.  A malformed or other-version file gives MRQ_EFORMAT, an
 * unreadable path MRQ_EIO. */
int mrq_save(const mrq_index* index, const char* path);
int mrq_load(const char* path, mrq_index** out);

int mrq_index_info(const mrq_index* index, mrq_index_info_t* info);

/* Number of queries of the last mrq_search on this index whose stage-1 survivors
 * overflowed their region (survivor_region, or the automatic one) and were searched
 * again with a larger region; 0 when the region held every query.  No GPU call. */
int mrq_last_search_redo(const mrq_index* index, int64_t* redone);

/* Copy one index array to host memory in the file's canonical layout (list-major,
 * unpadded).  field: 4-character tag of the file format (e.g. "CODE", "XD__"; "FRE1" and
 * "FER1" only when the index holds them, else MRQ_EINVAL), or one of the MR-SQ arrays
 * (made on demand): "SQ8C" u8[n*d] codes, "SQ8L" f32[d] grid start, "SQ8S" f32[d] grid
 * step. */
int mrq_index_export(const mrq_index* index, const char* field, void* host_dst,
                     size_t bytes);

/*
 * Train the OPQ of MRQ_MODE_PQ on the GPU (Appendix A.2, Exp-5; non-parametric OPQ):
 * R starts at the identity and the K initial centroids of every subspace are the rows
 * init_rows (K row positions of the list-major x_d', host int64; NULL = K distinct
 * rows drawn from `seed`); then opq_iters times: km_iters Lloyd rounds of every
 * subspace of x_d' R (assignment ties to the lower centroid, float64 means, an empty
 * centroid keeps its value) and a final assignment, then R = U V^T for
 * X^T Y = U S V^T (X the rows of x_d', Y their decoded rows; computed as
 * A (A^T A)^(-1/2) with the float64 Jacobi eigensolver); finally one more k-means of
 * x_d' R and the codes.  Replaces any earlier OPQ of the index; saved by mrq_save.
 *  d % M == 0, 2 <= K <= 256, K <= n, M * K <= 4096 (the per-warp lookup table of the
 *  scan), 0 <= opq_iters, km_iters <= 100, else MRQ_EINVAL.
 */
int mrq_pq_train(mrq_index* index, int M, int K, int opq_iters, int km_iters,
                 const int64_t* init_rows, uint64_t seed);

/*
 * List-sharded search (Section 5, distributed deployment: MRQ inside a distributed
 * IVF system).  The IVF lists are partitioned over nshards shards; every shard keeps
 * the global statistics (mu, lambda, W, all centroids) so that it probes the same
 * lists as the whole index, but holds only the members of its own lists.  A query
 * is searched on every shard (same k, nprobe and options), each shard returns its
 * top k under the threshold contract of its own candidates, and one exchange plus
 * mrq_merge_topk gives the answer.  Whenever every estimate's bounds hold, each
 * shard's answer is the exact top k of its probed candidates, so the merged answer
 * is the exact top k of all probed candidates: the single index's answer.
 */

/* Partition plan (host only, no GPU call): lists in decreasing size (ties: lower list
 * id first) each go to the shard holding the fewest vectors so far (ties: lower shard).
 *  list_sizes: int64[nlist] (host).  owner: int32[nlist] (host, caller-owned) receives
 *  each list's shard.  1 <= nshards <= nlist, else MRQ_EINVAL. */
int mrq_shard_plan(const int64_t* list_sizes, int nlist, int nshards, int32_t* owner);

/* A new index (on the current device) holding shard `shard` of `index` under
 * mrq_shard_plan: the same header, mu, lambda, W and centroids, and the members
 * (codes, factors, x_d', x_r, norms, ids) of the lists the plan gives it; the other
 * lists are empty.  *out is released with mrq_free.  0 <= shard < nshards <= nlist;
 * MRQ_EINVAL also when the shard would hold no vector. */
int mrq_index_shard(const mrq_index* index, int nshards, int shard, mrq_index** out);

/* Merge per-shard answers: ids / dists are nparts x nq x k (part-major, each part's rows
 * sorted by (dist, id), id -1 / dist +inf padding), out_ids / out_dists nq x k receive
 * the k smallest (dist, id) of each query over all parts, -1 / +inf padded.  All four
 * arrays host or all four device memory (the device merge runs on cuda_stream, NULL =
 * the legacy default stream, and returns after it completes); caller-owned.  Host merges
 * make no GPU call.  1 <= nparts <= 64, 1 <= k <= 1024, nq >= 0, else MRQ_EINVAL. */
int mrq_merge_topk(const int64_t* ids, const float* dists, int nparts, int64_t nq, int k,
                   void* cuda_stream, int64_t* out_ids, float* out_dists);

void mrq_free(mrq_index* index);

/* Message of the last failed call on this thread ("" if none). */
const char* mrq_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* MRQ_H */
