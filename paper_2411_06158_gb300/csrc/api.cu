// C ABI of libmrq (declared in include/mrq.h): argument checks, host/device
// staging, batching, index file I/O.  Every entry point catches internal
// errors and turns them into MRQ_E* codes plus a thread-local message.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <memory>
#include <string>

#include "common.cuh"

namespace {

thread_local std::string g_err;

// a nested public call inside a guarded body: rethrow its error
#define MRQ_CHECK_RC(call)                                \
  do {                                                    \
    const int rc_ = (call);                               \
    if (rc_ != MRQ_OK) ::mrq::fail(rc_, std::string(g_err)); \
  } while (0)

template <class F>
int guarded(F&& f) {
  try {
    f();
    g_err.clear();
    return MRQ_OK;
  } catch (const mrq::Error& e) {
    g_err = e.msg;
    return e.code;
  } catch (const std::bad_alloc&) {
    g_err = "host allocation failed";
    return MRQ_ENOMEM;
  } catch (const std::exception& e) {
    g_err = e.what();
    return MRQ_EINVAL;
  }
}

bool on_device(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// page-locked host memory (cudaHostAlloc / cudaHostRegister): copies from it can be
// asynchronous and captured in a CUDA graph
bool pinned_host(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

cudaStream_t stream_of(const mrq_search_opts& o) { return (cudaStream_t)o.cuda_stream; }

void use_device(const mrq_index* idx) { MRQ_CUDA(cudaSetDevice(idx->device)); }

mrq_search_opts resolve(const mrq_search_opts* opt) {
  mrq_search_opts o;
  mrq_search_opts_default(&o);
  if (opt) o = *opt;
  MRQ_REQUIRE(o.eps0 >= 0.f && o.m >= 0.f, "eps0 and m must be >= 0");
  MRQ_REQUIRE(o.mode == MRQ_MODE_MRQ || o.mode == MRQ_MODE_MRQ_PLUS || o.mode == MRQ_MODE_SQ8 ||
                  o.mode == MRQ_MODE_PQ,
              "mode must be MRQ_MODE_MRQ, MRQ_MODE_MRQ_PLUS, MRQ_MODE_SQ8 or MRQ_MODE_PQ");
  MRQ_REQUIRE((o.mode != MRQ_MODE_SQ8 && o.mode != MRQ_MODE_PQ) ||
                  (o.rerank >= 1 && o.rerank <= 65536),
              "rerank must be in [1, 65536]");
  MRQ_REQUIRE(o.precision >= MRQ_PREC_FP32 && o.precision <= MRQ_PREC_FP8, "unknown precision");
  MRQ_REQUIRE(o.query_bits >= 0 && o.query_bits <= 8, "query_bits must be in [0, 8]");
  MRQ_REQUIRE(o.batched >= MRQ_SCAN_PAIRS && o.batched <= MRQ_SCAN_BATCHED_TC,
              "batched must be MRQ_SCAN_PAIRS, MRQ_SCAN_BATCHED, MRQ_SCAN_AUTO or MRQ_SCAN_BATCHED_TC");
  MRQ_REQUIRE(o.refine == 0 || o.refine == 1, "refine must be 0 or 1");
  MRQ_REQUIRE(o.survivor_region >= 0, "survivor_region must be >= 0");
  return o;
}

// the 1 bit + refinement scan's own requirements (a 1-bit code has no refinement and
// searches as usual)
void check_refine(const mrq_index* idx, const mrq_search_opts& o, int k, int nprobe) {
  if (!mrq::refine_active(idx, o)) return;
  MRQ_REQUIRE(idx->fres1.p != nullptr,
              "refine needs the sign-plane factors (FRE1/FER1), which this index does not hold");
  MRQ_REQUIRE(o.query_bits > 0, "refine needs a quantized query (query_bits >= 1)");
  MRQ_REQUIRE(k <= 128, "refine needs k <= 128");
  MRQ_REQUIRE(nprobe <= mrq::REFINE_MAX_NPROBE, "refine needs nprobe <= 4096");
}

// ---------------------------------------------------------------- file format

constexpr char kMagic[8] = {'M', 'R', 'Q', 'I', 'N', 'D', 'E', 'X'};
constexpr uint32_t kVersion = 1;
enum : uint32_t { DT_F32 = 1, DT_F64 = 2, DT_I64 = 3, DT_U8 = 4 };

struct Section {
  char tag[4];
  uint32_t dtype;
  std::vector<uint8_t> data;
};

size_t dt_size(uint32_t dt) { return dt == DT_F32 ? 4 : dt == DT_F64 ? 8 : dt == DT_I64 ? 8 : 1; }

template <typename T>
std::vector<uint8_t> d2h_bytes(const T* dev, size_t count, cudaStream_t st) {
  std::vector<uint8_t> v(count * sizeof(T));
  if (count) MRQ_CUDA(cudaMemcpyAsync(v.data(), dev, v.size(), cudaMemcpyDeviceToHost, st));
  return v;
}

}  // namespace

namespace mrq {
void set_last_error(const std::string& m) { g_err = m; }
}  // namespace mrq

// ===================================================================== ABI

// The queries of the last search whose stage-1 survivors overflowed their region
// (listed by the scan) are searched again in rounds, each with a region eight times the
// last (the full worst case at most, which cannot overflow): their rows gathered, searched
// in batches that fit the budget, the answers and counters written back to their rows,
// and the queries that overflowed again kept for the next round.
static void redo_overflowed(mrq_index* idx, const float* queries, int k, int nprobe,
                            const mrq_search_opts& o, int64_t* ids, float* dists, int64_t cap,
                            int64_t budget, cudaStream_t st) {
  auto& ws = idx->ws;
  int count = 0;
  MRQ_CUDA(cudaMemcpy(&count, ws.ovf.p, sizeof(int), cudaMemcpyDeviceToHost));
  idx->last_redo = count;
  if (count <= 0) return;
  std::vector<int> bad(count);
  MRQ_CUDA(cudaMemcpy(bad.data(), ws.ovf.p + 1, sizeof(int) * count, cudaMemcpyDeviceToHost));
  std::sort(bad.begin(), bad.end());
  const bool qdev = on_device(queries), odev = on_device(ids);
  auto& rw = idx->ws_redo;
  const int D = idx->D;
  mrq_search_opts o2 = o;
  // a profiled search keeps profiling here: the rounds' stages add to the call's totals
  int64_t region = std::max<int64_t>(ws.cap_limit, 1);
  while (!bad.empty()) {
    region = std::min<int64_t>(cap, region * 8);
    rw.cap_limit = region < cap ? region : 0;
    rw.items_budget = budget / 4;
    const int64_t n = (int64_t)bad.size();
    int64_t qb = std::max<int64_t>(1, budget / (24 * region));
    qb = std::min<int64_t>({qb, n, (int64_t)131072, std::max<int64_t>(1, ((int64_t)1 << 30) / nprobe),
                            std::max<int64_t>(1, (int64_t)8e9 / (4 * (int64_t)idx->nlist))});
    mrq::DevBuf<float> qt((size_t)qb * D);
    mrq::DevBuf<int64_t> it((size_t)qb * k), stt((size_t)qb * 3);
    mrq::DevBuf<float> dt((size_t)qb * k);
    mrq::DevBuf<int> rows((size_t)n);
    MRQ_CUDA(cudaMemcpyAsync(rows.p, bad.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    if (rw.cap_limit > 0) {
      rw.ovf.reserve((size_t)n + 1);
      MRQ_CUDA(cudaMemsetAsync(rw.ovf.p, 0, sizeof(int), st));
    }
    std::vector<float> hq;
    std::vector<int64_t> hi;
    std::vector<float> hd;
    for (int64_t a = 0; a < n; a += qb) {
      const int64_t b = std::min<int64_t>(qb, n - a);
      if (qdev) {
        mrq::gather_query_rows(queries, D, rows.p + a, b, qt.p, st);
      } else {
        hq.resize((size_t)b * D);
        for (int64_t j = 0; j < b; ++j)
          std::memcpy(hq.data() + j * D, queries + (int64_t)bad[a + j] * D, 4 * (size_t)D);
        MRQ_CUDA(cudaMemcpyAsync(qt.p, hq.data(), 4 * hq.size(), cudaMemcpyHostToDevice, st));
      }
      rw.ovf_base = a;  // overflow entries are positions in this round's list
      rw.seed_tau = ws.ovf_tau.p;  // bounds recorded by row when the queries overflowed
      rw.seed_rows = rows.p + a;
      mrq::search_batch(idx, rw, qt.p, b, k, nprobe, o2, it.p, dt.p, stt.p, st);
      mrq::scatter_answers(it.p, dt.p, stt.p, k, rows.p + a, b, odev ? ids : nullptr,
                           odev ? dists : nullptr, ws.stats.p, st);
      if (!odev) {
        hi.resize((size_t)b * k);
        hd.resize((size_t)b * k);
        MRQ_CUDA(cudaMemcpyAsync(hi.data(), it.p, 8 * hi.size(), cudaMemcpyDeviceToHost, st));
        MRQ_CUDA(cudaMemcpyAsync(hd.data(), dt.p, 4 * hd.size(), cudaMemcpyDeviceToHost, st));
        MRQ_CUDA(cudaStreamSynchronize(st));
        for (int64_t j = 0; j < b; ++j) {
          std::memcpy(ids + (int64_t)bad[a + j] * k, hi.data() + j * k, 8 * (size_t)k);
          std::memcpy(dists + (int64_t)bad[a + j] * k, hd.data() + j * k, 4 * (size_t)k);
        }
      }
    }
    MRQ_CUDA(cudaStreamSynchronize(st));
    std::vector<int> next;
    if (rw.cap_limit > 0) {
      int c2 = 0;
      MRQ_CUDA(cudaMemcpy(&c2, rw.ovf.p, sizeof(int), cudaMemcpyDeviceToHost));
      if (c2 > 0) {
        std::vector<int> posl(c2);
        MRQ_CUDA(cudaMemcpy(posl.data(), rw.ovf.p + 1, sizeof(int) * c2, cudaMemcpyDeviceToHost));
        next.reserve(c2);
        for (int pidx : posl) next.push_back(bad[pidx]);
        std::sort(next.begin(), next.end());
      }
    }
    bad.swap(next);
  }
  rw.seed_tau = nullptr;
  rw.seed_rows = nullptr;
}

extern "C" {

const char* mrq_last_error(void) { return g_err.c_str(); }

void mrq_build_opts_default(mrq_build_opts* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->seed = 1;
  opt->kmeans_iters = 20;
  opt->auto_d_variance = 0.8;
}

void mrq_search_opts_default(mrq_search_opts* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->eps0 = 1.9f;
  opt->m = 4.0f;
  opt->mode = MRQ_MODE_MRQ_PLUS;
  opt->precision = MRQ_PREC_FP32;
  opt->query_bits = 0;
  opt->batched = 0;
  opt->rerank = 500;
  opt->cuda_stream = nullptr;
}

int mrq_build(const float* base, int64_t n, int D, int d, int bits, int nlist,
              const mrq_build_opts* opt, mrq_index** out) {
  return guarded([&] {
    MRQ_REQUIRE(out != nullptr, "out is NULL");
    *out = nullptr;
    MRQ_REQUIRE(base != nullptr, "base is NULL");
    MRQ_REQUIRE(n >= 1 && n < (int64_t(1) << 31), "n must be in [1, 2^31)");
    MRQ_REQUIRE(D >= 32 && D <= 16384, "D must be in [32, 16384]");
    MRQ_REQUIRE(d == 0 || (d >= 32 && d <= D && d % 32 == 0 && d <= MRQ_MAX_D),
                "d must be 0 (Eq. 8) or a multiple of 32 in [32, min(D, 1024)]");
    MRQ_REQUIRE(bits >= 1 && bits <= 8, "bits must be in [1, 8]");
    MRQ_REQUIRE(nlist >= 1 && nlist <= n && nlist <= (1 << 20), "nlist must be in [1, min(n, 2^20)]");
    mrq_build_opts o;
    mrq_build_opts_default(&o);
    if (opt) o = *opt;
    MRQ_REQUIRE(o.kmeans_iters >= 0 && o.kmeans_iters <= 1000, "kmeans_iters must be in [0, 1000]");
    MRQ_REQUIRE(o.auto_d_variance > 0.0 && o.auto_d_variance <= 1.0,
                "auto_d_variance must be in (0, 1]");
    MRQ_REQUIRE(d != 0 || o.rotation_gauss == nullptr,
                "d = 0 (chosen by Eq. 8) cannot take a rotation_gauss draw");
    if (o.pca_rows) {
      MRQ_REQUIRE(o.pca_n >= 2 && o.pca_n <= n, "pca_n must be in [2, n] with pca_rows");
      for (int64_t i = 0; i < o.pca_n; ++i)
        MRQ_REQUIRE(o.pca_rows[i] >= 0 && o.pca_rows[i] < n, "pca_rows out of range");
    }
    std::unique_ptr<mrq_index> idx(new mrq_index());
    MRQ_CUDA(cudaGetDevice(&idx->device));
    idx->n = n;
    idx->D = D;
    idx->d = d;
    idx->bits = bits;
    idx->nlist = nlist;
    cudaStream_t st = nullptr;
    mrq::DevBuf<float> staged;
    const float* X = base;
    if (!on_device(base)) {
      staged.alloc((size_t)n * D);
      MRQ_CUDA(cudaMemcpy(staged.p, base, staged.bytes(), cudaMemcpyHostToDevice));
      X = staged.p;
    }
    mrq::build_index(idx.get(), X, o, st);
    *out = idx.release();
  });
}

int mrq_search(mrq_index* idx, const float* queries, int64_t nq, int k, int nprobe,
               const mrq_search_opts* opt, int64_t* ids, float* dists) {
  return guarded([&] {
    MRQ_REQUIRE(idx != nullptr, "index is NULL");
    MRQ_REQUIRE(nq >= 0, "nq must be >= 0");
    MRQ_REQUIRE(k >= 1 && k <= 1024, "k must be in [1, 1024]");
    MRQ_REQUIRE(nprobe >= 1 && nprobe <= idx->nlist && nprobe <= 16384,
                "nprobe must be in [1, min(nlist, 16384)]");
    if (nq == 0) return;
    MRQ_REQUIRE(queries && ids && dists, "queries, ids and dists must not be NULL");
    const mrq_search_opts o = resolve(opt);
    check_refine(idx, o, k, nprobe);
    if (o.mode == MRQ_MODE_SQ8 || o.mode == MRQ_MODE_PQ) {
      MRQ_REQUIRE(k <= 128 && k <= o.rerank,
                  "MRQ_MODE_SQ8 and MRQ_MODE_PQ need k <= 128 and k <= rerank");
    }
    if (o.mode == MRQ_MODE_PQ)
      MRQ_REQUIRE(idx->pq_M > 0, "MRQ_MODE_PQ needs an OPQ (mrq_pq_train, or PQ sections in the file)");
    use_device(idx);
    cudaStream_t st = stream_of(o);
    if (o.mode == MRQ_MODE_SQ8) mrq::ensure_sq8(idx, st);  // before any graph capture
    const bool qdev = on_device(queries);
    const bool odev = on_device(ids);
    MRQ_REQUIRE(odev == on_device(dists), "ids and dists must both be host or both be device memory");
    const int D = idx->D;
    const int64_t cap = std::max<int64_t>(idx->cap_by_nprobe[nprobe], 1);
    // batch size: survivor scratch (6 arrays x 4 B x cap per query) within the budget
    // below, probe matrix within ~1 GB
    int64_t qb = std::min<int64_t>(nq, 16384);
    // the survivor scratch is sized for the worst case (every candidate of the nprobe
    // largest lists); give it up to a quarter of the free device memory (at least 6 GB,
    // at most 64 GB) so that indexes with very uneven lists still run large batches
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    int64_t budget =
        std::min<int64_t>((int64_t)64 << 30, std::max<int64_t>((int64_t)6e9, (int64_t)(free_b / 4)));
    // scratch this index already holds counts as available (the batch size stays put)
    budget = std::max<int64_t>(budget, (int64_t)idx->ws.spos.n * 24);
    auto& ws = idx->ws;
    // the bounded modes write only stage-1 survivors, a small fraction of the candidates:
    // when the worst-case region (every candidate of the nprobe largest lists) does not
    // fit a large batch, each query gets a smaller region and a query that overflows it
    // is searched again with the full region after the batch (exact either way)
    const bool bounded = o.mode == MRQ_MODE_MRQ || o.mode == MRQ_MODE_MRQ_PLUS;
    constexpr int64_t kMinRegion = 8192;
    ws.cap_limit = 0;
    if (bounded) {
      qb = std::min<int64_t>(nq, 131072);
      qb = std::min<int64_t>(qb, std::max<int64_t>(1, (int64_t)8e9 / (4 * (int64_t)idx->nlist)));
      qb = std::min<int64_t>(qb, std::max<int64_t>(1, ((int64_t)1 << 30) / nprobe));
      if (o.survivor_region > 0 && o.survivor_region < cap) {
        ws.cap_limit = o.survivor_region;
        qb = std::min<int64_t>(qb, std::max<int64_t>(1, budget / (24 * ws.cap_limit)));
      } else if (24 * cap * qb > budget) {
        int64_t c = budget / (24 * qb);
        if (c < kMinRegion) {
          c = std::min<int64_t>(kMinRegion, cap);
          qb = std::max<int64_t>(1, budget / (24 * c));
        }
        if (c < cap) ws.cap_limit = c;
      }
    } else {
      qb = std::min<int64_t>(qb, std::max<int64_t>(1, budget / (24 * cap)));
      qb = std::min<int64_t>(qb, std::max<int64_t>(1, (int64_t)1e9 / (4 * (int64_t)idx->nlist)));
    }
    ws.items_budget = budget / 4;
    if (ws.cap_limit > 0) {
      ws.ovf.reserve((size_t)nq + 1);
      ws.ovf_tau.reserve((size_t)nq);
    }
    ws.seed_out = ws.cap_limit > 0 ? ws.ovf_tau.p : nullptr;
    ws.stats.reserve((size_t)nq * 3);
    if (!odev) {
      ws.oids.reserve((size_t)qb * k);
      ws.odist.reserve((size_t)qb * k);
    }
    if (!qdev) ws.q.reserve((size_t)qb * D);
    idx->prof_on = o.profile != 0;
    idx->prof_batches = 0;
    idx->launches = 0;
    idx->last_redo = 0;
    // a captured graph also covers host buffers when they are page-locked (its copy
    // nodes then read and write those buffers on every replay)
    const bool use_graph = o.graph && !o.profile && (qdev || pinned_host(queries)) &&
                           (odev || (pinned_host(ids) && pinned_host(dists)));
    mrq_index::GraphKey key{queries, ids, dists, nq, k, nprobe, o.mode, o.precision,
                            o.query_bits, o.batched, o.refine,
                            (o.mode == MRQ_MODE_SQ8 || o.mode == MRQ_MODE_PQ) ? o.rerank : 0,
                            o.eps0, o.m, o.survivor_region};
    auto run_batches = [&](cudaStream_t s_) {
      if (ws.cap_limit > 0) MRQ_CUDA(cudaMemsetAsync(ws.ovf.p, 0, sizeof(int), s_));
      for (int64_t s = 0; s < nq; s += qb) {
        ws.ovf_base = s;
        const int64_t b = std::min(qb, nq - s);
        const float* qp = queries + s * D;
        if (!qdev) {  // host queries: one copy per batch into device memory
          MRQ_CUDA(cudaMemcpyAsync(ws.q.p, qp, 4 * b * D, cudaMemcpyHostToDevice, s_));
          qp = ws.q.p;
        }
        int64_t* oi = odev ? ids + s * k : ws.oids.p;
        float* od = odev ? dists + s * k : ws.odist.p;
        mrq::search_batch(idx, ws, qp, b, k, nprobe, o, oi, od, ws.stats.p + s * 3, s_);
        if (!odev) {
          MRQ_CUDA(cudaMemcpyAsync(ids + s * k, oi, 8 * b * k, cudaMemcpyDeviceToHost, s_));
          MRQ_CUDA(cudaMemcpyAsync(dists + s * k, od, 4 * b * k, cudaMemcpyDeviceToHost, s_));
        }
      }
    };
    if (use_graph) {
      if (!idx->graph_stream) {
        MRQ_CUDA(cudaStreamCreateWithFlags(&idx->graph_stream, cudaStreamNonBlocking));
        MRQ_CUDA(cudaEventCreateWithFlags(&idx->graph_ev[0], cudaEventDisableTiming));
        MRQ_CUDA(cudaEventCreateWithFlags(&idx->graph_ev[1], cudaEventDisableTiming));
      }
      if (!(idx->graph_valid && idx->graph_key == key &&
            idx->graph_epoch == mrq::g_ws_epoch.load())) {
        // first call with these arguments, or scratch that moved since the capture: run
        // once (sizes scratch), then capture
        run_batches(st);
        MRQ_CUDA(cudaStreamSynchronize(st));
        const int64_t l0 = idx->launches;
        if (idx->graph_exec) {
          cudaGraphExecDestroy(idx->graph_exec);
          idx->graph_exec = nullptr;
        }
        idx->graph_valid = false;
        cudaGraph_t g = nullptr;
        MRQ_CUDA(cudaStreamBeginCapture(idx->graph_stream, cudaStreamCaptureModeRelaxed));
        try {
          run_batches(idx->graph_stream);
        } catch (...) {
          cudaStreamEndCapture(idx->graph_stream, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        MRQ_CUDA(cudaStreamEndCapture(idx->graph_stream, &g));
        cudaError_t ie = cudaGraphInstantiate(&idx->graph_exec, g, 0);
        cudaGraphDestroy(g);
        MRQ_CUDA(ie);
        idx->graph_key = key;
        idx->graph_epoch = mrq::g_ws_epoch.load();
        idx->graph_valid = true;
        idx->graph_launches = idx->launches - l0;
      }
      MRQ_CUDA(cudaEventRecord(idx->graph_ev[0], st));
      MRQ_CUDA(cudaStreamWaitEvent(idx->graph_stream, idx->graph_ev[0], 0));
      MRQ_CUDA(cudaGraphLaunch(idx->graph_exec, idx->graph_stream));
      MRQ_CUDA(cudaEventRecord(idx->graph_ev[1], idx->graph_stream));
      MRQ_CUDA(cudaStreamWaitEvent(st, idx->graph_ev[1], 0));
      idx->launches = idx->graph_launches;
    }
    if (!use_graph) run_batches(st);
    // the tensor-core kernels' error word comes back with the results (one small
    // asynchronous copy); the per-query counters stay on the device until asked for
    int* herr = o.precision != MRQ_PREC_FP32 ? mrq::tc_error_mirror() : nullptr;
    if (herr) {
      *herr = 0;
      MRQ_CUDA(cudaMemcpyAsync(herr, mrq::tc_error_word(), sizeof(int), cudaMemcpyDeviceToHost, st));
    }
    MRQ_CUDA(cudaStreamSynchronize(st));
    if (herr && *herr && mrq::tc_check_error())
      mrq::fail(MRQ_ETIMEDOUT, "a tensor-core kernel gave up waiting on its pipeline");
    if (ws.cap_limit > 0) redo_overflowed(idx, queries, k, nprobe, o, ids, dists, cap, budget, st);
    idx->last_nq = nq;
    idx->last_stats_dev = true;
    for (int s = 0; s < MRQ_NSTAGES; ++s) idx->prof_ms[s] = 0.0;
    if (idx->prof_on) {
      for (int b = 0; b < idx->prof_batches; ++b)
        for (int s = 0; s < MRQ_NSTAGES; ++s) {
          float ms = 0.f;
          MRQ_CUDA(cudaEventElapsedTime(&ms, idx->prof_ev[(size_t)b * (MRQ_NSTAGES + 1) + s],
                                        idx->prof_ev[(size_t)b * (MRQ_NSTAGES + 1) + s + 1]));
          idx->prof_ms[s] += ms;
        }
    }
  });
}

int mrq_autotune(mrq_index* idx, const float* queries, int64_t nq, int k, int nprobe,
                 const mrq_search_opts* opt, mrq_tune_result_t* result) {
  return guarded([&] {
    MRQ_REQUIRE(idx && queries && result, "NULL argument");
    MRQ_REQUIRE(nq >= 1, "nq must be >= 1");
    mrq_search_opts o = resolve(opt);
    o.graph = 0;
    o.profile = 0;
    use_device(idx);
    cudaStream_t st = stream_of(o);
    const int D = idx->D;
    // device copies of the queries and two output sets (this config's, the first one's)
    mrq::DevBuf<float> qd_;
    const float* q = queries;
    if (!on_device(queries)) {
      qd_.alloc((size_t)nq * D);
      MRQ_CUDA(cudaMemcpyAsync(qd_.p, queries, 4 * nq * D, cudaMemcpyHostToDevice, st));
      q = qd_.p;
    }
    mrq::DevBuf<int64_t> ids(nq * k);
    mrq::DevBuf<float> dists(nq * k);
    std::vector<int64_t> ref_i((size_t)nq * k), got_i((size_t)nq * k);
    std::vector<float> ref_d((size_t)nq * k), got_d((size_t)nq * k);
    cudaEvent_t e0, e1;
    MRQ_CUDA(cudaEventCreate(&e0));
    MRQ_CUDA(cudaEventCreate(&e1));
    struct EvGuard {
      cudaEvent_t a, b;
      ~EvGuard() { cudaEventDestroy(a); cudaEventDestroy(b); }
    } evg{e0, e1};
    auto time_cfg = [&](const mrq::ScanConfig* c) {
      mrq::ScopedScanConfig force(c);
      MRQ_CHECK_RC(mrq_search(idx, q, nq, k, nprobe, &o, ids.p, dists.p));  // warm-up
      std::vector<float> t;
      for (int r = 0; r < 3; ++r) {
        MRQ_CUDA(cudaEventRecord(e0, st));
        MRQ_CHECK_RC(mrq_search(idx, q, nq, k, nprobe, &o, ids.p, dists.p));
        MRQ_CUDA(cudaEventRecord(e1, st));
        MRQ_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        MRQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        t.push_back(ms);
      }
      std::sort(t.begin(), t.end());
      return (double)t[1];
    };
    // candidates
    std::vector<mrq::ScanConfig> cands;
    for (int chunk : {1024, 4096, 16384}) {
      if (chunk != 4096 && idx->max_list <= 1024) continue;  // no list is long enough to cut
      cands.push_back({MRQ_SCAN_PAIRS, chunk, 16});
    }
    const int wds = idx->words, nch = idx->d / 32;
    const bool refine = mrq::refine_active(idx, o);  // scans pair by pair
    const bool sq8 = o.mode == MRQ_MODE_SQ8 || o.mode == MRQ_MODE_PQ;  // so do MR-SQ, MR-PQ
    const bool can_batch = !refine && !sq8 && o.query_bits > 0 && wds <= 16 && (wds & (wds - 1)) == 0 &&
                           (idx->bits & (idx->bits - 1)) == 0 && (nch & (nch - 1)) == 0 &&
                           !(wds == 16 && idx->d == 32);
    if (can_batch)
      for (int g : {4, 8, 16}) cands.push_back({MRQ_SCAN_BATCHED, 4096, g});
    if (!refine && !sq8 && mrq::tc_available() &&
        mrq::scan_tc_supported(idx->d, idx->bits, o.query_bits))
      cands.push_back({MRQ_SCAN_BATCHED_TC, 4096, mrq::TC_SCAN_GROUP});
    const mrq::ScanConfig dflt = mrq::scan_config(idx, o, nq, k, nprobe);
    result->consistent = 1;
    double best = 1e300;
    mrq::ScanConfig pick = cands[0];
    for (size_t c = 0; c < cands.size(); ++c) {
      const double ms = time_cfg(&cands[c]);
      MRQ_CUDA(cudaMemcpy(got_i.data(), ids.p, 8 * nq * k, cudaMemcpyDeviceToHost));
      MRQ_CUDA(cudaMemcpy(got_d.data(), dists.p, 4 * nq * k, cudaMemcpyDeviceToHost));
      if (c == 0) {
        ref_i = got_i;
        ref_d = got_d;
      } else if (got_i != ref_i ||
                 std::memcmp(got_d.data(), ref_d.data(), 4 * (size_t)nq * k) != 0) {
        result->consistent = 0;
      }
      if (ms < best) {
        best = ms;
        pick = cands[c];
      }
    }
    result->ms_default = time_cfg(&dflt);
    result->scan = pick.scan;
    result->chunk = pick.chunk;
    result->group = pick.group;
    result->ms = best;
    result->n_tried = (int)cands.size();
    {
      std::lock_guard<std::mutex> lk(idx->tune_mu);
      idx->tuned[std::make_tuple(mrq::scan_kclass(k), nprobe, o.query_bits, mrq::scan_variant(idx, o))] =
          pick;
    }
    idx->graph_valid = false;  // a captured graph may hold the old configuration
  });
}

int mrq_last_search_profile(const mrq_index* idx, double* stage_ms, int64_t* launches) {
  return guarded([&] {
    MRQ_REQUIRE(idx != nullptr, "index is NULL");
    if (stage_ms)
      for (int s = 0; s < MRQ_NSTAGES; ++s) stage_ms[s] = idx->prof_ms[s];
    if (launches) *launches = idx->launches;
  });
}

int mrq_project(mrq_index* idx, const float* queries, int64_t nq, const mrq_search_opts* opt,
                float* qp) {
  return guarded([&] {
    MRQ_REQUIRE(idx && queries && qp, "NULL argument");
    MRQ_REQUIRE(nq >= 1, "nq must be >= 1");
    const mrq_search_opts o = resolve(opt);
    use_device(idx);
    cudaStream_t st = stream_of(o);
    const int D = idx->D, d = idx->d, r = D - d;
    auto& ws = idx->ws;
    mrq::DevBuf<float> qin;
    const float* q = queries;
    if (!on_device(queries)) {
      qin.alloc((size_t)nq * D);
      MRQ_CUDA(cudaMemcpyAsync(qin.p, queries, 4 * nq * D, cudaMemcpyHostToDevice, st));
      q = qin.p;
    }
    ws.qd.reserve((size_t)nq * d);
    ws.qr.reserve((size_t)nq * std::max(r, 1));
    mrq::project_batch(idx, ws, q, nq, o.precision, ws.qd.p, ws.qr.p, st);
    MRQ_CUDA(cudaMemcpy2DAsync(qp, 4 * D, ws.qd.p, 4 * d, 4 * d, nq, cudaMemcpyDefault, st));
    if (r > 0)
      MRQ_CUDA(cudaMemcpy2DAsync(qp + d, 4 * D, ws.qr.p, 4 * r, 4 * r, nq, cudaMemcpyDefault, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
    if (o.precision != MRQ_PREC_FP32 && mrq::tc_check_error())
      mrq::fail(MRQ_ETIMEDOUT, "a tensor-core kernel gave up waiting on its pipeline");
  });
}

int mrq_project_noalloc(mrq_index* idx, const float* queries, int64_t nq,
                        const mrq_search_opts* opt, float* qp) {
  return guarded([&] {
    MRQ_REQUIRE(idx && queries && qp, "NULL argument");
    MRQ_REQUIRE(nq >= 1, "nq must be >= 1");
    const mrq_search_opts o = resolve(opt);
    use_device(idx);
    MRQ_REQUIRE(on_device(queries) && on_device(qp),
                "mrq_project_noalloc needs queries and qp in device memory");
    mrq::project_noalloc(idx, queries, nq, o.precision, qp, stream_of(o));
  });
}

int mrq_estimate(mrq_index* idx, const float* qp, int list, const mrq_search_opts* opt, float* ip,
                 float* dis, float* lb, float* ub, int32_t* int_dot) {
  return guarded([&] {
    MRQ_REQUIRE(idx && qp, "NULL argument");
    MRQ_REQUIRE(list >= 0 && list < idx->nlist, "list out of range");
    const mrq_search_opts o = resolve(opt);
    use_device(idx);
    cudaStream_t st = stream_of(o);
    const int64_t sz = idx->h_loff[list + 1] - idx->h_loff[list];
    if (sz == 0) return;
    MRQ_REQUIRE(ip && dis && lb && ub, "ip, dis, lb and ub must not be NULL");
    mrq::DevBuf<float> tmp(4 * sz);
    mrq::DevBuf<int32_t> ti(sz);
    mrq::DevBuf<float> qdev;
    const float* q = qp;
    if (!on_device(qp)) {
      qdev.alloc(idx->D);
      MRQ_CUDA(cudaMemcpyAsync(qdev.p, qp, 4 * idx->D, cudaMemcpyHostToDevice, st));
      q = qdev.p;
    }
    mrq::estimate_one(idx, q, list, o, tmp.p, tmp.p + sz, tmp.p + 2 * sz, tmp.p + 3 * sz,
                      o.query_bits > 0 ? ti.p : nullptr, st);
    MRQ_CUDA(cudaMemcpyAsync(ip, tmp.p, 4 * sz, cudaMemcpyDefault, st));
    MRQ_CUDA(cudaMemcpyAsync(dis, tmp.p + sz, 4 * sz, cudaMemcpyDefault, st));
    MRQ_CUDA(cudaMemcpyAsync(lb, tmp.p + 2 * sz, 4 * sz, cudaMemcpyDefault, st));
    MRQ_CUDA(cudaMemcpyAsync(ub, tmp.p + 3 * sz, 4 * sz, cudaMemcpyDefault, st));
    if (o.query_bits > 0 && int_dot)
      MRQ_CUDA(cudaMemcpyAsync(int_dot, ti.p, 4 * sz, cudaMemcpyDefault, st));
    MRQ_CUDA(cudaStreamSynchronize(st));
  });
}

int mrq_last_search_stats(const mrq_index* idx, int64_t nq, int64_t* n_cand, int64_t* n_s1,
                          int64_t* n_exact) {
  return guarded([&] {
    MRQ_REQUIRE(idx != nullptr, "index is NULL");
    MRQ_REQUIRE(nq == idx->last_nq, "nq differs from the last search on this index");
    if (idx->last_stats_dev) {
      use_device(idx);
      idx->last_stats.resize((size_t)nq * 3);
      MRQ_CUDA(cudaMemcpy(idx->last_stats.data(), idx->ws.stats.p, 8 * nq * 3,
                          cudaMemcpyDeviceToHost));
      idx->last_stats_dev = false;
    }
    for (int64_t i = 0; i < nq; ++i) {
      if (n_cand) n_cand[i] = idx->last_stats[i * 3 + 0];
      if (n_s1) n_s1[i] = idx->last_stats[i * 3 + 1];
      if (n_exact) n_exact[i] = idx->last_stats[i * 3 + 2];
    }
  });
}

int mrq_last_search_redo(const mrq_index* idx, int64_t* redone) {
  return guarded([&] {
    MRQ_REQUIRE(idx && redone, "NULL argument");
    *redone = idx->last_redo;
  });
}

int mrq_index_info(const mrq_index* idx, mrq_index_info_t* info) {
  return guarded([&] {
    MRQ_REQUIRE(idx && info, "NULL argument");
    info->n = idx->n;
    info->D = idx->D;
    info->d = idx->d;
    info->bits = idx->bits;
    info->nlist = idx->nlist;
    info->max_list = idx->max_list;
    info->device_bytes = (int64_t)(idx->mu.bytes() + idx->lam.bytes() + idx->W.bytes() +
                                   idx->W2.bytes() + idx->W8.bytes() + idx->W8s.bytes() +
                                   idx->cent2.bytes() + idx->cent.bytes() +
                                   idx->cent_n2.bytes() + idx->loff.bytes() + idx->ploff.bytes() +
                                   idx->ids.bytes() + idx->codes.bytes() + idx->fadd.bytes() +
                                   idx->fres.bytes() + idx->ferr.bytes() + idx->fres1.bytes() +
                                   idx->ferr1.bytes() + idx->sq_codes.bytes() +
                                   idx->sq_lo.bytes() + idx->sq_delta.bytes() +
                                   idx->sq_xr2.bytes() + idx->xd.bytes() +
                                   idx->xr.bytes() + idx->xn2.bytes() + idx->pq_R.bytes() +
                                   idx->pq_Rt.bytes() + idx->pq_C.bytes() +
                                   idx->pq_codes.bytes() + idx->pq_xr2.bytes());
    info->pq_M = idx->pq_M;
    info->pq_K = idx->pq_K;
  });
}

static void export_field(const mrq_index* idx, const std::string& f, std::vector<uint8_t>& out,
                         uint32_t& dtype, cudaStream_t st) {
  const int64_t n = idx->n;
  const int D = idx->D, d = idx->d, r = D - d;
  if (f == "MU__") { out = d2h_bytes(idx->mu.p, D, st); dtype = DT_F32; }
  else if (f == "LAM_") { out = d2h_bytes(idx->lam.p, D, st); dtype = DT_F32; }
  else if (f == "W___") { out = d2h_bytes(idx->W.p, (size_t)D * D, st); dtype = DT_F32; }
  else if (f == "CENT") { out = d2h_bytes(idx->cent.p, (size_t)idx->nlist * d, st); dtype = DT_F32; }
  else if (f == "LOFF") {
    out.resize(8 * idx->h_loff.size());
    std::memcpy(out.data(), idx->h_loff.data(), out.size());
    dtype = DT_I64;
  } else if (f == "IDS_") { out = d2h_bytes(idx->ids.p, n, st); dtype = DT_I64; }
  else if (f == "XD__") { out = d2h_bytes(idx->xd.p, (size_t)n * d, st); dtype = DT_F32; }
  else if (f == "XR__") { out = d2h_bytes(idx->xr.p, (size_t)n * r, st); dtype = DT_F32; }
  else if (f == "XN2_") { out = d2h_bytes(idx->xn2.p, n, st); dtype = DT_F32; }
  else if (f == "CODE") {
    mrq::DevBuf<uint8_t> lv((size_t)std::max<int64_t>(n * d, 1));
    mrq::export_levels(idx, lv.p, st);
    out = d2h_bytes(lv.p, (size_t)n * d, st);
    MRQ_CUDA(cudaStreamSynchronize(st));
    dtype = DT_U8;
  } else if (f == "SQ8C" || f == "SQ8L" || f == "SQ8S") {
    mrq::ensure_sq8(idx, st);
    if (f == "SQ8C") { out = d2h_bytes(idx->sq_codes.p, (size_t)n * d, st); dtype = DT_U8; }
    else { out = d2h_bytes(f == "SQ8L" ? idx->sq_lo.p : idx->sq_delta.p, d, st); dtype = DT_F32; }
  } else if ((f == "PQR_" || f == "PQC_" || f == "PQK_") && idx->pq_M > 0) {
    if (f == "PQR_") { out = d2h_bytes(idx->pq_R.p, (size_t)d * d, st); dtype = DT_F32; }
    else if (f == "PQC_") { out = d2h_bytes(idx->pq_C.p, (size_t)idx->pq_K * d, st); dtype = DT_F32; }
    else { out = d2h_bytes(idx->pq_codes.p, (size_t)n * idx->pq_M, st); dtype = DT_U8; }
  } else if (f == "FADD" || f == "FRES" || f == "FERR" ||
             ((f == "FRE1" || f == "FER1") && idx->fres1.p)) {
    const float* src = f == "FADD" ? idx->fadd.p : f == "FRES" ? idx->fres.p
                     : f == "FERR" ? idx->ferr.p : f == "FRE1" ? idx->fres1.p : idx->ferr1.p;
    mrq::DevBuf<float> t((size_t)std::max<int64_t>(n, 1));
    mrq::export_padded(idx, src, t.p, st);
    out = d2h_bytes(t.p, n, st);
    MRQ_CUDA(cudaStreamSynchronize(st));
    dtype = DT_F32;
  } else {
    mrq::fail(MRQ_EINVAL, "unknown field " + f);
  }
  MRQ_CUDA(cudaStreamSynchronize(st));
}

int mrq_index_export(const mrq_index* idx, const char* field, void* host_dst, size_t bytes) {
  return guarded([&] {
    MRQ_REQUIRE(idx && field && host_dst, "NULL argument");
    use_device(idx);
    std::vector<uint8_t> out;
    uint32_t dt = 0;
    export_field(idx, std::string(field, strnlen(field, 4)), out, dt, nullptr);
    MRQ_REQUIRE(bytes == out.size(), "destination size does not match the field size (" +
                                         std::to_string(out.size()) + " bytes)");
    std::memcpy(host_dst, out.data(), out.size());
  });
}

static const char* kTags[] = {"MU__", "LAM_", "W___", "CENT", "LOFF", "IDS_", "CODE",
                              "FADD", "FRES", "FERR", "XD__", "XR__", "XN2_", "FRE1", "FER1"};
constexpr uint32_t kRequiredTags = 13;  // FRE1 / FER1: written when the index holds them

int mrq_save(const mrq_index* idx, const char* path) {
  return guarded([&] {
    MRQ_REQUIRE(idx && path, "NULL argument");
    use_device(idx);
    FILE* f = std::fopen(path, "wb");
    if (!f) mrq::fail(MRQ_EIO, std::string("cannot open ") + path + " for writing");
    std::unique_ptr<FILE, int (*)(FILE*)> guard(f, std::fclose);
    auto put = [&](const void* p, size_t b) {
      if (b && std::fwrite(p, 1, b, f) != b) mrq::fail(MRQ_EIO, "write failed");
    };
    std::vector<const char*> tags(kTags, kTags + kRequiredTags);
    if (idx->fres1.p) { tags.push_back("FRE1"); tags.push_back("FER1"); }
    if (idx->pq_M > 0) { tags.push_back("PQR_"); tags.push_back("PQC_"); tags.push_back("PQK_"); }
    const uint32_t nsec = (uint32_t)tags.size();
    put(kMagic, 8);
    put(&kVersion, 4);
    put(&nsec, 4);
    const int32_t hdr[4] = {idx->D, idx->d, idx->bits, idx->nlist};
    put(&idx->n, 8);
    put(hdr, 16);
    for (uint32_t t = 0; t < nsec; ++t) {
      const char* tag = tags[t];
      std::vector<uint8_t> data;
      uint32_t dt = 0;
      export_field(idx, tag, data, dt, nullptr);
      uint64_t count = data.size() / dt_size(dt);
      put(tag, 4);
      put(&dt, 4);
      put(&count, 8);
      put(data.data(), data.size());
      static const uint8_t zeros[8] = {0};
      put(zeros, (8 - data.size() % 8) % 8);
    }
  });
}

// An index on the current device from the canonical (file) arrays: sections in the order
// MU__ LAM_ W___ CENT LOFF IDS_ CODE FADD FRES FERR XD__ XR__ XN2_ [FRE1 FER1], validated
// for sizes by the caller; the offsets, ids and code levels are checked here.
static std::unique_ptr<mrq_index> index_from_sections(int64_t n, int D, int d, int bits,
                                                      int nlist,
                                                      const std::vector<std::vector<uint8_t>>& sec,
                                                      bool sign_factors) {
  const int r = D - d;
  std::unique_ptr<mrq_index> idx(new mrq_index());
  MRQ_CUDA(cudaGetDevice(&idx->device));
  idx->n = n; idx->D = D; idx->d = d; idx->bits = bits; idx->nlist = nlist;
  idx->h_loff.resize(nlist + 1);
  std::memcpy(idx->h_loff.data(), sec[4].data(), 8 * (nlist + 1));
  if (idx->h_loff[0] != 0 || idx->h_loff[nlist] != n) mrq::fail(MRQ_EFORMAT, "bad list offsets");
  for (int j = 0; j < nlist; ++j)
    if (idx->h_loff[j + 1] < idx->h_loff[j]) mrq::fail(MRQ_EFORMAT, "bad list offsets");
  {
    const int64_t* ids = reinterpret_cast<const int64_t*>(sec[5].data());
    for (int64_t i = 0; i < n; ++i)
      if (ids[i] < 0 || ids[i] >= (int64_t(1) << 31)) mrq::fail(MRQ_EFORMAT, "id out of range");
    const uint8_t* lv = sec[6].data();
    for (size_t i = 0; i < sec[6].size(); ++i)
      if (lv[i] >> bits) mrq::fail(MRQ_EFORMAT, "code level exceeds 2^bits - 1");
  }
  cudaStream_t st = nullptr;
  auto up = [&](auto& buf, const std::vector<uint8_t>& data, size_t count) {
    buf.alloc(std::max<size_t>(count, 1));
    if (count) MRQ_CUDA(cudaMemcpyAsync(buf.p, data.data(), data.size(), cudaMemcpyHostToDevice, st));
  };
  up(idx->mu, sec[0], D);
  up(idx->lam, sec[1], D);
  up(idx->W, sec[2], (size_t)D * D);
  up(idx->cent, sec[3], (size_t)nlist * d);
  up(idx->ids, sec[5], n);
  up(idx->xd, sec[10], (size_t)n * d);
  up(idx->xr, sec[11], (size_t)n * r);
  up(idx->xn2, sec[12], n);
  mrq::DevBuf<uint8_t> lv;
  mrq::DevBuf<float> fa, fr, fe, fr1, fe1;
  up(lv, sec[6], (size_t)n * d);
  up(fa, sec[7], n);
  up(fr, sec[8], n);
  up(fe, sec[9], n);
  if (sign_factors) {
    up(fr1, sec[13], n);
    up(fe1, sec[14], n);
  }
  mrq::finalize_layout(idx.get(), lv.p, fa.p, fr.p, fe.p, st, fr1.p, fe1.p);
  MRQ_CUDA(cudaStreamSynchronize(st));
  return idx;
}

int mrq_load(const char* path, mrq_index** out) {
  return guarded([&] {
    MRQ_REQUIRE(path && out, "NULL argument");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) mrq::fail(MRQ_EIO, std::string("cannot open ") + path);
    std::unique_ptr<FILE, int (*)(FILE*)> guard(f, std::fclose);
    auto get = [&](void* p, size_t b) {
      if (b && std::fread(p, 1, b, f) != b) mrq::fail(MRQ_EFORMAT, "truncated index file");
    };
    char magic[8];
    uint32_t version = 0, nsec = 0;
    get(magic, 8);
    if (std::memcmp(magic, kMagic, 8) != 0) mrq::fail(MRQ_EFORMAT, "not an MRQ index file");
    get(&version, 4);
    if (version != kVersion) mrq::fail(MRQ_EFORMAT, "unsupported index file version");
    get(&nsec, 4);
    int64_t n = 0;
    int32_t hdr[4];
    get(&n, 8);
    get(hdr, 16);
    const int D = hdr[0], d = hdr[1], bits = hdr[2], nlist = hdr[3];
    if (!(n >= 1 && n < (int64_t(1) << 31) && D >= 32 && D <= 16384 && d >= 32 && d <= D &&
          d % 32 == 0 && d <= MRQ_MAX_D && bits >= 1 && bits <= 8 && nlist >= 1 &&
          nlist <= (1 << 20)))
      mrq::fail(MRQ_EFORMAT, "index header out of range");
    const int r = D - d;
    struct Want { const char* tag; uint32_t dt; uint64_t count; };
    const Want want[] = {
        {"MU__", DT_F32, (uint64_t)D}, {"LAM_", DT_F32, (uint64_t)D},
        {"W___", DT_F32, (uint64_t)D * D}, {"CENT", DT_F32, (uint64_t)nlist * d},
        {"LOFF", DT_I64, (uint64_t)nlist + 1}, {"IDS_", DT_I64, (uint64_t)n},
        {"CODE", DT_U8, (uint64_t)n * d}, {"FADD", DT_F32, (uint64_t)n},
        {"FRES", DT_F32, (uint64_t)n}, {"FERR", DT_F32, (uint64_t)n},
        {"XD__", DT_F32, (uint64_t)n * d}, {"XR__", DT_F32, (uint64_t)n * r},
        {"XN2_", DT_F32, (uint64_t)n}, {"FRE1", DT_F32, (uint64_t)n},
        {"FER1", DT_F32, (uint64_t)n}};
    constexpr int kWant = 15;
    std::vector<uint8_t> pq_sec[3];
    bool pq_seen[3] = {false, false, false};
    std::vector<std::vector<uint8_t>> sec(kWant);
    std::vector<bool> seen(kWant, false);
    for (uint32_t s = 0; s < nsec; ++s) {
      char tag[4];
      uint32_t dt;
      uint64_t count;
      get(tag, 4);
      get(&dt, 4);
      get(&count, 8);
      if (dt < DT_F32 || dt > DT_U8) mrq::fail(MRQ_EFORMAT, "bad section dtype");
      if (count > (uint64_t(1) << 40)) mrq::fail(MRQ_EFORMAT, "section too large");
      int which = -1;
      for (int w = 0; w < kWant; ++w)
        if (std::memcmp(tag, want[w].tag, 4) == 0) which = w;
      size_t bytes = count * dt_size(dt);
      std::vector<uint8_t> data(bytes);
      get(data.data(), bytes);
      uint8_t pad[8];
      get(pad, (8 - bytes % 8) % 8);
      const char* pq_tags[3] = {"PQR_", "PQC_", "PQK_"};
      for (int t = 0; t < 3; ++t)
        if (std::memcmp(tag, pq_tags[t], 4) == 0) {
          if (dt != (t == 2 ? DT_U8 : DT_F32)) mrq::fail(MRQ_EFORMAT, "PQ section has the wrong type");
          pq_sec[t] = std::move(data);
          pq_seen[t] = true;
        }
      if (which < 0) continue;  // unknown sections are skipped
      if (dt != want[which].dt || count != want[which].count)
        mrq::fail(MRQ_EFORMAT, std::string("section ") + want[which].tag + " has the wrong type or size");
      sec[which] = std::move(data);
      seen[which] = true;
    }
    for (int w = 0; w < (int)kRequiredTags; ++w)
      if (!seen[w]) mrq::fail(MRQ_EFORMAT, std::string("missing section ") + want[w].tag);
    if (seen[13] != seen[14]) mrq::fail(MRQ_EFORMAT, "FRE1 and FER1 come together");
    const bool sign_factors = seen[13] && bits > 1;
    if (pq_seen[0] || pq_seen[1] || pq_seen[2]) {
      if (!(pq_seen[0] && pq_seen[1] && pq_seen[2]))
        mrq::fail(MRQ_EFORMAT, "PQR_, PQC_ and PQK_ come together");
      const int64_t nr = pq_sec[0].size() / 4, nc = pq_sec[1].size() / 4, nk = pq_sec[2].size();
      const int64_t K = nc / d, M = nk / n;
      if (nr != (int64_t)d * d || nc % d || nk % n || M < 1 || d % M || K < 2 || K > 256 ||
          M * K > 4096)
        mrq::fail(MRQ_EFORMAT, "PQ sections have inconsistent sizes");
      for (uint8_t c : pq_sec[2])
        if (c >= K) mrq::fail(MRQ_EFORMAT, "PQ code exceeds K - 1");
    }
    std::unique_ptr<mrq_index> built = index_from_sections(n, D, d, bits, nlist, sec, sign_factors);
    if (pq_seen[0]) {
      const int K = (int)(pq_sec[1].size() / 4 / d), M = (int)(pq_sec[2].size() / n);
      mrq::pq_install(built.get(), M, K, reinterpret_cast<const float*>(pq_sec[0].data()),
                      reinterpret_cast<const float*>(pq_sec[1].data()), pq_sec[2].data(), nullptr);
    }
    *out = built.release();
  });
}

int mrq_pq_train(mrq_index* idx, int M, int K, int opq_iters, int km_iters,
                 const int64_t* init_rows, uint64_t seed) {
  return guarded([&] {
    MRQ_REQUIRE(idx != nullptr, "NULL index");
    MRQ_REQUIRE(M >= 1 && idx->d % M == 0, "M must divide d");
    MRQ_REQUIRE(K >= 2 && K <= 256 && K <= idx->n, "K must be in [2, min(256, n)]");
    MRQ_REQUIRE((int64_t)M * K <= 4096, "M * K must be <= 4096");
    MRQ_REQUIRE(opq_iters >= 0 && opq_iters <= 100 && km_iters >= 0 && km_iters <= 100,
                "opq_iters and km_iters must be in [0, 100]");
    std::vector<int64_t> rows(K);
    if (init_rows) {
      for (int c = 0; c < K; ++c) {
        MRQ_REQUIRE(init_rows[c] >= 0 && init_rows[c] < idx->n, "init_rows out of range");
        rows[c] = init_rows[c];
      }
    } else {  // K distinct rows: a partial Fisher-Yates shuffle driven by SplitMix64
      uint64_t x = seed ? seed : 1;
      auto next = [&x]() {
        uint64_t z = (x += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
      };
      std::map<int64_t, int64_t> swapped;
      auto at = [&](int64_t i) { auto it = swapped.find(i); return it == swapped.end() ? i : it->second; };
      for (int c = 0; c < K; ++c) {
        const int64_t j = c + (int64_t)(next() % (uint64_t)(idx->n - c));
        const int64_t vj = at(j), vc = at(c);
        swapped[j] = vc;
        swapped[c] = vj;
        rows[c] = vj;
      }
    }
    use_device(idx);
    mrq::pq_train(idx, M, K, opq_iters, km_iters, rows.data(), nullptr);
  });
}

int mrq_shard_plan(const int64_t* list_sizes, int nlist, int nshards, int32_t* owner) {
  return guarded([&] { mrq::shard_plan(list_sizes, nlist, nshards, owner); });
}

int mrq_index_shard(const mrq_index* idx, int nshards, int shard, mrq_index** out) {
  return guarded([&] {
    MRQ_REQUIRE(idx && out, "NULL argument");
    *out = nullptr;
    MRQ_REQUIRE(nshards >= 1 && nshards <= idx->nlist, "need 1 <= nshards <= nlist");
    MRQ_REQUIRE(shard >= 0 && shard < nshards, "need 0 <= shard < nshards");
    use_device(idx);
    const int nlist = idx->nlist, D = idx->D, d = idx->d, r = D - d;
    std::vector<int64_t> sizes(nlist), loff(nlist + 1, 0), keep;
    for (int j = 0; j < nlist; ++j) sizes[j] = idx->h_loff[j + 1] - idx->h_loff[j];
    std::vector<int32_t> owner(nlist);
    mrq::shard_plan(sizes.data(), nlist, nshards, owner.data());
    for (int j = 0; j < nlist; ++j) {
      if (owner[j] == shard)
        for (int64_t i = idx->h_loff[j]; i < idx->h_loff[j + 1]; ++i) keep.push_back(i);
      loff[j + 1] = (int64_t)keep.size();
    }
    const int64_t m = (int64_t)keep.size();
    MRQ_REQUIRE(m >= 1, "the shard would hold no vector");
    const bool sign = idx->fres1.p != nullptr;
    const int nsec = sign ? 15 : 13;
    // bytes per row of the list-major arrays (0: a global array, copied whole)
    const size_t row_bytes[15] = {0, 0, 0, 0, 0, 8, (size_t)d, 4, 4, 4, 4 * (size_t)d,
                                  4 * (size_t)r, 4, 4, 4};
    std::vector<std::vector<uint8_t>> sec(15);
    for (int t = 0; t < nsec; ++t) {
      if (t == 4) {  // LOFF
        sec[4].resize(8 * loff.size());
        std::memcpy(sec[4].data(), loff.data(), sec[4].size());
        continue;
      }
      std::vector<uint8_t> data;
      uint32_t dt = 0;
      export_field(idx, kTags[t], data, dt, nullptr);
      const size_t rb = row_bytes[t];
      if (rb == 0) {
        sec[t] = std::move(data);
        continue;
      }
      sec[t].resize(rb * (size_t)m);
      for (int64_t i = 0; i < m; ++i)
        std::memcpy(sec[t].data() + rb * i, data.data() + rb * keep[i], rb);
    }
    std::unique_ptr<mrq_index> built =
        index_from_sections(m, D, d, idx->bits, nlist, sec, sign && idx->bits > 1);
    if (idx->pq_M > 0) {  // the OPQ: the same rotation and codebooks, the shard's codes
      std::vector<uint8_t> R, C, K;
      uint32_t dt = 0;
      export_field(idx, "PQR_", R, dt, nullptr);
      export_field(idx, "PQC_", C, dt, nullptr);
      export_field(idx, "PQK_", K, dt, nullptr);
      const size_t M = (size_t)idx->pq_M;
      std::vector<uint8_t> ks(M * (size_t)m);
      for (int64_t i = 0; i < m; ++i) std::memcpy(ks.data() + M * i, K.data() + M * keep[i], M);
      mrq::pq_install(built.get(), idx->pq_M, idx->pq_K, reinterpret_cast<const float*>(R.data()),
                      reinterpret_cast<const float*>(C.data()), ks.data(), nullptr);
    }
    *out = built.release();
  });
}

int mrq_merge_topk(const int64_t* ids, const float* dists, int nparts, int64_t nq, int k,
                   void* cuda_stream, int64_t* out_ids, float* out_dists) {
  return guarded([&] {
    mrq::merge_topk(ids, dists, nparts, nq, k, (cudaStream_t)cuda_stream, out_ids, out_dists);
  });
}

void mrq_free(mrq_index* idx) {
  if (!idx) return;
  cudaSetDevice(idx->device);
  delete idx;
}

}  // extern "C"
