// Continuous-batching query server (the serving form of the query path).
//
// Requests (one query, its own k and nprobe) are queued by mrq_submit.  A
// scheduler thread groups pending requests with equal (k, nprobe), oldest
// first, and launches a group as one batch when a slot is free and the batch's
// scratch fits the device-memory budget; a group smaller than max_batch waits at
// most max_wait_us for company.  Every slot owns a stream, pinned staging
// buffers and its own search scratch, so batches admitted while others run
// overlap on the device.  Completed batches are detected with events; results
// and per-request latency (submit to completion) are kept until mrq_poll
// collects them.  Each request's answer is the same as a standalone mrq_search
// of that query (the thresholds do not depend on batch composition).
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <unordered_set>

#include "common.cuh"

namespace {

using Clock = std::chrono::steady_clock;
double now_us() {
  return std::chrono::duration<double, std::micro>(Clock::now().time_since_epoch()).count();
}

struct Req {
  uint64_t ticket;
  int k, nprobe;
  std::vector<float> q;
  double t_submit;
};
struct Result {
  int rc = MRQ_OK;
  std::vector<int64_t> ids;
  std::vector<float> dists;
};
struct Slot {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  mrq::Workspace ws;
  mrq::DevBuf<float> dq;
  mrq::DevBuf<int64_t> dids, dstats;
  mrq::DevBuf<float> dd;
  float* hq = nullptr;
  int64_t* hids = nullptr;
  float* hd = nullptr;
  size_t hcap = 0;  // queries the pinned buffers hold
  std::vector<Req> reqs;
  bool busy = false;
  size_t bytes = 0;
  int k = 0;
};

}  // namespace

struct mrq_server {
  mrq_index* idx = nullptr;
  mrq_server_opts opt{};
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::map<std::pair<int, int>, std::deque<Req>> pending;  // FIFO per (k, nprobe) group
  int64_t n_pending = 0;
  std::unordered_map<uint64_t, Result> done;
  std::unordered_set<uint64_t> live;  // submitted and not yet released by a poll
  std::deque<uint64_t> completed;     // tickets in completion order (mrq_poll_completed)
  std::vector<Slot> slots;
  uint64_t next_ticket = 1;
  bool stop = false;
  size_t inflight_bytes = 0;
  int64_t n_done = 0, n_batches = 0;
  std::vector<double> lat;  // latencies (us) of completed requests
  double t_first = 0, t_last = 0;
  int fatal = MRQ_OK;
  std::string fatal_msg;
};

namespace {

void release_slot(Slot& s) {
  if (s.hq) cudaFreeHost(s.hq);
  if (s.hids) cudaFreeHost(s.hids);
  if (s.hd) cudaFreeHost(s.hd);
  if (s.ev) cudaEventDestroy(s.ev);
  if (s.st) cudaStreamDestroy(s.st);
  s.hq = nullptr; s.hids = nullptr; s.hd = nullptr; s.ev = nullptr; s.st = nullptr;
}

// move finished batches into the result map (called with the lock held)
void collect(mrq_server* sv) {
  for (auto& s : sv->slots) {
    if (!s.busy) continue;
    cudaError_t e = cudaEventQuery(s.ev);
    if (e == cudaErrorNotReady) continue;
    const double t = now_us();
    for (size_t i = 0; i < s.reqs.size(); ++i) {
      Result r;
      if (e != cudaSuccess) {
        r.rc = MRQ_ECUDA;
      } else {
        r.ids.assign(s.hids + i * s.k, s.hids + (i + 1) * s.k);
        r.dists.assign(s.hd + i * s.k, s.hd + (i + 1) * s.k);
      }
      sv->lat.push_back(t - s.reqs[i].t_submit);
      sv->done.emplace(s.reqs[i].ticket, std::move(r));
      sv->completed.push_back(s.reqs[i].ticket);
    }
    if (e != cudaSuccess) cudaGetLastError();
    sv->n_done += (int64_t)s.reqs.size();
    sv->t_last = t;
    sv->inflight_bytes -= s.bytes;
    s.reqs.clear();
    s.busy = false;
    sv->cv_done.notify_all();
  }
}

// stage and launch one batch on a free slot (called without the lock: only the
// scheduler thread touches slots)
void launch(mrq_server* sv, Slot& s, std::vector<Req>&& batch, size_t bytes) {
  mrq_index* idx = sv->idx;
  const int64_t n = (int64_t)batch.size();
  const int D = idx->D, k = batch[0].k, nprobe = batch[0].nprobe;
  if ((size_t)n * std::max(k, 1) > s.hcap * (size_t)sv->opt.max_k || (size_t)n > s.hcap) {
    mrq::fail(MRQ_EINVAL, "batch larger than the slot");
  }
  for (int64_t i = 0; i < n; ++i) std::memcpy(s.hq + i * D, batch[i].q.data(), 4 * D);
  s.dq.reserve((size_t)n * D);
  s.dids.reserve((size_t)n * k);
  s.dd.reserve((size_t)n * k);
  s.dstats.reserve((size_t)n * 3);
  MRQ_CUDA(cudaMemcpyAsync(s.dq.p, s.hq, 4 * n * D, cudaMemcpyHostToDevice, s.st));
  mrq::search_batch(idx, s.ws, s.dq.p, n, k, nprobe, sv->opt.search, s.dids.p, s.dd.p,
                    s.dstats.p, s.st);
  MRQ_CUDA(cudaMemcpyAsync(s.hids, s.dids.p, 8 * n * k, cudaMemcpyDeviceToHost, s.st));
  MRQ_CUDA(cudaMemcpyAsync(s.hd, s.dd.p, 4 * n * k, cudaMemcpyDeviceToHost, s.st));
  MRQ_CUDA(cudaEventRecord(s.ev, s.st));
  s.k = k;
  s.bytes = bytes;
  s.reqs = std::move(batch);
}

void scheduler(mrq_server* sv) {
  cudaSetDevice(sv->idx->device);
  std::unique_lock<std::mutex> lk(sv->mu);
  while (true) {
    collect(sv);
    bool busy_any = false;
    for (auto& s : sv->slots) busy_any |= s.busy;
    if (sv->stop && sv->n_pending == 0 && !busy_any) break;
    bool launched = false;
    if (sv->n_pending > 0 && sv->fatal == MRQ_OK) {
      Slot* free_slot = nullptr;
      for (auto& s : sv->slots)
        if (!s.busy) { free_slot = &s; break; }
      if (free_slot) {
        // the group whose oldest request waited longest
        auto gsel = sv->pending.end();
        for (auto g = sv->pending.begin(); g != sv->pending.end(); ++g)
          if (!g->second.empty() &&
              (gsel == sv->pending.end() || g->second.front().t_submit < gsel->second.front().t_submit))
            gsel = g;
        auto& q = gsel->second;
        const int k = gsel->first.first, np = gsel->first.second;
        const int64_t cnt = std::min<int64_t>((int64_t)q.size(), sv->opt.max_batch);
        const bool full = cnt >= sv->opt.max_batch;
        const bool old = now_us() - q.front().t_submit >= sv->opt.max_wait_us;
        if (full || old || sv->stop) {
          const size_t bytes = mrq::batch_scratch_bytes(sv->idx, cnt, k, np);
          if (sv->inflight_bytes == 0 || sv->inflight_bytes + bytes <= sv->opt.mem_budget) {
            std::vector<Req> batch;
            batch.reserve(cnt);
            for (int64_t i = 0; i < cnt; ++i) {
              batch.push_back(std::move(q.front()));
              q.pop_front();
            }
            sv->n_pending -= cnt;
            if (q.empty()) sv->pending.erase(gsel);
            std::vector<uint64_t> tks;
            for (auto& r : batch) tks.push_back(r.ticket);
            free_slot->busy = true;
            sv->inflight_bytes += bytes;
            sv->n_batches++;
            bool ok = true;
            mrq::Error err{MRQ_OK, ""};
            lk.unlock();
            try {
              launch(sv, *free_slot, std::move(batch), bytes);
            } catch (const mrq::Error& e) {
              ok = false;
              err = e;
            }
            lk.lock();
            if (ok) {
              launched = true;
            } else {
              const mrq::Error& e = err;
              sv->inflight_bytes -= bytes;
              // the batch failed before it ran: its requests complete with the error
              sv->fatal = e.code;
              sv->fatal_msg = e.msg;
              for (uint64_t t : tks) {
                sv->done[t].rc = e.code;
                sv->completed.push_back(t);
              }
              free_slot->reqs.clear();
              free_slot->busy = false;
              sv->cv_done.notify_all();
            }
          }
        }
      }
    }
    if (!launched) {
      // nothing to launch now: sleep briefly (woken by submit/stop)
      sv->cv_work.wait_for(lk, std::chrono::microseconds(busy_any ? 20 : 200));
    }
  }
}

template <class F>
int srv_guard(F&& f) {
  try {
    f();
    mrq::set_last_error("");
    return MRQ_OK;
  } catch (const mrq::Error& e) {
    mrq::set_last_error(e.msg);
    return e.code;
  } catch (const std::exception& e) {
    mrq::set_last_error(e.what());
    return MRQ_EINVAL;
  }
}

}  // namespace

extern "C" {

void mrq_server_opts_default(mrq_server_opts* o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->mem_budget = (size_t)8 << 30;
  o->max_batch = 4096;
  o->max_inflight = 4;
  o->max_wait_us = 300;
  o->max_k = 128;
  mrq_search_opts_default(&o->search);
}

int mrq_server_start(mrq_index* idx, const mrq_server_opts* opt, mrq_server** out) {
  return srv_guard([&] {
    MRQ_REQUIRE(idx && out, "NULL argument");
    *out = nullptr;
    mrq_server_opts o;
    mrq_server_opts_default(&o);
    if (opt) o = *opt;
    MRQ_REQUIRE(o.max_batch >= 1 && o.max_batch <= 65536, "max_batch must be in [1, 65536]");
    MRQ_REQUIRE(o.max_inflight >= 1 && o.max_inflight <= 64, "max_inflight must be in [1, 64]");
    MRQ_REQUIRE(o.max_k >= 1 && o.max_k <= 1024, "max_k must be in [1, 1024]");
    MRQ_REQUIRE(o.max_wait_us >= 0, "max_wait_us must be >= 0");
    MRQ_REQUIRE(o.search.refine == 0 || o.search.refine == 1, "refine must be 0 or 1");
    MRQ_REQUIRE((o.search.mode != MRQ_MODE_SQ8 && o.search.mode != MRQ_MODE_PQ) ||
                    (o.max_k <= 128 && o.max_k <= o.search.rerank && o.search.rerank <= 65536),
                "MRQ_MODE_SQ8 and MRQ_MODE_PQ need max_k <= 128 and max_k <= rerank <= 65536");
    MRQ_REQUIRE(o.search.mode != MRQ_MODE_PQ || idx->pq_M > 0, "MRQ_MODE_PQ needs an OPQ");
    if (o.search.mode == MRQ_MODE_SQ8) mrq::ensure_sq8(idx, nullptr);
    if (mrq::refine_active(idx, o.search)) {
      MRQ_REQUIRE(idx->fres1.p != nullptr, "refine needs the sign-plane factors (FRE1/FER1)");
      MRQ_REQUIRE(o.search.query_bits > 0, "refine needs a quantized query (query_bits >= 1)");
      MRQ_REQUIRE(o.max_k <= 128, "refine needs max_k <= 128");
    }
    MRQ_CUDA(cudaSetDevice(idx->device));
    std::unique_ptr<mrq_server> sv(new mrq_server());
    idx->prof_on = false;  // the scheduler thread never records profiling events
    sv->idx = idx;
    sv->opt = o;
    sv->slots.resize(o.max_inflight);
    for (auto& s : sv->slots) {
      MRQ_CUDA(cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking));
      MRQ_CUDA(cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming));
      s.hcap = o.max_batch;
      MRQ_CUDA(cudaMallocHost(&s.hq, (size_t)4 * o.max_batch * idx->D));
      MRQ_CUDA(cudaMallocHost(&s.hids, (size_t)8 * o.max_batch * o.max_k));
      MRQ_CUDA(cudaMallocHost(&s.hd, (size_t)4 * o.max_batch * o.max_k));
    }
    sv->t_first = now_us();
    mrq_server* raw = sv.get();
    sv->th = std::thread(scheduler, raw);
    *out = sv.release();
  });
}

int mrq_submit(mrq_server* sv, const float* q, int k, int nprobe, uint64_t* ticket) {
  return srv_guard([&] {
    MRQ_REQUIRE(sv && q && ticket, "NULL argument");
    MRQ_REQUIRE(k >= 1 && k <= sv->opt.max_k, "k must be in [1, max_k]");
    MRQ_REQUIRE(nprobe >= 1 && nprobe <= sv->idx->nlist && nprobe <= 16384, "nprobe out of range");
    MRQ_REQUIRE(!mrq::refine_active(sv->idx, sv->opt.search) || nprobe <= mrq::REFINE_MAX_NPROBE,
                "refine needs nprobe <= 4096");
    Req r;
    r.k = k;
    r.nprobe = nprobe;
    r.q.assign(q, q + sv->idx->D);
    r.t_submit = now_us();
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->fatal != MRQ_OK) mrq::fail(sv->fatal, "server stopped after an error: " + sv->fatal_msg);
      MRQ_REQUIRE(!sv->stop, "server is stopping");
      r.ticket = sv->next_ticket++;
      *ticket = r.ticket;
      sv->live.insert(r.ticket);
      sv->pending[std::make_pair(r.k, r.nprobe)].push_back(std::move(r));
      sv->n_pending++;
    }
    sv->cv_work.notify_one();
  });
}

int mrq_poll(mrq_server* sv, uint64_t ticket, int64_t* ids, float* dists, int wait_ms) {
  int rc = srv_guard([&] {
    MRQ_REQUIRE(sv && ids && dists, "NULL argument");
    std::unique_lock<std::mutex> lk(sv->mu);
    MRQ_REQUIRE(sv->live.count(ticket) > 0, "unknown or already released ticket");
    auto ready = [&] { return sv->done.count(ticket) > 0; };
    if (!ready() && wait_ms > 0)
      sv->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), ready);
    auto it = sv->done.find(ticket);
    if (it == sv->done.end()) mrq::fail(1, "pending");
    sv->live.erase(ticket);
    if (it->second.rc != MRQ_OK) {
      int c = it->second.rc;
      sv->done.erase(it);
      mrq::fail(c, "the batch of this request failed");
    }
    std::copy(it->second.ids.begin(), it->second.ids.end(), ids);
    std::copy(it->second.dists.begin(), it->second.dists.end(), dists);
    sv->done.erase(it);
  });
  return rc;
}

int mrq_submit_many(mrq_server* sv, int64_t n, const float* q, const int* k, const int* nprobe,
                    uint64_t* tickets) {
  return srv_guard([&] {
    MRQ_REQUIRE(sv && q && k && nprobe && tickets && n >= 0, "bad argument");
    const int D = sv->idx->D;
    std::vector<Req> rs(n);
    const double t = now_us();
    for (int64_t i = 0; i < n; ++i) {
      MRQ_REQUIRE(k[i] >= 1 && k[i] <= sv->opt.max_k, "k must be in [1, max_k]");
      MRQ_REQUIRE(nprobe[i] >= 1 && nprobe[i] <= sv->idx->nlist && nprobe[i] <= 16384,
                  "nprobe out of range");
      MRQ_REQUIRE(!mrq::refine_active(sv->idx, sv->opt.search) ||
                      nprobe[i] <= mrq::REFINE_MAX_NPROBE,
                  "refine needs nprobe <= 4096");
      rs[i].k = k[i];
      rs[i].nprobe = nprobe[i];
      rs[i].q.assign(q + i * D, q + (i + 1) * D);
      rs[i].t_submit = t;
    }
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (sv->fatal != MRQ_OK) mrq::fail(sv->fatal, "server stopped after an error: " + sv->fatal_msg);
      MRQ_REQUIRE(!sv->stop, "server is stopping");
      for (int64_t i = 0; i < n; ++i) {
        rs[i].ticket = sv->next_ticket++;
        tickets[i] = rs[i].ticket;
        sv->live.insert(rs[i].ticket);
        sv->pending[std::make_pair(rs[i].k, rs[i].nprobe)].push_back(std::move(rs[i]));
        sv->n_pending++;
      }
    }
    sv->cv_work.notify_one();
  });
}

int mrq_poll_many(mrq_server* sv, int64_t n, const uint64_t* tickets, int kmax, int64_t* ids,
                  float* dists, int32_t* status) {
  return srv_guard([&] {
    MRQ_REQUIRE(sv && tickets && ids && dists && status && n >= 0 && kmax >= 1, "bad argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    for (int64_t i = 0; i < n; ++i) {
      auto it = sv->done.find(tickets[i]);
      if (it == sv->done.end()) {
        status[i] = sv->live.count(tickets[i]) ? 1 : MRQ_EINVAL;
        continue;
      }
      status[i] = it->second.rc;
      sv->live.erase(tickets[i]);
      const size_t kk = std::min<size_t>(it->second.ids.size(), (size_t)kmax);
      for (size_t j = 0; j < (size_t)kmax; ++j) {
        ids[i * kmax + j] = j < kk ? it->second.ids[j] : -1;
        dists[i * kmax + j] = j < kk ? it->second.dists[j] : __builtin_huge_valf();
      }
      sv->done.erase(it);
    }
  });
}

int64_t mrq_poll_completed(mrq_server* sv, int64_t max_n, int kmax, uint64_t* tickets,
                           int64_t* ids, float* dists, int32_t* status) {
  int64_t got = 0;
  int rc = srv_guard([&] {
    MRQ_REQUIRE(sv && tickets && ids && dists && status && max_n >= 0 && kmax >= 1, "bad argument");
    std::vector<std::pair<uint64_t, Result>> out;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      while ((int64_t)out.size() < max_n && !sv->completed.empty()) {
        const uint64_t t = sv->completed.front();
        sv->completed.pop_front();
        auto it = sv->done.find(t);
        if (it == sv->done.end()) continue;  // already released by mrq_poll
        out.emplace_back(t, std::move(it->second));
        sv->done.erase(it);
        sv->live.erase(t);
      }
    }
    for (size_t i = 0; i < out.size(); ++i) {
      tickets[i] = out[i].first;
      status[i] = out[i].second.rc;
      const auto& r = out[i].second;
      for (size_t j = 0; j < (size_t)kmax; ++j) {
        ids[i * kmax + j] = j < r.ids.size() ? r.ids[j] : -1;
        dists[i * kmax + j] = j < r.dists.size() ? r.dists[j] : __builtin_huge_valf();
      }
    }
    got = (int64_t)out.size();
  });
  return rc == MRQ_OK ? got : rc;
}

int mrq_server_stats(mrq_server* sv, mrq_server_stats_t* st) {
  return srv_guard([&] {
    MRQ_REQUIRE(sv && st, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(st, 0, sizeof(*st));
    st->completed = sv->n_done;
    st->batches = sv->n_batches;
    st->pending = sv->n_pending;
    std::vector<double> l = sv->lat;
    if (!l.empty()) {
      std::sort(l.begin(), l.end());
      st->p50_us = l[l.size() / 2];
      st->p99_us = l[std::min(l.size() - 1, (size_t)(0.99 * l.size()))];
      st->max_us = l.back();
      const double span = (sv->t_last - sv->t_first) * 1e-6;
      st->qps = span > 0 ? (double)sv->n_done / span : 0.0;
    }
  });
}

int mrq_server_reset_stats(mrq_server* sv) {
  return srv_guard([&] {
    MRQ_REQUIRE(sv, "NULL argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->lat.clear();
    sv->n_done = 0;
    sv->n_batches = 0;
    sv->t_first = sv->t_last = now_us();
  });
}

int mrq_server_stop(mrq_server* sv) {
  if (!sv) return MRQ_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
  }
  sv->cv_work.notify_all();
  if (sv->th.joinable()) sv->th.join();
  cudaSetDevice(sv->idx->device);
  for (auto& s : sv->slots) {
    if (s.st) cudaStreamSynchronize(s.st);
    release_slot(s);
  }
  const int rc = sv->fatal;
  delete sv;
  return rc;
}

}  // extern "C"
