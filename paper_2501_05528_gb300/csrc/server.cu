// Continuous-batching compression server.
//
// A worker thread owns the device side.  Requests (host buffers, ideally
// pinned) wait in a FIFO; a request is admitted when a stream slot is free and
// its first-phase memory fits in the budget.  Phase 1 copies the inputs in,
// tessellates and reads back the two sizes the outputs depend on; phase 2,
// admitted when its exact memory fits, runs the whole pipeline and copies the
// results out.  Every admitted request runs on its own stream, so requests
// that arrive while others are on the GPU overlap with them; memory comes
// from the stream-ordered allocator and is returned as soon as a request's
// stream reaches its end.  Kernels are deterministic, so a request's result
// does not depend on what runs beside it.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace tblr;

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
  return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

struct Job {
  tblr_request req;
  uint64_t ticket = 0;
  double t_submit = 0, t_done = 0;
  int phase = 0;  // 0 queued, 1 sizing, 2 compressing, 3 done
  int status = TBLR_OK;
  int slot = -1;
  size_t mem1 = 0, mem2 = 0;
  std::vector<void *> bufs1, bufs2;
  tblr_layout lay{};
  int64_t *nf_off = nullptr;
  int32_t *mmax_dev = nullptr;
  int32_t m_max = 0;
  int64_t total = 0;
};

}  // namespace

struct tblr_server {
  int device = 0;
  size_t budget = 0, in_use = 0, peak = 0;
  int slots = 1;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> events;
  std::vector<int> free_slots;
  int64_t *host_sizes = nullptr;  // pinned: [slot][2] = {nf total, m_max}
  std::mutex mu;
  std::condition_variable cv, done_cv;
  std::deque<Job *> pending;
  std::vector<Job *> active;
  std::map<uint64_t, Job *> jobs;
  std::vector<double> latencies;
  uint64_t next_ticket = 1;
  double t_first = -1, t_last = 0;
  uint64_t completed = 0, failed = 0;
  bool stop = false;
  std::thread worker;
};

namespace {

int dalloc(tblr_server *S, Job *j, std::vector<void *> &bag, void **p, size_t bytes) {
  bytes = align256(bytes == 0 ? 256 : bytes);
  TBLR_CUDA(cudaMallocAsync(p, bytes, S->streams[j->slot]));
  bag.push_back(*p);
  return TBLR_OK;
}

void release(tblr_server *S, Job *j, std::vector<void *> &bag) {
  for (void *p : bag) cudaFreeAsync(p, S->streams[j->slot]);
  bag.clear();
}

size_t phase1_bytes(const Prob &P) {
  const size_t n = P.n, b = P.b;
  return align256(8 * n * P.d) * 2 + align256(8 * b * P.ell) + 2 * align256(8 * n * P.r) +
         2 * align256(4 * n) + 4 * align256(4 * (b + 1)) + align256(4 * b * P.s3) +
         align256(8 * (b * P.s3 + 1)) + 256 + 4096;
}

size_t phase2_bytes(const Prob &P, const tblr_problem *prob, int32_t m_max, int64_t total) {
  const size_t n = P.n, b = P.b, k = P.k;
  return align256(8 * n * 2 * P.C) + align256(8 * b * P.ell) + align256(8 * b * b) +
         align256(8 * b) + 2 * align256(8 * n * k) + align256(4 * b) + align256(8 * b * b * k * k) +
         align256(8 * (size_t)std::max<int64_t>(total, 1)) +
         align256(std::max(tblr_compress_workspace(prob, m_max), tblr_tessellate_workspace(prob)));
}

int start_phase1(tblr_server *S, Job *j) {
  Prob P;
  TBLR_TRY(check_problem(&j->req.prob, &P));
  cudaStream_t s = S->streams[j->slot];
  void *pts, *T, *G, *H, *ws;
  auto &B = j->bufs1;
  TBLR_TRY(dalloc(S, j, B, &pts, 8 * P.n * P.d));
  TBLR_TRY(dalloc(S, j, B, &T, 8 * P.b * P.ell));
  TBLR_TRY(dalloc(S, j, B, &G, 8 * P.n * P.r));
  TBLR_TRY(dalloc(S, j, B, &H, 8 * P.n * P.r));
  void *perm, *box, *off, *nbr, *nnbr, *col, *spts, *nfo;
  TBLR_TRY(dalloc(S, j, B, &perm, 4 * P.n));
  TBLR_TRY(dalloc(S, j, B, &box, 4 * P.n));
  TBLR_TRY(dalloc(S, j, B, &off, 4 * (P.b + 1)));
  TBLR_TRY(dalloc(S, j, B, &nbr, 4 * P.b * P.s3));
  TBLR_TRY(dalloc(S, j, B, &nnbr, 4 * (P.b + 1)));
  TBLR_TRY(dalloc(S, j, B, &col, 4 * (P.b + 1)));
  TBLR_TRY(dalloc(S, j, B, &spts, 8 * P.n * P.d));
  TBLR_TRY(dalloc(S, j, B, &nfo, 8 * (P.b * P.s3 + 1) + 256));
  const size_t tws = tblr_tessellate_workspace(&j->req.prob);
  TBLR_TRY(dalloc(S, j, B, &ws, tws));
  j->lay = tblr_layout{(int32_t *)perm, (int32_t *)box, (int32_t *)off, (int32_t *)nbr,
                       (int32_t *)nnbr, (int32_t *)col, (double *)spts};
  j->nf_off = (int64_t *)nfo;
  j->mmax_dev = (int32_t *)((char *)nfo + align256(8 * (P.b * P.s3 + 1)));
  const tblr_request &q = j->req;
  TBLR_CUDA(cudaMemcpyAsync(pts, q.points_h, 8 * P.n * P.d, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(T, q.T_h, 8 * P.b * P.ell, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(G, q.G_h, 8 * P.n * P.r, cudaMemcpyHostToDevice, s));
  TBLR_CUDA(cudaMemcpyAsync(H, q.H_h, 8 * P.n * P.r, cudaMemcpyHostToDevice, s));
  TBLR_TRY(tblr_tessellate(&q.prob, (const double *)pts, &j->lay, ws, tws, s));
  TBLR_TRY(tblr_nearfield_offsets(&q.prob, &j->lay, j->nf_off, j->mmax_dev, s));
  int64_t *hs = S->host_sizes + 2 * j->slot;
  TBLR_CUDA(cudaMemsetAsync(j->mmax_dev + 1, 0, 4, s));
  TBLR_CUDA(cudaMemcpyAsync(hs, j->nf_off + P.b * P.s3, 8, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(hs + 1, j->mmax_dev, 8, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaEventRecord(S->events[j->slot], s));
  return TBLR_OK;
}

int start_phase2(tblr_server *S, Job *j) {
  Prob P;
  TBLR_TRY(check_problem(&j->req.prob, &P));
  const tblr_request &q = j->req;
  cudaStream_t s = S->streams[j->slot];
  if (j->total > q.bnear_capacity) {
    set_error("request needs %lld near-field doubles, capacity %lld", (long long)j->total,
              (long long)q.bnear_capacity);
    return TBLR_EWORKSPACE;
  }
  auto &B = j->bufs2;
  void *yz, *z, *tau, *rho, *u, *v, *ranks, *at, *bn, *ws;
  TBLR_TRY(dalloc(S, j, B, &yz, 8 * P.n * 2 * P.C));
  TBLR_TRY(dalloc(S, j, B, &z, 8 * P.b * P.ell));
  TBLR_TRY(dalloc(S, j, B, &tau, 8 * P.b * P.b));
  TBLR_TRY(dalloc(S, j, B, &rho, 8 * P.b));
  TBLR_TRY(dalloc(S, j, B, &u, 8 * P.n * P.k));
  TBLR_TRY(dalloc(S, j, B, &v, 8 * P.n * P.k));
  TBLR_TRY(dalloc(S, j, B, &ranks, 4 * P.b));
  TBLR_TRY(dalloc(S, j, B, &at, 8 * P.b * P.b * P.k * P.k));
  TBLR_TRY(dalloc(S, j, B, &bn, 8 * std::max<int64_t>(j->total, 1)));
  const size_t wsb = tblr_compress_workspace(&q.prob, j->m_max);
  TBLR_TRY(dalloc(S, j, B, &ws, wsb));
  const double *pts = (const double *)j->bufs1[0], *T = (const double *)j->bufs1[1];
  const double *G = (const double *)j->bufs1[2], *H = (const double *)j->bufs1[3];
  (void)pts;
  TBLR_TRY(tblr_compress(&q.prob, &j->lay, nullptr, T, G, H, (double *)yz, (double *)z,
                         (double *)tau, (double *)rho, (double *)u, (double *)v, (int32_t *)ranks,
                         (double *)at, j->nf_off, j->m_max, (double *)bn, ws, wsb, s));
  TBLR_CUDA(cudaMemcpyAsync(q.perm_h, j->lay.perm, 4 * P.n, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.offsets_h, j->lay.offsets, 4 * (P.b + 1), cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.nbr_h, j->lay.nbr, 4 * P.b * P.s3, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.ranks_h, ranks, 4 * P.b, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.u_h, u, 8 * P.n * P.k, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.v_h, v, 8 * P.n * P.k, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaMemcpyAsync(q.at_h, at, 8 * P.b * P.b * P.k * P.k, cudaMemcpyDeviceToHost, s));
  if (j->total > 0)
    TBLR_CUDA(cudaMemcpyAsync(q.bnear_h, bn, 8 * j->total, cudaMemcpyDeviceToHost, s));
  TBLR_CUDA(cudaEventRecord(S->events[j->slot], s));
  return TBLR_OK;
}

void finish(tblr_server *S, Job *j, int status) {
  release(S, j, j->bufs1);
  release(S, j, j->bufs2);
  S->in_use -= j->mem1 + j->mem2;
  j->mem1 = j->mem2 = 0;
  j->status = status;
  j->phase = 3;
  j->t_done = now_ms();
  if (status == TBLR_OK) {
    S->latencies.push_back(j->t_done - j->t_submit);
    S->completed++;
    S->t_last = j->t_done;
  } else {
    S->failed++;
  }
  S->free_slots.push_back(j->slot);
  S->done_cv.notify_all();
}

void worker_loop(tblr_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lock(S->mu);
  while (true) {
    bool progressed = false;
    // Admission: a free slot and the first phase's memory.
    while (!S->pending.empty() && !S->free_slots.empty()) {
      Job *j = S->pending.front();
      Prob P;
      if (check_problem(&j->req.prob, &P) != TBLR_OK) {
        S->pending.pop_front();
        j->slot = -1;
        j->status = TBLR_EINVAL;
        j->phase = 3;
        S->failed++;
        progressed = true;
        continue;
      }
      const size_t need = phase1_bytes(P);
      if (S->in_use + need > S->budget && !S->active.empty()) break;
      S->pending.pop_front();
      j->slot = S->free_slots.back();
      S->free_slots.pop_back();
      j->mem1 = need;
      S->in_use += need;
      S->peak = std::max(S->peak, S->in_use);
      j->phase = 1;
      S->active.push_back(j);
      const int st = start_phase1(S, j);
      if (st != TBLR_OK) finish(S, j, st);
      progressed = true;
    }
    // Progress of admitted requests.  A sized request that does not fit waits
    // for memory held by others, unless no request is compressing (nothing would
    // free memory): then the oldest sized request proceeds over budget.
    bool any_phase2 = false;
    for (Job *x : S->active) any_phase2 |= x->phase == 2;
    bool forced = false;
    for (size_t a = 0; a < S->active.size();) {
      Job *j = S->active[a];
      if (j->phase == 3) {
        S->active.erase(S->active.begin() + a);
        S->done_cv.notify_all();
        progressed = true;
        continue;
      }
      const cudaError_t q = cudaEventQuery(S->events[j->slot]);
      if (q == cudaErrorNotReady) {
        ++a;
        continue;
      }
      if (q != cudaSuccess) {
        set_error("request %llu failed on the device: %s", (unsigned long long)j->ticket,
                  cudaGetErrorString(q));
        finish(S, j, TBLR_ECUDA);
        progressed = true;
        continue;
      }
      if (j->phase == 1) {
        j->total = S->host_sizes[2 * j->slot];
        j->m_max = (int32_t)S->host_sizes[2 * j->slot + 1];
        Prob P;
        check_problem(&j->req.prob, &P);
        const size_t need = phase2_bytes(P, &j->req.prob, j->m_max, j->total);
        if (S->in_use + need > S->budget && (any_phase2 || forced)) {
          ++a;  // wait for memory held by others
          continue;
        }
        forced = forced || S->in_use + need > S->budget;
        any_phase2 = true;
        j->mem2 = need;
        S->in_use += need;
        S->peak = std::max(S->peak, S->in_use);
        j->phase = 2;
        const int st = start_phase2(S, j);
        if (st != TBLR_OK) finish(S, j, st);
      } else if (j->phase == 2) {
        finish(S, j, TBLR_OK);
      }
      progressed = true;
    }
    if (S->stop && S->pending.empty() && S->active.empty()) break;
    if (!progressed) S->cv.wait_for(lock, std::chrono::microseconds(50));
  }
}

}  // namespace

extern "C" int tblr_server_create(tblr_server **out, int device, size_t mem_budget_bytes,
                                  int max_inflight) {
  TBLR_REQUIRE(out != nullptr, "out is NULL");
  TBLR_REQUIRE(max_inflight >= 1 && max_inflight <= 64, "max_inflight must be in [1, 64]");
  TBLR_REQUIRE(mem_budget_bytes > 0, "memory budget must be positive");
  TBLR_CUDA(cudaSetDevice(device));
  tblr_server *S = new tblr_server;
  S->device = device;
  S->budget = mem_budget_bytes;
  S->slots = max_inflight;
  for (int i = 0; i < max_inflight; ++i) {
    cudaStream_t s;
    cudaEvent_t e;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      delete S;
      set_error("could not create streams/events");
      return TBLR_ECUDA;
    }
    S->streams.push_back(s);
    S->events.push_back(e);
    S->free_slots.push_back(max_inflight - 1 - i);
  }
  if (cudaMallocHost(&S->host_sizes, sizeof(int64_t) * 2 * max_inflight) != cudaSuccess) {
    delete S;
    set_error("could not allocate pinned size buffers");
    return TBLR_ECUDA;
  }
  S->worker = std::thread(worker_loop, S);
  *out = S;
  return TBLR_OK;
}

extern "C" int tblr_server_submit(tblr_server *S, const tblr_request *req, uint64_t *ticket) {
  TBLR_REQUIRE(S && req && ticket, "NULL argument");
  Prob P;
  TBLR_TRY(check_problem(&req->prob, &P));
  TBLR_REQUIRE(req->prob.kernel != TBLR_KERNEL_DENSE, "the server takes kernel operators");
  TBLR_REQUIRE(req->points_h && req->T_h && req->G_h && req->H_h && req->perm_h &&
                   req->offsets_h && req->nbr_h && req->ranks_h && req->u_h && req->v_h &&
                   req->at_h && req->bnear_h,
               "request buffers must be non-NULL");
  Job *j = new Job;
  j->req = *req;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    j->ticket = S->next_ticket++;
    j->t_submit = now_ms();
    if (S->t_first < 0) S->t_first = j->t_submit;
    S->jobs[j->ticket] = j;
    S->pending.push_back(j);
  }
  S->cv.notify_all();
  *ticket = j->ticket;
  return TBLR_OK;
}

extern "C" int tblr_server_wait(tblr_server *S, uint64_t ticket, int timeout_ms, int *status,
                                double *latency_ms) {
  TBLR_REQUIRE(S != nullptr, "server is NULL");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->jobs.find(ticket);
  TBLR_REQUIRE(it != S->jobs.end(), "unknown ticket %llu", (unsigned long long)ticket);
  Job *j = it->second;
  const bool ok = S->done_cv.wait_for(lock, std::chrono::milliseconds(timeout_ms),
                                      [&] { return j->phase == 3; });
  if (!ok) {
    set_error("request %llu not finished after %d ms", (unsigned long long)ticket, timeout_ms);
    return TBLR_ETIMEOUT;
  }
  if (status) *status = j->status;
  if (latency_ms) *latency_ms = j->t_done - j->t_submit;
  S->jobs.erase(it);
  delete j;
  return TBLR_OK;
}

extern "C" int tblr_server_stats(tblr_server *S, tblr_server_report *out) {
  TBLR_REQUIRE(S && out, "NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  std::vector<double> l = S->latencies;
  std::sort(l.begin(), l.end());
  auto pct = [&](double q) {
    if (l.empty()) return 0.0;
    const double pos = q * (l.size() - 1);
    const size_t lo = (size_t)pos;
    const size_t hi = std::min(lo + 1, l.size() - 1);
    return l[lo] + (pos - lo) * (l[hi] - l[lo]);
  };
  out->completed = S->completed;
  out->failed = S->failed;
  out->pending = S->pending.size();
  out->active = S->active.size();
  out->p50_ms = pct(0.5);
  out->p99_ms = pct(0.99);
  const double span = S->t_last - S->t_first;
  out->throughput = (S->completed > 0 && span > 0) ? S->completed / (span / 1e3) : 0.0;
  out->mem_in_use = S->in_use;
  out->mem_peak = S->peak;
  return TBLR_OK;
}

extern "C" void tblr_server_destroy(tblr_server *S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  for (auto &kv : S->jobs) delete kv.second;
  for (auto s : S->streams) cudaStreamDestroy(s);
  for (auto e : S->events) cudaEventDestroy(e);
  if (S->host_sizes) cudaFreeHost(S->host_sizes);
  delete S;
}
