// Batched compression of independent jobs (uneven N, box sizes, ranks and
// dimensions): planning, multi-stream execution and CUDA-graph capture.
//
// tblr_batch_plan tessellates every job once and reads back the sizes the
// near-field output depends on.  tblr_batch_run then enqueues every job's
// whole pipeline (tessellation, near-field offsets, tblr_compress) with no
// host synchronisation: jobs are dealt to worker streams largest first
// (estimated sketch work 2 n^2 (2 ell r)), the worker streams fork from and
// join back into the caller's stream with events, so small jobs fill the SMs
// that large ones leave idle and the whole batch can be captured into one CUDA
// graph (tblr_graph_create) and replayed with a single launch.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

using namespace tblr;

namespace {

constexpr int kMaxStreams = 32;

struct StreamPool {
  std::mutex mu;
  int device = -1;
  cudaStream_t s[kMaxStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kMaxStreams] = {};
};

StreamPool &pool() {
  static StreamPool p;
  return p;
}

int ensure_pool(int n) {
  StreamPool &P = pool();
  int dev = 0;
  TBLR_CUDA(cudaGetDevice(&dev));
  if (P.device != dev) {
    for (int i = 0; i < kMaxStreams; ++i) {
      P.s[i] = nullptr;
      P.join[i] = nullptr;
    }
    P.fork = nullptr;
    P.device = dev;
  }
  if (!P.fork) TBLR_CUDA(cudaEventCreateWithFlags(&P.fork, cudaEventDisableTiming));
  for (int i = 0; i < n; ++i) {
    if (!P.s[i]) TBLR_CUDA(cudaStreamCreateWithFlags(&P.s[i], cudaStreamNonBlocking));
    if (!P.join[i]) TBLR_CUDA(cudaEventCreateWithFlags(&P.join[i], cudaEventDisableTiming));
  }
  return TBLR_OK;
}

double job_cost(const tblr_job &j) {
  Prob P;
  if (check_problem(&j.prob, &P) != TBLR_OK) return 0.0;
  return 2.0 * (double)P.n * (double)P.n * 2.0 * (double)P.C;
}

int run_job(const tblr_job &j, void *stream) {
  TBLR_REQUIRE(j.ws_bytes >= tblr_tessellate_workspace(&j.prob), "job workspace too small");
  TBLR_TRY(tblr_tessellate(&j.prob, j.points, &j.lay, j.ws, j.ws_bytes, stream));
  TBLR_TRY(tblr_nearfield_offsets(&j.prob, &j.lay, j.nf_off, j.m_max_dev, stream));
  return tblr_compress(&j.prob, &j.lay, j.dense, j.T, j.G, j.H, j.yz, j.z, j.tau, j.rho, j.u, j.v,
                       j.ranks, j.at, j.nf_off, j.m_max, j.bnear, j.ws, j.ws_bytes, stream);
}

}  // namespace

extern "C" int tblr_batch_plan(int n_jobs, tblr_job *jobs, void *stream) {
  TBLR_REQUIRE(n_jobs >= 0 && (n_jobs == 0 || jobs != nullptr), "bad job list");
  cudaStream_t s = as_stream(stream);
  std::vector<int32_t> mmax(n_jobs);
  std::vector<int64_t> total(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    tblr_job &j = jobs[i];
    Prob P;
    TBLR_TRY(check_problem(&j.prob, &P));
    TBLR_REQUIRE(j.ws_bytes >= tblr_tessellate_workspace(&j.prob), "job %d: workspace too small", i);
    TBLR_TRY(tblr_tessellate(&j.prob, j.points, &j.lay, j.ws, j.ws_bytes, stream));
    TBLR_TRY(tblr_nearfield_offsets(&j.prob, &j.lay, j.nf_off, j.m_max_dev, stream));
    TBLR_CUDA(cudaMemcpyAsync(&mmax[i], j.m_max_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    TBLR_CUDA(cudaMemcpyAsync(&total[i], j.nf_off + P.b * P.s3, sizeof(int64_t),
                              cudaMemcpyDeviceToHost, s));
  }
  TBLR_CUDA(cudaStreamSynchronize(s));
  for (int i = 0; i < n_jobs; ++i) {
    jobs[i].m_max = mmax[i];
    jobs[i].nf_total = total[i];
  }
  return TBLR_OK;
}

extern "C" int tblr_batch_run(int n_jobs, const tblr_job *jobs, int n_streams, void *stream) {
  TBLR_REQUIRE(n_jobs >= 0 && (n_jobs == 0 || jobs != nullptr), "bad job list");
  TBLR_REQUIRE(n_streams >= 1 && n_streams <= kMaxStreams, "n_streams must be in [1, %d]",
               kMaxStreams);
  for (int i = 0; i < n_jobs; ++i) {
    TBLR_REQUIRE(jobs[i].bnear && jobs[i].ws, "job %d: missing output or workspace", i);
    TBLR_REQUIRE(jobs[i].ws_bytes >= tblr_compress_workspace(&jobs[i].prob, jobs[i].m_max),
                 "job %d: workspace smaller than tblr_compress_workspace", i);
  }
  StreamPool &P = pool();
  std::lock_guard<std::mutex> lock(P.mu);
  TBLR_TRY(ensure_pool(n_streams));
  cudaStream_t origin = as_stream(stream);
  // Longest-processing-time-first assignment to the least loaded stream.
  std::vector<int> order(n_jobs);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(),
            [&](int a, int b) { return job_cost(jobs[a]) > job_cost(jobs[b]); });
  std::vector<double> load(n_streams, 0.0);
  std::vector<std::vector<int>> lanes(n_streams);
  for (int id : order) {
    const int w = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    load[w] += job_cost(jobs[id]);
    lanes[w].push_back(id);
  }
  TBLR_CUDA(cudaEventRecord(P.fork, origin));
  for (int w = 0; w < n_streams; ++w) {
    TBLR_CUDA(cudaStreamWaitEvent(P.s[w], P.fork, 0));
    for (int id : lanes[w]) TBLR_TRY(run_job(jobs[id], P.s[w]));
    TBLR_CUDA(cudaEventRecord(P.join[w], P.s[w]));
    TBLR_CUDA(cudaStreamWaitEvent(origin, P.join[w], 0));
  }
  return TBLR_OK;
}

struct tblr_graph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

extern "C" int tblr_graph_create(int n_jobs, const tblr_job *jobs, int n_streams, void *stream,
                                 tblr_graph **out) {
  TBLR_REQUIRE(out != nullptr, "out is NULL");
  TBLR_REQUIRE(stream != nullptr, "capture needs a non-default stream");
  cudaStream_t s = as_stream(stream);
  TBLR_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  const int st = tblr_batch_run(n_jobs, jobs, n_streams, stream);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s, &g);
  if (st != TBLR_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) {
    set_error("stream capture failed: %s", cudaGetErrorString(e));
    return TBLR_ECUDA;
  }
  tblr_graph *G = new tblr_graph;
  G->graph = g;
  const cudaError_t ie = cudaGraphInstantiate(&G->exec, g, 0);
  if (ie != cudaSuccess) {
    cudaGraphDestroy(g);
    delete G;
    set_error("graph instantiation failed: %s", cudaGetErrorString(ie));
    return TBLR_ECUDA;
  }
  *out = G;
  return TBLR_OK;
}

extern "C" int tblr_graph_launch(tblr_graph *g, void *stream) {
  TBLR_REQUIRE(g != nullptr && g->exec != nullptr, "graph is NULL");
  TBLR_CUDA(cudaGraphLaunch(g->exec, as_stream(stream)));
  return TBLR_OK;
}

extern "C" void tblr_graph_destroy(tblr_graph *g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}
