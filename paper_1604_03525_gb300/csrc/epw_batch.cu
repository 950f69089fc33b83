// Batched linewidth over many systems of uneven size (Eq. (linewidthel) per
// system): one device workspace (jobs that run one after another on a branch
// share a region of it), tile parameters from a timing
// autotuner, and the whole batch captured as one CUDA graph whose jobs run
// on parallel branches.  Replaying the graph costs one launch on the host
// however many kernels the jobs hold.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <vector>

#include "epw_host.cuh"

#define BCK(call)                                                                                             \
  do {                                                                                                        \
    cudaError_t e_ = (call);                                                                                  \
    if (e_ != cudaSuccess)                                                                                    \
      return epwi_fail(e_ == cudaErrorMemoryAllocation ? EPW_ERR_OOM : EPW_ERR_CUDA, "%s: %s", #call,         \
                       cudaGetErrorString(e_));                                                               \
  } while (0)
#define BCKS(expr)                \
  do {                            \
    epw_status s_ = (expr);       \
    if (s_ != EPW_OK) return s_;  \
  } while (0)

namespace {

// ----------------------------------------------------------------- autotuner
// A job's path: the fused tensor-core kernel, the wide-shape form (one fused
// kernel or two per chunk of k), the staged tensor-core form, or the SIMT
// per-pair kernel (no tile knob).
enum Path { PATH_SIMT = 0, PATH_FUSED = 1, PATH_STAGED = 2, PATH_WIDE = 3 };

int job_path(const epw_model *m, int prec) {
  if (prec != EPW_BF16X3 && prec != EPW_TF32X3) return PATH_SIMT;
  if (tc_supported(m)) return PATH_FUSED;
  if (tcw_supported(m)) return PATH_WIDE;
  if (tc_staged_supported(m)) return PATH_STAGED;
  return -1;
}

int log2_floor(long x) {
  int b = 0;
  while (x > 1) {
    x >>= 1;
    b++;
  }
  return b;
}

// Tile choices move with the order of magnitude of the sizes: the key buckets
// nk and nq by powers of two.
std::string tune_key(const epw_model *m, int nk, int nq, int prec, int path) {
  char buf[160];
  snprintf(buf, sizeof(buf), "path%d nw%d nm%d nR%d k2^%d q2^%d prec%d", path, m->nw, m->nm, m->nRe,
           log2_floor(nk), log2_floor(nq), prec);
  return buf;
}

std::mutex g_mu;
std::map<std::string, EpwTune> g_cache;
bool g_loaded = false;

// File format, one entry per line: <key>|<a_block_bytes>|<staged_ct_bytes>[|<wide_form>]
void load_cache_file_locked() {
  if (g_loaded) return;
  g_loaded = true;
  const char *path = getenv("EPW_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "r");
  if (!f) return;
  char line[512];
  while (fgets(line, sizeof(line), f)) {
    char *b1 = strchr(line, '|');
    if (!b1) continue;
    char *b2 = strchr(b1 + 1, '|');
    if (!b2) continue;
    *b1 = 0;
    EpwTune t = epwi_default_tune();
    t.a_block_bytes = strtoull(b1 + 1, nullptr, 10);
    t.staged_ct_bytes = strtoull(b2 + 1, nullptr, 10);
    char *b3 = strchr(b2 + 1, '|');
    t.wide_form = b3 ? atoi(b3 + 1) : 0;
    g_cache[line] = t;
  }
  fclose(f);
}

void append_cache_file_locked(const std::string &key, const EpwTune &t) {
  const char *path = getenv("EPW_TUNE_CACHE");
  if (!path || !*path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%zu|%zu|%d\n", key.c_str(), t.a_block_bytes, t.staged_ct_bytes, t.wide_form);
  fclose(f);
}

std::vector<EpwTune> candidates(int path) {
  const EpwTune d = epwi_default_tune();
  std::vector<EpwTune> c;
  if (path == PATH_FUSED) {
    for (size_t mib : {16, 32, 48, 96}) c.push_back(EpwTune{mib << 20, d.staged_ct_bytes, 0, d.k_side_bytes});
  } else if (path == PATH_STAGED) {
    for (size_t gib : {1, 2, 4}) c.push_back(EpwTune{d.a_block_bytes, gib << 30, 0, d.k_side_bytes});
  } else {
    // wide shapes: the form single calls take (EPW_WIDE_FORM, default the paired fused kernel), so that
    // batch and single-call results agree bit for bit
    c.push_back(d);
  }
  return c;
}

// Times one candidate on the first nk_t k-points of the job (two runs, the
// second timed), in a scratch workspace of ws_bytes.
epw_status trial(const epw_linewidth_job &j, int nk_t, const EpwTune &t, char *ws, size_t ws_bytes, double *out,
                 cudaStream_t st, cudaEvent_t e0, cudaEvent_t e1, float *ms) {
  epw_model *m = const_cast<epw_model *>(j.model);
  Arena A{ws, ws_bytes, 0};
  LwPlan L;
  BCKS(epwi_plan_linewidth(A, m, nk_t, j.nq, j.params.precision, false, false, false, false, t, L));
  if (A.off > ws_bytes) return epwi_fail(EPW_ERR_OOM, "autotuner workspace too small");
  BCKS(epwi_linewidth_exec(m, nk_t, j.k, j.nq, j.q, j.wq, &j.params, L, out, st));
  BCK(cudaEventRecord(e0, st));
  BCKS(epwi_linewidth_exec(m, nk_t, j.k, j.nq, j.q, j.wq, &j.params, L, out, st));
  BCK(cudaEventRecord(e1, st));
  BCK(cudaEventSynchronize(e1));
  BCK(cudaEventElapsedTime(ms, e0, e1));
  return EPW_OK;
}

// Tile choice of a job: cached, or picked by timing every candidate.
epw_status tune_job(const epw_linewidth_job &j, int path, cudaStream_t st, EpwTune *out) {
  const std::string key = tune_key(j.model, j.nk, j.nq, j.params.precision, path);
  std::lock_guard<std::mutex> lk(g_mu);
  load_cache_file_locked();
  auto it = g_cache.find(key);
  if (it != g_cache.end()) {
    *out = it->second;
    return EPW_OK;
  }
  const std::vector<EpwTune> cand = candidates(path);
  if (cand.size() == 1) {
    *out = cand[0];
    g_cache[key] = cand[0];
    return EPW_OK;
  }
  // enough k for the tiles to repeat: the fused kernel's k groups fill the
  // SMs a few times over; the staged form runs a few chunks (16 k: its heaviest
  // shapes take seconds per trial over a 48^3 q grid)
  const int nk_t = std::min(j.nk, path == PATH_FUSED ? 608 : 16);
  size_t need = 0;
  for (const EpwTune &t : cand) {
    Arena A{nullptr, 0, 0};
    LwPlan L;
    BCKS(epwi_plan_linewidth(A, j.model, nk_t, j.nq, j.params.precision, false, false, false, false, t, L));
    need = std::max(need, A.off);
  }
  const size_t out_bytes = sizeof(double) * (size_t)nk_t * j.model->nw;
  char *ws = nullptr;
  BCK(cudaMalloc((void **)&ws, need + out_bytes + 512));
  double *outp = (double *)(ws + ((need + 255) & ~size_t(255)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 0.0f;
  int ib = -1;
  epw_status s = EPW_OK;
  for (size_t i = 0; i < cand.size() && s == EPW_OK; i++) {
    float ms = 0.0f;
    s = trial(j, nk_t, cand[i], ws, need, outp, st, e0, e1, &ms);
    if (s == EPW_OK && (ib < 0 || ms < best)) {
      best = ms;
      ib = (int)i;
    }
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(ws);
  if (s != EPW_OK) return s;
  *out = cand[ib];
  g_cache[key] = cand[ib];
  append_cache_file_locked(key, cand[ib]);
  return EPW_OK;
}

// Cost estimate (ms) used to balance the graph branches: algorithmic
// contraction flops over a per-form rate.
double job_cost(const epw_linewidth_job &j) {
  const epw_model *m = j.model;
  const double flops = 8.0 * m->nRe * m->nw * m->nw * (m->nm + 1) * (double)j.nk * j.nq;
  const int p = j.params.precision;
  const double rate = p == EPW_FP64 ? 0.5e12 : p == EPW_FP32 ? 10e12 : 200e12;
  return flops / rate * 1e3 + 0.05;
}

}  // namespace

struct epw_batch {
  int device = 0;
  std::vector<epw_linewidth_job> jobs;
  std::vector<LwPlan> plans;
  std::vector<EpwTune> tunes;
  std::vector<double> cost;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<cudaStream_t> streams;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> joins;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int nbranch = 1;
  size_t nodes = 0;
  std::vector<int> region;  // workspace region of each job (its branch in the 4-branch graph)
};

namespace {

constexpr int MAX_BRANCHES = 4;
constexpr int LONG_BATCH_MS = 5000;  // eager pass above which the branch count is not timed

// Enqueues every job on its branch stream (branch[i] < nb), forked from and
// joined back into streams[0].
epw_status enqueue_all(epw_batch *b, const std::vector<int> &branch, int nb) {
  BCK(cudaEventRecord(b->fork, b->streams[0]));
  for (int i = 1; i < nb; i++) BCK(cudaStreamWaitEvent(b->streams[i], b->fork, 0));
  for (size_t j = 0; j < b->jobs.size(); j++) {
    const epw_linewidth_job &J = b->jobs[j];
    if (J.nk == 0) continue;
    cudaStream_t st = b->streams[branch[j]];
    if (J.nq == 0) {
      BCK(cudaMemsetAsync(J.imsigma, 0, sizeof(double) * (size_t)J.nk * J.model->nw, st));
      continue;
    }
    BCKS(epwi_linewidth_exec(const_cast<epw_model *>(J.model), J.nk, J.k, J.nq, J.q, J.wq, &J.params, b->plans[j],
                             J.imsigma, st));
  }
  for (int i = 1; i < nb; i++) {
    BCK(cudaEventRecord(b->joins[i], b->streams[i]));
    BCK(cudaStreamWaitEvent(b->streams[0], b->joins[i], 0));
  }
  return EPW_OK;
}

// Longest-processing-time assignment of jobs to nb branches.
std::vector<int> assign(const epw_batch *b, int nb) {
  std::vector<int> order(b->jobs.size());
  for (size_t i = 0; i < order.size(); i++) order[i] = (int)i;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
  std::vector<double> load(nb, 0.0);
  std::vector<int> br(b->jobs.size(), 0);
  for (int j : order) {
    int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    br[j] = best;
    load[best] += b->cost[j];
  }
  return br;
}

epw_status capture(epw_batch *b, const std::vector<int> &branch, int nb, cudaGraph_t *g, cudaGraphExec_t *x) {
  BCK(cudaStreamBeginCapture(b->streams[0], cudaStreamCaptureModeThreadLocal));
  epw_status s = enqueue_all(b, branch, nb);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(b->streams[0], &graph);
  if (s != EPW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return s;
  }
  if (e != cudaSuccess) return epwi_fail(EPW_ERR_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
  e = cudaGraphInstantiate(x, graph, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(graph);
    return epwi_fail(EPW_ERR_CUDA, "graph instantiation failed: %s", cudaGetErrorString(e));
  }
  *g = graph;
  return EPW_OK;
}

void destroy(epw_batch *b) {
  if (!b) return;
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  if (b->fork) cudaEventDestroy(b->fork);
  for (cudaEvent_t e : b->joins)
    if (e) cudaEventDestroy(e);
  if (b->ws) cudaFree(b->ws);
  delete b;
}

epw_status create_impl(int njobs, const epw_linewidth_job *jobs, epw_batch *b) {
  BCK(cudaGetDevice(&b->device));
  b->jobs.assign(jobs, jobs + njobs);
  const int nj = njobs;
  b->plans.resize(nj);
  b->tunes.assign(nj, epwi_default_tune());
  b->cost.assign(nj, 0.0);
  // checks
  for (int j = 0; j < nj; j++) {
    const epw_linewidth_job &J = b->jobs[j];
    BCKS(epwi_check_common(J.model, J.nk, J.k, J.nq, J.q));
    BCKS(epwi_check_params(&J.params));
    if (J.model->timing) return epwi_fail(EPW_ERR_INVALID_ARG, "job %d: the model has timing enabled", j);
    if (J.nk > 0 && !J.imsigma) return epwi_fail(EPW_ERR_INVALID_ARG, "job %d: null imsigma", j);
    if ((J.nk > 0 && !epwi_is_device_ptr(J.k)) || (J.nq > 0 && !epwi_is_device_ptr(J.q)) ||
        (J.wq && J.nq > 0 && !epwi_is_device_ptr(J.wq)) || (J.nk > 0 && !epwi_is_device_ptr(J.imsigma)))
      return epwi_fail(EPW_ERR_INVALID_ARG, "job %d: batch buffers must be device pointers", j);
    if (J.nk > 0 && J.nq > 0 && job_path(J.model, J.params.precision) < 0)
      return epwi_fail(EPW_ERR_UNSUPPORTED, "job %d: no tensor-core form for nw=%d, 3nat=%d", j,
                       J.model->nw, J.model->nm);
    if (J.nk > 0 && J.nq > 0 && (J.model->nw > 18 || J.model->nm > 18))
      return epwi_fail(EPW_ERR_UNSUPPORTED, "job %d: no per-pair kernel for nw=%d, 3nat=%d", j, J.model->nw,
                       J.model->nm);
  }
  for (int i = 0; i < MAX_BRANCHES; i++) {
    cudaStream_t s = nullptr;
    BCK(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    b->streams.push_back(s);
    cudaEvent_t e = nullptr;
    BCK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    b->joins.push_back(e);
  }
  BCK(cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming));
  // tiles
  for (int j = 0; j < nj; j++) {
    const epw_linewidth_job &J = b->jobs[j];
    if (J.nk == 0 || J.nq == 0) continue;
    BCKS(tune_job(J, job_path(J.model, J.params.precision), b->streams[0], &b->tunes[j]));
    b->cost[j] = job_cost(J);
  }
  // one workspace in MAX_BRANCHES regions: the jobs of a region always run one after
  // another on one stream (every candidate graph maps regions onto branches), so they
  // share the region, which is as large as its largest job
  b->region = assign(b, MAX_BRANCHES);
  std::vector<size_t> rsize(MAX_BRANCHES, 0), roff(MAX_BRANCHES, 0);
  for (int j = 0; j < nj; j++) {
    const epw_linewidth_job &J = b->jobs[j];
    if (J.nk == 0 || J.nq == 0) continue;
    Arena A{nullptr, 0, 0};
    BCKS(epwi_plan_linewidth(A, J.model, J.nk, J.nq, J.params.precision, false, false, false, false, b->tunes[j],
                             b->plans[j]));
    rsize[b->region[j]] = std::max(rsize[b->region[j]], (A.off + 255) & ~size_t(255));
  }
  size_t total = 0;
  for (int r = 0; r < MAX_BRANCHES; r++) {
    roff[r] = total;
    total += rsize[r];
  }
  if (total) BCK(cudaMalloc((void **)&b->ws, total));
  b->ws_bytes = total;
  for (int j = 0; j < nj; j++) {
    const epw_linewidth_job &J = b->jobs[j];
    if (J.nk == 0 || J.nq == 0) continue;
    Arena A{b->ws + roff[b->region[j]], rsize[b->region[j]], 0};
    BCKS(epwi_plan_linewidth(A, J.model, J.nk, J.nq, J.params.precision, false, false, false, false, b->tunes[j],
                             b->plans[j]));
  }
  // one eager pass (validates every job and sets kernel attributes outside capture)
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  std::vector<int> one(nj, 0);
  BCK(cudaEventRecord(e0, b->streams[0]));
  BCKS(enqueue_all(b, one, 1));
  BCK(cudaEventRecord(e1, b->streams[0]));
  BCK(cudaStreamSynchronize(b->streams[0]));
  float eager_ms = 0.0f;
  BCK(cudaEventElapsedTime(&eager_ms, e0, e1));
  // candidate graphs: 1, 2 and 4 branches, the fastest kept; a batch whose eager pass
  // takes seconds gains nothing measurable from the choice and takes the 4-branch graph
  // without timing replays
  const bool long_batch = eager_ms > (float)LONG_BATCH_MS;
  int busy = 0;
  for (int j = 0; j < nj; j++) busy += (b->jobs[j].nk > 0) ? 1 : 0;
  float best = 0.0f;
  epw_status s = EPW_OK;
  for (int nb : {1, 2, 4}) {
    if (nb > 1 && nb > busy) break;
    if (long_batch && nb != (busy >= 4 ? 4 : busy >= 2 ? 2 : 1)) continue;
    std::vector<int> br(nj);
    for (int j = 0; j < nj; j++) br[j] = b->region[j] * nb / MAX_BRANCHES;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t x = nullptr;
    s = capture(b, br, nb, &g, &x);
    if (s != EPW_OK) break;
    float ms = 0.0f;
    cudaError_t e = cudaSuccess;
    if (!long_batch) {
      cudaEventRecord(e0, b->streams[0]);
      e = cudaGraphLaunch(x, b->streams[0]);
      cudaEventRecord(e1, b->streams[0]);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e != cudaSuccess) {
      cudaGraphExecDestroy(x);
      cudaGraphDestroy(g);
      s = epwi_fail(EPW_ERR_CUDA, "graph replay failed: %s", cudaGetErrorString(e));
      break;
    }
    if (!b->exec || ms < best) {
      if (b->exec) {
        cudaGraphExecDestroy(b->exec);
        cudaGraphDestroy(b->graph);
      }
      b->exec = x;
      b->graph = g;
      b->nbranch = nb;
      best = ms;
    } else {
      cudaGraphExecDestroy(x);
      cudaGraphDestroy(g);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != EPW_OK) return s;
  if (b->graph) {
    // kernel nodes: the kernels one replay launches
    size_t n = 0;
    BCK(cudaGraphGetNodes(b->graph, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    if (n) BCK(cudaGraphGetNodes(b->graph, nodes.data(), &n));
    b->nodes = 0;
    for (size_t i = 0; i < n; i++) {
      cudaGraphNodeType t;
      BCK(cudaGraphNodeGetType(nodes[i], &t));
      if (t == cudaGraphNodeTypeKernel) b->nodes++;
    }
  }
  return EPW_OK;
}

}  // namespace

extern "C" epw_status epw_batch_create(int njobs, const epw_linewidth_job *jobs, epw_batch **out) {
  if (!out) return epwi_fail(EPW_ERR_INVALID_ARG, "null output handle");
  *out = nullptr;
  if (njobs < 0 || (njobs > 0 && !jobs)) return epwi_fail(EPW_ERR_INVALID_ARG, "bad job list");
  epw_batch *b = new epw_batch();
  epw_status s = create_impl(njobs, jobs, b);
  if (s != EPW_OK) {
    destroy(b);
    return s;
  }
  *out = b;
  return EPW_OK;
}

extern "C" epw_status epw_batch_run(epw_batch *b, void *stream) {
  if (!b) return epwi_fail(EPW_ERR_INVALID_ARG, "null batch");
  if (!b->exec) return EPW_OK;  // no job with work
  int cur = -1;
  BCK(cudaGetDevice(&cur));
  if (cur != b->device) return epwi_fail(EPW_ERR_INVALID_ARG, "batch lives on device %d, current is %d", b->device, cur);
  BCK(cudaGraphLaunch(b->exec, (cudaStream_t)stream));
  return EPW_OK;
}

extern "C" epw_status epw_batch_info(const epw_batch *b, int *branches, size_t *workspace_bytes, size_t *graph_nodes) {
  if (!b) return epwi_fail(EPW_ERR_INVALID_ARG, "null batch");
  if (branches) *branches = b->nbranch;
  if (workspace_bytes) *workspace_bytes = b->ws_bytes;
  if (graph_nodes) *graph_nodes = b->nodes;
  return EPW_OK;
}

extern "C" void epw_batch_free(epw_batch *b) { destroy(b); }

extern "C" epw_status epw_linewidth_batched(int njobs, const epw_linewidth_job *jobs, void *stream) {
  epw_batch *b = nullptr;
  BCKS(epw_batch_create(njobs, jobs, &b));
  epw_status s = epw_batch_run(b, stream);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (s == EPW_OK && e != cudaSuccess) s = epwi_fail(EPW_ERR_CUDA, "batch: %s", cudaGetErrorString(e));
  std::set<const epw_model *> models;
  for (int j = 0; j < njobs; j++) models.insert(jobs[j].model);
  for (const epw_model *m : models) {
    epw_status t = epw_sync(m, stream);
    if (s == EPW_OK) s = t;
  }
  destroy(b);
  return s;
}
