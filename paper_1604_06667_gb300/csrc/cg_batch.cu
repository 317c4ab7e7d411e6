// cg_batch.cu -- many independent gridding jobs as one CUDA graph.
//
// A batch holds jobs of uneven sample count, channel count, target grid and
// kernel width (each with its own cg_grid handle).  The planner assigns the
// jobs to parallel branch streams by longest-processing-time first (estimated
// cost n_samples * (C + 16)), the capture records every job's one-shot
// pipeline (keys, sort, index, gridder, normalisation) on its branch between
// one fork and one join event, and cg_batch_run replays the instantiated
// graph with a single launch.  The autotuner times, per job, the FP32
// gridder's register-blocking shapes near the default for its channel count
// and, for BF16 data, the tensor-core form, and keeps the fastest.
#include <algorithm>
#include <cstdio>
#include <new>
#include <vector>

#include "cg_internal.h"

struct cg_batch {
  int device = 0;
  std::vector<cg_job> jobs;
  std::vector<cudaStream_t> streams;
  std::vector<int> stream_of;
  std::vector<cudaEvent_t> ev_join;
  cudaEvent_t ev_fork = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<int32_t> path, cfg;
  std::vector<double> tuned_ms;
  int64_t graph_kernels = 0;
};

namespace {

void release_graph(cg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

cg_status run_job(cg_batch* b, int j, cudaStream_t s) {
  const cg_job& J = b->jobs[(size_t)j];
  cg_grid* g = J.grid;
  cudaStream_t old = g->stream;
  g->stream = s;
  const int32_t keep_path = g->path, keep_cfg = g->f32_cfg;
  g->path = b->path[(size_t)j];
  g->f32_cfg = b->cfg[(size_t)j];
  const cg_status st = cg_grid_oneshot(g, J.lon_deg, J.lat_deg, J.data, J.data_dtype, J.weights,
                                       J.n_samples, J.out, J.layout_channel_major,
                                       J.out_weights);
  g->path = keep_path;
  g->f32_cfg = keep_cfg;
  g->stream = old;
  return st;
}

}  // namespace

extern "C" {

cg_status cg_batch_create(cg_batch** out, const cg_job* jobs, int32_t n_jobs,
                          int32_t n_streams) {
  if (!out) return cg::batch_fail(CG_EINVAL, "cg_batch_create: out is null");
  *out = nullptr;
  if (!jobs || n_jobs < 1) return cg::batch_fail(CG_EINVAL, "cg_batch_create: no jobs");
  if (n_streams < 1 || n_streams > 64)
    return cg::batch_fail(CG_EINVAL, "cg_batch_create: n_streams must be in [1, 64]");
  std::vector<cg_grid*> seen;
  for (int j = 0; j < n_jobs; ++j) {
    const cg_job& J = jobs[j];
    if (!J.grid || !J.grid->kernel_set)
      return cg::batch_fail(CG_EINVAL, "cg_batch_create: job %d has no handle with a kernel", j);
    if (std::find(seen.begin(), seen.end(), J.grid) != seen.end())
      return cg::batch_fail(CG_EINVAL, "cg_batch_create: job %d shares its handle with another "
                                       "job (one handle per job)", j);
    seen.push_back(J.grid);
    if (J.n_samples < 1 || !J.lon_deg || !J.lat_deg || !J.data || !J.out)
      return cg::batch_fail(CG_EINVAL, "cg_batch_create: job %d: null pointer or no samples", j);
    if (J.data_dtype != CG_F32 && J.data_dtype != CG_BF16)
      return cg::batch_fail(CG_EINVAL, "cg_batch_create: job %d: bad data_dtype", j);
    if (J.grid->device != jobs[0].grid->device)
      return cg::batch_fail(CG_EINVAL, "cg_batch_create: jobs on different devices");
  }
  cg_batch* b = new (std::nothrow) cg_batch();
  if (!b) return cg::batch_fail(CG_ENOMEM, "cg_batch_create: host allocation failed");
  b->device = jobs[0].grid->device;
  b->jobs.assign(jobs, jobs + n_jobs);
  b->path.assign((size_t)n_jobs, CG_PATH_AUTO);
  b->cfg.assign((size_t)n_jobs, -1);
  b->tuned_ms.assign((size_t)n_jobs, 0.0);
  for (int j = 0; j < n_jobs; ++j) {
    b->path[(size_t)j] = jobs[j].grid->path;
    b->cfg[(size_t)j] = jobs[j].grid->f32_cfg;
  }
  cudaSetDevice(b->device);
  const int ns = std::min(n_streams, n_jobs);
  b->streams.resize((size_t)ns, nullptr);
  b->ev_join.resize((size_t)ns, nullptr);
  cudaError_t e = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
  for (int i = 0; i < ns && e == cudaSuccess; ++i) {
    e = cudaStreamCreateWithFlags(&b->streams[(size_t)i], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_join[(size_t)i], cudaEventDisableTiming);
  }
  if (e != cudaSuccess) {
    cg_batch_destroy(b);
    return cg::batch_fail(CG_ECUDA, "cg_batch_create: %s", cudaGetErrorString(e));
  }
  // longest processing time first onto the least loaded branch
  std::vector<int> order((size_t)n_jobs);
  for (int j = 0; j < n_jobs; ++j) order[(size_t)j] = j;
  auto cost = [&](int j) {
    return (double)jobs[j].n_samples * (double)(jobs[j].grid->C + 16);
  };
  std::sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  std::vector<double> load((size_t)ns, 0.0);
  b->stream_of.assign((size_t)n_jobs, 0);
  for (int j : order) {
    const int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    b->stream_of[(size_t)j] = s;
    load[(size_t)s] += cost(j);
  }
  *out = b;
  return CG_OK;
}

cg_status cg_batch_autotune(cg_batch* b, int32_t reps, int32_t allow_tc) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_autotune: null batch");
  if (reps < 1 || reps > 100) return cg::batch_fail(CG_EINVAL, "cg_batch_autotune: reps in [1, 100]");
  cudaSetDevice(b->device);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return cg::batch_fail(CG_ECUDA, "cg_batch_autotune: event creation failed");
  cg_status result = CG_OK;
  for (size_t j = 0; j < b->jobs.size() && result == CG_OK; ++j) {
    const cg_job& J = b->jobs[j];
    cg_grid* g = J.grid;
    cudaStream_t s = b->streams[(size_t)b->stream_of[j]];
    // candidates: (path, FP32 shape)
    std::vector<std::pair<int32_t, int32_t>> cand;
    const int d = cg::f32_default_config(g->C);
    for (int c = d - 1; c <= d + 1; ++c)
      if (c >= 0 && c < cg::kF32Configs) cand.push_back({CG_PATH_FP32, c});
    if (allow_tc && cg::tc_supported(g, J.data_dtype, J.data)) cand.push_back({CG_PATH_TC, -1});
    double best = 1e300;
    std::pair<int32_t, int32_t> win = cand.front();
    for (const auto& c : cand) {
      b->path[j] = c.first;
      b->cfg[j] = c.second;
      cg_status st = run_job(b, (int)j, s);          // warm-up (allocations, index)
      if (st != CG_OK) { result = st; break; }
      cudaEventRecord(e0, s);
      for (int r = 0; r < reps && st == CG_OK; ++r) st = run_job(b, (int)j, s);
      cudaEventRecord(e1, s);
      if (st != CG_OK) { result = st; break; }
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        result = cg::batch_fail(CG_ECUDA, "cg_batch_autotune: job %d failed", (int)j);
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms / reps < best) {
        best = ms / reps;
        win = c;
      }
    }
    b->path[j] = win.first;
    b->cfg[j] = win.second;
    b->tuned_ms[j] = best;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  release_graph(b);   // a captured graph no longer reflects the choices
  return result;
}

cg_status cg_batch_capture(cg_batch* b, void* stream) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_capture: null batch");
  cudaSetDevice(b->device);
  cudaStream_t cap = static_cast<cudaStream_t>(stream);
  bool own = false;
  if (!cap) {
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      return cg::batch_fail(CG_ECUDA, "cg_batch_capture: stream creation failed");
    own = true;
  }
  // one eager pass first: workspaces reach their final sizes, so the capture
  // records no allocation
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    const cg_status st = run_job(b, (int)j, b->streams[(size_t)b->stream_of[j]]);
    if (st != CG_OK) {
      if (own) cudaStreamDestroy(cap);
      return st;
    }
  }
  for (cudaStream_t s : b->streams) cudaStreamSynchronize(s);
  release_graph(b);
  int64_t launches0 = 0;
  for (const cg_job& J : b->jobs) launches0 += J.grid->n_launches;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  cg_status st = CG_OK;
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, cap);
  for (size_t i = 0; i < b->streams.size() && e == cudaSuccess; ++i)
    e = cudaStreamWaitEvent(b->streams[i], b->ev_fork, 0);
  for (size_t j = 0; j < b->jobs.size() && e == cudaSuccess && st == CG_OK; ++j)
    st = run_job(b, (int)j, b->streams[(size_t)b->stream_of[j]]);
  for (size_t i = 0; i < b->streams.size() && e == cudaSuccess; ++i) {
    e = cudaEventRecord(b->ev_join[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, b->ev_join[i], 0);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t e_end = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e_end;
  if (e == cudaSuccess && st == CG_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (e == cudaSuccess && st == CG_OK) {
    b->graph = graph;
  } else if (graph) {
    cudaGraphDestroy(graph);
  }
  int64_t launches1 = 0;
  for (const cg_job& J : b->jobs) launches1 += J.grid->n_launches;
  b->graph_kernels = launches1 - launches0;
  if (own) cudaStreamDestroy(cap);
  if (st != CG_OK) return st;
  if (e != cudaSuccess)
    return cg::batch_fail(CG_ECUDA, "cg_batch_capture: %s", cudaGetErrorString(e));
  return CG_OK;
}

cg_status cg_batch_run(cg_batch* b, void* stream) {
  if (!b || !b->exec)
    return cg::batch_fail(CG_ESTATE, "cg_batch_run: capture the batch first");
  cudaSetDevice(b->device);
  const cudaError_t e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_run: %s", cudaGetErrorString(e));
  return CG_OK;
}

cg_status cg_batch_get_choice(cg_batch* b, int32_t job, int32_t* path, int32_t* f32_shape,
                              double* ms, int32_t* stream_index) {
  if (!b || job < 0 || job >= (int32_t)b->jobs.size())
    return cg::batch_fail(CG_EINVAL, "cg_batch_get_choice: bad batch or job index");
  if (path) *path = b->path[(size_t)job];
  if (f32_shape) *f32_shape = b->cfg[(size_t)job];
  if (ms) *ms = b->tuned_ms[(size_t)job];
  if (stream_index) *stream_index = b->stream_of[(size_t)job];
  return CG_OK;
}

cg_status cg_batch_info(cg_batch* b, int64_t* graph_kernels, int32_t* n_streams) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_info: null batch");
  if (graph_kernels) *graph_kernels = b->graph_kernels;
  if (n_streams) *n_streams = (int32_t)b->streams.size();
  return CG_OK;
}

cg_status cg_batch_destroy(cg_batch* b) {
  if (!b) return CG_OK;
  cudaSetDevice(b->device);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamSynchronize(s);
  release_graph(b);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
  return CG_OK;
}

}  // extern "C"
