// cg_batch.cu -- many independent gridding jobs as one CUDA graph.
//
// A batch holds jobs of uneven sample count, channel count, target grid and
// kernel width (each with its own cg_grid handle).  Two ways to capture it:
//
// per job   the planner assigns the jobs to parallel branch streams by
//           longest-processing-time first (estimated cost n_samples *
//           (C + 16)), the capture records every job's one-shot pipeline
//           (keys, sort, index, gridder, normalisation) on its branch
//           between one fork and one join event;
// fused     one pipeline for all jobs: one keys pass, one sort of every
//           job's samples by a composite key, one gather and one candidate
//           range pass, then one persistent FP32 gridder launch whose CTAs
//           take (job, tile, slab, split) items from a queue ordered by
//           estimated cost (up to 96 jobs per launch), one split reduction,
//           one non-finite fix-up and one normalisation over all jobs; jobs
//           on the tensor-core form run the tensor-core gridder on their
//           segment of the shared index.
//
// cg_batch_run replays the instantiated graph with a single launch.  The
// autotuner times, per job, the FP32 gridder's register-blocking shapes near
// the default for its channel count and, for BF16 data, the tensor-core
// form, and keeps the fastest.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "cg_common.cuh"
#include "cg_internal.h"

namespace {

// The fused pipeline's device state (built by the eager pass before capture).
struct FusedPlan {
  cg::BatchIndex bi;
  std::vector<cg::BatchIndexJob> ijobs;
  struct Group {
    cg::F32Multi m;
    std::vector<cg::F32MultiJob> hjobs;
    std::vector<cg::F32Multi::Out> houts;
  };
  std::vector<Group> groups;
  std::vector<int> tc_jobs;          // jobs on the tensor-core form
  std::vector<void*> owned;          // device buffers to release
  int64_t kernels = 0;               // launches of one pass
};

}  // namespace

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
  // fused capture
  bool fused = false;
  FusedPlan* plan = nullptr;
  cudaStream_t own = nullptr;        // eager work of the fused plan
  unsigned* d_err = nullptr;         // device errors of the fused pipeline
  int32_t* d_hold = nullptr;         // testing hook: a word nothing sets
  bool hold = false;
  int64_t hold_cycles = 0;
  cudaEvent_t ev_done = nullptr;     // end of the last replay
};

namespace {

void release_graph(cg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void release_plan(cg_batch* b) {
  FusedPlan* p = b->plan;
  if (!p) return;
  cudaStream_t s = b->own;
  if (s) cudaStreamSynchronize(s);
  cg::batch_index_free(p->bi, s);
  for (void* q : p->owned) cudaFreeAsync(q, s);
  if (s) cudaStreamSynchronize(s);
  delete p;
  b->plan = nullptr;
}

template <typename T>
cudaError_t plan_alloc(FusedPlan* p, T** out, size_t count, cudaStream_t s) {
  cudaError_t e = cg::dalloc(out, count, s);
  if (e == cudaSuccess) p->owned.push_back(*out);
  return e;
}

template <typename T>
cudaError_t plan_upload(FusedPlan* p, T** out, const std::vector<T>& h, cudaStream_t s) {
  cudaError_t e = plan_alloc(p, out, h.size(), s);
  if (e == cudaSuccess && !h.empty())
    e = cudaMemcpyAsync(*out, h.data(), sizeof(T) * h.size(), cudaMemcpyHostToDevice, s);
  return e;
}

// The job's form, as a one-job call would choose it (CG_PATH_AUTO: tensor
// cores for BF16 data with C >= 16), where the fused pipeline supports it.
bool job_on_tc(const cg_batch* b, int j) {
  const cg_job& J = b->jobs[(size_t)j];
  const int32_t path = b->path[(size_t)j];
  if (path == CG_PATH_FP32) return false;
  if (!cg::tc_supported(J.grid, J.data_dtype, J.data) || J.layout_channel_major) return false;
  return path == CG_PATH_TC || path == CG_PATH_TC_FAST || J.grid->C >= 16;
}

// The FP32 register-blocking shape of a job: the autotuner's, else the
// default for its channel count.
int job_shape(const cg_batch* b, int j) {
  const int32_t c = b->cfg[(size_t)j];
  return (c >= 0 && c < cg::kF32MultiShapes) ? c : cg::f32_multi_shape(b->jobs[(size_t)j].grid->C);
}

// Build the fused plan: the shared sample index, the FP32 groups (their job
// arguments, item counts, split counts and scratch) and the tensor-core
// job list.  Host work plus allocations on b->own; nothing is launched.
cg_status build_plan(cg_batch* b) {
  release_plan(b);
  FusedPlan* p = new (std::nothrow) FusedPlan();
  if (!p) return cg::batch_fail(CG_ENOMEM, "cg_batch_capture: host allocation failed");
  b->plan = p;
  cudaStream_t s = b->own;
  const int nj = (int)b->jobs.size();
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  // ---- the shared sample index ----
  std::vector<int64_t> samp_off(1, 0), key_blk(1, 0), gth_blk(1, 0), tile_off(1, 0);
  uint64_t key_base = 0;
  int64_t ring_base = 0;
  for (int j = 0; j < nj; ++j) {
    const cg_job& J = b->jobs[(size_t)j];
    cg_grid* g = J.grid;
    const bool tc = job_on_tc(b, j);
    cg::Tiling& t = tc ? g->t128 : g->t64;
    cg::BatchIndexJob q;
    q.lon = J.lon_deg;
    q.lat = J.lat_deg;
    q.weights = J.weights;
    q.n = J.n_samples;
    q.off = samp_off.back();
    q.nside = g->nside;
    q.lg = -1;
    if ((g->nside & (g->nside - 1)) == 0)
      for (q.lg = 0; (1LL << q.lg) < g->nside; ++q.lg) {
      }
    q.key_base = key_base;
    q.ring_base = ring_base;
    q.ranges = t.ranges;
    q.range_off = t.range_off;
    q.n_tiles = t.n_tiles;
    q.range_s = t.range_s;
    q.range_c = t.range_c;
    q.tile_cand = t.tile_cand;
    p->ijobs.push_back(q);
    const int64_t ns = g->nside;
    key_base += (uint64_t)(12 * ns * ns) + 1;
    ring_base += 4 * ns + 1;
    samp_off.push_back(q.off + J.n_samples);
    key_blk.push_back(key_blk.back() + (J.n_samples + 255) / 256);
    gth_blk.push_back(gth_blk.back() + (J.n_samples + 1 + 255) / 256);
    tile_off.push_back(tile_off.back() + t.n_tiles);
    if (tc) p->tc_jobs.push_back(j);
  }
  cg::BatchIndex& bi = p->bi;
  bi.n_jobs = nj;
  bi.N = samp_off.back();
  bi.n_ring = ring_base;
  bi.n_tiles = tile_off.back();
  bi.key_bits = 1;
  while (bi.key_bits < 64 && ((key_base - 1) >> bi.key_bits) != 0) ++bi.key_bits;
  bi.sw.err = b->d_err;
  cudaError_t e = cg::batch_index_alloc(bi, s);
  if (e == cudaSuccess) e = cg::dalloc(&bi.jobs, (size_t)nj, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(bi.jobs, p->ijobs.data(), sizeof(cg::BatchIndexJob) * (size_t)nj,
                        cudaMemcpyHostToDevice, s);
  auto up64 = [&](int64_t** d, const std::vector<int64_t>& h) {
    if (e != cudaSuccess) return;
    e = cg::dalloc(d, h.size(), s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(*d, h.data(), sizeof(int64_t) * h.size(), cudaMemcpyHostToDevice, s);
  };
  bi.n_key_blk = key_blk.back();
  bi.n_gth_blk = gth_blk.back();
  up64(&bi.key_blk, key_blk);
  up64(&bi.gth_blk, gth_blk);
  up64(&bi.tile_off, tile_off);
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_capture: %s", cudaGetErrorString(e));

  // ---- FP32 groups ----
  // FP32 jobs grouped by register-blocking shape (one launch per shape)
  std::vector<int> f32;
  for (int j = 0; j < nj; ++j)
    if (!job_on_tc(b, j)) f32.push_back(j);
  std::stable_sort(f32.begin(), f32.end(),
                   [&](int x, int y) { return job_shape(b, x) < job_shape(b, y); });
  // candidate splits: items of about 1 / (16 x CTAs) of the FP32 work each
  double total = 0.0;
  for (int j : f32) {
    const cg_job& J = b->jobs[(size_t)j];
    const int shape = job_shape(b, j);
    const int cp = cg::f32_multi_cpad(shape);
    const int nb = (J.grid->C + cp - 1) / cp;
    total += (double)J.n_samples * (double)(cg::kTile + cp) * nb;
  }
  const double quantum = std::max(1.0, total / (16.0 * 2.0 * nsm));
  for (size_t g0 = 0, g1 = 0; g0 < f32.size(); g0 = g1) {
    p->groups.emplace_back();
    FusedPlan::Group& G = p->groups.back();
    std::vector<int64_t> item_off(1, 0), fin_blk(1, 0), red_blk(1, 0), word_off(1, 0);
    const int shape0 = job_shape(b, f32[g0]);
    for (g1 = g0; g1 < f32.size() && g1 - g0 < (size_t)cg::kF32MultiMaxJobs &&
                  job_shape(b, f32[g1]) == shape0;
         ++g1) {
    }
    G.m.shape = shape0;
    for (size_t k = g0; k < g1 && e == cudaSuccess; ++k) {
      const int j = f32[k];
      const cg_job& J = b->jobs[(size_t)j];
      cg_grid* g = J.grid;
      const cg::BatchIndexJob& q = p->ijobs[(size_t)j];
      cg::F32MultiJob mj;
      std::memset(&mj, 0, sizeof(mj));
      mj.shape = shape0;
      mj.dtype = J.data_dtype;
      mj.pad = cg::f32_multi_cpad(mj.shape);
      mj.n_slabs = (g->C + mj.pad - 1) / mj.pad;
      cg::GridArgs& a = mj.a;
      a.tile_chi = g->t64.chi;
      a.tile_clo = g->t64.clo;
      a.tgt_a = g->t64.a;
      a.tgt_f1 = g->tgt_f1;
      a.tgt_f2 = g->tgt_f2;
      a.tgt_ll = g->tgt_ll;
      a.tgt_perm = g->tgt_perm;
      a.range_off = g->t64.range_off;
      a.range_s = g->t64.range_s;
      a.s_hi = bi.s_hi + q.off;
      a.s_lo = bi.s_lo + q.off;
      a.sll = bi.sll + q.off;
      // the sorted values are known once the sort's pass count is (ping-pong)
      a.perm = nullptr;
      a.data = J.data;
      a.C = g->C;
      const size_t esz = (J.data_dtype == CG_BF16) ? 2 : 4;
      a.vec4 = (g->C % 4 == 0) && ((reinterpret_cast<uintptr_t>(J.data) % (4 * esz)) == 0);
      a.kd = g->kdev;
      a.kd.dscale = 0.f;
      a.acc_num = g->acc_num;
      a.acc_w = g->acc_w;
      a.accumulate = 0;
      a.pairs = nullptr;
      a.tile_cand = g->t64.tile_cand;
      const double per_tile = (double)J.n_samples / std::max<int64_t>(1, g->t64.n_tiles) *
                              (double)(cg::kTile + mj.pad);
      a.n_split = (int)std::min(64.0, std::max(1.0, std::ceil(per_tile / quantum)));
      a.n_slots = g->n_slots;
      if (a.n_split > 1) {
        e = plan_alloc(p, &a.part_num, (size_t)a.n_split * g->n_slots * g->C, s);
        if (e == cudaSuccess) e = plan_alloc(p, &a.part_w, (size_t)a.n_split * g->n_slots, s);
      }
      const int64_t nbits = g->n_slots * (int64_t)mj.n_slabs;
      {
        cudaStream_t keep = g->stream;
        g->stream = s;
        if (e == cudaSuccess) e = cg::nonfinite_prepare(g, nbits);
        g->stream = keep;
      }
      a.nf_bits = g->nf_bits;
      // without splits, [P][C] maps are written by the gridder itself
      const bool direct = a.n_split == 1 && !J.layout_channel_major;
      a.out = direct ? J.out : nullptr;
      a.out_w = direct ? J.out_weights : nullptr;
      G.hjobs.push_back(mj);
      const int vec4 = !J.layout_channel_major && g->C % 4 == 0 &&
                       reinterpret_cast<uintptr_t>(J.out) % 16 == 0;
      G.houts.push_back({J.out, J.out_weights, J.layout_channel_major, vec4, g->P});
      item_off.push_back(item_off.back() + g->t64.n_tiles * mj.n_slabs * a.n_split);
      fin_blk.push_back(fin_blk.back() +
                        (direct ? 0
                                : (g->n_slots * (int64_t)g->C + cg::kMultiFinElems - 1) /
                                      cg::kMultiFinElems));
      red_blk.push_back(red_blk.back() +
                        (a.n_split > 1 ? (g->n_slots * (int64_t)(g->C + 1) + cg::kMultiRedElems - 1) /
                                             cg::kMultiRedElems
                                       : 0));
      word_off.push_back(word_off.back() + (nbits + 31) / 32);
    }
    cg::F32Multi& m = G.m;
    m.n_jobs = (int)G.hjobs.size();
    m.n_items = item_off.back();
    m.n_fin_blk = fin_blk.back();
    m.n_red_blk = red_blk.back();
    m.n_words = word_off.back();
    m.err = b->d_err;
    if (e == cudaSuccess) e = plan_alloc(p, &m.nf_any, 1, s);
    for (auto& mj : G.hjobs) mj.a.nf_any = m.nf_any;
    if (e == cudaSuccess) e = plan_upload(p, &m.item_off, item_off, s);
    if (e == cudaSuccess) e = plan_upload(p, &m.fin_blk, fin_blk, s);
    if (e == cudaSuccess) e = plan_upload(p, &m.red_blk, red_blk, s);
    if (e == cudaSuccess) e = plan_upload(p, &m.word_off, word_off, s);
    if (e == cudaSuccess) e = plan_upload(p, &m.outs, G.houts, s);
    if (e == cudaSuccess) e = plan_alloc(p, &m.order, (size_t)std::max<int64_t>(1, m.n_items), s);
    if (e == cudaSuccess) e = plan_alloc(p, &m.head, 1, s);
    if (e == cudaSuccess) e = plan_alloc(p, &m.jobs, G.hjobs.size(), s);
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_capture: %s", cudaGetErrorString(e));
  return CG_OK;
}

// One pass of the fused pipeline on stream st: eager (upload = true: the
// jobs' arguments are copied to the device once the sort's output buffers are
// known) or under capture (upload = false).
cg_status run_fused(cg_batch* b, cudaStream_t st, bool upload) {
  FusedPlan* p = b->plan;
  cg::BatchIndex& bi = p->bi;
  int64_t launches = 0;
  cudaError_t e = cg::batch_index_run(bi, b->d_err, st, &launches);
  // the tensor-core jobs (the planner's branch assignment) and the FP32
  // groups (group k on branch k) run on the branch streams, side by side
  const size_t ns = b->streams.size();
  std::vector<char> used(ns, 0);
  for (int j : p->tc_jobs) used[(size_t)b->stream_of[(size_t)j]] = 1;
  for (size_t k = 0; k < p->groups.size(); ++k) used[k % ns] = 1;
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, st);
  for (size_t i = 0; i < ns && e == cudaSuccess; ++i)
    if (used[i]) e = cudaStreamWaitEvent(b->streams[i], b->ev_fork, 0);
  for (size_t k = 0; k < p->tc_jobs.size() && e == cudaSuccess; ++k) {
    const int j = p->tc_jobs[k];
    const cg_job& J = b->jobs[(size_t)j];
    cg_grid* g = J.grid;
    const cg::BatchIndexJob& q = p->ijobs[(size_t)j];
    cudaStream_t bs = b->streams[(size_t)b->stream_of[(size_t)j]];
    // the handle sees its segment of the shared index for this call
    struct {
      cudaStream_t stream;
      float4 *s_hi, *s_lo;
      double2* s_ll;
      uint32_t *sorted_val, *sorted_key;
      int32_t* ring_off;
      int64_t last_n;
    } keep = {g->stream, g->s_hi, g->s_lo, g->s_ll, g->sorted_val, g->sorted_key, g->ring_off,
              g->last_n};
    g->stream = bs;
    g->s_hi = bi.s_hi + q.off;
    g->s_lo = bi.s_lo + q.off;
    g->s_ll = bi.sll + q.off;
    g->sorted_val = bi.sorted_val + q.off;
    g->sorted_key = bi.skey + q.off;
    g->ring_off = bi.ring_off + q.ring_base;
    g->last_n = J.n_samples;
    const int64_t l0 = g->n_launches;
    e = cg::grid_tiles_tc(g, J.data, 2, J.out, J.out_weights,
                          b->path[(size_t)j] != CG_PATH_TC_FAST);
    launches += g->n_launches - l0;
    // restore the handle's own sample arrays (allocations made by the call,
    // such as the bitmap or the item order, stay with the handle)
    g->stream = keep.stream;
    g->s_hi = keep.s_hi;
    g->s_lo = keep.s_lo;
    g->s_ll = keep.s_ll;
    g->sorted_val = keep.sorted_val;
    g->sorted_key = keep.sorted_key;
    g->ring_off = keep.ring_off;
    g->last_n = keep.last_n;
  }
  // the FP32 groups, launched after the tensor-core jobs so that their
  // persistent CTAs fill what the tensor-core kernels leave free; the jobs'
  // arguments point into the sort's output (known now)
  for (size_t k = 0; k < p->groups.size() && e == cudaSuccess; ++k) {
    FusedPlan::Group& G = p->groups[k];
    cudaStream_t gs = b->streams[k % ns];
    for (size_t i = 0; i < G.hjobs.size(); ++i) {
      const int64_t off = (int64_t)(G.hjobs[i].a.s_hi - bi.s_hi);
      G.hjobs[i].a.perm = bi.sorted_val + off;
    }
    G.m.hjobs = G.hjobs.data();
    G.m.hold = b->hold ? b->d_hold : nullptr;
    G.m.hold_cycles = b->hold_cycles;
    if (upload) {
      e = cudaMemcpyAsync(G.m.jobs, G.hjobs.data(), sizeof(cg::F32MultiJob) * G.hjobs.size(),
                          cudaMemcpyHostToDevice, gs);
      if (e == cudaSuccess) e = cudaStreamSynchronize(gs);
    }
    if (e == cudaSuccess) e = cg::grid_f32_multi(G.m, gs, &launches);
  }
  for (size_t i = 0; i < used.size() && e == cudaSuccess; ++i) {
    if (!used[i]) continue;
    e = cudaEventRecord(b->ev_join[i], b->streams[i]);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->ev_join[i], 0);
  }
  // the shared index wrote every job's candidate ranges: the handles' own
  // adds compute theirs again
  for (const cg_job& J : b->jobs) {
    J.grid->t64.ranges_gen = -1;
    J.grid->t128.ranges_gen = -1;
  }
  p->kernels = launches;
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch (fused): %s", cudaGetErrorString(e));
  return CG_OK;
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

cg_status ensure_own(cg_batch* b) {
  cudaError_t e = cudaSuccess;
  if (!b->own) e = cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking);
  if (e == cudaSuccess && !b->ev_done) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess && !b->d_err) {
    e = cg::dalloc(&b->d_err, 1, b->own);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->own);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch: %s", cudaGetErrorString(e));
  return CG_OK;
}

// Fused capture: plan, one eager pass (allocations, the jobs' arguments on
// the device), then the same pass recorded on cap.
cg_status capture_fused(cg_batch* b, cudaStream_t cap) {
  cg_status st = ensure_own(b);
  if (st == CG_OK) st = build_plan(b);
  if (st == CG_OK) st = run_fused(b, b->own, true);
  if (st != CG_OK) return st;
  cudaError_t e = cudaStreamSynchronize(b->own);
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_capture: %s", cudaGetErrorString(e));
  release_graph(b);
  e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) st = run_fused(b, cap, false);
  cudaGraph_t graph = nullptr;
  const cudaError_t e_end = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e_end;
  if (e == cudaSuccess && st == CG_OK) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (e == cudaSuccess && st == CG_OK) {
    b->graph = graph;
  } else if (graph) {
    cudaGraphDestroy(graph);
  }
  b->graph_kernels = b->plan ? b->plan->kernels : 0;
  if (st != CG_OK) return st;
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_capture: %s", cudaGetErrorString(e));
  return CG_OK;
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
  if (b->fused) {
    const cg_status st = capture_fused(b, cap);
    if (own) cudaStreamDestroy(cap);
    return st;
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
  cudaError_t e = cudaSuccess;
  if (!b->ev_done) e = cudaEventCreateWithFlags(&b->ev_done, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_done, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_run: %s", cudaGetErrorString(e));
  return CG_OK;
}

cg_status cg_batch_set_fused(cg_batch* b, int32_t fused) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_set_fused: null batch");
  cudaSetDevice(b->device);
  if ((fused != 0) != b->fused) {
    release_graph(b);
    release_plan(b);
  }
  b->fused = fused != 0;
  return CG_OK;
}

cg_status cg_batch_sync(cg_batch* b) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_sync: null batch");
  cudaSetDevice(b->device);
  cudaError_t e = cudaSuccess;
  if (b->ev_done) e = cudaEventSynchronize(b->ev_done);
  if (e == cudaSuccess && b->own) e = cudaStreamSynchronize(b->own);
  unsigned h = 0;
  if (e == cudaSuccess && b->d_err) {
    e = cudaMemcpy(&h, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && h) e = cudaMemset(b->d_err, 0, sizeof(unsigned));
  }
  if (e != cudaSuccess) return cg::batch_fail(CG_ECUDA, "cg_batch_sync: %s", cudaGetErrorString(e));
  if (h & cg::ERR_BAD_SAMPLE)
    return cg::batch_fail(CG_EINVAL, "cg_batch_sync: sample coordinates must be finite with "
                                     "|lat| <= 90 and weights finite and >= 0 (offending "
                                     "samples were skipped)");
  if (h & cg::ERR_TIMEOUT)
    return cg::batch_fail(CG_ETIMEOUT, "cg_batch_sync: a bounded device wait gave up");
  if (h) return cg::batch_fail(CG_EDEVICE, "cg_batch_sync: device error word 0x%x", h);
  // the tensor-core jobs of a fused batch, and every job of a per-job batch,
  // report through their handles
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    const cg_status st = cg_sync(b->jobs[j].grid);
    if (st != CG_OK) return st;
  }
  return CG_OK;
}

cg_status cg_batch_debug_hold(cg_batch* b, int32_t enable, int64_t wait_cycles) {
  if (!b) return cg::batch_fail(CG_EINVAL, "cg_batch_debug_hold: null batch");
  cudaSetDevice(b->device);
  cg_status st = ensure_own(b);
  if (st != CG_OK) return st;
  if (enable && !b->d_hold) {
    cudaError_t e = cg::dalloc(&b->d_hold, 1, b->own);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_hold, 0, sizeof(int32_t), b->own);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->own);
    if (e != cudaSuccess)
      return cg::batch_fail(CG_ECUDA, "cg_batch_debug_hold: %s", cudaGetErrorString(e));
  }
  b->hold = enable != 0;
  b->hold_cycles = wait_cycles > 0 ? wait_cycles : 2000000;
  release_graph(b);   // the hook is recorded in the captured launches
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
  release_plan(b);
  if (b->own) {
    cudaStreamSynchronize(b->own);
    if (b->d_err) cudaFreeAsync(b->d_err, b->own);
    if (b->d_hold) cudaFreeAsync(b->d_hold, b->own);
    cudaStreamSynchronize(b->own);
    cudaStreamDestroy(b->own);
  }
  if (b->ev_done) cudaEventDestroy(b->ev_done);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev_join)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
  return CG_OK;
}

}  // extern "C"
