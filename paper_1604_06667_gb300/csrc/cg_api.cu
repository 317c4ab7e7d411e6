// cg_api.cu -- the C ABI (include/cygrid_gb300.h): argument checks, the
// planner (nside rule, kernel constants) and the ordering of the kernels on
// the handle's stream.
#include <cmath>
#include <cstdarg>
#include <vector>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "cg_common.cuh"
#include "cg_internal.h"

using namespace cg;

namespace {

thread_local std::string g_last_error;

cg_status fail(cg_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
cg_status fail(cg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

cg_status cuda_fail(cudaError_t e, const char* where) {
  if (e == cudaErrorMemoryAllocation)
    return fail(CG_ENOMEM, "%s: device allocation failed", where);
  return fail(CG_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CG_CUDA(call, where)                       \
  do {                                             \
    cudaError_t e_ = (call);                       \
    if (e_ != cudaSuccess) return cuda_fail(e_, where); \
  } while (0)

// ---- stage timing -------------------------------------------------------
cudaEvent_t tmark(cg_grid* g) {
  if (!g->timing) return nullptr;
  cudaEvent_t e = nullptr;
  if (!g->ev_pool.empty()) {
    e = g->ev_pool.back();
    g->ev_pool.pop_back();
  } else if (cudaEventCreate(&e) != cudaSuccess) {
    return nullptr;
  }
  cudaEventRecord(e, g->stream);
  g->ev_used.push_back(e);  // owned once here; stage records only refer to it
  return e;
}

void tstage(cg_grid* g, int stage, cudaEvent_t a, cudaEvent_t b) {
  if (a && b) g->timing_recs.push_back(cg_grid::TimingRec{stage, a, b});
}

// Consecutive stages share their boundary event, so events are returned to
// the pool from the ownership list (each exactly once), not from the records.
void release_events(cg_grid* g) {
  for (cudaEvent_t e : g->ev_used) g->ev_pool.push_back(e);
  g->ev_used.clear();
  g->timing_recs.clear();
}

// Read and clear the device error word (synchronises the stream).
cg_status check_device(cg_grid* g, const char* where) {
  unsigned h = 0;
  CG_CUDA(cudaMemcpyAsync(&h, g->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream),
          where);
  CG_CUDA(cudaStreamSynchronize(g->stream), where);
  if (h) {
    CG_CUDA(cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), g->stream), where);
    CG_CUDA(cudaStreamSynchronize(g->stream), where);
  }
  if (h & ERR_BAD_TARGET)
    return fail(CG_EINVAL, "%s: target coordinates must be finite with |lat| <= 90", where);
  if (h & ERR_BAD_SAMPLE)
    return fail(CG_EINVAL,
                "%s: sample coordinates must be finite with |lat| <= 90 and weights finite "
                "and >= 0 (offending samples were skipped)",
                where);
  if (h & ERR_TIMEOUT) return fail(CG_ETIMEOUT, "%s: a bounded device wait gave up", where);
  if (h) return fail(CG_EDEVICE, "%s: device error word 0x%x", where, h);
  return CG_OK;
}

void free_all(cg_grid* g) {
  cudaStream_t s = g->stream;
  dfree(g->tgt_perm, s);
  tiling_free(g->t64, s);
  tiling_free(g->t128, s);
  dfree(g->tgt_e, s);
  dfree(g->tgt_n, s);
  dfree(g->tgt_f1, s);
  dfree(g->tgt_f2, s);
  dfree(g->tgt_ll, s);
  dfree(g->key, s);
  dfree(g->val, s);
  if (g->sw.keys_alt) cudaFreeAsync(g->sw.keys_alt, s);
  g->sw.keys_alt = nullptr;
  dfree(g->sw.vals_alt, s);
  dfree(g->sw.hist, s);
  dfree(g->sw.totals, s);
  dfree(g->sw.status, s);
  dfree(g->sw.os_meta, s);
  dfree(g->s_hi, s);
  dfree(g->s_lo, s);
  dfree(g->u_rec, s);
  dfree(g->s_ll, s);
  dfree(g->ring_off, s);
  dfree(g->tix_key, s);
  dfree(g->tix_val, s);
  dfree(g->tix_uhi, s);
  dfree(g->tix_ulo, s);
  dfree(g->tix_hi, s);
  dfree(g->tix_lo, s);
  dfree(g->tix_ring_off, s);
  dfree(g->tix_invw, s);
  if (g->tix_sw.keys_alt) cudaFreeAsync(g->tix_sw.keys_alt, s);
  g->tix_sw.keys_alt = nullptr;
  dfree(g->tix_sw.vals_alt, s);
  dfree(g->tix_sw.hist, s);
  dfree(g->tix_sw.totals, s);
  dfree(g->tix_sw.status, s);
  dfree(g->tix_sw.os_meta, s);
  dfree(g->ds_num, s);
  dfree(g->ds_w, s);
  dfree(g->ds_num0, s);
  dfree(g->ds_w0, s);
  dfree(g->ds_part, s);
  dfree(g->pcw_data, s);
  dfree(g->pcw_acc, s);
  dfree(g->pcw_w, s);
  g->pcw_cap_data = 0;
  dfree(g->part_num, s);
  dfree(g->part_w, s);
  dfree(g->acc_num, s);
  dfree(g->acc_w, s);
  dfree(g->d_err, s);
  dfree(g->d_pairs, s);
  dfree(g->nf_bits, s);
  dfree(g->nf_any, s);
  g->nf_words = 0;
  dfree(g->d_hold, s);
  dfree(g->md_part, s);
  g->md_cap = 0;
  release_events(g);
  for (cudaEvent_t e : g->ev_pool) cudaEventDestroy(e);
  g->ev_pool.clear();
}

bool finite_pos(double x) { return std::isfinite(x) && x > 0.0; }

// Reset: the first add after it stores instead of accumulating (both
// gridders write every valid slot of every tile), so the accumulators are
// only cleared when a finalize finds no add since the reset.
cg_status zero_acc(cg_grid* g) {
  CG_CUDA(cudaMemsetAsync(g->d_pairs, 0, sizeof(unsigned long long), g->stream), "reset");
  g->acc_empty = true;
  g->total_n = 0;
  return CG_OK;
}

cg_status clear_if_empty(cg_grid* g, const char* where) {
  if (!g->acc_empty) return CG_OK;
  const int64_t slots = g->n_slots;
  CG_CUDA(cudaMemsetAsync(g->acc_num, 0, sizeof(float) * (size_t)slots * g->C, g->stream), where);
  CG_CUDA(cudaMemsetAsync(g->acc_w, 0, sizeof(float2) * (size_t)slots, g->stream), where);
  return CG_OK;
}

// Channel-accumulation form for this add.
bool use_tc(const cg_grid* g, int dtype, const void* data) {
  if (g->path == CG_PATH_FP32) return false;
  if (g->path == CG_PATH_TC || g->path == CG_PATH_TC_FAST) return true;
  return tc_supported(g, dtype, data) && g->C >= 16;
}

// out != nullptr: one-shot call whose normalised [P][C] result the
// tensor-core epilogue writes directly (the accumulators are left empty).
cg_status do_add(cg_grid* g, const double* lon, const double* lat, const void* data,
                 int32_t dtype, const float* weights, int64_t n, const char* where,
                 float* out = nullptr, float* out_w = nullptr, bool* fused = nullptr) {
  if (fused) *fused = false;
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (dtype != CG_F32 && dtype != CG_BF16)
    return fail(CG_EINVAL, "%s: data_dtype must be CG_F32 or CG_BF16", where);
  if (n < 0 || n > 0x7fffffffLL) return fail(CG_EINVAL, "%s: n_samples out of range", where);
  if (n == 0) return CG_OK;
  // lon = lat = NULL: the samples (and weights) of the previous add, whose
  // sample index is reused; only the channel data are new
  const bool reuse = !lon && !lat;
  if (reuse && (!g->index_valid || n != g->last_n || weights))
    return fail(CG_EINVAL,
                "%s: lon = lat = NULL reuses the previous add's samples: needs a previous add "
                "since cg_set_kernel with the same n_samples and weights = NULL",
                where);
  if ((!reuse && (!lon || !lat)) || !data)
    return fail(CG_EINVAL, "%s: null coordinate or data pointer", where);
  const bool tc = use_tc(g, dtype, data);
  if (tc && !tc_supported(g, dtype, data))
    return fail(CG_EINVAL,
                "%s: the tensor-core form needs BF16 data, n_channels %% 8 == 0 and a "
                "16-byte aligned data pointer",
                where);
  CG_CUDA(cudaSetDevice(g->device), where);
  Tiling& t = tc ? g->t128 : g->t64;
  cudaEvent_t t0 = tmark(g);
  if (!reuse) {
    g->index_valid = false;
    CG_CUDA(samples_keys(g, lon, lat, weights, n), where);
  }
  cudaEvent_t t1 = tmark(g);
  if (!reuse) CG_CUDA(samples_sort(g, n), where);
  cudaEvent_t t2 = tmark(g);
  if (!reuse) {
    CG_CUDA(samples_prepare(g, n), where);
    g->index_gen += 1;
    g->index_valid = true;
  }
  if (t.ranges_gen != g->index_gen) {
    CG_CUDA(tiles_ranges(g, t), where);
    t.ranges_gen = g->index_gen;
  }
  cudaEvent_t t3 = tmark(g);
  // host-buffer calls: the index is built while the channel data still copy
  if (g->data_ready) CG_CUDA(cudaStreamWaitEvent(g->stream, g->data_ready, 0), where);
  if (tc) {
    const bool fuse = out != nullptr && g->acc_empty;
    const int mode = fuse ? 2 : (g->acc_empty ? 0 : 1);
    CG_CUDA(grid_tiles_tc(g, data, mode, out, out_w, g->path != CG_PATH_TC_FAST), where);
    if (fused) *fused = fuse;
  } else {
    // one-shot calls: the gridder writes R = N / W itself where it can
    const bool want = out != nullptr && g->acc_empty;
    bool direct = false;
    CG_CUDA(grid_tiles_f32(g, data, dtype, want ? out : nullptr, want ? out_w : nullptr, &direct),
            where);
    if (fused) *fused = direct;
  }
  cudaEvent_t t4 = tmark(g);
  tstage(g, 0, t0, t1);
  tstage(g, 1, t1, t2);
  tstage(g, 2, t2, t3);
  tstage(g, 3, t3, t4);
  g->last_path = tc ? (g->path == CG_PATH_TC_FAST ? CG_PATH_TC_FAST : CG_PATH_TC) : CG_PATH_FP32;
  g->total_n += n;
  if (!(fused && *fused)) g->acc_empty = false;
  return CG_OK;
}

// Reset, add, finalize (the body of the one-shot calls).
cg_status oneshot_impl(cg_grid* g, const double* lon, const double* lat, const void* data,
                       int32_t dtype, const float* weights, int64_t n, float* out,
                       int32_t layout_channel_major, float* out_w, const char* where) {
  cg_status st = zero_acc(g);
  if (st != CG_OK) return st;
  bool fused = false;
  st = do_add(g, lon, lat, data, dtype, weights, n, where, layout_channel_major ? nullptr : out,
              out_w, &fused);
  if (st != CG_OK) return st;
  if (fused) return CG_OK;  // the gridder's epilogue already wrote Eq. 3
  st = clear_if_empty(g, where);
  if (st != CG_OK) return st;
  cudaEvent_t t0 = tmark(g);
  CG_CUDA(finalize_maps(g, out, layout_channel_major ? 1 : 0, out_w), where);
  tstage(g, 4, t0, tmark(g));
  return CG_OK;
}

void free_pipe(cg_grid* g) {
  HostPipe* p = g->pipe;
  if (!p) return;
  if (p->s_in) cudaStreamSynchronize(p->s_in);
  if (p->s_out) cudaStreamSynchronize(p->s_out);
  for (int i = 0; i < 2; ++i) {
    cudaFree(p->lon[i]);
    cudaFree(p->lat[i]);
    cudaFree(p->data[i]);
    cudaFree(p->weights[i]);
    cudaFree(p->out[i]);
    cudaFree(p->out_w[i]);
    if (p->coords[i]) cudaEventDestroy(p->coords[i]);
    if (p->in_done[i]) cudaEventDestroy(p->in_done[i]);
    if (p->comp_done[i]) cudaEventDestroy(p->comp_done[i]);
    if (p->out_done[i]) cudaEventDestroy(p->out_done[i]);
  }
  if (p->s_in) cudaStreamDestroy(p->s_in);
  if (p->s_out) cudaStreamDestroy(p->s_out);
  delete p;
  g->pipe = nullptr;
}

}  // namespace

// error reporting for the other host translation units (the batch API)
cg_status cg::batch_fail(cg_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}

extern "C" {

const char* cg_last_error(void) { return g_last_error.c_str(); }

cg_status cg_grid_create(cg_grid** out, const double* lon_deg, const double* lat_deg,
                         int64_t n_targets, int32_t n_channels, void* stream) {
  g_last_error.clear();
  if (!out) return fail(CG_EINVAL, "cg_grid_create: out is null");
  *out = nullptr;
  if (!lon_deg || !lat_deg) return fail(CG_EINVAL, "cg_grid_create: null target coordinates");
  if (n_targets < 1 || n_targets > 0x7fffffffLL)
    return fail(CG_EINVAL, "cg_grid_create: n_targets must be in [1, 2^31-1]");
  if (n_channels < 1 || n_channels > 65536)
    return fail(CG_EINVAL, "cg_grid_create: n_channels must be in [1, 65536]");
  cg_grid* g = new (std::nothrow) cg_grid();
  if (!g) return fail(CG_ENOMEM, "cg_grid_create: host allocation failed");
  g->stream = static_cast<cudaStream_t>(stream);
  g->P = n_targets;
  g->C = n_channels;
  cudaError_t e = cudaGetDevice(&g->device);
  if (e == cudaSuccess) e = dalloc(&g->d_err, 1, g->stream);
  if (e == cudaSuccess) e = dalloc(&g->d_pairs, 1, g->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(g->d_err, 0, sizeof(unsigned), g->stream);
  if (e == cudaSuccess) e = targets_build(g, lon_deg, lat_deg);
  const int64_t slots = g->n_slots;
  if (e == cudaSuccess) e = dalloc(&g->acc_num, (size_t)slots * g->C, g->stream);
  if (e == cudaSuccess) e = dalloc(&g->acc_w, (size_t)slots, g->stream);
  if (e != cudaSuccess) {
    cg_status st = cuda_fail(e, "cg_grid_create");
    free_all(g);
    cudaStreamSynchronize(g->stream);
    delete g;
    return st;
  }
  cg_status st = zero_acc(g);
  if (st == CG_OK) st = check_device(g, "cg_grid_create");
  if (st != CG_OK) {
    free_all(g);
    cudaStreamSynchronize(g->stream);
    delete g;
    return st;
  }
  *out = g;
  return CG_OK;
}

cg_status cg_set_kernel(cg_grid* g, int32_t kernel_type, const double* params, int32_t n_params,
                        double support_deg, int32_t nside, double hpx_maxres_deg) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_set_kernel: null handle");
  if (!params) return fail(CG_EINVAL, "cg_set_kernel: params is null");
  double sig1 = 0, sig2 = 0, pa = 0;
  if (kernel_type == CG_GAUSS1D) {
    if (n_params < 1 || !finite_pos(params[0]))
      return fail(CG_EINVAL, "cg_set_kernel: gauss1d needs params = {sigma > 0}");
    sig1 = sig2 = params[0];
  } else if (kernel_type == CG_GAUSS2D) {
    if (n_params < 3 || !finite_pos(params[0]) || !finite_pos(params[1]) ||
        !std::isfinite(params[2]))
      return fail(CG_EINVAL,
                  "cg_set_kernel: gauss2d needs params = {sigma_maj > 0, sigma_min > 0, PA}");
    sig1 = params[0];
    sig2 = params[1];
    pa = params[2];
  } else if (kernel_type == CG_TSINC) {
    if (n_params < 2 || !finite_pos(params[0]) || !finite_pos(params[1]))
      return fail(CG_EINVAL, "cg_set_kernel: tsinc needs params = {a > 0, b > 0}");
    sig1 = sig2 = params[1];
  } else {
    return fail(CG_EINVAL, "cg_set_kernel: unknown kernel type %d", kernel_type);
  }
  if (!finite_pos(support_deg) || support_deg > 180.0)
    return fail(CG_EINVAL, "cg_set_kernel: support must be in (0, 180] degrees");
  int ns = nside;
  if (ns == 0) {
    if (!finite_pos(hpx_maxres_deg))
      return fail(CG_EINVAL, "cg_set_kernel: hpx_maxres must be > 0 when nside = 0");
    // Sect. 3.5: hpx-max-resolution ~ sigma/2; smallest power of two nside
    // with pixel size sqrt(pi/3)/nside <= hpx_maxres
    const double target = hpx_maxres_deg * kDeg2Rad;
    ns = 1;
    while (ns < 8192 && std::sqrt(kPi / 3.0) / ns > target) ns *= 2;
  }
  if (ns < 1 || ns > 8192) return fail(CG_EINVAL, "cg_set_kernel: nside must be in [1, 8192]");
  CG_CUDA(cudaSetDevice(g->device), "cg_set_kernel");
  g->kernel_type = kernel_type;
  g->kparams[0] = params[0];
  g->kparams[1] = (kernel_type == CG_GAUSS2D || kernel_type == CG_TSINC) ? params[1] : 0.0;
  g->kparams[2] = (kernel_type == CG_GAUSS2D) ? params[2] : 0.0;
  g->support_deg = support_deg;
  g->nside = ns;
  KernelDev kd{};
  kd.type = kernel_type;
  const double log2e = 1.4426950408889634;
  const double s1 = sig1 * kDeg2Rad, s2 = sig2 * kDeg2Rad;
  kd.k1 = (float)(-log2e / (2.0 * s1 * s1));
  kd.k2 = (float)(-log2e / (2.0 * s2 * s2));
  if (kernel_type == CG_TSINC) {   // taper exp(-d^2 / b^2), zeros of the sinc at d = a, 2a, ...
    kd.k1 = (float)(-log2e / (s1 * s1));
    kd.inv_a = (float)(1.0 / (params[0] * kDeg2Rad));
  }
  const double r = support_deg * kDeg2Rad;
  const double chord = 2.0 * std::sin(0.5 * std::fmin(r, kPi));
  kd.r_rad = r;
  {
    const double c2r = chord * chord;
    kd.c2r_hi = (float)c2r;
    kd.c2r_lo = (float)(c2r - (double)kd.c2r_hi);
    kd.c2r_tol = (float)(1e-9 * c2r + 1e-12 * chord);
  }
  kd.c2_cut = (float)(chord * chord);
  kd.c2_in = (float)(chord * chord * (1.0 - 1e-5));
  kd.c2_out = (float)(chord * chord * (1.0 + 1e-5));
  kd.big_support = chord > 0.1 ? 1 : 0;
  g->kdev = kd;
  if (kernel_type == CG_GAUSS2D) CG_CUDA(targets_set_axes(g, pa), "cg_set_kernel");
  CG_CUDA(tiles_query(g, g->t64), "cg_set_kernel");
  CG_CUDA(tiles_query(g, g->t128), "cg_set_kernel");
  // nside and tiles may have changed: the sample and target indices are stale
  g->index_valid = false;
  g->t64.ranges_gen = g->t128.ranges_gen = -1;
  g->tix_valid = false;
  cg_status st = zero_acc(g);
  if (st != CG_OK) return st;
  g->kernel_set = true;
  return check_device(g, "cg_set_kernel");
}

cg_status cg_grid_add(cg_grid* g, const double* lon_deg, const double* lat_deg,
                      const void* data, int32_t data_dtype, const float* weights,
                      int64_t n_samples) {
  g_last_error.clear();
  return do_add(g, lon_deg, lat_deg, data, data_dtype, weights, n_samples, "cg_grid_add");
}

cg_status cg_grid_finalize(cg_grid* g, float* out, int32_t layout_channel_major,
                           float* out_weights) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_grid_finalize: null handle");
  if (!out) return fail(CG_EINVAL, "cg_grid_finalize: out is null");
  CG_CUDA(cudaSetDevice(g->device), "cg_grid_finalize");
  cg_status st = clear_if_empty(g, "cg_grid_finalize");
  if (st != CG_OK) return st;
  cudaEvent_t t0 = tmark(g);
  CG_CUDA(finalize_maps(g, out, layout_channel_major ? 1 : 0, out_weights), "cg_grid_finalize");
  tstage(g, 4, t0, tmark(g));
  return check_device(g, "cg_grid_finalize");
}

cg_status cg_grid_oneshot(cg_grid* g, const double* lon_deg, const double* lat_deg,
                          const void* data, int32_t data_dtype, const float* weights,
                          int64_t n_samples, float* out, int32_t layout_channel_major,
                          float* out_weights) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_grid_oneshot: null handle");
  if (!out) return fail(CG_EINVAL, "cg_grid_oneshot: out is null");
  if (!g->kernel_set) return fail(CG_ESTATE, "cg_grid_oneshot: call cg_set_kernel first");
  CG_CUDA(cudaSetDevice(g->device), "cg_grid_oneshot");
  return oneshot_impl(g, lon_deg, lat_deg, data, data_dtype, weights, n_samples, out,
                      layout_channel_major, out_weights, "cg_grid_oneshot");
}

cg_status cg_grid_oneshot_host(cg_grid* g, const double* h_lon, const double* h_lat,
                               const void* h_data, int32_t data_dtype, const float* h_weights,
                               int64_t n_samples, float* h_out, int32_t layout_channel_major,
                               float* h_out_weights) {
  const char* where = "cg_grid_oneshot_host";
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (!h_lon || !h_lat || !h_data || !h_out)
    return fail(CG_EINVAL, "%s: null coordinate, data or output pointer", where);
  if (data_dtype != CG_F32 && data_dtype != CG_BF16)
    return fail(CG_EINVAL, "%s: data_dtype must be CG_F32 or CG_BF16", where);
  if (n_samples < 0 || n_samples > 0x7fffffffLL)
    return fail(CG_EINVAL, "%s: n_samples out of range", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  if (!g->pipe) {
    HostPipe* p = new HostPipe();
    g->pipe = p;
    CG_CUDA(cudaStreamCreateWithFlags(&p->s_in, cudaStreamNonBlocking), where);
    CG_CUDA(cudaStreamCreateWithFlags(&p->s_out, cudaStreamNonBlocking), where);
    for (int i = 0; i < 2; ++i) {
      CG_CUDA(cudaEventCreateWithFlags(&p->coords[i], cudaEventDisableTiming), where);
      CG_CUDA(cudaEventCreateWithFlags(&p->in_done[i], cudaEventDisableTiming), where);
      CG_CUDA(cudaEventCreateWithFlags(&p->comp_done[i], cudaEventDisableTiming), where);
      CG_CUDA(cudaEventCreateWithFlags(&p->out_done[i], cudaEventDisableTiming), where);
    }
  }
  HostPipe* p = g->pipe;
  const int s = p->next;
  p->next ^= 1;
  const size_t n = (size_t)n_samples;
  const size_t dbytes = n * (size_t)g->C * (data_dtype == CG_BF16 ? 2 : 4);
  const size_t obytes = (size_t)g->P * (size_t)g->C * sizeof(float);
  // (re)allocate this slot's staging once its previous use has drained
  if (p->cap_n[s] < n || p->cap_data[s] < dbytes || !p->have_out[s] ||
      (h_out_weights && !p->have_w[s])) {
    if (p->used[s]) CG_CUDA(cudaEventSynchronize(p->out_done[s]), where);
    if (p->cap_n[s] < n) {
      cudaFree(p->lon[s]);
      cudaFree(p->lat[s]);
      cudaFree(p->weights[s]);
      p->lon[s] = p->lat[s] = nullptr;
      p->weights[s] = nullptr;
      p->cap_n[s] = 0;
      const size_t m = n > 0 ? n : 1;
      CG_CUDA(cudaMalloc(&p->lon[s], m * sizeof(double)), where);
      CG_CUDA(cudaMalloc(&p->lat[s], m * sizeof(double)), where);
      CG_CUDA(cudaMalloc(&p->weights[s], m * sizeof(float)), where);
      p->cap_n[s] = n;
    }
    if (p->cap_data[s] < dbytes) {
      cudaFree(p->data[s]);
      p->data[s] = nullptr;
      p->cap_data[s] = 0;
      CG_CUDA(cudaMalloc(&p->data[s], dbytes > 0 ? dbytes : 16), where);
      p->cap_data[s] = dbytes;
    }
    if (!p->have_out[s]) {
      CG_CUDA(cudaMalloc(&p->out[s], obytes > 0 ? obytes : 16), where);
      p->have_out[s] = true;
    }
    if (h_out_weights && !p->have_w[s]) {
      CG_CUDA(cudaMalloc(&p->out_w[s], (size_t)(g->P > 0 ? g->P : 1) * sizeof(float)), where);
      p->have_w[s] = true;
    }
  }
  // copy-in: after the compute that last read this slot's inputs
  if (p->used[s]) CG_CUDA(cudaStreamWaitEvent(p->s_in, p->comp_done[s], 0), where);
  CG_CUDA(cudaMemcpyAsync(p->lon[s], h_lon, n * sizeof(double), cudaMemcpyHostToDevice, p->s_in),
          where);
  CG_CUDA(cudaMemcpyAsync(p->lat[s], h_lat, n * sizeof(double), cudaMemcpyHostToDevice, p->s_in),
          where);
  if (h_weights)
    CG_CUDA(cudaMemcpyAsync(p->weights[s], h_weights, n * sizeof(float), cudaMemcpyHostToDevice,
                            p->s_in),
            where);
  CG_CUDA(cudaEventRecord(p->coords[s], p->s_in), where);
  CG_CUDA(cudaMemcpyAsync(p->data[s], h_data, dbytes, cudaMemcpyHostToDevice, p->s_in), where);
  CG_CUDA(cudaEventRecord(p->in_done[s], p->s_in), where);
  // compute: the index waits for the coordinates only, the gridder for the
  // data; the map buffer must have been copied out by this slot's last use
  CG_CUDA(cudaStreamWaitEvent(g->stream, p->coords[s], 0), where);
  if (p->used[s]) CG_CUDA(cudaStreamWaitEvent(g->stream, p->out_done[s], 0), where);
  g->data_ready = p->in_done[s];
  cg_status st = oneshot_impl(g, p->lon[s], p->lat[s], p->data[s], data_dtype,
                              h_weights ? p->weights[s] : nullptr, n_samples, p->out[s],
                              layout_channel_major, h_out_weights ? p->out_w[s] : nullptr, where);
  g->data_ready = nullptr;
  if (st != CG_OK) return st;
  // the gridder may have been skipped (no samples): order the data copy anyway
  CG_CUDA(cudaStreamWaitEvent(g->stream, p->in_done[s], 0), where);
  CG_CUDA(cudaEventRecord(p->comp_done[s], g->stream), where);
  // copy-out
  CG_CUDA(cudaStreamWaitEvent(p->s_out, p->comp_done[s], 0), where);
  CG_CUDA(cudaMemcpyAsync(h_out, p->out[s], obytes, cudaMemcpyDeviceToHost, p->s_out), where);
  if (h_out_weights)
    CG_CUDA(cudaMemcpyAsync(h_out_weights, p->out_w[s], (size_t)g->P * sizeof(float),
                            cudaMemcpyDeviceToHost, p->s_out),
            where);
  CG_CUDA(cudaEventRecord(p->out_done[s], p->s_out), where);
  p->used[s] = true;
  return CG_OK;
}

cg_status cg_grid_reset(cg_grid* g) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_grid_reset: null handle");
  CG_CUDA(cudaSetDevice(g->device), "cg_grid_reset");
  return zero_acc(g);
}

cg_status cg_grid_destroy(cg_grid* g) {
  g_last_error.clear();
  if (!g) return CG_OK;
  cudaSetDevice(g->device);
  free_pipe(g);
  free_all(g);
  cudaError_t e = cudaStreamSynchronize(g->stream);
  delete g;
  if (e != cudaSuccess) return cuda_fail(e, "cg_grid_destroy");
  return CG_OK;
}

cg_status cg_set_stream(cg_grid* g, void* stream) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_set_stream: null handle");
  // order the new stream after all work already enqueued on the old one
  CG_CUDA(cudaStreamSynchronize(g->stream), "cg_set_stream");
  g->stream = static_cast<cudaStream_t>(stream);
  return CG_OK;
}

cg_status cg_set_path(cg_grid* g, int32_t path) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_set_path: null handle");
  if (path < CG_PATH_AUTO || path > CG_PATH_TC_FAST)
    return fail(CG_EINVAL, "cg_set_path: bad path");
  g->path = path;
  return CG_OK;
}

cg_status cg_sync(cg_grid* g) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_sync: null handle");
  CG_CUDA(cudaSetDevice(g->device), "cg_sync");
  if (g->pipe) {
    CG_CUDA(cudaStreamSynchronize(g->pipe->s_in), "cg_sync");
    CG_CUDA(cudaStreamSynchronize(g->pipe->s_out), "cg_sync");
  }
  return check_device(g, "cg_sync");
}

cg_status cg_get_info(cg_grid* g, cg_info* info) {
  g_last_error.clear();
  if (!g || !info) return fail(CG_EINVAL, "cg_get_info: null argument");
  info->n_targets = g->P;
  info->n_channels = g->C;
  info->nside = g->nside;
  const bool tc = g->last_path == CG_PATH_TC || g->last_path == CG_PATH_TC_FAST;
  info->n_tiles = tc ? g->t128.n_tiles : g->t64.n_tiles;
  info->tile_size = tc ? kTile2 : kTile;
  info->path = g->last_path;
  info->n_ranges = tc ? g->t128.n_ranges : g->t64.n_ranges;
  info->n_samples_total = g->total_n;
  info->n_launches = g->n_launches;
  unsigned long long pairs = 0;
  CG_CUDA(cudaSetDevice(g->device), "cg_get_info");
  CG_CUDA(cudaMemcpyAsync(&pairs, g->d_pairs, sizeof pairs, cudaMemcpyDeviceToHost, g->stream),
          "cg_get_info");
  CG_CUDA(cudaStreamSynchronize(g->stream), "cg_get_info");
  info->n_pairs = (int64_t)pairs;
  info->n_candidates = 0;
  const Tiling& t = tc ? g->t128 : g->t64;
  if (t.tile_cand && t.ranges_gen == g->index_gen && t.n_tiles > 0) {
    std::vector<int32_t> h((size_t)t.n_tiles);
    CG_CUDA(cudaMemcpy(h.data(), t.tile_cand, sizeof(int32_t) * (size_t)t.n_tiles,
                       cudaMemcpyDeviceToHost),
            "cg_get_info");
    int64_t sum = 0;
    for (int32_t v : h) sum += v;
    info->n_candidates = sum;
  }
  return CG_OK;
}

cg_status cg_set_timing(cg_grid* g, int32_t enable) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_set_timing: null handle");
  g->timing = enable != 0;
  return CG_OK;
}

cg_status cg_read_timing(cg_grid* g, double* ms, int64_t* n_grid_launches) {
  g_last_error.clear();
  if (!g || !ms) return fail(CG_EINVAL, "cg_read_timing: null argument");
  CG_CUDA(cudaSetDevice(g->device), "cg_read_timing");
  CG_CUDA(cudaStreamSynchronize(g->stream), "cg_read_timing");
  for (int i = 0; i < CG_N_STAGES; ++i) ms[i] = 0.0;
  int64_t ng = 0;
  for (auto& r : g->timing_recs) {
    float t = 0.f;
    CG_CUDA(cudaEventElapsedTime(&t, r.a, r.b), "cg_read_timing");
    if (r.stage >= 0 && r.stage < CG_N_STAGES) ms[r.stage] += t;
    if (r.stage == 3) ++ng;
  }
  if (n_grid_launches) *n_grid_launches = ng;
  release_events(g);
  return CG_OK;
}

cg_status cg_ang2pix_ring(int32_t nside, const double* lon_deg, const double* lat_deg, int64_t n,
                          int64_t* pix, void* stream) {
  g_last_error.clear();
  if (nside < 1 || nside > (1 << 20)) return fail(CG_EINVAL, "cg_ang2pix_ring: bad nside");
  if (n < 0) return fail(CG_EINVAL, "cg_ang2pix_ring: n < 0");
  if (n > 0 && (!lon_deg || !lat_deg || !pix))
    return fail(CG_EINVAL, "cg_ang2pix_ring: null pointer");
  CG_CUDA(ang2pix_export(nside, lon_deg, lat_deg, n, pix, static_cast<cudaStream_t>(stream)),
          "cg_ang2pix_ring");
  return CG_OK;
}

cg_status cg_set_f32_shape(cg_grid* g, int32_t shape) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_set_f32_shape: null handle");
  if (shape < -1 || shape >= kF32Configs)
    return fail(CG_EINVAL, "cg_set_f32_shape: shape must be -1 or in [0, %d)", kF32Configs);
  g->f32_cfg = shape;
  return CG_OK;
}

cg_status cg_degrid(cg_grid* g, const float* map, const float* map_weights, float* out,
                    int64_t n) {
  g_last_error.clear();
  const char* where = "cg_degrid";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (!g->index_valid)
    return fail(CG_ESTATE, "%s: no sample index: call cg_grid_add (or oneshot) first", where);
  if (n != g->last_n)
    return fail(CG_EINVAL, "%s: n (%lld) must equal the last add's n_samples (%lld)", where,
                (long long)n, (long long)g->last_n);
  if (!map || !out) return fail(CG_EINVAL, "%s: null map or out pointer", where);
  if (!map_weights && g->acc_empty)
    return fail(CG_ESTATE,
                "%s: no accumulated weight map (one-shot calls leave none): pass map_weights",
                where);
  CG_CUDA(cudaSetDevice(g->device), where);
  CG_CUDA(grid_degrid(g, map, map_weights, out), where);
  return CG_OK;
}

cg_status cg_interp(cg_grid* g, const float* map, float* out, float* out_weights, int64_t n) {
  g_last_error.clear();
  const char* where = "cg_interp";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (!g->index_valid)
    return fail(CG_ESTATE, "%s: no sample index: call cg_grid_add (or oneshot) first", where);
  if (n != g->last_n)
    return fail(CG_EINVAL, "%s: n (%lld) must equal the last add's n_samples (%lld)", where,
                (long long)n, (long long)g->last_n);
  if (!map || !out) return fail(CG_EINVAL, "%s: null map or out pointer", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  CG_CUDA(grid_degrid(g, map, nullptr, out, true, out_weights), where);
  return CG_OK;
}

cg_status cg_grid_oneshot_pcw(cg_grid* g, const double* lon_deg, const double* lat_deg,
                              const void* data, int32_t data_dtype, const float* pc_weights,
                              int64_t n_samples, float* out, int32_t layout_channel_major,
                              float* out_weights) {
  g_last_error.clear();
  const char* where = "cg_grid_oneshot_pcw";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (data_dtype != CG_F32 && data_dtype != CG_BF16)
    return fail(CG_EINVAL, "%s: data_dtype must be CG_F32 or CG_BF16", where);
  if (n_samples < 0 || n_samples > 0x7fffffffLL)
    return fail(CG_EINVAL, "%s: n_samples out of range", where);
  if (!lon_deg || !lat_deg || !data || !pc_weights || !out)
    return fail(CG_EINVAL, "%s: null coordinate, data, weight or output pointer", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  const int64_t n = n_samples;
  g->index_valid = false;
  if (n > 0) {
    CG_CUDA(samples_keys(g, lon_deg, lat_deg, nullptr, n), where);
    CG_CUDA(samples_sort(g, n), where);
    CG_CUDA(samples_prepare(g, n), where);
  } else {
    g->last_n = 0;
  }
  g->index_gen += 1;
  g->index_valid = n > 0;
  Tiling& t = g->t64;
  if (n > 0 && t.ranges_gen != g->index_gen) {
    CG_CUDA(tiles_ranges(g, t), where);
    t.ranges_gen = g->index_gen;
  }
  CG_CUDA(pcw_pack(g, data, data_dtype, pc_weights, n), where);
  if (n > 0) {
    CG_CUDA(grid_tiles_f32_to(g, g->pcw_data, CG_F32, g->pcw_acc, g->pcw_w, 0, 0.f, 2 * g->C),
            where);
  } else {
    CG_CUDA(cudaMemsetAsync(g->pcw_acc, 0, sizeof(float) * (size_t)g->n_slots * 2 * g->C,
                            g->stream),
            where);
  }
  CG_CUDA(pcw_finalize(g, out, layout_channel_major ? 1 : 0, out_weights), where);
  g->last_path = CG_PATH_FP32;
  return CG_OK;
}

cg_status cg_grid_dsigma(cg_grid* g, const void* data, int32_t data_dtype, const float* grad_out,
                         float* dR, double* dsigma) {
  g_last_error.clear();
  const char* where = "cg_grid_dsigma";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (!g->kernel_set) return fail(CG_ESTATE, "%s: call cg_set_kernel first", where);
  if (g->kernel_type != CG_GAUSS1D)
    return fail(CG_EINVAL, "%s: d/dsigma is defined for the circular gauss1d kernel", where);
  if (!g->index_valid)
    return fail(CG_ESTATE, "%s: no sample index: call cg_grid_add (or oneshot) first", where);
  if (data_dtype != CG_F32 && data_dtype != CG_BF16)
    return fail(CG_EINVAL, "%s: data_dtype must be CG_F32 or CG_BF16", where);
  if (!data) return fail(CG_EINVAL, "%s: null data pointer", where);
  if (dsigma && !grad_out)
    return fail(CG_EINVAL, "%s: the scalar dsigma needs grad_out", where);
  if (!dR && !dsigma) return fail(CG_EINVAL, "%s: nothing to compute (dR and dsigma NULL)", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  CG_CUDA(grid_dsigma(g, data, data_dtype, grad_out, dR, dsigma), where);
  return CG_OK;
}

cg_status cg_unit_vectors(const double* lon_deg, const double* lat_deg, int64_t n, double* xyz,
                          void* stream) {
  g_last_error.clear();
  if (n < 0) return fail(CG_EINVAL, "cg_unit_vectors: n < 0");
  if (n > 0 && (!lon_deg || !lat_deg || !xyz))
    return fail(CG_EINVAL, "cg_unit_vectors: null pointer");
  CG_CUDA(unit_vectors(lon_deg, lat_deg, n, xyz, static_cast<cudaStream_t>(stream)),
          "cg_unit_vectors");
  return CG_OK;
}

cg_status cg_grid_export_index(cg_grid* g, int64_t* sorted_pix, int64_t* perm,
                               int64_t* ring_off, int64_t n) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_grid_export_index: null handle");
  if (n != g->last_n)
    return fail(CG_EINVAL, "cg_grid_export_index: n (%lld) != samples of the last add (%lld)",
                (long long)n, (long long)g->last_n);
  if (n > 0 && (!sorted_pix || !perm)) return fail(CG_EINVAL, "cg_grid_export_index: null pointer");
  CG_CUDA(cudaSetDevice(g->device), "cg_grid_export_index");
  CG_CUDA(export_index(g, sorted_pix, perm, ring_off, n), "cg_grid_export_index");
  return CG_OK;
}

cg_status cg_md_residual(cg_grid* g, float* r, const float* data, int64_t n, double* loss) {
  g_last_error.clear();
  const char* where = "cg_md_residual";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (n < 0 || (n > 0 && (!r || !data)) || !loss)
    return fail(CG_EINVAL, "%s: null pointer or negative size", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  CG_CUDA(md_residual(g, r, data, n, loss), where);
  return CG_OK;
}

cg_status cg_md_update(cg_grid* g, float* m, const float* grad, float alpha, int64_t n) {
  g_last_error.clear();
  const char* where = "cg_md_update";
  if (!g) return fail(CG_EINVAL, "%s: null handle", where);
  if (n < 0 || (n > 0 && (!m || !grad))) return fail(CG_EINVAL, "%s: null pointer or negative size", where);
  if (!std::isfinite(alpha)) return fail(CG_EINVAL, "%s: alpha must be finite", where);
  CG_CUDA(cudaSetDevice(g->device), where);
  CG_CUDA(md_update(g, m, grad, alpha, n), where);
  return CG_OK;
}

cg_status cg_debug_hold(cg_grid* g, int32_t enable, int64_t wait_cycles) {
  g_last_error.clear();
  if (!g) return fail(CG_EINVAL, "cg_debug_hold: null handle");
  CG_CUDA(cudaSetDevice(g->device), "cg_debug_hold");
  if (enable && !g->d_hold) {
    CG_CUDA(dalloc(&g->d_hold, 1, g->stream), "cg_debug_hold");
    CG_CUDA(cudaMemsetAsync(g->d_hold, 0, sizeof(int32_t), g->stream), "cg_debug_hold");
  }
  g->hold = enable != 0;
  g->hold_cycles = wait_cycles > 0 ? wait_cycles : 2000000;
  return CG_OK;
}

cg_status cg_sort_samples_noalloc(int32_t nside, const double* lon_deg, const double* lat_deg,
                                  int64_t n, int64_t* sorted_pix, int64_t* perm, void* stream) {
  g_last_error.clear();
  if (nside < 1 || nside > 8192)
    return fail(CG_EINVAL, "cg_sort_samples_noalloc: nside must be in [1, 8192]");
  if (n < 0 || n > CG_NOALLOC_MAX_SAMPLES)
    return fail(CG_EINVAL,
                "cg_sort_samples_noalloc: n = %lld exceeds the no-allocation limit of %d samples",
                (long long)n, CG_NOALLOC_MAX_SAMPLES);
  if (n > 0 && (!lon_deg || !lat_deg || !sorted_pix || !perm))
    return fail(CG_EINVAL, "cg_sort_samples_noalloc: null pointer");
  CG_CUDA(sort_samples_noalloc(nside, lon_deg, lat_deg, n, sorted_pix, perm,
                               static_cast<cudaStream_t>(stream)),
          "cg_sort_samples_noalloc");
  return CG_OK;
}

}  // extern "C"
