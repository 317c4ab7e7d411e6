// cg_internal.h -- the handle and the host-side launch wrappers shared by the
// translation units of the library.  Not part of the public C ABI.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include <vector>

// the public C ABI is the only thing the shared library exports
#pragma GCC visibility push(default)
#include "../../include/cygrid_gb300.h"
#pragma GCC visibility pop

namespace cg {

// Tile sizes: targets grouped per CTA (FP32 form: 64; tensor-core form: 128,
// the M dimension of one tcgen05 MMA).  The 128-tiles are unions of two
// sibling 64-tiles, so both tilings share one slot layout.
constexpr int kTile = 64;
constexpr int kTile2 = 128;
// Candidate samples staged per chunk.
constexpr int kChunk = 32;

struct Range {            // one contiguous pixel interval of one ring
  int32_t pix_lo;         // first pixel (inclusive)
  int32_t pix_hi;         // last pixel (inclusive)
  int32_t ring;           // ring number 1 .. 4ns-1
  int32_t pad;
};

struct KernelDev {        // kernel constants used by the gridder
  int type;               // CG_GAUSS1D / CG_GAUSS2D
  float k1, k2;           // -log2(e) / (2 sigma^2) [rad^-2] (gauss2d: major, minor)
  float c2_in, c2_out;    // chord^2 below c2_in: inside; above c2_out: outside
  float c2_cut;           // chord^2 of the support radius
  double r_rad;           // support radius (FP64 guard-band decision)
  float c2r_hi, c2r_lo;   // FP64 squared chord of r as a double-float pair
  float c2r_tol;          // tolerance of the double-float squared chord of a pair
  int big_support;        // 1 if the chord series for d^2 is not accurate enough
  float dscale;           // 0; else the weight is w d^2 dscale (d/dsigma pass)
  float inv_a;            // CG_TSINC: 1 / a (rad^-1); k1 then holds the taper -log2(e)/b^2
};

struct Tiling {           // geometry of one tiling of the targets
  int T = 0;
  int64_t n_tiles = 0;
  float4* chi = nullptr;          // [n_tiles] centre hi (xyz), w = radius (rad)
  float4* clo = nullptr;          // [n_tiles] centre lo (xyz)
  double4* c64 = nullptr;         // [n_tiles] FP64 centre, w = radius
  float4* a = nullptr;            // [n_tiles*T] u_t - centre (FP32)
  int64_t n_ranges = 0;
  int64_t* range_off = nullptr;   // [n_tiles + 1]
  Range* ranges = nullptr;        // [n_ranges]
  int2* range_s = nullptr;        // [n_ranges] sample ranges [lo, hi) of the last add
  int32_t* range_c = nullptr;     // [n_ranges] the tile's candidates before each range
  int32_t* tile_cand = nullptr;   // [n_tiles] candidates per tile of the last add
  int32_t* order = nullptr;       // [cap_order] persistent schedule: waves of neighbouring items
  int64_t cap_order = 0;
  // 128-target tiles only: the four 32-target quarters (one TMEM lane quarter
  // each; k-d leaves), FP64 centre + radius, and the centre relative to the
  // tile centre in FP32 with the radius as a chord
  double4* sub64 = nullptr;       // [n_tiles * 4]
  float4* subf = nullptr;         // [n_tiles * 4]
  // every tile: its 4-target groups (compact k-d leaves), FP64 centre + radius
  // (radius < 0: an empty group); the candidate query's discs
  double4* grp64 = nullptr;       // [n_tiles * T / 4]
  int64_t ranges_gen = -1;        // sample index the per-add ranges belong to
};

struct SortWork {         // radix-sort scratch
  void* keys_alt = nullptr;
  uint32_t* vals_alt = nullptr;
  uint32_t* hist = nullptr;     // [256 * nblk]
  uint32_t* totals = nullptr;   // [256]
  size_t cap_n = 0, cap_hist = 0, key_bytes = 0;
  // one-sweep passes (32-bit keys)
  uint64_t* status = nullptr;   // [nblk * 256] epoch-tagged look-back words
  uint32_t* os_meta = nullptr;  // digit totals [4][256] + tickets [4]
  size_t cap_status = 0;
  uint32_t epoch = 0;
  unsigned* err = nullptr;      // device error word for bounded waits
};

}  // namespace cg

namespace cg {
// Staging for cg_grid_oneshot_host: two slots of device buffers, a copy-in
// and a copy-out stream, and the events that order the three streams.
struct HostPipe {
  cudaStream_t s_in = nullptr, s_out = nullptr;
  cudaEvent_t coords[2] = {}, in_done[2] = {}, comp_done[2] = {}, out_done[2] = {};
  bool used[2] = {false, false};
  double* lon[2] = {};
  double* lat[2] = {};
  void* data[2] = {};
  float* weights[2] = {};
  float* out[2] = {};
  float* out_w[2] = {};
  size_t cap_n[2] = {0, 0}, cap_data[2] = {0, 0};
  bool have_out[2] = {false, false}, have_w[2] = {false, false};
  int next = 0;
};
}  // namespace cg

struct cg_grid {
  int device = 0;
  cudaStream_t stream = nullptr;
  cg::HostPipe* pipe = nullptr;   // cg_grid_oneshot_host staging (created on first use)
  cudaEvent_t data_ready = nullptr;  // if set: the gridder waits for it (channel data copy)
  int64_t P = 0;
  int32_t C = 0;
  int32_t path = CG_PATH_AUTO;
  int32_t f32_cfg = -1;           // FP32 gridder shape (-1: by channel count)
  int32_t last_path = CG_PATH_FP32;

  // targets, in tile order (slot = tile * T + lane; empty slots marked)
  cg::Tiling t64, t128;
  int64_t n_slots = 0;            // t128.n_tiles * kTile2 (>= t64.n_tiles * kTile)
  uint32_t* tgt_perm = nullptr;   // [n_slots] user index or 0xffffffff
  float4* tgt_e = nullptr;        // [slots] local east unit vector
  float4* tgt_n = nullptr;        // [slots] local north unit vector
  float4* tgt_f1 = nullptr;       // [slots] major-axis direction (set_kernel)
  float4* tgt_f2 = nullptr;       // [slots] minor-axis direction (set_kernel)
  double2* tgt_ll = nullptr;      // [slots] lon/lat degrees (FP64)

  // kernel and candidate query
  bool kernel_set = false;
  int32_t kernel_type = 0;
  double kparams[3] = {0, 0, 0};
  double support_deg = 0;
  int32_t nside = 0;
  cg::KernelDev kdev{};

  // per-add sample workspace
  size_t cap_n = 0;
  uint32_t* key = nullptr;        // [cap_n] RING index of each sample
  uint32_t* val = nullptr;        // [cap_n] sample index
  cg::SortWork sw;
  uint32_t* sorted_key = nullptr; // points at key or sw.keys_alt after the sort
  uint32_t* sorted_val = nullptr;
  float4* s_hi = nullptr;         // [cap_n] sorted samples: unit vector hi, w = omega
  float4* s_lo = nullptr;         // [cap_n] unit vector lo
  // [2 cap_n] input order: per sample one 32-byte record, unit vector hi
  // (w = omega) then lo, so that the gather into sorted order reads one sector
  float4* u_rec = nullptr;
  double2* s_ll = nullptr;        // [cap_n] input order: FP64 lon/lat (guard-band decisions)
  int32_t* ring_off = nullptr;    // [4*nside + 1]
  int64_t last_n = 0;
  int64_t total_n = 0;
  bool index_valid = false;       // the sample index of the last add is usable
  int64_t index_gen = 0;          // bumped by every new sample index

  // target index of the degridder (RING keys of the targets, sorted; built on
  // the first cg_degrid after cg_set_kernel)
  bool tix_valid = false;
  uint32_t* tix_key = nullptr;    // [n_slots] RING key per slot (npix: empty slot)
  uint32_t* tix_val = nullptr;    // [n_slots] slot
  uint32_t* tix_skey = nullptr;   // sorted keys (into tix_key or tix_sw)
  uint32_t* tix_sslot = nullptr;  // slot of each sorted key
  float4* tix_uhi = nullptr;      // [n_slots] slot order unit vector hi
  float4* tix_ulo = nullptr;
  float4* tix_hi = nullptr;       // [n_slots] sorted order
  float4* tix_lo = nullptr;
  int32_t* tix_ring_off = nullptr;  // [4 nside + 1]
  float* tix_invw = nullptr;      // [n_slots] 1 / W of the operator being transposed
  cg::SortWork tix_sw;
  // scratch accumulators of cg_grid_dsigma (w' = dw/dsigma pass)
  float* ds_num = nullptr;        // [slots][C]
  float2* ds_w = nullptr;         // [slots]
  float* ds_num0 = nullptr;       // [slots][C] (w pass)
  float2* ds_w0 = nullptr;        // [slots]
  double* ds_part = nullptr;      // per-block partial sums
  double* md_part = nullptr;      // map making: per-block partial sums of r^2
  size_t md_cap = 0;
  // one weight per sample and channel: [N][2C] (omega D | omega) and its
  // [slots][2C] accumulators (cg_grid_oneshot_pcw)
  float* pcw_data = nullptr;
  float* pcw_acc = nullptr;
  float2* pcw_w = nullptr;
  size_t pcw_cap_data = 0;

  // candidate-split partial sums of the FP32 gridder
  float* part_num = nullptr;      // [n_split][slots][C]
  float2* part_w = nullptr;       // [n_split][slots]
  size_t part_cap_num = 0, part_cap_w = 0;

  // accumulators (tile order)
  float* acc_num = nullptr;       // [slots][C]
  float2* acc_w = nullptr;        // [slots] double-float weight sum
  bool acc_empty = true;

  unsigned* d_err = nullptr;      // device error word
  unsigned long long* d_pairs = nullptr;  // pairs with d <= r since the last reset
  // (target slot, channel slab) rows of a gridder pass whose numerator came
  // out non-finite: one bit each, and a word set when any bit is (the fix-up
  // pass recomputes those rows and clears their bits)
  uint32_t* nf_bits = nullptr;
  uint32_t* nf_any = nullptr;
  size_t nf_words = 0;
  // cg_debug_hold: the tensor-core producers wait for d_hold (never set)
  bool hold = false;
  int64_t hold_cycles = 0;
  int32_t* d_hold = nullptr;
  int64_t n_launches = 0;         // kernels launched by this handle

  // optional stage timing (CUDA events on the handle's stream)
  struct TimingRec {
    int stage;
    cudaEvent_t a, b;
  };
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;   // idle events
  std::vector<cudaEvent_t> ev_used;   // events handed out since the last read
  std::vector<TimingRec> timing_recs; // stages refer to events in ev_used
};

namespace cg {

// k_sort.cu -- stable LSD radix sort of (key, value) pairs.
cudaError_t radix_sort_u32(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                           SortWork& w, cudaStream_t s, uint32_t** out_keys,
                           uint32_t** out_vals);
cudaError_t radix_sort_u32_scratch(uint32_t* keys, uint32_t* vals, int64_t n, int key_bits,
                                   uint32_t* keys_alt, uint32_t* vals_alt, uint32_t* hist,
                                   uint32_t* totals, cudaStream_t s, uint32_t** out_keys,
                                   uint32_t** out_vals);
cudaError_t radix_sort_u64(uint64_t* keys, uint32_t* vals, int64_t n, int key_bits,
                           SortWork& w, cudaStream_t s, uint64_t** out_keys,
                           uint32_t** out_vals);

// k_targets.cu -- target geometry and tiling.
cudaError_t targets_build(cg_grid* g, const double* lon, const double* lat);
cudaError_t targets_set_axes(cg_grid* g, double pa_deg);

// k_healpix.cu -- ang2pix, ring offsets, tile disc queries, sample ranges.
cudaError_t ang2pix_export(int nside, const double* lon, const double* lat, int64_t n,
                           int64_t* pix, cudaStream_t s);
cudaError_t samples_keys(cg_grid* g, const double* lon, const double* lat, const float* weights,
                         int64_t n);
cudaError_t unit_vectors(const double* lon, const double* lat, int64_t n, double* out,
                         cudaStream_t s);
cudaError_t samples_sort(cg_grid* g, int64_t n);
cudaError_t samples_prepare(cg_grid* g, int64_t n);
int key_bits_for(int64_t ns);   // bits of a RING key at nside (incl. the invalid sentinel)
// gather (hi, lo) records into sorted order and build ring offsets [4 ns + 1];
// record i is u_hi[i * stride], u_lo[i * stride]
cudaError_t sorted_gather(int64_t ns, const uint32_t* skey, const uint32_t* sval,
                          const float4* u_hi, const float4* u_lo, int stride, int64_t n,
                          float4* s_hi, float4* s_lo, int32_t* ring_off, cudaStream_t s);
cudaError_t tiles_ranges(cg_grid* g, Tiling& t);
cudaError_t tiles_query(cg_grid* g, Tiling& t);
void tiling_free(Tiling& t, cudaStream_t s);
cudaError_t export_index(cg_grid* g, int64_t* sorted_pix, int64_t* perm, int64_t* ring_off,
                         int64_t n);

// k_grid.cu -- the tile gridder (FP32 CUDA-core form).  Arguments of one
// gridder pass (one job): the t64 tiling, the sorted samples, the data.
struct GridArgs {
  const float4* tile_chi;
  const float4* tile_clo;
  const float4* tgt_a;
  const float4* tgt_f1;
  const float4* tgt_f2;
  const double2* tgt_ll;
  const uint32_t* tgt_perm;
  const int64_t* range_off;
  const int2* range_s;
  const float4* s_hi;
  const float4* s_lo;
  const uint32_t* perm;
  const double2* sll;   // FP64 lon/lat of each sample (input order, degrees)
  const void* data;
  int C;
  int vec4;  // data rows are 16-byte (f32) / 8-byte (bf16) aligned in groups of 4
  KernelDev kd;
  float* acc_num;
  float2* acc_w;
  int accumulate;
  unsigned long long* pairs;
  // candidate splits: a tile's candidates are shared by n_split
  // CTAs that write partial sums, summed by k_split_reduce in split order
  const int32_t* tile_cand;
  int n_split;
  int64_t n_slots;
  float* part_num;      // [n_split][slots][C]
  float2* part_w;       // [n_split][slots]
  // rows with a non-finite numerator (bit slot * n_slabs + slab)
  uint32_t* nf_bits;
  uint32_t* nf_any;
  // one-shot output (no candidate splits, no accumulation): R = N / W
  // written straight into the caller's [P][C] map and W into out_w (if
  // set); null: numerator and W into the accumulators
  float* out;
  float* out_w;
};
// out != null (one-shot call, pixel-major map): R = N / W straight into out
// when the pass has no candidate splits (*direct = true), else the
// accumulators as usual.
cudaError_t grid_tiles_f32(cg_grid* g, const void* data, int dtype, float* out = nullptr,
                           float* out_w = nullptr, bool* direct = nullptr);
constexpr int kF32Configs = 7;   // register-blocking shapes of the FP32 gridder
int f32_default_config(int C);
// the same into given accumulators; dscale != 0 evaluates w d^2 dscale
// instead of w (the d/dsigma pass) and counts no pairs
cudaError_t grid_tiles_f32_to(cg_grid* g, const void* data, int dtype, float* acc_num,
                              float2* acc_w, int accumulate, float dscale, int C = -1,
                              float* out = nullptr, float* out_w = nullptr,
                              bool* direct = nullptr);
cg_status batch_fail(cg_status st, const char* fmt, ...) __attribute__((format(printf, 2, 3)));

// ---- fused batches: one sample index for all jobs (k_healpix.cu) --------
// The samples of all jobs sorted together by a composite key: the job's key
// base (the RING index ranges of the jobs before it, each npix + 1 long) plus
// the sample's RING index at the job's nside, so that every job's samples
// form one segment of the sorted order, in the job's own key order.
struct BatchIndexJob {
  const double* lon;
  const double* lat;
  const float* weights;
  int64_t n;              // samples
  int64_t off;            // first position of the job in the batch sample arrays
  int64_t nside;
  int lg;                 // log2 nside (-1: not a power of two)
  uint64_t key_base;
  int64_t ring_base;      // first of the job's 4 nside + 1 ring offsets
  // the tiling of the job's gridder form: its candidate ranges are written
  const Range* ranges;
  const int64_t* range_off;
  int64_t n_tiles;
  int2* range_s;
  int32_t* range_c;
  int32_t* tile_cand;
};
struct BatchIndex {
  int n_jobs = 0;
  int64_t N = 0;                    // samples of all jobs
  int64_t n_ring = 0;               // ring offsets of all jobs
  int64_t n_tiles = 0;              // tiles of all jobs
  int key_bits = 0;
  BatchIndexJob* jobs = nullptr;    // device [n_jobs]
  int64_t* key_blk = nullptr;       // device [n_jobs + 1]: prefix of ceil(n / 256)
  int64_t n_key_blk = 0;
  int64_t* gth_blk = nullptr;       // device [n_jobs + 1]: prefix of ceil((n + 1) / 256)
  int64_t n_gth_blk = 0;
  int64_t* tile_off = nullptr;      // device [n_jobs + 1]: prefix of n_tiles
  uint64_t* key = nullptr;          // [N] composite keys, input order
  uint32_t* val = nullptr;          // [N] the sample's index within its job
  float4* u_rec = nullptr;          // [2 N] input order: (hi, lo) records
  double2* sll = nullptr;
  float4* s_hi = nullptr;           // [N] sorted order
  float4* s_lo = nullptr;
  uint32_t* skey = nullptr;         // [N] sorted RING keys (the job's own)
  int32_t* ring_off = nullptr;      // [n_ring] relative to the job's segment
  uint64_t* sorted_key = nullptr;   // set by the sort
  uint32_t* sorted_val = nullptr;
  SortWork sw;
};
// Allocate the sample arrays (jobs, prefixes and sizes set by the caller).
cudaError_t batch_index_alloc(BatchIndex& bi, cudaStream_t s);
// keys, one sort, gather + ring offsets, every job's candidate ranges
cudaError_t batch_index_run(BatchIndex& bi, unsigned* err, cudaStream_t s, int64_t* launches);
void batch_index_free(BatchIndex& bi, cudaStream_t s);

// ---- fused batches: one FP32 gridder launch for all jobs (k_grid.cu) ----
// Items (job, tile, channel slab, candidate split) are taken from a queue
// ordered by decreasing estimated cost; one launch per register-blocking
// shape of the one-job gridder (by channel count, or the autotuner's choice)
// and up to kF32MultiMaxJobs jobs.
constexpr int kF32MultiShapes = kF32Configs;
constexpr int kF32MultiMaxJobs = 96;  // jobs per launch (their arguments fill the parameter space)
int f32_multi_shape(int C);           // default shape for C channels (f32_default_config)
int f32_multi_cpad(int shape);        // channels per slab of a shape
struct F32MultiJob {
  GridArgs a;
  int shape;
  int dtype;
  int n_slabs;
  int pad;                            // channels per slab of the shape
};
struct F32Multi {
  int shape = 0;                      // the register-blocking shape of all its jobs
  F32MultiJob* jobs = nullptr;        // device [n_jobs]
  const F32MultiJob* hjobs = nullptr; // host copy (the launcher reads it)
  int n_jobs = 0;
  int64_t* item_off = nullptr;        // device [n_jobs + 1]: prefix of items
  int64_t n_items = 0;
  int32_t* order = nullptr;           // device [n_items]: items, costliest first
  unsigned* head = nullptr;           // queue head (cleared by the order pass)
  unsigned* err = nullptr;
  const int* hold = nullptr;          // testing hook: a word nothing sets
  long long hold_cycles = 0;
  // split reduction, normalisation and non-finite fix-up of all jobs
  struct Out {
    float* out;                       // caller's map
    float* out_w;
    int channel_major;
    int vec4;                         // [P][C], C % 4 == 0, 16-byte aligned map
    int64_t P;
  };
  Out* outs = nullptr;                // device [n_jobs]
  // CTAs of the normalisation (every job) and of the split reduction (jobs
  // with candidate splits): prefix over the jobs of their CTA counts
  int64_t* fin_blk = nullptr;         // device [n_jobs + 1]
  int64_t n_fin_blk = 0;
  int64_t* red_blk = nullptr;         // device [n_jobs + 1]
  int64_t n_red_blk = 0;
  int64_t* word_off = nullptr;        // device [n_jobs + 1]: prefix of bitmap words
  int64_t n_words = 0;
  uint32_t* nf_any = nullptr;
};
cudaError_t grid_f32_multi(const F32Multi& m, cudaStream_t s, int64_t* launches);
constexpr int kMultiFinElems = 1024;  // map values per CTA of the normalisation
constexpr int kMultiRedElems = 256;   // values per CTA of the split reduction
// k_grid_tc.cu -- the tile gridder, BF16 tcgen05 form (TMEM accumulators).
// mode 0: store into the accumulators, 1: add into them, 2: one-shot
// normalised output in the caller's [P][C] layout (out, out_w).
bool tc_supported(const cg_grid* g, int dtype, const void* data);
cudaError_t grid_tiles_tc(cg_grid* g, const void* data, int mode, float* out, float* out_w,
                          int split);
// k_grid.cu -- rows a gridder flagged as non-finite, computed again in FP32
// with only the pairs inside the support taking part; the pass returns at
// once when nothing is flagged.  Bit e = slot * n_slabs + slab of nf_bits.
struct NonfiniteRows {
  const Tiling* tiling;   // the tiling whose candidate ranges the gridder used
  const void* data;       // [n_samples][C] channel values, dtype
  int dtype;
  int C;
  int cp;                 // channels per slab (<= 256)
  int n_slabs;
  int mode;               // 0 store, 1 add (into acc_num), 2 divide by W into out
  float* out;             // mode 2: user-order map
  float* acc_num;         // modes 0, 1: slot-order numerator
  KernelDev kd;
};
// Grow the bitmap to n_bits (zeroed) and clear the "any" word.
cudaError_t nonfinite_prepare(cg_grid* g, int64_t n_bits);
cudaError_t nonfinite_fixup(cg_grid* g, const NonfiniteRows& rows);
// k_noalloc.cu -- sample index on the library's static scratch array.
cudaError_t sort_samples_noalloc(int nside, const double* lon, const double* lat, int64_t n,
                                 int64_t* sorted_pix, int64_t* perm, cudaStream_t s);
// k_finalize.cu -- normalisation and output layout.
// k_degrid.cu -- adjoint (degridding) and d/dsigma
cudaError_t target_index_build(cg_grid* g);
// one weight per sample and channel (k_variants.cu)
cudaError_t pcw_pack(cg_grid* g, const void* data, int dtype, const float* omega, int64_t n);
cudaError_t pcw_finalize(cg_grid* g, float* out, int channel_major, float* out_w);

cudaError_t grid_degrid(cg_grid* g, const float* y, const float* wmap, float* out,
                        bool interp = false, float* vsum = nullptr);
cudaError_t grid_dsigma(cg_grid* g, const void* data, int dtype, const float* grad, float* dR,
                        double* dsigma);
// map making: r <- r - d with *loss = 1/2 sum r^2 (FP64); m <- m - alpha grad
cudaError_t md_residual(cg_grid* g, float* r, const float* d, int64_t n, double* loss);
cudaError_t md_update(cg_grid* g, float* m, const float* grad, float alpha, int64_t n);

cudaError_t finalize_maps(cg_grid* g, float* out, int channel_major, float* out_w);

// device allocation helper (stream ordered); returns cudaErrorMemoryAllocation on failure
template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), s);
}
template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

inline unsigned ceil_div(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

}  // namespace cg
