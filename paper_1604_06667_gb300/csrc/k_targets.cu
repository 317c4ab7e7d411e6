// k_targets.cu -- target geometry and tiling (set-up, once per handle).
//
// The paper grids onto the pixel centres of a WCS map or onto a list of sight
// lines (Sect. 3.5, WcsGrid / SlGrid).  Here targets are always a list of
// directions.  To give each CTA a compact group of targets (its "tile"), the
// targets are split by a k-d tree over their unit vectors: every node is cut
// along its widest axis at a multiple of the leaf size, so all leaves hold
// exactly that many targets (except the last) and each leaf is a compact box.
// The tree is cut to 128-target leaves, then each leaf into 64 + 64, 32 + 32
// and on down to groups of 4, so a 128-tile is two 64-tiles, four 32-target
// quarters and thirty-two 4-target groups, all compact (consecutive slots).
// The tree is built level by level with one stable 64-bit radix sort per
// level keyed by (child node, coordinate along the child's widest axis).
// Each tile stores
//   - its centre e_c (FP64, and as a double-float pair) and angular radius;
//   - for every member, u_t - e_c in FP32 (accurate relative to its size);
//   - the local east / north unit vectors (for the elliptical kernel);
//   - the member's longitude / latitude in FP64 (guard-band recomputation).
// FP64 is acceptable here: this runs once per target set, not per sample.
#include "cg_common.cuh"
#include "cg_internal.h"

namespace cg {
namespace {

__device__ __forceinline__ uint32_t orderable(float f) {
  const uint32_t b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ bool valid_coord(double lon, double lat) {
  return isfinite(lon) && isfinite(lat) && lat >= -90.0 && lat <= 90.0;
}

__device__ __forceinline__ void unit_vec(double lon, double lat, double& x, double& y,
                                         double& z) {
  double sb, cb, sl, cl;
  sincos(lat * kDeg2Rad, &sb, &cb);
  sincos(lon * kDeg2Rad, &sl, &cl);
  x = cb * cl;
  y = cb * sl;
  z = sb;
}

__global__ void k_target_init(const double* __restrict__ lon, const double* __restrict__ lat,
                              int64_t P, float4* __restrict__ pos, uint32_t* __restrict__ ord,
                              uint32_t* __restrict__ nid, unsigned* err) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const double lo = lon[i], la = lat[i];
  float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
  if (valid_coord(lo, la)) {
    double x, y, z;
    unit_vec(lo, la, x, y, z);
    v = make_float4((float)x, (float)y, (float)z, 0.f);
  } else {
    set_error(err, ERR_BAD_TARGET);
  }
  pos[i] = v;
  ord[i] = (uint32_t)i;
  nid[i] = 0;
}

// First / one-past-last position of every node in the current order.
__global__ void k_node_bounds(const uint32_t* __restrict__ nid, int64_t P,
                              uint32_t* __restrict__ nstart, uint32_t* __restrict__ nend) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  const uint32_t n = nid[s];
  if (s == 0 || nid[s - 1] != n) nstart[n] = (uint32_t)s;
  if (s == P - 1 || nid[s + 1] != n) nend[n] = (uint32_t)(s + 1);
}

// Child of every position (left part = a multiple of kTile targets) and the
// bounding box of every child (order-preserving integer min / max).
__global__ void k_node_split(const uint32_t* __restrict__ nid, const uint32_t* __restrict__ ord,
                             const float4* __restrict__ pos, int64_t P, uint32_t leaf,
                             const uint32_t* __restrict__ nstart,
                             const uint32_t* __restrict__ nend, uint32_t* __restrict__ child,
                             uint32_t* __restrict__ bmin, uint32_t* __restrict__ bmax) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  const uint32_t n = nid[s];
  const uint32_t st = nstart[n], cnt = nend[n] - st;
  uint32_t c = 2u * n;
  if (cnt > leaf) {
    const uint32_t m = (cnt + leaf - 1) / leaf;
    const uint32_t left = leaf * (m / 2);
    if ((uint32_t)s - st >= left) c += 1u;
  }
  child[s] = c;
  const float4 v = pos[ord[s]];
  atomicMin(&bmin[3 * c + 0], orderable(v.x));
  atomicMin(&bmin[3 * c + 1], orderable(v.y));
  atomicMin(&bmin[3 * c + 2], orderable(v.z));
  atomicMax(&bmax[3 * c + 0], orderable(v.x));
  atomicMax(&bmax[3 * c + 1], orderable(v.y));
  atomicMax(&bmax[3 * c + 2], orderable(v.z));
}

__device__ __forceinline__ float from_orderable(uint32_t u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// Sort key: (child node, coordinate along the child's widest axis).
__global__ void k_node_keys(const uint32_t* __restrict__ child, const uint32_t* __restrict__ ord,
                            const float4* __restrict__ pos, int64_t P,
                            const uint32_t* __restrict__ bmin, const uint32_t* __restrict__ bmax,
                            uint64_t* __restrict__ key, uint32_t* __restrict__ val) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= P) return;
  const uint32_t c = child[s];
  const float ex = from_orderable(bmax[3 * c + 0]) - from_orderable(bmin[3 * c + 0]);
  const float ey = from_orderable(bmax[3 * c + 1]) - from_orderable(bmin[3 * c + 1]);
  const float ez = from_orderable(bmax[3 * c + 2]) - from_orderable(bmin[3 * c + 2]);
  const uint32_t o = ord[s];
  const float4 v = pos[o];
  const float coord = (ex >= ey && ex >= ez) ? v.x : ((ey >= ez) ? v.y : v.z);
  key[s] = ((uint64_t)c << 32) | orderable(coord);
  val[s] = o;
}

__global__ void k_node_unpack(const uint64_t* __restrict__ key, int64_t P,
                              uint32_t* __restrict__ nid) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < P) nid[s] = (uint32_t)(key[s] >> 32);
}

// One CTA of T threads per tile: centre, radius and tile-relative vectors.
// The T = kTile2 build also writes the per-slot data shared by both tilings.
template <int T>
__global__ void __launch_bounds__(T) k_tile_build(
    const double* __restrict__ lon, const double* __restrict__ lat, int64_t P,
    const uint32_t* __restrict__ order, float4* __restrict__ tile_chi,
    float4* __restrict__ tile_clo, double4* __restrict__ tile_c64, float4* __restrict__ tgt_a,
    uint32_t* __restrict__ tgt_perm, float4* __restrict__ tgt_e, float4* __restrict__ tgt_n,
    double2* __restrict__ tgt_ll, double4* __restrict__ sub64, float4* __restrict__ subf,
    double4* __restrict__ grp64) {
  __shared__ double red[3][T];
  const int64_t tile = blockIdx.x;
  const int j = threadIdx.x;
  const int64_t s = tile * T + j;
  const bool valid = s < P;
  double x = 0, y = 0, z = 0, lo = 0, la = 0;
  uint32_t u = 0xffffffffu;
  if (valid) {
    u = order[s];
    lo = lon[u];
    la = lat[u];
    unit_vec(lo, la, x, y, z);
  }
  red[0][j] = x;
  red[1][j] = y;
  red[2][j] = z;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (j < o) {
      red[0][j] += red[0][j + o];
      red[1][j] += red[1][j + o];
      red[2][j] += red[2][j + o];
    }
    __syncthreads();
  }
  double cx = red[0][0], cy = red[1][0], cz = red[2][0];
  double nrm = sqrt(cx * cx + cy * cy + cz * cz);
  __syncthreads();
  if (!(nrm > 1e-9)) {  // degenerate spread: use the first member
    const uint32_t u0 = order[tile * T];
    unit_vec(lon[u0], lat[u0], cx, cy, cz);
    nrm = 1.0;
  }
  cx /= nrm;
  cy /= nrm;
  cz /= nrm;
  const double dx = x - cx, dy = y - cy, dz = z - cz;
  double ang = 0.0;
  if (valid) {
    const double ch = sqrt(dx * dx + dy * dy + dz * dz);
    ang = 2.0 * asin(fmin(1.0, 0.5 * ch));
  }
  red[0][j] = ang;
  __syncthreads();
  for (int o = T / 2; o > 0; o >>= 1) {
    if (j < o) red[0][j] = fmax(red[0][j], red[0][j + o]);
    __syncthreads();
  }
  const double radius = red[0][0] * (1.0 + 1e-9) + 1e-12;
  // an empty slot sits far outside every support radius
  tgt_a[s] = valid ? make_float4((float)dx, (float)dy, (float)dz, 0.f)
                   : make_float4(4.f, 4.f, 4.f, 0.f);
  if (tgt_perm) {
    tgt_perm[s] = valid ? u : 0xffffffffu;
    if (valid) {
      double sl, cl, sb, cb;
      sincos(lo * kDeg2Rad, &sl, &cl);
      sincos(la * kDeg2Rad, &sb, &cb);
      tgt_e[s] = make_float4((float)(-sl), (float)cl, 0.f, 0.f);
      tgt_n[s] = make_float4((float)(-sb * cl), (float)(-sb * sl), (float)cb, 0.f);
      tgt_ll[s] = make_double2(lo, la);
    } else {
      tgt_e[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      tgt_n[s] = make_float4(0.f, 0.f, 0.f, 0.f);
      tgt_ll[s] = make_double2(0.0, 0.0);
    }
  }
  if (sub64) {
    // 32-target quarters: warp-level centroid and radius (empty slots ignored)
    double sx = x, sy = y, sz = z;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      sx += __shfl_xor_sync(0xffffffffu, sx, o);
      sy += __shfl_xor_sync(0xffffffffu, sy, o);
      sz += __shfl_xor_sync(0xffffffffu, sz, o);
    }
    double qn = sqrt(sx * sx + sy * sy + sz * sz);
    if (!(qn > 1e-9)) {  // empty or degenerate quarter: use the tile centre
      sx = cx; sy = cy; sz = cz; qn = 1.0;
    }
    sx /= qn; sy /= qn; sz /= qn;
    double qa = 0.0;
    if (valid) {
      const double ex = x - sx, ey = y - sy, ez = z - sz;
      qa = 2.0 * asin(fmin(1.0, 0.5 * sqrt(ex * ex + ey * ey + ez * ez)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) qa = fmax(qa, __shfl_xor_sync(0xffffffffu, qa, o));
    qa = qa * (1.0 + 1e-9) + 1e-12;
    if ((j & 31) == 0) {
      const int64_t qi = tile * (T / 32) + (j >> 5);
      sub64[qi] = make_double4(sx, sy, sz, qa);
      subf[qi] = make_float4((float)(sx - cx), (float)(sy - cy), (float)(sz - cz),
                             (float)(2.0 * sin(0.5 * qa)));
    }
  }
  {
    // 4-target groups (lanes 4 g .. 4 g + 3): centroid of the valid members
    // and their largest angular distance from it; empty groups get radius -1
    double gx = x, gy = y, gz = z;
    int gv = valid ? 1 : 0;
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) {
      gx += __shfl_xor_sync(0xffffffffu, gx, o);
      gy += __shfl_xor_sync(0xffffffffu, gy, o);
      gz += __shfl_xor_sync(0xffffffffu, gz, o);
      gv += __shfl_xor_sync(0xffffffffu, gv, o);
    }
    double gn = sqrt(gx * gx + gy * gy + gz * gz);
    if (!(gn > 1e-9)) {  // degenerate spread: the tile centre (radius still covers)
      gx = cx; gy = cy; gz = cz; gn = 1.0;
    }
    gx /= gn; gy /= gn; gz /= gn;
    double ga = 0.0;
    if (valid) {
      const double ex = x - gx, ey = y - gy, ez = z - gz;
      ga = 2.0 * asin(fmin(1.0, 0.5 * sqrt(ex * ex + ey * ey + ez * ez)));
    }
#pragma unroll
    for (int o = 1; o < 4; o <<= 1) ga = fmax(ga, __shfl_xor_sync(0xffffffffu, ga, o));
    ga = ga * (1.0 + 1e-9) + 1e-12;
    if ((j & 3) == 0) grp64[tile * (T / 4) + (j >> 2)] = make_double4(gx, gy, gz, gv ? ga : -1.0);
  }
  if (j == 0) {
    float hx, lx, hy, ly, hz, lz;
    split_f64(cx, hx, lx);
    split_f64(cy, hy, ly);
    split_f64(cz, hz, lz);
    tile_chi[tile] = make_float4(hx, hy, hz, (float)radius);
    tile_clo[tile] = make_float4(lx, ly, lz, 0.f);
    tile_c64[tile] = make_double4(cx, cy, cz, radius);
  }
}

__global__ void k_set_axes(const float4* __restrict__ e, const float4* __restrict__ n,
                           float4* __restrict__ f1, float4* __restrict__ f2, int64_t slots,
                           float cpa, float spa) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= slots) return;
  const float4 E = e[i], N = n[i];
  // major axis at position angle PA from north through east
  f1[i] = make_float4(N.x * cpa + E.x * spa, N.y * cpa + E.y * spa, N.z * cpa + E.z * spa, 0.f);
  f2[i] = make_float4(E.x * cpa - N.x * spa, E.y * cpa - N.y * spa, E.z * cpa - N.z * spa, 0.f);
}

}  // namespace

static cudaError_t tiling_alloc(Tiling& t, int T, int64_t P, cudaStream_t s) {
  t.T = T;
  t.n_tiles = (P + T - 1) / T;
  cudaError_t e;
  if ((e = dalloc(&t.chi, (size_t)t.n_tiles, s)) != cudaSuccess) return e;
  if ((e = dalloc(&t.clo, (size_t)t.n_tiles, s)) != cudaSuccess) return e;
  if ((e = dalloc(&t.c64, (size_t)t.n_tiles, s)) != cudaSuccess) return e;
  if ((e = dalloc(&t.a, (size_t)(t.n_tiles * T), s)) != cudaSuccess) return e;
  if ((e = dalloc(&t.tile_cand, (size_t)t.n_tiles, s)) != cudaSuccess) return e;
  if ((e = dalloc(&t.grp64, (size_t)(t.n_tiles * (T / 4)), s)) != cudaSuccess) return e;
  if (T == kTile2) {
    if ((e = dalloc(&t.sub64, (size_t)(t.n_tiles * 4), s)) != cudaSuccess) return e;
    if ((e = dalloc(&t.subf, (size_t)(t.n_tiles * 4), s)) != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t targets_build(cg_grid* g, const double* lon, const double* lat) {
  cudaStream_t s = g->stream;
  const int64_t P = g->P;
  cudaError_t e;
  if ((e = tiling_alloc(g->t64, kTile, P, s)) != cudaSuccess) return e;
  if ((e = tiling_alloc(g->t128, kTile2, P, s)) != cudaSuccess) return e;
  g->n_slots = g->t128.n_tiles * kTile2;
  const int64_t slots = g->n_slots;
  if ((e = dalloc(&g->tgt_perm, slots, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->tgt_e, slots, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->tgt_n, slots, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->tgt_f1, slots, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->tgt_f2, slots, s)) != cudaSuccess) return e;
  if ((e = dalloc(&g->tgt_ll, slots, s)) != cudaSuccess) return e;

  // k-d tree levels: leaves of kTile2 targets, then five more levels that split
  // every leaf into kTile halves, 32-target quarters and on down to groups of 4
  int levels2 = 0;
  while (((int64_t)1 << levels2) < g->t128.n_tiles) ++levels2;
  const int levels = levels2 + 5;
  const int64_t max_nodes = (int64_t)1 << (levels + 1);
  float4* pos = nullptr;
  uint32_t *ord = nullptr, *nid = nullptr, *child = nullptr, *val = nullptr;
  uint32_t *nstart = nullptr, *nend = nullptr, *bmin = nullptr, *bmax = nullptr;
  uint64_t* key = nullptr;
  SortWork w;
  e = dalloc(&pos, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&ord, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&nid, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&child, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&val, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&key, (size_t)P, s);
  if (e == cudaSuccess) e = dalloc(&nstart, (size_t)max_nodes, s);
  if (e == cudaSuccess) e = dalloc(&nend, (size_t)max_nodes, s);
  if (e == cudaSuccess) e = dalloc(&bmin, (size_t)(3 * max_nodes), s);
  if (e == cudaSuccess) e = dalloc(&bmax, (size_t)(3 * max_nodes), s);
  const unsigned nb = ceil_div(P, 256);
  if (e == cudaSuccess) {
    k_target_init<<<nb, 256, 0, s>>>(lon, lat, P, pos, ord, nid, g->d_err);
    g->n_launches += 1;
  }
  for (int l = 0; l < levels && e == cudaSuccess; ++l) {
    const uint32_t leaf = (l < levels2) ? (uint32_t)kTile2 : ((uint32_t)kTile >> (l - levels2));
    const int64_t nchild = (int64_t)1 << (l + 1);
    e = cudaMemsetAsync(bmin, 0xff, sizeof(uint32_t) * (size_t)(3 * nchild), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(bmax, 0x00, sizeof(uint32_t) * (size_t)(3 * nchild), s);
    if (e != cudaSuccess) break;
    k_node_bounds<<<nb, 256, 0, s>>>(nid, P, nstart, nend);
    k_node_split<<<nb, 256, 0, s>>>(nid, ord, pos, P, leaf, nstart, nend, child, bmin, bmax);
    k_node_keys<<<nb, 256, 0, s>>>(child, ord, pos, P, bmin, bmax, key, val);
    g->n_launches += 3;
    uint64_t* sk = nullptr;
    uint32_t* sv = nullptr;
    const int bits = 32 + l + 1;
    e = radix_sort_u64(key, val, P, bits, w, s, &sk, &sv);
    g->n_launches += 3 * ((bits + 7) / 8);
    if (e != cudaSuccess) break;
    k_node_unpack<<<nb, 256, 0, s>>>(sk, P, nid);
    g->n_launches += 1;
    if (sv != ord) e = cudaMemcpyAsync(ord, sv, sizeof(uint32_t) * (size_t)P,
                                       cudaMemcpyDeviceToDevice, s);
  }
  if (e == cudaSuccess) {
    k_tile_build<kTile2><<<(unsigned)g->t128.n_tiles, kTile2, 0, s>>>(
        lon, lat, P, ord, g->t128.chi, g->t128.clo, g->t128.c64, g->t128.a, g->tgt_perm,
        g->tgt_e, g->tgt_n, g->tgt_ll, g->t128.sub64, g->t128.subf, g->t128.grp64);
    k_tile_build<kTile><<<(unsigned)g->t64.n_tiles, kTile, 0, s>>>(
        lon, lat, P, ord, g->t64.chi, g->t64.clo, g->t64.c64, g->t64.a, nullptr, nullptr,
        nullptr, nullptr, nullptr, nullptr, g->t64.grp64);
    g->n_launches += 2;
    e = cudaGetLastError();
  }
  if (w.keys_alt) cudaFreeAsync(w.keys_alt, s);
  dfree(w.vals_alt, s);
  dfree(w.hist, s);
  dfree(w.totals, s);
  dfree(pos, s);
  dfree(ord, s);
  dfree(nid, s);
  dfree(child, s);
  dfree(val, s);
  dfree(key, s);
  dfree(nstart, s);
  dfree(nend, s);
  dfree(bmin, s);
  dfree(bmax, s);
  return e;
}

cudaError_t targets_set_axes(cg_grid* g, double pa_deg) {
  const int64_t slots = g->n_slots;
  const double pa = pa_deg * kDeg2Rad;
  k_set_axes<<<ceil_div(slots, 256), 256, 0, g->stream>>>(g->tgt_e, g->tgt_n, g->tgt_f1,
                                                          g->tgt_f2, slots, (float)cos(pa),
                                                          (float)sin(pa));
  return cudaGetLastError();
}

}  // namespace cg
