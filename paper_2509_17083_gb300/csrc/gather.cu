// Hash-grid gather (Eq. 3) and its reverse for the BF16 tensor-core path.
//
// The decoders run on the tensor cores over tiles of 128 rows, a shape that
// needs most of an SM's shared memory and therefore runs only a few warps per
// SM. The hash gathers and the gradient scatter are latency-bound memory work
// that wants the opposite: as many independent loads and atomics in flight as
// possible. So they run here, in their own kernels, with one thread per
// (row, level) pair: a CTA holds 32 rows (the lanes) x 16 levels (the warps),
// 512 threads, 4 CTAs per SM.
//
//   k_gather   rows -> bf16 features X [rows][32] per field (row-major; the
//              decoder kernels stage them into their operand tiles)
//   k_scatter  f32 feature gradients dX [rows][32] per field -> float2
//              atomics into the f32 table gradients, and, for Gaussians,
//              dL/dp through the trilinear weights and the contraction
//              Jacobian (App. A.1, Eq. 2)
//
// A row is a visible Gaussian (position via vis_ids) or a pixel (the hit of
// its ray with the background sphere, App. A.2). A lane works on one row at a
// fixed level, so when neighbouring rows are neighbours in space (pixels of
// an image row; Gaussians stored in Morton order), runs of lanes hit the
// same corner at all but the finest levels; the scatter sums each run with
// shuffles and issues one atomic per run.
#include "tc_ops.cuh"

namespace hyrf {

namespace {

constexpr int kRows = 32;    // rows per CTA (lanes)
constexpr int kLevels = 16;  // levels (warps)
constexpr int kThreads = kRows * kLevels;

__device__ __forceinline__ int row_count(const RowSource& S, const CamDev& cam) {
  const int all = S.pixels ? cam.W * cam.H : min(*S.n_vis, S.n);
  return S.list ? min(*S.n_list, all) : all;
}

// Contracted position (and, for Gaussians, the Gaussian index and the
// contraction Jacobian) of row `row`; rows past the end, or with an
// out-of-range id, get a harmless in-box point and ok = false.
__device__ __forceinline__ void row_point(const RowSource& S, const FieldsDev& F, const CamDev& cam,
                                          int row, int nrows, float y[3], float* J, int& g, bool& ok) {
  ok = row < nrows;
  g = 0;
  if (S.pixels) {
    const int p = ok ? (S.list ? S.list[row] : row) : 0;
    float ps[3], dir[3];
    tc::bg_ray(cam, F, S.radius, p % cam.W, p / cam.W, ps, dir);
    contract_n(ps, y);
    return;
  }
  if (ok) {
    const int v = S.list ? S.list[row] : row;
    g = (v >= 0 && v < S.n) ? S.vis_ids[v] : -1;
    if (g < 0 || g >= S.n) {
      set_status(S.status, HYRF_ERR_BOUNDS);
      ok = false;
      g = 0;
    }
  }
  float p[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) p[k] = ok ? S.pos[3 * (int64_t)g + k] : F.lo[k] + 1.0f / F.sx[k];
  contract_p(F, p, y, J);
}

// Eq. 3 at one level: the two interpolated features, summed over the corners
// in the same order as the fused field kernels.
template <int DT>
__device__ __forceinline__ float2 level_feature(const GridDev& G, int l, const float y[3]) {
  uint32_t idx[8];
  float f[3];
  level_cell(G, l, y, idx, f);
  float2 e[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) e[c] = load_entry_t<DT>(G, (size_t)l * G.T + idx[c]);
  float a0 = 0.0f, a1 = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = corner_w(f, c);
    a0 = fmaf(w, e[c].x, a0);
    a1 = fmaf(w, e[c].y, a1);
  }
  return make_float2(a0, a1);
}

// Eq. 3 at one level in two grids with the same cell arithmetic (same
// levels, resolutions, table size and dense levels): each corner's index
// and weight serve both tables. Same sums, in the same order, as two calls
// of level_feature.
template <int DT>
__device__ __forceinline__ void level_feature2(const GridDev& A, const GridDev& B, int l, const float y[3],
                                               float2& fa, float2& fb) {
  uint32_t idx[8];
  float f[3];
  level_cell(A, l, y, idx, f);
  float2 ea[8], eb[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const size_t e = (size_t)l * A.T + idx[c];
    ea[c] = load_entry_t<DT>(A, e);
    eb[c] = load_entry_t<DT>(B, e);
  }
  float a0 = 0.0f, a1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float w = corner_w(f, c);
    a0 = fmaf(w, ea[c].x, a0);
    a1 = fmaf(w, ea[c].y, a1);
    b0 = fmaf(w, eb[c].x, b0);
    b1 = fmaf(w, eb[c].y, b1);
  }
  fa = make_float2(a0, a1);
  fb = make_float2(b0, b1);
}

// Lanes that start a run of consecutive lanes in the same grid cell (cell
// from level_cell): lanes hold neighbouring points (pixels of an image row;
// Gaussians in Morton order), so lanes sharing a cell form runs, and every
// corner of the cell has the same runs. Found once per level.
__device__ __forceinline__ unsigned cell_heads(uint64_t cell) {
  const int lane = threadIdx.x & 31;
  const uint64_t prev = __shfl_up_sync(0xffffffffu, cell, 1);
  return __ballot_sync(0xffffffffu, lane == 0 || prev != cell);
}

// Length of the longest run of the heads (warp-uniform): a segmented scan
// over runs no longer than this needs only its offsets below it; the later
// steps would add nothing to any lane.
__device__ __forceinline__ int longest_run(unsigned heads) {
  const int lane = threadIdx.x & 31;
  const unsigned above = heads & ~(0xffffffffu >> (31 - lane));  // heads after this lane
  const int len = ((heads >> lane) & 1u) ? (above ? __ffs(above) - 1 : 32) - lane : 0;
  return (int)__reduce_max_sync(0xffffffffu, (unsigned)len);
}

// Sums over the 32 lanes of eight float2 values by recursive halving (a
// lane keeps half of its partial sums and adds its partner's copy of that
// half): the lanes with (lane & 3) == 0 return the sum of value
// ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1).
// Used when the whole warp is one run (every lane in one cell).
__device__ __forceinline__ float2 warp_sum8x2(float2* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int h = 4, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float2 send = up ? v[j] : v[j + h];
      const float2 keep = up ? v[j + h] : v[j];
      v[j] = make_float2(keep.x + __shfl_xor_sync(0xffffffffu, send.x, o),
                         keep.y + __shfl_xor_sync(0xffffffffu, send.y, o));
    }
  }
  float2 s = v[0];
#pragma unroll
  for (int o = 2; o >= 1; o >>= 1)
    s = make_float2(s.x + __shfl_xor_sync(0xffffffffu, s.x, o), s.y + __shfl_xor_sync(0xffffffffu, s.y, o));
  return s;
}

// Corner whose sum warp_sum8x2 leaves in this lane, and its table index.
__device__ __forceinline__ uint32_t lane_corner_index(const uint32_t idx[8]) {
  const int lane = threadIdx.x & 31;
  const int c8 = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
  uint32_t ic = idx[0];
#pragma unroll
  for (int c = 1; c < 8; ++c) ic = c == c8 ? idx[c] : ic;
  return ic;
}

// One float2 atomic per run (heads from cell_heads, span = longest_run) of
// lanes that target the same table entry e: each run's contributions are
// summed by a segmented shuffle scan and its last lane issues the atomic.
// Warp-uniform fast paths: no run longer than one lane, or one run over the
// whole warp.
__device__ __forceinline__ void run_atomic(float* __restrict__ gtab, size_t e, unsigned heads, int span, float g0,
                                           float g1) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  if (heads == full) {
    if (g0 != 0.0f || g1 != 0.0f) atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
    return;
  }
  if (heads == 1u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      g0 += __shfl_xor_sync(full, g0, o);
      g1 += __shfl_xor_sync(full, g1, o);
    }
    if (lane == 0 && (g0 != 0.0f || g1 != 0.0f))
      atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
    return;
  }
  const int start = 31 - __clz(heads & (full >> (31 - lane)));  // first lane of this run
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    if (o >= span) break;  // warp-uniform
    const float a0 = __shfl_up_sync(full, g0, o), a1 = __shfl_up_sync(full, g1, o);
    if (lane - o >= start) {
      g0 += a0;
      g1 += a1;
    }
  }
  const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
  if (tail && (g0 != 0.0f || g1 != 0.0f)) atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
}

// Reverse of level_feature: (d0, d1) = dL/d features of level l. Adds
// w_c (d0, d1) to the table gradient of every corner and returns the level's
// dL/dy if WANT_DY. COHERENT: lanes hold neighbouring points (run_atomic).
template <bool COHERENT, bool WANT_DY, int DT>
__device__ __forceinline__ void level_scatter(const GridDev& G, int l, const float y[3], float d0, float d1,
                                              float* __restrict__ gtab, float dy[3]) {
  if (WANT_DY) dy[0] = dy[1] = dy[2] = 0.0f;
  // A zero feature gradient adds nothing to the table and nothing to dL/dy
  // (every term carries d0 or d1): skip the level; in COHERENT mode, whose
  // lanes must all reach the shuffles, only when the whole warp may.
  const bool zero = d0 == 0.0f && d1 == 0.0f;
  if (COHERENT ? __all_sync(0xffffffffu, zero) : zero) return;
  uint32_t idx[8];
  float f[3];
  uint64_t cell;
  level_cell(G, l, y, idx, f, &cell);
  const unsigned heads = COHERENT ? cell_heads(cell) : 0u;
  const bool one_run = COHERENT && heads == 1u;  // the whole warp in one cell (warp-uniform)
  const int span = COHERENT ? longest_run(heads) : 1;
  if (one_run) {  // the eight corners' sums at once, one atomic per corner
    float2 v[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = corner_w(f, c);
      v[c] = make_float2(w * d0, w * d1);
    }
    const float2 sm = warp_sum8x2(v);
    if ((threadIdx.x & 3) == 0 && (sm.x != 0.0f || sm.y != 0.0f))
      atomicAdd(reinterpret_cast<float2*>(gtab) + (size_t)l * G.T + lane_corner_index(idx), sm);
  }
  float g[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const size_t e = (size_t)l * G.T + idx[c];
    const float w = corner_w(f, c);
    const float g0 = w * d0, g1 = w * d1;
    if (COHERENT) {
      if (!one_run) run_atomic(gtab, e, heads, span, g0, g1);
    } else if (g0 != 0.0f || g1 != 0.0f) {
      atomicAdd(reinterpret_cast<float2*>(gtab) + e, make_float2(g0, g1));
    }
    if (WANT_DY && !zero) {
      const float2 v = load_entry_t<DT>(G, e);
      const float dot = v.x * d0 + v.y * d1;
      const float wx = (c & 1) ? f[0] : 1.0f - f[0];
      const float wy = (c & 2) ? f[1] : 1.0f - f[1];
      const float wz = (c & 4) ? f[2] : 1.0f - f[2];
      g[0] += dot * ((c & 1) ? 1.0f : -1.0f) * wy * wz;
      g[1] += dot * ((c & 2) ? 1.0f : -1.0f) * wx * wz;
      g[2] += dot * ((c & 4) ? 1.0f : -1.0f) * wx * wy;
    }
  }
  if (WANT_DY) {
    const float N = (float)G.res[l];
    dy[0] = g[0] * N;
    dy[1] = g[1] * N;
    dy[2] = g[2] * N;
  }
}

// run_atomic for the same entry e of two tables (ga, gb) at once: the four
// sums scanned together.
__device__ __forceinline__ void run_atomic2(float* __restrict__ ga, float* __restrict__ gb, size_t e, unsigned heads,
                                            int span, float a0, float a1, float b0, float b1) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  bool issue = true;
  if (heads == 1u) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a0 += __shfl_xor_sync(full, a0, o);
      a1 += __shfl_xor_sync(full, a1, o);
      b0 += __shfl_xor_sync(full, b0, o);
      b1 += __shfl_xor_sync(full, b1, o);
    }
    issue = lane == 0;
  } else if (heads != full) {
    const int start = 31 - __clz(heads & (full >> (31 - lane)));
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (o >= span) break;  // warp-uniform
      const float x0 = __shfl_up_sync(full, a0, o), x1 = __shfl_up_sync(full, a1, o);
      const float z0 = __shfl_up_sync(full, b0, o), z1 = __shfl_up_sync(full, b1, o);
      if (lane - o >= start) {
        a0 += x0;
        a1 += x1;
        b0 += z0;
        b1 += z1;
      }
    }
    issue = lane == 31 || ((heads >> (lane + 1)) & 1u);
  }
  if (!issue) return;
  if (a0 != 0.0f || a1 != 0.0f) atomicAdd(reinterpret_cast<float2*>(ga) + e, make_float2(a0, a1));
  if (b0 != 0.0f || b1 != 0.0f) atomicAdd(reinterpret_cast<float2*>(gb) + e, make_float2(b0, b1));
}

// level_scatter of two grids with the same cell arithmetic (Gaussians,
// coherent lanes): (a0, a1) and (b0, b1) are the feature gradients of grid
// A and B; dy receives the sum of both grids' dL/dy.
template <int DT>
__device__ __forceinline__ void level_scatter2(const GridDev& A, const GridDev& B, int l, const float y[3],
                                               float2 da, float2 db, float* __restrict__ ga,
                                               float* __restrict__ gb, float dy[3]) {
  dy[0] = dy[1] = dy[2] = 0.0f;
  const bool zero = da.x == 0.0f && da.y == 0.0f && db.x == 0.0f && db.y == 0.0f;
  if (__all_sync(0xffffffffu, zero)) return;
  uint32_t idx[8];
  float f[3];
  uint64_t cell;
  level_cell(A, l, y, idx, f, &cell);
  const unsigned heads = cell_heads(cell);
  const bool one_run = heads == 1u;  // the whole warp in one cell (warp-uniform)
  const int span = longest_run(heads);
  float g[3] = {0.0f, 0.0f, 0.0f};
  // dL/dy first: the corner values of both tables are loaded together (one
  // round trip), not each behind the previous corner's atomics
  if (!zero) {
    float dot[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t e = (size_t)l * A.T + idx[c];
      const float2 va = load_entry_t<DT>(A, e), vb = load_entry_t<DT>(B, e);
      dot[c] = va.x * da.x + va.y * da.y + (vb.x * db.x + vb.y * db.y);
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float wx = (c & 1) ? f[0] : 1.0f - f[0];
      const float wy = (c & 2) ? f[1] : 1.0f - f[1];
      const float wz = (c & 4) ? f[2] : 1.0f - f[2];
      g[0] += dot[c] * ((c & 1) ? 1.0f : -1.0f) * wy * wz;
      g[1] += dot[c] * ((c & 2) ? 1.0f : -1.0f) * wx * wz;
      g[2] += dot[c] * ((c & 4) ? 1.0f : -1.0f) * wx * wy;
    }
  }
  if (one_run) {  // the eight corners' sums at once, one atomic per corner and table
    float2 va[8], vb[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = corner_w(f, c);
      va[c] = make_float2(w * da.x, w * da.y);
      vb[c] = make_float2(w * db.x, w * db.y);
    }
    const float2 sa = warp_sum8x2(va), sb = warp_sum8x2(vb);
    if ((threadIdx.x & 3) == 0) {
      const size_t e = (size_t)l * A.T + lane_corner_index(idx);
      if (sa.x != 0.0f || sa.y != 0.0f) atomicAdd(reinterpret_cast<float2*>(ga) + e, sa);
      if (sb.x != 0.0f || sb.y != 0.0f) atomicAdd(reinterpret_cast<float2*>(gb) + e, sb);
    }
  } else {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float w = corner_w(f, c);
      run_atomic2(ga, gb, (size_t)l * A.T + idx[c], heads, span, w * da.x, w * da.y, w * db.x, w * db.y);
    }
  }
  const float N = (float)A.res[l];
  dy[0] = g[0] * N;
  dy[1] = g[1] * N;
  dy[2] = g[2] * N;
}

// Features of both fields (Gaussians) or of the radiance field only (pixels).
// X*: [rows][16] uint32 = [rows][32] bf16 (f16 when H16: the decoders'
// operand type), level-major (2l, 2l+1).
// SAME: both grids have the same cell arithmetic (level_feature2).
template <bool BOTH, int DT, bool H16, bool SAME>
__global__ void __launch_bounds__(kThreads, 4)
    k_gather(FieldsDev F, CamDev cam, RowSource S, uint32_t* __restrict__ Xg, uint32_t* __restrict__ Xr) {
  __shared__ float ys[kRows][3];
  __shared__ uint32_t xs[2][kRows][kLevels + 1];
  const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int nrows = row_count(S, cam);
  const int row0 = blockIdx.x * kRows;
  if (row0 >= nrows) return;  // CTA-uniform
  if (l == 0) {
    float y[3];
    int g;
    bool ok;
    row_point(S, F, cam, row0 + lane, nrows, y, nullptr, g, ok);
#pragma unroll
    for (int k = 0; k < 3; ++k) ys[lane][k] = y[k];
  }
  __syncthreads();
  const float y[3] = {ys[lane][0], ys[lane][1], ys[lane][2]};
  if (BOTH && SAME) {
    float2 a, b;
    level_feature2<DT>(F.geo, F.rad, l, y, a, b);
    xs[0][lane][l] = tc::pack2<H16>(a.x, a.y);
    xs[1][lane][l] = tc::pack2<H16>(b.x, b.y);
  } else {
    if (BOTH) {
      const float2 a = level_feature<DT>(F.geo, l, y);
      xs[0][lane][l] = tc::pack2<H16>(a.x, a.y);
    }
    const float2 b = level_feature<DT>(F.rad, l, y);
    xs[1][lane][l] = tc::pack2<H16>(b.x, b.y);
  }
  __syncthreads();
  // coalesced write-out: thread t -> row t/16, word t%16
  const int r = threadIdx.x >> 4, wd = threadIdx.x & 15;
  if (row0 + r < nrows) {
    const size_t o = (size_t)(row0 + r) * 16 + wd;
    if (BOTH) __stcs(Xg + o, xs[0][r][wd]);
    __stcs(Xr + o, xs[1][r][wd]);
  }
}

// FP32 path: the same gather from f32 tables with f32 features out, X*:
// [rows][32] float (level-major, features 2l and 2l + 1), for the decoders
// on the CUDA cores.
template <bool BOTH, bool SAME>
__global__ void __launch_bounds__(kThreads, 4)
    k_gather_f32(FieldsDev F, CamDev cam, RowSource S, float2* __restrict__ Xg, float2* __restrict__ Xr) {
  __shared__ float ys[kRows][3];
  __shared__ float2 xs[2][kRows][kLevels + 1];
  const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int nrows = row_count(S, cam);
  const int row0 = blockIdx.x * kRows;
  if (row0 >= nrows) return;  // CTA-uniform
  if (l == 0) {
    float y[3];
    int g;
    bool ok;
    row_point(S, F, cam, row0 + lane, nrows, y, nullptr, g, ok);
#pragma unroll
    for (int k = 0; k < 3; ++k) ys[lane][k] = y[k];
  }
  __syncthreads();
  const float y[3] = {ys[lane][0], ys[lane][1], ys[lane][2]};
  if (BOTH && SAME) {
    float2 a, b;
    level_feature2<0>(F.geo, F.rad, l, y, a, b);
    xs[0][lane][l] = a;
    xs[1][lane][l] = b;
  } else {
    if (BOTH) xs[0][lane][l] = level_feature<0>(F.geo, l, y);
    xs[1][lane][l] = level_feature<0>(F.rad, l, y);
  }
  __syncthreads();
  // coalesced write-out: thread t -> row t/16, level t%16
  const int r = threadIdx.x >> 4, wd = threadIdx.x & 15;
  if (row0 + r < nrows) {
    const size_t o = (size_t)(row0 + r) * 16 + wd;
    if (BOTH) __stcs(Xg + o, xs[0][r][wd]);
    __stcs(Xr + o, xs[1][r][wd]);
  }
}

// Reverse of k_gather. dXg/dXr: [rows][32] f32 feature gradients (already
// unscaled; streamed with evict-first loads). Gaussians: both fields, and
// d_pos[g] += J^T sum_l dL/dy_l; pixels: the radiance field. SAME: both
// grids have the same cell arithmetic (level_scatter2).
template <bool GAUSS, int DT, bool SAME>
__global__ void __launch_bounds__(kThreads, 4)
    k_scatter(FieldsDev F, CamDev cam, RowSource S, const float* __restrict__ dXg,
              const float* __restrict__ dXr, float* __restrict__ g_geo, float* __restrict__ g_rad,
              float* __restrict__ d_pos) {
  __shared__ float ys[kRows][3];
  __shared__ float Js[kRows][9];
  __shared__ int gs[kRows];
  __shared__ float dys[kLevels][kRows][3];
  const int lane = threadIdx.x & 31, l = threadIdx.x >> 5;
  const int nrows = row_count(S, cam);
  const int row0 = blockIdx.x * kRows;
  if (row0 >= nrows) return;  // CTA-uniform
  const int row = row0 + lane;
  // this thread's feature gradients, loaded while warp 0 finds the rows'
  // points (kept only for rows found valid)
  const size_t o = (size_t)(row < nrows ? row : row0) * 32 + 2 * l;
  const float2 zero = make_float2(0.0f, 0.0f);
  float2 dg0 = zero, dr0 = zero;
  if (row < nrows) {
    if (GAUSS) dg0 = __ldcs(reinterpret_cast<const float2*>(dXg + o));
    dr0 = __ldcs(reinterpret_cast<const float2*>(dXr + o));
  }
  if (l == 0) {
    float y[3], J[9];
    int g;
    bool ok;
    row_point(S, F, cam, row, nrows, y, GAUSS ? J : nullptr, g, ok);
#pragma unroll
    for (int k = 0; k < 3; ++k) ys[lane][k] = y[k];
    if (GAUSS) {
#pragma unroll
      for (int k = 0; k < 9; ++k) Js[lane][k] = J[k];
    }
    gs[lane] = ok ? g : -1;
  }
  __syncthreads();
  const bool ok = gs[lane] >= 0;
  const float y[3] = {ys[lane][0], ys[lane][1], ys[lane][2]};
  if (GAUSS) {
    const float2 dg = ok ? dg0 : zero;
    const float2 dr = ok ? dr0 : zero;
    float dy[3], dy2[3];
    if (SAME) {
      level_scatter2<DT>(F.geo, F.rad, l, y, dg, dr, g_geo, g_rad, dy);
      dy2[0] = dy2[1] = dy2[2] = 0.0f;
    } else {
      level_scatter<true, true, DT>(F.geo, l, y, dg.x, dg.y, g_geo, dy);
      level_scatter<true, true, DT>(F.rad, l, y, dr.x, dr.y, g_rad, dy2);
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) dys[l][lane][k] = dy[k] + dy2[k];
    __syncthreads();
    if (l == 0 && ok) {
      float s[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
      for (int m = 0; m < kLevels; ++m) {
#pragma unroll
        for (int k = 0; k < 3; ++k) s[k] += dys[m][lane][k];
      }
      const float* J = Js[lane];
      const int g = gs[lane];
#pragma unroll
      for (int j = 0; j < 3; ++j) atomicAdd(d_pos + 3 * (int64_t)g + j, J[j] * s[0] + J[3 + j] * s[1] + J[6 + j] * s[2]);
    }
  } else {
    const float2 dr = ok ? dr0 : zero;
    float dy[3];
    level_scatter<true, false, DT>(F.rad, l, y, dr.x, dr.y, g_rad, dy);
  }
}

int grid_for(int rows) { return rows > 0 ? (rows + kRows - 1) / kRows : 0; }

}  // namespace

// rows: an upper bound of the device row count (n for Gaussians, W*H for
// pixels). Gaussians gather and scatter both fields, pixels the radiance
// field only.
// Both grids index their tables identically at every level.
static bool same_cells(const GridDev& a, const GridDev& b) {
  if (a.L != b.L || a.T != b.T || a.dense != b.dense) return false;
  for (int l = 0; l < a.L; ++l)
    if (a.res[l] != b.res[l]) return false;
  return true;
}

template <int DT, bool H16>
static hyrf_status gather_dt(const FieldsDev& F, const CamDev& cam, const RowSource& S, int grid, uint32_t* Xg,
                             uint32_t* Xr, cudaStream_t s) {
  if (S.pixels)
    HYRF_LAUNCH("k_gather<pixels>", s,
                k_gather<false, DT, H16, false><<<grid, kThreads, 0, s>>>(F, cam, S, nullptr, Xr));
  else if (same_cells(F.geo, F.rad))
    HYRF_LAUNCH("k_gather<gaussians>", s,
                k_gather<true, DT, H16, true><<<grid, kThreads, 0, s>>>(F, cam, S, Xg, Xr));
  else
    HYRF_LAUNCH("k_gather<gaussians>", s,
                k_gather<true, DT, H16, false><<<grid, kThreads, 0, s>>>(F, cam, S, Xg, Xr));
  return HYRF_OK;
}

template <int DT>
static hyrf_status scatter_dt(const FieldsDev& F, const CamDev& cam, const RowSource& S, int grid,
                              const float* dXg, const float* dXr, float* g_geo, float* g_rad, float* d_pos,
                              cudaStream_t s) {
  if (S.pixels)
    HYRF_LAUNCH("k_scatter<pixels>", s,
                k_scatter<false, DT, false><<<grid, kThreads, 0, s>>>(F, cam, S, nullptr, dXr, nullptr, g_rad, nullptr));
  else if (same_cells(F.geo, F.rad))
    HYRF_LAUNCH("k_scatter<gaussians>", s,
                k_scatter<true, DT, true><<<grid, kThreads, 0, s>>>(F, cam, S, dXg, dXr, g_geo, g_rad, d_pos));
  else
    HYRF_LAUNCH("k_scatter<gaussians>", s,
                k_scatter<true, DT, false><<<grid, kThreads, 0, s>>>(F, cam, S, dXg, dXr, g_geo, g_rad, d_pos));
  return HYRF_OK;
}

// rows: an upper bound of the device row count (n for Gaussians, W*H for
// pixels). Gaussians gather and scatter both fields, pixels the radiance
// field only. The table type (both grids alike) picks the instantiation.
hyrf_status launch_gather(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows, uint32_t* Xg,
                          uint32_t* Xr, cudaStream_t s) {
  const int grid = grid_for(rows);
  if (grid == 0) return HYRF_OK;
  if (F.cm.f16) {  // the real-time f16 path: f16 or 8-bit grids
    if (F.rad.u8) return gather_dt<2, true>(F, cam, S, grid, Xg, Xr, s);
    if (F.rad.f16) return gather_dt<3, true>(F, cam, S, grid, Xg, Xr, s);
    return HYRF_ERR_UNSUPPORTED;
  }
  if (F.rad.u8) return gather_dt<2, false>(F, cam, S, grid, Xg, Xr, s);
  if (F.rad.bf16) return gather_dt<1, false>(F, cam, S, grid, Xg, Xr, s);
  if (F.rad.f16) return HYRF_ERR_UNSUPPORTED;
  return gather_dt<0, false>(F, cam, S, grid, Xg, Xr, s);
}

// f32 tables, f32 features (the FP32 path's split field query).
hyrf_status launch_gather_f32(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows, float* Xg,
                              float* Xr, cudaStream_t s) {
  const int grid = grid_for(rows);
  if (grid == 0) return HYRF_OK;
  if (F.rad.u8 || F.rad.bf16 || F.rad.f16 || F.rad.L != kLevels) return HYRF_ERR_UNSUPPORTED;
  float2* g2 = reinterpret_cast<float2*>(Xg);
  float2* r2 = reinterpret_cast<float2*>(Xr);
  if (S.pixels)
    HYRF_LAUNCH("k_gather_f32<pixels>", s, k_gather_f32<false, false><<<grid, kThreads, 0, s>>>(F, cam, S, nullptr, r2));
  else if (same_cells(F.geo, F.rad))
    HYRF_LAUNCH("k_gather_f32<gaussians>", s, k_gather_f32<true, true><<<grid, kThreads, 0, s>>>(F, cam, S, g2, r2));
  else
    HYRF_LAUNCH("k_gather_f32<gaussians>", s, k_gather_f32<true, false><<<grid, kThreads, 0, s>>>(F, cam, S, g2, r2));
  return HYRF_OK;
}

hyrf_status launch_scatter(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows,
                           const float* dXg, const float* dXr, float* g_geo, float* g_rad, float* d_pos,
                           cudaStream_t s) {
  const int grid = grid_for(rows);
  if (grid == 0) return HYRF_OK;
  if (F.rad.u8 || F.rad.f16 || F.cm.f16) return HYRF_ERR_UNSUPPORTED;  // render-only types
  if (F.rad.bf16) return scatter_dt<1>(F, cam, S, grid, dXg, dXr, g_geo, g_rad, d_pos, s);
  return scatter_dt<0>(F, cam, S, grid, dXg, dXr, g_geo, g_rad, d_pos, s);
}

}  // namespace hyrf
