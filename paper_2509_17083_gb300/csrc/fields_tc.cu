// BF16 field query and background forward with the decoders (Eqs. 4, 6) on
// the 5th-generation tensor cores. A CTA owns a tile of 128 points (the MMA
// M dimension): every thread copies one point's bf16 hash features (Eq. 3,
// gathered by k_gather in gather.cu) and, for the colour decoder, its
// positional encoding into its row of the A operand in shared memory; one
// thread issues tcgen05.mma (kind::f16, bf16 x bf16 -> f32) per
// layer with the weights staged once per CTA as the B operand; the f32
// accumulators live in tensor memory and come back with tcgen05.ld for the
// bias + ReLU epilogue, which writes the next layer's bf16 A operand. The
// field query runs three CTAs per SM (inputs share the hidden activations'
// buffers, 128 tensor-memory columns each), its geometry and colour
// decoders as two independent 128-thread groups (own MMA issuer, mbarrier
// and named barrier), and fetches the next tile's rows into registers
// while the current tile's MMA chain runs.
//
// Shared-memory operands use the no-swizzle K-major core-matrix layout: an
// 8-row x 16-byte core matrix is 128 contiguous bytes; core matrices
// adjacent along K are 128 bytes apart (leading byte offset) and 8-row
// groups are K/8 * 128 bytes apart (stride byte offset).
//
// Every wait on an mbarrier is bounded; on expiry the kernel records
// HYRF_ERR_TIMEOUT in the status word, waits (bounded) for its MMAs, frees
// its tensor memory and returns.
#include "tc_ops.cuh"

namespace hyrf {
namespace tc {

// ---------------------------------------------------------------- field query

struct QueryIO {
  int n;
  const float* pos;
  const float* alpha_e;
  const float* scale_e;
  const float* color_e;
  const int32_t* vis_ids;
  const int32_t* n_vis;
  const uint32_t* Xg;   // [n_vis][32] bf16 geometry features (k_gather)
  const uint32_t* Xr;   // [n_vis][32] bf16 radiance features
  float* alpha;
  float* scale;
  float* quat;
  float* color;
  int32_t* status;
};

// smem byte offsets. A tile's inputs (A operands) share the buffers of its
// hidden activations: layer 0's MMA has finished reading them when the
// epilogue overwrites them.
constexpr int oW0g = 0, oW1g = oW0g + 64 * 32 * 2, oW2g = oW1g + 64 * 64 * 2, oW0c = oW2g + 16 * 64 * 2,
              oW1c = oW0c + 64 * 64 * 2, oW2c = oW1c + 64 * 64 * 2, oHg = oW2c + 16 * 64 * 2,
              oHc = oHg + 128 * 64 * 2, oAg = oHg, oAc = oHc, oBias = oHc + 128 * 64 * 2,
              kQuerySmem = oBias + 288 * 4;
// tensor memory: geometry accumulators in columns [0, 64), colour in
// [64, 128); the output layers reuse [0, 16) and [64, 80)
constexpr uint32_t kQueryTmemCols = 128;

// One point's inputs, fetched a tile ahead into registers so that their
// global loads overlap the previous tile's MMA chain: its features (by row
// index), position and explicit parameters (by its Gaussian id, itself
// read one tile earlier still), so no load waits on another. Nothing
// branches on a loaded value until the next tile uses it.
struct QueryRow {
  uint4 x[4];  // 32 bf16 hash features of this thread's field
  float p[3];  // position
  float e[3];  // explicit parameters: alpha_e, scale_e (geometry) or colour_e (colour)
  int i, g;
  bool ok;
};

__device__ __forceinline__ void fetch_row(const QueryIO& io, bool geo, int i, int g, bool ok, QueryRow& q) {
  q.i = i;
  q.g = g;
  q.ok = ok;
  const int ii = ok ? i : 0, gg = ok ? g : 0;  // (row 0 and Gaussian 0 exist whenever a tile runs)
  const uint4* s4 = reinterpret_cast<const uint4*>((geo ? io.Xg : io.Xr) + (size_t)ii * 16);
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) q.x[kc] = __ldg(s4 + kc);
#pragma unroll
  for (int k = 0; k < 3; ++k) q.p[k] = io.pos[3 * (int64_t)gg + k];
  if (geo) {
    q.e[0] = io.alpha_e ? io.alpha_e[gg] : 0.0f;
    q.e[1] = io.scale_e ? io.scale_e[gg] : 0.0f;
    q.e[2] = 0.0f;
  } else {
#pragma unroll
    for (int k = 0; k < 3; ++k) q.e[k] = io.color_e ? io.color_e[3 * (int64_t)gg + k] : 0.0f;
  }
}

// Visible row i of a tile (or none) and its Gaussian id g, read earlier:
// whether the row is processed; an id out of range is reported.
__device__ __forceinline__ bool row_ok(const QueryIO& io, int i, int nv, int g) {
  if (i >= nv) return false;
  if (g < 0 || g >= io.n) {
    set_status(io.status, HYRF_ERR_BOUNDS);
    return false;
  }
  return true;
}

template <bool H16>
__global__ void __launch_bounds__(256, 3) k_query_fwd_tc(FieldsDev F, CamDev cam, QueryIO io) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bars[2];  // one per decoder group
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, w = t >> 5, r = t & 127;
  const bool geo = t < 128;
  // the two decoders run as independent 128-thread groups: own MMA issuer,
  // barrier and named barrier (1, 2), so neither waits for the other's phases
  uint64_t* bar = &bars[geo ? 0 : 1];
  float* bias = reinterpret_cast<float*>(sm + oBias);
  float *b0g = bias, *b1g = bias + 64, *b2g = bias + 128, *b0c = bias + 144, *b1c = bias + 208,
        *b2c = bias + 272;
  stage_w<64, 32>(sm + oW0g, F.gm.W[0], 64);
  stage_w<64, 64>(sm + oW1g, F.gm.W[1], 64);
  stage_w<16, 64>(sm + oW2g, F.gm.W[2], 8);
  stage_w<64, 64>(sm + oW0c, F.cm.W[0], 64);
  stage_w<64, 64>(sm + oW1c, F.cm.W[1], 64);
  stage_w<16, 64>(sm + oW2c, F.cm.W[2], 3);
  if (t < 64) {
    b0g[t] = F.gm.b[0][t];
    b1g[t] = F.gm.b[1][t];
    b0c[t] = F.cm.b[0][t];
    b1c[t] = F.cm.b[1][t];
  }
  if (t < 16) {
    b2g[t] = t < 8 ? F.gm.b[2][t] : 0.0f;
    b2c[t] = t < 3 ? F.cm.b[2][t] : 0.0f;
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bars[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bars[1])));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kQueryTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_smem_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tm = tmem_base;
  const uint32_t lane = ((uint32_t)((w & 3) * 32)) << 16;
  const uint32_t colD = geo ? 0u : 64u;
  uint8_t* Hs = sm + (geo ? oHg : oHc);
  const float* b0 = geo ? b0g : b0c;
  const float* b1 = geo ? b1g : b1c;
  const float* b2 = geo ? b2g : b2c;
  float pc[3];
  cam_center(cam, pc);
  const int nv = min(*io.n_vis, io.n);
  const int ntile = (nv + 127) / 128;
  uint32_t phase = 0;
  bool failed = false;
  const int G = gridDim.x;
  QueryRow cur;
  int gn = 0;  // Gaussian id of this thread's row of the next tile (read a tile ahead)
  if ((int)blockIdx.x < ntile) {
    const int i0 = blockIdx.x * 128 + r, i1 = (blockIdx.x + G) * 128 + r;
    const int g0 = i0 < nv ? io.vis_ids[i0] : 0;
    fetch_row(io, geo, i0, g0, row_ok(io, i0, nv, g0), cur);
    if ((int)blockIdx.x + G < ntile && i1 < nv) gn = io.vis_ids[i1];
  }
  for (int tile = blockIdx.x; tile < ntile && !failed; tile += G) {
    // this tile's rows -> A operands (the previous tile's last MMA, the
    // only reader of these buffers, has completed): the features, and
    // half of the colour input's positional encoding from each of the
    // row's two threads
#pragma unroll
    for (int kc = 0; kc < 4; ++kc)
      *reinterpret_cast<uint4*>(sm + (geo ? oAg : oAc) + kmaj(r, 8 * kc, geo ? 32 : 64)) = cur.x[kc];
    if (!geo) {
      float p[3];
#pragma unroll
      for (int k = 0; k < 3; ++k) p[k] = cur.ok ? cur.p[k] : F.lo[k] + 1.0f / F.sx[k];  // box centre when idle
      float v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
      const float vn = sqrtf(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
      const float dir[3] = {v[0] / vn, v[1] / vn, v[2] / vn};
      float pe[32];
      pos_enc(dir, pe);
      store_cols<64, 32, 32, H16>(sm + oAc, r, pe);
    }
    fence_smem_async();
    fence_before();
    if (geo) group_sync<1>();
    else group_sync<2>();
    fence_after();
    if (r == 0) {
      if (geo) gemm<64, 32, H16>(tm + 0, sm + oAg, sm + oW0g);
      else gemm<64, 64, H16>(tm + 64, sm + oAc, sm + oW0c);
      commit(bar);
    }
    // the next tile's inputs, in flight during this tile's MMA chain, and
    // the Gaussian ids of the one after
    const QueryRow q = cur;
    if (tile + G < ntile) {
      const int i1 = (tile + G) * 128 + r, i2 = (tile + 2 * G) * 128 + r;
      fetch_row(io, geo, i1, gn, row_ok(io, i1, nv, gn), cur);
      gn = (tile + 2 * G < ntile && i2 < nv) ? io.vis_ids[i2] : 0;
    }
    if (!(geo ? wait_phase_group<1>(bar, phase) : wait_phase_group<2>(bar, phase))) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu64<H16>(tm + lane + colD, b0, Hs, r);
    fence_smem_async();
    fence_before();
    if (geo) group_sync<1>();
    else group_sync<2>();
    fence_after();
    if (r == 0) {
      if (geo) gemm<64, 64, H16>(tm + 0, sm + oHg, sm + oW1g);
      else gemm<64, 64, H16>(tm + 64, sm + oHc, sm + oW1c);
      commit(bar);
    }
    if (!(geo ? wait_phase_group<1>(bar, phase) : wait_phase_group<2>(bar, phase))) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu64<H16>(tm + lane + colD, b1, Hs, r);
    fence_smem_async();
    fence_before();
    if (geo) group_sync<1>();
    else group_sync<2>();
    fence_after();
    if (r == 0) {
      if (geo) gemm<16, 64, H16>(tm + 0, sm + oHg, sm + oW2g);
      else gemm<16, 64, H16>(tm + 64, sm + oHc, sm + oW2c);
      commit(bar);
    }
    if (!(geo ? wait_phase_group<1>(bar, phase) : wait_phase_group<2>(bar, phase))) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    float o[16];
    ld16(tm + lane + colD, o);
    const int i = q.i;
    if (q.ok) {
      if (geo) {
        // Eq. 7: alpha, scale from the geometry decoder, rotation normalised
        io.alpha[i] = sigmoidf_(o[0] + b2[0] + q.e[0]);
        const float se = q.e[1];
#pragma unroll
        for (int k = 0; k < 3; ++k) io.scale[3 * i + k] = sigmoidf_(o[1 + k] + b2[1 + k] + se);
        float qq[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) qq[k] = o[4 + k] + b2[4 + k];
        const float rn = sqrtf(qq[0] * qq[0] + qq[1] * qq[1] + qq[2] * qq[2] + qq[3] * qq[3]);
        const float den = fmaxf(rn, 1e-12f);
#pragma unroll
        for (int k = 0; k < 4; ++k) io.quat[4 * i + k] = qq[k] / den;
      } else {
#pragma unroll
        for (int k = 0; k < 3; ++k)
          io.color[3 * i + k] = sigmoidf_(o[k] + b2[k] + q.e[k]);
      }
    }
    // (the next tile's first MMA, which overwrites these tensor-memory
    // columns, is issued after its operand barrier)
    fence_before();
  }
  if (failed) {
    set_status(io.status, HYRF_ERR_TIMEOUT);
    for (uint32_t it = 0; it < kSpin; ++it)
      if (try_wait(bar, phase)) break;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kQueryTmemCols));
}

// ---------------------------------------------------------------- background, exact mode

// The pixels' inputs share the hidden activations' buffer (bAc = bHc), and
// the output layer reuses tensor-memory columns [0, 16): six CTAs per SM.
constexpr int bW0c = 0, bW1c = bW0c + 64 * 64 * 2, bW2c = bW1c + 64 * 64 * 2, bHc = bW2c + 16 * 64 * 2,
              bAc = bHc, bBias = bHc + 128 * 64 * 2, kBgSmem = bBias + 144 * 4;
constexpr uint32_t kBgTmemCols = 64;

template <bool H16>
__global__ void __launch_bounds__(128, 6) k_bg_exact_fwd_tc(FieldsDev F, CamDev cam, float radius,
                                                           const uint32_t* __restrict__ Xb,
                                                           const int32_t* __restrict__ px_ids,
                                                           const int32_t* __restrict__ n_px,
                                                           const float* __restrict__ C_fg,
                                                           const float* __restrict__ T_final,
                                                           float* __restrict__ C, int32_t* status) {
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, w = t >> 5;
  float* bias = reinterpret_cast<float*>(sm + bBias);
  float *b0 = bias, *b1 = bias + 64, *b2 = bias + 128;
  stage_w<64, 64>(sm + bW0c, F.cm.W[0], 64);
  stage_w<64, 64>(sm + bW1c, F.cm.W[1], 64);
  stage_w<16, 64>(sm + bW2c, F.cm.W[2], 3);
  if (t < 64) {
    b0[t] = F.cm.b[0][t];
    b1[t] = F.cm.b[1][t];
  }
  if (t < 16) b2[t] = t < 3 ? F.cm.b[2][t] : 0.0f;
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kBgTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_smem_async();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tm = tmem_base;
  const uint32_t lane = ((uint32_t)(w * 32)) << 16;
  const int P = cam.W * cam.H;
  const int rows = px_ids ? min(*n_px, P) : P;  // listed pixels, or all
  const int ntile = (rows + 127) / 128;
  uint32_t phase = 0;
  bool failed = false;
  // this thread's next row (pixel id and bf16 features), fetched a tile ahead
  uint4 xn[4];
  int pn = 0;
  bool okn = false;
  auto fetch = [&](int tile) {
    const int row = tile * 128 + t;
    okn = row < rows;
    pn = okn ? (px_ids ? px_ids[row] : row) : 0;
    const uint4* s4 = reinterpret_cast<const uint4*>(Xb + (size_t)(okn ? row : 0) * 16);
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) xn[kc] = okn ? __ldg(s4 + kc) : make_uint4(0u, 0u, 0u, 0u);
  };
  if ((int)blockIdx.x < ntile) fetch(blockIdx.x);
  for (int tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
    const bool ok = okn;
    const int p = pn;
    {
#pragma unroll
      for (int kc = 0; kc < 4; ++kc) *reinterpret_cast<uint4*>(sm + bAc + kmaj(t, 8 * kc, 64)) = xn[kc];
      float ps[3], dir[3], pe[32];
      bg_ray(cam, F, radius, p % cam.W, p / cam.W, ps, dir);
      pos_enc(dir, pe);
      store_cols<64, 32, 32, H16>(sm + bAc, t, pe);
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      gemm<64, 64, H16>(tm, sm + bAc, sm + bW0c);
      commit(&bar);
    }
    if (tile + (int)gridDim.x < ntile) fetch(tile + gridDim.x);
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu64<H16>(tm + lane, b0, sm + bHc, t);
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      gemm<64, 64, H16>(tm, sm + bHc, sm + bW1c);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu64<H16>(tm + lane, b1, sm + bHc, t);
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    if (t == 0) {
      gemm<16, 64, H16>(tm, sm + bHc, sm + bW2c);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    float o[16];
    ld16(tm + lane, o);
    if (ok) {
      const float T = T_final[p];
#pragma unroll
      for (int k = 0; k < 3; ++k)
        C[3 * (int64_t)p + k] = C_fg[3 * (int64_t)p + k] + T * sigmoidf_(o[k] + b2[k]);
    }
    // (the next tile's first MMA, which overwrites these columns, is issued
    // after its operand barrier)
    fence_before();
  }
  if (failed) {
    set_status(status, HYRF_ERR_TIMEOUT);
    for (uint32_t it = 0; it < kSpin; ++it)
      if (try_wait(&bar, phase)) break;
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kBgTmemCols));
}

// The bounded wait of the tensor-core kernels on a barrier that nothing
// completes (hyrf_check_bounded_wait): gives up after `polls` polls, sets
// HYRF_ERR_TIMEOUT and returns.
__global__ void __launch_bounds__(128) k_wait_check(int32_t* status, uint32_t polls) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  __syncthreads();
  if (!wait_phase(&bar, 0u, polls) && threadIdx.x == 0) set_status(status, HYRF_ERR_TIMEOUT);
}

}  // namespace tc

// ---------------------------------------------------------------- launchers

size_t precull_workspace(int n);

// Workspace of the BF16 forward calls beyond their own: bf16 features of
// `rows` rows for `fields` fields.
size_t tc_fwd_feature_bytes(int64_t rows, int fields) { return align_up((size_t)fields * rows * 64); }

hyrf_status launch_query_fwd_tc(const hyrf_query_fields_args& a, const FieldsDev& F, void* ws, cudaStream_t s) {
  if (a.n == 0) return HYRF_OK;
  Carver c(ws);
  c.take<char>(precull_workspace(a.n));
  uint32_t* X = a.features ? static_cast<uint32_t*>(a.features) : c.take<uint32_t>((size_t)2 * a.n * 16);
  uint32_t *Xg = X, *Xr = X + (size_t)a.n * 16;
  const CamDev cam = to_dev(a.cam);
  const RowSource RS{0, a.n, a.vis_ids, a.n_vis, a.pos, 0.0f, a.status, nullptr, nullptr};
  hyrf_status st = launch_gather(F, cam, RS, a.n, Xg, Xr, s);
  if (st != HYRF_OK) return st;
  tc::QueryIO io{a.n,     a.pos, a.alpha_e, a.scale_e, a.color_e, a.vis_ids, a.n_vis,
                 Xg,      Xr,    a.alpha,   a.scale,   a.quat,    a.color,   a.status};
  int tiles = (a.n + 127) / 128;
  int grid = num_sms() * 3;
  if (tiles < grid) grid = tiles;
  if (F.cm.f16) {
    set_smem_limit<tc::k_query_fwd_tc<true>>(tc::kQuerySmem);
    HYRF_LAUNCH("k_query_fwd_tc", s, tc::k_query_fwd_tc<true><<<grid, 256, tc::kQuerySmem, s>>>(F, cam, io));
  } else {
    set_smem_limit<tc::k_query_fwd_tc<false>>(tc::kQuerySmem);
    HYRF_LAUNCH("k_query_fwd_tc", s, tc::k_query_fwd_tc<false><<<grid, 256, tc::kQuerySmem, s>>>(F, cam, io));
  }
  return HYRF_OK;
}

// Render-time background skip (tau_T > 0): C = C_fg where T_final < tau_T;
// the other pixels are listed, in image order within each CTA, for the
// gather and the decoder.
__global__ void __launch_bounds__(256) k_bg_select(int P, float tau, const float* __restrict__ T_final,
                                                   const float* __restrict__ C_fg, float* __restrict__ C,
                                                   int32_t* __restrict__ list, int32_t* __restrict__ count) {
  __shared__ int wsum[8];
  __shared__ int base;
  const int t = threadIdx.x, lane = t & 31, w = t >> 5;
  for (int p0 = blockIdx.x * 256; p0 < P; p0 += gridDim.x * 256) {
    const int p = p0 + t;
    const bool in = p < P;
    const bool keep = in && T_final[p] >= tau;
    if (in && !keep) {
#pragma unroll
      for (int k = 0; k < 3; ++k) C[3 * (int64_t)p + k] = C_fg[3 * (int64_t)p + k];
    }
    const unsigned bal = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) wsum[w] = __popc(bal);
    __syncthreads();
    if (t == 0) {
      int tot = 0;
      for (int q = 0; q < 8; ++q) {
        const int c = wsum[q];
        wsum[q] = tot;
        tot += c;
      }
      base = atomicAdd(count, tot);
    }
    __syncthreads();
    if (keep) list[base + wsum[w] + __popc(bal & ((1u << lane) - 1u))] = p;
    __syncthreads();
  }
}

// Workspace of the BF16 exact background forward: features, and with tau_T
// the pixel list and its count.
size_t tc_bg_fwd_workspace(int64_t P, bool have_features, bool skip) {
  Carver c(nullptr);
  if (!have_features) c.take<uint32_t>((size_t)P * 16);
  if (skip) {
    c.take<int32_t>((size_t)P);
    c.take<int32_t>(1);
  }
  return c.size();
}

hyrf_status launch_bg_gather(const hyrf_composite_background_args& a, const FieldsDev& F, cudaStream_t s) {
  const CamDev cam = to_dev(a.cam);
  const RowSource RS{1, 0, nullptr, nullptr, nullptr, a.bg.radius, a.status, nullptr, nullptr};
  return launch_gather(F, cam, RS, cam.W * cam.H, nullptr, static_cast<uint32_t*>(a.features), s);
}

hyrf_status launch_bg_exact_fwd_tc(const hyrf_composite_background_args& a, const FieldsDev& F, void* ws,
                                   cudaStream_t s) {
  const CamDev cam = to_dev(a.cam);
  const int P = cam.W * cam.H;
  const bool skip = a.bg.tau_T > 0.0f;
  Carver c(ws);
  // with the skip the rows are the listed pixels: the caller's feature buffer
  // (pixel-indexed, for the reverse) is not written
  uint32_t* Xb = a.features && !skip ? static_cast<uint32_t*>(a.features) : c.take<uint32_t>((size_t)P * 16);
  int32_t* list = nullptr;
  int32_t* count = nullptr;
  if (skip) {
    list = c.take<int32_t>((size_t)P);
    count = c.take<int32_t>(1);
    cudaMemsetAsync(count, 0, sizeof(int32_t), s);
    int blocks = (P + 255) / 256;
    if (blocks > num_sms() * 8) blocks = num_sms() * 8;
    HYRF_LAUNCH("k_bg_select", s,
                k_bg_select<<<blocks, 256, 0, s>>>(P, a.bg.tau_T, a.T_final, a.C_fg, a.C, list, count));
  }
  const RowSource RS{1, 0, nullptr, nullptr, nullptr, a.bg.radius, a.status, list, count};
  const bool ready = a.features && a.features_ready && !skip;  // gathered ahead (hyrf_gather_background)
  hyrf_status st = ready ? HYRF_OK : launch_gather(F, cam, RS, P, nullptr, Xb, s);
  if (st != HYRF_OK) return st;
  int tiles = (P + 127) / 128;
  int grid = num_sms() * 6;
  if (tiles < grid) grid = tiles;
  if (F.cm.f16) {
    set_smem_limit<tc::k_bg_exact_fwd_tc<true>>(tc::kBgSmem);
    HYRF_LAUNCH("k_bg_exact_fwd_tc", s,
                tc::k_bg_exact_fwd_tc<true><<<grid, 128, tc::kBgSmem, s>>>(F, cam, a.bg.radius, Xb, list, count,
                                                                          a.C_fg, a.T_final, a.C, a.status));
  } else {
    set_smem_limit<tc::k_bg_exact_fwd_tc<false>>(tc::kBgSmem);
    HYRF_LAUNCH("k_bg_exact_fwd_tc", s,
                tc::k_bg_exact_fwd_tc<false><<<grid, 128, tc::kBgSmem, s>>>(F, cam, a.bg.radius, Xb, list, count,
                                                                           a.C_fg, a.T_final, a.C, a.status));
  }
  return HYRF_OK;
}

hyrf_status launch_wait_check(int32_t* status, uint32_t polls, cudaStream_t s) {
  HYRF_LAUNCH("k_wait_check", s, tc::k_wait_check<<<1, 128, 0, s>>>(status, polls));
  return HYRF_OK;
}

}  // namespace hyrf
