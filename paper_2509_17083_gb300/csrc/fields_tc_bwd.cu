// Reverse of the BF16 decoders (Eqs. 4, 6) and of the aggregation (Eq. 7)
// on the tensor cores. One CTA of 256 threads owns a tile of 128 rows (the
// MMA M dimension; two threads per row, each taking half of every row's
// columns) and one decoder:
//
//   X = bf16 hash features of the rows (written by k_gather, gather.cu)
//   forward recompute  X -> H1 -> H2 -> O          (K-major A, K-major B)
//   dZ2 = reverse of Eq. 7 (or of Eq. 10 for background pixels), x loss scale
//   dH2 = dZ2 W2,  dW2 += dZ2^T H2                  (B MN-major; A and B MN-major)
//   dZ1 = dH2 * [H2 > 0] -> dH1 = dZ1 W1, dW1 += dZ1^T H1
//   dZ0 = dH1 * [H1 > 0] -> dX  = dZ0 W0, dW0 += dZ0^T X
//   dX: the feature part goes to global memory (f32) for k_scatter, the
//   positional-encoding part of the colour decoder to dL/dposition here
//
// dX products read the forward weight tile as an MN-major B operand, so no
// transposed copy exists. Weight gradients are formed transposed, dW^T =
// A^T dZ with the layer input A read as an MN-major operand (M = 128 output
// rows: A's columns and, from a column of ones the row tiles carry, the bias
// gradient), and stay in tensor memory over every tile the persistent CTA
// takes; at the end each CTA writes them to its f32 slab and one reduction
// kernel sums the slabs. Hidden activations are recomputed, never stored in
// global memory.
#include "tc_ops.cuh"

namespace hyrf {
namespace tc {

// Sums of 16 columns over the 32 lanes of a warp by recursive halving: at
// each step a lane keeps half of its partial sums and adds its partner's
// copy of that half (16 shuffles instead of 16 x 5). On return lane l holds
// the sum of column col_of_lane(l); lanes l and l ^ 1 hold the same column.
__device__ __forceinline__ float col_sum16(const float* in) {
  const int lane = threadIdx.x & 31;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = in[j];
#pragma unroll
  for (int h = 8, o = 16; h >= 1; h >>= 1, o >>= 1) {
    const bool up = lane & o;
#pragma unroll
    for (int j = 0; j < h; ++j) {
      const float send = up ? v[j] : v[j + h];
      const float keep = up ? v[j + h] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__device__ __forceinline__ int col_of_lane(int lane) {
  return ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
}

__device__ __forceinline__ void unpack8(uint4 u, float* v) {
  const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&w[k]));
    v[2 * k] = f.x;
    v[2 * k + 1] = f.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float* v) {
  uint4 u;
  u.x = pack2(v[0], v[1]);
  u.y = pack2(v[2], v[3]);
  u.z = pack2(v[4], v[5]);
  u.w = pack2(v[6], v[7]);
  return u;
}

// ---------------------------------------------------------------- point sources

struct GaussP {
  int n;
  const float* pos;
  const float* alpha_e;
  const float* scale_e;
  const float* color_e;
  const int32_t* vis_ids;
  const int32_t* n_vis;
  const float* d_alpha;
  const float* d_scale;
  const float* d_quat;
  const float* d_color;
  const uint32_t* Xg;   // [n_vis][32] bf16 features of the geometry field
  const uint32_t* Xr;   // [n_vis][32] bf16 features of the radiance field
  float* dXg;           // [n_vis][32] f32 out
  float* dXr;           // [n_vis][32] f32 out
  float* d_pos;
  float* d_alpha_e;
  float* d_scale_e;
  float* d_color_e;
  int32_t* status;
  // Optional list of the visible rows to process (those with a non-zero
  // upstream gradient) and its device count; NULL: every visible row. Row k
  // of dXg / dXr belongs to list[k]; Xg / Xr and the upstream gradients are
  // indexed by visible row.
  const int32_t* list;
  const int32_t* n_list;
};

__device__ __forceinline__ void store_dx16(float* dst, const float* dx) {
  float4* d4 = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int k = 0; k < 4; ++k) __stcs(d4 + k, make_float4(dx[4 * k], dx[4 * k + 1], dx[4 * k + 2], dx[4 * k + 3]));
}

// Two threads serve each row: half h = 0 (warps 0-3) and h = 1 (warps 4-7).
// begin() fills the row's operand columns and the state its half needs;
// dz_out() runs on half 0 only; finish() gets the half's share of dX.

// Visible row v of list position idx, and its Gaussian g; false (with v =
// g = 0) past the end or for an out-of-range index.
__device__ __forceinline__ bool gauss_row(const GaussP& P, int idx, bool ok, int& v, int& g) {
  v = ok ? (P.list ? P.list[idx] : idx) : 0;
  g = ok && v >= 0 && v < P.n ? P.vis_ids[v] : 0;
  if (ok && (v < 0 || v >= P.n || g < 0 || g >= P.n)) {
    set_status(P.status, HYRF_ERR_BOUNDS);
    v = g = 0;
    return false;
  }
  return ok;
}

__device__ __forceinline__ int gauss_count(const GaussP& P) {
  const int nv = min(*P.n_vis, P.n);
  return P.list ? min(*P.n_list, nv) : nv;
}

// Geometry decoder at visible Gaussians: inputs enc(y; Theta_geo), outputs
// (alpha_n, s_n[3], r_n[4]).
struct GeoGauss {
  static constexpr int IN = 32, OUT = 8, DEC = 0, DXC = 32;
  static constexpr const char* kName = "k_decoder_bwd_tc<GeoGauss>";
  using Params = GaussP;
  struct Row {
    int i, g;
    bool ok;
    float da, ds[3], dq[4], ae, se;
  };
  __device__ static int count(const Params& P) { return gauss_count(P); }
  __device__ static const MlpDev& mlp(const FieldsDev& F) { return F.gm; }
  __device__ static void begin(const Params& P, const FieldsDev&, const CamDev&, int idx, bool ok, Row& R,
                               uint8_t* X, int r, int h) {
    R.i = idx;
    int v;
    R.ok = gauss_row(P, idx, ok, v, R.g);
    // half h copies feature columns [16h, 16h + 16)
    const uint4* src = reinterpret_cast<const uint4*>(P.Xg + (size_t)v * 16) + 2 * h;
#pragma unroll
    for (int kc = 0; kc < 2; ++kc) {
      const uint4 v = R.ok ? __ldcs(src + kc) : make_uint4(0u, 0u, 0u, 0u);
      *reinterpret_cast<uint4*>(X + kmaj(r, 16 * h + 8 * kc, IN + 8)) = v;
    }
    if (h != 0) return;
    R.da = R.ok ? P.d_alpha[v] : 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) R.ds[k] = R.ok ? P.d_scale[3 * v + k] : 0.0f;
#pragma unroll
    for (int k = 0; k < 4; ++k) R.dq[k] = R.ok ? P.d_quat[4 * v + k] : 0.0f;
    R.ae = R.ok && P.alpha_e ? P.alpha_e[R.g] : 0.0f;
    R.se = R.ok && P.scale_e ? P.scale_e[R.g] : 0.0f;
  }
  // Reverse of Eq. 7 for alpha, scale and rotation; o = raw decoder outputs.
  __device__ static void dz_out(const Params& P, Row& R, const float* o, float* dz) {
    const float a = sigmoidf_(o[0] + R.ae);
    dz[0] = R.da * a * (1.0f - a);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float s = sigmoidf_(o[1 + k] + R.se);
      dz[1 + k] = R.ds[k] * s * (1.0f - s);
    }
    const float rn = sqrtf(o[4] * o[4] + o[5] * o[5] + o[6] * o[6] + o[7] * o[7]);
    if (rn > 1e-12f) {
      const float irn = 1.0f / rn;
      float qd = 0.0f;
#pragma unroll
      for (int k = 0; k < 4; ++k) qd += o[4 + k] * irn * R.dq[k];
#pragma unroll
      for (int k = 0; k < 4; ++k) dz[4 + k] = (R.dq[k] - o[4 + k] * irn * qd) * irn;
    } else {
#pragma unroll
      for (int k = 0; k < 4; ++k) dz[4 + k] = R.dq[k] / 1e-12f;
    }
    if (!R.ok) {
#pragma unroll
      for (int k = 0; k < 8; ++k) dz[k] = 0.0f;
      return;
    }
    // one row per Gaussian: the adds never meet; reductions do not wait
    if (P.d_alpha_e) atomicAdd(P.d_alpha_e + R.g, dz[0]);
    if (P.d_scale_e) atomicAdd(P.d_scale_e + R.g, dz[1] + dz[2] + dz[3]);
  }
  // dx = dX columns [16h, 16h + 16)
  __device__ static void finish(const Params& P, const FieldsDev&, const CamDev&, Row& R, const float* dx,
                                int h) {
    if (R.ok) store_dx16(P.dXg + (size_t)R.i * 32 + 16 * h, dx);
  }
};

// Colour decoder at visible Gaussians: inputs enc(y; Theta_rad) (+) PE(dir).
// The PE part of dX goes to dL/dp here (half 1); the feature part goes out
// for the scatter (half 0).
struct ColGauss {
  static constexpr int IN = 64, OUT = 3, DEC = 1, DXC = 64;
  using Params = GaussP;
  static constexpr const char* kName = "k_decoder_bwd_tc<ColGauss>";
  struct Row {
    int i, g;
    bool ok;
    float dir[3], vn, dc[3], ce[3];
  };
  __device__ static int count(const Params& P) { return gauss_count(P); }
  __device__ static const MlpDev& mlp(const FieldsDev& F) { return F.cm; }
  __device__ static void begin(const Params& P, const FieldsDev& F, const CamDev& cam, int idx, bool ok,
                               Row& R, uint8_t* X, int r, int h) {
    R.i = idx;
    int v;
    R.ok = gauss_row(P, idx, ok, v, R.g);
    if (h == 0) {
      load_row32<IN + 8>(X, r, P.Xr + (size_t)v * 16, R.ok);
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        R.dc[k] = R.ok ? P.d_color[3 * v + k] : 0.0f;
        R.ce[k] = R.ok && P.color_e ? P.color_e[3 * (int64_t)R.g + k] : 0.0f;
      }
      return;
    }
    float p[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) p[k] = R.ok ? P.pos[3 * (int64_t)R.g + k] : F.lo[k] + 1.0f / F.sx[k];
    float pc[3];
    cam_center(cam, pc);
    const float d[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
    R.vn = sqrtf(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) R.dir[k] = d[k] / R.vn;
    float pe[32];
    pos_enc(R.dir, pe);
    store_cols<IN + 8, 32, 32>(X, r, pe);
  }
  __device__ static void dz_out(const Params& P, Row& R, const float* o, float* dz) {
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float c = sigmoidf_(o[k] + R.ce[k]);
      dz[k] = R.ok ? R.dc[k] * c * (1.0f - c) : 0.0f;
    }
    if (R.ok && P.d_color_e) {
#pragma unroll
      for (int k = 0; k < 3; ++k) atomicAdd(P.d_color_e + 3 * (int64_t)R.g + k, dz[k]);
    }
  }
  // dx = dX columns [32h, 32h + 32)
  __device__ static void finish(const Params& P, const FieldsDev&, const CamDev&, Row& R, const float* dx,
                                int h) {
    if (!R.ok) return;
    if (h == 0) {
      store_dx16(P.dXr + (size_t)R.i * 32, dx);
      store_dx16(P.dXr + (size_t)R.i * 32 + 16, dx + 16);
      return;
    }
    float ddir[3];
    pos_enc_bwd(R.dir, dx, ddir);
    const float dd = R.dir[0] * ddir[0] + R.dir[1] * ddir[1] + R.dir[2] * ddir[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) atomicAdd(P.d_pos + 3 * (int64_t)R.g + j, (ddir[j] - R.dir[j] * dd) / R.vn);
  }
};

struct PixelP {
  float radius;
  const float* T_final;
  const float* dC;
  const uint32_t* Xb;   // [W*H][32] bf16 radiance features at the sphere hits
  float* dXb;           // [W*H][32] f32 out
  float* dC_fg;
  float* dT;
};

// Colour decoder at the background-sphere hit of every pixel (exact mode):
// reverse of C = C_fg + T_final sigma(c_n).
struct BgPixel {
  static constexpr int IN = 64, OUT = 3, DEC = 1, DXC = 32;
  using Params = PixelP;
  static constexpr const char* kName = "k_decoder_bwd_tc<BgPixel>";
  struct Row {
    int p;
    bool ok;
    float T, g[3];
  };
  __device__ static int count_px(const CamDev& cam) { return cam.W * cam.H; }
  __device__ static const MlpDev& mlp(const FieldsDev& F) { return F.cm; }
  __device__ static void begin(const Params& P, const FieldsDev& F, const CamDev& cam, int idx, bool ok,
                               Row& R, uint8_t* X, int r, int h) {
    R.ok = ok;
    R.p = ok ? idx : 0;
    if (h == 0) {
      load_row32<IN + 8>(X, r, P.Xb + (size_t)R.p * 16, ok);
      R.T = ok ? P.T_final[R.p] : 0.0f;
#pragma unroll
      for (int k = 0; k < 3; ++k) R.g[k] = ok ? P.dC[3 * (int64_t)R.p + k] : 0.0f;
      return;
    }
    float ps[3], dir[3], pe[32];
    bg_ray(cam, F, P.radius, R.p % cam.W, R.p / cam.W, ps, dir);
    pos_enc(dir, pe);
    store_cols<IN + 8, 32, 32>(X, r, pe);
  }
  __device__ static void dz_out(const Params& P, Row& R, const float* o, float* dz) {
    float dt = 0.0f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float cs = sigmoidf_(o[k]);
      dt += R.g[k] * cs;
      dz[k] = R.g[k] * R.T * cs * (1.0f - cs);
    }
    if (R.ok) {
      if (P.dT) P.dT[R.p] = dt;
      if (P.dC_fg) {
#pragma unroll
        for (int k = 0; k < 3; ++k) P.dC_fg[3 * (int64_t)R.p + k] = R.g[k];
      }
    }
  }
  // dx = dX columns [16h, 16h + 16)
  __device__ static void finish(const Params& P, const FieldsDev&, const CamDev&, Row& R, const float* dx,
                                int h) {
    if (R.ok) store_dx16(P.dXb + (size_t)R.p * 32 + 16 * h, dx);
  }
};

template <class S>
__device__ __forceinline__ int point_count(const typename S::Params& P, const CamDev& cam) {
  if constexpr (std::is_same<S, BgPixel>::value) {
    return BgPixel::count_px(cam);
  } else {
    return S::count(P);
  }
}

// ---------------------------------------------------------------- the kernel

// Shared-memory map. The row tiles X, H1 and H2 carry 8 columns past their
// data: a column of ones (column IN, resp. 64) and seven zeros, so that the
// weight-gradient products A^T dZ also give the bias gradients (the row of
// ones sums dZ over the tile's points). Those products read A with 128
// output rows; rows past a tile's columns come from the bytes that follow it
// (always inside this map: each tile is followed by another or the guard).
template <int IN>
struct BwdSmem {
  static constexpr int XP = IN + 8, HP = 64 + 8;
  static constexpr int W0 = 0, W1 = W0 + 64 * IN * 2, W2 = W1 + 64 * 64 * 2, X = W2 + 16 * 64 * 2,
                       H1 = X + 128 * XP * 2, H2 = H1 + 128 * HP * 2, Z2 = H2 + 128 * HP * 2,
                       GUARD = Z2 + 128 * 16 * 2, BIAS = GUARD + 2048, SIZE = BIAS + 144 * 4;
};
// Tensor memory of a CTA: [0, 64) the products of the current tile; the
// weight gradients (transposed: lane = input column, column = output),
// accumulated over every tile the CTA takes: dW2^T [64, 80), dW1^T
// [80, 144), dW0^T [144, 208).
constexpr uint32_t kBwdTmemCols = 256;
constexpr uint32_t kTmW2 = 64, kTmW1 = 80, kTmW0 = 144;

// ReLU(D + b) of NC accumulator columns [c0, c0 + NC) of this thread's lane
// -> the same columns of its row of the HP-column tile H. taddr points at
// column c0.
template <int NC, int HP>
__device__ __forceinline__ void epilogue_relu(uint32_t taddr, const float* b, uint8_t* H, int r, int c0) {
  float v[NC];
  ldcols<NC>(taddr, v);
#pragma unroll
  for (int c = 0; c < NC; c += 8) {
    const float4 bl = *reinterpret_cast<const float4*>(b + c0 + c),
                 bh = *reinterpret_cast<const float4*>(b + c0 + c + 4);
    uint4 u;
    u.x = add_relu_pack2(v[c], v[c + 1], bl.x, bl.y);
    u.y = add_relu_pack2(v[c + 2], v[c + 3], bl.z, bl.w);
    u.z = add_relu_pack2(v[c + 4], v[c + 5], bh.x, bh.y);
    u.w = add_relu_pack2(v[c + 6], v[c + 7], bh.z, bh.w);
    *reinterpret_cast<uint4*>(H + kmaj(r, c0 + c, HP)) = u;
  }
}

// ReLU mask from the bf16 activations of this row, applied to NC columns
// [c0, c0 + NC) of D read from tensor memory (taddr at column c0); the
// masked gradient replaces the activations in place (bf16).
template <int NC, int HP>
__device__ __forceinline__ void relu_back(uint32_t taddr, uint8_t* Hbuf, int r, bool ok, int c0) {
  float v[NC];
  ldcols<NC>(taddr, v);
#pragma unroll
  for (int c = 0; c < NC; c += 8) {
    float hv[8];
    unpack8(*reinterpret_cast<const uint4*>(Hbuf + kmaj(r, c0 + c, HP)), hv);
#pragma unroll
    for (int j = 0; j < 8; ++j) v[c + j] = (ok && hv[j] > 0.0f) ? v[c + j] : 0.0f;
    *reinterpret_cast<uint4*>(Hbuf + kmaj(r, c0 + c, HP)) = pack8(v + c);
  }
}

// Columns 8 * (this thread's share) of a ones-column block: column `at` of
// the row's tile is 1, the seven after it 0.
template <int P_>
__device__ __forceinline__ void ones_block(uint8_t* tile, int r, int at) {
  float v[8] = {1.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
  *reinterpret_cast<uint4*>(tile + kmaj(r, at, P_)) = pack8(v);
}

// One transposed weight-gradient accumulator (lanes 0 .. NI - 1: input
// column i, lane NI: the bias; columns: outputs 0 .. NO - 1) written into
// the CTA's slab, W [NO][NI] and b [NO] (plain stores: the slab is this
// CTA's alone and every entry of it is written here). Zeros if the CTA took
// no tile.
template <int NCOL>
__device__ __forceinline__ void store_dw(uint32_t tm_acc, int NI, int NO, float* slab_W, float* slab_b, bool any) {
  const int w = threadIdx.x >> 5, q = w & 3, h = w >> 2, lane = threadIdx.x & 31;
  constexpr int HALF = NCOL >= 32 ? NCOL / 2 : NCOL;
  if (q * 32 > NI || (NCOL < 32 && h != 0)) return;  // warp-uniform
  const int i = q * 32 + lane, c0 = NCOL >= 32 ? h * HALF : 0;
  float v[HALF];
  ldcols<HALF>(tm_acc + ((uint32_t)(q * 32) << 16) + c0, v);
#pragma unroll
  for (int k = 0; k < HALF; ++k) {
    const int o = c0 + k;
    if (o >= NO) break;
    const float x = any ? v[k] : 0.0f;
    if (i < NI) slab_W[o * NI + i] = x;
    else if (i == NI) slab_b[o] = x;
  }
}

__device__ __forceinline__ void sync_for_mma() {
  fence_smem_async();
  fence_before();
  __syncthreads();
  fence_after();
}

// 256 threads: row r = t % 128 of the tile, half h = t / 128. Warps w and
// w + 4 read the same TMEM lanes (32 (w % 4) ...) and split the columns.
// Persistent: the CTA takes tiles blockIdx.x, blockIdx.x + gridDim.x, ...
// and keeps its weight and bias gradients in tensor memory until the end.
template <class S>
__global__ void __launch_bounds__(256, 2) k_decoder_bwd_tc(typename S::Params P, FieldsDev F, CamDev cam,
                                                           float loss_scale, SlabLayout SL, float* slabs,
                                                           int32_t* status) {
  constexpr int IN = S::IN, OUT = S::OUT;
  using L = BwdSmem<IN>;
  constexpr int XP = L::XP, HP = L::HP;
  extern __shared__ __align__(1024) uint8_t sm[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ uint32_t tmem_base;
  const int t = threadIdx.x, w = t >> 5, h = t >> 7, r = t & 127;
  const MlpDev& M = S::mlp(F);
  float* bias = reinterpret_cast<float*>(sm + L::BIAS);
  stage_w<64, IN>(sm + L::W0, M.W[0], 64);
  stage_w<64, 64>(sm + L::W1, M.W[1], 64);
  stage_w<16, 64>(sm + L::W2, M.W[2], OUT);
  if (t < 64) {
    bias[t] = M.b[0][t];
    bias[64 + t] = M.b[1][t];
  }
  if (t < 16) bias[128 + t] = t < OUT ? M.b[2][t] : 0.0f;
  if (h == 0) ones_block<XP>(sm + L::X, r, IN);
  else {
    ones_block<HP>(sm + L::H1, r, 64);
    ones_block<HP>(sm + L::H2, r, 64);
  }
  if (t == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(saddr(&bar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  if (w == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(saddr(&tmem_base)),
                 "r"(kBwdTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  sync_for_mma();
  const uint32_t tm = tmem_base;
  const uint32_t lane_off = ((uint32_t)((w & 3) * 32)) << 16;
  float* slab = slabs + (size_t)blockIdx.x * SL.total;
  const float inv_ls = 1.0f / loss_scale;
  const int n = point_count<S>(P, cam);
  const int ntile = (n + 127) / 128;
  const int hc = 32 * h;  // this half's first column of 64
  uint32_t phase = 0;
  bool failed = false, any = false;
  for (int tile = blockIdx.x; tile < ntile && !failed; tile += gridDim.x) {
    const int idx = tile * 128 + r;
    const bool ok = idx < n;
    typename S::Row R;
    S::begin(P, F, cam, idx, ok, R, sm + L::X, r, h);
    // ---- forward recompute
    sync_for_mma();
    if (t == 0) {
      gemm_ap<64, IN, XP>(tm, sm + L::X, sm + L::W0);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu<32, HP>(tm + lane_off + hc, bias, sm + L::H1, r, hc);
    sync_for_mma();
    if (t == 0) {
      gemm_ap<64, 64, HP>(tm, sm + L::H1, sm + L::W1);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    epilogue_relu<32, HP>(tm + lane_off + hc, bias + 64, sm + L::H2, r, hc);
    sync_for_mma();
    if (t == 0) {
      gemm_ap<16, 64, HP>(tm, sm + L::H2, sm + L::W2);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    if (h == 0) {  // warp-uniform
      float o[16], dz[16];
      ld16(tm + lane_off, o);
#pragma unroll
      for (int k = 0; k < 16; ++k) o[k] += bias[128 + k];
      S::dz_out(P, R, o, dz);
#pragma unroll
      for (int k = 0; k < 16; ++k) dz[k] = k < OUT ? dz[k] * loss_scale : 0.0f;
      *reinterpret_cast<uint4*>(sm + L::Z2 + kmaj(r, 0, 16)) = pack8(dz);
      *reinterpret_cast<uint4*>(sm + L::Z2 + kmaj(r, 8, 16)) = pack8(dz + 8);
    }
    // ---- layer 2: dH2 = dZ2 W2, dW2^T (and db2) += [H2 1]^T dZ2
    sync_for_mma();
    if (t == 0) {
      gemm_dx_ap<64, 16, 16>(tm, sm + L::Z2, sm + L::W2);
      gemm_at<16, HP, 16>(tm + kTmW2, sm + L::H2, sm + L::Z2, any);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    relu_back<32, HP>(tm + lane_off + hc, sm + L::H2, r, ok, hc);  // dZ1 replaces H2
    // ---- layer 1: dH1 = dZ1 W1, dW1^T (and db1) += [H1 1]^T dZ1
    sync_for_mma();
    if (t == 0) {
      gemm_dx_ap<64, 64, HP>(tm, sm + L::H2, sm + L::W1);
      gemm_at<64, HP, HP>(tm + kTmW1, sm + L::H1, sm + L::H2, any);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    relu_back<32, HP>(tm + lane_off + hc, sm + L::H1, r, ok, hc);  // dZ0 replaces H1
    // ---- layer 0: dX = dZ0 W0, dW0^T (and db0) += [X 1]^T dZ0
    sync_for_mma();
    if (t == 0) {
      gemm_dx_ap<IN, 64, HP>(tm, sm + L::H1, sm + L::W0);
      gemm_at<64, XP, HP>(tm + kTmW0, sm + L::X, sm + L::H1, any);
      commit(&bar);
    }
    if (!wait_phase(&bar, phase)) { failed = true; break; }
    phase ^= 1u;
    fence_after();
    any = true;
    {
      constexpr int HALF = S::DXC / 2;
      float dx[HALF];
      ldcols<HALF>(tm + lane_off + h * HALF, dx);
#pragma unroll
      for (int k = 0; k < HALF; ++k) dx[k] *= inv_ls;
      S::finish(P, F, cam, R, dx, h);
    }
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
  // the CTA's weight and bias gradients (x loss scale) into its slab
  const int d = S::DEC;
  store_dw<16>(tm + kTmW2, 64, OUT, slab + SL.off_W[d][2], slab + SL.off_b[d][2], any && !failed);
  store_dw<64>(tm + kTmW1, 64, 64, slab + SL.off_W[d][1], slab + SL.off_b[d][1], any && !failed);
  store_dw<64>(tm + kTmW0, IN, 64, slab + SL.off_W[d][0], slab + SL.off_b[d][0], any && !failed);
  fence_before();
  __syncthreads();
  if (w == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kBwdTmemCols));
}

}  // namespace tc

// ---------------------------------------------------------------- rows with a gradient

// Visible rows whose upstream gradient (dL/d opacity, scale, rotation or
// colour) is not exactly zero (a NaN counts as non-zero). For every other
// row the reverse of the aggregation, of both decoders and of the gather
// adds exactly zero (dZ = 0, so dX = 0 and the row's share of dW and of the
// table gradients is 0), so the reverse runs on the listed rows only, in
// ascending order (the storage order the gather's coherence relies on).
constexpr int kActChunk = 2048;  // rows per compaction CTA (256 threads x 8)

struct GradRows {
  int n;
  const int32_t* n_vis;
  const float* d_alpha;  // [n]
  const float* d_scale;  // [n][3]
  const float* d_quat;   // [n][4]
  const float* d_color;  // [n][3]
};

__device__ __forceinline__ bool row_has_grad(const GradRows& P, int i) {
  bool a = P.d_alpha[i] != 0.0f;
#pragma unroll
  for (int k = 0; k < 3; ++k) a |= (P.d_scale[3 * i + k] != 0.0f) | (P.d_color[3 * i + k] != 0.0f);
#pragma unroll
  for (int k = 0; k < 4; ++k) a |= P.d_quat[4 * i + k] != 0.0f;
  return a;
}

__global__ void __launch_bounds__(256) k_active_count(GradRows P, int32_t* __restrict__ counts) {
  __shared__ int red[8];
  const int nv = min(*P.n_vis, P.n);
  const int base = blockIdx.x * kActChunk;
  int c = 0;
  for (int k = 0; k < kActChunk / 256; ++k) {
    const int i = base + k * 256 + threadIdx.x;
    if (i < nv && row_has_grad(P, i)) ++c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) t += red[w];
    counts[blockIdx.x] = t;
  }
}

// Ordered compaction: the rows of chunk b land at offsets[b] + rank.
__global__ void __launch_bounds__(256) k_active_list(GradRows P, const int32_t* __restrict__ offsets,
                                                     int32_t* __restrict__ list) {
  __shared__ int wsum[8];
  const int nv = min(*P.n_vis, P.n);
  const int base = blockIdx.x * kActChunk;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int run = offsets[blockIdx.x];
  for (int k = 0; k < kActChunk / 256; ++k) {
    const int i = base + k * 256 + threadIdx.x;
    const bool f = i < nv && row_has_grad(P, i);
    const unsigned m = __ballot_sync(0xffffffffu, f);
    if (lane == 0) wsum[w] = __popc(m);
    __syncthreads();
    int before = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      before += j < w ? wsum[j] : 0;
      tot += wsum[j];
    }
    if (f) list[run + before + __popc(m & ((1u << lane) - 1u))] = i;
    run += tot;
    __syncthreads();
  }
}

hyrf_status launch_scan_small(int32_t* counts, int m, int32_t* total, cudaStream_t s);

static int act_chunks(int n) { return n > 0 ? (n + kActChunk - 1) / kActChunk : 0; }

// Workspace of the list of rows with a gradient (n rows at most).
size_t active_rows_workspace(int n) {
  Carver c(nullptr);
  c.take<int32_t>((size_t)act_chunks(n) + 1);
  c.take<int32_t>(1);
  c.take<int32_t>((size_t)(n > 0 ? n : 1));
  return c.size();
}

// The visible rows with a non-zero upstream gradient, ascending, into the
// workspace carved by `c` (active_rows_workspace); *list / *n_list point
// at the list and its device count.
hyrf_status launch_active_rows(int n, const int32_t* n_vis, const float* d_alpha, const float* d_scale,
                               const float* d_quat, const float* d_color, Carver& c, int32_t** list,
                               int32_t** n_list, cudaStream_t s) {
  const int chunks = act_chunks(n);
  int32_t* offsets = c.take<int32_t>((size_t)chunks + 1);
  *n_list = c.take<int32_t>(1);
  *list = c.take<int32_t>((size_t)(n > 0 ? n : 1));
  if (chunks == 0) return cudaMemsetAsync(*n_list, 0, sizeof(int32_t), s) == cudaSuccess ? HYRF_OK : HYRF_ERR_CUDA;
  const GradRows P{n, n_vis, d_alpha, d_scale, d_quat, d_color};
  HYRF_LAUNCH("k_active_count", s, k_active_count<<<chunks, 256, 0, s>>>(P, offsets));
  hyrf_status st = launch_scan_small(offsets, chunks, *n_list, s);
  if (st != HYRF_OK) return st;
  HYRF_LAUNCH("k_active_list", s, k_active_list<<<chunks, 256, 0, s>>>(P, offsets, *list));
  return HYRF_OK;
}

// ---------------------------------------------------------------- launchers

int bwd_ctas();
size_t slab_bytes(const FieldsDev& F, bool geo);
hyrf_status launch_slab_reduce(const float* slabs, int nslabs, const SlabLayout& SL,
                               const SlabTargets& T, float scale, cudaStream_t s);
SlabTargets slab_targets(const hyrf_field_grads& g, bool geo);

// Persistent CTAs of the tensor-core reverse: two per SM (each holds 256
// tensor-memory columns; the shared-memory request below keeps a third
// from being placed on the SM). Each writes every entry of its slab.
static int tc_bwd_ctas() { return 2 * num_sms(); }
constexpr int kBwdSmemMin = 80 * 1024;

template <class S>
static hyrf_status launch_dec_bwd(const typename S::Params& P, const FieldsDev& F, const CamDev& cam,
                                  float ls, const SlabLayout& SL, float* slabs, int32_t* status,
                                  cudaStream_t s) {
  constexpr int smem = tc::BwdSmem<S::IN>::SIZE > kBwdSmemMin ? tc::BwdSmem<S::IN>::SIZE : kBwdSmemMin;
  set_smem_limit<tc::k_decoder_bwd_tc<S>>(smem);
  HYRF_LAUNCH(S::kName, s,
              tc::k_decoder_bwd_tc<S><<<tc_bwd_ctas(), 256, smem, s>>>(P, F, cam, ls, SL, slabs, status));
  return HYRF_OK;
}

// Workspace of the BF16 backward calls: CTA slabs, bf16 features (unless
// the caller saved them in the forward) and f32 feature gradients of `rows`
// rows for one or both fields.
size_t tc_bwd_workspace(const FieldsDev& F, bool geo, int64_t rows, bool have_features) {
  Carver c(nullptr);
  c.take<char>(slab_bytes(F, geo));
  const int fields = geo ? 2 : 1;
  if (!have_features) c.take<uint32_t>((size_t)fields * rows * 16);
  c.take<float>((size_t)fields * rows * 32);
  if (geo) c.take<char>(active_rows_workspace((int)rows));  // the Gaussian rows with a gradient
  return c.size();
}

hyrf_status launch_query_bwd_tc(const hyrf_query_fields_backward_args& a, const FieldsDev& F, void* ws,
                                cudaStream_t s) {
  if (a.n == 0) return HYRF_OK;
  const CamDev cam = to_dev(a.cam);
  const SlabLayout SL = make_slab_layout(&F.gm, &F.cm);
  Carver c(ws);
  float* slabs = reinterpret_cast<float*>(c.take<char>(slab_bytes(F, true)));
  const bool saved = a.features != nullptr;
  uint32_t* X = saved ? const_cast<uint32_t*>(static_cast<const uint32_t*>(a.features))
                      : c.take<uint32_t>((size_t)2 * a.n * 16);
  float* dX = c.take<float>((size_t)2 * a.n * 32);
  uint32_t *Xg = X, *Xr = X + (size_t)a.n * 16;
  float *dXg = dX, *dXr = dX + (size_t)a.n * 32;
  Carver ca(c.take<char>(active_rows_workspace(a.n)));
  const RowSource RS{0, a.n, a.vis_ids, a.n_vis, a.pos, 0.0f, a.status, nullptr, nullptr};
  hyrf_status st = saved ? HYRF_OK : launch_gather(F, cam, RS, a.n, Xg, Xr, s);
  if (st != HYRF_OK) return st;
  tc::GaussP P{a.n,       a.pos,     a.alpha_e, a.scale_e, a.color_e, a.vis_ids,   a.n_vis,
               a.d_alpha, a.d_scale, a.d_quat,  a.d_color, Xg,        Xr,          dXg,
               dXr,       a.d_pos,   a.d_alpha_e, a.d_scale_e, a.d_color_e, a.status, nullptr, nullptr};
  // the rows with a non-zero upstream gradient, in ascending order
  int32_t *list = nullptr, *n_list = nullptr;
  st = launch_active_rows(a.n, a.n_vis, a.d_alpha, a.d_scale, a.d_quat, a.d_color, ca, &list, &n_list, s);
  if (st != HYRF_OK) return st;
  P.list = list;
  P.n_list = n_list;
  st = launch_dec_bwd<tc::GeoGauss>(P, F, cam, a.loss_scale, SL, slabs, a.status, s);
  if (st != HYRF_OK) return st;
  st = launch_dec_bwd<tc::ColGauss>(P, F, cam, a.loss_scale, SL, slabs, a.status, s);
  if (st != HYRF_OK) return st;
  const RowSource RSL{0, a.n, a.vis_ids, a.n_vis, a.pos, 0.0f, a.status, list, n_list};
  st = launch_scatter(F, cam, RSL, a.n, dXg, dXr, a.grads.geo_table, a.grads.rad_table, a.d_pos, s);
  if (st != HYRF_OK) return st;
  return launch_slab_reduce(slabs, tc_bwd_ctas(), SL, slab_targets(a.grads, true), 1.0f / a.loss_scale, s);
}

hyrf_status launch_bg_bwd_tc(const hyrf_composite_background_backward_args& b, const FieldsDev& F,
                             void* ws, cudaStream_t s) {
  const hyrf_composite_background_args& a = b.fwd;
  const CamDev cam = to_dev(a.cam);
  const int P_ = cam.W * cam.H;
  const SlabLayout SL = make_slab_layout(nullptr, &F.cm);
  Carver c(ws);
  float* slabs = reinterpret_cast<float*>(c.take<char>(slab_bytes(F, false)));
  const bool saved = a.features != nullptr;
  uint32_t* Xb = saved ? static_cast<uint32_t*>(a.features) : c.take<uint32_t>((size_t)P_ * 16);
  float* dXb = c.take<float>((size_t)P_ * 32);
  const RowSource RS{1, 0, nullptr, nullptr, nullptr, a.bg.radius, a.status, nullptr, nullptr};
  hyrf_status st = saved ? HYRF_OK : launch_gather(F, cam, RS, P_, nullptr, Xb, s);
  if (st != HYRF_OK) return st;
  tc::PixelP P{a.bg.radius, a.T_final, b.d_C, Xb, dXb, b.d_C_fg, b.d_T_final};
  st = launch_dec_bwd<tc::BgPixel>(P, F, cam, b.loss_scale, SL, slabs, a.status, s);
  if (st != HYRF_OK) return st;
  // decoder gradients first (a plain read-modify-write of the caller's
  // buffers, kept on the caller's stream); the table scatter (atomics only)
  // may then run on the caller's second stream
  st = launch_slab_reduce(slabs, tc_bwd_ctas(), SL, slab_targets(b.grads, false), 1.0f / b.loss_scale, s);
  if (st != HYRF_OK) return st;
  cudaStream_t ss = s;
  if (b.scatter_stream) {
    ss = static_cast<cudaStream_t>(b.scatter_stream);
    st = fork_stream(s, ss);
    if (st != HYRF_OK) return st;
  }
  return launch_scatter(F, cam, RS, P_, nullptr, dXb, nullptr, b.grads.rad_table, nullptr, ss);
}

}  // namespace hyrf
