// tcgen05 building blocks shared by the BF16 decoder kernels: shared-memory
// matrix descriptors (no-swizzle core-matrix layouts), instruction
// descriptors, MMA issue and commit, bounded mbarrier waits, tensor-memory
// loads and the bf16 tile writers.
//
// Core-matrix layout of an R x C bf16 tile, "row-major in core matrices":
// element (r, c) sits at ((r/8) * (C/8) + c/8) * 128 + (r%8) * 16 + (c%8) * 2
// bytes. Read as a K-major operand (rows = M or N, columns = K) its leading
// byte offset (K direction) is 128 and its stride byte offset (M/N
// direction) is C/8 * 128. Read as an MN-major operand (rows = K, columns =
// M or N) the leading byte offset (K direction) is C/8 * 128 and the stride
// byte offset (M/N direction) is 128.
#pragma once
#include <type_traits>

#include "field_ops.cuh"

namespace hyrf {

// Rows of the BF16 field kernels: visible Gaussians or camera pixels.
struct RowSource {
  int pixels;               // 0: visible Gaussians, 1: pixels of the camera
  int n;                    // Gaussians (capacity of vis_ids)
  const int32_t* vis_ids;   // [n]
  const int32_t* n_vis;     // device count
  const float* pos;         // [n][3]
  float radius;             // background sphere radius (pixels)
  int32_t* status;
  // Optional list of the rows to process (pixels, or indices into vis_ids)
  // and its device count; NULL: every row. Row k of the features X written
  // and of the feature gradients dX read belongs to list[k].
  const int32_t* list;
  const int32_t* n_list;
};

// gather.cu: bf16 features X [rows][32] per field, and the reverse scatter
// of f32 feature gradients dX [rows][32]. Gaussians use both fields, pixels
// the radiance field only; `rows` bounds the device row count.
hyrf_status launch_gather(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows, uint32_t* Xg,
                          uint32_t* Xr, cudaStream_t s);
hyrf_status launch_scatter(const FieldsDev& F, const CamDev& cam, const RowSource& S, int rows,
                           const float* dXg, const float* dXr, float* g_geo, float* g_rad, float* d_pos,
                           cudaStream_t s);

namespace tc {

// Polls of a bounded mbarrier wait before it gives up: each poll
// (mbarrier.try_wait, which may suspend the thread) takes ~3.8 us on a
// GB300, so a wait that never completes ends after ~4 s.
constexpr uint32_t kSpin = 1u << 20;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__host__ __device__ constexpr uint32_t kmaj(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D f32, A and B bf16 (or both f16 when
// H16), M = 128; A and B K-major unless AMN / BMN (MN-major).
template <int N, bool AMN = false, bool BMN = false, bool H16 = false>
__device__ __forceinline__ constexpr uint32_t idesc() {
  static_assert(N % 16 == 0 && N >= 16 && N <= 256, "N");
  constexpr uint32_t fmt = H16 ? 0u : ((1u << 7) | (1u << 10));
  return (1u << 4) | fmt | ((AMN ? 1u : 0u) << 15) | ((BMN ? 1u : 0u) << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(saddr(bar)));
}

__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(saddr(bar)), "r"(phase));
  return ok != 0;
}

// Bounded wait on the given phase (at most `polls` polls); returns false
// (on every thread) if any thread of the CTA gave up.
__device__ __forceinline__ bool wait_phase(uint64_t* bar, uint32_t phase, uint32_t polls = kSpin) {
  bool ok = false;
  for (uint32_t it = 0; it < polls && !ok; ++it) ok = try_wait(bar, phase);
  return !__syncthreads_or(!ok);
}

// Named barrier ID over the 128 threads of one group of a CTA (ids from 1;
// id 0 is __syncthreads), and its OR-reduction of a predicate.
template <int ID>
__device__ __forceinline__ void group_sync() {
  asm volatile("bar.sync %0, 128;" ::"n"(ID) : "memory");
}
template <int ID>
__device__ __forceinline__ bool group_or(bool pred) {
  uint32_t r;
  asm volatile(
      "{\n.reg .pred a, b;\nsetp.ne.u32 a, %1, 0;\nbar.red.or.pred b, %2, 128, a;\nselp.u32 %0, 1, 0, b;\n}"
      : "=r"(r)
      : "r"((uint32_t)pred), "n"(ID)
      : "memory");
  return r != 0;
}

// wait_phase for the 128-thread group of named barrier ID.
template <int ID>
__device__ __forceinline__ bool wait_phase_group(uint64_t* bar, uint32_t phase, uint32_t polls = kSpin) {
  bool ok = false;
  for (uint32_t it = 0; it < polls && !ok; ++it) ok = try_wait(bar, phase);
  return !group_or<ID>(!ok);
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 16 consecutive f32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// 32 consecutive f32 accumulator columns of this thread's TMEM lane, one
// load and one wait.
__device__ __forceinline__ void ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// NC consecutive accumulator columns (16 or a multiple of 32) with as few
// load-and-wait round trips as the load shapes allow.
template <int NC>
__device__ __forceinline__ void ldcols(uint32_t taddr, float* v) {
  static_assert(NC == 16 || NC % 32 == 0, "columns");
  if constexpr (NC == 16) {
    ld16(taddr, v);
  } else {
#pragma unroll
    for (int c = 0; c < NC; c += 32) ld32(taddr + c, v + c);
  }
}

// D[128 x N] (+)= A[128 x K] B[N x K]^T with both operands K-major in smem.
template <int N, int K, bool H16 = false>
__device__ __forceinline__ void gemm(uint32_t d, const uint8_t* A, const uint8_t* B) {
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = sdesc(saddr(A) + ks * 256, 128, (K / 8) * 128);
    const uint64_t db = sdesc(saddr(B) + ks * 256, 128, (K / 8) * 128);
    mma(d, da, db, idesc<N, false, false, H16>(), ks > 0 ? 1u : 0u);
  }
}

// As gemm, with A stored with AP >= K columns per row (its core-matrix row
// groups AP / 8 * 128 bytes apart); the first K columns are multiplied.
template <int N, int K, int AP>
__device__ __forceinline__ void gemm_ap(uint32_t d, const uint8_t* A, const uint8_t* B) {
  static_assert(AP >= K && AP % 8 == 0, "A columns");
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = sdesc(saddr(A) + ks * 256, 128, (AP / 8) * 128);
    const uint64_t db = sdesc(saddr(B) + ks * 256, 128, (K / 8) * 128);
    mma(d, da, db, idesc<N>(), ks > 0 ? 1u : 0u);
  }
}

// Two operand values (bf16, or f16 when H16), round to nearest even.
template <bool H16 = false>
__device__ __forceinline__ uint32_t pack2(float a, float b) {
  if constexpr (H16) {
    const __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  } else {
    const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<const uint32_t*>(&h);
  }
}

// Row r of a K-major bf16 tile from 8*n floats.
template <int K>
__device__ __forceinline__ void store_row(uint8_t* tile, int r, const float* v) {
#pragma unroll
  for (int kc = 0; kc < K / 8; ++kc) {
    uint4 u;
    u.x = pack2(v[8 * kc], v[8 * kc + 1]);
    u.y = pack2(v[8 * kc + 2], v[8 * kc + 3]);
    u.z = pack2(v[8 * kc + 4], v[8 * kc + 5]);
    u.w = pack2(v[8 * kc + 6], v[8 * kc + 7]);
    *reinterpret_cast<uint4*>(tile + kmaj(r, 8 * kc, K)) = u;
  }
}

// Columns [C0, C0 + NC) of row r of a K-major bf16 (f16) tile from NC floats.
template <int K, int C0, int NC, bool H16 = false>
__device__ __forceinline__ void store_cols(uint8_t* tile, int r, const float* v) {
#pragma unroll
  for (int kc = 0; kc < NC / 8; ++kc) {
    uint4 u;
    u.x = pack2<H16>(v[8 * kc], v[8 * kc + 1]);
    u.y = pack2<H16>(v[8 * kc + 2], v[8 * kc + 3]);
    u.z = pack2<H16>(v[8 * kc + 4], v[8 * kc + 5]);
    u.w = pack2<H16>(v[8 * kc + 6], v[8 * kc + 7]);
    *reinterpret_cast<uint4*>(tile + kmaj(r, C0 + 8 * kc, K)) = u;
  }
}

// Columns [0, 32) of row r of a K-major bf16 tile from 32 bf16 values in
// global memory (16-byte aligned); zeros if !ok.
template <int K>
__device__ __forceinline__ void load_row32(uint8_t* tile, int r, const uint32_t* src, bool ok) {
  const uint4* s4 = reinterpret_cast<const uint4*>(src);
#pragma unroll
  for (int kc = 0; kc < 4; ++kc) {
    const uint4 v = ok ? __ldg(s4 + kc) : make_uint4(0u, 0u, 0u, 0u);
    *reinterpret_cast<uint4*>(tile + kmaj(r, 8 * kc, K)) = v;
  }
}

// Weights W [rows][K] bf16 (row-major, rows_real valid rows) into a K-major
// tile of N rows (rows >= rows_real zero).
template <int N, int K>
__device__ __forceinline__ void stage_w(uint8_t* tile, const void* W, int rows_real) {
  const uint4* src = static_cast<const uint4*>(W);
  for (int e = threadIdx.x; e < N * (K / 8); e += blockDim.x) {
    const int r = e / (K / 8), kc = e % (K / 8);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (r < rows_real) v = __ldg(src + r * (K / 8) + kc);
    *reinterpret_cast<uint4*>(tile + kmaj(r, 8 * kc, K)) = v;
  }
}

// ReLU(x + bx), ReLU(y + by) rounded to the operand type (bf16, or f16 when
// H16) and packed, x in the low half: one paired f32 add (two independent
// round-to-nearest adds) and one converting instruction that clamps
// negative values to zero. Same values as max(x + bx, 0) rounded to
// nearest even.
template <bool H16 = false>
__device__ __forceinline__ uint32_t add_relu_pack2(float x, float y, float bx, float by) {
  uint32_t r;
  if constexpr (H16) {
    asm("{\n.reg .b64 p, q;\n.reg .f32 lo, hi;\n"
        "mov.b64 p, {%1, %2};\nmov.b64 q, {%3, %4};\n"
        "add.rn.f32x2 p, p, q;\nmov.b64 {lo, hi}, p;\n"
        "cvt.rn.relu.f16x2.f32 %0, hi, lo;\n}"
        : "=r"(r)
        : "f"(x), "f"(y), "f"(bx), "f"(by));
  } else {
    asm("{\n.reg .b64 p, q;\n.reg .f32 lo, hi;\n"
        "mov.b64 p, {%1, %2};\nmov.b64 q, {%3, %4};\n"
        "add.rn.f32x2 p, p, q;\nmov.b64 {lo, hi}, p;\n"
        "cvt.rn.relu.bf16x2.f32 %0, hi, lo;\n}"
        : "=r"(r)
        : "f"(x), "f"(y), "f"(bx), "f"(by));
  }
  return r;
}

// ReLU(D + b) of this thread's 64 accumulator columns -> its row of H
// (bf16, or f16 when H16).
template <bool H16 = false>
__device__ __forceinline__ void epilogue_relu64(uint32_t taddr, const float* b, uint8_t* H, int r) {
#pragma unroll
  for (int c0 = 0; c0 < 64; c0 += 32) {
    float v[32];
    ld32(taddr + c0, v);
    const float4* b4 = reinterpret_cast<const float4*>(b + c0);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float4 bl = b4[2 * h], bh = b4[2 * h + 1];
      uint4 u;
      u.x = add_relu_pack2<H16>(v[8 * h], v[8 * h + 1], bl.x, bl.y);
      u.y = add_relu_pack2<H16>(v[8 * h + 2], v[8 * h + 3], bl.z, bl.w);
      u.z = add_relu_pack2<H16>(v[8 * h + 4], v[8 * h + 5], bh.x, bh.y);
      u.w = add_relu_pack2<H16>(v[8 * h + 6], v[8 * h + 7], bh.z, bh.w);
      *reinterpret_cast<uint4*>(H + kmaj(r, c0 + 8 * h, 64)) = u;
    }
  }
}

__device__ __forceinline__ void cam_center(const CamDev& c, float pc[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) pc[i] = -(c.R[i] * c.t[0] + c.R[3 + i] * c.t[1] + c.R[6 + i] * c.t[2]);
}

// dX-type product D[128 x N] = dZ[128 x K] W[K x N]: dZ a K-major tile of K
// columns, W the forward weight tile (rows = K outputs, columns = N inputs)
// read as an MN-major B operand.
template <int N, int K>
__device__ __forceinline__ void gemm_dx(uint32_t d, const uint8_t* dZ, const uint8_t* W, bool acc) {
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = sdesc(saddr(dZ) + ks * 256, 128, (K / 8) * 128);
    const uint64_t db = sdesc(saddr(W) + ks * 2 * (N / 8) * 128, (N / 8) * 128, 128);
    mma(d, da, db, idesc<N, false, true>(), (acc || ks > 0) ? 1u : 0u);
  }
}

// As gemm_dx, with dZ stored with AP >= K columns per row.
template <int N, int K, int AP>
__device__ __forceinline__ void gemm_dx_ap(uint32_t d, const uint8_t* dZ, const uint8_t* W) {
  static_assert(AP >= K && AP % 8 == 0, "dZ columns");
#pragma unroll
  for (int ks = 0; ks < K / 16; ++ks) {
    const uint64_t da = sdesc(saddr(dZ) + ks * 256, 128, (AP / 8) * 128);
    const uint64_t db = sdesc(saddr(W) + ks * 2 * (N / 8) * 128, (N / 8) * 128, 128);
    mma(d, da, db, idesc<N, false, true>(), ks > 0 ? 1u : 0u);
  }
}

// Transposed weight-gradient product over the 128 points (rows) of a tile,
// D[128 x N] (+)= A^T dZ: A a point-row tile of AP columns read as an
// MN-major A operand (D row m = column m of A; rows m >= AP read the bytes
// that follow the tile and are never used), dZ a point-row tile of BP >= N
// columns read as an MN-major B operand (its first N columns). With a
// column of ones in A, that row of D is the column sum of dZ.
template <int N, int AP, int BP>
__device__ __forceinline__ void gemm_at(uint32_t d, const uint8_t* A, const uint8_t* dZ, bool acc) {
  static_assert(AP % 8 == 0 && BP % 8 == 0 && BP >= N, "columns");
#pragma unroll
  for (int ks = 0; ks < 128 / 16; ++ks) {
    const uint64_t da = sdesc(saddr(A) + ks * 2 * (AP / 8) * 128, (AP / 8) * 128, 128);
    const uint64_t db = sdesc(saddr(dZ) + ks * 2 * (BP / 8) * 128, (BP / 8) * 128, 128);
    mma(d, da, db, idesc<N, true, true>(), (acc || ks > 0) ? 1u : 0u);
  }
}

// dW-type product D[128 x N] = dZ^T X over the 128 points of a tile: dZ a
// point-row tile with OC columns read as an MN-major A operand (D row o =
// output o; rows >= OC read neighbouring bytes and are never used), X a
// point-row tile with N columns read as an MN-major B operand.
template <int N, int OC>
__device__ __forceinline__ void gemm_dw(uint32_t d, const uint8_t* dZ, const uint8_t* X, bool acc) {
#pragma unroll
  for (int ks = 0; ks < 128 / 16; ++ks) {
    const uint64_t da = sdesc(saddr(dZ) + ks * 2 * (OC / 8) * 128, (OC / 8) * 128, 128);
    const uint64_t db = sdesc(saddr(X) + ks * 2 * (N / 8) * 128, (N / 8) * 128, 128);
    mma(d, da, db, idesc<N, true, true>(), (acc || ks > 0) ? 1u : 0u);
  }
}

// Pixel (i, j): hit point p_s of the ray with the sphere |x| = r in the
// normalised box space (App. A.2, positive root) and the unit ray direction.
__device__ __forceinline__ void bg_ray(const CamDev& c, const FieldsDev& F, float radius, int i, int j,
                                       float ps[3], float dirw[3]) {
  float oc[3];
  cam_center(c, oc);
  const float dc[3] = {((float)i + 0.5f - c.cx) / c.fx, ((float)j + 0.5f - c.cy) / c.fy, 1.0f};
  float on[3], dn[3], dw[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    dw[k] = c.R[k] * dc[0] + c.R[3 + k] * dc[1] + c.R[6 + k] * dc[2];
    on[k] = (oc[k] - F.lo[k]) * F.sx[k] - 1.0f;
    dn[k] = dw[k] * F.sx[k];
  }
  const float A = dn[0] * dn[0] + dn[1] * dn[1] + dn[2] * dn[2];
  const float B = 2.0f * (on[0] * dn[0] + on[1] * dn[1] + on[2] * dn[2]);
  const float C = on[0] * on[0] + on[1] * on[1] + on[2] * on[2] - radius * radius;
  const float tt = (-B + sqrtf(B * B - 4.0f * A * C)) / (2.0f * A);
#pragma unroll
  for (int k = 0; k < 3; ++k) ps[k] = on[k] + tt * dn[k];
  const float nd = sqrtf(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
#pragma unroll
  for (int k = 0; k < 3; ++k) dirw[k] = dw[k] / nd;
}

}  // namespace tc
}  // namespace hyrf
