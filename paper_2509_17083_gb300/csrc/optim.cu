// Fused multi-tensor Adam (hyrf_adam_step): every tensor of the model in one
// launch. A CTA owns a 4096-element block of one tensor; the block table is
// laid out on the host and passed by value. Elements are processed as float4
// where the whole vector is inside the tensor.
#include "common.cuh"

namespace hyrf {

constexpr int kAdamBlock = 4096;

struct AdamLaunch {
  hyrf_adam_tensor t[HYRF_ADAM_MAX_TENSORS];
  int64_t first_block[HYRF_ADAM_MAX_TENSORS + 1];  // prefix of blocks per tensor
  int count;
  float lr, b1, b2, omb1, omb2, eps, c1, c2, gs;    // omb = 1 - b; c1 = 1 - b1^t, c2 = 1 - b2^t
};

__device__ __forceinline__ float adam_one(float& p, float g, float& m, float& v, const AdamLaunch& A,
                                          float lr) {
  g *= A.gs;
  m = A.b1 * m + A.omb1 * g;
  v = A.b2 * v + A.omb2 * g * g;
  const float mh = m / A.c1, vh = v / A.c2;
  p -= lr * mh / (sqrtf(vh) + A.eps);
  return p;
}

__global__ void __launch_bounds__(256) k_adam(const AdamLaunch A) {
  const int64_t b = blockIdx.x;
  int k = 0;
  while (k + 1 < A.count && A.first_block[k + 1] <= b) ++k;
  const hyrf_adam_tensor& T = A.t[k];
  const int64_t e0 = (b - A.first_block[k]) * kAdamBlock;
  const int64_t e1 = e0 + kAdamBlock < T.n ? e0 + kAdamBlock : T.n;
  const float lr = A.lr * T.lr_scale;
  __nv_bfloat16* sh = static_cast<__nv_bfloat16*>(T.shadow);
  for (int64_t e = e0 + 4 * threadIdx.x; e < e1; e += 4 * blockDim.x) {
    if (e + 4 <= e1) {
      float4 p = *reinterpret_cast<float4*>(T.param + e);
      const float4 g = *reinterpret_cast<const float4*>(T.grad + e);
      float4 m = *reinterpret_cast<float4*>(T.m + e);
      float4 v = *reinterpret_cast<float4*>(T.v + e);
      adam_one(p.x, g.x, m.x, v.x, A, lr);
      adam_one(p.y, g.y, m.y, v.y, A, lr);
      adam_one(p.z, g.z, m.z, v.z, A, lr);
      adam_one(p.w, g.w, m.w, v.w, A, lr);
      *reinterpret_cast<float4*>(T.param + e) = p;
      *reinterpret_cast<float4*>(T.m + e) = m;
      *reinterpret_cast<float4*>(T.v + e) = v;
      if (sh) {
        *reinterpret_cast<__nv_bfloat162*>(sh + e) = __floats2bfloat162_rn(p.x, p.y);
        *reinterpret_cast<__nv_bfloat162*>(sh + e + 2) = __floats2bfloat162_rn(p.z, p.w);
      }
    } else {
      for (int64_t i = e; i < e1; ++i) {
        float p = T.param[i], m = T.m[i], v = T.v[i];
        adam_one(p, T.grad[i], m, v, A, lr);
        T.param[i] = p;
        T.m[i] = m;
        T.v[i] = v;
        if (sh) sh[i] = __float2bfloat16_rn(p);
      }
    }
  }
}

}  // namespace hyrf

using namespace hyrf;

extern "C" hyrf_status hyrf_adam_step(const hyrf_adam_tensor* tensors, int32_t count,
                                      const hyrf_adam_hparams* hp, void* stream) {
  if (!tensors || !hp || count < 0 || count > HYRF_ADAM_MAX_TENSORS) return HYRF_ERR_INVALID_ARG;
  if (hp->step < 1 || !(hp->beta1 >= 0.0f && hp->beta1 < 1.0f) || !(hp->beta2 >= 0.0f && hp->beta2 < 1.0f) ||
      !(hp->eps > 0.0f) || !(hp->lr >= 0.0f))
    return HYRF_ERR_INVALID_ARG;
  AdamLaunch A{};
  A.lr = hp->lr;
  A.b1 = hp->beta1;
  A.b2 = hp->beta2;
  A.eps = hp->eps;
  A.gs = hp->grad_scale;
  A.omb1 = (float)(1.0 - (double)hp->beta1);  // exact difference, then one rounding
  A.omb2 = (float)(1.0 - (double)hp->beta2);
  A.c1 = (float)(1.0 - pow((double)hp->beta1, (double)hp->step));
  A.c2 = (float)(1.0 - pow((double)hp->beta2, (double)hp->step));
  int64_t blocks = 0;
  int k = 0;
  for (int i = 0; i < count; ++i) {
    const hyrf_adam_tensor& t = tensors[i];
    if (t.n < 0) return HYRF_ERR_INVALID_ARG;
    if (t.n == 0) continue;
    auto al = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
    if (!t.param || !t.grad || !t.m || !t.v || !al(t.param) || !al(t.grad) || !al(t.m) || !al(t.v) ||
        (t.shadow && (reinterpret_cast<uintptr_t>(t.shadow) & 7u) != 0))
      return HYRF_ERR_INVALID_ARG;
    A.t[k] = t;
    A.first_block[k] = blocks;
    blocks += (t.n + kAdamBlock - 1) / kAdamBlock;
    ++k;
  }
  A.count = k;
  A.first_block[k] = blocks;
  if (blocks == 0) return HYRF_OK;
  if (blocks > 0x7fffffff) return HYRF_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  HYRF_LAUNCH("k_adam", s, k_adam<<<(unsigned)blocks, 256, 0, s>>>(A));
  return HYRF_OK;
}
