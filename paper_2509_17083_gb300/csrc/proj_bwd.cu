// Reverse of the EWA projection: dL/d(mean2d, conic) -> dL/d(p, s, q).
// conic = (c, -b, a) / det of Sigma' = [[a, b], [b, c]], det = a c - b^2;
// Sigma' = T Sigma T^T + 0.3 I with T = J R; Sigma = M M^T, M = R_q diag(s);
// J is the perspective Jacobian with the tangent clamped (the clamped
// coordinate passes no gradient). For near-singular Sigma'
// (|det| < 1e-2 a c) the derivative of the inverse is taken in FP64.
#include "common.cuh"

namespace hyrf {

__device__ __noinline__ void conic_grad_fp64(const float T0[3], const float T1[3], const float S[9],
                                             float gA, float gB, float gC, float out[3]) {
  double a = 0.3, b = 0.0, c = 0.3;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a += (double)T0[i] * S[3 * i + j] * T0[j];
      b += (double)T0[i] * S[3 * i + j] * T1[j];
      c += (double)T1[i] * S[3 * i + j] * T1[j];
    }
  const double det = a * c - b * b, d2 = det * det;
  out[0] = (float)(gA * (-c * c / d2) + gB * (b * c / d2) + gC * (-b * b / d2));
  out[1] = (float)(gA * (2 * b * c / d2) + gB * (-1.0 / det - 2 * b * b / d2) + gC * (2 * a * b / d2));
  out[2] = (float)(gA * (-b * b / d2) + gB * (b * a / d2) + gC * (-a * a / d2));
}

__global__ void __launch_bounds__(256) k_project_bwd(CamDev cam, int n, const float* __restrict__ pos,
                                                     const int32_t* __restrict__ vis_ids,
                                                     const int32_t* __restrict__ n_vis,
                                                     const float* __restrict__ scale,
                                                     const float* __restrict__ quat,
                                                     const float* __restrict__ d_mean2d,
                                                     const float* __restrict__ d_conic,
                                                     float* __restrict__ d_pos,
                                                     float* __restrict__ d_scale,
                                                     float* __restrict__ d_quat, int32_t* status) {
  const int nv = min(*n_vis, n);
  const float* R = cam.R;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += gridDim.x * blockDim.x) {
    const int g = vis_ids[i];
    if (g < 0 || g >= n) {
      set_status(status, HYRF_ERR_BOUNDS);
      continue;
    }
    const float p[3] = {pos[3 * (int64_t)g], pos[3 * (int64_t)g + 1], pos[3 * (int64_t)g + 2]};
    const float s[3] = {scale[3 * i], scale[3 * i + 1], scale[3 * i + 2]};
    const float q[4] = {quat[4 * i], quat[4 * i + 1], quat[4 * i + 2], quat[4 * i + 3]};
    float tc[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) tc[k] = R[3 * k] * p[0] + R[3 * k + 1] * p[1] + R[3 * k + 2] * p[2] + cam.t[k];
    const float x = tc[0], y = tc[1], z = tc[2];
    const float fx = cam.fx, fy = cam.fy;
    const float limx = 1.3f * (0.5f * (float)cam.W / fx), limy = 1.3f * (0.5f * (float)cam.H / fy);
    const float rx = x / z, ry = y / z;
    const bool clx = rx < -limx || rx > limx, cly = ry < -limy || ry > limy;
    const float mx = fminf(limx, fmaxf(-limx, rx)), my = fminf(limy, fmaxf(-limy, ry));
    const float J00 = fx / z, J02 = -fx * mx / z, J11 = fy / z, J12 = -fy * my / z;
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      T0[k] = J00 * R[k] + J02 * R[6 + k];
      T1[k] = J11 * R[3 + k] + J12 * R[6 + k];
    }
    const float w = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float Rq[9] = {1.f - 2.f * (qy * qy + qz * qz), 2.f * (qx * qy - w * qz), 2.f * (qx * qz + w * qy),
                         2.f * (qx * qy + w * qz), 1.f - 2.f * (qx * qx + qz * qz), 2.f * (qy * qz - w * qx),
                         2.f * (qx * qz - w * qy), 2.f * (qy * qz + w * qx), 1.f - 2.f * (qx * qx + qy * qy)};
    float M[9], S[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int k = 0; k < 3; ++k) M[3 * a + k] = Rq[3 * a + k] * s[k];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
    float ST0[3], ST1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      ST0[k] = S[3 * k] * T0[0] + S[3 * k + 1] * T0[1] + S[3 * k + 2] * T0[2];
      ST1[k] = S[3 * k] * T1[0] + S[3 * k + 1] * T1[1] + S[3 * k + 2] * T1[2];
    }
    const float a = T0[0] * ST0[0] + T0[1] * ST0[1] + T0[2] * ST0[2] + 0.3f;
    const float b = T1[0] * ST0[0] + T1[1] * ST0[1] + T1[2] * ST0[2];
    const float c = T1[0] * ST1[0] + T1[1] * ST1[1] + T1[2] * ST1[2] + 0.3f;
    const float det = a * c - b * b;
    const float gA = d_conic[3 * i], gB = d_conic[3 * i + 1], gC = d_conic[3 * i + 2];
    float dabc[3];
    if (fabsf(det) < 1e-2f * a * c) {
      conic_grad_fp64(T0, T1, S, gA, gB, gC, dabc);
    } else {
      const float id = 1.0f / det, id2 = id * id;
      dabc[0] = (-gA * c * c + gB * b * c - gC * b * b) * id2;
      dabc[1] = (2.f * gA * b * c - 2.f * gB * b * b + 2.f * gC * a * b) * id2 - gB * id;
      dabc[2] = (-gA * b * b + gB * a * b - gC * a * a) * id2;
    }
    const float da = dabc[0], db = dabc[1], dc = dabc[2];
    // Sigma gradient (full, non-symmetric) and dT.
    float GS[9];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int v = 0; v < 3; ++v) GS[3 * u + v] = da * T0[u] * T0[v] + db * T0[u] * T1[v] + dc * T1[u] * T1[v];
    float dT0[3], dT1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      dT0[k] = 2.f * da * ST0[k] + db * ST1[k];
      dT1[k] = db * ST0[k] + 2.f * dc * ST1[k];
    }
    // T = J R
    const float dJ00 = dT0[0] * R[0] + dT0[1] * R[1] + dT0[2] * R[2];
    const float dJ02 = dT0[0] * R[6] + dT0[1] * R[7] + dT0[2] * R[8];
    const float dJ11 = dT1[0] * R[3] + dT1[1] * R[4] + dT1[2] * R[5];
    const float dJ12 = dT1[0] * R[6] + dT1[1] * R[7] + dT1[2] * R[8];
    // Sigma = M M^T, M = Rq diag(s)
    float dM[9];
#pragma unroll
    for (int u = 0; u < 3; ++u)
#pragma unroll
      for (int k = 0; k < 3; ++k)
        dM[3 * u + k] = (GS[3 * u] + GS[u]) * M[k] + (GS[3 * u + 1] + GS[3 + u]) * M[3 + k] +
                        (GS[3 * u + 2] + GS[6 + u]) * M[6 + k];
#pragma unroll
    for (int k = 0; k < 3; ++k) d_scale[3 * i + k] = Rq[k] * dM[k] + Rq[3 + k] * dM[3 + k] + Rq[6 + k] * dM[6 + k];
    float dR[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) dR[e] = dM[e] * s[e % 3];
    // d Rq / d (w, x, y, z)
    d_quat[4 * i] = 2.f * (-qz * dR[1] + qy * dR[2] + qz * dR[3] - qx * dR[5] - qy * dR[6] + qx * dR[7]);
    d_quat[4 * i + 1] = 2.f * (qy * dR[1] + qz * dR[2] + qy * dR[3] - 2.f * qx * dR[4] - w * dR[5] +
                               qz * dR[6] + w * dR[7] - 2.f * qx * dR[8]);
    d_quat[4 * i + 2] = 2.f * (-2.f * qy * dR[0] + qx * dR[1] + w * dR[2] + qx * dR[3] + qz * dR[5] -
                               w * dR[6] + qz * dR[7] - 2.f * qy * dR[8]);
    d_quat[4 * i + 3] = 2.f * (-2.f * qz * dR[0] - w * dR[1] + qx * dR[2] + w * dR[3] - 2.f * qz * dR[4] +
                               qy * dR[5] + qx * dR[6] + qy * dR[7]);
    // camera-space point
    const float du = d_mean2d[2 * i], dv = d_mean2d[2 * i + 1];
    const float iz = 1.0f / z, iz2 = iz * iz;
    float gx = du * fx * iz, gy = dv * fy * iz;
    float gz = -(du * fx * x + dv * fy * y) * iz2 - (dJ00 * fx + dJ11 * fy) * iz2;
    const float dmx_dx = clx ? 0.f : iz, dmx_dz = clx ? 0.f : -x * iz2;
    const float dmy_dy = cly ? 0.f : iz, dmy_dz = cly ? 0.f : -y * iz2;
    gx += dJ02 * (-fx * dmx_dx * iz);
    gz += dJ02 * (fx * mx * iz2 - fx * dmx_dz * iz);
    gy += dJ12 * (-fy * dmy_dy * iz);
    gz += dJ12 * (fy * my * iz2 - fy * dmy_dz * iz);
#pragma unroll
    for (int k = 0; k < 3; ++k) d_pos[3 * (int64_t)g + k] += R[k] * gx + R[3 + k] * gy + R[6 + k] * gz;
  }
}

hyrf_status launch_project_bwd(const hyrf_project_backward_args& a, cudaStream_t s) {
  if (a.n == 0) return HYRF_OK;
  int blocks = (a.n + 255) / 256;
  if (blocks > num_sms() * 8) blocks = num_sms() * 8;
  HYRF_LAUNCH("k_project_bwd", s,
              k_project_bwd<<<blocks, 256, 0, s>>>(to_dev(a.cam), a.n, a.pos, a.vis_ids, a.n_vis, a.scale,
                                       a.quat, a.d_mean2d, a.d_conic, a.d_pos, a.d_scale,
                                       a.d_quat, a.status));
  return HYRF_OK;
}

}  // namespace hyrf
