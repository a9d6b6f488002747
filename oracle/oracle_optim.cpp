// Adam, written out from its published definition (Kingma & Ba 2015,
// Algorithm 1), in FP64. Test infrastructure only (see hyrf_oracle.h).
#include <cmath>

#include "hyrf_oracle.h"

extern "C" int32_t orc_adam_step(int64_t n, double* p, const double* grad, double* m, double* v, double lr,
                                 double b1, double b2, double eps, int32_t t, double grad_scale) {
  if (n < 0 || t < 1 || !(eps > 0.0)) return -1;
  const double c1 = 1.0 - std::pow(b1, t), c2 = 1.0 - std::pow(b2, t);
  for (int64_t i = 0; i < n; ++i) {
    const double g = grad_scale * grad[i];
    m[i] = b1 * m[i] + (1.0 - b1) * g;
    v[i] = b2 * v[i] + (1.0 - b2) * g * g;
    const double mhat = m[i] / c1, vhat = v[i] / c2;
    p[i] -= lr * mhat / (std::sqrt(vhat) + eps);
  }
  return 0;
}

// ---------------- adaptive density control (3DGS rules, the paper's Sec. 3.3
// end and Sec. 4.1 "as the original 3DGS")

extern "C" int32_t orc_densify_stats(int32_t n, int32_t n_vis, const int32_t* vis_ids, const float* d_mean2d,
                                     const int32_t* ntiles, int32_t width, int32_t height, float* accum,
                                     int32_t* count) {
  if (n < 0 || n_vis < 0 || n_vis > n) return -1;
  const float hw = 0.5f * (float)width, hh = 0.5f * (float)height;
  for (int32_t i = 0; i < n_vis; ++i) {
    if (ntiles[i] <= 0) continue;
    const int32_t g = vis_ids[i];
    if (g < 0 || g >= n) return -2;
    const float gx = d_mean2d[2 * i] * hw, gy = d_mean2d[2 * i + 1] * hh;
    const float sq = gx * gx + gy * gy;  // each operation rounded to float (no contraction)
    accum[g] = accum[g] + std::sqrt(sq);
    count[g] += 1;
  }
  return 0;
}

extern "C" int64_t orc_densify_plan(int32_t n, int32_t n_vis, const int32_t* vis_ids, const float* alpha,
                                    const float* scale, const float* accum, const int32_t* count,
                                    float grad_threshold, float dense_scale, float min_opacity, uint8_t* action,
                                    int32_t* row, int64_t* offset) {
  if (n < 0 || n_vis < 0 || n_vis > n) return -1;
  for (int32_t g = 0; g < n; ++g) row[g] = -1;
  for (int32_t i = 0; i < n_vis; ++i) row[vis_ids[i]] = i;
  int64_t total = 0;
  for (int32_t g = 0; g < n; ++g) {
    uint8_t act = 0;  // keep
    const int32_t r = row[g];
    if (r >= 0) {
      if (alpha[r] < min_opacity) {
        act = 1;  // prune
      } else if (count[g] > 0 && accum[g] / (float)count[g] >= grad_threshold) {
        float s = scale[3 * r];
        if (scale[3 * r + 1] > s) s = scale[3 * r + 1];
        if (scale[3 * r + 2] > s) s = scale[3 * r + 2];
        act = s > dense_scale ? 3 : 2;  // split : clone
      }
    }
    action[g] = act;
    offset[g] = total;
    total += act == 1 ? 0 : (act == 0 ? 1 : 2);
  }
  offset[n] = total;
  return total;
}

extern "C" int32_t orc_densify_apply(int32_t n, const uint8_t* action, const int32_t* row, const int64_t* offset,
                                     const double* scale, const double* quat, const double* noise,
                                     double split_log_scale, int32_t width, int32_t kind, const double* src,
                                     double* dst) {
  if (n < 0 || width < 1) return -1;
  for (int32_t g = 0; g < n; ++g) {
    const int act = action[g];
    if (act == 1) continue;
    double* d0 = dst + offset[g] * width;
    const double* s = src + (int64_t)g * width;
    if (act == 0) {
      for (int c = 0; c < width; ++c) d0[c] = s[c];
      continue;
    }
    double* d1 = d0 + width;
    if (act == 2) {  // clone: the original, then a copy (new optimiser state)
      for (int c = 0; c < width; ++c) {
        d0[c] = s[c];
        d1[c] = kind == 1 ? 0.0 : s[c];
      }
      continue;
    }
    // split: two new Gaussians
    if (kind == 1) {
      for (int c = 0; c < width; ++c) d0[c] = d1[c] = 0.0;
    } else if (kind == 2) {
      const int32_t r = row[g];
      const double* q = quat + 4 * (int64_t)r;
      const double w = q[0], x = q[1], y = q[2], z = q[3];
      const double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                           2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                           2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
      for (int k = 0; k < 2; ++k) {
        double u[3];
        for (int j = 0; j < 3; ++j) u[j] = scale[3 * (int64_t)r + j] * noise[6 * (int64_t)g + 3 * k + j];
        double* d = k == 0 ? d0 : d1;
        for (int i = 0; i < 3; ++i) d[i] = s[i] + R[3 * i] * u[0] + R[3 * i + 1] * u[1] + R[3 * i + 2] * u[2];
      }
    } else if (kind == 3) {
      d0[0] = d1[0] = s[0] - split_log_scale;
    } else {
      for (int c = 0; c < width; ++c) d0[c] = d1[c] = s[c];
    }
  }
  return 0;
}
