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
