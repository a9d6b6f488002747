// 8-bit min-max codec of a hash table (the compressed model's grids, Sec.
// 4.4), written from its definition: per level, lo = min, hi = max,
// step = (hi - lo) / 255 and code = rint((x - lo) / step) clamped to
// [0, 255] (0 if step = 0). The range and the codes are float operations
// (FP32 replay, no contraction), so they compare bit for bit; the decoded
// value lo + step * code is returned in FP64. Test infrastructure only.
#include <cmath>

#include "hyrf_oracle.h"

extern "C" int32_t orc_quantize_grid(int32_t n_levels, int64_t per_level, const float* table, uint8_t* codes,
                                     float* qparams, double* decoded) {
  if (n_levels < 1 || per_level < 1) return -1;
  for (int32_t l = 0; l < n_levels; ++l) {
    const float* t = table + (int64_t)l * per_level;
    float lo = t[0], hi = t[0];
    for (int64_t i = 1; i < per_level; ++i) {
      if (t[i] < lo) lo = t[i];
      if (t[i] > hi) hi = t[i];
    }
    const float step = (hi - lo) / 255.0f;
    qparams[2 * l] = lo;
    qparams[2 * l + 1] = step;
    for (int64_t i = 0; i < per_level; ++i) {
      float c = 0.0f;
      if (step > 0.0f) c = std::rint((t[i] - lo) / step);
      c = c < 0.0f ? 0.0f : (c > 255.0f ? 255.0f : c);
      codes[(int64_t)l * per_level + i] = (uint8_t)c;
      if (decoded) decoded[(int64_t)l * per_level + i] = (double)lo + (double)step * (double)c;
    }
  }
  return 0;
}
