// Internal declarations shared by the two oracle translation units.
// Test infrastructure only (see hyrf_oracle.h).
#ifndef HYRF_ORACLE_INTERNAL_H
#define HYRF_ORACLE_INTERNAL_H
#include <vector>

#include "hyrf_oracle.h"

namespace orc {
void contract_point(const orc_aabb& box, const double p[3], double y[3], double J[9]);
int level_res(const orc_grid& g, int l);
uint32_t level_index(const orc_grid& g, int l, uint32_t ix, uint32_t iy, uint32_t iz);
void hash_encode(const orc_grid& g, const double y[3], double* f);
void hash_encode_backward(const orc_grid& g, const double y[3], const double* df,
                          double* d_table, double dy[3]);
void mlp_forward(const orc_mlp& m, const double* x, double* y);
void mlp_backward(const orc_mlp& m, const double* x, const double* dy, const orc_mlp_grad* grad,
                  double* dx);
void pos_enc(const double d[3], int n_freq, double* out);
void camera_center(const orc_camera& cam, double c[3]);
void bg_color(const orc_fields& fl, const double y[3], const double dir[3], double c[3]);
double bg_margin(const orc_fields& fl, const double y[3], const double dir[3]);
void bg_color_backward(const orc_fields& fl, const double y[3], const double dir[3],
                       const double dc[3], double* d_rad_table, const orc_mlp_grad* d_col);
}  // namespace orc
#endif
