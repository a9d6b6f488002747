// HyRF oracle, part 1: neural fields (Sec. 3.2, Eqs. 2-7; App. A.1).
// Test infrastructure only (see hyrf_oracle.h). Plain FP64, one point at a time.
#include "oracle_internal.h"

#include <atomic>
#include <cmath>
#include <cstring>
#include <vector>

namespace orc {

// App. A.1: the box B0 is mapped affinely onto [-1, 1]^3 (the printed
// "p / B0" read as this affine map). Eq. 2 / Eq. A2 then contract to (0, 1)
// with the offset read as +0.5 (the printed +1 contradicts the stated range).
void contract_point(const orc_aabb& box, const double p[3], double y[3], double J[9]) {
  double x[3], sx[3];
  for (int k = 0; k < 3; ++k) {
    sx[k] = 2.0 / (box.hi[k] - box.lo[k]);
    x[k] = (p[k] - box.lo[k]) * sx[k] - 1.0;
  }
  double n = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double Jx[9];
  if (n <= 1.0) {
    for (int k = 0; k < 3; ++k) y[k] = 0.25 * x[k] + 0.5;
    for (int i = 0; i < 9; ++i) Jx[i] = (i % 4 == 0) ? 0.25 : 0.0;
  } else {
    // y = 0.25 * (2 - 1/n) * x / n + 0.5 = 0.25 * g(n) * x + 0.5, g(n) = 2/n - 1/n^2
    double g = 2.0 / n - 1.0 / (n * n);
    double gp = -2.0 / (n * n) + 2.0 / (n * n * n);  // dg/dn
    for (int k = 0; k < 3; ++k) y[k] = 0.25 * g * x[k] + 0.5;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        Jx[i * 3 + j] = 0.25 * ((i == j ? g : 0.0) + gp * x[i] * x[j] / n);
  }
  if (J) {
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) J[i * 3 + j] = Jx[i * 3 + j] * sx[j];
  }
}

int level_res(const orc_grid& g, int l) {
  return (int)std::floor((double)g.base_res * std::pow(g.growth, (double)l));
}

// Eq. 3 (Instant-NGP): a level is stored densely when its (N+1)^3 vertices fit
// in the table, otherwise vertices are hashed with the spatial hash of
// Instant-NGP (XOR of coordinates times the primes 1, 2654435761, 805459861,
// in 32-bit wrap-around arithmetic) modulo the table size.
uint32_t level_index(const orc_grid& g, int l, uint32_t ix, uint32_t iy, uint32_t iz) {
  const uint64_t T = 1ull << g.log2_T;
  const uint64_t n1 = (uint64_t)level_res(g, l) + 1;
  if (n1 * n1 * n1 <= T) return (uint32_t)(ix + iy * n1 + iz * n1 * n1);
  uint32_t h = ix * 1u;
  h ^= iy * 2654435761u;
  h ^= iz * 805459861u;
  return (uint32_t)(h & (uint32_t)(T - 1));
}

// Trilinear interpolation cell of one level: corners c = 0..7 with bit 0 = x,
// bit 1 = y, bit 2 = z; weights w[c] and dw[c][d] = d w[c] / d u_d.
struct Cell {
  uint32_t idx[8];
  double w[8];
  double dw[8][3];
  int res;
};

static void level_cell(const orc_grid& g, int l, const double y[3], Cell& cell) {
  int N = level_res(g, l);
  cell.res = N;
  int i0[3];
  double f[3];
  for (int d = 0; d < 3; ++d) {
    double u = y[d] * (double)N;
    double fl = std::floor(u);
    if (fl < 0.0) fl = 0.0;
    if (fl > (double)(N - 1)) fl = (double)(N - 1);
    i0[d] = (int)fl;
    f[d] = u - fl;
  }
  for (int c = 0; c < 8; ++c) {
    int b[3] = {c & 1, (c >> 1) & 1, (c >> 2) & 1};
    double wd[3];
    for (int d = 0; d < 3; ++d) wd[d] = b[d] ? f[d] : 1.0 - f[d];
    cell.w[c] = wd[0] * wd[1] * wd[2];
    for (int d = 0; d < 3; ++d) {
      double s = b[d] ? 1.0 : -1.0;
      double prod = 1.0;
      for (int e = 0; e < 3; ++e)
        if (e != d) prod *= wd[e];
      cell.dw[c][d] = s * prod;
    }
    cell.idx[c] = level_index(g, l, (uint32_t)(i0[0] + b[0]), (uint32_t)(i0[1] + b[1]),
                              (uint32_t)(i0[2] + b[2]));
  }
}

void hash_encode(const orc_grid& g, const double y[3], double* f) {
  const size_t T = (size_t)1 << g.log2_T;
  for (int l = 0; l < g.n_levels; ++l) {
    Cell cell;
    level_cell(g, l, y, cell);
    for (int k = 0; k < g.n_feat; ++k) {
      double acc = 0.0;
      for (int c = 0; c < 8; ++c)
        acc += cell.w[c] * g.table[((size_t)l * T + cell.idx[c]) * g.n_feat + k];
      f[l * g.n_feat + k] = acc;
    }
  }
}

// Reverse of hash_encode: table gradient (accumulated) and dL/dy (accumulated).
void hash_encode_backward(const orc_grid& g, const double y[3], const double* df,
                          double* d_table, double dy[3]) {
  const size_t T = (size_t)1 << g.log2_T;
  for (int l = 0; l < g.n_levels; ++l) {
    Cell cell;
    level_cell(g, l, y, cell);
    for (int c = 0; c < 8; ++c) {
      double dot = 0.0;
      for (int k = 0; k < g.n_feat; ++k) {
        size_t e = ((size_t)l * T + cell.idx[c]) * g.n_feat + k;
        if (d_table) d_table[e] += cell.w[c] * df[l * g.n_feat + k];
        dot += g.table[e] * df[l * g.n_feat + k];
      }
      if (dy)
        for (int d = 0; d < 3; ++d) dy[d] += dot * cell.dw[c][d] * (double)cell.res;
    }
  }
}

// Layer sizes of the decoder (Sec. 4.1: hidden ReLU layers, linear output).
static void layer_dims(const orc_mlp& m, int l, int& n_out, int& n_in) {
  n_in = (l == 0) ? m.n_in : m.width;
  n_out = (l == m.n_hidden) ? m.n_out : m.width;
}

// Round to the nearest bfloat16 through float (ties to even), as a kernel
// that converts its FP32 values to bfloat16 does.
static double to_bf16(double v) {
  float f = (float)v;
  uint32_t u;
  std::memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0x7fffu + ((u >> 16) & 1u)) & 0xffff0000u;
  std::memcpy(&f, &u, 4);
  return f;
}

// Sum of the branch-pattern mixes of every decoder evaluation (see
// orc_branch_sum); atomic so that evaluations on several threads add up.
static std::atomic<uint64_t> g_branch_sum{0};

// splitmix64 finaliser: a 64-bit mix of the pattern's running hash.
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

// ReLU branches of the hidden units for input x: on[l][o] = 1 where unit o of
// hidden layer l is active, decided in the precision m.relu_replay selects
// (see hyrf_oracle.h). Returns the smallest relative margin
// min |z| / (sum_i |W_i a_i| + |b|) of the pre-activations decided on.
static double relu_branches(const orc_mlp& m, const double* x, std::vector<std::vector<char>>& on) {
  const bool rep = m.relu_replay == 1;
  std::vector<double> a(x, x + m.n_in), next;
  if (rep)
    for (double& v : a) v = to_bf16(v);
  double mg = 1e300;
  on.assign(m.n_hidden, {});
  for (int l = 0; l < m.n_hidden; ++l) {
    int no, ni;
    layer_dims(m, l, no, ni);
    next.assign(no, 0.0);
    on[l].assign(no, 0);
    for (int o = 0; o < no; ++o) {
      double z = m.b[l][o], mag = std::fabs(m.b[l][o]);
      for (int i = 0; i < ni; ++i) {
        z += m.W[l][(size_t)o * ni + i] * a[i];
        mag += std::fabs(m.W[l][(size_t)o * ni + i] * a[i]);
      }
      if (mag > 0.0) mg = std::min(mg, std::fabs(z) / mag);
      on[l][o] = z > 0.0;
      double h = z > 0.0 ? z : 0.0;
      next[o] = rep ? to_bf16(h) : h;
    }
    a.swap(next);
  }
  uint64_t h = 0x9e3779b97f4a7c15ull;
  for (const auto& layer : on)
    for (char b : layer) h = mix64(h ^ (uint64_t)(b + 1));
  g_branch_sum.fetch_add(h, std::memory_order_relaxed);
  return mg;
}

static double mlp_margin(const orc_mlp& m, const double* x) {
  std::vector<std::vector<char>> on;
  return relu_branches(m, x, on);
}

// Forward keeping every layer input (acts[l]), pre-activation (pre[l]) and
// ReLU branch (on[l]). The values are FP64; each hidden unit passes its
// pre-activation where its branch is active, else 0 (Sec. 4.1: ReLU hidden
// layers, linear output).
static void mlp_forward_acts(const orc_mlp& m, const double* x,
                             std::vector<std::vector<double>>& acts,
                             std::vector<std::vector<double>>& pre,
                             std::vector<std::vector<char>>& on, double* y) {
  relu_branches(m, x, on);
  acts.assign(m.n_hidden + 1, {});
  pre.assign(m.n_hidden + 1, {});
  acts[0].assign(x, x + m.n_in);
  for (int l = 0; l <= m.n_hidden; ++l) {
    int no, ni;
    layer_dims(m, l, no, ni);
    pre[l].assign(no, 0.0);
    for (int o = 0; o < no; ++o) {
      double s = m.b[l][o];
      for (int i = 0; i < ni; ++i) s += m.W[l][(size_t)o * ni + i] * acts[l][i];
      pre[l][o] = s;
    }
    if (l < m.n_hidden) {
      acts[l + 1].resize(no);
      for (int o = 0; o < no; ++o) acts[l + 1][o] = on[l][o] ? pre[l][o] : 0.0;
    }
  }
  for (int o = 0; o < m.n_out; ++o) y[o] = pre[m.n_hidden][o];
}

void mlp_forward(const orc_mlp& m, const double* x, double* y) {
  std::vector<std::vector<double>> acts, pre;
  std::vector<std::vector<char>> on;
  mlp_forward_acts(m, x, acts, pre, on, y);
}

// Reverse pass: accumulates dW, db (if grad is given) and writes dL/dx.
void mlp_backward(const orc_mlp& m, const double* x, const double* dy, const orc_mlp_grad* grad,
                  double* dx) {
  std::vector<std::vector<double>> acts, pre;
  std::vector<std::vector<char>> on;
  std::vector<double> y(m.n_out);
  mlp_forward_acts(m, x, acts, pre, on, y.data());
  std::vector<double> dz(dy, dy + m.n_out);
  for (int l = m.n_hidden; l >= 0; --l) {
    int no, ni;
    layer_dims(m, l, no, ni);
    if (grad) {
      for (int o = 0; o < no; ++o) {
        grad->b[l][o] += dz[o];
        for (int i = 0; i < ni; ++i) grad->W[l][(size_t)o * ni + i] += dz[o] * acts[l][i];
      }
    }
    std::vector<double> da(ni, 0.0);
    for (int o = 0; o < no; ++o)
      for (int i = 0; i < ni; ++i) da[i] += m.W[l][(size_t)o * ni + i] * dz[o];
    if (l == 0) {
      for (int i = 0; i < ni; ++i) dx[i] = da[i];
    } else {
      // ReLU of hidden layer l-1: derivative 1 on its active branch.
      dz.assign(ni, 0.0);
      for (int i = 0; i < ni; ++i) dz[i] = on[l - 1][i] ? da[i] : 0.0;
    }
  }
}

// Eq. 5: NeRF positional encoding [d, sin(2^k pi d), cos(2^k pi d)] for
// k = 0..n_freq-1 (sin block then cos block per frequency).
void pos_enc(const double d[3], int n_freq, double* out) {
  for (int j = 0; j < 3; ++j) out[j] = d[j];
  for (int k = 0; k < n_freq; ++k) {
    double w = std::ldexp(M_PI, k);
    for (int j = 0; j < 3; ++j) {
      out[3 + 6 * k + j] = std::sin(w * d[j]);
      out[3 + 6 * k + 3 + j] = std::cos(w * d[j]);
    }
  }
}

void pos_enc_backward(const double d[3], int n_freq, const double* dout, double dd[3]) {
  for (int j = 0; j < 3; ++j) dd[j] += dout[j];
  for (int k = 0; k < n_freq; ++k) {
    double w = std::ldexp(M_PI, k);
    for (int j = 0; j < 3; ++j) {
      dd[j] += dout[3 + 6 * k + j] * w * std::cos(w * d[j]);
      dd[j] -= dout[3 + 6 * k + 3 + j] * w * std::sin(w * d[j]);
    }
  }
}

void camera_center(const orc_camera& cam, double c[3]) {
  // x_c = R x_w + t = 0  =>  x_w = -R^T t
  for (int i = 0; i < 3; ++i) {
    c[i] = 0.0;
    for (int k = 0; k < 3; ++k) c[i] -= cam.R[k * 3 + i] * cam.t[k];
  }
}

static double sigmoid(double x) { return 1.0 / (1.0 + std::exp(-x)); }

// Colour-MLP input: [f_rad (L*F), PE(dir) (3 + 6 n_freq), zeros up to pe_pad].
static void color_input(const orc_fields& fl, const double* f_rad, const double dir[3],
                        std::vector<double>& in) {
  int nf = fl.rad.n_levels * fl.rad.n_feat;
  in.assign(fl.col_mlp.n_in, 0.0);
  for (int i = 0; i < nf; ++i) in[i] = f_rad[i];
  pos_enc(dir, fl.pe_freq, in.data() + nf);
}

// Colour of a background point: sigma(dec(enc(y; Theta_rad) (+) PE(dir); Phi_c)).
void bg_color(const orc_fields& fl, const double y[3], const double dir[3], double c[3]) {
  std::vector<double> f(fl.rad.n_levels * fl.rad.n_feat), in;
  hash_encode(fl.rad, y, f.data());
  color_input(fl, f.data(), dir, in);
  double cn[3];
  mlp_forward(fl.col_mlp, in.data(), cn);
  for (int k = 0; k < 3; ++k) c[k] = sigmoid(cn[k]);
}

double bg_margin(const orc_fields& fl, const double y[3], const double dir[3]) {
  std::vector<double> f(fl.rad.n_levels * fl.rad.n_feat), in;
  hash_encode(fl.rad, y, f.data());
  color_input(fl, f.data(), dir, in);
  return mlp_margin(fl.col_mlp, in.data());
}

void bg_color_backward(const orc_fields& fl, const double y[3], const double dir[3],
                       const double dc[3], double* d_rad_table, const orc_mlp_grad* d_col) {
  std::vector<double> f(fl.rad.n_levels * fl.rad.n_feat), in;
  hash_encode(fl.rad, y, f.data());
  color_input(fl, f.data(), dir, in);
  double cn[3], dcn[3];
  mlp_forward(fl.col_mlp, in.data(), cn);
  for (int k = 0; k < 3; ++k) {
    double s = sigmoid(cn[k]);
    dcn[k] = dc[k] * s * (1.0 - s);
  }
  std::vector<double> din(fl.col_mlp.n_in);
  mlp_backward(fl.col_mlp, in.data(), dcn, d_col, din.data());
  hash_encode_backward(fl.rad, y, din.data(), d_rad_table, nullptr);
}

}  // namespace orc

using namespace orc;

extern "C" {

void orc_contract(const orc_aabb* box, const double p[3], double y[3], double J[9]) {
  contract_point(*box, p, y, J);
}

void orc_hash_encode(const orc_grid* g, const double y[3], double* f) { hash_encode(*g, y, f); }

int32_t orc_level_res(const orc_grid* g, int32_t l) { return level_res(*g, l); }

uint32_t orc_level_index(const orc_grid* g, int32_t l, uint32_t ix, uint32_t iy, uint32_t iz) {
  return level_index(*g, l, ix, iy, iz);
}

void orc_mlp_forward(const orc_mlp* m, const double* x, double* y) { mlp_forward(*m, x, y); }

void orc_pos_enc(const double d[3], int32_t n_freq, double* out) { pos_enc(d, n_freq, out); }

void orc_branch_sum_reset(void) { g_branch_sum.store(0); }

uint64_t orc_branch_sum(void) { return g_branch_sum.load(); }

static bool fields_ok(const orc_fields* fl) {
  if (!fl) return false;
  int ng = fl->geo.n_levels * fl->geo.n_feat;
  int nr = fl->rad.n_levels * fl->rad.n_feat;
  if (fl->geo_mlp.n_in != ng || fl->geo_mlp.n_out != 8) return false;
  if (fl->pe_pad < 3 + 6 * fl->pe_freq) return false;
  if (fl->col_mlp.n_in != nr + fl->pe_pad || fl->col_mlp.n_out != 3) return false;
  return true;
}

int32_t orc_decoder_margins(int32_t n, const double* pos, const orc_camera* cam,
                            const orc_fields* fl, double* margin_geo, double* margin_col) {
  if (!fields_ok(fl) || n < 0) return -1;
  double pc[3];
  camera_center(*cam, pc);
  std::vector<double> fg(fl->geo.n_levels * fl->geo.n_feat), fr(fl->rad.n_levels * fl->rad.n_feat), in;
  for (int i = 0; i < n; ++i) {
    const double* p = pos + 3 * i;
    double y[3];
    contract_point(fl->box, p, y, nullptr);
    hash_encode(fl->geo, y, fg.data());
    hash_encode(fl->rad, y, fr.data());
    double v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
    double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double dir[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
    color_input(*fl, fr.data(), dir, in);
    margin_geo[i] = mlp_margin(fl->geo_mlp, fg.data());
    margin_col[i] = mlp_margin(fl->col_mlp, in.data());
  }
  return 0;
}

// Eqs. 3-7 for n visible Gaussians.
int32_t orc_query_fields(int32_t n, const double* pos, const double* alpha_e,
                         const double* scale_e, const double* color_e, const orc_camera* cam,
                         const orc_fields* fl, double* alpha, double* scale, double* quat,
                         double* color) {
  if (!fields_ok(fl) || n < 0) return -1;
  double pc[3];
  camera_center(*cam, pc);
  std::vector<double> fg(fl->geo.n_levels * fl->geo.n_feat), fr(fl->rad.n_levels * fl->rad.n_feat);
  std::vector<double> in;
  for (int i = 0; i < n; ++i) {
    const double* p = pos + 3 * i;
    double y[3];
    contract_point(fl->box, p, y, nullptr);
    hash_encode(fl->geo, y, fg.data());
    hash_encode(fl->rad, y, fr.data());
    double g[8];
    mlp_forward(fl->geo_mlp, fg.data(), g);  // (alpha_n, s_n[3], r_n[4]), raw (Eq. 4)
    double v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
    double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double dir[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
    color_input(*fl, fr.data(), dir, in);
    double cn[3];
    mlp_forward(fl->col_mlp, in.data(), cn);  // Eq. 6, raw
    // Eq. 7 aggregation.
    alpha[i] = sigmoid(g[0] + alpha_e[i]);
    for (int k = 0; k < 3; ++k) scale[3 * i + k] = sigmoid(g[1 + k] + scale_e[i]);
    double rn = std::sqrt(g[4] * g[4] + g[5] * g[5] + g[6] * g[6] + g[7] * g[7]);
    double den = rn > 1e-12 ? rn : 1e-12;
    for (int k = 0; k < 4; ++k) quat[4 * i + k] = g[4 + k] / den;
    for (int k = 0; k < 3; ++k) color[3 * i + k] = sigmoid(cn[k] + color_e[3 * i + k]);
  }
  return 0;
}

int32_t orc_query_fields_backward(int32_t n, const double* pos, const double* alpha_e,
                                  const double* scale_e, const double* color_e,
                                  const orc_camera* cam, const orc_fields* fl,
                                  const double* d_alpha, const double* d_scale,
                                  const double* d_quat, const double* d_color, double* d_pos,
                                  double* d_alpha_e, double* d_scale_e, double* d_color_e,
                                  double* d_geo_table, double* d_rad_table,
                                  const orc_mlp_grad* d_geo_mlp, const orc_mlp_grad* d_col_mlp) {
  if (!fields_ok(fl) || n < 0) return -1;
  double pc[3];
  camera_center(*cam, pc);
  const int ng = fl->geo.n_levels * fl->geo.n_feat, nr = fl->rad.n_levels * fl->rad.n_feat;
  std::vector<double> fg(ng), fr(nr), in, dfg(ng), din(fl->col_mlp.n_in);
  for (int i = 0; i < n; ++i) {
    const double* p = pos + 3 * i;
    double y[3], J[9];
    contract_point(fl->box, p, y, J);
    hash_encode(fl->geo, y, fg.data());
    hash_encode(fl->rad, y, fr.data());
    double g[8];
    mlp_forward(fl->geo_mlp, fg.data(), g);
    double v[3] = {p[0] - pc[0], p[1] - pc[1], p[2] - pc[2]};
    double nv = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    double dir[3] = {v[0] / nv, v[1] / nv, v[2] / nv};
    color_input(*fl, fr.data(), dir, in);
    double cn[3];
    mlp_forward(fl->col_mlp, in.data(), cn);

    // Reverse of Eq. 7.
    double dg[8], dcn[3];
    double a = sigmoid(g[0] + alpha_e[i]);
    dg[0] = d_alpha[i] * a * (1.0 - a);
    d_alpha_e[i] += dg[0];
    for (int k = 0; k < 3; ++k) {
      double s = sigmoid(g[1 + k] + scale_e[i]);
      dg[1 + k] = d_scale[3 * i + k] * s * (1.0 - s);
      d_scale_e[i] += dg[1 + k];
    }
    double rn = std::sqrt(g[4] * g[4] + g[5] * g[5] + g[6] * g[6] + g[7] * g[7]);
    if (rn > 1e-12) {
      double q[4], qd = 0.0;
      for (int k = 0; k < 4; ++k) {
        q[k] = g[4 + k] / rn;
        qd += q[k] * d_quat[4 * i + k];
      }
      for (int k = 0; k < 4; ++k) dg[4 + k] = (d_quat[4 * i + k] - q[k] * qd) / rn;
    } else {
      for (int k = 0; k < 4; ++k) dg[4 + k] = d_quat[4 * i + k] / 1e-12;
    }
    for (int k = 0; k < 3; ++k) {
      double c = sigmoid(cn[k] + color_e[3 * i + k]);
      dcn[k] = d_color[3 * i + k] * c * (1.0 - c);
      d_color_e[3 * i + k] += dcn[k];
    }
    // Decoders, then encodings.
    mlp_backward(fl->geo_mlp, fg.data(), dg, d_geo_mlp, dfg.data());
    mlp_backward(fl->col_mlp, in.data(), dcn, d_col_mlp, din.data());
    double dy[3] = {0, 0, 0};
    hash_encode_backward(fl->geo, y, dfg.data(), d_geo_table, dy);
    hash_encode_backward(fl->rad, y, din.data(), d_rad_table, dy);
    double dp[3] = {0, 0, 0};
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) dp[j] += J[k * 3 + j] * dy[k];
    // View direction (Eq. 5): dir = v / |v|.
    double ddir[3] = {0, 0, 0};
    pos_enc_backward(dir, fl->pe_freq, din.data() + nr, ddir);
    double dd = dir[0] * ddir[0] + dir[1] * ddir[1] + dir[2] * ddir[2];
    for (int k = 0; k < 3; ++k) dp[k] += (ddir[k] - dir[k] * dd) / nv;
    for (int k = 0; k < 3; ++k) d_pos[3 * i + k] += dp[k];
  }
  return 0;
}

}  // extern "C"
