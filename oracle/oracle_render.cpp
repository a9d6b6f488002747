// HyRF oracle, part 2: pre-cull, projection, binning, compositing, background
// and loss (Secs. 3.1, 3.3, 3.4; App. A.2), each with its reverse pass.
// Test infrastructure only (see hyrf_oracle.h). Plain FP64 except the FP32
// replays of integer decisions, which follow the operation order written
// out below (compiled with -ffp-contract=off so no multiply-add is fused).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "oracle_internal.h"

using namespace orc;

namespace {

struct CamF {
  float R[9], t[3], fx, fy, cx, cy, z_near, tol;
  int W, H;
};

CamF cam_f32(const orc_camera& c) {
  CamF f;
  for (int i = 0; i < 9; ++i) f.R[i] = (float)c.R[i];
  for (int i = 0; i < 3; ++i) f.t[i] = (float)c.t[i];
  f.fx = (float)c.fx;
  f.fy = (float)c.fy;
  f.cx = (float)c.cx;
  f.cy = (float)c.cy;
  f.z_near = (float)c.z_near;
  f.tol = (float)c.cull_tol;
  f.W = c.width;
  f.H = c.height;
  return f;
}

// x_c = R p + t in float, each row summed left to right.
void cam_point_f32(const CamF& c, const float p[3], float tc[3]) {
  tc[0] = c.R[0] * p[0] + c.R[1] * p[1] + c.R[2] * p[2] + c.t[0];
  tc[1] = c.R[3] * p[0] + c.R[4] * p[1] + c.R[5] * p[2] + c.t[1];
  tc[2] = c.R[6] * p[0] + c.R[7] * p[1] + c.R[8] * p[2] + c.t[2];
}

// Rotation matrix of the quaternion q = (w, x, y, z) and its derivative
// dR[k][i] = d R_i / d q_k (i = row-major entry).
void quat_rot(const double* q, double R[9], double dR[4][9]) {
  double w = q[0], x = q[1], y = q[2], z = q[3];
  R[0] = 1 - 2 * (y * y + z * z);
  R[1] = 2 * (x * y - w * z);
  R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);
  R[4] = 1 - 2 * (x * x + z * z);
  R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);
  R[7] = 2 * (y * z + w * x);
  R[8] = 1 - 2 * (x * x + y * y);
  if (!dR) return;
  const double d[4][9] = {
      {0, -2 * z, 2 * y, 2 * z, 0, -2 * x, -2 * y, 2 * x, 0},
      {0, 2 * y, 2 * z, 2 * y, -4 * x, -2 * w, 2 * z, 2 * w, -4 * x},
      {-4 * y, 2 * x, 2 * w, 2 * x, 0, 2 * z, -2 * w, 2 * z, -4 * y},
      {-4 * z, -2 * w, 2 * x, 2 * w, -4 * z, 2 * y, 2 * x, 2 * y, 0},
  };
  std::memcpy(dR, d, sizeof(d));
}

// Everything the FP64 projection computes for one Gaussian.
struct Proj {
  double tc[3], u, v, J[6], T[6], Rq[9], M[9], S[9], a, b, c, det;
  bool clx, cly;
};

void project_one(const orc_camera& cam, const double* p, const double* s, const double* q, Proj& P) {
  for (int i = 0; i < 3; ++i)
    P.tc[i] = cam.R[3 * i] * p[0] + cam.R[3 * i + 1] * p[1] + cam.R[3 * i + 2] * p[2] + cam.t[i];
  const double x = P.tc[0], y = P.tc[1], z = P.tc[2];
  P.u = cam.fx * x / z + cam.cx;
  P.v = cam.fy * y / z + cam.cy;
  // EWA Jacobian of the perspective map, with the 3DGS clamp of the tangent
  // at 1.3 times the half field of view.
  const double limx = 1.3 * (0.5 * cam.width / cam.fx), limy = 1.3 * (0.5 * cam.height / cam.fy);
  double mx = x / z, my = y / z;
  P.clx = mx < -limx || mx > limx;
  P.cly = my < -limy || my > limy;
  mx = std::min(limx, std::max(-limx, mx));
  my = std::min(limy, std::max(-limy, my));
  double J[6] = {cam.fx / z, 0, -cam.fx * mx / z, 0, cam.fy / z, -cam.fy * my / z};
  std::memcpy(P.J, J, sizeof(J));
  for (int i = 0; i < 2; ++i)
    for (int k = 0; k < 3; ++k) {
      double acc = 0;
      for (int j = 0; j < 3; ++j) acc += J[3 * i + j] * cam.R[3 * j + k];
      P.T[3 * i + k] = acc;
    }
  quat_rot(q, P.Rq, nullptr);
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) P.M[3 * i + k] = P.Rq[3 * i + k] * s[k];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double acc = 0;
      for (int k = 0; k < 3; ++k) acc += P.M[3 * i + k] * P.M[3 * j + k];
      P.S[3 * i + j] = acc;
    }
  double ab[3] = {0, 0, 0};  // (T S T^T)_00, _01, _11
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      ab[0] += P.T[i] * P.S[3 * i + j] * P.T[j];
      ab[1] += P.T[i] * P.S[3 * i + j] * P.T[3 + j];
      ab[2] += P.T[3 + i] * P.S[3 * i + j] * P.T[3 + j];
    }
  P.a = ab[0] + 0.3;  // 3DGS low-pass dilation
  P.b = ab[1];
  P.c = ab[2] + 0.3;
  P.det = P.a * P.c - P.b * P.b;
}

// Per-pixel compositing record used by the forward and the reverse pass.
struct Hit {
  int g;
  double alpha, T, G, dx, dy;
  bool clamped;
};

const double kAlphaMin = 1.0 / 255.0, kAlphaMax = 0.99, kTMin = 1e-4;

// Eq. 1 for one pixel over one list of Gaussian indices.
void composite_pixel(double px, double py, const int32_t* list, int64_t len, const double* mean2d,
                     const double* conic, const double* opacity, const double* color,
                     double C[3], double* T_out, int32_t* last, double* margin,
                     std::vector<Hit>* hits) {
  double T = 1.0, mg = 1e300;
  C[0] = C[1] = C[2] = 0.0;
  int32_t lst = 0;
  if (hits) hits->clear();
  for (int64_t k = 0; k < len; ++k) {
    int g = list[k];
    double dx = mean2d[2 * g] - px, dy = mean2d[2 * g + 1] - py;
    const double* cn = conic + 3 * g;
    double power = -0.5 * (cn[0] * dx * dx + cn[2] * dy * dy) - cn[1] * dx * dy;
    if (power > 0.0) continue;
    double G = std::exp(power);
    double oG = opacity[g] * G;
    mg = std::min(mg, std::fabs(oG - kAlphaMin) / kAlphaMin);
    mg = std::min(mg, std::fabs(oG - kAlphaMax) / kAlphaMax);
    double alpha = std::min(kAlphaMax, oG);
    if (alpha < kAlphaMin) continue;
    double Tn = T * (1.0 - alpha);
    mg = std::min(mg, std::fabs(Tn - kTMin) / kTMin);
    if (Tn < kTMin) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += color[3 * g + ch] * alpha * T;
    if (hits) hits->push_back({g, alpha, T, G, dx, dy, oG > kAlphaMax});
    T = Tn;
    lst = (int32_t)(k + 1);
  }
  *T_out = T;
  if (last) *last = lst;
  if (margin) *margin = mg;
}

// Background colour c_s seen by pixel (i, j).
struct BgSample {
  double y[3], dir[3];       // exact mode: contracted hit point, ray direction
  int a[2], b[2];            // map mode: texel rows / columns
  double wa[2], wb[2];       // map mode: bilinear weights
};

void map_texel_dir(const orc_bg& bg, int a, int b, double w[3]) {
  double phi = (b + 0.5) / bg.map_w * 2.0 * M_PI - M_PI;
  double th = (a + 0.5) / bg.map_h * M_PI - 0.5 * M_PI;
  w[0] = std::cos(th) * std::sin(phi);
  w[1] = std::sin(th);
  w[2] = std::cos(th) * std::cos(phi);
}

void map_texel_point(const orc_bg& bg, int a, int b, double y[3], double dir[3]) {
  map_texel_dir(bg, a, b, dir);
  double x[3] = {bg.radius * dir[0], bg.radius * dir[1], bg.radius * dir[2]};
  // x is already in the normalised space: only the contraction applies.
  double n = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double g = n <= 1.0 ? 1.0 : (2.0 / n - 1.0 / (n * n));
  for (int k = 0; k < 3; ++k) y[k] = 0.25 * g * x[k] + 0.5;
}

void contract_normalised(const double x[3], double y[3]) {
  double n = std::sqrt(x[0] * x[0] + x[1] * x[1] + x[2] * x[2]);
  double g = n <= 1.0 ? 1.0 : (2.0 / n - 1.0 / (n * n));
  for (int k = 0; k < 3; ++k) y[k] = 0.25 * g * x[k] + 0.5;
}

void bg_sample(const orc_camera& cam, const orc_aabb& box, const orc_bg& bg, int i, int j,
               BgSample& s) {
  double ps[3], t, o[3], d[3];
  orc_ray_sphere(&cam, &box, bg.radius, i, j, ps, &t, o, d);
  if (bg.mode == 0) {
    contract_normalised(ps, s.y);
    // View direction of the background PE: the world-space ray direction.
    double dc[3] = {(i + 0.5 - cam.cx) / cam.fx, (j + 0.5 - cam.cy) / cam.fy, 1.0};
    double dw[3];
    for (int k = 0; k < 3; ++k) dw[k] = cam.R[k] * dc[0] + cam.R[3 + k] * dc[1] + cam.R[6 + k] * dc[2];
    double nd = std::sqrt(dw[0] * dw[0] + dw[1] * dw[1] + dw[2] * dw[2]);
    for (int k = 0; k < 3; ++k) s.dir[k] = dw[k] / nd;
  } else {
    double n = std::sqrt(ps[0] * ps[0] + ps[1] * ps[1] + ps[2] * ps[2]);
    double w[3] = {ps[0] / n, ps[1] / n, ps[2] / n};
    double th = std::asin(std::max(-1.0, std::min(1.0, w[1])));
    double phi = std::atan2(w[0], w[2]);
    double bf = (phi + M_PI) / (2.0 * M_PI) * bg.map_w - 0.5;
    double af = (th + 0.5 * M_PI) / M_PI * bg.map_h - 0.5;
    double b0 = std::floor(bf), a0 = std::floor(af);
    double fb = bf - b0, fa = af - a0;
    int ib = (int)b0, ia = (int)a0;
    for (int k = 0; k < 2; ++k) {
      int bb = ((ib + k) % bg.map_w + bg.map_w) % bg.map_w;  // wrap in longitude
      int aa = std::min(bg.map_h - 1, std::max(0, ia + k));   // clamp in latitude
      s.b[k] = bb;
      s.a[k] = aa;
    }
    s.wb[0] = 1.0 - fb;
    s.wb[1] = fb;
    s.wa[0] = 1.0 - fa;
    s.wa[1] = fa;
  }
}

// 11-tap Gaussian window, sigma 1.5, normalised to sum 1 (Wang et al. 2004).
void ssim_window(double w[11]) {
  double s = 0;
  for (int i = 0; i < 11; ++i) {
    w[i] = std::exp(-(double)((i - 5) * (i - 5)) / (2.0 * 1.5 * 1.5));
    s += w[i];
  }
  for (int i = 0; i < 11; ++i) w[i] /= s;
}

// SSIM over one channel; if dS is given, also d(mean SSIM)/dx * scale added to dx.
double ssim_channel(int W, int H, const double* x, const double* y, int ch, double scale,
                    double* dx) {
  const double C1 = 0.01 * 0.01, C2 = 0.03 * 0.03;
  double w1[11];
  ssim_window(w1);
  const size_t P = (size_t)W * H;
  std::vector<double> dmu(P), dsxx(P), dsxy(P);
  double total = 0.0;
  for (int py = 0; py < H; ++py)
    for (int px = 0; px < W; ++px) {
      double mx = 0, my = 0, sxx = 0, syy = 0, sxy = 0;
      for (int dy = -5; dy <= 5; ++dy)
        for (int dxx = -5; dxx <= 5; ++dxx) {
          int qy = py + dy, qx = px + dxx;
          if (qy < 0 || qy >= H || qx < 0 || qx >= W) continue;  // zero padding
          double w = w1[dy + 5] * w1[dxx + 5];
          double a = x[((size_t)qy * W + qx) * 3 + ch], b = y[((size_t)qy * W + qx) * 3 + ch];
          mx += w * a;
          my += w * b;
          sxx += w * a * a;
          syy += w * b * b;
          sxy += w * a * b;
        }
      double vx = sxx - mx * mx, vy = syy - my * my, cxy = sxy - mx * my;
      double A1 = 2 * mx * my + C1, A2 = 2 * cxy + C2;
      double B1 = mx * mx + my * my + C1, B2 = vx + vy + C2;
      double S = (A1 * A2) / (B1 * B2);
      total += S;
      size_t p = (size_t)py * W + px;
      dmu[p] = S * (2 * my / A1 - 2 * my / A2 - 2 * mx / B1 + 2 * mx / B2);
      dsxx[p] = -S / B2;
      dsxy[p] = 2 * S / A2;
    }
  if (dx) {
    for (int qy = 0; qy < H; ++qy)
      for (int qx = 0; qx < W; ++qx) {
        double a = x[((size_t)qy * W + qx) * 3 + ch], b = y[((size_t)qy * W + qx) * 3 + ch];
        double acc = 0;
        for (int dy = -5; dy <= 5; ++dy)
          for (int dxx = -5; dxx <= 5; ++dxx) {
            int py = qy + dy, px = qx + dxx;
            if (py < 0 || py >= H || px < 0 || px >= W) continue;
            double w = w1[dy + 5] * w1[dxx + 5];
            size_t p = (size_t)py * W + px;
            acc += w * (dmu[p] + 2 * a * dsxx[p] + b * dsxy[p]);
          }
        dx[((size_t)qy * W + qx) * 3 + ch] += scale * acc;
      }
  }
  return total;
}

}  // namespace

extern "C" {

// Eqs. 8-9, with the tolerance test on normalised device coordinates
// x_ndc = 2u/W - 1, y_ndc = 2v/H - 1 and the near test z > z_near.
int32_t orc_precull_f32(int32_t n, const float* pos, const orc_camera* cam, uint8_t* vis) {
  if (n < 0 || !cam) return -1;
  CamF c = cam_f32(*cam);
  int32_t kept = 0;
  for (int i = 0; i < n; ++i) {
    float tc[3];
    cam_point_f32(c, pos + 3 * i, tc);
    bool keep = false;
    if (tc[2] > c.z_near) {
      float u = c.fx * tc[0] / tc[2] + c.cx;
      float v = c.fy * tc[1] / tc[2] + c.cy;
      float xn = 2.0f * u / (float)c.W - 1.0f;
      float yn = 2.0f * v / (float)c.H - 1.0f;
      float lim = 1.0f + c.tol;
      keep = std::fabs(xn) <= lim && std::fabs(yn) <= lim;
    }
    vis[i] = keep ? 1 : 0;
    kept += keep;
  }
  return kept;
}

int32_t orc_project(int32_t n, const double* pos, const double* scale, const double* quat,
                    const orc_camera* cam, double* mean2d, double* conic, double* depth) {
  if (n < 0 || !cam) return -1;
  for (int i = 0; i < n; ++i) {
    Proj P;
    project_one(*cam, pos + 3 * i, scale + 3 * i, quat + 4 * i, P);
    mean2d[2 * i] = P.u;
    mean2d[2 * i + 1] = P.v;
    conic[3 * i] = P.c / P.det;
    conic[3 * i + 1] = -P.b / P.det;
    conic[3 * i + 2] = P.a / P.det;
    depth[i] = P.tc[2];
  }
  return 0;
}

// FP32 replay of the integer outputs of the projection. The operation order
// below is the specification the GPU kernel follows.
// ---- opacity-aware footprint (FP32 replay of the binning's culling) ----
//
// Eq. 1 skips a pixel where alpha = o exp(-q / 2) < 1/255 with
// q = d^T Sigma'^-1 d, so a Gaussian shows nowhere with q > 2 ln(255 o).
// The footprint keeps, per tile row of the rectangle, the tile columns
// whose pixel-centre box meets the ellipse q <= t with t = 1.02 x 2 ln(255 o)
// + 0.05 (a margin far above FP32 rounding). Written with plain FP32 + - * /
// sqrt in a fixed order (no fused multiply-add) so the GPU's binning takes
// the same decisions bit for bit.

// t for opacity o (-1: no footprint at all, o < 1/255). ln x by the
// exponent and the series ln m = 2 atanh(s), s = (m - 1) / (m + 1), to s^9
// (Abramowitz & Stegun 4.1.27; truncation below 2e-6 for m in [1, 2)).
static float fp_qlimit(float o) {
  if (!(o >= 1.0f / 255.0f)) return -1.0f;
  const float x = 255.0f * o;  // >= 1
  uint32_t u;
  std::memcpy(&u, &x, 4);
  const int e = (int)((u >> 23) & 0xffu) - 127;
  const uint32_t um = (u & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &um, 4);  // x = m 2^e, m in [1, 2)
  const float s = (m - 1.0f) / (m + 1.0f);
  const float s2 = s * s;
  float pz = 1.0f / 9.0f;
  pz = pz * s2 + 1.0f / 7.0f;
  pz = pz * s2 + 1.0f / 5.0f;
  pz = pz * s2 + 1.0f / 3.0f;
  pz = pz * s2 + 1.0f;
  const float ln = (float)e * 0.693147180559945f + 2.0f * s * pz;
  return 1.02f * (2.0f * ln) + 0.05f;
}

// Tile columns [*tx0, *tx1) of tile row ty (within [cx0, cx1)) whose pixel
// centres (16 tx + 0.5 ... 16 tx + 15.5) meet the ellipse
// {(u, v) + d : d^T Sigma'^-1 d <= t}, Sigma' = [[a, b], [b, c]]: the ellipse
// cut to the row's pixel-centre strip spans x in [u + xmin, u + xmax], where
// the boundary at height dy is x = (b / c) dy +- sqrt((a - b^2 / c)(t - dy^2 / c))
// and the extremes +-sqrt(t a) sit at dy = +-b sqrt(t / a). t = +inf: the
// whole row of the rectangle.
static void fp_row_span(float u, float v, float a, float b, float c, float t, int ty, int tile, int cx0,
                        int cx1, int* tx0, int* tx1) {
  *tx0 = *tx1 = cx0;
  if (!(t >= 0.0f)) return;
  if (std::isinf(t)) {
    *tx1 = cx1;
    return;
  }
  const float tw = (float)tile;
  const float Y0 = (float)(ty * tile) + 0.5f, Y1 = Y0 + (tw - 1.0f);
  const float dy0 = Y0 - v, dy1 = Y1 - v;
  const float hy = std::sqrt(t * c);
  const float ya = std::fmax(dy0, -hy), yb = std::fmin(dy1, hy);
  if (!(ya <= yb)) return;
  const float k = b / c;
  const float mm = std::fmax(a - b * k, 0.0f);
  const float wa = std::sqrt(std::fmax(mm * (t - ya * ya / c), 0.0f));
  const float wb = std::sqrt(std::fmax(mm * (t - yb * yb / c), 0.0f));
  const float hx = std::sqrt(t * a);
  const float yr = b * std::sqrt(t / a);
  const float xmax = (yr >= ya && yr <= yb) ? hx : std::fmax(k * ya + wa, k * yb + wb);
  const float xmin = (-yr >= ya && -yr <= yb) ? -hx : std::fmin(k * ya - wa, k * yb - wb);
  float f0 = std::ceil(((u + xmin) - (tw - 0.5f)) / tw);
  float f1 = std::floor(((u + xmax) - 0.5f) / tw) + 1.0f;
  f0 = std::fmin(std::fmax(f0, (float)cx0), (float)cx1);
  f1 = std::fmin(std::fmax(f1, (float)cx0), (float)cx1);
  if (f1 > f0) {
    *tx0 = (int)f0;
    *tx1 = (int)f1;
  }
}

int32_t orc_project_f32(int32_t n, const float* pos, const float* scale, const float* quat,
                        const orc_camera* cam, int32_t tile, int32_t* rect, int32_t* ntiles,
                        float* depth, uint8_t* flag) {
  return orc_project_f32_fp(n, pos, scale, quat, nullptr, cam, tile, rect, ntiles, depth, flag, nullptr,
                            nullptr);
}

int32_t orc_project_f32_fp(int32_t n, const float* pos, const float* scale, const float* quat,
                           const float* alpha, const orc_camera* cam, int32_t tile, int32_t* rect,
                           int32_t* ntiles, float* depth, uint8_t* flag, float* mean2d, float* foot) {
  if (n < 0 || !cam || tile <= 0) return -1;
  CamF c = cam_f32(*cam);
  const int TX = (c.W + tile - 1) / tile, TY = (c.H + tile - 1) / tile;
  for (int i = 0; i < n; ++i) {
    const float* p = pos + 3 * i;
    const float* s = scale + 3 * i;
    const float* q = quat + 4 * i;
    float tc[3];
    cam_point_f32(c, p, tc);
    const float x = tc[0], y = tc[1], z = tc[2];
    if (!(z > c.z_near)) {  // behind the near plane: no footprint (3DGS's own near culling)
      rect[4 * i] = rect[4 * i + 1] = rect[4 * i + 2] = rect[4 * i + 3] = 0;
      ntiles[i] = 0;
      depth[i] = z;
      flag[i] = 0;
      continue;
    }
    const float u = c.fx * x / z + c.cx;
    const float v = c.fy * y / z + c.cy;
    const float limx = 1.3f * (0.5f * (float)c.W / c.fx);
    const float limy = 1.3f * (0.5f * (float)c.H / c.fy);
    const float mx = std::fmin(limx, std::fmax(-limx, x / z));
    const float my = std::fmin(limy, std::fmax(-limy, y / z));
    const float j00 = c.fx / z, j02 = -(c.fx * mx) / z;
    const float j11 = c.fy / z, j12 = -(c.fy * my) / z;
    float T0[3], T1[3];
    for (int k = 0; k < 3; ++k) {
      T0[k] = j00 * c.R[k] + j02 * c.R[6 + k];
      T1[k] = j11 * c.R[3 + k] + j12 * c.R[6 + k];
    }
    const float w = q[0], qx = q[1], qy = q[2], qz = q[3];
    const float r[9] = {1.0f - 2.0f * (qy * qy + qz * qz), 2.0f * (qx * qy - w * qz),
                        2.0f * (qx * qz + w * qy),         2.0f * (qx * qy + w * qz),
                        1.0f - 2.0f * (qx * qx + qz * qz), 2.0f * (qy * qz - w * qx),
                        2.0f * (qx * qz - w * qy),         2.0f * (qy * qz + w * qx),
                        1.0f - 2.0f * (qx * qx + qy * qy)};
    float M[9], S[9];
    for (int a = 0; a < 3; ++a)
      for (int k = 0; k < 3; ++k) M[3 * a + k] = r[3 * a + k] * s[k];
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        S[3 * a + b] = M[3 * a] * M[3 * b] + M[3 * a + 1] * M[3 * b + 1] + M[3 * a + 2] * M[3 * b + 2];
    float U0[3], U1[3];
    for (int k = 0; k < 3; ++k) {
      U0[k] = T0[0] * S[k] + T0[1] * S[3 + k] + T0[2] * S[6 + k];
      U1[k] = T1[0] * S[k] + T1[1] * S[3 + k] + T1[2] * S[6 + k];
    }
    const float a = U0[0] * T0[0] + U0[1] * T0[1] + U0[2] * T0[2] + 0.3f;
    const float b = U0[0] * T1[0] + U0[1] * T1[1] + U0[2] * T1[2];
    const float cc = U1[0] * T1[0] + U1[1] * T1[1] + U1[2] * T1[2] + 0.3f;
    const float det = a * cc - b * b;
    const float mid = 0.5f * (a + cc);
    const float disc = std::fmax(mid * mid - det, 0.0f);
    const float lam = mid + std::sqrt(disc);
    const float rad = std::ceil(3.0f * std::sqrt(lam));
    const float tw = (float)tile;
    float x0 = std::floor((u - rad) / tw), x1 = std::floor((u + rad) / tw) + 1.0f;
    float y0 = std::floor((v - rad) / tw), y1 = std::floor((v + rad) / tw) + 1.0f;
    x0 = std::fmin(std::fmax(x0, 0.0f), (float)TX);
    x1 = std::fmin(std::fmax(x1, 0.0f), (float)TX);
    y0 = std::fmin(std::fmax(y0, 0.0f), (float)TY);
    y1 = std::fmin(std::fmax(y1, 0.0f), (float)TY);
    int ix0 = (int)x0, ix1 = (int)x1, iy0 = (int)y0, iy1 = (int)y1;
    rect[4 * i] = ix0;
    rect[4 * i + 1] = iy0;
    rect[4 * i + 2] = ix1;
    rect[4 * i + 3] = iy1;
    ntiles[i] = (ix1 > ix0 && iy1 > iy0) ? (ix1 - ix0) * (iy1 - iy0) : 0;
    depth[i] = z;
    const bool near_singular = std::fabs(det) < 1e-2f * a * cc;
    flag[i] = near_singular ? 1 : 0;
    if (foot) {
      // the footprint; near-singular Gaussians keep their whole rectangle
      // (their conic comes from an FP64 recomputation of Sigma') unless
      // o < 1/255, where no pixel shows them at all
      float t = fp_qlimit(alpha ? alpha[i] : 1.0f);
      if (near_singular && t >= 0.0f) t = INFINITY;
      float* fr = foot + 12 * i;
      fr[0] = a;
      fr[1] = b;
      fr[2] = cc;
      fr[3] = t;
      // row spans packed as 16-bit fields (first column - x0, length) when
      // the rectangle has at most 16 rows and 255 columns; else zero words
      uint32_t w[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      const bool packed = iy1 - iy0 <= 16 && ix1 - ix0 <= 255;
      int cnt = 0;
      if (ix1 > ix0 && iy1 > iy0) {
        for (int ty = iy0; ty < iy1; ++ty) {
          int t0, t1;
          fp_row_span(u, v, a, b, cc, t, ty, tile, ix0, ix1, &t0, &t1);
          cnt += t1 - t0;
          if (packed) {
            const int j = ty - iy0;
            w[j / 2] |= (uint32_t)((t0 - ix0) | ((t1 - t0) << 8)) << (16 * (j % 2));
          }
        }
      }
      std::memcpy(fr + 4, w, sizeof(w));
      ntiles[i] = cnt;
    }
    if (mean2d) {
      mean2d[2 * i] = u;
      mean2d[2 * i + 1] = v;
    }
  }
  return 0;
}

int32_t orc_project_backward(int32_t n, const double* pos, const double* scale,
                             const double* quat, const orc_camera* cam, const double* d_mean2d,
                             const double* d_conic, double* d_pos, double* d_scale,
                             double* d_quat) {
  if (n < 0 || !cam) return -1;
  for (int i = 0; i < n; ++i) {
    Proj P;
    const double* s = scale + 3 * i;
    project_one(*cam, pos + 3 * i, s, quat + 4 * i, P);
    const double a = P.a, b = P.b, c = P.c, det = P.det, d2 = det * det;
    const double gA = d_conic[3 * i], gB = d_conic[3 * i + 1], gC = d_conic[3 * i + 2];
    // conic = (c, -b, a) / det, with det = a c - b^2.
    const double da = gA * (-c * c / d2) + gB * (b * c / d2) + gC * (-b * b / d2);
    const double db = gA * (2 * b * c / d2) + gB * (-1.0 / det - 2 * b * b / d2) + gC * (2 * a * b / d2);
    const double dc = gA * (-b * b / d2) + gB * (b * a / d2) + gC * (-a * a / d2);
    // (a, b, c) = entries of T S T^T (+0.3 on the diagonal).
    double GS[9], dT[6];
    for (int p = 0; p < 3; ++p)
      for (int q = 0; q < 3; ++q)
        GS[3 * p + q] = da * P.T[p] * P.T[q] + db * P.T[p] * P.T[3 + q] + dc * P.T[3 + p] * P.T[3 + q];
    double ST0[3], ST1[3];
    for (int p = 0; p < 3; ++p) {
      ST0[p] = ST1[p] = 0;
      for (int q = 0; q < 3; ++q) {
        ST0[p] += P.S[3 * p + q] * P.T[q];
        ST1[p] += P.S[3 * p + q] * P.T[3 + q];
      }
    }
    for (int k = 0; k < 3; ++k) {
      dT[k] = 2 * da * ST0[k] + db * ST1[k];
      dT[3 + k] = db * ST0[k] + 2 * dc * ST1[k];
    }
    // T = J R.
    double dJ[6];
    for (int r = 0; r < 2; ++r)
      for (int j = 0; j < 3; ++j) {
        double acc = 0;
        for (int k = 0; k < 3; ++k) acc += dT[3 * r + k] * cam->R[3 * j + k];
        dJ[3 * r + j] = acc;
      }
    // S = M M^T, M = Rq diag(s).
    double dM[9];
    for (int p = 0; p < 3; ++p)
      for (int k = 0; k < 3; ++k) {
        double acc = 0;
        for (int q = 0; q < 3; ++q) acc += (GS[3 * p + q] + GS[3 * q + p]) * P.M[3 * q + k];
        dM[3 * p + k] = acc;
      }
    double Rq[9], dRq[4][9];
    quat_rot(quat + 4 * i, Rq, dRq);
    for (int k = 0; k < 3; ++k) {
      double acc = 0;
      for (int p = 0; p < 3; ++p) acc += Rq[3 * p + k] * dM[3 * p + k];
      d_scale[3 * i + k] += acc;
    }
    for (int k = 0; k < 4; ++k) {
      double acc = 0;
      for (int e = 0; e < 9; ++e) acc += dRq[k][e] * dM[e] * s[e % 3];
      d_quat[4 * i + k] += acc;
    }
    // Camera-space point: mean2d and J depend on it.
    const double x = P.tc[0], y = P.tc[1], z = P.tc[2];
    const double fx = cam->fx, fy = cam->fy;
    const double du = d_mean2d[2 * i], dv = d_mean2d[2 * i + 1];
    double gx = du * fx / z, gy = dv * fy / z;
    double gz = du * (-fx * x / (z * z)) + dv * (-fy * y / (z * z));
    gz += dJ[0] * (-fx / (z * z)) + dJ[4] * (-fy / (z * z));
    const double limx = 1.3 * (0.5 * cam->width / fx), limy = 1.3 * (0.5 * cam->height / fy);
    double mx = std::min(limx, std::max(-limx, x / z)), my = std::min(limy, std::max(-limy, y / z));
    // J02 = -fx mx / z, J12 = -fy my / z, mx = x / z unless clamped.
    double dmx_dx = P.clx ? 0.0 : 1.0 / z, dmx_dz = P.clx ? 0.0 : -x / (z * z);
    double dmy_dy = P.cly ? 0.0 : 1.0 / z, dmy_dz = P.cly ? 0.0 : -y / (z * z);
    gx += dJ[2] * (-fx * dmx_dx / z);
    gz += dJ[2] * (fx * mx / (z * z) - fx * dmx_dz / z);
    gy += dJ[5] * (-fy * dmy_dy / z);
    gz += dJ[5] * (fy * my / (z * z) - fy * dmy_dz / z);
    for (int k = 0; k < 3; ++k)
      d_pos[3 * i + k] += cam->R[k] * gx + cam->R[3 + k] * gy + cam->R[6 + k] * gz;
  }
  return 0;
}

int64_t orc_bin_sort(int32_t n, const int32_t* rect, const float* depth, int32_t tiles_x,
                     int32_t tiles_y, int64_t cap, uint64_t* keys, int32_t* vals,
                     int32_t* ranges) {
  return orc_bin_sort_fp(n, rect, depth, nullptr, nullptr, 16, tiles_x, tiles_y, cap, keys, vals, ranges);
}

int64_t orc_bin_sort_fp(int32_t n, const int32_t* rect, const float* depth, const float* mean2d,
                        const float* foot, int32_t tile, int32_t tiles_x, int32_t tiles_y, int64_t cap,
                        uint64_t* keys, int32_t* vals, int32_t* ranges) {
  if (n < 0 || tiles_x <= 0 || tiles_y <= 0 || tile <= 0) return -2;
  std::vector<std::pair<uint64_t, int32_t>> inst;
  for (int g = 0; g < n; ++g) {
    const int32_t* r = rect + 4 * g;
    if (!(r[2] > r[0] && r[3] > r[1])) continue;
    uint32_t bits;
    std::memcpy(&bits, depth + g, 4);
    for (int ty = r[1]; ty < r[3]; ++ty) {
      int t0 = r[0], t1 = r[2];
      if (foot)
        fp_row_span(mean2d[2 * g], mean2d[2 * g + 1], foot[12 * g], foot[12 * g + 1], foot[12 * g + 2],
                    foot[12 * g + 3], ty, tile, r[0], r[2], &t0, &t1);
      for (int tx = t0; tx < t1; ++tx) inst.push_back({((uint64_t)(ty * tiles_x + tx) << 32) | bits, g});
    }
  }
  std::stable_sort(inst.begin(), inst.end(),
                   [](const std::pair<uint64_t, int32_t>& A, const std::pair<uint64_t, int32_t>& B) {
                     return A.first < B.first;
                   });
  const int64_t K = (int64_t)inst.size();
  for (int64_t t = 0; t < 2LL * tiles_x * tiles_y; ++t) ranges[t] = 0;
  if (K > cap) return -1;
  for (int64_t k = 0; k < K; ++k) {
    keys[k] = inst[k].first;
    vals[k] = inst[k].second;
    int32_t t = (int32_t)(inst[k].first >> 32);
    if (k == 0 || (int32_t)(inst[k - 1].first >> 32) != t) ranges[2 * t] = (int32_t)k;
    if (k == K - 1 || (int32_t)(inst[k + 1].first >> 32) != t) ranges[2 * t + 1] = (int32_t)(k + 1);
  }
  return K;
}

int32_t orc_rasterize(int32_t width, int32_t height, int32_t tile, const int32_t* ranges,
                      const int32_t* vals, const double* mean2d, const double* conic,
                      const double* opacity, const double* color, double* C_fg, double* T_final,
                      int32_t* n_contrib, double* margin) {
  if (width <= 0 || height <= 0 || tile <= 0) return -1;
  const int TX = (width + tile - 1) / tile;
  for (int py = 0; py < height; ++py)
    for (int px = 0; px < width; ++px) {
      int t = (py / tile) * TX + px / tile;
      size_t p = (size_t)py * width + px;
      composite_pixel(px + 0.5, py + 0.5, vals + ranges[2 * t], ranges[2 * t + 1] - ranges[2 * t],
                      mean2d, conic, opacity, color, C_fg + 3 * p, T_final + p,
                      n_contrib ? n_contrib + p : nullptr, margin ? margin + p : nullptr, nullptr);
    }
  return 0;
}

int32_t orc_rasterize_untiled(int32_t width, int32_t height, int32_t tile, int32_t n,
                              const int32_t* rect, const float* depth, const double* mean2d,
                              const double* conic, const double* opacity, const double* color,
                              double* C_fg, double* T_final) {
  if (width <= 0 || height <= 0 || tile <= 0 || n < 0) return -1;
  std::vector<int32_t> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int A, int B) { return depth[A] < depth[B]; });
  std::vector<int32_t> list;
  for (int py = 0; py < height; ++py)
    for (int px = 0; px < width; ++px) {
      int tx = px / tile, ty = py / tile;
      list.clear();
      for (int g : order) {
        const int32_t* r = rect + 4 * g;
        if (tx >= r[0] && tx < r[2] && ty >= r[1] && ty < r[3]) list.push_back(g);
      }
      size_t p = (size_t)py * width + px;
      composite_pixel(px + 0.5, py + 0.5, list.data(), (int64_t)list.size(), mean2d, conic, opacity,
                      color, C_fg + 3 * p, T_final + p, nullptr, nullptr, nullptr);
    }
  return 0;
}

// Reverse of Eq. 1 (and of the T_final factor of Eq. 10), computed from the
// full per-pixel list of contributions.
int32_t orc_rasterize_backward(int32_t width, int32_t height, int32_t tile, const int32_t* ranges,
                               const int32_t* vals, const double* mean2d, const double* conic,
                               const double* opacity, const double* color, const double* d_C_fg,
                               const double* d_T_final, double* d_mean2d, double* d_conic,
                               double* d_opacity, double* d_color) {
  if (width <= 0 || height <= 0 || tile <= 0) return -1;
  const int TX = (width + tile - 1) / tile;
  std::vector<Hit> hits;
  for (int py = 0; py < height; ++py)
    for (int px = 0; px < width; ++px) {
      int t = (py / tile) * TX + px / tile;
      size_t p = (size_t)py * width + px;
      double C[3], Tf;
      composite_pixel(px + 0.5, py + 0.5, vals + ranges[2 * t], ranges[2 * t + 1] - ranges[2 * t],
                      mean2d, conic, opacity, color, C, &Tf, nullptr, nullptr, &hits);
      const double* G = d_C_fg + 3 * p;
      const double gT = d_T_final[p];
      double S[3] = {0, 0, 0};  // sum over later contributors of c_k alpha_k T_k
      for (int h = (int)hits.size() - 1; h >= 0; --h) {
        const Hit& H = hits[h];
        const double* c = color + 3 * H.g;
        double dalpha = 0;
        for (int ch = 0; ch < 3; ++ch) {
          d_color[3 * H.g + ch] += H.alpha * H.T * G[ch];
          dalpha += G[ch] * (c[ch] * H.T - S[ch] / (1.0 - H.alpha));
          S[ch] += c[ch] * H.alpha * H.T;
        }
        dalpha -= gT * Tf / (1.0 - H.alpha);
        if (H.clamped) continue;  // alpha = 0.99 does not depend on o or the power
        d_opacity[H.g] += dalpha * H.G;
        double dpow = dalpha * H.alpha;
        const double* cn = conic + 3 * H.g;
        d_mean2d[2 * H.g] += dpow * (-cn[0] * H.dx - cn[1] * H.dy);
        d_mean2d[2 * H.g + 1] += dpow * (-cn[2] * H.dy - cn[1] * H.dx);
        d_conic[3 * H.g] += dpow * (-0.5 * H.dx * H.dx);
        d_conic[3 * H.g + 1] += dpow * (-H.dx * H.dy);
        d_conic[3 * H.g + 2] += dpow * (-0.5 * H.dy * H.dy);
      }
    }
  return 0;
}

// App. A.2: ray o + t d against the sphere |x| = r centred at the origin of
// the normalised space; the larger root is the forward hit.
void orc_ray_sphere(const orc_camera* cam, const orc_aabb* box, double radius, int32_t i,
                    int32_t j, double p_s[3], double* t_hit, double o_n[3], double d_n[3]) {
  double oc[3];
  camera_center(*cam, oc);
  double dc[3] = {(i + 0.5 - cam->cx) / cam->fx, (j + 0.5 - cam->cy) / cam->fy, 1.0};
  for (int k = 0; k < 3; ++k) {
    double dw = cam->R[k] * dc[0] + cam->R[3 + k] * dc[1] + cam->R[6 + k] * dc[2];
    double sx = 2.0 / (box->hi[k] - box->lo[k]);
    o_n[k] = (oc[k] - box->lo[k]) * sx - 1.0;
    d_n[k] = dw * sx;
  }
  double A = d_n[0] * d_n[0] + d_n[1] * d_n[1] + d_n[2] * d_n[2];
  double B = 2.0 * (o_n[0] * d_n[0] + o_n[1] * d_n[1] + o_n[2] * d_n[2]);
  double C = o_n[0] * o_n[0] + o_n[1] * o_n[1] + o_n[2] * o_n[2] - radius * radius;
  double t = (-B + std::sqrt(B * B - 4.0 * A * C)) / (2.0 * A);
  *t_hit = t;
  for (int k = 0; k < 3; ++k) p_s[k] = o_n[k] + t * d_n[k];
}

static bool bg_ok(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg) {
  if (!cam || !fl || !bg) return false;
  if (bg->mode == 1 && (bg->map_h <= 0 || bg->map_w <= 0)) return false;
  return bg->mode == 0 || bg->mode == 1;
}

// Eqs. 10-11: C = C_fg + T_final * c_s.
int32_t orc_background(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg,
                       const double* C_fg, const double* T_final, double* C, double* c_s) {
  if (!bg_ok(cam, fl, bg)) return -1;
  const int W = cam->width, H = cam->height;
  std::vector<double> map;
  if (bg->mode == 1) {
    map.resize((size_t)bg->map_h * bg->map_w * 3);
    for (int a = 0; a < bg->map_h; ++a)
      for (int b = 0; b < bg->map_w; ++b) {
        double y[3], dir[3];
        map_texel_point(*bg, a, b, y, dir);
        bg_color(*fl, y, dir, &map[((size_t)a * bg->map_w + b) * 3]);
      }
  }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      size_t p = (size_t)j * W + i;
      BgSample s;
      bg_sample(*cam, fl->box, *bg, i, j, s);
      double cs[3] = {0, 0, 0};
      if (bg->mode == 0) {
        bg_color(*fl, s.y, s.dir, cs);
      } else {
        for (int ka = 0; ka < 2; ++ka)
          for (int kb = 0; kb < 2; ++kb) {
            const double* m = &map[((size_t)s.a[ka] * bg->map_w + s.b[kb]) * 3];
            for (int ch = 0; ch < 3; ++ch) cs[ch] += s.wa[ka] * s.wb[kb] * m[ch];
          }
      }
      for (int ch = 0; ch < 3; ++ch) {
        C[3 * p + ch] = C_fg[3 * p + ch] + T_final[p] * cs[ch];
        if (c_s) c_s[3 * p + ch] = cs[ch];
      }
    }
  return 0;
}

int32_t orc_background_backward(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg,
                                const double* T_final, const double* d_C, double* d_C_fg,
                                double* d_T_final, double* d_rad_table,
                                const orc_mlp_grad* d_col_mlp) {
  if (!bg_ok(cam, fl, bg)) return -1;
  const int W = cam->width, H = cam->height;
  std::vector<double> map, dmap;
  if (bg->mode == 1) {
    map.resize((size_t)bg->map_h * bg->map_w * 3);
    dmap.assign(map.size(), 0.0);
    for (int a = 0; a < bg->map_h; ++a)
      for (int b = 0; b < bg->map_w; ++b) {
        double y[3], dir[3];
        map_texel_point(*bg, a, b, y, dir);
        bg_color(*fl, y, dir, &map[((size_t)a * bg->map_w + b) * 3]);
      }
  }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      size_t p = (size_t)j * W + i;
      BgSample s;
      bg_sample(*cam, fl->box, *bg, i, j, s);
      double cs[3] = {0, 0, 0};
      if (bg->mode == 0) {
        bg_color(*fl, s.y, s.dir, cs);
      } else {
        for (int ka = 0; ka < 2; ++ka)
          for (int kb = 0; kb < 2; ++kb) {
            const double* m = &map[((size_t)s.a[ka] * bg->map_w + s.b[kb]) * 3];
            for (int ch = 0; ch < 3; ++ch) cs[ch] += s.wa[ka] * s.wb[kb] * m[ch];
          }
      }
      double dcs[3];
      for (int ch = 0; ch < 3; ++ch) {
        d_C_fg[3 * p + ch] += d_C[3 * p + ch];
        d_T_final[p] += d_C[3 * p + ch] * cs[ch];
        dcs[ch] = d_C[3 * p + ch] * T_final[p];
      }
      if (bg->mode == 0) {
        bg_color_backward(*fl, s.y, s.dir, dcs, d_rad_table, d_col_mlp);
      } else {
        for (int ka = 0; ka < 2; ++ka)
          for (int kb = 0; kb < 2; ++kb) {
            double* dm = &dmap[((size_t)s.a[ka] * bg->map_w + s.b[kb]) * 3];
            for (int ch = 0; ch < 3; ++ch) dm[ch] += s.wa[ka] * s.wb[kb] * dcs[ch];
          }
      }
    }
  if (bg->mode == 1) {
    for (int a = 0; a < bg->map_h; ++a)
      for (int b = 0; b < bg->map_w; ++b) {
        double y[3], dir[3];
        map_texel_point(*bg, a, b, y, dir);
        bg_color_backward(*fl, y, dir, &dmap[((size_t)a * bg->map_w + b) * 3], d_rad_table,
                          d_col_mlp);
      }
  }
  return 0;
}

int32_t orc_bg_margins(const orc_camera* cam, const orc_fields* fl, const orc_bg* bg,
                       double* margin) {
  if (!bg_ok(cam, fl, bg)) return -1;
  const int W = cam->width, H = cam->height;
  std::vector<double> tm;
  if (bg->mode == 1) {
    tm.resize((size_t)bg->map_h * bg->map_w);
    for (int a = 0; a < bg->map_h; ++a)
      for (int b = 0; b < bg->map_w; ++b) {
        double y[3], dir[3];
        map_texel_point(*bg, a, b, y, dir);
        tm[(size_t)a * bg->map_w + b] = bg_margin(*fl, y, dir);
      }
  }
  for (int j = 0; j < H; ++j)
    for (int i = 0; i < W; ++i) {
      BgSample s;
      bg_sample(*cam, fl->box, *bg, i, j, s);
      double m = 1e300;
      if (bg->mode == 0) {
        m = bg_margin(*fl, s.y, s.dir);
      } else {
        for (int ka = 0; ka < 2; ++ka)
          for (int kb = 0; kb < 2; ++kb) m = std::min(m, tm[(size_t)s.a[ka] * bg->map_w + s.b[kb]]);
      }
      margin[(size_t)j * W + i] = m;
    }
  return 0;
}

double orc_ssim(int32_t width, int32_t height, const double* x, const double* y) {
  double t = 0;
  for (int ch = 0; ch < 3; ++ch) t += ssim_channel(width, height, x, y, ch, 0.0, nullptr);
  return t / (3.0 * width * height);
}

// Eq. 12 with L_ssim read as 1 - SSIM (D-SSIM, as in 3DGS).
double orc_loss(int32_t width, int32_t height, const double* C, const double* target,
                double lambda, double* d_C) {
  const size_t n = (size_t)width * height * 3;
  double l1 = 0;
  for (size_t e = 0; e < n; ++e) {
    double d = C[e] - target[e];
    l1 += std::fabs(d);
    if (d_C) d_C[e] = (1.0 - lambda) * (d > 0 ? 1.0 : (d < 0 ? -1.0 : 0.0)) / (double)n;
  }
  l1 /= (double)n;
  double loss = (1.0 - lambda) * l1;
  if (lambda != 0.0) {
    double t = 0;
    for (int ch = 0; ch < 3; ++ch)
      t += ssim_channel(width, height, C, target, ch, -lambda / (double)n, d_C);
    loss += lambda * (1.0 - t / (double)n);
  }
  return loss;
}

}  // extern "C"
