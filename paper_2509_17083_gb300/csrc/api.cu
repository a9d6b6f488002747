// extern "C" entry points of libhyrf (declared in include/hyrf.h): argument
// checks on the host, workspace sizing and kernel dispatch.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace hyrf {

// launchers (one per translation unit)
size_t precull_workspace(int n);
size_t depth_order_workspace(int n);
hyrf_status launch_depth_order(const hyrf_depth_order_args& a, void* ws, cudaStream_t s);
hyrf_status launch_precull(const CamDev& cam, const float* pos, int n, int32_t* vis_ids,
                           int32_t* n_vis, void* ws, cudaStream_t s);
hyrf_status launch_project(const CamDev& cam, int n, const float* pos, const int32_t* vis_ids,
                           const int32_t* n_vis, const float* scale, const float* quat, float* mean2d,
                           float* conic, float* depth, int32_t* rect, int32_t* ntiles, uint8_t* flag,
                           int32_t* status, const float* alpha, float* footprint, cudaStream_t s);
hyrf_status launch_project_bwd(const hyrf_project_backward_args& a, cudaStream_t s);
hyrf_status launch_query_fwd(const hyrf_query_fields_args& a, const FieldsDev& F, void* ws, cudaStream_t s);
size_t query_fwd_workspace_f32(const hyrf_fields& f, const FieldsDev& F, int n);
hyrf_status launch_query_fwd_tc(const hyrf_query_fields_args& a, const FieldsDev& F, void* ws, cudaStream_t s);
hyrf_status launch_query_explicit(const hyrf_query_fields_args& a, cudaStream_t s);
hyrf_status launch_query_explicit_bwd(const hyrf_query_fields_backward_args& a, cudaStream_t s);
hyrf_status launch_bg_none(const hyrf_composite_background_args& a, cudaStream_t s);
hyrf_status launch_bg_gather(const hyrf_composite_background_args& a, const FieldsDev& F, cudaStream_t s);
hyrf_status launch_bg_none_bwd(const hyrf_composite_background_backward_args& b, cudaStream_t s);
size_t tc_fwd_feature_bytes(int64_t rows, int fields);
size_t tc_bwd_workspace(const FieldsDev& F, bool geo, int64_t rows, bool have_features);
hyrf_status launch_bg_exact_fwd_tc(const hyrf_composite_background_args& a, const FieldsDev& F, void* ws,
                                   cudaStream_t s);
hyrf_status launch_query_bwd(const hyrf_query_fields_backward_args& a, const FieldsDev& F, void* ws,
                             cudaStream_t s);
hyrf_status launch_query_bwd_tc(const hyrf_query_fields_backward_args& a, const FieldsDev& F, void* ws,
                                cudaStream_t s);
hyrf_status launch_bg_bwd_tc(const hyrf_composite_background_backward_args& b, const FieldsDev& F,
                             void* ws, cudaStream_t s);
size_t slab_bytes(const FieldsDev& F, bool geo);
size_t query_bwd_workspace(const hyrf_fields& f, const FieldsDev& F, int n);
size_t bg_workspace(const hyrf_composite_background_args& a, const FieldsDev& F, bool backward);
hyrf_status launch_bg_fwd(const hyrf_composite_background_args& a, const FieldsDev& F, void* ws,
                          cudaStream_t s);
hyrf_status launch_bg_bwd(const hyrf_composite_background_backward_args& b, const FieldsDev& F,
                          void* ws, cudaStream_t s);
size_t bin_sort_workspace(int n, int64_t cap);
hyrf_status launch_bin_sort(const hyrf_bin_sort_args& a, void* ws, cudaStream_t s);
size_t raster_workspace(int n, int width, int height, bool reverse);
hyrf_status launch_raster_fwd(const hyrf_rasterize_args& a, void* ws, cudaStream_t s);
size_t tile_order_workspace(int width, int height);
hyrf_status launch_wait_check(int32_t* status, uint32_t polls, cudaStream_t s);
hyrf_status launch_tile_order(const hyrf_tile_order_args& a, void* ws, cudaStream_t s);
hyrf_status launch_raster_bwd(const hyrf_rasterize_backward_args& b, void* ws, cudaStream_t s);
size_t loss_workspace(const hyrf_loss_args& a);
hyrf_status launch_loss(const hyrf_loss_args& a, void* ws, cudaStream_t s);

static std::atomic<uint64_t> g_launches{0};
void count_launch(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

// ---------------------------------------------------------------- stream forks
hyrf_status fork_stream(cudaStream_t before, cudaStream_t after) {
  constexpr int kPool = 64;
  static std::mutex mu;
  static cudaEvent_t pool[64][kPool];
  static int next[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return HYRF_ERR_CUDA;
  cudaEvent_t ev;
  {
    std::lock_guard<std::mutex> lock(mu);
    cudaEvent_t& slot = pool[dev][next[dev]];
    if (!slot && cudaEventCreateWithFlags(&slot, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return HYRF_ERR_CUDA;
    }
    ev = slot;
    next[dev] = (next[dev] + 1) % kPool;
  }
  if (cudaEventRecord(ev, before) != cudaSuccess || cudaStreamWaitEvent(after, ev, 0) != cudaSuccess) {
    cudaGetLastError();
    return HYRF_ERR_CUDA;
  }
  return HYRF_OK;
}

// ---------------------------------------------------------------- kernel timer
namespace {
struct TimedLaunch {
  const char* name;
  cudaEvent_t a, b;
};
struct KernelTotal {
  const char* name;
  uint64_t launches;
  double ms;
};
std::atomic<bool> g_timer_on{false};
std::mutex g_timer_mu;
std::vector<TimedLaunch> g_pending;
std::vector<cudaEvent_t> g_free_events;
std::vector<KernelTotal> g_totals;

cudaEvent_t take_event() {
  if (!g_free_events.empty()) {
    cudaEvent_t e = g_free_events.back();
    g_free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

KernelTimer::KernelTimer(const char* name, cudaStream_t s) : name_(name), s_(s) {
  if (!g_timer_on.load(std::memory_order_relaxed)) return;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return;
  }
  std::lock_guard<std::mutex> lock(g_timer_mu);
  a_ = take_event();
  b_ = take_event();
  if (!a_ || !b_ || cudaEventRecord(a_, s) != cudaSuccess) {
    cudaGetLastError();
    if (a_) g_free_events.push_back(a_);
    if (b_) g_free_events.push_back(b_);
    a_ = b_ = nullptr;
  }
}

KernelTimer::~KernelTimer() {
  if (!a_) return;
  std::lock_guard<std::mutex> lock(g_timer_mu);
  if (cudaEventRecord(b_, s_) != cudaSuccess) {
    cudaGetLastError();
    g_free_events.push_back(a_);
    g_free_events.push_back(b_);
    return;
  }
  g_pending.push_back({name_, a_, b_});
}

int num_sms() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
      sms = 148;
  }
  return sms;
}

static bool cam_ok(const hyrf_camera& c) {
  return c.width > 0 && c.height > 0 && c.width <= 16384 && c.height <= 16384 && c.fx > 0.0f &&
         c.fy > 0.0f && c.z_near >= 0.0f && c.cull_tol >= 0.0f;
}

// The field query's camera may carry a negative near distance: the pre-cull
// then keeps Gaussians behind the camera too (the "w/o Pre-culling"
// ablation queries every Gaussian; the projection drops them).
static bool query_cam_ok(const hyrf_camera& c) {
  hyrf_camera d = c;
  if (!(c.z_near == c.z_near)) return false;
  d.z_near = 0.0f;
  return cam_ok(d);
}

static bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// bf16 decoder weights are staged with 16-byte vector loads
static bool bf16_weights_ok(const hyrf_mlp& m) {
  if (m.dtype != HYRF_BF16 && m.dtype != HYRF_F16) return true;
  for (int l = 0; l <= m.n_hidden && l < 3; ++l)
    if (!aligned(m.W[l], 16)) return false;
  return true;
}

static bool ws_ok(void* ws, size_t have, size_t need) {
  return have >= need && (need == 0 || (ws != nullptr && aligned(ws, 256)));
}

}  // namespace hyrf

using namespace hyrf;

#define S(x) static_cast<cudaStream_t>(x)

namespace hyrf {
// Host-side argument checks shared by hyrf_bin_sort, its reverse and
// hyrf_bin_sort_noalloc (no device work, no workspace).
hyrf_status bin_sort_check(const hyrf_bin_sort_args* a) {
  if (!a || a->n < 0 || a->tiles_x <= 0 || a->tiles_y <= 0 || a->capacity < 0 ||
      a->capacity > 0x7fffffffLL || (int64_t)a->tiles_x * a->tiles_y > (1 << 24))
    return HYRF_ERR_INVALID_ARG;
  if (!a->n_vis || !a->ranges || !a->n_instances) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->rect || !a->ntiles || !a->depth)) return HYRF_ERR_INVALID_ARG;
  if (a->capacity > 0 && !a->vals) return HYRF_ERR_INVALID_ARG;
  if ((a->mean2d == nullptr) != (a->footprint == nullptr)) return HYRF_ERR_INVALID_ARG;
  if (a->footprint && !aligned(a->footprint, 16)) return HYRF_ERR_INVALID_ARG;
  return HYRF_OK;
}
}  // namespace hyrf

extern "C" {

// ------------------------------------------------------------------ query fields

size_t hyrf_query_fields_workspace_size(const hyrf_query_fields_args* a) {
  if (!a || a->n < 0) return 0;
  if (a->explicit_only) return align_up(precull_workspace(a->n));
  FieldsDev F;
  const bool tc = make_fields(a->fields, F, true) && F.cm.bf16;
  return align_up(precull_workspace(a->n)) + (tc && !a->features ? tc_fwd_feature_bytes(a->n, 2) : 0) +
         (tc ? 0 : query_fwd_workspace_f32(a->fields, F, a->n));
}

hyrf_status hyrf_query_fields(const hyrf_query_fields_args* a, void* ws, size_t ws_bytes,
                              void* stream) {
  if (!a || a->n < 0 || !query_cam_ok(a->cam)) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids || !a->alpha || !a->scale || !a->quat || !a->color))
    return HYRF_ERR_INVALID_ARG;
  if (!a->n_vis || !ws_ok(ws, ws_bytes, hyrf_query_fields_workspace_size(a)))
    return HYRF_ERR_INVALID_ARG;
  if (a->explicit_only) {  // "w/o Neural": no field is read
    if (a->features) return HYRF_ERR_INVALID_ARG;
    hyrf_status st = a->vis_ready ? HYRF_OK
                                  : launch_precull(to_dev(a->cam), a->pos, a->n, a->vis_ids, a->n_vis, ws, S(stream));
    return st != HYRF_OK ? st : launch_query_explicit(*a, S(stream));
  }
  FieldsDev F;
  if (!make_fields(a->fields, F, true)) return HYRF_ERR_UNSUPPORTED;
  if (F.gm.bf16 != F.cm.bf16 || (F.cm.bf16 && a->fields.rad.n_levels != 16))
    return HYRF_ERR_UNSUPPORTED;
  // both grids of one type; 8-bit codes only with the tensor-core decoders;
  // f16 decoders with f16 or 8-bit grids, f16 grids only with f16 decoders
  if (F.geo.bf16 != F.rad.bf16 || F.geo.u8 != F.rad.u8 || F.geo.f16 != F.rad.f16 || F.gm.f16 != F.cm.f16 ||
      (F.rad.u8 && !F.cm.bf16) || (F.cm.f16 && !(F.rad.f16 || F.rad.u8)) || (F.rad.f16 && !F.cm.f16))
    return HYRF_ERR_UNSUPPORTED;
  if (!bf16_weights_ok(a->fields.geo_mlp) || !bf16_weights_ok(a->fields.col_mlp)) return HYRF_ERR_INVALID_ARG;
  if (a->features && (!F.cm.bf16 || !aligned(a->features, 16))) return HYRF_ERR_INVALID_ARG;
  hyrf_status st = a->vis_ready ? HYRF_OK
                                : launch_precull(to_dev(a->cam), a->pos, a->n, a->vis_ids, a->n_vis, ws, S(stream));
  if (st != HYRF_OK) return st;
  // BF16 decoders run on the tensor cores, FP32 decoders on the CUDA cores
  return F.cm.bf16 ? launch_query_fwd_tc(*a, F, ws, S(stream)) : launch_query_fwd(*a, F, ws, S(stream));
}

size_t hyrf_precull_workspace_size(const hyrf_precull_args* a) {
  return a && a->n >= 0 ? align_up(precull_workspace(a->n)) : 0;
}

hyrf_status hyrf_precull(const hyrf_precull_args* a, void* ws, size_t ws_bytes, void* stream) {
  if (!a || a->n < 0 || !query_cam_ok(a->cam) || !a->n_vis) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids)) return HYRF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, hyrf_precull_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_precull(to_dev(a->cam), a->pos, a->n, a->vis_ids, a->n_vis, ws, S(stream));
}

size_t hyrf_depth_order_workspace_size(const hyrf_depth_order_args* a) {
  return a && a->n >= 0 ? depth_order_workspace(a->n) : 0;
}

hyrf_status hyrf_depth_order(const hyrf_depth_order_args* a, void* ws, size_t ws_bytes, void* stream) {
  if (!a || a->n < 0 || !query_cam_ok(a->cam) || !a->n_vis) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids || !a->order)) return HYRF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, hyrf_depth_order_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_depth_order(*a, ws, S(stream));
}

size_t hyrf_query_fields_backward_workspace_size(const hyrf_query_fields_backward_args* a) {
  if (!a || a->explicit_only) return 0;
  FieldsDev F;
  if (!make_fields(a->fields, F, true) || a->n < 0) return 0;
  return F.cm.bf16 ? tc_bwd_workspace(F, true, a->n, a->features != nullptr) : query_bwd_workspace(a->fields, F, a->n);
}

hyrf_status hyrf_query_fields_backward(const hyrf_query_fields_backward_args* a, void* ws,
                                       size_t ws_bytes, void* stream) {
  if (!a || a->n < 0 || !query_cam_ok(a->cam) || !(a->loss_scale > 0.0f)) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids || !a->n_vis || !a->d_alpha || !a->d_scale || !a->d_quat ||
                   !a->d_color || !a->d_pos))
    return HYRF_ERR_INVALID_ARG;
  if (a->explicit_only) return launch_query_explicit_bwd(*a, S(stream));
  FieldsDev F;
  if (!make_fields(a->fields, F, true)) return HYRF_ERR_UNSUPPORTED;
  if (F.geo.u8 || F.rad.u8 || F.rad.f16 || F.cm.f16) return HYRF_ERR_UNSUPPORTED;  // render-only types
  if (F.gm.bf16 != F.cm.bf16 || (F.cm.bf16 && a->fields.rad.n_levels != 16))
    return HYRF_ERR_UNSUPPORTED;
  if (!ws_ok(ws, ws_bytes, hyrf_query_fields_backward_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  if (!bf16_weights_ok(a->fields.geo_mlp) || !bf16_weights_ok(a->fields.col_mlp)) return HYRF_ERR_INVALID_ARG;
  if (a->features && (!F.cm.bf16 || !aligned(a->features, 16))) return HYRF_ERR_INVALID_ARG;
  return F.cm.bf16 ? launch_query_bwd_tc(*a, F, ws, S(stream)) : launch_query_bwd(*a, F, ws, S(stream));
}

// ------------------------------------------------------------------ project

size_t hyrf_project_workspace_size(const hyrf_project_args*) { return 0; }

hyrf_status hyrf_project(const hyrf_project_args* a, void* ws, size_t ws_bytes, void* stream) {
  (void)ws;
  (void)ws_bytes;
  if (!a || a->n < 0 || !cam_ok(a->cam) || a->tile != kTile) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids || !a->n_vis || !a->scale || !a->quat || !a->mean2d ||
                   !a->conic || !a->depth || !a->rect || !a->ntiles))
    return HYRF_ERR_INVALID_ARG;
  if (a->footprint && !aligned(a->footprint, 16)) return HYRF_ERR_INVALID_ARG;
  return launch_project(to_dev(a->cam), a->n, a->pos, a->vis_ids, a->n_vis, a->scale, a->quat,
                        a->mean2d, a->conic, a->depth, a->rect, a->ntiles, a->fp64_flag, a->status,
                        a->alpha, a->footprint, S(stream));
}

size_t hyrf_project_backward_workspace_size(const hyrf_project_backward_args*) { return 0; }

hyrf_status hyrf_project_backward(const hyrf_project_backward_args* a, void* ws, size_t ws_bytes,
                                  void* stream) {
  (void)ws;
  (void)ws_bytes;
  if (!a || a->n < 0 || !cam_ok(a->cam)) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->pos || !a->vis_ids || !a->n_vis || !a->scale || !a->quat || !a->d_mean2d ||
                   !a->d_conic || !a->d_pos || !a->d_scale || !a->d_quat))
    return HYRF_ERR_INVALID_ARG;
  return launch_project_bwd(*a, S(stream));
}

// ------------------------------------------------------------------ bin + sort

size_t hyrf_bin_sort_workspace_size(const hyrf_bin_sort_args* a) {
  return a && a->n >= 0 && a->capacity >= 0 ? bin_sort_workspace(a->n, a->capacity) : 0;
}


hyrf_status hyrf_bin_sort(const hyrf_bin_sort_args* a, void* ws, size_t ws_bytes, void* stream) {
  hyrf_status st = bin_sort_check(a);
  if (st != HYRF_OK) return st;
  if (!ws_ok(ws, ws_bytes, hyrf_bin_sort_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_bin_sort(*a, ws, S(stream));
}

hyrf_status hyrf_bin_sort_backward(const hyrf_bin_sort_args* a, void* ws, size_t ws_bytes,
                                   void* stream) {
  (void)ws;
  (void)ws_bytes;
  (void)stream;
  return bin_sort_check(a);
}

// ------------------------------------------------------------------ rasterize

static hyrf_status raster_check(const hyrf_rasterize_args* a) {
  if (!a || a->n < 0 || a->width <= 0 || a->height <= 0 || a->tile != kTile) return HYRF_ERR_INVALID_ARG;
  if (!a->n_vis || !a->ranges || !a->C_fg || !a->T_final || !a->n_contrib) return HYRF_ERR_INVALID_ARG;
  if (a->n > 0 && (!a->vals || !a->mean2d || !a->conic || !a->alpha || !a->color))
    return HYRF_ERR_INVALID_ARG;
  if (a->records && (reinterpret_cast<uintptr_t>(a->records) & 15u)) return HYRF_ERR_INVALID_ARG;
  return HYRF_OK;
}

size_t hyrf_tile_order_workspace_size(const hyrf_tile_order_args* a) {
  return a && a->width > 0 && a->height > 0 ? tile_order_workspace(a->width, a->height) : 0;
}

hyrf_status hyrf_check_bounded_wait(int32_t* status, uint32_t polls, void* stream) {
  if (!status || polls < 1 || polls > (1u << 24)) return HYRF_ERR_INVALID_ARG;
  return launch_wait_check(status, polls, S(stream));
}

hyrf_status hyrf_tile_order(const hyrf_tile_order_args* a, void* ws, size_t ws_bytes, void* stream) {
  if (!a || a->width <= 0 || a->height <= 0 || a->tile != kTile || !a->n_contrib || !a->order)
    return HYRF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, hyrf_tile_order_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_tile_order(*a, ws, S(stream));
}

size_t hyrf_rasterize_workspace_size(const hyrf_rasterize_args* a) {
  return a ? raster_workspace(a->n, a->width, a->height, false) : 0;
}

hyrf_status hyrf_rasterize(const hyrf_rasterize_args* a, void* ws, size_t ws_bytes, void* stream) {
  hyrf_status st = raster_check(a);
  if (st != HYRF_OK) return st;
  if (!ws_ok(ws, ws_bytes, hyrf_rasterize_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_raster_fwd(*a, ws, S(stream));
}

size_t hyrf_rasterize_backward_workspace_size(const hyrf_rasterize_backward_args* a) {
  return a ? raster_workspace(a->fwd.n, a->fwd.width, a->fwd.height, true) : 0;
}

hyrf_status hyrf_rasterize_backward(const hyrf_rasterize_backward_args* a, void* ws, size_t ws_bytes,
                                    void* stream) {
  if (!a) return HYRF_ERR_INVALID_ARG;
  hyrf_status st = raster_check(&a->fwd);
  if (st != HYRF_OK) return st;
  if (!a->d_C_fg || (!a->d_T_final && !a->C)) return HYRF_ERR_INVALID_ARG;
  if (a->fwd.n > 0 && (!a->d_mean2d || !a->d_conic || !a->d_alpha || !a->d_color))
    return HYRF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, hyrf_rasterize_backward_workspace_size(a))) return HYRF_ERR_INVALID_ARG;
  return launch_raster_bwd(*a, ws, S(stream));
}

// ------------------------------------------------------------------ background

static hyrf_status bg_check(const hyrf_composite_background_args* a, FieldsDev& F) {
  if (!a || !cam_ok(a->cam) || !a->C_fg || !a->T_final) return HYRF_ERR_INVALID_ARG;
  if (!(a->bg.radius > 0.0f)) return HYRF_ERR_INVALID_ARG;
  if (a->bg.mode == 1 && (a->bg.map_h <= 0 || a->bg.map_w <= 0 || a->bg.map_h > 4096 || a->bg.map_w > 4096))
    return HYRF_ERR_INVALID_ARG;
  if (a->bg.mode != 0 && a->bg.mode != 1 && a->bg.mode != 2) return HYRF_ERR_INVALID_ARG;
  if (a->bg.mode == 2) return a->features ? HYRF_ERR_INVALID_ARG : HYRF_OK;  // no field is read
  if (!make_fields(a->fields, F, false)) return HYRF_ERR_UNSUPPORTED;
  if (F.cm.bf16 && a->fields.rad.n_levels != 16) return HYRF_ERR_UNSUPPORTED;
  if (F.rad.u8 && (!F.cm.bf16 || a->bg.mode != 0)) return HYRF_ERR_UNSUPPORTED;
  if ((F.cm.f16 && (a->bg.mode != 0 || !(F.rad.f16 || F.rad.u8))) || (F.rad.f16 && !F.cm.f16))
    return HYRF_ERR_UNSUPPORTED;
  if (a->features && (a->bg.mode != 0 || !F.cm.bf16 || !aligned(a->features, 16))) return HYRF_ERR_INVALID_ARG;
  if (!(a->bg.tau_T >= 0.0f)) return HYRF_ERR_INVALID_ARG;
  if (a->bg.tau_T > 0.0f && (a->bg.mode != 0 || !F.cm.bf16)) return HYRF_ERR_UNSUPPORTED;
  return HYRF_OK;
}

size_t hyrf_composite_background_workspace_size(const hyrf_composite_background_args* a) {
  if (a && a->bg.mode == 2) return 0;
  FieldsDev F;
  if (!a || !make_fields(a->fields, F, false)) return 0;
  return bg_workspace(*a, F, false);
}

hyrf_status hyrf_composite_background(const hyrf_composite_background_args* a, void* ws,
                                      size_t ws_bytes, void* stream) {
  FieldsDev F;
  hyrf_status st = bg_check(a, F);
  if (st != HYRF_OK) return st;
  if (a->bg.mode == 2) return a->C ? launch_bg_none(*a, S(stream)) : HYRF_ERR_INVALID_ARG;
  if (!a->C || !ws_ok(ws, ws_bytes, bg_workspace(*a, F, false))) return HYRF_ERR_INVALID_ARG;
  if (!bf16_weights_ok(a->fields.col_mlp)) return HYRF_ERR_INVALID_ARG;
  if (a->bg.mode == 0 && F.cm.bf16) return launch_bg_exact_fwd_tc(*a, F, ws, S(stream));
  return launch_bg_fwd(*a, F, ws, S(stream));
}

hyrf_status hyrf_gather_background(const hyrf_composite_background_args* a, void* stream) {
  FieldsDev F;
  hyrf_status st = bg_check(a, F);
  if (st != HYRF_OK) return st;
  if (a->bg.mode != 0 || !F.cm.bf16 || !a->features || a->bg.tau_T > 0.0f) return HYRF_ERR_INVALID_ARG;
  return launch_bg_gather(*a, F, S(stream));
}

size_t hyrf_composite_background_backward_workspace_size(
    const hyrf_composite_background_backward_args* b) {
  if (b && b->fwd.bg.mode == 2) return 0;
  FieldsDev F;
  if (!b || !make_fields(b->fwd.fields, F, false)) return 0;
  return bg_workspace(b->fwd, F, true);
}

hyrf_status hyrf_composite_background_backward(const hyrf_composite_background_backward_args* b,
                                               void* ws, size_t ws_bytes, void* stream) {
  if (!b) return HYRF_ERR_INVALID_ARG;
  FieldsDev F;
  hyrf_status st = bg_check(&b->fwd, F);
  if (st != HYRF_OK) return st;
  if (!b->d_C || !(b->loss_scale > 0.0f)) return HYRF_ERR_INVALID_ARG;
  if (b->fwd.bg.mode == 2) return launch_bg_none_bwd(*b, S(stream));
  if (b->fwd.bg.tau_T > 0.0f) return HYRF_ERR_INVALID_ARG;  // render-only rule
  if (F.rad.u8 || F.rad.f16 || F.cm.f16) return HYRF_ERR_UNSUPPORTED;  // render-only types
  if (!ws_ok(ws, ws_bytes, bg_workspace(b->fwd, F, true))) return HYRF_ERR_INVALID_ARG;
  if (!bf16_weights_ok(b->fwd.fields.col_mlp)) return HYRF_ERR_INVALID_ARG;
  if (b->fwd.bg.mode == 0 && F.cm.bf16) return launch_bg_bwd_tc(*b, F, ws, S(stream));
  return launch_bg_bwd(*b, F, ws, S(stream));
}

// ------------------------------------------------------------------ loss

size_t hyrf_loss_workspace_size(const hyrf_loss_args* a) { return a ? loss_workspace(*a) : 0; }

hyrf_status hyrf_loss(const hyrf_loss_args* a, void* ws, size_t ws_bytes, void* stream) {
  if (!a || a->width <= 0 || a->height <= 0 || !a->C || !a->target || !a->loss) return HYRF_ERR_INVALID_ARG;
  if (!(a->lambda >= 0.0f && a->lambda <= 1.0f)) return HYRF_ERR_INVALID_ARG;
  if (!ws_ok(ws, ws_bytes, loss_workspace(*a))) return HYRF_ERR_INVALID_ARG;
  return launch_loss(*a, ws, S(stream));
}

// ------------------------------------------------------------------ misc

hyrf_status hyrf_read_status(const int32_t* status, void* stream, int32_t* host_out) {
  if (!status || !host_out) return HYRF_ERR_INVALID_ARG;
  if (cudaMemcpyAsync(host_out, status, sizeof(int32_t), cudaMemcpyDeviceToHost, S(stream)) != cudaSuccess)
    return HYRF_ERR_CUDA;
  if (cudaStreamSynchronize(S(stream)) != cudaSuccess) return HYRF_ERR_CUDA;
  return static_cast<hyrf_status>(*host_out);
}

const char* hyrf_error_string(int32_t st) {
  if (st == HYRF_OK) return "ok";
  if (st & HYRF_ERR_CUDA) return "CUDA launch or copy failed";
  if (st & HYRF_ERR_INVALID_ARG) return "invalid argument";
  if (st & HYRF_ERR_UNSUPPORTED) return "unsupported configuration";
  if (st & HYRF_ERR_OVERFLOW) return "tile instances exceeded the capacity";
  if (st & HYRF_ERR_BOUNDS) return "an index read from memory was out of range";
  if (st & HYRF_ERR_TIMEOUT) return "a bounded wait on a tensor-core completion gave up";
  return "unknown status";
}

uint64_t hyrf_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

void hyrf_timer_enable(int on) { hyrf::g_timer_on.store(on != 0, std::memory_order_relaxed); }

int hyrf_timer_read(hyrf_kernel_time* out, int max_entries) {
  using namespace hyrf;
  std::lock_guard<std::mutex> lock(g_timer_mu);
  for (const TimedLaunch& t : g_pending) {
    float ms = 0.0f;
    if (cudaEventSynchronize(t.b) != cudaSuccess || cudaEventElapsedTime(&ms, t.a, t.b) != cudaSuccess) {
      cudaGetLastError();
      ms = 0.0f;
    }
    KernelTotal* k = nullptr;
    for (KernelTotal& x : g_totals)
      if (std::strcmp(x.name, t.name) == 0) k = &x;
    if (!k) {
      g_totals.push_back({t.name, 0, 0.0});
      k = &g_totals.back();
    }
    k->launches += 1;
    k->ms += ms;
    g_free_events.push_back(t.a);
    g_free_events.push_back(t.b);
  }
  g_pending.clear();
  const int n = (int)g_totals.size();
  for (int i = 0; out && i < n && i < max_entries; ++i)
    out[i] = {g_totals[i].name, g_totals[i].launches, g_totals[i].ms};
  g_totals.clear();
  return n;
}

}  // extern "C"
