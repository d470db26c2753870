// C ABI of the tracking library (include/dri.h): argument checks, the stream's
// device workspace, IMU bookkeeping on the host and the per-frame launch
// sequence.  All arithmetic of a frame runs in the kernels of maps.cu,
// track.cu and solve.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "dri_internal.h"

using namespace dri;

namespace {

constexpr size_t kAlign = 256;
inline size_t align_up(size_t v, size_t a = kAlign) { return (v + a - 1) / a * a; }

int valid_config(const dri_stream_config* c) {
  if (!c) return DRI_EINVAL;
  if (c->width < 8 || c->height < 8 || c->width > 8192 || c->height > 8192) return DRI_EINVAL;
  if (c->levels < 1 || c->levels > kMaxLevels) return DRI_EINVAL;
  if ((c->width >> (c->levels - 1)) < 4 || (c->height >> (c->levels - 1)) < 4) return DRI_EINVAL;
  for (int l = 0; l < c->levels; ++l)
    if (c->iters[l] < 0 || c->iters[l] > 1000) return DRI_EINVAL;
  if (!(c->fx > 0) || !(c->fy > 0) || !std::isfinite(c->cx) || !std::isfinite(c->cy)) return DRI_EINVAL;
  if (!(c->sigma_I > 0) || !(c->sigma_d > 0) || !(c->gyr_nd > 0) || !(c->acc_nd > 0)) return DRI_EINVAL;
  if (!(c->gyr_rw > 0) || !(c->acc_rw > 0) || !(c->g > 0) || !(c->sigma_grav_rw > 0)) return DRI_EINVAL;
  for (int i = 0; i < 5; ++i)
    if (!(c->prior_sigma[i] > 0)) return DRI_EINVAL;
  if (!(c->icp_dist_thr > 0) || !(c->icp_angle_thr_deg > 0) || !(c->icp_angle_thr_deg < 180))
    return DRI_EINVAL;
  if (!(c->depth_min >= 0) || !(c->depth_max > c->depth_min)) return DRI_EINVAL;
  if (c->max_imu < 2 || c->max_imu > 65536) return DRI_EINVAL;
  const double qn = c->T_CS[3] * c->T_CS[3] + c->T_CS[4] * c->T_CS[4] + c->T_CS[5] * c->T_CS[5] +
                    c->T_CS[6] * c->T_CS[6];
  if (!(std::fabs(qn - 1.0) < 1e-6)) return DRI_EINVAL;
  return DRI_OK;
}

void quat_to_rot_h(const double* q, double* R) {
  const double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  const double w = q[0] / n, x = q[1] / n, y = q[2] / n, z = q[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

DState to_dstate(const dri_state& s) {
  DState d;
  for (int i = 0; i < 3; ++i) {
    d.r[i] = s.r_WC[i];
    d.v[i] = s.v_I[i];
    d.bg[i] = s.bg[i];
    d.ba[i] = s.ba[i];
  }
  double nq = 0, ng = 0;
  for (int i = 0; i < 4; ++i) {
    nq += s.q_WC[i] * s.q_WC[i];
    ng += s.q_IW[i] * s.q_IW[i];
  }
  nq = std::sqrt(nq);
  ng = std::sqrt(ng);
  for (int i = 0; i < 4; ++i) {
    d.q[i] = s.q_WC[i] / nq;
    d.qg[i] = s.q_IW[i] / ng;
  }
  return d;
}

dri_state from_dstate(const DState& d, double t) {
  dri_state s;
  for (int i = 0; i < 3; ++i) {
    s.r_WC[i] = d.r[i];
    s.v_I[i] = d.v[i];
    s.bg[i] = d.bg[i];
    s.ba[i] = d.ba[i];
  }
  for (int i = 0; i < 4; ++i) {
    s.q_WC[i] = d.q[i];
    s.q_IW[i] = d.qg[i];
  }
  s.t = t;
  return s;
}

bool finite_state(const dri_state& s) {
  const double* p = reinterpret_cast<const double*>(&s);
  for (size_t i = 0; i < sizeof(dri_state) / sizeof(double) - 1; ++i)
    if (!std::isfinite(p[i])) return false;
  double nq = 0, ng = 0;
  for (int i = 0; i < 4; ++i) {
    nq += s.q_WC[i] * s.q_WC[i];
    ng += s.q_IW[i] * s.q_IW[i];
  }
  return nq > 1e-12 && ng > 1e-12;
}

}  // namespace

namespace dri {

LevelGeom level_geom(const dri_stream_config& cfg, int level) {
  LevelGeom g;
  const double s = std::ldexp(1.0, level);
  g.w = cfg.width >> level;
  g.h = cfg.height >> level;
  g.fx = (float)(cfg.fx / s);
  g.fy = (float)(cfg.fy / s);
  g.cx = (float)((cfg.cx + 0.5) / s - 0.5);
  g.cy = (float)((cfg.cy + 0.5) / s - 0.5);
  g.ifx = (float)(s / cfg.fx);
  g.ify = (float)(s / cfg.fy);
  return g;
}

StreamLayout make_layout(const dri_stream_config& cfg) {
  StreamLayout L;
  std::memset(&L, 0, sizeof(L));
  const bool fp16 = (cfg.precision_flags & DRI_FP16_MAPS) != 0;
  const bool fp32p = (cfg.precision_flags & DRI_FP32_PARTIALS) != 0;
  L.map_elem_bytes = fp16 ? 2 : 4;
  L.imu_cap = cfg.max_imu;
  size_t off = 0;
  L.ctrl = off;
  off = align_up(off + sizeof(Ctrl));
  L.imu = off;
  off = align_up(off + sizeof(ImuHeader) + (size_t)L.imu_cap * sizeof(dri_imu_sample));
  const size_t npx = (size_t)cfg.width * cfg.height;
  L.in_depth = off;
  off = align_up(off + npx * 4);
  L.in_inten = off;
  off = align_up(off + npx * 4);
  for (int l = 0; l < cfg.levels; ++l) {
    const size_t n = (size_t)(cfg.width >> l) * (cfg.height >> l);
    const size_t plane = (n + 63) / 64 * 64;
    L.plane[l] = (int64_t)plane;
    for (int s = 0; s < 2; ++s) {
      L.level_off[l][s][0] = off;
      off = align_up(off + plane * 4);
      L.level_off[l][s][1] = off;
      off = align_up(off + 3 * plane * L.map_elem_bytes);
      L.level_off[l][s][2] = off;
      off = align_up(off + plane * 4);
      L.level_off[l][s][3] = off;
      off = align_up(off + 2 * plane * L.map_elem_bytes);
    }
  }
  int maxb = 1;
  for (int l = 0; l < cfg.levels; ++l)
    maxb = std::max(maxb, track_grid_blocks(cfg.width >> l, cfg.height >> l, 1));
  L.max_blocks = maxb;
  L.counters = off;
  off = align_up(off + (size_t)(1 + fold_groups(maxb)) * sizeof(uint32_t));
  L.partials = off;
  off = align_up(off + (size_t)maxb * kSumsAll * (fp32p ? 4 : 8));
  L.gpartials = off;
  off = align_up(off + (size_t)fold_groups(maxb) * kSumsAll * (fp32p ? 4 : 8));
  L.flags = off;
  off = align_up(off + npx);
  L.lin_out = off;
  off = align_up(off + sizeof(dri_linearisation));
  L.total = off;
  return L;
}

}  // namespace dri

struct dri_stream_s {
  dri_stream_config cfg;
  StreamLayout L;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  bool own_ws = false;
  Ctrl* ctrl = nullptr;
  ImuHeader* imu_dev = nullptr;
  float* in_depth = nullptr;
  float* in_inten = nullptr;
  void* partials = nullptr;
  void* gpartials = nullptr;
  uint32_t* counters = nullptr;
  uint8_t* flags = nullptr;
  dri_linearisation* lin_dev = nullptr;
  LevelMaps maps[kMaxLevels];
  LevelGeom geom[kMaxLevels];
  int ppt[kMaxLevels];
  DState x_init;
  // host bookkeeping
  std::vector<dri_imu_sample> imu;
  bool initialised = false;        // host view: the init frame was enqueued
  double t_prev = 0.0;             // time of the state the next frame starts from
  double t_frame = 0.0;
  bool frame_pending = false;
  char* pin_imu = nullptr;         // pinned staging, one slot per frame in flight (+1)
  size_t imu_slot_bytes = 0;
  Ctrl* pin_ctrl = nullptr;        // pinned copy of the whole control block
  // frames in flight: each copies its result head into a pinned ring slot and
  // records an event; completed frames are settled in order on the host
  static constexpr int kRing = 64;
  char* pin_ring = nullptr;        // kRing result heads
  cudaEvent_t ring_ev[kRing] = {};
  struct InFlight { int slot; };
  std::deque<InFlight> inflight;
  int ring_next = 0;
  double t_confirmed = 0.0;        // time of the last state known to be good
  int64_t frames_ok = 0, frames_failed = 0;
  double t_prev_before = 0.0;      // t_prev before the last optimistic advance
  int64_t launches = 0;
  int64_t h2d_last = 0, d2h_last = 0;   // bytes copied for the last frame
  // profiling: event pairs around launches
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec { int cls; size_t e0, e1; double pixels; };
  std::vector<Rec> recs;
  dri_profile counted;
};

namespace {

constexpr size_t kMaxTimed = 65536;

cudaEvent_t prof_event(dri_stream_s* s, size_t* idx) {
  if (s->ev_used == s->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    s->ev_pool.push_back(e);
  }
  *idx = s->ev_used;
  return s->ev_pool[s->ev_used++];
}

// Runs one kernel launcher; counts it and, while profiling, brackets it with events.
template <class F>
cudaError_t launch(dri_stream_s* s, int cls, double pixels, F&& f) {
  s->launches++;
  if (!s->profiling) return f();
  s->counted.launches[cls]++;
  s->counted.pixels[cls] += pixels;
  if (s->recs.size() >= kMaxTimed) return f();
  size_t i0 = 0, i1 = 0;
  cudaEvent_t e0 = prof_event(s, &i0);
  cudaEvent_t e1 = e0 ? prof_event(s, &i1) : nullptr;
  if (!e0 || !e1) return f();
  cudaEventRecord(e0, s->stream);
  cudaError_t r = f();
  cudaEventRecord(e1, s->stream);
  s->recs.push_back({cls, i0, i1, pixels});
  return r;
}

SolveParams solve_params(const dri_stream_s* s, int level, int last) {
  SolveParams p;
  std::memset(&p, 0, sizeof(p));
  p.ctrl = s->ctrl;
  p.imu = s->imu_dev;
  p.level = level;
  p.last = last;
  const dri_stream_config& c = s->cfg;
  double R[9];
  quat_to_rot_h(c.T_CS + 3, R);
  for (int i = 0; i < 9; ++i) p.R_CS[i] = R[i];
  for (int i = 0; i < 3; ++i) p.r_CS[i] = c.T_CS[i];
  p.W_icp = 1.0 / (c.sigma_d * c.sigma_d);
  p.W_rgb = 1.0 / (c.sigma_I * c.sigma_I);
  p.gyr_nd = c.gyr_nd;
  p.acc_nd = c.acc_nd;
  p.gyr_rw = c.gyr_rw;
  p.acc_rw = c.acc_rw;
  p.g = c.g;
  p.sigma_grav = c.sigma_grav_rw;
  for (int i = 0; i < 5; ++i) p.prior_sigma[i] = c.prior_sigma[i];
  p.min_valid = c.min_valid;
  p.imu_cap = s->L.imu_cap;
  return p;
}

TrackParams track_params(const dri_stream_s* s, int level, uint8_t* flags) {
  TrackParams p;
  std::memset(&p, 0, sizeof(p));
  p.g = s->geom[level];
  p.m = s->maps[level];
  p.ctrl = s->ctrl;
  p.partials = s->partials;
  p.gpartials = s->gpartials;
  p.counters = s->counters;
  p.flags = flags;
  p.ppt = s->ppt[level];
  p.nblocks = track_grid_blocks(p.g.w, p.g.h, p.ppt);
  p.depth_min = (float)s->cfg.depth_min;
  p.depth_max = (float)s->cfg.depth_max;
  p.icp_dist2 = (float)(s->cfg.icp_dist_thr * s->cfg.icp_dist_thr);
  p.icp_cos = (float)std::cos(s->cfg.icp_angle_thr_deg * 3.14159265358979323846 / 180.0);
  return p;
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return DRI_ECUDA;       \
  } while (0)

// Level maps of the uploaded frame in the live map set.
int enqueue_maps(dri_stream_s* s) {
  const bool fp16 = (s->cfg.precision_flags & DRI_FP16_MAPS) != 0;
  const double npx = (double)s->cfg.width * s->cfg.height;
  CK(launch(s, DRI_KC_MAPS, npx, [&] {
    return launch_copy_input(s->in_depth, s->in_inten, s->maps[0], s->ctrl, s->cfg.width,
                             s->cfg.height, s->stream);
  }));
  for (int l = 1; l < s->cfg.levels; ++l) {
    CK(launch(s, DRI_KC_MAPS, (double)s->geom[l].w * s->geom[l].h, [&] {
      return launch_pyr_down(s->maps[l - 1], s->maps[l], s->ctrl, s->geom[l - 1].w,
                             s->geom[l - 1].h, s->geom[l].w, s->geom[l].h, s->stream);
    }));
  }
  for (int l = 0; l < s->cfg.levels; ++l) {
    CK(launch(s, DRI_KC_MAPS, (double)s->geom[l].w * s->geom[l].h, [&] {
      return launch_normals(s->maps[l], s->ctrl, s->geom[l], (float)s->cfg.depth_min,
                            (float)s->cfg.depth_max, fp16, -1, s->stream);
    }));
  }
  return DRI_OK;
}

int enqueue_gradients(dri_stream_s* s) {
  const bool fp16 = (s->cfg.precision_flags & DRI_FP16_MAPS) != 0;
  for (int l = 0; l < s->cfg.levels; ++l) {
    CK(launch(s, DRI_KC_GRAD, (double)s->geom[l].w * s->geom[l].h, [&] {
      return launch_gradient(s->maps[l], s->ctrl, s->geom[l].w, s->geom[l].h, fp16, s->stream);
    }));
  }
  return DRI_OK;
}

// Stage header + samples covering [t0, t1] and copy them to the device.
int stage_imu(dri_stream_s* s, int slot, double t0, double t1, bool need_cover) {
  ImuHeader h;
  std::memset(&h, 0, sizeof(h));
  h.t0 = t0;
  h.t1 = t1;
  size_t k0 = 0, k1 = 0;
  if (need_cover) {
    const auto& v = s->imu;
    if (v.empty() || v.front().t > t0 || v.back().t < t1) return DRI_ENOTREADY;
    size_t a = 0;
    while (a + 1 < v.size() && v[a + 1].t <= t0) ++a;
    size_t b = a;
    while (b < v.size() && v[b].t < t1) ++b;
    if (b >= v.size()) return DRI_ENOTREADY;
    k0 = a;
    k1 = b + 1;
    if ((int64_t)(k1 - k0) > s->L.imu_cap) return DRI_ENOMEM;
    if ((int64_t)(k1 - k0) - 1 > solver_max_imu_pieces()) return DRI_ENOMEM;
    h.n = (int32_t)(k1 - k0);
  }
  // a slot is rewritten only after the frame that last used it has completed
  char* stage = s->pin_imu + (size_t)slot * s->imu_slot_bytes;
  std::memcpy(stage, &h, sizeof(h));
  if (h.n) std::memcpy(stage + sizeof(h), s->imu.data() + k0, (size_t)h.n * sizeof(dri_imu_sample));
  CK(cudaMemcpyAsync(s->imu_dev, stage, sizeof(h) + (size_t)h.n * sizeof(dri_imu_sample),
                     cudaMemcpyHostToDevice, s->stream));
  s->h2d_last += (int64_t)(sizeof(h) + (size_t)h.n * sizeof(dri_imu_sample));
  return DRI_OK;
}

const Ctrl* ring_head(const dri_stream_s* s, int slot) {
  return reinterpret_cast<const Ctrl*>(s->pin_ring + (size_t)slot * kCtrlHeadBytes);
}

// Settles, in order, the frames whose result copy has completed (all of them
// when wait is set): a failed frame rolls the host's start time back to the
// state the device kept.
int settle(dri_stream_s* s, bool wait) {
  while (!s->inflight.empty()) {
    const int slot = s->inflight.front().slot;
    cudaError_t q = wait ? cudaEventSynchronize(s->ring_ev[slot]) : cudaEventQuery(s->ring_ev[slot]);
    if (q == cudaErrorNotReady) return DRI_OK;
    if (q != cudaSuccess) return DRI_ECUDA;
    const Ctrl* h = ring_head(s, slot);
    s->t_confirmed = h->t_state;
    if (h->status != DRI_OK) {
      s->t_prev = h->t_state;
      s->frames_failed++;
    } else {
      s->frames_ok++;
    }
    s->inflight.pop_front();
  }
  return DRI_OK;
}

}  // namespace

extern "C" {

const char* dri_status_string(int code) {
  switch (code) {
    case DRI_OK: return "ok";
    case DRI_EINVAL: return "invalid argument";
    case DRI_ENOMEM: return "out of memory";
    case DRI_EADMIT: return "over the HBM budget";
    case DRI_ENOTREADY: return "frame or IMU coverage missing";
    case DRI_ELOST: return "tracking lost";
    case DRI_ETIMEDOUT: return "bounded wait expired";
    case DRI_ECUDA: return "CUDA error";
    default: return "unknown status";
  }
}

int dri_config_default(int32_t width, int32_t height, dri_stream_config* cfg) {
  if (!cfg || width < 8 || height < 8 || width > 8192 || height > 8192) return DRI_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->width = width;
  cfg->height = height;
  cfg->fx = cfg->fy = 277.0 * width / 320.0;
  cfg->cx = width / 2.0;
  cfg->cy = height / 2.0;
  cfg->levels = 3;
  cfg->iters[0] = 10;
  cfg->iters[1] = 5;
  cfg->iters[2] = 4;
  cfg->T_CS[3] = 1.0;
  cfg->sigma_I = 0.01;
  cfg->sigma_d = 0.002;
  cfg->gyr_nd = 12.0e-4;
  cfg->acc_nd = 8.0e-3;
  cfg->gyr_rw = 4.0e-6;
  cfg->acc_rw = 2.0e-5;
  cfg->g = 9.81;
  cfg->sigma_grav_rw = 1e-4;
  cfg->prior_sigma[0] = 1e-6;
  cfg->prior_sigma[1] = 0.1;
  cfg->prior_sigma[2] = 0.03;
  cfg->prior_sigma[3] = 0.1;
  cfg->prior_sigma[4] = 0.1;
  cfg->icp_dist_thr = 0.10;
  cfg->icp_angle_thr_deg = 20.0;
  cfg->depth_min = 0.3;
  cfg->depth_max = 8.0;
  cfg->min_valid = 64;
  cfg->precision_flags = 0;
  cfg->max_imu = 512;
  return DRI_OK;
}

int dri_stream_workspace_bytes(const dri_stream_config* cfg, size_t* bytes) {
  if (!bytes) return DRI_EINVAL;
  const int v = valid_config(cfg);
  if (v != DRI_OK) return v;
  *bytes = make_layout(*cfg).total;
  return DRI_OK;
}

int dri_create_stream(const dri_stream_config* cfg, const dri_state* x_init, void* cuda_stream,
                      void* workspace, size_t workspace_bytes, dri_stream* out) {
  if (!out || !x_init) return DRI_EINVAL;
  *out = nullptr;
  int v = valid_config(cfg);
  if (v != DRI_OK) return v;
  if (!finite_state(*x_init)) return DRI_EINVAL;
  StreamLayout L = make_layout(*cfg);
  if (prepare_solver_kernels() != cudaSuccess) return DRI_ECUDA;
  if (workspace && (workspace_bytes < L.total || ((uintptr_t)workspace % kAlign) != 0))
    return DRI_EINVAL;
  dri_stream_s* s = new (std::nothrow) dri_stream_s();
  if (!s) return DRI_ENOMEM;
  s->cfg = *cfg;
  s->L = L;
  s->stream = (cudaStream_t)cuda_stream;
  if (workspace) {
    s->ws = (char*)workspace;
  } else {
    if (cudaMalloc(&s->ws, L.total) != cudaSuccess) {
      delete s;
      return DRI_ENOMEM;
    }
    s->own_ws = true;
  }
  s->imu_slot_bytes = align_up(sizeof(ImuHeader) + (size_t)L.imu_cap * sizeof(dri_imu_sample), 64);
  if (cudaMallocHost(&s->pin_imu, (size_t)(dri_stream_s::kRing + 1) * s->imu_slot_bytes) != cudaSuccess ||
      cudaMallocHost(&s->pin_ctrl, sizeof(Ctrl)) != cudaSuccess ||
      cudaMallocHost(&s->pin_ring, (size_t)dri_stream_s::kRing * kCtrlHeadBytes) != cudaSuccess) {
    dri_destroy_stream(s);
    return DRI_ENOMEM;
  }
  for (int i = 0; i < dri_stream_s::kRing; ++i) {
    if (cudaEventCreateWithFlags(&s->ring_ev[i], cudaEventDisableTiming) != cudaSuccess) {
      dri_destroy_stream(s);
      return DRI_ENOMEM;
    }
  }
  s->ctrl = (Ctrl*)(s->ws + L.ctrl);
  s->imu_dev = (ImuHeader*)(s->ws + L.imu);
  s->in_depth = (float*)(s->ws + L.in_depth);
  s->in_inten = (float*)(s->ws + L.in_inten);
  s->partials = (void*)(s->ws + L.partials);
  s->gpartials = (void*)(s->ws + L.gpartials);
  s->counters = (uint32_t*)(s->ws + L.counters);
  s->flags = (uint8_t*)(s->ws + L.flags);
  s->lin_dev = (dri_linearisation*)(s->ws + L.lin_out);
  for (int l = 0; l < cfg->levels; ++l) {
    s->geom[l] = level_geom(*cfg, l);
    LevelMaps& m = s->maps[l];
    m.plane = L.plane[l];
    for (int k = 0; k < 2; ++k) {
      m.depth[k] = (float*)(s->ws + L.level_off[l][k][0]);
      m.normal[k] = (void*)(s->ws + L.level_off[l][k][1]);
      m.inten[k] = (float*)(s->ws + L.level_off[l][k][2]);
      m.grad[k] = (void*)(s->ws + L.level_off[l][k][3]);
    }
    s->ppt[l] = track_default_ppt(s->geom[l].w, s->geom[l].h);
  }
  s->x_init = to_dstate(*x_init);
  // control block: zero, then the initial state
  Ctrl* h = s->pin_ctrl;
  std::memset(h, 0, sizeof(Ctrl));
  h->x = s->x_init;
  h->x0 = h->x1 = h->xbar = h->xstart = h->x;
  h->ref_index = 0;
  h->t_state = x_init->t;
  if (cudaMemcpyAsync(s->ctrl, h, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream) != cudaSuccess ||
      cudaMemsetAsync(s->ws + L.level_off[0][0][0], 0, L.flags - L.level_off[0][0][0], s->stream) !=
          cudaSuccess ||
      cudaStreamSynchronize(s->stream) != cudaSuccess) {
    dri_destroy_stream(s);
    return DRI_ECUDA;
  }
  *out = s;
  return DRI_OK;
}

int dri_destroy_stream(dri_stream s) {
  if (!s) return DRI_EINVAL;
  if (s->stream || s->ws) cudaStreamSynchronize(s->stream);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  if (s->pin_imu) cudaFreeHost(s->pin_imu);
  if (s->pin_ctrl) cudaFreeHost(s->pin_ctrl);
  if (s->pin_ring) cudaFreeHost(s->pin_ring);
  for (int i = 0; i < dri_stream_s::kRing; ++i)
    if (s->ring_ev[i]) cudaEventDestroy(s->ring_ev[i]);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  delete s;
  return DRI_OK;
}

int dri_upload_frame(dri_stream s, double t, const float* depth, const float* intensity,
                     size_t pitch_bytes, int32_t mem_kind) {
  if (!s || !depth || !intensity || !std::isfinite(t)) return DRI_EINVAL;
  if (mem_kind != DRI_HOST && mem_kind != DRI_DEVICE) return DRI_EINVAL;
  const size_t row = (size_t)s->cfg.width * sizeof(float);
  const size_t pitch = pitch_bytes ? pitch_bytes : row;
  if (pitch < row) return DRI_EINVAL;
  if (s->initialised && !(t > s->t_prev)) return DRI_EINVAL;
  const cudaMemcpyKind kind = mem_kind == DRI_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  s->h2d_last = mem_kind == DRI_HOST ? (int64_t)(2 * row * s->cfg.height) : 0;
  CK(cudaMemcpy2DAsync(s->in_depth, row, depth, pitch, row, s->cfg.height, kind, s->stream));
  CK(cudaMemcpy2DAsync(s->in_inten, row, intensity, pitch, row, s->cfg.height, kind, s->stream));
  s->t_frame = t;
  s->frame_pending = true;
  return DRI_OK;
}

int dri_push_imu(dri_stream s, const dri_imu_sample* samples, size_t n) {
  if (!s || (n && !samples)) return DRI_EINVAL;
  double last = s->imu.empty() ? -INFINITY : s->imu.back().t;
  for (size_t i = 0; i < n; ++i) {
    const dri_imu_sample& m = samples[i];
    bool ok = std::isfinite(m.t) && m.t > last;
    for (int k = 0; k < 3; ++k) ok = ok && std::isfinite(m.gyr[k]) && std::isfinite(m.acc[k]);
    if (!ok) return DRI_EINVAL;
    last = m.t;
  }
  s->imu.insert(s->imu.end(), samples, samples + n);
  return DRI_OK;
}

static int fill_result(dri_stream s, const Ctrl* h, dri_track_result* out, bool init) {
  std::memset(out, 0, sizeof(*out));
  out->x1 = from_dstate(h->x, h->t_state);
  out->x0 = from_dstate(h->x0, s->t_prev_before);
  for (int l = 0; l < kMaxLevels; ++l) {
    out->n_icp[l] = h->n_icp[l];
    out->n_rgb[l] = h->n_rgb[l];
  }
  out->cost = h->cost;
  out->status = h->status;
  out->initialised = init ? 1 : 0;
  return h->status;
}

int dri_track(dri_stream s, dri_track_result* out) {
  if (!s) return DRI_EINVAL;
  if (!s->frame_pending) return DRI_ENOTREADY;
  if (settle(s, false) != DRI_OK) return DRI_ECUDA;
  if ((int)s->inflight.size() >= dri_stream_s::kRing) {
    // ring full: wait for the oldest frame only, so its slots can be reused
    CK(cudaEventSynchronize(s->ring_ev[s->inflight.front().slot]));
    if (settle(s, false) != DRI_OK) return DRI_ECUDA;
  }
  const bool init = !s->initialised;
  const int slot = s->ring_next;   // staging + result slot of this frame
  if (init) {
    int r = stage_imu(s, slot, s->t_frame, s->t_frame, false);
    if (r != DRI_OK) return r;
    if ((r = enqueue_maps(s)) != DRI_OK) return r;
    CK(launch(s, DRI_KC_FRAME, 0.0, [&] { return launch_frame_init(solve_params(s, 0, 0), s->stream); }));
    if ((r = enqueue_gradients(s)) != DRI_OK) return r;
    s->initialised = true;
    s->t_prev_before = s->t_frame;
    s->t_prev = s->t_frame;
    s->t_confirmed = s->t_frame;
  } else {
    int r = stage_imu(s, slot, s->t_prev, s->t_frame, true);
    if (r != DRI_OK) return r;
    if ((r = enqueue_maps(s)) != DRI_OK) return r;
    CK(launch(s, DRI_KC_FRAME, 0.0, [&] { return launch_frame_begin(solve_params(s, 0, 0), s->stream); }));
    int remaining = 0;
    for (int l = 0; l < s->cfg.levels; ++l) remaining += s->cfg.iters[l];
    for (int l = s->cfg.levels - 1; l >= 0; --l) {
      const TrackParams tp = track_params(s, l, nullptr);
      const bool fp16 = (s->cfg.precision_flags & DRI_FP16_MAPS) != 0;
      const bool fp32p = (s->cfg.precision_flags & DRI_FP32_PARTIALS) != 0;
      for (int it = 0; it < s->cfg.iters[l]; ++it) {
        --remaining;
        CK(launch(s, DRI_KC_TRACK, (double)tp.g.w * tp.g.h,
                  [&] { return launch_track(tp, fp16, fp32p, s->stream); }));
        CK(launch(s, DRI_KC_SOLVE, 0.0,
                  [&] { return launch_gn_step(solve_params(s, l, remaining == 0), s->stream); }));
      }
    }
    CK(launch(s, DRI_KC_FRAME, 0.0, [&] { return launch_frame_end(solve_params(s, 0, 0), s->stream); }));
    if ((r = enqueue_gradients(s)) != DRI_OK) return r;
    // drop samples no later frame can need: all before the one covering the
    // earliest time a frame may still start from (a failed frame in flight
    // rolls the start back to t_confirmed)
    const double keep_from = std::min(s->t_prev, s->t_confirmed);
    size_t a = 0;
    while (a + 1 < s->imu.size() && s->imu[a + 1].t <= keep_from) ++a;
    if (a) s->imu.erase(s->imu.begin(), s->imu.begin() + a);
    s->t_prev_before = s->t_prev;
    s->t_prev = s->t_frame;   // optimistic; rolled back when the frame is known to fail
  }
  s->frame_pending = false;
  s->ring_next = (s->ring_next + 1) % dri_stream_s::kRing;
  CK(cudaMemcpyAsync(s->pin_ring + (size_t)slot * kCtrlHeadBytes, s->ctrl, kCtrlHeadBytes,
                     cudaMemcpyDeviceToHost, s->stream));
  s->d2h_last = (int64_t)kCtrlHeadBytes;
  CK(cudaEventRecord(s->ring_ev[slot], s->stream));
  s->inflight.push_back({slot});
  if (!out) return DRI_OK;
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  return fill_result(s, ring_head(s, slot), out, init);
}

int dri_get_state(dri_stream s, dri_state* x1, double* H_prior, double* b_prior) {
  if (!s || !x1) return DRI_EINVAL;
  CK(cudaMemcpyAsync(s->pin_ctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  const Ctrl* h = s->pin_ctrl;
  *x1 = from_dstate(h->x, h->t_state);
  if (H_prior) std::memcpy(H_prior, h->Hs, sizeof(h->Hs));
  if (b_prior) std::memcpy(b_prior, h->bs, sizeof(h->bs));
  return DRI_OK;
}

int dri_set_state(dri_stream s, const dri_state* x1, const double* H_prior, const double* b_prior) {
  if (!s || !x1 || !finite_state(*x1)) return DRI_EINVAL;
  CK(cudaMemcpyAsync(s->pin_ctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  Ctrl* h = s->pin_ctrl;
  h->x = to_dstate(*x1);
  h->xbar = h->x;
  h->t_state = x1->t;
  if (H_prior) std::memcpy(h->Hs, H_prior, sizeof(h->Hs));
  if (b_prior) std::memcpy(h->bs, b_prior, sizeof(h->bs));
  h->status = DRI_OK;
  CK(cudaMemcpyAsync(s->ctrl, h, sizeof(Ctrl), cudaMemcpyHostToDevice, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  s->t_prev = x1->t;
  s->t_confirmed = x1->t;
  return DRI_OK;
}

int dri_linearise(dri_stream s, int32_t level, const dri_state* x0, const dri_state* x1,
                  dri_linearisation* out, uint8_t* flags) {
  if (!s || !x0 || !x1 || !out || level < 0 || level >= s->cfg.levels) return DRI_EINVAL;
  if (!finite_state(*x0) || !finite_state(*x1)) return DRI_EINVAL;
  if (!s->initialised || !s->frame_pending) return DRI_ENOTREADY;
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  int r = stage_imu(s, dri_stream_s::kRing, s->t_prev, s->t_frame, true);
  if (r != DRI_OK) return r;
  if ((r = enqueue_maps(s)) != DRI_OK) return r;
  const SolveParams sp = solve_params(s, level, 0);
  const bool fp16 = (s->cfg.precision_flags & DRI_FP16_MAPS) != 0;
  const bool fp32p = (s->cfg.precision_flags & DRI_FP32_PARTIALS) != 0;
  const TrackParams tp = track_params(s, level, flags ? s->flags : nullptr);
  CK(launch(s, DRI_KC_FRAME, 0.0,
            [&] { return launch_linearise_begin(sp, to_dstate(*x0), to_dstate(*x1), s->stream); }));
  CK(launch(s, DRI_KC_TRACK, (double)tp.g.w * tp.g.h, [&] { return launch_track(tp, fp16, fp32p, s->stream); }));
  CK(launch(s, DRI_KC_SOLVE, 0.0, [&] { return launch_linearise_end(sp, s->lin_dev, s->stream); }));
  CK(cudaMemcpyAsync(out, s->lin_dev, sizeof(*out), cudaMemcpyDeviceToHost, s->stream));
  if (flags) {
    const size_t n = (size_t)s->geom[level].w * s->geom[level].h;
    CK(cudaMemcpyAsync(flags, s->flags, n, cudaMemcpyDeviceToHost, s->stream));
  }
  CK(cudaMemcpyAsync(s->pin_ctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  return s->pin_ctrl->status;
}

int dri_profile_enable(dri_stream s, int32_t enable) {
  if (!s) return DRI_EINVAL;
  if (enable) {
    CK(cudaStreamSynchronize(s->stream));
    s->recs.clear();
    s->ev_used = 0;
    std::memset(&s->counted, 0, sizeof(s->counted));
  }
  s->profiling = enable != 0;
  return DRI_OK;
}

int dri_profile_read(dri_stream s, dri_profile* out) {
  if (!s || !out) return DRI_EINVAL;
  CK(cudaStreamSynchronize(s->stream));
  *out = s->counted;
  for (int k = 0; k < DRI_KC_COUNT; ++k) out->ms[k] = 0.0;
  for (const auto& r : s->recs) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->ev_pool[r.e0], s->ev_pool[r.e1]));
    out->ms[r.cls] += ms;
  }
  return DRI_OK;
}

int dri_frame_counts(dri_stream s, int64_t* ok, int64_t* failed) {
  if (!s || !ok || !failed) return DRI_EINVAL;
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  *ok = s->frames_ok;
  *failed = s->frames_failed;
  return DRI_OK;
}

int dri_io_bytes(dri_stream s, int64_t* h2d, int64_t* d2h) {
  if (!s || !h2d || !d2h) return DRI_EINVAL;
  *h2d = s->h2d_last;
  *d2h = s->d2h_last;
  return DRI_OK;
}

int dri_launch_count(dri_stream s, int64_t* count) {
  if (!s || !count) return DRI_EINVAL;
  *count = s->launches;
  return DRI_OK;
}

}  // extern "C"
