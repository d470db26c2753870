// C ABI of the tracking library (include/dri.h): argument checks, the stream's
// device workspace, IMU bookkeeping on the host and the per-frame launch
// sequence ("plan") over one stream (dri_track) or many (dri_track_batch),
// captured once as a CUDA graph and replayed per frame.  All arithmetic of a
// frame runs in the kernels of maps.cu, track.cu and solve.cu.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <vector>

#include <cuda_runtime.h>

#include "dri_internal.h"
#include "host.h"

using namespace dri;

namespace {

constexpr size_t kAlign = 256;
constexpr int kStreamRing = 64;   // frames of one stream in flight (dri_track, out = NULL)
constexpr int kBatchRing = 8;     // launches of one batch plan in flight
constexpr int kMaxBatch = 4096;
constexpr int kMaxRowsPerThread = 64;
constexpr int kMaxGroups = 8;     // slot groups of a batch plan's Gauss-Newton loop
constexpr size_t kImuDropBatch = 4096;   // consumed IMU samples dropped at once (~10 s at 400 Hz)
// Slot groups of a new batch plan: one per 16 slots, at most 4 (64 x 640x480:
// 1 group 10.3k frames/s, 2 11.8k, 3 12.1k, 4 12.3k, 5 11.1k).
inline int default_groups(int n) { return std::max(1, std::min(4, n / 16)); }
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
  // below 90 degrees: the angle test then also rejects a zero (invalid) normal
  if (!(c->icp_dist_thr > 0) || !(c->icp_angle_thr_deg > 0) || !(c->icp_angle_thr_deg < 90))
    return DRI_EINVAL;
  if (!(c->depth_min >= 0) || !(c->depth_max > c->depth_min)) return DRI_EINVAL;
  if (c->max_imu < 2 || c->max_imu > 65536) return DRI_EINVAL;
  if (c->imu_mode != DRI_IMU_REINTEGRATE && c->imu_mode != DRI_IMU_FIRST_ORDER) return DRI_EINVAL;
  if (!(c->bias_relin_g >= 0) || !(c->bias_relin_a >= 0) || !std::isfinite(c->bias_relin_g) ||
      !std::isfinite(c->bias_relin_a))
    return DRI_EINVAL;
  if (c->track_mode != DRI_TRACK_INERTIAL && c->track_mode != DRI_TRACK_RGBD_ONLY &&
      c->track_mode != DRI_TRACK_GYRO_ONLY)
    return DRI_EINVAL;
  if (!(c->rgbd_lambda >= 0) || !std::isfinite(c->rgbd_lambda)) return DRI_EINVAL;
  if (!(c->occlusion_thr >= 0) || !std::isfinite(c->occlusion_thr)) return DRI_EINVAL;
  if (c->icp_depth_weight != 0 && c->icp_depth_weight != 1) return DRI_EINVAL;
  if (c->gravity_dof != 0 && c->gravity_dof != DRI_GRAVITY_2DOF && c->gravity_dof != DRI_GRAVITY_3D)
    return DRI_EINVAL;
  if (c->gravity_dof == DRI_GRAVITY_3D && c->track_mode != DRI_TRACK_INERTIAL) return DRI_EINVAL;
  if (c->count_margins != 0 && c->count_margins != 1) return DRI_EINVAL;
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

TableView table_view(int nslots, int levels, int groups) {
  TableView v;
  std::memset(&v, 0, sizeof(v));
  size_t off = align_up((size_t)nslots * sizeof(SlotStatic), 16);
  const size_t pre = (size_t)(nslots + 1) * sizeof(int32_t);
  const size_t pre_g = (size_t)(nslots + groups) * sizeof(int32_t);
  v.copy_off = off;
  off = align_up(off + pre, 16);
  for (int l = 0; l < levels; ++l) {
    v.map_off[l] = off;
    off = align_up(off + pre, 16);
    v.track_off[l] = off;
    off = align_up(off + pre_g, 16);
  }
  v.bytes = align_up(off);
  return v;
}

}  // namespace dri

namespace {

// Staged bytes of one launch: SlotDyn[nslots], then one IMU block per slot.
size_t dyn_header_bytes(int nslots) { return align_up((size_t)nslots * sizeof(SlotDyn), 64); }
size_t imu_block_bytes(int imu_cap) {
  return align_up(sizeof(ImuHeader) + (size_t)imu_cap * sizeof(dri_imu_sample), 16);
}

}  // namespace

namespace dri {

StreamLayout make_layout(const dri_stream_config& cfg) {
  StreamLayout L;
  std::memset(&L, 0, sizeof(L));
  const bool fp16 = (cfg.precision_flags & DRI_FP16_MAPS) != 0;
  const bool fp32p = (cfg.precision_flags & DRI_FP32_PARTIALS) != 0;
  L.pack_bytes = fp16 ? 8 : 16;
  L.imu_cap = cfg.max_imu;
  size_t off = 0;
  L.ctrl = off;
  off = align_up(off + sizeof(Ctrl));
  L.dyn = off;
  L.dyn_bytes = dyn_header_bytes(1) + imu_block_bytes(L.imu_cap);
  off = align_up(off + L.dyn_bytes);
  L.table = off;
  off = align_up(off + table_view(1, cfg.levels, 1).bytes);
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
      off = align_up(off + plane * 4);
      L.level_off[l][s][2] = off;
      off = align_up(off + plane * L.pack_bytes);
      L.level_off[l][s][3] = off;
      off = align_up(off + plane * L.pack_bytes);
    }
  }
  int maxb = 1;
  for (int l = 0; l < cfg.levels; ++l)
    maxb = std::max(maxb, std::max(track_grid_blocks(cfg.width >> l, cfg.height >> l, 1),
                                   track_mixed_blocks(cfg.width >> l, cfg.height >> l, 1)));
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

namespace dri_host {

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

// Runs one kernel launcher; while profiling, brackets it with events recorded
// into stream s's counters.
template <class F>
cudaError_t launch(dri_stream_s* s, int cls, double pixels, F&& f) {
  if (!s || !s->profiling) return f();
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
  p.imu = reinterpret_cast<const ImuHeader*>(s->ws + s->L.dyn + dyn_header_bytes(1));
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
  p.imu_mode = c.imu_mode;
  p.gdof = c.gravity_dof == DRI_GRAVITY_3D ? 3 : 2;
  p.relin_g = c.bias_relin_g;
  p.relin_a = c.bias_relin_a;
  p.track_mode = c.track_mode;
  p.rgbd_lambda = c.rgbd_lambda;
  return p;
}

TrackParams track_params(const dri_stream_s* s, int level, int ppt, uint8_t* flags) {
  TrackParams p;
  std::memset(&p, 0, sizeof(p));
  p.g = s->geom[level];
  p.m = s->maps[level];
  p.ctrl = s->ctrl;
  p.partials = s->partials;
  p.gpartials = s->gpartials;
  p.counters = s->counters;
  p.flags = flags;
  p.ppt = ppt;
  p.nblocks = track_grid_blocks(p.g.w, p.g.h, p.ppt);
  p.depth_min = (float)s->cfg.depth_min;
  p.depth_max = (float)s->cfg.depth_max;
  p.icp_dist2 = (float)(s->cfg.icp_dist_thr * s->cfg.icp_dist_thr);
  p.icp_cos = (float)std::cos(s->cfg.icp_angle_thr_deg * 3.14159265358979323846 / 180.0);
  p.occ_thr = (float)s->cfg.occlusion_thr;
  p.icp_dw = s->cfg.icp_depth_weight;
  return p;
}

#define CK(expr)                                   \
  do {                                             \
    cudaError_t e_ = (expr);                       \
    if (e_ != cudaSuccess) return DRI_ECUDA;       \
  } while (0)

// ---- plans ------------------------------------------------------------------

// Block prefixes and static slot records from the slots' configurations and
// the chosen rows per thread.
void plan_fill_tables(Plan* p) {
  p->host_slots.assign(p->S, SlotStatic());
  p->pre_copy.assign(p->S + 1, 0);
  for (int l = 0; l < p->levels; ++l) {
    p->pre_map[l].assign(p->S + 1, 0);
    p->pre_track[l].assign(p->S + p->groups, 0);
  }
  for (int i = 0; i < p->S; ++i) {
    const dri_stream_s* s = p->slots[i];
    SlotStatic& st = p->host_slots[i];
    std::memset(&st, 0, sizeof(st));
    for (int l = 0; l < p->levels; ++l) st.tp[l] = track_params(s, l, p->ppt[i][l], nullptr);
    st.sp = solve_params(s, 0, 0);
    st.sp.imu = nullptr;
    st.in_depth = s->in_depth;
    st.in_inten = s->in_inten;
    st.levels = p->levels;
    p->pre_copy[i + 1] = p->pre_copy[i] + copy_tiles(s->cfg.width, s->cfg.height);
    for (int l = 0; l < p->levels; ++l)
      p->pre_map[l][i + 1] = p->pre_map[l][i] + map_tiles(s->geom[l].w, s->geom[l].h);
  }
  for (int g = 0; g < p->groups; ++g) {       // local prefix of each group's slots
    const int base = p->gfirst[g] + g;
    for (int l = 0; l < p->levels; ++l)
      for (int k = 0; k < p->gcount[g]; ++k)
        p->pre_track[l][base + k + 1] =
            p->pre_track[l][base + k] + p->host_slots[p->gfirst[g] + k].tp[l].nblocks;
  }
}

// Pixel-kernel blocks of group g at level l, and the byte offset of its prefix.
int track_blocks(const Plan* p, int l, int g) {
  return p->pre_track[l][p->gfirst[g] + g + p->gcount[g]];
}
size_t track_start(const Plan* p, int l, int g) {
  return p->tv.track_off[l] + (size_t)(p->gfirst[g] + g) * sizeof(int32_t);
}

int plan_upload_tables(Plan* p) {
  std::vector<char> img(p->tv.bytes, 0);
  std::memcpy(img.data(), p->host_slots.data(), (size_t)p->S * sizeof(SlotStatic));
  const size_t pre = (size_t)(p->S + 1) * sizeof(int32_t);
  std::memcpy(img.data() + p->tv.copy_off, p->pre_copy.data(), pre);
  for (int l = 0; l < p->levels; ++l) {
    std::memcpy(img.data() + p->tv.map_off[l], p->pre_map[l].data(), pre);
    std::memcpy(img.data() + p->tv.track_off[l], p->pre_track[l].data(),
                (size_t)(p->S + p->groups) * sizeof(int32_t));
  }
  CK(cudaMemcpyAsync(p->table, img.data(), img.size(), cudaMemcpyHostToDevice, p->stream));
  CK(cudaStreamSynchronize(p->stream));
  return DRI_OK;
}

void plan_free(Plan* p) {
  if (!p) return;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  for (cudaStream_t a : p->aux)
    if (a) cudaStreamDestroy(a);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_grad) cudaEventDestroy(p->ev_grad);
  if (p->ev_maps) cudaEventDestroy(p->ev_maps);
  if (p->ev_start) cudaEventDestroy(p->ev_start);
  if (p->ev_begin) cudaEventDestroy(p->ev_begin);
  if (p->ev_norm) cudaEventDestroy(p->ev_norm);
  for (cudaEvent_t e : p->ev_join)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : p->ev)
    if (e) cudaEventDestroy(e);
  if (p->pin_dyn) cudaFreeHost(p->pin_dyn);
  if (p->pin_heads) cudaFreeHost(p->pin_heads);
  if (p->owns_device) {
    if (p->table) cudaFree(p->table);
    if (p->dyn) cudaFree(p->dyn);
    if (p->heads) cudaFree(p->heads);
  }
  delete p;
}

// Creates a plan over the given streams.  Single-slot plans use the stream's
// workspace; batch plans allocate their own table, staging and head buffers.
// Splits the plan's slots into `groups` contiguous groups of near-equal size.
void plan_set_groups(Plan* p, int groups) {
  p->groups = groups;
  p->gfirst.assign(groups, 0);
  p->gcount.assign(groups, 0);
  for (int g = 0; g < groups; ++g) {
    p->gfirst[g] = (int)((int64_t)p->S * g / groups);
    p->gcount[g] = (int)((int64_t)p->S * (g + 1) / groups) - p->gfirst[g];
  }
}

int plan_create(dri_stream_s* const* streams, int n, int ring, bool in_workspace, int groups,
                Plan** out) {
  *out = nullptr;
  Plan* p = new (std::nothrow) Plan();
  if (!p) return DRI_ENOMEM;
  p->slots.assign(streams, streams + n);
  p->S = n;
  p->stream = streams[0]->stream;
  p->levels = streams[0]->cfg.levels;
  for (int l = 0; l < kMaxLevels; ++l) p->iters[l] = l < p->levels ? streams[0]->cfg.iters[l] : 0;
  p->fp16 = (streams[0]->cfg.precision_flags & DRI_FP16_MAPS) != 0;
  p->fp32p = (streams[0]->cfg.precision_flags & DRI_FP32_PARTIALS) != 0;
  p->opt = pixel_options(streams[0]->cfg);
  for (int i = 0; i < n; ++i) p->g3 = p->g3 || streams[i]->cfg.gravity_dof == DRI_GRAVITY_3D;
  for (int i = 0; i < n; ++i) p->margins = p->margins || streams[i]->cfg.count_margins == 1;
  plan_set_groups(p, groups);
  // a batch plan's table has room for any group count; a stream's own plan has
  // one group and exactly the workspace's table region
  p->tv = table_view(n, p->levels, in_workspace ? 1 : kMaxGroups);
  p->R = ring;
  p->ppt.resize(n);
  for (int i = 0; i < n; ++i)
    for (int l = 0; l < kMaxLevels; ++l) p->ppt[i][l] = streams[i]->ppt[l];
  int imu_cap = 0;
  for (int i = 0; i < n; ++i) imu_cap = std::max(imu_cap, streams[i]->L.imu_cap);
  p->dyn_cap = dyn_header_bytes(n) + (size_t)n * imu_block_bytes(imu_cap);
  if (in_workspace) {             // the one-slot plan of dri_track
    dri_stream_s* s = streams[0];
    if (n != 1 || groups != 1 || p->tv.bytes > s->L.in_depth - s->L.table) {
      plan_free(p);
      return DRI_EINVAL;
    }
    p->table = s->ws + s->L.table;
    p->dyn = reinterpret_cast<unsigned char*>(s->ws + s->L.dyn);
  } else {
    p->owns_device = true;
    if (cudaMalloc(&p->table, p->tv.bytes) != cudaSuccess ||
        cudaMalloc(&p->dyn, p->dyn_cap) != cudaSuccess ||
        cudaMalloc(&p->heads, (size_t)n * kCtrlHeadBytes) != cudaSuccess) {
      plan_free(p);
      return DRI_ENOMEM;
    }
  }
  if (cudaMallocHost(&p->pin_dyn, (size_t)ring * p->dyn_cap) != cudaSuccess ||
      cudaMallocHost(&p->pin_heads, (size_t)ring * n * kCtrlHeadBytes) != cudaSuccess) {
    plan_free(p);
    return DRI_ENOMEM;
  }
  p->aux.assign(kMaxGroups - 1, nullptr);
  p->ev_join.assign(kMaxGroups - 1, nullptr);
  if (!in_workspace) {
    if (cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_grad, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_maps, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_begin, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_norm, cudaEventDisableTiming) != cudaSuccess) {
      plan_free(p);
      return DRI_ENOMEM;
    }
    for (int g = 0; g < kMaxGroups - 1; ++g) {
      if (cudaStreamCreateWithFlags(&p->aux[g], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&p->ev_join[g], cudaEventDisableTiming) != cudaSuccess) {
        plan_free(p);
        return DRI_ENOMEM;
      }
    }
  }
  p->ev.assign(ring, nullptr);
  p->ring_used.assign(ring, 0);
  for (int i = 0; i < ring; ++i) {
    if (cudaEventCreateWithFlags(&p->ev[i], cudaEventDisableTiming) != cudaSuccess) {
      plan_free(p);
      return DRI_ENOMEM;
    }
  }
  plan_fill_tables(p);
  const int r = plan_upload_tables(p);
  if (r != DRI_OK) {
    plan_free(p);
    return r;
  }
  *out = p;
  return DRI_OK;
}

const Ctrl* ring_head(const Plan* p, int slot, int i) {
  return reinterpret_cast<const Ctrl*>(p->pin_heads + ((size_t)slot * p->S + i) * kCtrlHeadBytes);
}

// Settles, in order, the frames whose result copy has completed (all of them
// when wait is set): a failed frame rolls the host's start time back to the
// state the device kept.
int settle(dri_stream_s* s, bool wait) {
  while (!s->inflight.empty()) {
    const dri_stream_s::InFlight f = s->inflight.front();
    cudaError_t q = wait ? cudaEventSynchronize(f.ev) : cudaEventQuery(f.ev);
    if (q == cudaErrorNotReady) return DRI_OK;
    if (q != cudaSuccess) return DRI_ECUDA;
    s->t_confirmed = f.head->t_state;
    if (f.head->status != DRI_OK) {
      s->t_prev = f.head->t_state;
      s->frames_failed++;
    } else {
      s->frames_ok++;
    }
    s->inflight.pop_front();
  }
  return DRI_OK;
}

// Next staging slot of the plan; waits for the launch that last used it and
// settles the streams whose results it held.
int plan_acquire(Plan* p, int* slot) {
  const int r = p->next;
  if (p->ring_used[r]) {
    CK(cudaEventSynchronize(p->ev[r]));
    for (dri_stream_s* s : p->slots)
      if (settle(s, false) != DRI_OK) return DRI_ECUDA;
    p->ring_used[r] = 0;
  }
  *slot = r;
  return DRI_OK;
}

// Samples covering [t0, t1] (the last one at or before t0 through the first at
// or after t1): [k0, k1).
// Index of the last sample at or before t (samples strictly increasing in t;
// the first sample is at or before t).
size_t imu_at_or_before(const std::vector<dri_imu_sample>& v, double t) {
  const auto it = std::upper_bound(v.begin(), v.end(), t,
                                   [](double x, const dri_imu_sample& m) { return x < m.t; });
  return it == v.begin() ? 0 : (size_t)(it - v.begin()) - 1;
}

int select_imu(const dri_stream_s* s, double t0, double t1, size_t* k0, size_t* k1) {
  const auto& v = s->imu;
  if (v.empty() || v.front().t > t0 || v.back().t < t1) return DRI_ENOTREADY;
  const size_t a = imu_at_or_before(v, t0);
  // first sample at or after t1
  const size_t b = (size_t)(std::lower_bound(v.begin() + a, v.end(), t1,
                                             [](const dri_imu_sample& m, double x) { return m.t < x; }) -
                            v.begin());
  if (b >= v.size()) return DRI_ENOTREADY;
  *k0 = a;
  *k1 = b + 1;
  if ((int64_t)(*k1 - *k0) > s->L.imu_cap) return DRI_ENOMEM;
  if ((int64_t)(*k1 - *k0) - 1 > solver_max_imu_pieces()) return DRI_ENOMEM;
  return DRI_OK;
}

// One slot's staged record: mode, image pointers and the IMU block of
// [t0, t1] at byte `off` of the staging image.  Returns the block's size.
size_t stage_slot(const dri_stream_s* s, char* img, int i, int mode, double t0, double t1, size_t k0,
                  size_t k1, size_t off) {
  SlotDyn d;
  std::memset(&d, 0, sizeof(d));
  d.mode = mode;
  d.pitch = s->src_pitch;
  d.imu_off = (int64_t)off;
  d.src_depth = s->src_depth;
  d.src_inten = s->src_inten;
  std::memcpy(img + (size_t)i * sizeof(SlotDyn), &d, sizeof(d));
  ImuHeader h;
  std::memset(&h, 0, sizeof(h));
  h.t0 = t0;
  h.t1 = t1;
  h.n = (int32_t)(k1 - k0);
  std::memcpy(img + off, &h, sizeof(h));
  if (h.n) std::memcpy(img + off + sizeof(h), s->imu.data() + k0, (size_t)h.n * sizeof(dri_imu_sample));
  return align_up(sizeof(h) + (size_t)h.n * sizeof(dri_imu_sample), 16);
}

BatchArgs plan_args(const Plan* p, size_t start_off, int level, int last, int slot0 = 0,
                    int nslots = -1) {
  BatchArgs a;
  std::memset(&a, 0, sizeof(a));
  a.slots = reinterpret_cast<const SlotStatic*>(p->table);
  a.dyn = p->dyn;
  a.start = reinterpret_cast<const int32_t*>(p->table + start_off);
  a.slot0 = slot0;
  a.nslots = nslots < 0 ? p->S : nslots;
  a.level = level;
  a.last = last;
  return a;
}

double plan_pixels(const Plan* p, int level) {
  double n = 0;
  for (const dri_stream_s* s : p->slots) n += (double)s->geom[level].w * s->geom[level].h;
  return n;
}

// The spare stream of a batch plan (the last of its group streams when the
// groups leave it free; none while profiling or for a stream's own plan).
cudaStream_t side_stream(const Plan* p, bool profiling) {
  if (profiling || p->groups >= kMaxGroups || !p->aux[kMaxGroups - 2]) return p->stream;
  return p->aux[kMaxGroups - 2];
}

// Kernel launches of one frame, in order.  phase 1: maps and frame begin;
// phase 2: the Gauss-Newton loop, frame end, gradients and the head gather.
// On a batch plan's spare stream: the frame start, beside the map kernels
// (it reads and writes the slots' control blocks and their IMU blocks, the map
// kernels only which set is the reference, which changes at the frame end),
// and beside the loop the normal maps of the finer levels (the loop starts at
// the coarsest; each group waits for them before its first finer-level pixel
// kernel) and the gradient maps.
int plan_enqueue(Plan* p, int phases, int64_t* kernels) {
  dri_stream_s* prof = p->slots[0];
  cudaStream_t st = p->stream;
  const int L = p->levels;
  const cudaStream_t sside = side_stream(p, prof->profiling);
  int64_t k = 0;
  if (phases & 1) {
    const bool side = sside != st;
    const BatchArgs ab = plan_args(p, p->tv.copy_off, 0, 0);
    if (side) {
      CK(cudaEventRecord(p->ev_start, st));
      CK(cudaStreamWaitEvent(sside, p->ev_start, 0));
      CK(launch(prof, DRI_KC_FRAME, 0.0, [&] { return launch_frame_begin_batch(ab, sside); }));
      ++k;
      CK(cudaEventRecord(p->ev_begin, sside));
    }
    const BatchArgs a0 = plan_args(p, p->tv.copy_off, 0, 0);
    CK(launch(prof, DRI_KC_MAPS, plan_pixels(p, 0),
              [&] { return launch_copy_batch(a0, p->pre_copy[p->S], st); }));
    ++k;
    for (int l = 1; l < L; ++l) {
      const BatchArgs a = plan_args(p, p->tv.map_off[l], l, 0);
      CK(launch(prof, DRI_KC_MAPS, plan_pixels(p, l),
                [&] { return launch_pyr_down_batch(a, p->pre_map[l][p->S], st); }));
      ++k;
    }
    p->norm_side = sside != st && L > 1;
    if (p->norm_side) {
      CK(cudaEventRecord(p->ev_maps, st));
      CK(cudaStreamWaitEvent(sside, p->ev_maps, 0));
    }
    for (int l = L - 1; l >= 0; --l) {          // coarsest first
      const BatchArgs a = plan_args(p, p->tv.map_off[l], l, 0);
      const cudaStream_t sn = (p->norm_side && l < L - 1) ? sside : st;
      CK(launch(prof, DRI_KC_MAPS, plan_pixels(p, l),
                [&] { return launch_normals_batch(a, p->pre_map[l][p->S], p->fp16, sn); }));
      ++k;
    }
    if (p->norm_side) CK(cudaEventRecord(p->ev_norm, sside));
    if (side) {
      CK(cudaStreamWaitEvent(st, p->ev_begin, 0));
    } else {
      CK(launch(prof, DRI_KC_FRAME, 0.0, [&] { return launch_frame_begin_batch(ab, st); }));
      ++k;
    }
  }
  if (phases & 2) {
    // Gauss-Newton loop per slot group; groups run on their own streams (forked
    // from and joined back into the plan's stream) so that one group's FP64
    // solves overlap another group's pixel kernels.  With several groups a
    // pixel kernel starts only when its group's step has ended: launched early
    // (programmatic dependent launch) its blocks would hold the SMs for the
    // whole step, waiting, instead of leaving them to the other groups (4 groups
    // of 16 x 640x480: 7.4k frames/s early, 12.3k not).  While profiling, the
    // groups run one after the other on the plan's stream.
    const bool fork = p->groups > 1 && !prof->profiling;
    // The gradient maps of the frame's own set (the next reference's pack B)
    // depend on its intensity pyramid only: they run on a spare stream beside
    // the Gauss-Newton loop and are joined before the frame end.
    const cudaStream_t sgrad = sside;
    if (fork || sgrad != st) CK(cudaEventRecord(p->ev_fork, st));
    if (sgrad != st) CK(cudaStreamWaitEvent(sgrad, p->ev_fork, 0));
    for (int l = 0; l < L; ++l) {
      const BatchArgs a = plan_args(p, p->tv.map_off[l], l, 0);
      CK(launch(prof, DRI_KC_GRAD, plan_pixels(p, l),
                [&] { return launch_gradient_batch(a, p->pre_map[l][p->S], p->fp16, sgrad); }));
      ++k;
    }
    if (sgrad != st) CK(cudaEventRecord(p->ev_grad, sgrad));
    for (int g = 0; g < p->groups; ++g) {
      cudaStream_t sg = (fork && g > 0) ? p->aux[g - 1] : st;
      if (fork && g > 0) CK(cudaStreamWaitEvent(sg, p->ev_fork, 0));
      const double px_scale = (double)p->gcount[g] / p->S;
      const int prio = launch_priority(false);
      int remaining = 0;
      for (int l = 0; l < L; ++l) remaining += p->iters[l];
      for (int l = L - 1; l >= 0; --l) {
        if (p->norm_side && l == L - 2) CK(cudaStreamWaitEvent(sg, p->ev_norm, 0));
        for (int it = 0; it < p->iters[l]; ++it) {
          --remaining;
          BatchArgs at = plan_args(p, track_start(p, l, g), l, 0, p->gfirst[g], p->gcount[g]);
          at.margin = p->margins && it == p->iters[l] - 1;   // the level's margin decisions
          const int nb = track_blocks(p, l, g);
          CK(launch(prof, DRI_KC_TRACK, plan_pixels(p, l) * px_scale,
                    [&] {
                      return launch_track_batch(at, nb, p->fp16, p->fp32p, p->opt, prio, p->groups == 1, sg);
                    }));
          const BatchArgs as = plan_args(p, p->tv.copy_off, l, remaining == 0, p->gfirst[g], p->gcount[g]);
          CK(launch(prof, DRI_KC_SOLVE, 0.0, [&] { return launch_gn_step_batch(as, p->g3, sg); }));
          k += 2;
        }
      }
      if (fork && g > 0) {
        CK(cudaEventRecord(p->ev_join[g - 1], sg));
        CK(cudaStreamWaitEvent(st, p->ev_join[g - 1], 0));
      }
    }
    if (sgrad != st) CK(cudaStreamWaitEvent(st, p->ev_grad, 0));
    const BatchArgs ae = plan_args(p, p->tv.copy_off, 0, 0);
    CK(launch(prof, DRI_KC_FRAME, 0.0, [&] { return launch_frame_end_batch(ae, st); }));
    ++k;
    if (p->heads) {
      CK(launch_gather_heads(ae, p->heads, st));
      ++k;
    }
  }
  if (kernels) *kernels += k;
  return DRI_OK;
}

// Chooses each level's rows per thread by timing the pixel kernel on the
// frames just staged (their maps and frame start are already enqueued):
// candidates 2, 4, 8, 16 and 32, three launches each, the fastest mean wins.
int plan_autotune(Plan* p, int64_t* kernels) {
  static const int cand[] = {2, 4, 8, 16, 32};
  if (p->norm_side) CK(cudaStreamWaitEvent(p->stream, p->ev_norm, 0));   // every level's maps
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = DRI_OK;
  for (int l = 0; l < p->levels && rc == DRI_OK; ++l) {
    float best = 1e30f;
    int best_ppt = p->ppt[0][l];
    for (int c : cand) {
      for (auto& v : p->ppt) v[l] = c;
      plan_fill_tables(p);
      if ((rc = plan_upload_tables(p)) != DRI_OK) break;
      auto all_groups = [&] {
        for (int g = 0; g < p->groups; ++g) {
          const BatchArgs at = plan_args(p, track_start(p, l, g), l, 0, p->gfirst[g], p->gcount[g]);
          if (launch_track_batch(at, track_blocks(p, l, g), p->fp16, p->fp32p, p->opt, launch_priority(false),
                                 true, p->stream) !=
              cudaSuccess)
            return false;
        }
        return true;
      };
      if (!all_groups() || cudaEventRecord(e0, p->stream) != cudaSuccess) {
        rc = DRI_ECUDA;
        break;
      }
      for (int rep = 0; rep < 3; ++rep)
        if (!all_groups()) rc = DRI_ECUDA;
      float ms = 0.f;
      if (rc != DRI_OK || cudaEventRecord(e1, p->stream) != cudaSuccess ||
          cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
        rc = DRI_ECUDA;
        break;
      }
      *kernels += 4 * p->groups;
      if (ms < best) {
        best = ms;
        best_ppt = c;
      }
    }
    for (auto& v : p->ppt) v[l] = best_ppt;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != DRI_OK) return rc;
  plan_fill_tables(p);
  return plan_upload_tables(p);
}

// Captures the per-frame launch sequence once as a CUDA graph; a stream that
// cannot be captured (the legacy default stream) keeps launching directly.
int plan_run(Plan* p, int64_t* kernels) {
  const bool profiling = p->slots[0]->profiling;
  if (!profiling && !p->graph && !p->graph_failed && p->stream != nullptr &&
      (!p->autotune || p->tuned)) {
    cudaGraph_t g = nullptr;
    int64_t k = 0;
    if (cudaStreamBeginCapture(p->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
      const int r = plan_enqueue(p, 3, &k);
      const cudaError_t e = cudaStreamEndCapture(p->stream, &g);
      if (r == DRI_OK && e == cudaSuccess && g &&
          cudaGraphInstantiate(&p->graph, g, cudaGraphInstantiateFlagUseNodePriority) == cudaSuccess) {
        p->kernels_per_frame = k;
      } else {
        p->graph = nullptr;
        p->graph_failed = true;
      }
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
    } else {
      cudaGetLastError();
      p->graph_failed = true;
    }
  }
  if (p->graph && !profiling) {
    CK(cudaGraphLaunch(p->graph, p->stream));
    *kernels += p->kernels_per_frame;
    return DRI_OK;
  }
  return plan_enqueue(p, 3, kernels);
}

SlotWork plan_slot_work(const dri_stream_s* s) {
  SlotWork w;
  if (!s->frame_pending) return w;
  if (!s->initialised) {
    w.mode = kSlotInit;
    w.status = DRI_OK;
    return w;
  }
  if (s->cfg.track_mode == DRI_TRACK_RGBD_ONLY) {   // no IMU term: no samples staged
    w.mode = kSlotTrack;
    w.status = DRI_OK;
    return w;
  }
  const int r = select_imu(s, s->t_prev, s->t_frame, &w.k0, &w.k1);
  if (r != DRI_OK) {
    w.status = r;
    return w;
  }
  w.mode = kSlotTrack;
  w.status = DRI_OK;
  return w;
}

// Stages and launches one frame of every slot with work; records the result
// copies and the streams' bookkeeping.  *ring_slot receives the staging slot
// (-1 if nothing ran).
int plan_launch(Plan* p, const std::vector<SlotWork>& work, int* ring_slot) {
  *ring_slot = -1;
  int r = settle(p->slots[0], false);
  if (r != DRI_OK) return r;
  int rs = 0;
  if ((r = plan_acquire(p, &rs)) != DRI_OK) return r;
  char* img = p->pin_dyn + (size_t)rs * p->dyn_cap;
  std::memset(img, 0, dyn_header_bytes(p->S));
  size_t off = dyn_header_bytes(p->S);
  bool any_track = false;
  for (int i = 0; i < p->S; ++i) {
    const dri_stream_s* s = p->slots[i];
    const SlotWork& w = work[i];
    if (w.mode == kSlotIdle) continue;
    const double t0 = w.mode == kSlotInit ? s->t_frame : s->t_prev;
    off += stage_slot(s, img, i, w.mode, t0, s->t_frame, w.k0, w.k1, off);
    any_track = any_track || w.mode == kSlotTrack;
  }
  CK(cudaMemcpyAsync(p->dyn, img, off, cudaMemcpyHostToDevice, p->stream));
  int64_t kernels = 0;
  if (p->autotune && !p->tuned && any_track && !p->slots[0]->profiling) {
    if ((r = plan_enqueue(p, 1, &kernels)) != DRI_OK) return r;
    if ((r = plan_autotune(p, &kernels)) != DRI_OK) return r;
    p->tuned = true;
    if ((r = plan_enqueue(p, 2, &kernels)) != DRI_OK) return r;
  } else if ((r = plan_run(p, &kernels)) != DRI_OK) {
    return r;
  }
  const void* src = p->heads ? (const void*)p->heads : (const void*)p->slots[0]->ctrl;
  CK(cudaMemcpyAsync(p->pin_heads + (size_t)rs * p->S * kCtrlHeadBytes, src,
                     (size_t)p->S * kCtrlHeadBytes, cudaMemcpyDeviceToHost, p->stream));
  CK(cudaEventRecord(p->ev[rs], p->stream));
  p->ring_used[rs] = 1;
  p->next = (p->next + 1) % p->R;
  for (int i = 0; i < p->S; ++i) {
    dri_stream_s* s = p->slots[i];
    s->launches += kernels;
    const SlotWork& w = work[i];
    if (w.mode == kSlotIdle) continue;
    s->h2d_last = s->h2d_frame + (int64_t)(sizeof(SlotDyn) + sizeof(ImuHeader) +
                                           (w.k1 - w.k0) * sizeof(dri_imu_sample));
    s->d2h_last = (int64_t)kCtrlHeadBytes;
    if (w.mode == kSlotInit) {
      s->initialised = true;
      s->t_prev_before = s->t_frame;
      s->t_prev = s->t_frame;
      s->t_confirmed = s->t_frame;
    } else {
      // drop samples no later frame can need: all before the one covering the
      // earliest time a frame may still start from (a failed frame in flight
      // rolls the start back to t_confirmed).  Erasing moves every later
      // sample, and a client may push minutes of samples ahead, so they are
      // dropped in batches of at least kImuDropBatch.
      const double keep_from = std::min(s->t_prev, s->t_confirmed);
      if (!s->imu.empty() && s->imu.front().t <= keep_from) {
        const size_t a = imu_at_or_before(s->imu, keep_from);
        if (a >= kImuDropBatch) s->imu.erase(s->imu.begin(), s->imu.begin() + a);
      }
      s->t_prev_before = s->t_prev;
      s->t_prev = s->t_frame;   // optimistic; rolled back when the frame is known to fail
    }
    s->frame_pending = false;
    s->inflight.push_back({p->ev[rs], ring_head(p, rs, i)});
  }
  *ring_slot = rs;
  return DRI_OK;
}

std::mutex g_batch_mu;   // guards every stream's batch-plan list and the plan cache
std::vector<Plan*> g_batch_plans;

void forget_plan_locked(Plan* p) {
  for (dri_stream_s* s : p->slots) {
    auto& v = s->batches;
    v.erase(std::remove(v.begin(), v.end(), p), v.end());
  }
  g_batch_plans.erase(std::remove(g_batch_plans.begin(), g_batch_plans.end(), p), g_batch_plans.end());
}

void release_batch_plan(const std::vector<dri_stream_s*>& key) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (Plan* q : g_batch_plans) {
    if (q->slots != key) continue;
    cudaStreamSynchronize(q->stream);
    for (dri_stream_s* o : q->slots) settle(o, true);
    forget_plan_locked(q);
    plan_free(q);
    return;
  }
}

}  // namespace dri_host

using namespace dri_host;

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
  cfg->imu_mode = DRI_IMU_REINTEGRATE;
  cfg->bias_relin_g = 0.01;
  cfg->bias_relin_a = 0.1;
  cfg->track_mode = DRI_TRACK_INERTIAL;
  cfg->rgbd_lambda = 1.0;
  cfg->occlusion_thr = 0.0;
  cfg->icp_depth_weight = 0;
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
  if (cudaMallocHost(&s->pin_ctrl, sizeof(Ctrl)) != cudaSuccess) {
    dri_destroy_stream(s);
    return DRI_ENOMEM;
  }
  s->ctrl = (Ctrl*)(s->ws + L.ctrl);
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
    for (int k = 0; k < 2; ++k) {
      m.depth[k] = (float*)(s->ws + L.level_off[l][k][0]);
      m.inten[k] = (float*)(s->ws + L.level_off[l][k][1]);
      m.packA[k] = (void*)(s->ws + L.level_off[l][k][2]);
      m.packB[k] = (void*)(s->ws + L.level_off[l][k][3]);
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
  dri_stream_s* one[1] = {s};
  const int r = plan_create(one, 1, kStreamRing, true, 1, &s->own);
  if (r != DRI_OK) {
    dri_destroy_stream(s);
    return r;
  }
  *out = s;
  return DRI_OK;
}

int dri_destroy_stream(dri_stream s) {
  if (!s) return DRI_EINVAL;
  if (s->stream || s->ws) cudaStreamSynchronize(s->stream);
  {
    std::lock_guard<std::mutex> lk(g_batch_mu);
    while (!s->batches.empty()) {
      Plan* p = s->batches.back();
      cudaStreamSynchronize(p->stream);
      for (dri_stream_s* o : p->slots) settle(o, true);
      forget_plan_locked(p);
      plan_free(p);
    }
  }
  settle(s, true);
  plan_free(s->own);
  if (s->ref_stage) cudaFree(s->ref_stage);
  if (s->own_ws && s->ws) cudaFree(s->ws);
  if (s->pin_ctrl) cudaFreeHost(s->pin_ctrl);
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  delete s;
  return DRI_OK;
}

namespace {

// Device address of pinned (page-locked) host memory, which the GPU reads
// directly; false for pageable memory or an unknown pointer.
bool pinned_device_ptr(const void* p, const void** dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type != cudaMemoryTypeHost || a.devicePointer == nullptr) return false;
  *dev = a.devicePointer;
  return true;
}

}  // namespace

int dri_upload_frame(dri_stream s, double t, const float* depth, const float* intensity,
                     size_t pitch_bytes, int32_t mem_kind) {
  if (!s || !depth || !intensity || !std::isfinite(t)) return DRI_EINVAL;
  if (mem_kind != DRI_HOST && mem_kind != DRI_DEVICE) return DRI_EINVAL;
  const size_t row = (size_t)s->cfg.width * sizeof(float);
  const size_t pitch = pitch_bytes ? pitch_bytes : row;
  if (pitch < row || pitch % sizeof(float) != 0 || pitch / sizeof(float) > (size_t)INT32_MAX)
    return DRI_EINVAL;
  if (s->initialised && !(t > s->t_prev)) return DRI_EINVAL;
  const void *pd = nullptr, *pi = nullptr;
  if (mem_kind == DRI_HOST && pinned_device_ptr(depth, &pd) && pinned_device_ptr(intensity, &pi)) {
    // pinned: the frame's first kernel reads the images over the host link
    s->src_depth = static_cast<const float*>(pd);
    s->src_inten = static_cast<const float*>(pi);
    s->src_pitch = (int32_t)(pitch / sizeof(float));
    s->h2d_frame = (int64_t)(2 * row * s->cfg.height);
  } else if (mem_kind == DRI_HOST) {
    CK(cudaMemcpy2DAsync(s->in_depth, row, depth, pitch, row, s->cfg.height, cudaMemcpyHostToDevice,
                         s->stream));
    CK(cudaMemcpy2DAsync(s->in_inten, row, intensity, pitch, row, s->cfg.height,
                         cudaMemcpyHostToDevice, s->stream));
    s->src_depth = s->in_depth;
    s->src_inten = s->in_inten;
    s->src_pitch = s->cfg.width;
    s->h2d_frame = (int64_t)(2 * row * s->cfg.height);
  } else {
    s->src_depth = depth;
    s->src_inten = intensity;
    s->src_pitch = (int32_t)(pitch / sizeof(float));
    s->h2d_frame = 0;
  }
  s->t_frame = t;
  s->frame_pending = true;
  return DRI_OK;
}

int dri_upload_reference(dri_stream s, const float* vertex_W, const float* normal_W,
                         const float* intensity, const double* T_WC_ref, size_t pitch_px,
                         int32_t mem_kind) {
  if (!s || !vertex_W || !normal_W || !intensity || !T_WC_ref) return DRI_EINVAL;
  if (mem_kind != DRI_HOST && mem_kind != DRI_DEVICE) return DRI_EINVAL;
  const int w = s->cfg.width, h = s->cfg.height;
  const size_t pitch = pitch_px ? pitch_px : (size_t)w;
  if (pitch < (size_t)w || pitch > (size_t)INT32_MAX) return DRI_EINVAL;
  for (int i = 0; i < 7; ++i)
    if (!std::isfinite(T_WC_ref[i])) return DRI_EINVAL;
  const double qn = std::sqrt(T_WC_ref[3] * T_WC_ref[3] + T_WC_ref[4] * T_WC_ref[4] +
                              T_WC_ref[5] * T_WC_ref[5] + T_WC_ref[6] * T_WC_ref[6]);
  if (!(qn > 1e-12)) return DRI_EINVAL;
  if (!s->initialised) return DRI_ENOTREADY;
  RefUpload up;
  std::memset(&up, 0, sizeof(up));
  quat_to_rot_h(T_WC_ref + 3, up.R);
  for (int i = 0; i < 3; ++i) up.r[i] = T_WC_ref[i];
  if (mem_kind == DRI_HOST) {
    const size_t npx = (size_t)w * h;
    if (!s->ref_stage && cudaMalloc(&s->ref_stage, npx * 7 * sizeof(float)) != cudaSuccess) {
      s->ref_stage = nullptr;
      return DRI_ENOMEM;
    }
    float* sv = s->ref_stage;
    float* sn = sv + 3 * npx;
    float* si = sn + 3 * npx;
    const size_t row3 = (size_t)w * 3 * sizeof(float), row1 = (size_t)w * sizeof(float);
    CK(cudaMemcpy2DAsync(sv, row3, vertex_W, pitch * 3 * sizeof(float), row3, h, cudaMemcpyHostToDevice,
                         s->stream));
    CK(cudaMemcpy2DAsync(sn, row3, normal_W, pitch * 3 * sizeof(float), row3, h, cudaMemcpyHostToDevice,
                         s->stream));
    CK(cudaMemcpy2DAsync(si, row1, intensity, pitch * sizeof(float), row1, h, cudaMemcpyHostToDevice,
                         s->stream));
    up.V = sv;
    up.N = sn;
    up.I = si;
    up.pitch = w;
  } else {
    up.V = vertex_W;
    up.N = normal_W;
    up.I = intensity;
    up.pitch = (int64_t)pitch;
  }
  const bool fp16 = (s->cfg.precision_flags & DRI_FP16_MAPS) != 0;
  CK(launch(s, DRI_KC_MAPS, (double)w * h, [&] {
    return launch_upload_reference(s->maps, s->geom, s->cfg.levels, s->ctrl, (float)s->cfg.depth_min,
                                   (float)s->cfg.depth_max, fp16, up, s->stream);
  }));
  s->launches += 2 * s->cfg.levels + 1;
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


int dri_track(dri_stream s, dri_track_result* out) {
  if (!s) return DRI_EINVAL;
  if (!s->frame_pending) return DRI_ENOTREADY;
  std::vector<SlotWork> work(1, plan_slot_work(s));
  if (work[0].mode == kSlotIdle) return work[0].status;
  const bool init = work[0].mode == kSlotInit;
  int rs = -1;
  const int r = plan_launch(s->own, work, &rs);
  if (r != DRI_OK) return r;
  if (!out) return DRI_OK;
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  const Ctrl* h = ring_head(s->own, rs, 0);
  fill_result(s, h, out, init, s->t_prev_before);
  return h->status;
}

}  // extern "C"

namespace dri_host {

void fill_result(const dri_stream_s* s, const Ctrl* h, dri_track_result* out, bool init,
                        double t0) {
  std::memset(out, 0, sizeof(*out));
  out->x1 = from_dstate(h->x, h->t_state);
  out->x0 = from_dstate(h->x0, t0);
  for (int l = 0; l < kMaxLevels; ++l) {
    out->n_icp[l] = h->n_icp[l];
    out->n_rgb[l] = h->n_rgb[l];
    out->n_margin[l] = h->n_margin[l];
  }
  out->cost = h->cost;
  out->status = h->status;
  out->initialised = init ? 1 : 0;
  (void)s;
}

// The plan of a stream list: a stream's own plan for one stream, else the
// cached batch plan of exactly this list (created on first use).
int batch_plan(const dri_stream* streams, int32_t n, Plan** out) {
  *out = nullptr;
  if (!streams || n < 1 || n > kMaxBatch) return DRI_EINVAL;
  for (int i = 0; i < n; ++i) {
    const dri_stream_s* s = streams[i];
    if (!s) return DRI_EINVAL;
    for (int j = 0; j < i; ++j)
      if (streams[j] == s) return DRI_EINVAL;
    const dri_stream_s* s0 = streams[0];
    if (s->stream != s0->stream || s->cfg.levels != s0->cfg.levels ||
        s->cfg.precision_flags != s0->cfg.precision_flags ||
        pixel_options(s->cfg) != pixel_options(s0->cfg))
      return DRI_EINVAL;
    for (int l = 0; l < s->cfg.levels; ++l)
      if (s->cfg.iters[l] != s0->cfg.iters[l]) return DRI_EINVAL;
  }
  if (n == 1) {
    *out = streams[0]->own;
    return DRI_OK;
  }
  std::vector<dri_stream_s*> key(streams, streams + n);
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (Plan* q : g_batch_plans)
    if (q->slots == key) *out = q;
  if (*out) return DRI_OK;
  Plan* p = nullptr;
  const int r = plan_create(key.data(), n, kBatchRing, false, default_groups(n), &p);
  if (r != DRI_OK) return r;
  p->autotune = true;
  g_batch_plans.push_back(p);
  for (dri_stream_s* s : key) s->batches.push_back(p);
  *out = p;
  return DRI_OK;
}

}  // namespace dri_host

extern "C" {

int dri_track_batch(const dri_stream* streams, int32_t n, dri_track_result* out) {
  Plan* p = nullptr;
  const int rp = batch_plan(streams, n, &p);
  if (rp != DRI_OK) return rp;
  const std::vector<dri_stream_s*>& key = p->slots;
  std::vector<SlotWork> work(n);
  bool any = false;
  for (int i = 0; i < n; ++i) {
    if (settle(key[i], false) != DRI_OK) return DRI_ECUDA;
    work[i] = plan_slot_work(key[i]);
    any = any || work[i].mode != kSlotIdle;
  }
  if (!any) return DRI_ENOTREADY;
  std::vector<double> t0(n);
  for (int i = 0; i < n; ++i) t0[i] = key[i]->t_prev;
  int rs = -1;
  const int r = plan_launch(p, work, &rs);
  if (r != DRI_OK) return r;
  if (!out) return DRI_OK;
  CK(cudaEventSynchronize(p->ev[rs]));
  for (int i = 0; i < n; ++i) {
    if (settle(key[i], true) != DRI_OK) return DRI_ECUDA;
    if (work[i].mode == kSlotIdle) {
      std::memset(&out[i], 0, sizeof(out[i]));
      out[i].status = work[i].status;
      continue;
    }
    fill_result(key[i], ring_head(p, rs, i), &out[i], work[i].mode == kSlotInit, t0[i]);
  }
  return DRI_OK;
}

namespace {
// Tangent dimension of one state of the stream (the prior's size).
size_t prior_dim(const dri_stream_s* s) { return s->cfg.gravity_dof == DRI_GRAVITY_3D ? 18 : 17; }
}  // namespace

int dri_get_state(dri_stream s, dri_state* x1, double* H_prior, double* b_prior) {
  if (!s || !x1) return DRI_EINVAL;
  CK(cudaMemcpyAsync(s->pin_ctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  const Ctrl* h = s->pin_ctrl;
  *x1 = from_dstate(h->x, h->t_state);
  const size_t ns = prior_dim(s);
  if (H_prior) std::memcpy(H_prior, h->Hs, ns * ns * sizeof(double));
  if (b_prior) std::memcpy(b_prior, h->bs, ns * sizeof(double));
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
  const size_t ns = prior_dim(s);
  if (H_prior) std::memcpy(h->Hs, H_prior, ns * ns * sizeof(double));
  if (b_prior) std::memcpy(h->bs, b_prior, ns * sizeof(double));
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
  if (s->cfg.gravity_dof == DRI_GRAVITY_3D) return DRI_EINVAL;   // the output holds the 34-D system
  if (!s->initialised || !s->frame_pending) return DRI_ENOTREADY;
  if (settle(s, true) != DRI_OK) return DRI_ECUDA;
  size_t k0 = 0, k1 = 0;
  int r = select_imu(s, s->t_prev, s->t_frame, &k0, &k1);
  if (r != DRI_OK) return r;
  Plan* p = s->own;
  int rs = 0;
  if ((r = plan_acquire(p, &rs)) != DRI_OK) return r;
  char* img = p->pin_dyn + (size_t)rs * p->dyn_cap;
  std::memset(img, 0, dyn_header_bytes(1));
  const size_t off = dyn_header_bytes(1);
  const size_t used = off + stage_slot(s, img, 0, kSlotTrack, s->t_prev, s->t_frame, k0, k1, off);
  CK(cudaMemcpyAsync(p->dyn, img, used, cudaMemcpyHostToDevice, s->stream));
  CK(cudaEventRecord(p->ev[rs], s->stream));
  p->ring_used[rs] = 1;
  p->next = (p->next + 1) % p->R;
  // the maps of the pending frame (the frame itself stays pending)
  const int L = s->cfg.levels;
  const BatchArgs a0 = plan_args(p, p->tv.copy_off, 0, 0);
  CK(launch(s, DRI_KC_MAPS, 0.0, [&] { return launch_copy_batch(a0, p->pre_copy[1], s->stream); }));
  for (int l = 1; l < L; ++l) {
    const BatchArgs a = plan_args(p, p->tv.map_off[l], l, 0);
    CK(launch(s, DRI_KC_MAPS, 0.0, [&] { return launch_pyr_down_batch(a, p->pre_map[l][1], s->stream); }));
  }
  for (int l = 0; l < L; ++l) {
    const BatchArgs a = plan_args(p, p->tv.map_off[l], l, 0);
    CK(launch(s, DRI_KC_MAPS, 0.0,
              [&] { return launch_normals_batch(a, p->pre_map[l][1], p->fp16, s->stream); }));
  }
  const SolveParams sp = solve_params(s, level, 0);
  CK(launch(s, DRI_KC_FRAME, 0.0,
            [&] { return launch_linearise_begin(sp, to_dstate(*x0), to_dstate(*x1), s->stream); }));
  // The pixel terms come from the batched kernel that tracking runs, over the
  // stream's own one-slot plan (its rows per thread included).  The per-pixel
  // validity bits come from the same kernel's flag-writing instantiation,
  // launched first; the instantiation a level's last iteration runs (margin
  // decisions counted) then recomputes the sums the system is assembled from.
  const BatchArgs at = plan_args(p, track_start(p, level, 0), level, 0, 0, 1);
  const int nb = track_blocks(p, level, 0);
  const double px = (double)s->geom[level].w * s->geom[level].h;
  const size_t nflags = (size_t)s->geom[level].w * s->geom[level].h;
  if (flags) {
    BatchArgs af = at;
    af.flags = s->flags;
    CK(cudaMemsetAsync(s->flags, 0, nflags, s->stream));
    CK(launch(s, DRI_KC_TRACK, px, [&] {
      return launch_track_batch(af, nb, p->fp16, p->fp32p, p->opt, launch_priority(false), false, s->stream);
    }));
    // the flag-writing launch counted the margin decisions too: count once
    CK(cudaMemsetAsync(s->ctrl->margin_acc, 0, sizeof(s->ctrl->margin_acc), s->stream));
  }
  BatchArgs am = at;
  am.margin = 1;                   // the margin decisions, counted as a level's last iteration does
  CK(launch(s, DRI_KC_TRACK, px, [&] {
    return launch_track_batch(am, nb, p->fp16, p->fp32p, p->opt, launch_priority(false), false, s->stream);
  }));
  CK(launch(s, DRI_KC_SOLVE, 0.0, [&] { return launch_linearise_end(sp, s->lin_dev, s->stream); }));
  s->launches += 1 + 2 * L - 1 + 3 + (flags ? 1 : 0);
  CK(cudaMemcpyAsync(out, s->lin_dev, sizeof(*out), cudaMemcpyDeviceToHost, s->stream));
  if (flags) CK(cudaMemcpyAsync(flags, s->flags, nflags, cudaMemcpyDeviceToHost, s->stream));
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

int dri_batch_get_options(const dri_stream* streams, int32_t n, dri_batch_options* out) {
  if (!streams || n < 1 || !out) return DRI_EINVAL;
  const Plan* p = nullptr;
  if (n == 1) {
    if (!streams[0]) return DRI_EINVAL;
    p = streams[0]->own;
  } else {
    std::vector<dri_stream_s*> key(streams, streams + n);
    std::lock_guard<std::mutex> lk(g_batch_mu);
    for (const Plan* q : g_batch_plans)
      if (q->slots == key) p = q;
  }
  if (!p) return DRI_ENOTREADY;
  std::memset(out, 0, sizeof(*out));
  for (int l = 0; l < kMaxLevels; ++l) out->rows_per_thread[l] = l < p->levels ? p->ppt[0][l] : 0;
  out->groups = p->groups;
  out->autotune = p->autotune && !p->tuned ? 1 : 0;
  return DRI_OK;
}

int dri_batch_set_options(const dri_stream* streams, int32_t n, const dri_batch_options* opt) {
  if (!opt) return DRI_EINVAL;
  Plan* p = nullptr;
  const int r = batch_plan(streams, n, &p);
  if (r != DRI_OK) return r;
  if (opt->groups < 0 || opt->groups > std::min(p->S, kMaxGroups)) return DRI_EINVAL;
  if (!opt->autotune)
    for (int l = 0; l < p->levels; ++l)
      if (opt->rows_per_thread[l] < 1 || opt->rows_per_thread[l] > kMaxRowsPerThread) return DRI_EINVAL;
  CK(cudaStreamSynchronize(p->stream));      // in-flight frames read the current tables
  if (!opt->autotune)
    for (auto& v : p->ppt)
      for (int l = 0; l < p->levels; ++l) v[l] = opt->rows_per_thread[l];
  p->autotune = opt->autotune != 0;
  p->tuned = !p->autotune;
  if (opt->groups > 0) plan_set_groups(p, opt->groups);
  if (p->graph) {
    cudaGraphExecDestroy(p->graph);
    p->graph = nullptr;
  }
  p->graph_failed = false;
  plan_fill_tables(p);
  return plan_upload_tables(p);
}

}  // extern "C"
