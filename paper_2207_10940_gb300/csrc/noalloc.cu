// Linearisation of one image pair with no allocation of any kind.
//
// Who needs this: code that may not call cudaMalloc / cudaFree when it runs --
// for example a host framework that owns all device memory and forbids
// allocation inside its per-frame callback, a real-time thread that must not
// block in the allocator, or work recorded while a CUDA stream capture is
// active (allocation calls are illegal there).  Creating a tracking stream
// allocates (its workspace, pinned staging, events), so such code cannot use
// the stream API on the fly.  This entry point takes the caller's device images
// and a caller-owned device output and keeps every intermediate it needs (the
// normal and gradient maps, the pixel kernel's per-block partial sums and its
// completion counter, the per-call transforms, the per-pixel flag bytes before
// they are copied to the caller) in one file-scope static device
// array, held until the process exits.  The array is device memory of the
// library's module: the CUDA runtime reserves it when it loads the module on a
// device, which with lazy module loading (the default since CUDA 12.2) happens
// at the first call made with that device current, so that first call itself
// reserves about 4 MB; later calls reserve nothing.
//
// Limits and rules:
//  * at most kNoallocMaxPixels = 320 * 240 pixels per image; larger images are
//    rejected with DRI_EINVAL before anything is launched;
//  * the static array is shared by every call on a device and keeps the last
//    call's contents; each call re-initialises what must start at zero (the
//    fold counters and the status word) before its kernels run;
//  * calls whose GPU work overlaps (different streams or host threads, without
//    ordering between them) race on the array: order them on one stream;
//  * the device address of the array is looked up once per device, on the first
//    call made with that device current (cudaGetSymbolAddress); make that first
//    call before any stream capture begins.
#include <cmath>
#include <cstring>
#include <mutex>

#include "dri_internal.h"
#include "so3.cuh"

namespace dri {
namespace {

constexpr int kNoallocMaxW = 320;
constexpr int kNoallocMaxH = 240;
constexpr int64_t kNoallocMaxPixels = (int64_t)kNoallocMaxW * kNoallocMaxH;
constexpr size_t kAlignNA = 256;
constexpr size_t na_align(size_t v) { return (v + kAlignNA - 1) / kAlignNA * kAlignNA; }

constexpr int64_t kPlane = (kNoallocMaxPixels + 63) / 64 * 64;
constexpr size_t kOffCtrl = 0;
constexpr size_t kOffPackA0 = na_align(kOffCtrl + sizeof(Ctrl));       // reference normals + depth
constexpr size_t kOffPackA1 = na_align(kOffPackA0 + kPlane * 16);         // live normals + depth
constexpr size_t kOffPackB = na_align(kOffPackA1 + kPlane * 16);          // reference intensity + gradient
// one row per thread: at most ceil(320/32) * ceil(240/4) blocks
constexpr int kNoallocMaxBlocks = ((kNoallocMaxW + kTrackThreadsX - 1) / kTrackThreadsX) *
                                  ((kNoallocMaxH + kTrackRows - 1) / kTrackRows);
constexpr int kNoallocMaxGroups = (kNoallocMaxBlocks + kFoldGroup - 1) / kFoldGroup;
constexpr size_t kOffCounters = na_align(kOffPackB + kPlane * 16);
constexpr size_t kOffPartials = na_align(kOffCounters + (1 + kNoallocMaxGroups) * sizeof(uint32_t));
constexpr size_t kOffGPartials = na_align(kOffPartials + (size_t)kNoallocMaxBlocks * kSumsAll * sizeof(double));
// per-pixel flag bytes, or-ed in by 32-bit words, then copied to the caller's buffer
constexpr size_t kOffFlags = na_align(kOffGPartials + (size_t)kNoallocMaxGroups * kSumsAll * sizeof(double));
constexpr size_t kNoallocBytes = na_align(kOffFlags + (size_t)kPlane);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Per-call set-up: transforms of the pixel kernel from (x_ref, x0, x1) exactly as
// the stream path computes them, status and counter cleared, set 0 = reference.
__global__ void k_noalloc_begin(Ctrl* c, uint32_t* counters, DState xref, DState x0, DState x1) {
  for (int i = threadIdx.x; i < 1 + kNoallocMaxGroups; i += blockDim.x) counters[i] = 0u;
  if (threadIdx.x != 0) return;
  double Rref[9], R0[9], R1[9], M[9], dr[3], t[3];
  quat_to_rot(xref.q, Rref);
  quat_to_rot(x0.q, R0);
  quat_to_rot(x1.q, R1);
  for (int i = 0; i < 9; ++i) c->Rref[i] = Rref[i];
  for (int i = 0; i < 3; ++i) c->rref[i] = xref.r[i];
  c->x0 = x0;
  c->x1 = x1;
  m3_tmul(Rref, R1, M);
  for (int i = 0; i < 3; ++i) dr[i] = x1.r[i] - xref.r[i];
  m3_tvec(Rref, dr, t);
  for (int i = 0; i < 9; ++i) c->xf_icp[i] = (float)(M[i] - ((i % 4 == 0) ? 1.0 : 0.0));
  for (int i = 0; i < 3; ++i) c->xf_icp[9 + i] = (float)t[i];
  m3_tmul(R0, R1, M);
  for (int i = 0; i < 3; ++i) dr[i] = x1.r[i] - x0.r[i];
  m3_tvec(R0, dr, t);
  for (int i = 0; i < 9; ++i) c->xf_rgb[i] = (float)(M[i] - ((i % 4 == 0) ? 1.0 : 0.0));
  for (int i = 0; i < 3; ++i) c->xf_rgb[9 + i] = (float)t[i];
  c->status = 0;
  c->ref_index = 0;
  c->block_counter = 0u;
  c->margin_acc[0] = c->margin_acc[1] = 0u;
}

// Weighted world-frame systems of both terms from the folded sums (the pixel
// kernel works in the reference / x0 camera frames: H_W = Q H Q^T, Q = diag(R, R)).
__global__ void k_noalloc_end(const Ctrl* c, double W_icp, double W_rgb, dri_linearisation* out) {
  const int tid = threadIdx.x;
  if (tid < 2 * 36) {
    const int term = tid / 36, idx = tid % 36;
    const int i = idx / 6, j = idx % 6;
    double R[9];
    if (term == 0) {
      for (int k = 0; k < 9; ++k) R[k] = c->Rref[k];
    } else {
      quat_to_rot(c->x0.q, R);
    }
    const double* s = c->sums + term * kSums;
    auto hloc = [&](int a, int b) {
      const int lo = a < b ? a : b, hi = a < b ? b : a;
      return s[lo * 6 - lo * (lo - 1) / 2 + (hi - lo)];
    };
    double acc = 0.0;
    const int bi = i / 3, ri = i % 3, bj = j / 3, rj = j % 3;
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) acc += R[ri * 3 + k] * hloc(bi * 3 + k, bj * 3 + l) * R[rj * 3 + l];
    const double w = term == 0 ? W_icp : W_rgb;
    (term == 0 ? out->H_icp : out->H_rgb)[idx] = w * acc;
    if (j == 0) {
      double g = 0.0;
      for (int k = 0; k < 3; ++k) g += R[ri * 3 + k] * s[21 + bi * 3 + k];
      (term == 0 ? out->b_icp : out->b_rgb)[i] = -w * g;
    }
  }
  for (int idx = tid; idx < 34 * 34; idx += blockDim.x) out->H[idx] = 0.0;
  if (tid < 34) out->b[tid] = 0.0;
  if (tid < 18) out->e_imu[tid] = 0.0;
  if (tid == 0) {
    out->cost_icp = W_icp * c->sums[27];
    out->cost_rgb = W_rgb * c->sums[kSums + 27];
    out->cost_imu = 0.0;
    out->n_icp = (int64_t)c->sums[28];
    out->n_rgb = (int64_t)c->sums[kSums + 28];
    out->n_margin_icp = c->margin_acc[0];
    out->n_margin_rgb = c->margin_acc[1];
  }
}

// A state the kernels can use: finite, with a non-zero orientation quaternion.
bool usable_state(const dri_state& s) {
  double nq = 0.0;
  for (int i = 0; i < 4; ++i) nq += s.q_WC[i] * s.q_WC[i];
  if (!(nq > 0.0) || !std::isfinite(nq)) return false;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(s.r_WC[i]) || !std::isfinite(s.v_I[i]) || !std::isfinite(s.bg[i]) ||
        !std::isfinite(s.ba[i]))
      return false;
  for (int i = 0; i < 4; ++i)
    if (!std::isfinite(s.q_IW[i])) return false;
  return true;
}

DState dstate_of(const dri_state& s) {
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
  nq = sqrt(nq);
  ng = sqrt(ng);
  for (int i = 0; i < 4; ++i) {
    d.q[i] = s.q_WC[i] / nq;
    d.qg[i] = ng > 0 ? s.q_IW[i] / ng : (i == 0 ? 1.0 : 0.0);
  }
  return d;
}

// Device address of the static array for the current device, looked up once.
int scratch_address(unsigned char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return DRI_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return DRI_EINVAL;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return DRI_ECUDA;
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
  return DRI_OK;
}

}  // namespace
}  // namespace dri

using namespace dri;

extern "C" int dri_linearise_pair_noalloc(const dri_stream_config* cfg, const float* ref_depth,
                                          const float* ref_intensity, const float* live_depth,
                                          const float* live_intensity, const dri_state* x_ref,
                                          const dri_state* x0, const dri_state* x1,
                                          dri_linearisation* out, uint8_t* flags, void* cuda_stream) {
  if (!cfg || !ref_depth || !ref_intensity || !live_depth || !live_intensity || !x_ref || !x0 ||
      !x1 || !out)
    return DRI_EINVAL;
  if (cfg->width < 8 || cfg->height < 8 || cfg->width > kNoallocMaxW || cfg->height > kNoallocMaxH ||
      (int64_t)cfg->width * cfg->height > kNoallocMaxPixels)
    return DRI_EINVAL;
  if (!(cfg->fx > 0) || !(cfg->fy > 0) || !(cfg->sigma_I > 0) || !(cfg->sigma_d > 0) ||
      !(cfg->depth_max > cfg->depth_min) || !(cfg->icp_dist_thr > 0) ||
      !(cfg->icp_angle_thr_deg > 0) || !(cfg->icp_angle_thr_deg < 90))
    return DRI_EINVAL;
  if ((cfg->precision_flags & ~(DRI_FP16_MAPS | DRI_FP32_PARTIALS)) != 0 ||
      !(cfg->occlusion_thr >= 0.0) || !std::isfinite(cfg->occlusion_thr) ||
      (cfg->icp_depth_weight != 0 && cfg->icp_depth_weight != 1))
    return DRI_EINVAL;
  if (!usable_state(*x_ref) || !usable_state(*x0) || !usable_state(*x1)) return DRI_EINVAL;
  const bool fp16 = (cfg->precision_flags & DRI_FP16_MAPS) != 0;
  const bool fp32p = (cfg->precision_flags & DRI_FP32_PARTIALS) != 0;
  unsigned char* base = nullptr;
  const int r = scratch_address(&base);
  if (r != DRI_OK) return r;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Ctrl* ctrl = reinterpret_cast<Ctrl*>(base + kOffCtrl);

  LevelGeom g = level_geom(*cfg, 0);
  LevelMaps m;
  std::memset(&m, 0, sizeof(m));
  m.depth[0] = const_cast<float*>(ref_depth);      // set 0: reference
  m.inten[0] = const_cast<float*>(ref_intensity);
  m.depth[1] = const_cast<float*>(live_depth);     // set 1: live frame
  m.inten[1] = const_cast<float*>(live_intensity);
  m.packA[0] = base + kOffPackA0;
  m.packA[1] = base + kOffPackA1;
  m.packB[0] = base + kOffPackB;
  m.packB[1] = base + kOffPackB;                    // the live set's pack B is never read

  uint32_t* counters = reinterpret_cast<uint32_t*>(base + kOffCounters);
  k_noalloc_begin<<<1, 32, 0, s>>>(ctrl, counters, dstate_of(*x_ref), dstate_of(*x0), dstate_of(*x1));
  if (cudaGetLastError() != cudaSuccess) return DRI_ECUDA;
  const float dmin = (float)cfg->depth_min, dmax = (float)cfg->depth_max;
  if (launch_normals(m, ctrl, g, dmin, dmax, fp16, 0, s) != cudaSuccess) return DRI_ECUDA;
  if (launch_normals(m, ctrl, g, dmin, dmax, fp16, 1, s) != cudaSuccess) return DRI_ECUDA;
  if (launch_gradient(m, ctrl, g.w, g.h, fp16, s) != cudaSuccess) return DRI_ECUDA;

  TrackParams p;
  std::memset(&p, 0, sizeof(p));
  p.g = g;
  p.m = m;
  p.ctrl = ctrl;
  p.partials = base + kOffPartials;
  p.gpartials = base + kOffGPartials;
  p.counters = counters;
  p.flags = flags ? base + kOffFlags : nullptr;
  p.ppt = 1;
  p.nblocks = track_mixed_blocks(g.w, g.h, 1);
  if (p.nblocks > kNoallocMaxBlocks) return DRI_EINVAL;
  p.depth_min = dmin;
  p.depth_max = dmax;
  p.icp_dist2 = (float)(cfg->icp_dist_thr * cfg->icp_dist_thr);
  p.icp_cos = (float)std::cos(cfg->icp_angle_thr_deg * 3.14159265358979323846 / 180.0);
  p.occ_thr = (float)cfg->occlusion_thr;
  p.icp_dw = cfg->icp_depth_weight;
  if (flags && cudaMemsetAsync(p.flags, 0, (size_t)g.w * g.h, s) != cudaSuccess) return DRI_ECUDA;
  if (launch_track(p, fp16, fp32p, s) != cudaSuccess) return DRI_ECUDA;
  if (flags && cudaMemcpyAsync(flags, p.flags, (size_t)g.w * g.h, cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return DRI_ECUDA;
  k_noalloc_end<<<1, 128, 0, s>>>(ctrl, 1.0 / (cfg->sigma_d * cfg->sigma_d),
                                  1.0 / (cfg->sigma_I * cfg->sigma_I), out);
  if (cudaGetLastError() != cudaSuccess) return DRI_ECUDA;
  return DRI_OK;
}
