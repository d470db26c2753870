// Host-side state of the tracking library shared by the C ABI (api.cpp) and
// the serving loop (server.cpp): a stream's workspace views and bookkeeping,
// and the plan (the launch sequence of one frame over one or more streams).
#pragma once

#include <array>
#include <deque>
#include <mutex>
#include <vector>

#include <cuda_runtime.h>

#include "dri_internal.h"

using dri::Ctrl;
using dri::DState;
using dri::LevelGeom;
using dri::LevelMaps;
using dri::SlotStatic;
using dri::StreamLayout;
using dri::TableView;
using dri::kMaxLevels;
using dri::kSlotIdle;
using dri::kSlotInit;
using dri::kSlotTrack;

struct Plan;

struct dri_stream_s {
  dri_stream_config cfg;
  StreamLayout L;
  cudaStream_t stream = nullptr;
  char* ws = nullptr;
  bool own_ws = false;
  Ctrl* ctrl = nullptr;
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
  Plan* own = nullptr;              // one-slot plan of dri_track (in the workspace)
  std::vector<Plan*> batches;       // batch plans this stream is a slot of
  // host bookkeeping
  std::vector<dri_imu_sample> imu;
  bool initialised = false;         // host view: the init frame was enqueued
  double t_prev = 0.0;              // time of the state the next frame starts from
  double t_frame = 0.0;
  bool frame_pending = false;
  const float* src_depth = nullptr; // the pending frame's level-0 images on the device
  const float* src_inten = nullptr;
  int32_t src_pitch = 0;            // floats
  int64_t h2d_frame = 0;            // bytes of the pending frame's host upload
  Ctrl* pin_ctrl = nullptr;         // pinned copy of the whole control block
  // frames in flight, settled in order once their result copy has completed
  struct InFlight { cudaEvent_t ev; const Ctrl* head; };
  std::deque<InFlight> inflight;
  double t_confirmed = 0.0;         // time of the last state known to be good
  int64_t frames_ok = 0, frames_failed = 0;
  double t_prev_before = 0.0;       // t_prev before the last optimistic advance
  int64_t launches = 0;
  int64_t h2d_last = 0, d2h_last = 0;   // bytes copied for the last frame
  // profiling: event pairs around launches
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  struct Rec { int cls; size_t e0, e1; double pixels; };
  std::vector<Rec> recs;
  dri_profile counted;
  float* ref_stage = nullptr;       // device staging of host reference uploads (allocated on demand)
};

// The launch sequence of one frame over nslots streams: the device table of
// the slots' static parameters, the staging ring, the captured graph.
struct Plan {
  std::vector<dri_stream_s*> slots;
  cudaStream_t stream = nullptr;
  int S = 0, levels = 0;
  int iters[kMaxLevels] = {};
  bool fp16 = false, fp32p = false;
  int opt = 0;                      // pixel-kernel options of every slot: 1 occlusion test, 2 depth weight
  bool g3 = false;                  // some slot has the 3-D gravity form (its step's shared memory)
  bool margins = false;             // some slot counts margin decisions (count_margins)
  bool owns_device = false;         // table / dyn / heads allocated by the plan
  int groups = 1;                   // slot groups of the Gauss-Newton loop, one CUDA stream each
  std::vector<int> gfirst, gcount;
  std::vector<cudaStream_t> aux;    // streams of groups 1 .. groups - 1
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_grad = nullptr;    // the gradient maps' side stream is done
  cudaEvent_t ev_start = nullptr;   // the frame's inputs are staged (frame start may run)
  cudaEvent_t ev_begin = nullptr;   // the frame start is done
  cudaEvent_t ev_maps = nullptr;    // the pyramid is built (fine-level normals may start)
  cudaEvent_t ev_norm = nullptr;    // the fine-level normal maps are built
  bool norm_side = false;           // this frame's fine-level normals are on the side stream
  std::vector<cudaEvent_t> ev_join;
  char* table = nullptr;
  TableView tv;
  unsigned char* dyn = nullptr;
  size_t dyn_cap = 0;
  unsigned char* heads = nullptr;   // S result heads (batch plans)
  std::vector<SlotStatic> host_slots;
  std::vector<int32_t> pre_copy, pre_map[kMaxLevels], pre_track[kMaxLevels];
  int R = 0;                        // staging ring
  char* pin_dyn = nullptr;
  char* pin_heads = nullptr;
  std::vector<cudaEvent_t> ev;
  std::vector<char> ring_used;
  int next = 0;
  cudaGraphExec_t graph = nullptr;
  bool graph_failed = false;
  bool autotune = false;            // choose rows per thread by timing, on the first tracked frame
  bool tuned = false;
  std::vector<std::array<int, kMaxLevels>> ppt;   // rows per thread of each slot's pixel kernel
  int64_t kernels_per_frame = 0;
};

// Pixel-kernel variant a stream's configuration selects: bit 0 the photometric
// occlusion test, bit 1 the depth-dependent ICP weight.  The streams of one
// batch or server share it.
inline int pixel_options(const dri_stream_config& c) {
  return (c.occlusion_thr > 0 ? 1 : 0) | (c.icp_depth_weight ? 2 : 0);
}

namespace dri_host {

// Per-slot decision for one launch of plan p.
struct SlotWork {
  int mode = kSlotIdle;
  int status = DRI_ENOTREADY;       // result for a slot that does not run
  size_t k0 = 0, k1 = 0;
};

// Settles, in order, the stream's frames whose result copy has completed
// (all of them when wait is set).
int settle(dri_stream_s* s, bool wait);
// Mode and IMU range of the stream's pending frame for the next launch.
SlotWork plan_slot_work(const dri_stream_s* s);
// Stages and launches one frame of every slot with work; *ring_slot receives
// the staging slot whose event and result heads belong to this launch.
int plan_launch(Plan* p, const std::vector<SlotWork>& work, int* ring_slot);
// Result head of slot i of the launch staged in ring slot `slot`.
const Ctrl* ring_head(const Plan* p, int slot, int i);
// The plan of a stream list (the stream's own for one stream, else the cached
// batch plan of exactly this list, created on first use).
int batch_plan(const dri_stream* streams, int32_t n, Plan** out);
// Frees the cached batch plan of exactly this list (after waiting for it), if any.
void release_batch_plan(const std::vector<dri_stream_s*>& key);
void fill_result(const dri_stream_s* s, const Ctrl* h, dri_track_result* out, bool init, double t0);

}  // namespace dri_host
