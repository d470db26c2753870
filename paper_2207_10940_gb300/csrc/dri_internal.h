// Internal layout shared by the host API and the kernels of the tracking library.
//
// Device memory of one stream (one workspace allocation, 256-byte aligned parts):
//   Ctrl           FP64 state block: x, the iterates x0 / x1, the prior (H*, b*, xbar),
//                  W_IMU, the reference pose, the per-iteration pixel transforms, the
//                  folded sums and the last joint system (Sec. IV-D/E).
//   dyn            per-frame staging of the stream's own launch sequence: SlotDyn,
//                  then an ImuHeader and the samples covering [t0, t1].
//   table          SlotStatic of the stream and the block-count prefixes of its
//                  launches (the one-slot plan of dri_track).
//   input depth/I  level-0 host-upload target.
//   2 map sets     per level: depth and intensity planes, pack A (normal + depth) and
//                  pack B (intensity + gradient) per pixel, FP32 or FP16 (packs.cuh).
//                  Set ctrl.ref_index is the reference, the other the live frame; a
//                  tracked frame flips the index on the device (no host round trip).
//   partials       per-block sums of the pixel kernel (FP64 or FP32).
//   flags          per-pixel validity bytes for the parity entry point.
//
// Every launch of a frame is "batched": its blocks are spread over one or more
// slots (streams) by a prefix of per-slot block counts, each slot reading its
// static parameters (SlotStatic) from a device table and its per-frame mode,
// image pointers and IMU block from the staged dyn buffer.  dri_track runs the
// sequence over one slot, dri_track_batch over many.
#pragma once

#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "dri.h"

namespace dri {

constexpr int kMaxLevels = DRI_MAX_LEVELS;
constexpr int kSums = 29;             // per term: 21 (upper J J^T) + 6 (J e) + e^2 + count
constexpr int kSumsAll = 2 * kSums;   // ICP then photometric
constexpr int kTrackThreadsX = 32;
constexpr int kTrackThreadsY = 8;      // warps of a pixel-kernel block
constexpr int kTrackRows = 4;          // mixed-term tiles: rows per unit of rows-per-thread
constexpr int kFoldGroup = 16;        // blocks per first-level fold of the pixel kernel

struct DState {                       // Eq. 1
  double r[3];
  double q[4];
  double v[3];
  double bg[3];
  double ba[3];
  double qg[4];
};

struct Ctrl {
  // ---- result head: copied to the host after every frame ----
  DState x;                           // state after the last tracked frame
  DState x0, x1;                      // Gauss-Newton iterates of the current frame
  double cost;
  double t_state;                     // time of x
  int32_t n_icp[kMaxLevels], n_rgb[kMaxLevels];
  int32_t n_margin[kMaxLevels];       // margin decisions of the last iteration per level
  int32_t status;                     // DRI_OK or the frame's error
  int32_t ref_index;                  // map set holding the reference
  int32_t initialised;                // reference exists
  int32_t iterations;
  uint32_t block_counter;             // last-block detection of the pixel kernel
  uint32_t margin_acc[2];             // margin decisions of the running pixel kernel (ICP, photometric)
  uint32_t pad1;
  // ---- solver state ----
  DState xbar;                        // prior mean
  DState xstart;                      // state at frame start (restored on DRI_ELOST)
  double Hs[18 * 18];                 // prior information H* (Eq. 8a), ns x ns (ns = 17 or 18)
  double bs[18];                      // prior vector b* (Eq. 8b)
  double Wimu[18 * 18];               // IMU weight
  double Rref[9], rref[3];            // pose T_ref the reference maps were made at
  double sums[64];                    // folded pixel sums of the current iteration
  double H[36 * 36], b[36], d[36];    // last joint system and step (marginalisation), 2 ns
  float xf_icp[12];                   // R_ref^T R_1 - I (row-major), R_ref^T (r_1 - r_ref)
  float xf_rgb[12];                   // R_0^T R_1 - I, R_0^T (r_1 - r_0)
  // DRI_IMU_FIRST_ORDER: the frame's pre-integration at its linearisation point
  // (dR 9, dv 3, dp 3, Phi_g 9, V_g 9, P_g 9, V_a 9, P_a 9, T) and those biases
  double pre_lin[61];
  double b_lin[6];
};

// Bytes of the result head (x .. pad1) copied back after each frame.
constexpr size_t kCtrlHeadBytes = offsetof(Ctrl, xbar);

struct ImuHeader {
  double t0, t1;
  int32_t n;
  int32_t pad;
};

struct LevelGeom {
  int32_t w, h;
  float fx, fy, cx, cy, ifx, ify;
};

// Pointers of one pyramid level in both map sets (row-major, w * h pixels).
struct LevelMaps {
  float* depth[2];
  float* inten[2];
  void* packA[2];                     // per pixel normal + depth (packs.cuh)
  void* packB[2];                     // per pixel intensity + gradient (packs.cuh)
};

struct StreamLayout {
  size_t ctrl, dyn, dyn_bytes, table, in_depth, in_inten, counters, partials, gpartials, flags,
      lin_out, total;
  size_t level_off[kMaxLevels][2][4];  // per level, per set: depth, inten, pack A, pack B
  int64_t plane[kMaxLevels];
  int max_blocks;
  int imu_cap;
  int pack_bytes;                     // 16 (FP32) or 8 (FP16) per pack element
};

struct TrackParams {
  LevelGeom g;
  LevelMaps m;
  Ctrl* ctrl;
  void* partials;                     // per-block partial sums
  void* gpartials;                    // per-group partial sums
  uint32_t* counters;                 // [0]: groups done, [1 + g]: blocks of group g done
  uint8_t* flags;
  int32_t nblocks;
  int32_t ppt;                        // pixel rows per thread
  float depth_min, depth_max;
  float icp_dist2, icp_cos;
  float occ_thr;                      // > 0: photometric depth-consistency test (m)
  int32_t icp_dw;                     // 1: ICP weight 1 / d^4 (depth-dependent noise)
};

struct SolveParams {
  Ctrl* ctrl;
  const ImuHeader* imu;               // followed by the samples
  int32_t level;
  int32_t last;                       // 1 on the frame's last iteration
  // configuration (copied from dri_stream_config)
  double R_CS[9], r_CS[3];
  double W_icp, W_rgb;
  double gyr_nd, acc_nd, gyr_rw, acc_rw, g, sigma_grav;
  double prior_sigma[5];
  int32_t min_valid;
  int32_t imu_cap;
  int32_t imu_mode;                   // DRI_IMU_REINTEGRATE or DRI_IMU_FIRST_ORDER
  int32_t gdof;                       // gravity degrees of freedom: 2 or 3 (state dimension 15 + gdof)
  double relin_g, relin_a;            // first order: re-integration thresholds
  int32_t track_mode;                 // DRI_TRACK_INERTIAL, _RGBD_ONLY or _GYRO_ONLY
  int32_t pad2;
  double rgbd_lambda;                 // RGB-D-only: photometric weight
};

// ---- batched launches --------------------------------------------------------
enum SlotMode : int32_t { kSlotIdle = 0, kSlotTrack = 1, kSlotInit = 2 };

constexpr int kCopyTileW = 128;       // level-0 input copy: 32 x 8 threads, 4 pixels each
constexpr int kCopyTileH = 8;
constexpr int kMapTileW = 32;         // pyramid, normal and gradient maps: 32 x 8 threads
constexpr int kMapTileH = 8;          // block rows; a thread takes kMapRows rows of its tile
constexpr int kMapRows = 8;           // 32 x 64 tiles: 8 rows per thread measured 1.4-1.6x faster
                                      // than one (block scheduling dominated 256-pixel blocks)

// Per-slot parameters fixed for the life of a plan.
struct SlotStatic {
  TrackParams tp[kMaxLevels];         // flags = nullptr; ppt / nblocks as planned
  SolveParams sp;                     // imu, level and last are set per launch
  const float* in_depth;              // level-0 host-upload target
  const float* in_inten;
  int32_t levels;
  int32_t pad;
};

// Per-slot record staged with every launch of a frame.
struct SlotDyn {
  int32_t mode;                       // SlotMode
  int32_t pitch;                      // source row pitch, floats
  int64_t imu_off;                    // byte offset of the slot's ImuHeader in the dyn buffer
  const float* src_depth;             // this frame's level-0 images (device)
  const float* src_inten;
};

// Table of one plan in device memory: SlotStatic[nslots], then the int32
// block prefixes copy[n + 1], map[levels][n + 1] and, per level, one prefix of
// n_g + 1 entries for each of the G slot groups of the Gauss-Newton loop
// (group g's at entry first_slot(g) + g).
struct TableView {
  size_t copy_off, map_off[kMaxLevels], track_off[kMaxLevels], bytes;
};
TableView table_view(int nslots, int levels, int groups);

// Kernel argument of every batched launch: it covers slots slot0 ..
// slot0 + nslots - 1 of the plan (all of them, or one group of the
// Gauss-Newton loop).
struct BatchArgs {
  const SlotStatic* slots;            // every slot of the plan
  const unsigned char* dyn;           // SlotDyn[all slots], then the IMU blocks
  const int32_t* start;               // block prefix over this launch's slots (nslots + 1)
  int32_t slot0;
  int32_t nslots;
  int32_t level;
  int32_t last;                       // 1 on the frame's last Gauss-Newton iteration
  int32_t margin;                     // pixel kernel: count margin decisions (a level's last iteration)
  uint8_t* flags;                     // pixel kernel, parity entry only: per-pixel validity and
                                      // margin bits (one slot, zeroed before the launch); nullptr
                                      // otherwise
};

// Index (0 .. nslots - 1, relative to slot0) of the launch slot owning `block`.
__device__ __forceinline__ int batch_slot(const BatchArgs& a, int block) {
  int lo = 0, hi = a.nslots;          // start[lo] <= block < start[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(a.start + mid) <= block) lo = mid;
    else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ const SlotDyn& batch_dyn(const BatchArgs& a, int slot) {
  return reinterpret_cast<const SlotDyn*>(a.dyn)[slot];
}

StreamLayout make_layout(const dri_stream_config& cfg);
LevelGeom level_geom(const dri_stream_config& cfg, int level);

// ---- kernel launchers (return cudaGetLastError()) ------------------------
// Uploaded reference: level-0 vertex / normal maps (x, y, z per pixel, W frame),
// intensity, rows `pitch` pixels apart, and the pose T_ref they were rendered at.
struct RefUpload {
  const float* V;
  const float* N;
  const float* I;
  int64_t pitch;
  double R[9], r[3];
};
cudaError_t launch_upload_reference(const LevelMaps* m, const LevelGeom* g, int levels, Ctrl* ctrl,
                                    float dmin, float dmax, bool fp16, const RefUpload& up,
                                    cudaStream_t s);
cudaError_t launch_copy_batch(const BatchArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_pyr_down_batch(const BatchArgs& a, int blocks, cudaStream_t s);
cudaError_t launch_normals_batch(const BatchArgs& a, int blocks, bool fp16, cudaStream_t s);
cudaError_t launch_gradient_batch(const BatchArgs& a, int blocks, bool fp16, cudaStream_t s);
inline int copy_tiles(int w, int h) {
  return ((w + kCopyTileW - 1) / kCopyTileW) * ((h + kCopyTileH - 1) / kCopyTileH);
}
inline int map_tiles(int w, int h) {
  return ((w + kMapTileW - 1) / kMapTileW) * ((h + kMapTileH * kMapRows - 1) / (kMapTileH * kMapRows));
}
cudaError_t launch_normals(const LevelMaps& m, const Ctrl* ctrl, const LevelGeom& g,
                           float dmin, float dmax, bool fp16, int which_set, cudaStream_t s);
cudaError_t launch_gradient(const LevelMaps& m, const Ctrl* ctrl, int w, int h, bool fp16,
                            cudaStream_t s);
cudaError_t launch_track(const TrackParams& p, bool fp16, bool fp32_partials, cudaStream_t s);

#ifdef __CUDACC__
// Programmatic dependent launch between the batched pixel kernel and the
// Gauss-Newton step (each launched with programmatic stream serialization):
// grid_dep_wait blocks until the preceding kernel has completed and its writes
// are visible (immediately when there is no programmatic dependency);
// grid_dep_launch lets the next kernel's blocks start once every block of this
// one has reached it.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" :::); }
#endif
// Block-scheduling priority of a batched launch: the greatest for the
// Gauss-Newton steps (solver), one below for the pixel kernels, so that a slot
// group's step takes the SMs that free up before the pixel blocks of the other
// groups that wait for them (measured on 4 groups of 16 x 640x480: 10.9k frames/s
// without priorities, 12.3k with; an order among the groups' pixel kernels
// gained nothing).
int launch_priority(bool solver);
// opt: the pixel-kernel variant, bit 0 the occlusion test, bit 1 the depth-dependent ICP weight;
// early: programmatic dependent launch after the preceding Gauss-Newton step (its
// blocks then wait on the SMs for the step's end, which only pays when no other
// slot group could use those SMs meanwhile)
cudaError_t launch_track_batch(const BatchArgs& a, int blocks, bool fp16, bool fp32_partials, int opt,
                               int priority, bool early, cudaStream_t s);
int track_grid_blocks(int w, int h, int ppt);   // batched kernel: single-term blocks
int track_mixed_blocks(int w, int h, int ppt);  // by-value kernel: mixed-term blocks
int track_default_ppt(int w, int h);
inline int fold_groups(int nblocks) { return (nblocks + kFoldGroup - 1) / kFoldGroup; }

cudaError_t prepare_solver_kernels();   // opt-in shared memory sizes (current device)
int solver_max_imu_pieces();
cudaError_t launch_frame_begin_batch(const BatchArgs& a, cudaStream_t s);
// g3: some slot of the launch has the 3-D gravity form (larger shared memory)
cudaError_t launch_gn_step_batch(const BatchArgs& a, bool g3, cudaStream_t s);
cudaError_t launch_frame_end_batch(const BatchArgs& a, cudaStream_t s);
cudaError_t launch_gather_heads(const BatchArgs& a, unsigned char* out, cudaStream_t s);
cudaError_t launch_linearise_begin(const SolveParams& p, const DState& x0, const DState& x1,
                                   cudaStream_t s);
cudaError_t launch_linearise_end(const SolveParams& p, dri_linearisation* out, cudaStream_t s);

}  // namespace dri
