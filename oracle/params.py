"""Constants and tracker configuration of the oracle.

Oracle code (test infrastructure only).

Table I (Sec. VI), synthetic-dataset column: noise densities, bias priors,
bias random walks ("drift noise density"), gravity and IMU rate.  Saturation
limits (7.8 rad/s, 176 m/s^2) are never reached by the synthetic workloads and
are not applied.

Readings where the paper is silent (Sec. IV-B/D give no thresholds, weights
or schedule):
* W_RGB = 1 / sigma_I^2 with sigma_I = 0.01 (intensity in [0, 1]) and
  W_ICP = 1 / sigma_d^2 with sigma_d = 0.002 m: the inverse covariances the
  text asks for (Sec. III, Sec. IV-D), constant per pixel.  Table I's
  "intensity noise 4.0" (no units) and "disparity noise 5.5 px" do not map onto
  these synthetic images.
* Data association: nearest reference pixel floor(x + 0.5), accepted when
  the points are closer than 0.10 m and their normals differ by less than
  20 degrees; depths are valid in [0.3, 8.0] m.  No robust kernel, no
  occlusion test, no photometric gradient threshold.
* Prior for the first frame (W is the first camera frame, Sec. II): diagonal
  with pose 1e-6 (m, rad), velocity 0.1 m/s, gyro / accelerometer bias
  0.03 rad/s and 0.1 m/s^2 (Table I bias priors), gravity direction 0.1 rad.
* Gravity-direction process noise between consecutive frames: 1e-4 rad.
* IMU term per Gauss-Newton iteration (imu_mode): 0 re-integrates the samples
  at x_0's current biases (exact); 1 applies Forster et al.'s first-order bias
  update to the pre-integration made at the frame's linearisation point (x_0's
  biases when the frame starts) and re-integrates, making the current biases
  the new linearisation point, once |db_g| > 0.01 rad/s or |db_a| > 0.1 m/s^2
  (Euclidean norms; the paper gives no thresholds).
* RGB-D-only baseline (track_mode 1; the vision-only tracker the paper
  compares with, Sec. III: ElasticFusion estimates the current pose only and
  weighs the photometric against the geometric term with a tuning parameter
  lambda): the unknowns are x_1's pose; x_0 (the previous result) stays fixed
  and the photometric term still warps with it; x_1 starts at x_0; the system
  is H_icp + lambda H_rgb on x_1's pose (the per-pixel weights W_ICP, W_RGB
  kept, lambda = 1 by default); no IMU term, prior or marginalisation.
* Gyro-only variant (track_mode 2; Sec. VII, Fig. 5 and Table VI, where the
  accelerometer-related residuals are ignored): the IMU term keeps its rotation
  rows and the gyro-bias random walk, weighted by the inverse of their own
  covariance (the (rotation, b_g) block of Sigma, so that the dropped rows'
  correlations do not leak in); the position, velocity, accelerometer-bias and
  gravity rows are dropped.  Nothing then measures the velocity, the
  accelerometer bias or the gravity direction, so they are held at their
  values (removed from both states' tangent spaces: identity rows in the
  system, no prior on them).  x_1 starts at x_0's position with the gyro's
  rotation prediction R_WC0 R_CS dR R_CS^T; the prior and the marginalisation
  act on the remaining 9 components of each state (pose and b_g).
* Occlusion test (occlusion_thr > 0; off by default, the paper gives none):
  a photometric residual is used only where the warped point's depth in x_0's
  camera agrees within occlusion_thr with the reference depth at the nearest
  reference pixel floor(x + 0.5), when that depth is valid (> 0); a point
  behind or in front of what the reference saw there changed visibility.
* Depth-dependent ICP weight (icp_depth_weight = 1; off by default, the
  synthetic sensor's depth noise is constant): the axial noise of a
  structured-light or stereo sensor grows with the square of the depth, so
  sigma_d(z) = sigma_d (z / 1 m)^2 and a pixel's ICP weight is W_ICP / z^4
  with z its live depth in metres.
"""
from __future__ import annotations

from dataclasses import dataclass, field

GRAVITY = 9.81                 # Table I, m s^-2
GYR_NOISE_DENSITY = 12.0e-4    # Table I, rad s^-1 Hz^-0.5
ACC_NOISE_DENSITY = 8.0e-3     # Table I, m s^-2 Hz^-0.5
GYR_BIAS_PRIOR = 0.03          # Table I, rad s^-1
ACC_BIAS_PRIOR = 0.1           # Table I, m s^-2
GYR_DRIFT_DENSITY = 4.0e-6     # Table I, rad s^-2 Hz^-0.5
ACC_DRIFT_DENSITY = 2.0e-5     # Table I, m s^-3 Hz^-0.5
IMU_RATE = 200.0               # Table I, Hz


@dataclass
class TrackerConfig:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float
    levels: int = 3
    iters: tuple = (10, 5, 4)           # iterations per level, index 0 = finest
    R_CS: object = None                 # 3x3, IMU frame S in camera frame C
    r_CS: object = None                 # position of S in C
    sigma_I: float = 0.01
    sigma_d: float = 0.002
    gyr_nd: float = GYR_NOISE_DENSITY
    acc_nd: float = ACC_NOISE_DENSITY
    gyr_rw: float = GYR_DRIFT_DENSITY
    acc_rw: float = ACC_DRIFT_DENSITY
    g: float = GRAVITY
    sigma_grav_rw: float = 1e-4
    icp_dist_thr: float = 0.10
    icp_angle_thr_deg: float = 20.0
    depth_min: float = 0.3
    depth_max: float = 8.0
    prior_sigma: dict = field(default_factory=lambda: dict(
        pose=1e-6, v=0.1, bg=GYR_BIAS_PRIOR, ba=ACC_BIAS_PRIOR, grav=0.1))
    min_valid: int = 64                 # level-0 correspondences below this: tracking lost
    fp16_maps: bool = False             # normals and intensity gradients rounded to FP16
    imu_mode: int = 0                   # 0 re-integrate per iteration, 1 first-order bias update
    bias_relin_g: float = 0.01          # |db_g| (rad/s) above which mode 1 re-integrates
    bias_relin_a: float = 0.1           # |db_a| (m/s^2) above which mode 1 re-integrates
    track_mode: int = 0                 # 0 RGB-D-inertial (joint), 1 RGB-D-only pose, 2 gyro only
    rgbd_lambda: float = 1.0            # track_mode 1: weight of the photometric term
    occlusion_thr: float = 0.0          # > 0: photometric depth-consistency test (m)
    icp_depth_weight: int = 0           # 1: ICP weight W_ICP / z^4 (sigma_d at 1 m)

    def level_camera(self, level):
        """Intrinsics at pyramid level l: f_l = f / 2^l, c_l = (c + 0.5) / 2^l - 0.5
        (the centre of a 2x2 block of the finer level)."""
        s = 2.0 ** level
        return dict(width=self.width >> level, height=self.height >> level,
                    fx=self.fx / s, fy=self.fy / s,
                    cx=(self.cx + 0.5) / s - 0.5, cy=(self.cy + 0.5) / s - 0.5)
