"""Seeded synthetic RGB-D + IMU inputs (test and benchmark data only).

This module renders the inputs both the FP64 oracle and the CUDA path consume:
depth and intensity images of an analytic scene, ground-truth trajectories and
the IMU samples measured along them.  It holds none of the tracking method's
arithmetic (no pyramid, no residual, no pre-integration, no solve): only a
scene description, a ray caster and the closed-form kinematics of two
trajectory families.

Stand-in for the paper's data (Sec. VI-A: ICL-NUIM living room re-rendered
with POV-Ray, IMU simulated along spline-fitted trajectories with the Table I
noise parameters; Sec. VI-B: ZR300 recordings).  Neither dataset is available,
so scenes are an analytic box room (4 x 3 x 2.5 m) with five textured spheres,
the texture a 3-D value noise that is view independent (brightness constancy
holds exactly before noise is added).

Frames: I is gravity aligned (z up, g_I = (0, 0, -9.81)); W is the first
camera frame and shares I's origin (Sec. II).  Poses T_AB = (R_AB, r_AB) map B
coordinates into A.  Quaternions are Hamilton, stored (w, x, y, z).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

GRAVITY = 9.81  # Table I

# Table I, synthetic-dataset column (Sec. VI): noise densities used to draw IMU noise.
GYR_NOISE_DENSITY = 12.0e-4   # rad s^-1 Hz^-0.5
ACC_NOISE_DENSITY = 8.0e-3    # m s^-2 Hz^-0.5


# ----------------------------------------------------------------------------
# Generator-local rotation helpers (independent of the oracle's and the CUDA code)
# ----------------------------------------------------------------------------

def _hat(w):
    return np.array([[0.0, -w[2], w[1]], [w[2], 0.0, -w[0]], [-w[1], w[0], 0.0]])


def _rotvec_to_matrix(w):
    w = np.asarray(w, dtype=np.float64)
    th = float(np.linalg.norm(w))
    if th < 1e-12:
        return np.eye(3) + _hat(w)
    k = _hat(w / th)
    return np.eye(3) + np.sin(th) * k + (1.0 - np.cos(th)) * (k @ k)


def _rx(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1, 0, 0], [0, c, -s], [0, s, c]], dtype=np.float64)


def _ry(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]], dtype=np.float64)


def _rz(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]], dtype=np.float64)


def matrix_to_quat(R):
    """Rotation matrix -> unit quaternion (w, x, y, z), w >= 0."""
    R = np.asarray(R, dtype=np.float64)
    tr = R[0, 0] + R[1, 1] + R[2, 2]
    if tr > 0:
        s = np.sqrt(tr + 1.0) * 2
        q = [0.25 * s, (R[2, 1] - R[1, 2]) / s, (R[0, 2] - R[2, 0]) / s, (R[1, 0] - R[0, 1]) / s]
    elif R[0, 0] > R[1, 1] and R[0, 0] > R[2, 2]:
        s = np.sqrt(1.0 + R[0, 0] - R[1, 1] - R[2, 2]) * 2
        q = [(R[2, 1] - R[1, 2]) / s, 0.25 * s, (R[0, 1] + R[1, 0]) / s, (R[0, 2] + R[2, 0]) / s]
    elif R[1, 1] > R[2, 2]:
        s = np.sqrt(1.0 + R[1, 1] - R[0, 0] - R[2, 2]) * 2
        q = [(R[0, 2] - R[2, 0]) / s, (R[0, 1] + R[1, 0]) / s, 0.25 * s, (R[1, 2] + R[2, 1]) / s]
    else:
        s = np.sqrt(1.0 + R[2, 2] - R[0, 0] - R[1, 1]) * 2
        q = [(R[1, 0] - R[0, 1]) / s, (R[0, 2] + R[2, 0]) / s, (R[1, 2] + R[2, 1]) / s, 0.25 * s]
    q = np.array(q)
    q /= np.linalg.norm(q)
    if q[0] < 0:
        q = -q
    return q


def quat_to_matrix(q):
    w, x, y, z = np.asarray(q, dtype=np.float64) / np.linalg.norm(q)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
        [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
        [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)],
    ])


# ----------------------------------------------------------------------------
# Cameras
# ----------------------------------------------------------------------------

@dataclass(frozen=True)
class Camera:
    width: int
    height: int
    fx: float
    fy: float
    cx: float
    cy: float


CAM_320 = Camera(320, 240, 277.0, 277.0, 160.0, 120.0)
CAM_640 = Camera(640, 480, 554.0, 554.0, 320.0, 240.0)
CAM_1280 = Camera(1280, 720, 1108.0, 1108.0, 640.0, 360.0)


def scaled_camera(width, height):
    """Camera with the 320x240 focal scale (277 px per 320 px of width)."""
    f = 277.0 * width / 320.0
    return Camera(width, height, f, f, width / 2.0, height / 2.0)


# ----------------------------------------------------------------------------
# Scene: box room + spheres with 3-D value-noise albedo
# ----------------------------------------------------------------------------

@dataclass
class Scene:
    lo: np.ndarray          # room minimum corner (I frame), shape (3,)
    hi: np.ndarray          # room maximum corner
    centers: np.ndarray     # sphere centres, (S, 3)
    radii: np.ndarray       # sphere radii, (S,)
    perm: np.ndarray        # value-noise permutation table, int64 (512,)
    lattice: np.ndarray     # value-noise lattice values in [0, 1], (256,)
    seed: int = 0


def make_scene(seed, center=(0.0, 0.0, 0.0), size=(4.0, 3.0, 2.5), n_spheres=5,
               keep_clear=None, clearance=0.3):
    """Seeded box room of the given size centred at `center`.

    Spheres have radius U[0.2, 0.5] m, stay >= `clearance` from every wall and
    from every point in `keep_clear` (camera path samples, (N, 3))."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5CE4E]))
    c = np.asarray(center, dtype=np.float64)
    half = 0.5 * np.asarray(size, dtype=np.float64)
    lo, hi = c - half, c + half
    pts = np.zeros((1, 3)) + c if keep_clear is None else np.asarray(keep_clear, dtype=np.float64)
    centers, radii = [], []
    tries = 0
    while len(centers) < n_spheres and tries < 100000:
        tries += 1
        r = rng.uniform(0.2, 0.5)
        p = rng.uniform(lo + r + clearance, hi - r - clearance)
        if np.min(np.linalg.norm(pts - p, axis=1)) < r + clearance:
            continue
        if any(np.linalg.norm(p - q) < r + s + 0.05 for q, s in zip(centers, radii)):
            continue
        centers.append(p)
        radii.append(r)
    perm = rng.permutation(256).astype(np.int64)
    return Scene(lo=lo, hi=hi, centers=np.array(centers).reshape(-1, 3),
                 radii=np.array(radii), perm=np.concatenate([perm, perm]),
                 lattice=rng.uniform(0.0, 1.0, 256), seed=int(seed))


def albedo(scene, pts):
    """3-D value noise of world points: 4 octaves, base 4 cycles/m, persistence 0.5,
    smoothstep-trilinear between lattice values, mapped to [0.1, 0.9]."""
    pts = np.asarray(pts, dtype=np.float64)
    perm, lat = scene.perm, scene.lattice
    total = np.zeros(pts.shape[:-1])
    amp, norm = 1.0, 0.0
    for octave in range(4):
        p = pts * (4.0 * (2 ** octave)) + 17.0 * octave
        i0 = np.floor(p)
        f = p - i0
        i0 = i0.astype(np.int64)
        s = f * f * (3.0 - 2.0 * f)
        acc = np.zeros(pts.shape[:-1])
        for dz in (0, 1):
            wz = s[..., 2] if dz else 1.0 - s[..., 2]
            for dy in (0, 1):
                wy = s[..., 1] if dy else 1.0 - s[..., 1]
                for dx in (0, 1):
                    wx = s[..., 0] if dx else 1.0 - s[..., 0]
                    h = perm[(perm[(perm[(i0[..., 0] + dx) & 255] + i0[..., 1] + dy) & 255]
                              + i0[..., 2] + dz) & 255]
                    acc += wx * wy * wz * lat[h]
        total += amp * acc
        norm += amp
        amp *= 0.5
    return 0.1 + 0.8 * total / norm


def render(scene, R_IC, r_IC, cam, rng=None, sigma_d=0.002, sigma_I=0.01, dropout=0.0,
           spheres=True):
    """Ray-cast z-depth (m) and intensity in [0, 1] of the scene seen from camera
    pose T_IC.  Returns float32 (H, W) arrays; dropped-out depth is 0."""
    R_IC = np.asarray(R_IC, dtype=np.float64)
    o = np.asarray(r_IC, dtype=np.float64)
    u = np.arange(cam.width, dtype=np.float64)
    v = np.arange(cam.height, dtype=np.float64)
    uu, vv = np.meshgrid(u, v)
    d_c = np.stack([(uu - cam.cx) / cam.fx, (vv - cam.cy) / cam.fy, np.ones_like(uu)], axis=-1)
    d = d_c @ R_IC.T                       # ray directions in I, camera z component = 1
    with np.errstate(divide="ignore", invalid="ignore"):
        t_hi = (scene.hi - o) / d
        t_lo = (scene.lo - o) / d
    t_wall = np.where(d > 0, t_hi, np.where(d < 0, t_lo, np.inf))
    t = np.min(t_wall, axis=-1)
    if spheres:
        a = np.sum(d * d, axis=-1)
        for c, r in zip(scene.centers, scene.radii):
            oc = o - c
            b = d @ oc
            cc = float(oc @ oc - r * r)
            disc = b * b - a * cc
            hit = disc >= 0
            ts = np.where(hit, (-b - np.sqrt(np.where(hit, disc, 0.0))) / a, np.inf)
            ts = np.where(ts > 1e-9, ts, np.inf)
            t = np.minimum(t, ts)
    pts = o + d * t[..., None]
    inten = albedo(scene, pts)
    depth = t.copy()                       # camera-frame z of the hit point (ray z = 1)
    if rng is not None:
        if sigma_d > 0:
            depth = depth + rng.normal(0.0, sigma_d, depth.shape)
        if sigma_I > 0:
            inten = inten + rng.normal(0.0, sigma_I, inten.shape)
        if dropout > 0:
            depth = np.where(rng.uniform(size=depth.shape) < dropout, 0.0, depth)
    inten = np.clip(inten, 0.0, 1.0)
    return depth.astype(np.float32), inten.astype(np.float32)


# ----------------------------------------------------------------------------
# Camera-IMU rig
# ----------------------------------------------------------------------------

# Camera C looks along the IMU's x axis: C's x = -S's y, C's y = -S's z, C's z = S's x.
_R_SC_NOMINAL = np.array([[0.0, 0.0, 1.0], [-1.0, 0.0, 0.0], [0.0, -1.0, 0.0]])


def default_extrinsics():
    """T_CS (IMU frame S expressed in camera frame C): a nominal rig with a small
    mounting rotation and lever arm, so the extrinsic is never the identity."""
    R_SC = _R_SC_NOMINAL @ _rotvec_to_matrix([0.01, -0.02, 0.015])
    R_CS = R_SC.T
    r_CS = np.array([0.03, -0.01, 0.02])   # position of S's origin in C
    return R_CS, r_CS


# ----------------------------------------------------------------------------
# Trajectories (closed-form kinematics of the IMU frame S in I)
# ----------------------------------------------------------------------------

@dataclass
class ConstantRateTrajectory:
    """R_IS(t) = R_IS0 Exp(omega_S t), r_IS(t) = r_IS0 + v_I t.

    With zero world acceleration and constant body rate, a zero-order hold of
    the sampled gyro and specific-force readings is exact."""
    R_IS0: np.ndarray
    r_IS0: np.ndarray
    omega_S: np.ndarray
    v_I: np.ndarray

    def pose_IS(self, t):
        return self.R_IS0 @ _rotvec_to_matrix(self.omega_S * t), self.r_IS0 + self.v_I * t

    def velocity_I(self, t):
        return self.v_I.copy()

    def omega_S_at(self, t):
        return self.omega_S.copy()

    def accel_I(self, t):
        return np.zeros(3)


@dataclass
class SinusoidTrajectory:
    """r_IS(t) = c + A sin(w t + phi) per axis; R_IS = Rz(psi) Ry(theta) Rx(phi_r)
    with each angle a0 + amplitude * sin(w t + phase)."""
    c: np.ndarray
    A: np.ndarray
    phase: np.ndarray
    w: float
    ang0: np.ndarray        # (yaw, pitch, roll) offsets
    ang_amp: np.ndarray     # amplitudes
    ang_phase: np.ndarray

    def _angles(self, t):
        a = self.ang0 + self.ang_amp * np.sin(self.w * t + self.ang_phase)
        ad = self.ang_amp * self.w * np.cos(self.w * t + self.ang_phase)
        return a, ad

    def pose_IS(self, t):
        (psi, th, ph), _ = self._angles(t)
        R = _rz(psi) @ _ry(th) @ _rx(ph)
        return R, self.c + self.A * np.sin(self.w * t + self.phase)

    def velocity_I(self, t):
        return self.A * self.w * np.cos(self.w * t + self.phase)

    def accel_I(self, t):
        return -self.A * self.w * self.w * np.sin(self.w * t + self.phase)

    def omega_S_at(self, t):
        (psi, th, ph), (dpsi, dth, dph) = self._angles(t)
        return np.array([
            dph - dpsi * np.sin(th),
            dth * np.cos(ph) + dpsi * np.sin(ph) * np.cos(th),
            -dth * np.sin(ph) + dpsi * np.cos(ph) * np.cos(th),
        ])


@dataclass
class Sequence:
    """Everything one synthetic camera stream provides."""
    cam: Camera
    scene: Scene
    R_CS: np.ndarray
    r_CS: np.ndarray
    R_IW: np.ndarray                # gravity alignment of W (= first camera frame)
    frame_times: np.ndarray         # (F,)
    depth: list                     # F float32 (H, W)
    intensity: list
    gt: list                        # F dicts: r_WC, q_WC, R_WC, v_I, bg, ba, q_IW
    imu: np.ndarray                 # (N, 7): t, gyr(3), acc(3)
    bg: np.ndarray
    ba: np.ndarray
    meta: dict = field(default_factory=dict)
    traj: object = None


def _camera_pose_I(traj, t, R_CS, r_CS):
    R_IS, r_IS = traj.pose_IS(t)
    R_IC = R_IS @ R_CS.T
    r_IC = r_IS - R_IC @ r_CS
    return R_IC, r_IC


def imu_samples(traj, rate, t_start, t_end, bg, ba, rng=None,
                gyr_nd=GYR_NOISE_DENSITY, acc_nd=ACC_NOISE_DENSITY):
    """Samples at t_k = k / rate covering [t_start, t_end]: gyro = omega_S + bg + n_g,
    accelerometer = R_IS^T (a_I - g_I) + ba + n_a, n ~ N(0, density^2 * rate)."""
    k0 = int(np.floor(t_start * rate)) - 1
    k1 = int(np.ceil(t_end * rate)) + 1
    g_I = np.array([0.0, 0.0, -GRAVITY])
    rows = []
    for k in range(k0, k1 + 1):
        t = k / rate
        R_IS, _ = traj.pose_IS(t)
        gyr = traj.omega_S_at(t) + bg
        acc = R_IS.T @ (traj.accel_I(t) - g_I) + ba
        if rng is not None:
            gyr = gyr + rng.normal(0.0, gyr_nd * np.sqrt(rate), 3)
            acc = acc + rng.normal(0.0, acc_nd * np.sqrt(rate), 3)
        rows.append(np.concatenate([[t], gyr, acc]))
    return np.array(rows)


def _state_from(traj, t, R_CS, r_CS, R_IW, bg, ba):
    R_IC, r_IC = _camera_pose_I(traj, t, R_CS, r_CS)
    R_WC = R_IW.T @ R_IC
    r_WC = R_IW.T @ r_IC            # I and W share their origin
    return dict(t=float(t), r_WC=r_WC, R_WC=R_WC, q_WC=matrix_to_quat(R_WC),
                v_I=traj.velocity_I(t), bg=np.array(bg, dtype=np.float64),
                ba=np.array(ba, dtype=np.float64), q_IW=matrix_to_quat(R_IW), R_IW=R_IW.copy())


def _make_sequence(traj, cam, scene, R_CS, r_CS, frame_times, rate, bg, ba, rng,
                   sigma_d, sigma_I, dropout, imu_noise, render_frames=True):
    R_IC0, r_IC0 = _camera_pose_I(traj, frame_times[0], R_CS, r_CS)
    R_IW = R_IC0                                   # W = first camera frame
    depth, inten, gt = [], [], []
    for t in frame_times:
        st = _state_from(traj, t, R_CS, r_CS, R_IW, bg, ba)
        gt.append(st)
        if render_frames:
            R_IC, r_IC = _camera_pose_I(traj, t, R_CS, r_CS)
            d, i = render(scene, R_IC, r_IC, cam, rng, sigma_d, sigma_I, dropout)
            depth.append(d)
            inten.append(i)
    imu = imu_samples(traj, rate, frame_times[0], frame_times[-1], bg, ba,
                      rng if imu_noise else None)
    return Sequence(cam=cam, scene=scene, R_CS=R_CS, r_CS=r_CS, R_IW=R_IW,
                    frame_times=np.asarray(frame_times, dtype=np.float64), depth=depth,
                    intensity=inten, gt=gt, imu=imu, bg=np.asarray(bg), ba=np.asarray(ba),
                    traj=traj)


def _random_unit(rng):
    v = rng.normal(size=3)
    return v / np.linalg.norm(v)


def frame_pair(seed=1, cam=CAM_320, rot_deg=2.0, trans_m=0.03, dt=1.0 / 30.0, rate=200.0,
               bias=True, sigma_d=0.002, sigma_I=0.01, dropout=0.0, imu_noise=True,
               spheres=True, t0=0.0):
    """One frame pair: a seeded 2 deg rotation and 3 cm translation over `dt` from
    constant body rate and constant velocity, IMU biases of 1e-3 rad/s and
    0.05 m/s^2 per axis (seeded signs), Table I white noise."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xF4A1]))
    R_CS, r_CS = default_extrinsics()
    # level camera looking along +x of I, with a small seeded tilt and yaw
    R_IS0 = _rz(rng.uniform(-0.3, 0.3)) @ _ry(rng.uniform(-0.1, 0.1)) @ _rx(rng.uniform(-0.1, 0.1))
    omega = _random_unit(rng) * np.deg2rad(rot_deg) / dt
    vel = _random_unit(rng) * trans_m / dt
    R_IC0 = R_IS0 @ R_CS.T
    r_IS0 = R_IC0 @ r_CS                               # camera starts at I's origin
    traj = ConstantRateTrajectory(R_IS0=R_IS0, r_IS0=r_IS0, omega_S=omega, v_I=vel)
    bg = (np.where(rng.uniform(size=3) < 0.5, -1.0, 1.0) * 1e-3) if bias else np.zeros(3)
    ba = (np.where(rng.uniform(size=3) < 0.5, -1.0, 1.0) * 0.05) if bias else np.zeros(3)
    path = np.array([_camera_pose_I(traj, s, R_CS, r_CS)[1] for s in np.linspace(t0, t0 + dt, 5)])
    scene = make_scene(seed, center=(0.0, 0.0, 0.0), keep_clear=path,
                       n_spheres=5 if spheres else 0)
    times = np.array([t0, t0 + dt])
    seq = _make_sequence(traj, cam, scene, R_CS, r_CS, times, rate, bg, ba, rng,
                         sigma_d, sigma_I, dropout, imu_noise)
    seq.meta = dict(kind="pair", seed=seed, rate=rate, dt=dt)
    return seq


def sinusoid_sequence(seed=2, cam=CAM_640, n_frames=300, fps=30.0, rate=400.0,
                      peak_speed=1.5, peak_yaw_rate_deg=90.0, period_frames=100, bias=True,
                      sigma_d=0.002, sigma_I=0.01, dropout=0.0, imu_noise=True,
                      render_frames=True):
    """A sequence along a sinusoidal path (peak 1.5 m/s, peak yaw rate 90 deg/s, period
    100 frames so it loops seamlessly), IMU at 400 Hz from the analytic derivatives."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x51D0]))
    R_CS, r_CS = default_extrinsics()
    w = 2.0 * np.pi * fps / period_frames
    A = np.array([peak_speed / w, 0.5 * peak_speed / w, 0.2 * peak_speed / w])
    phase = rng.uniform(0, 2 * np.pi, 3)
    yaw_amp = np.deg2rad(peak_yaw_rate_deg) / w
    ang0 = np.array([rng.uniform(-np.pi, np.pi), 0.0, 0.0])
    ang_amp = np.array([yaw_amp, 0.08, 0.06])
    ang_phase = rng.uniform(0, 2 * np.pi, 3)
    traj0 = SinusoidTrajectory(c=np.zeros(3), A=A, phase=phase, w=w, ang0=ang0,
                               ang_amp=ang_amp, ang_phase=ang_phase)
    # shift so the first camera position is I's origin
    R_IC0, r_IC0 = _camera_pose_I(traj0, 0.0, R_CS, r_CS)
    traj = SinusoidTrajectory(c=-r_IC0, A=A, phase=phase, w=w, ang0=ang0, ang_amp=ang_amp,
                              ang_phase=ang_phase)
    ts = np.linspace(0.0, period_frames / fps, 200)
    path = np.array([_camera_pose_I(traj, s, R_CS, r_CS)[1] for s in ts])
    center = 0.5 * (path.min(axis=0) + path.max(axis=0))
    scene = make_scene(seed, center=center, keep_clear=path)
    bg = (np.where(rng.uniform(size=3) < 0.5, -1.0, 1.0) * 1e-3) if bias else np.zeros(3)
    ba = (np.where(rng.uniform(size=3) < 0.5, -1.0, 1.0) * 0.05) if bias else np.zeros(3)
    times = np.arange(n_frames) / fps
    seq = _make_sequence(traj, cam, scene, R_CS, r_CS, times, rate, bg, ba, rng,
                         sigma_d, sigma_I, dropout, imu_noise, render_frames)
    seq.meta = dict(kind="sinusoid", seed=seed, rate=rate, fps=fps)
    return seq


def initial_state(seq, rng=None, v_sigma=0.0, grav_sigma=0.0):
    """Initial state for the first frame: identity pose (W = first camera frame),
    GT velocity (+ optional noise), zero biases, GT gravity alignment (+ optional
    seeded tilt).  Returned as a plain dict of float64 arrays."""
    g0 = seq.gt[0]
    v = g0["v_I"].copy()
    R_IW = g0["R_IW"].copy()
    if rng is not None:
        if v_sigma > 0:
            v = v + rng.normal(0.0, v_sigma, 3)
        if grav_sigma > 0:
            ax = rng.normal(size=2)
            R_IW = _rotvec_to_matrix(np.array([ax[0], ax[1], 0.0]) * grav_sigma) @ R_IW
    return dict(t=float(seq.frame_times[0]), r_WC=np.zeros(3), q_WC=np.array([1.0, 0, 0, 0]),
                v_I=v, bg=np.zeros(3), ba=np.zeros(3), q_IW=matrix_to_quat(R_IW))


def render_frame(seq, i, seed=0, sigma_d=0.002, sigma_I=0.01, dropout=0.0):
    """Renders frame i of a sequence made with render_frames=False, with its own
    noise stream (seeded by (seed, i)), so frames can be rendered in parallel."""
    g = seq.gt[i]
    R_IC = seq.R_IW @ g["R_WC"]
    r_IC = seq.R_IW @ g["r_WC"]
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), int(i), 0xF7A3]))
    return render(seq.scene, R_IC, r_IC, seq.cam, rng, sigma_d, sigma_I, dropout)


def sequence_imu(seq, t_end, seed=0):
    """IMU samples of the sequence's trajectory from its first frame to t_end
    (periodic trajectories can be extended beyond the rendered frames)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x1A0]))
    return imu_samples(seq.traj, seq.meta["rate"], seq.frame_times[0], t_end, seq.bg, seq.ba, rng)
