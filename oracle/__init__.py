"""FP64 CPU oracle of the dense RGB-D-inertial tracking hot path.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously
correct reference that the CUDA path is checked against.  Only the tests, the
smoke check of the build entry point and the CPU-baseline leg of the benchmark
may import it; the product path never does, and it shares no code, table or
helper with the CUDA library (it reads the same seeded synthetic inputs).

Contents, each following the paper (Laidlow et al., "Dense RGB-D-Inertial
SLAM with Map Deformations", IROS 2017):

* so3     -- state, Hamilton quaternions, boxplus / boxminus (Sec. IV-A, Eq. 1-2)
* maps    -- image pyramid, vertex / normal / gradient maps, reference maps
             (Sec. IV-D: three-level coarse-to-fine pyramid; Eq. 3-4 inputs)
* photogeo-- photometric (Eq. 3) and point-to-plane ICP (Eq. 4) residuals,
             Jacobians and their weighted normal equations, with the margin
             flags used for the bit-exact count comparison
* imu     -- inertial pre-integration and the IMU error term (Sec. IV-C, Eq. 5)
             with its weight (Table I noise densities)
* gn      -- joint cost (Eq. 6), Gauss-Newton system (Eq. 7), marginalisation
             (Eq. 8) and first-order prior correction (Eq. 9), and the per-frame
             tracker that chains them
* gravity3-- the paper's 3-D gravity-with-gauge form of the state (Sec. II,
             IV-A) with a damped step, beside the 2-DoF form the rest uses

Every floating-point step is FP64 (inputs are FP32 images, which convert
exactly).  Where the paper is silent (Jacobians, pyramid construction, data
association, thresholds, integration scheme) the reading chosen is stated in
the docstring of the function that implements it.

Parity status per function: pinned by the CPU tests (finite differences,
closed forms, invariants, brute force, textbook identities) except the
end-to-end accuracy against the paper's own experiments, which is parity
unpinned (the paper prints no intermediate values and its datasets are not
available).
"""
