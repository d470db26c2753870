import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")


def oracle_config(seq, levels=2, iters=(10, 5), **kw):
    from oracle.params import TrackerConfig
    cam = seq.cam
    return TrackerConfig(cam.width, cam.height, cam.fx, cam.fy, cam.cx, cam.cy, levels=levels,
                         iters=tuple(iters), R_CS=seq.R_CS, r_CS=seq.r_CS, **kw)


@pytest.fixture(scope="session")
def small_cam():
    from paper_2207_10940_gb300.synth import scaled_camera
    return scaled_camera(96, 72)


@pytest.fixture(scope="session")
def pair_small(small_cam):
    from paper_2207_10940_gb300 import synth
    return synth.frame_pair(seed=7, cam=small_cam)


@pytest.fixture(scope="session")
def pair_c1():
    """320x240 frame pair of the 1-pair workload (seed 1)."""
    from paper_2207_10940_gb300 import synth
    return synth.frame_pair(seed=1)


@pytest.fixture
def rng():
    return np.random.default_rng(1234)
