import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: long-running CPU test")


@pytest.fixture(scope="session")
def cfg1():
    import tbsystems
    return tbsystems.make_system(1)


@pytest.fixture(scope="session")
def cfg1_exact(cfg1):
    import oracle
    return oracle.full_diag(cfg1)


@pytest.fixture(scope="session")
def cfg1_dc0(cfg1):
    """Plain DC density with core-only clusters: the start of an LNO step."""
    import oracle
    return oracle.plain_dc_density(cfg1, cfg1.r_core)


@pytest.fixture(scope="session")
def mixed_system():
    """Small open system with two species of different basis sizes (3 and 4)."""
    import tbsystems
    from tbsystems import _sc_lattice, assemble_system
    pos, ijk = _sc_lattice(3, 3, 2, 2.6)
    pos = pos + np.random.default_rng(5).normal(0, 0.05, pos.shape)
    sp = (ijk.sum(1) % 2).astype(np.int32)
    exps = [np.array([0.25, 0.7, 2.0]) if s == 0 else np.array([0.18, 0.45, 1.1, 2.8]) for s in sp]
    ons = [np.array([-0.45, -0.2, 0.3]) if s == 0 else np.array([-0.55, -0.35, 0.05, 0.5]) for s in sp]
    ne = float(sum(2.0 if s == 0 else 3.0 for s in sp))
    return assemble_system("mixed18", pos, np.eye(3) * 20.0, np.zeros(3, bool), sp, exps, ons,
                           ne, 0.02, 3.0, 6.0, 2)
