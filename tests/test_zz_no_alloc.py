"""dclno_find_mu_noalloc: the chemical-potential search for callers that cannot
allocate device memory (graph capture, caller-owned memory pools, loops that
must not allocate).  Its scratch is a static device array inside the library.

Checked against the ordinary entry point dclno_find_mu on the same spectrum,
twice in a row (the static scratch keeps the previous call's contents).  This
file is collected last so that a failure here leaves every other test run.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle as O  # noqa: E402
from gpu_helpers import gpu_context  # noqa: E402
from paper_1809_05637_gb300 import DclnoError, find_mu_noalloc  # noqa: E402


def _reference(system):
    ctx = gpu_context(system, system.r_core, system.r_core, 0)
    ctx.solve_clusters()
    mu, n = ctx.find_mu(system.n_electrons, system.kT)
    spec = ctx.spectrum()
    ctx.close()
    eps = np.concatenate([e for e, _ in spec])
    q = np.concatenate([w for _, w in spec])
    return mu, n, eps, q


def test_noalloc_mu_matches_find_mu(mixed_system):
    s = mixed_system
    mu_ref, n_ref, eps, q = _reference(s)
    d_eps = torch.from_numpy(eps).to("cuda:0")
    d_q = torch.from_numpy(q).to("cuda:0")
    for _ in range(2):
        mu, n = find_mu_noalloc(d_eps, d_q, s.n_electrons, s.kT)
        assert abs(n - s.n_electrons) <= 1e-10 * s.n_electrons
        assert abs(mu - mu_ref) <= 1e-9
        assert abs(n - n_ref) <= 1e-9 * s.n_electrons
        # N(mu) recomputed on the host from the same pairs
        assert abs(O.n_of_mu(eps, q, mu, s.kT) - s.n_electrons) <= 1e-9 * s.n_electrons


def test_noalloc_mu_rejects_oversized_input():
    d = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    from paper_1809_05637_gb300 import _lib as L
    lib = L.load_library()
    import ctypes
    mu = ctypes.c_double()
    st = lib.dclno_find_mu_noalloc(L._ptr(d), L._ptr(d), 8388608 + 1, 1.0, 0.01, L._dptr(mu), None, None)
    assert st == 1  # DCLNO_ERR_ARG, before any GPU work
    with pytest.raises(DclnoError):
        find_mu_noalloc(d[:0], d[:0], 1.0, 0.01)  # empty input


def _synthetic_pairs(count, seed):
    """Seeded (eps, q) pairs shaped like a DC spectrum: eigenvalues spread over a
    few hartree with a dense occupied window, positive Mulliken-like weights."""
    rng = np.random.default_rng(seed)
    eps = np.concatenate([rng.uniform(-1.0, 0.5, count - count // 4), rng.uniform(0.5, 40.0, count // 4)])
    q = rng.uniform(0.0, 0.05, count)
    return eps, q


@pytest.mark.parametrize("count", [100_003, 8_388_608])
def test_noalloc_mu_many_blocks_against_oracle(count):
    """Many partial-sum blocks (100,003 pairs: 49 blocks with a ragged last one) and
    exactly the largest count the static scratch covers (4096 blocks).  mu is
    checked against the oracle's bisection and N(mu) against the oracle's sum."""
    eps, q = _synthetic_pairs(count, seed=count)
    kT = 0.01
    n_e = 0.6 * 2.0 * float(q.sum())
    d_eps = torch.from_numpy(eps).to("cuda:0")
    d_q = torch.from_numpy(q).to("cuda:0")
    mu_or, _ = O.find_mu(eps, q, n_e, kT)
    # slope of N at mu: turns the 1e-12 N_e stopping rule of both searches into a mu tolerance
    h = 1e-6
    slope = (O.n_of_mu(eps, q, mu_or + h, kT) - O.n_of_mu(eps, q, mu_or - h, kT)) / (2 * h)
    mu_tol = 1e-12 + 4e-12 * n_e / slope
    for _ in range(2):
        mu, n = find_mu_noalloc(d_eps, d_q, n_e, kT)
        assert abs(mu - mu_or) <= mu_tol, (mu, mu_or, mu_tol)
        n_host = O.n_of_mu(eps, q, mu, kT)
        assert abs(n_host - n_e) <= 1e-9 * n_e
        assert abs(n - n_host) <= 1e-9 * n_e


def test_noalloc_binding_rejects_unsafe_arrays():
    """The binding refuses arrays the C entry point would read past or misread."""
    d = torch.zeros(16, dtype=torch.float64, device="cuda:0")
    with pytest.raises(ValueError):
        find_mu_noalloc(d, d[:8], 1.0, 0.01)  # q shorter than eps
    with pytest.raises(ValueError):
        find_mu_noalloc(d.float(), d.float(), 1.0, 0.01)  # float32
    with pytest.raises(ValueError):
        find_mu_noalloc(d[::2], d[::2], 1.0, 0.01)  # not contiguous
    with pytest.raises(ValueError):
        find_mu_noalloc(d.cpu(), d.cpu(), 1.0, 0.01)  # host memory
