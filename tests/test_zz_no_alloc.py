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
