"""The QL launch-shape autotuner: the first eager solve times the candidate lanes
per warp, keeps the fastest, and the results are bit for bit those of a context
with the tuner off (every lane's arithmetic is independent of the grouping)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import tbsystems as T  # noqa: E402
from gpu_helpers import gpu_context, to_dev  # noqa: E402
from paper_1809_05637_gb300 import DCLNO_MIXED  # noqa: E402


def _run(s, rho_in, tune, prec=0):
    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno)
    ctx.set_autotune(tune)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    r = ctx.step(to_dev(rho_in), out, s.n_electrons, s.kT, precision=prec)
    spec = ctx.spectrum()
    lanes, ms = ctx.tuning(0)
    ctx.close()
    return r, out.cpu().numpy(), np.concatenate([e for e, _ in spec]), lanes, ms


@pytest.mark.parametrize("prec", [0, DCLNO_MIXED])
def test_tuned_equals_untuned(cfg1, prec):
    s = cfg1
    rho_in = T.synthetic_density(s, seed=3)
    r1, rho1, eps1, lanes1, ms1 = _run(s, rho_in, True, prec)
    r0, rho0, eps0, lanes0, ms0 = _run(s, rho_in, False, prec)
    assert lanes0 == 0 and np.all(ms0 == -1)
    assert lanes1 in (4, 8, 12, 16, 24, 32)
    tried = ms1[ms1 >= 0]
    assert len(tried) >= 1 and ms1[[4, 8, 12, 16, 24, 32].index(lanes1)] == tried.min()
    assert r1 == r0
    np.testing.assert_array_equal(rho1, rho0)
    np.testing.assert_array_equal(eps1, eps0)
