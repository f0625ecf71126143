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


def _step_with(s, rho_in, prec, schedule, engine, tridiag, cache=None, steps=1, bucket_min=1):
    from gpu_helpers import gpu_context

    ctx = gpu_context(s, s.r_core, s.r_lno, s.k_lno, tridiag=tridiag)
    ctx.set_bucket_min(bucket_min)
    if cache is not None:
        ctx.set_tuning_cache(cache)
    ctx.set_schedule(schedule)
    ctx.set_mixed_engine(engine)
    out = torch.zeros(len(s.S), dtype=torch.float64, device="cuda:0")
    runs = []
    for _ in range(steps):
        r = ctx.step(to_dev(rho_in), out, s.n_electrons, s.kT, precision=prec)
        runs.append((r, out.cpu().numpy().copy(), np.concatenate([e for e, _ in ctx.spectrum()])))
    report = ctx.tuning_report()
    ctx.close()
    return runs, report


@pytest.mark.parametrize("prec,tridiag", [(0, 1), (0, 2), (DCLNO_MIXED, 1), (DCLNO_MIXED, 2)])
def test_schedules_and_engines_give_the_same_bits(cfg1, prec, tridiag):
    """Size buckets (every 64-wide bucket kept) launched with one CTA per cluster or as
    persistent grids on an atomic work counter, and (mixed path) either tensor-core engine for the K <= 32 products:
    the results are bit for bit the same (a cluster's arithmetic does not depend on the
    CTA that runs it; both engines combine the same exact integer level sums)."""
    s = cfg1
    rho_in = T.synthetic_density(s, seed=3)
    forms = [(1, 1), (2, 2), (2, 1), (1, 2)] if prec else [(1, 0), (2, 0)]
    ref = None
    for schedule, engine in forms:
        runs, report = _step_with(s, rho_in, prec, schedule, engine, tridiag)
        buckets = report["batches"][0]["buckets"]
        assert len(buckets) >= 2  # cluster dimensions span more than one bucket
        r, rho, eps = runs[0]
        if ref is None:
            ref = (r, rho, eps)
            continue
        assert r == ref[0]
        np.testing.assert_array_equal(rho, ref[1])
        np.testing.assert_array_equal(eps, ref[2])


def test_tuner_decides_and_caches(cfg1, tmp_path):
    """The tuner times one candidate schedule per bucket and kernel per eager solve
    (results unchanged), decides after four solves, writes the decisions to the cache,
    and a new context reading the cache starts with them."""
    s = cfg1
    rho_in = T.synthetic_density(s, seed=3)
    cache = str(tmp_path / "schedules.txt")
    runs, report = _step_with(s, rho_in, DCLNO_MIXED, 0, 0, 2, cache=cache, steps=5)
    for r, rho, eps in runs[1:]:
        assert r == runs[0][0]
        np.testing.assert_array_equal(rho, runs[0][1])
        np.testing.assert_array_equal(eps, runs[0][2])
    scheds = [v for b in report["batches"][0]["buckets"] for v in b["schedules"].values()]
    assert scheds and all(v["decided"] for v in scheds)
    assert any(len(v["ms"]) == 4 and min(v["ms"]) > 0 for v in scheds)
    lines = [ln for ln in open(cache).read().splitlines() if ln and not ln.startswith("#")]
    assert len(lines) >= 3
    runs2, report2 = _step_with(s, rho_in, DCLNO_MIXED, 0, 0, 2, cache=cache, steps=1)
    scheds2 = [v for b in report2["batches"][0]["buckets"] for v in b["schedules"].values()]
    assert any(v["from_cache"] for v in scheds2)
    assert runs2[0][0] == runs[0][0]
    np.testing.assert_array_equal(runs2[0][1], runs[0][1])


def test_small_buckets_merge(cfg1):
    """With the default minimum (twice the SM count) the 64 clusters form one bucket,
    and the results equal those of the unmerged buckets bit for bit."""
    s = cfg1
    rho_in = T.synthetic_density(s, seed=3)
    runs1, rep1 = _step_with(s, rho_in, 0, 1, 0, 1, bucket_min=1)
    runs0, rep0 = _step_with(s, rho_in, 0, 1, 0, 1, bucket_min=0)
    assert len(rep1["batches"][0]["buckets"]) >= 2
    b0 = rep0["batches"][0]["buckets"]
    assert len(b0) == 1 and b0[0]["clusters"] == s.natoms
    assert runs1[0][0] == runs0[0][0]
    np.testing.assert_array_equal(runs1[0][1], runs0[0][1])
