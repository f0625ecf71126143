#!/usr/bin/env python3
"""DC-LNO clusters per second on one GB300: FP64 path (value) and mixed path ("mixed").

A step is one pass of the whole hot path on the 1,728-atom gapped rock-salt
workload (12x12x12 simple-cubic sites, a = 3.0 bohr, two species, 9 s-Gaussians
per atom, r_core = 6, r_lno = 10 bohr, 3 LNOs per atom): Lambda blocks and LNOs
of every atom, assembly and generalised eigensolve of all 1,728 clusters,
common chemical potential, density-matrix rows of every central atom.  The
input density is the seeded synthetic density of ``tbsystems`` (the same for
the reference arm).  Inputs (S, H, rho: 5.2 GB) are larger than L2, so no L2
flush is inserted between steps.

N > 1 (torchrun): replicas.  Every rank runs the whole workload on its own GPU
(one GPU holds the problem; no data-path collective), value = clusters of all
ranks / max-over-ranks time ("scaling": "weak").

--impl reference times the FP64 oracle (the plain CPU statement of the method)
on the host cores on a bounded sample of the same workload (rank 0 only).
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "DC-LNO clusters/s at 1 GB300; mixed vs FP64 at ≤1e-6 Ha/atom, % of roofline"
WORKLOAD = ("DC-LNO step, 1728-atom gapped rock-salt (12^3 SC sites, a=3.0 bohr, jitter 0.05, "
            "9 s-Gaussians/atom, r_core=6, r_lno=10 bohr, 3 LNOs/atom, kT=0.01 Ha), FP64")
# kernels whose time is reported per step (CUDA events around each launch on the context's stream)
KERNELS = ["k_lambda", "k_lno_eig", "k_lno_blocks", "k_assemble", "k_cholesky", "k_congruence", "k_tridiag",
           "k_band", "k_chase", "k_ql", "k_merge", "k_apply_q_rows", "k_replay_fwd", "k_mgemm_fwd", "k_weights",
           "k_mu_partial", "k_mu_update", "k_rho_prep", "k_mgemm_rev", "k_replay_rev", "k_rho_qx", "k_rho_scatter"]
ROOFLINE_KERNELS = ("k_tridiag", "k_band", "k_chase")  # kernels with a roofline model (roofline_report)
# oracle sample: one cluster per host core (at least 8, at most 32), evenly spaced atoms
CPU_SAMPLE_CLUSTERS = max(8, min(32, os.cpu_count() or 1))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-scf", action="store_true", help="skip the SCF-loop measurement on the bcc slab")
    p.add_argument("--no-amorphous", action="store_true",
                   help="skip the one-step measurement of the 32,000-atom amorphous workload (run on one GPU only)")
    p.add_argument("--no-refine", action="store_true",
                   help="skip the measurement of the refinement sweeps (dclno_refine_eigenpairs)")
    p.add_argument("--workload", choices=["rocksalt1728", "rocksalt512", "rocksalt216", "small64", "amorphous32000"],
                   default="rocksalt1728",
                   help="rocksalt512: the same rock-salt recipe on 8^3 sites (the same cluster dimensions, one "
                        "wave of clusters in flight); rocksalt216: on 6^3 sites (the same cluster dimensions, "
                        "under 5 GB on the device: the case for DRAM-traffic captures of the cubic kernels); "
                        "small64: a 64-cluster periodic lattice (n ~ 525) for ncu captures of single kernels; "
                        "amorphous32000: the 32,000-atom random packing, generated row range by row range "
                        "into device memory and solved through memory-admitted batches")
    p.add_argument("--atoms", type=int, default=32000, help="atoms of the amorphous workload (same density)")
    p.add_argument("--tridiag", type=int, choices=[0, 1, 2], default=0,
                   help="tridiagonalisation form of both paths: 0 the library's automatic choice, 1 one-stage, "
                        "2 two-stage (dense -> band -> tridiagonal)")
    p.add_argument("--mixed-engine", type=int, choices=[0, 1, 2], default=0,
                   help="tensor-core engine of the mixed path's Cholesky, congruence and one-stage "
                        "tridiagonalisation: 0 tuned per size bucket, 1 mma.sync, 2 tcgen05 with tensor memory "
                        "(the band reduction's long-K products always run on tcgen05)")
    return p.parse_args()


def make_workload(name):
    import tbsystems as T
    if name == "small64":
        return T.small_lattice(4, 4, 4, a=2.5, jitter=0.05, exps=(0.1, 0.2, 0.45, 1.0, 2.2, 5.0),
                               onsite=(-0.6, -0.4, -0.2, 0.0, 0.2, 0.4), e_per_atom=3.0, r_core=5.0, r_lno=8.0,
                               k_lno=3, periodic=True, name="small64")
    if name == "rocksalt512":
        return T.make_system(2, n_cells=8)
    if name == "rocksalt216":
        return T.make_system(2, n_cells=6)
    return T.make_system(2)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows),
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()), default=None)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and reference arm)
# ---------------------------------------------------------------------------
def oracle_sample(s, rho_in, mu_fixed, threads, detail=False):
    """Per-cluster DC-LNO work of the oracle on a sample of clusters: LNOs of the
    LNO-region atoms, assembly, FP64 generalised eigensolve, weights and the
    central density-matrix rows at a fixed chemical potential.  Returns the
    number of clusters and the wall time (and, with detail, the LNOs, the
    per-cluster results and the rows, for comparisons made after the timing)."""
    import numpy as np

    import oracle as O

    n = s.natoms
    sample = sorted({int(x) for x in np.linspace(0, n - 1, CPU_SAMPLE_CLUSTERS)})
    t0 = time.perf_counter()
    need = set()
    for i in sample:
        cl = O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno)
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, rho_in, s.k_lno, atoms=sorted(need))
    V = {j: v[0] for j, v in lno.items()}
    res = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=sample, threads=threads)
    rows = np.zeros_like(s.S)
    for r in res.values():
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu_fixed, s.kT, rows)
    wall = time.perf_counter() - t0
    if detail:
        return len(sample), wall, V, res, rows
    return len(sample), wall


def cpu_threads():
    return max(1, min(CPU_SAMPLE_CLUSTERS, os.cpu_count() or 1))


def sample_text(natoms=1728):
    return (f"{CPU_SAMPLE_CLUSTERS} of the {natoms} clusters (evenly spaced atoms): LNOs of their LNO-region "
            "atoms, assembly, FP64 Cholesky+Jacobi eigensolve, weights and central density rows at a fixed mu; "
            "the global mu search needs every cluster and is not in the sample")


def oracle_errors(s, res, orows, spec, rows_gpu):
    """A GPU solve against the oracle on the sampled clusters: the largest
    eigenvalue difference (Ha), the same over each state's first-order bound (a
    backward error n u in H^(i), S^(i), c^T S c = 1), and the largest density-row
    difference relative to the row's largest element."""
    import numpy as np

    deps = dbound = drho = 0.0
    for i, r in res.items():
        d = np.abs(np.sort(spec[i][0]) - r.eps)
        bound = 1e-10 + 2.0 * len(r.eps) * 2.0 ** -53 * (r.h_norm + np.abs(r.eps) * r.s_norm) * np.einsum(
            "am,am->m", r.C, r.C)
        deps = max(deps, float(np.max(d)))
        dbound = max(dbound, float(np.max(d / bound)))
        b0, b1 = int(s.row_ptr[i]), int(s.row_ptr[i + 1])
        o0 = int(s.blk_off[b0])
        o1 = int(s.blk_off[b1 - 1] + s.norb[i] * s.norb[s.col[b1 - 1]])
        big = float(np.max(np.abs(orows[o0:o1])))
        drho = max(drho, float(np.max(np.abs(rows_gpu[o0:o1] - orows[o0:o1]))) / big)
    return {"clusters": sorted(res), "max_abs_eps_diff_ha": deps, "max_eps_diff_over_first_order_bound": dbound,
            "max_rho_row_diff_rel_to_row_max": drho}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import tbsystems as T

    s = T.make_system(2)
    rho_in = T.synthetic_density(s, seed=11)
    th = cpu_threads()
    for _ in range(args.warmup):
        oracle_sample(s, rho_in, -0.27, th)
    times = []
    ncl = 0
    for _ in range(args.steps):
        ncl, dt = oracle_sample(s, rho_in, -0.27, th)
        times.append(dt)
    total = sum(times)
    value = ncl * args.steps / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample_clusters_per_step": ncl},
            "cpu_baseline": {"value": value, "unit": "clusters/s", "cores": th, "host_cores": os.cpu_count(),
                             "kind": "oracle", "sample": sample_text(s.natoms)},
            "e2e": {"value": value, "unit": "clusters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# multi-rank bookkeeping (replicas: one whole workload per rank)
# ---------------------------------------------------------------------------
def max_over_ranks(x, world, device=None):
    """The largest of the ranks' values (a job's time is its slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, clusters, steps, seconds):
    """Clusters per second of the whole job: every rank solves all clusters of its
    own copy of the workload, the job takes the slowest rank's time."""
    return world * clusters * steps / seconds


# ---------------------------------------------------------------------------
# the SCF loop (mixing) on the metallic bcc slab
# ---------------------------------------------------------------------------
SCF_WORKLOAD = ("SCF loop, 7840-atom bcc slab (20x20x10 cells, a=5.4 bohr, 2% vacancies, vacuum in z, "
                "9 s-Gaussians/atom, r_core=6, r_lno=11 bohr, 3 LNOs/atom, kT=0.005 Ha): 5 steps of LNO "
                "regeneration, solve, mu search, rho rows and linear mixing 0.3, one CUDA graph per step")
SCF_STEPS = 5


def measure_scf(world):
    """Five SCF steps (dclno_scf_run, captured graph) in each precision, CUDA events
    on the context's stream; inputs resident on the device."""
    import torch
    import torch.distributed as dist

    import tbsystems as T
    from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, Context

    s = T.make_system(4)
    rho0 = torch.from_numpy(T.synthetic_density(s, seed=4)).cuda()
    H = torch.from_numpy(s.H).cuda()
    S = torch.from_numpy(s.S).cuda()
    stream = torch.cuda.Stream()
    out = {"workload": SCF_WORKLOAD, "steps": SCF_STEPS, "clusters": s.natoms}
    with torch.cuda.stream(stream):
        ctx = Context(stream=stream.cuda_stream)
        ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                           s.r_core, s.r_lno, s.k_lno)
        dims = ctx.cluster_info()[0]
        out["cluster_dim_min"], out["cluster_dim_max"] = int(dims.min()), int(dims.max())
        for name, prec in (("fp64", DCLNO_FP64), ("mixed", DCLNO_MIXED)):
            # eager steps first: the schedule tuner decides outside graph capture
            tmp = torch.zeros_like(rho0)
            for _ in range(TUNE_STEPS):
                ctx.step(rho0, tmp, s.n_electrons, s.kT, precision=prec)
            rho = rho0.clone()
            ctx.scf_run(rho, 1, 0.3, s.n_electrons, s.kT, prec, use_graph=True)  # warm-up
            rho = rho0.clone()
            stream.synchronize()
            if world > 1:
                dist.barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            mu, n, eb = ctx.scf_run(rho, SCF_STEPS, 0.3, s.n_electrons, s.kT, prec, use_graph=True)
            e1.record(stream)
            stream.synchronize()
            if world > 1:
                dist.barrier()
            # the reduction's tensor lives on this rank's GPU (NCCL reduces device tensors only)
            ms = max_over_ranks(e0.elapsed_time(e1), world, torch.device("cuda", torch.cuda.current_device()))
            out[name] = {"value": replica_throughput(world, s.natoms, SCF_STEPS, ms / 1e3), "unit": "clusters/s",
                         "ms_per_step": ms / SCF_STEPS, "mu_last": float(mu[-1]), "e_band_last": float(eb[-1])}
        out["schedules"] = schedule_summary(ctx.tuning_report())
        ctx.close()
    out["e_band_diff_per_atom_mixed_vs_fp64"] = abs(out["mixed"]["e_band_last"] - out["fp64"]["e_band_last"]) / s.natoms
    return out


# ---------------------------------------------------------------------------
# Ogita-Aishima refinement sweeps (dclno_refine_eigenpairs) at the benchmark's
# cluster dimension
# ---------------------------------------------------------------------------
REFINE_PENCILS, REFINE_N, REFINE_SWEEPS = 32, 680, 2
REFINE_WORKLOAD = (f"{REFINE_PENCILS} pencils (H, S) of dimension {REFINE_N} (the 1728-atom step's cluster "
                   "dimension) with known eigenpairs (cond(S) = 100, eigenvalues over [-2, 2]), starts "
                   f"X = C (I + 1e-6 P); {REFINE_SWEEPS} sweeps per call")


def measure_refinement(dfma):
    """Refinement sweeps on a batch of pencils whose eigenpairs are known: time of one
    call of REFINE_SWEEPS sweeps (CUDA events on the current stream; the call allocates
    its workspace and synchronises inside), FP64 roofline of its 10 n^3 flops per pencil
    and sweep against the measured FP64 FMA rate, errors against the known pairs."""
    import numpy as np
    import torch

    import tbsystems as T
    from paper_1809_05637_gb300 import refine_eigenpairs

    H, S, C, w = T.known_pencils(REFINE_PENCILS, REFINE_N, seed=41)
    rng = np.random.default_rng(42)
    X0 = np.stack([C[p] @ (np.eye(REFINE_N) + 1e-6 * rng.standard_normal((REFINE_N, REFINE_N)))
                   for p in range(REFINE_PENCILS)])
    dH, dS, dX0 = (torch.from_numpy(a).cuda() for a in (H, S, X0))
    dX = dX0.clone()
    refine_eigenpairs(dH, dS, dX, nsweeps=1)  # warm-up (module load, allocator)
    dX.copy_(dX0)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lam = refine_eigenpairs(dH, dS, dX, nsweeps=REFINE_SWEEPS)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    flops = 10.0 * REFINE_N ** 3 * REFINE_PENCILS * REFINE_SWEEPS
    achieved = flops / (ms / 1e3) / 1e12
    lam = lam.cpu().numpy()
    X = dX.cpu().numpy()
    return {"workload": REFINE_WORKLOAD, "ms_per_sweep": ms / REFINE_SWEEPS,
            "pencil_sweeps_per_s": REFINE_PENCILS * REFINE_SWEEPS / (ms / 1e3),
            "roofline": {"bound": "alu", "kernel": "k_refine_gemm", "achieved": achieved, "peak": dfma,
                         "unit": "TFLOP/s", "frac": achieved / dfma, "traffic": None,
                         "peak_source": "measured in-process FP64 FMA rate (the products run on FP64 FMA)",
                         "flops_per_call": flops},
            "max_abs_eig_err": float(np.max(np.abs(lam - w))), "max_abs_vec_err": float(np.max(np.abs(X - C))),
            "start_vec_err": float(np.max(np.abs(X0 - C)))}


# ---------------------------------------------------------------------------
# the 32,000-atom amorphous workload, streamed
# ---------------------------------------------------------------------------
AMORPHOUS = ("DC-LNO step, {n}-atom amorphous two-species packing (random sequential addition at 0.012 "
             "atoms/bohr^3, d_min 3.8 bohr, periodic cube), 13 s-Gaussians/atom, r_core=6, r_lno=10 bohr, "
             "4 LNOs/atom, kT=0.01 Ha, memory-admitted batches")


def measure_amorphous(n_atoms):
    """One LNO step of the amorphous workload in FP64 and in mixed precision: S, H
    and the input density are generated row range by row range (host threads) straight
    into device memory (the host never holds them), the context admits the cluster
    workspace in batches; invariants on the device and, for both paths, sampled
    clusters against the oracle (host blocks computed only for the rows those clusters
    touch)."""
    import numpy as np
    import torch

    import tbsystems as T
    from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, Context

    def ddot(a, b, chunk=1 << 30):  # cuBLAS dot takes at most 2^31 - 1 elements
        return sum(float(torch.dot(a[k:k + chunk], b[k:k + chunk])) for k in range(0, a.numel(), chunk))

    t0 = time.perf_counter()
    s = T.make_system_streamed(5, n_atoms=n_atoms)
    t_struct = time.perf_counter() - t0
    nval = len(s.S)
    dev = torch.device("cuda", torch.cuda.current_device())
    H = torch.empty(nval, dtype=torch.float64, device=dev)
    S = torch.empty_like(H)
    R = torch.empty_like(H)
    for i0, i1, o0, sv, hv, rv in T.row_chunks(s, 128, density_seed=11):
        S[o0:o0 + len(sv)].copy_(torch.from_numpy(sv))
        H[o0:o0 + len(hv)].copy_(torch.from_numpy(hv))
        R[o0:o0 + len(rv)].copy_(torch.from_numpy(rv))
    torch.cuda.synchronize()
    t_fill = time.perf_counter() - t0 - t_struct
    out = torch.zeros_like(H)
    stream = torch.cuda.current_stream(dev)
    ctx = Context(stream=stream.cuda_stream)
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                       s.r_core, s.r_lno, s.k_lno)
    t_build = time.perf_counter() - t0 - t_struct - t_fill
    nb, ws = ctx.batch_info()
    dims = ctx.cluster_info()[0]
    print(f"amorphous {s.natoms}: structure {t_struct:.0f} s, device fill {t_fill:.0f} s, clusters {t_build:.0f} s, "
          f"{nb} batches of <= {ws / 1e9:.1f} GB", file=sys.stderr, flush=True)
    res = {}
    for name, prec in (("fp64", DCLNO_FP64), ("mixed", DCLNO_MIXED)):
        # warm-up: tunes the QL launch shape and (batches share tuner slots) the schedules
        ctx.step(R, out, s.n_electrons, s.kT, precision=prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        mu, n, eb = ctx.step(R, out, s.n_electrons, s.kT, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        res[name] = {"value": s.natoms / (ms / 1e3), "unit": "clusters/s", "ms_per_step": ms, "mu": mu,
                     "n_electrons": n, "e_band": eb,
                     "trace_rho_s_minus_n": abs(2.0 * ddot(out, S) - n) / s.n_electrons,
                     "trace_rho_h_minus_eband": abs(2.0 * ddot(out, H) - eb) / abs(eb)}
    # sampled clusters against the oracle (both paths, rows at the FP64 step's mu)
    import oracle as O

    mu_fix = res["fp64"]["mu"]
    sample = [0, s.natoms // 2]
    cls = {i: O.cluster_members(s, i, s.r_core, s.r_lno, s.k_lno) for i in sample}
    rows_needed = set()
    for cl in cls.values():
        rows_needed |= {int(a) for a in cl.atoms}
    T.fill_rows(s, rows_needed)
    rho_host = np.zeros(nval)  # untouched pages stay unallocated
    for i in rows_needed:
        T.synthetic_density_rows(s, i, i + 1, rho_host, seed=11)
    need = set()
    for cl in cls.values():
        need |= {int(a) for a, c in zip(cl.atoms, cl.core) if not c}
    lno = O.compute_lnos(s, rho_host, s.k_lno, atoms=sorted(need))
    V = {j: v[0] for j, v in lno.items()}
    ores = O.dclno_solve(s, V, s.r_core, s.r_lno, s.k_lno, atoms=sample, threads=len(sample))
    out_rows = np.zeros(nval)
    for i, r in ores.items():
        O.density_rows(s, r.cluster, r.eps, r.C, V, mu_fix, s.kT, out_rows)
    for name, prec in (("fp64", DCLNO_FP64), ("mixed", DCLNO_MIXED)):
        ctx.step(R, out, s.n_electrons, s.kT, precision=prec)
        ctx.density_matrix(mu_fix, s.kT, out)
        spec = ctx.spectrum()
        deps, deps_b, drho = 0.0, 0.0, 0.0
        for i, r in ores.items():
            d = np.abs(np.sort(spec[i][0]) - r.eps)
            # first-order bound of a backward error n u in H^(i), S^(i) (c^T S c = 1)
            bound = 1e-10 + 2.0 * len(r.eps) * 2.0 ** -53 * (r.h_norm + np.abs(r.eps) * r.s_norm) * np.einsum(
                "am,am->m", r.C, r.C)
            deps = max(deps, float(np.max(d)))
            deps_b = max(deps_b, float(np.max(d / bound)))
            o0, o1 = int(s.blk_off[s.row_ptr[i]]), int(s.blk_off[s.row_ptr[i + 1]])
            g = out[o0:o1].cpu().numpy()
            drho = max(drho, float(np.max(np.abs(g - out_rows[o0:o1])) / np.max(np.abs(out_rows[o0:o1]))))
        res[name]["oracle_sample"] = {"clusters": sample, "max_abs_eps_diff_ha": deps,
                                      "max_eps_diff_over_first_order_bound": deps_b,
                                      "max_rho_row_diff_rel_to_row_max": drho, "mu": mu_fix}
    schedules = schedule_summary(ctx.tuning_report())
    ctx.close()
    del H, S, R, out
    torch.cuda.empty_cache()
    return {"workload": AMORPHOUS.format(n=s.natoms), "clusters": s.natoms, "cluster_dim_min": int(dims.min()),
            "cluster_dim_max": int(dims.max()), "stored_blocks": int(len(s.col)), "matrix_gb": nval * 8 / 1e9,
            "batches": nb, "workspace_gb": ws / 1e9, "host_structure_s": t_struct, "fill_s": t_fill,
            "clusters_build_s": t_build, "fp64": res["fp64"], "mixed": res["mixed"],
            "e_band_diff_per_atom_mixed_vs_fp64": abs(res["mixed"]["e_band"] - res["fp64"]["e_band"]) / s.natoms,
            "schedules": schedules}


def run_streamed(args):
    print(json.dumps(measure_amorphous(args.atoms)))
    return 0


# ---------------------------------------------------------------------------
# rooflines
# ---------------------------------------------------------------------------
SLICE_PRODUCTS = 36  # BF16 slice products per emulated FP64 multiply-add (levels t + u <= 7 of 8 x 8 slices)


def bf16_peak():
    """Dense BF16 tensor rate (TFLOP/s) the emulated contractions are measured against:
    the sustained cuBLAS figure of MEASURED_PEAKS.json (the kernels run inside a
    seconds-long step), else the fallback of one earlier GB300 measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops_sustained"])
        return v, "measured (MEASURED_PEAKS.json bf16_tflops_sustained)"
    except (OSError, KeyError, ValueError):
        return 1700.0, "fallback (1.7 PFLOP/s sustained bf16, an earlier GB300 measurement)"


def roofline_report(kernel, path, n, k_ms, k_n, dfma, dmma, bf16, bf16_src):
    """Roofline of one launch of a tridiagonalisation kernel over all clusters
    (dimensions n), against that kernel's own floor: the time its flop mix takes at
    the measured peaks.  frac = floor / measured launch time; peak = algorithmic
    flops / floor (the kernel's own effective peak, FP64-equivalent for emulated work).

    k_tridiag  one-stage Householder, 4 n^3/3: half symmetric matrix-vector products
               (FP64 FMA in both paths), half rank-2k updates (FP64 MMA, or emulated on
               BF16 tensor cores at 36 slice products per FP64 multiply-add).
    k_band     dense -> band of half-width BW = 32, 4 n^3/3 in tile products (FP64 MMA or
               emulated) plus the panel work (QR, T, W: about 4 n^2 BW FP64 flops).
    k_chase    band -> tridiagonal by bulge chasing, about 6 n^2 BW FP64 flops."""
    import numpy as np

    n = np.asarray(n, dtype=np.float64)
    bw = 32.0
    if kernel == "k_tridiag":
        flops = float(np.sum(4.0 * n ** 3 / 3.0))
        fma_f, mma_f = flops / 2.0, flops / 2.0
    elif kernel == "k_band":
        gemm = float(np.sum(4.0 * n ** 3 / 3.0))
        fma_f, mma_f = float(np.sum(4.0 * n ** 2 * bw)), gemm
        flops = gemm + fma_f
    else:  # k_chase
        flops = float(np.sum(6.0 * n ** 2 * bw))
        fma_f, mma_f = flops, 0.0
    if path == "fp64":
        floor_s = fma_f / (dfma * 1e12) + mma_f / (dmma * 1e12)
        src = f"measured in-process: FP64 FMA {dfma:.3f}, FP64 MMA {dmma:.3f} TFLOP/s"
    else:
        floor_s = fma_f / (dfma * 1e12) + SLICE_PRODUCTS * mma_f / (bf16 * 1e12)
        src = (f"FP64 part on measured FP64 FMA {dfma:.3f} TFLOP/s; tile products as {SLICE_PRODUCTS} BF16 slice "
               f"products per FP64 multiply-add at {bf16:.0f} TFLOP/s BF16, {bf16_src}")
    launch_s = k_ms / max(k_n, 1) / 1e3 if k_n else None
    per = TRAFFIC_PER_CLUSTER.get((kernel, path))
    traffic = per * len(n) if per is not None else None
    traffic_src = ("ncu dram__bytes_read.sum + dram__bytes_write.sum per cluster of this kernel on the 216-cluster "
                   "rock-salt case (same cluster dimensions), times the clusters of this launch"
                   if per is not None else "no capture of this kernel on this path")
    achieved = flops / launch_s / 1e12 if launch_s else None
    peak = flops / floor_s / 1e12
    return {"bound": "alu", "kernel": kernel, "path": path, "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s (FP64-equivalent)" if path == "mixed" else "TFLOP/s",
            "frac": (achieved / peak) if achieved else None, "traffic": traffic,
            "traffic_source": traffic_src,
            "peak_source": src, "flops_per_launch": flops, "floor_ms": floor_s * 1e3,
            "launch_ms": launch_s * 1e3 if launch_s else None}


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per cluster of one launch,
# from an ncu capture of each kernel on the 216-cluster rock-salt case (the benchmark's
# recipe on 6^3 sites: the same cluster dimensions, 654-702), scaled to a launch by its
# clusters: in both cases each cluster's trailing matrix (3.7 MB) is many times its
# share of the L2, so every pass over it goes to DRAM.  Taken on the kernels as they
# are now; a change to a kernel voids its entry.
TRAFFIC_PER_CLUSTER = {
    ("k_tridiag", "fp64"): (83441013504 + 7083535104) / 216,
    ("k_band", "mixed"): (15157292800 + 10908427520) / 216,
}

TUNE_STEPS = 4  # eager solves the schedule tuner needs to decide (its largest candidate set)


def schedule_summary(report):
    """Per precision and kernel: (rounded cluster dimension, engine, persistent grid) of
    every size bucket, from the library's tuning report."""
    out = {}
    for b in report.get("batches", []):
        for bk in b["buckets"]:
            for name, v in bk["schedules"].items():
                out.setdefault(name, []).append([bk["n_rounded"], v["engine"], v["persistent"], v["decided"]])
    return out


def dominant(times):
    """The roofline kernel with the largest time in a {kernel: (ms, launches)} map."""
    have = [(times[k][0], k) for k in ROOFLINE_KERNELS if times.get(k, (0.0, 0))[1] > 0]
    return max(have)[1] if have else "k_tridiag"


def step_fmin_report(path, n3, step_ms, dfma, dmma, bf16, two_stage=False):
    """The whole step against its algorithmic minimum F_min = sum 8 n^3 / 3 (Cholesky
    n^3/3, symmetric congruence n^3, tridiagonalisation 4 n^3/3): FP64 path at the
    1:1 FP64 FMA/MMA rate; mixed path emulated at 36 BF16 slice products per FP64
    multiply-add, except the one-stage tridiagonalisation's symv half (2 n^3/3),
    which stays on FP64 FMA (with the two-stage form everything cubic is emulated)."""
    fmin = float(n3.sum() * 8.0 / 3.0)
    if path == "fp64":
        floor_s = fmin / (1e12 / (0.5 / dfma + 0.5 / dmma))
    else:
        f64 = 0.0 if two_stage else float(n3.sum() * 2.0 / 3.0)
        floor_s = f64 / (dfma * 1e12) + SLICE_PRODUCTS * (fmin - f64) / (bf16 * 1e12)
    return {"fmin_flops": fmin, "achieved_tflops": fmin / (step_ms / 1e3) / 1e12, "floor_ms": floor_s * 1e3,
            "frac": floor_s * 1e3 / step_ms}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import tbsystems as T
    from paper_1809_05637_gb300 import DCLNO_FP64, DCLNO_MIXED, Context, measure_fp64_peaks

    dev = torch.device("cuda", local)
    s = make_workload(args.workload)
    rho_host = T.synthetic_density(s, seed=11)
    H = torch.from_numpy(s.H).to(dev)
    S = torch.from_numpy(s.S).to(dev)
    rho_in = torch.from_numpy(rho_host).to(dev)
    rho_out = torch.zeros_like(rho_in)
    stream = torch.cuda.current_stream(dev)
    ctx = Context(stream=stream.cuda_stream)
    ctx.set_tridiag(args.tridiag)  # before the build: the two-stage form lays out its reflector log there
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift, s.blk_off, H, S,
                       s.r_core, s.r_lno, s.k_lno)
    ctx.set_mixed_engine(args.mixed_engine)
    dims = ctx.cluster_info()[0]
    ncl = int(s.natoms)

    def step(prec=DCLNO_FP64):
        return ctx.step(rho_in, rho_out, s.n_electrons, s.kT, precision=prec)

    # warm-up: at least TUNE_STEPS eager steps, so that the schedule tuner (which times one
    # candidate per size bucket and kernel per eager solve) has decided before the timing
    warmup = max(args.warmup, 3, TUNE_STEPS)
    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    l0 = ctx.launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            mu, n_mu, e_band = step()
        ev1.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
    ms = ev0.elapsed_time(ev1)
    launches = ctx.launch_count() - l0
    t64 = {k: ctx.kernel_time(k) for k in KERNELS}
    ctx.set_profiling(False)
    clocks = clk.summary()
    gpu_samples = {}  # per path: spectra and the density rows at the FP64 step's mu (oracle comparison)

    def keep_sample(name):
        out = torch.zeros_like(rho_in)
        ctx.density_matrix(mu, s.kT, out)
        gpu_samples[name] = (ctx.spectrum(), out.cpu().numpy())

    keep_sample("fp64")
    ms = max_over_ranks(ms, world, dev)
    value = replica_throughput(world, ncl, args.steps, ms / 1e3)

    # the mixed-precision form of the same step (BF16 tensor-core emulation of the FP64
    # contractions), timed the same way; accuracy against the FP64 step above
    for _ in range(warmup):
        step(DCLNO_MIXED)
    torch.cuda.synchronize()
    ctx.set_profiling(True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        mu_mx, n_mx, e_mx = step(DCLNO_MIXED)
    ev1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms_mx = ev0.elapsed_time(ev1)
    tmx = {k: ctx.kernel_time(k) for k in KERNELS}
    ctx.set_profiling(False)
    ms_mx = max_over_ranks(ms_mx, world, dev)
    keep_sample("mixed")

    # e2e: the C-ABI step with host buffers (H2D of rho_in and D2H of rho_out inside)
    e2e = None
    if not args.no_e2e:
        h_in = torch.from_numpy(rho_host).pin_memory()
        h_out = torch.empty_like(h_in).pin_memory()
        ctx.step(h_in, h_out, s.n_electrons, s.kT, host_buffers=True)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.step(h_in, h_out, s.n_electrons, s.kT, host_buffers=True)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        dt = max_over_ranks(dt, world, dev)
        nbytes = int(rho_host.nbytes)
        e2e = {"value": replica_throughput(world, ncl, args.steps, dt), "unit": "clusters/s",
               "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes}

    # roofline of the dominant kernel of each path, against that kernel's own floor
    # (see roofline_report); the whole step's algorithmic minimum F_min beside it
    dfma, dmma = measure_fp64_peaks()
    bf16, bf16_src = bf16_peak()
    n3 = dims.astype(np.float64) ** 3
    k64 = dominant(t64)
    roofline = roofline_report(k64, "fp64", dims, *t64[k64], dfma, dmma, bf16, bf16_src)
    roofline["step_fmin"] = step_fmin_report("fp64", n3, ms / args.steps, dfma, dmma, bf16)
    roofline["kernels_ms_per_step"] = {k: v[0] / args.steps for k, v in t64.items() if v[1]}
    kmx = dominant(tmx)
    mixed = {"value": replica_throughput(world, ncl, args.steps, ms_mx / 1e3), "unit": "clusters/s",
             "ms_per_step": ms_mx / args.steps,
             "speedup_vs_fp64": ms / ms_mx, "e_band_err_per_atom_vs_fp64": abs(e_mx - e_band) / s.natoms,
             "mu_diff_vs_fp64": abs(mu_mx - mu),
             "dtype": "bf16 slices (8 x 8 bit) emulating f64 contractions; f64 elsewhere",
             "roofline": roofline_report(kmx, "mixed", dims, *tmx[kmx], dfma, dmma, bf16, bf16_src)}
    mixed["roofline"]["step_fmin"] = step_fmin_report("mixed", n3, ms_mx / args.steps, dfma, dmma, bf16,
                                                      two_stage=tmx.get("k_band", (0, 0))[1] > 0)
    mixed["roofline"]["kernels_ms_per_step"] = {k: v[0] / args.steps for k, v in tmx.items() if v[1]}
    mixed["tridiagonalisation"] = "two-stage (k_band + k_chase)" if tmx.get("k_band", (0, 0))[1] else "one-stage"
    schedules = schedule_summary(ctx.tuning_report())

    scf = None
    if not args.no_scf:
        ctx.close()
        scf = measure_scf(world)

    # the 32,000-atom amorphous workload (memory-admitted batches), one GPU only
    amorphous = None
    if world == 1 and args.workload == "rocksalt1728" and not args.no_amorphous:
        ctx.close()
        del H, S, rho_in, rho_out
        torch.cuda.empty_cache()
        amorphous = measure_amorphous(args.atoms)

    refinement = None
    if world == 1 and not args.no_refine:
        torch.cuda.empty_cache()  # the library allocates the sweeps' workspace itself
        refinement = measure_refinement(dfma)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        th = cpu_threads()
        ncs, wall, _, ores, orows = oracle_sample(s, rho_host, mu, th, detail=True)
        cpu = {"value": ncs / wall, "unit": "clusters/s", "cores": th, "host_cores": os.cpu_count(),
               "kind": "oracle", "sample": sample_text(s.natoms)}
        # both GPU paths against the oracle on the sampled clusters (rows at the FP64 step's mu)
        line_err = {}
        for name, (spec_g, rows_g) in gpu_samples.items():
            line_err[name] = oracle_errors(s, ores, orows, spec_g, rows_g)
        roofline["oracle_sample"] = line_err["fp64"]
        mixed["oracle_sample"] = line_err["mixed"]

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "clusters/s", "n_gpus": world, "steps": args.steps,
                "warmup": warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": WORKLOAD if args.workload == "rocksalt1728" else args.workload,
                           "precision": "fp64", "clusters": ncl,
                           "cluster_dim_min": int(dims.min()), "cluster_dim_max": int(dims.max()),
                           "parallelism": f"replicas x{world}", "tridiag_option": args.tridiag,
                           "mixed_engine": args.mixed_engine,
                           "l2": "no flush: S, H and rho (5.2 GB) exceed the 129 MB L2"},
                "clocks": clocks, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
                "schedules": schedules,
                "cpu_baseline": cpu, "mixed": mixed, "scf": scf, "amorphous32000": amorphous, "refinement": refinement, "mu": mu,
                "n_electrons": n_mu, "e_band": e_band}
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "amorphous32000":
        return run_streamed(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
