"""GB300-native DC-LNO hot path (Ozaki, Fukuda, Jiang: O(N) divide-conquer with
localized natural orbitals).

The work runs in ``libdclno.so`` (hand-written sm_103a CUDA behind a C ABI,
declared in ``include/dclno.h``).  This package is its thin Python binding:
argument marshalling only.  Importing it fails loudly if the library has not
been built; there is no CPU fallback.

One step on device arrays (``s`` holds the BSR structure and values of H, S)::

    ctx = Context()                                   # torch's current stream
    ctx.build_clusters(s.pos, s.cell, s.pbc, s.norb, s.row_ptr, s.col, s.shift,
                       s.blk_off, H, S, r_core, r_lno, k_lno)   # or kappa=0.3
    ctx.compute_lnos(rho_in)                          # Lambda, LNOs
    ctx.solve_clusters(DCLNO_FP64)                    # or DCLNO_MIXED
    mu, n_mu = ctx.find_mu(n_electrons, kT)
    e_band = ctx.density_matrix(mu, kT, rho_out)

or ``ctx.step(rho_in, rho_out, n_electrons, kT)`` for all of it, and
``ctx.scf_run(rho, nsteps, 0.3, n_electrons, kT, use_graph=True)`` for an SCF
loop with linear mixing.  ``set_workspace_limit`` (memory-admitted batches),
``set_lno_threshold`` (lambda_th selection), ``set_lno_mode`` (the symmetric
projector form of the LNO eigenproblem) and ``set_autotune`` adjust the run.
``refine_eigenpairs`` applies Ogita-Aishima refinement sweeps with FP64
residuals to batched approximate eigendecompositions of pencils (H, S).
"""
from ._lib import (  # noqa: F401
    DCLNO_FP64, DCLNO_MIXED, DCLNO_LNO_PAPER, DCLNO_LNO_SYM, LIB_PATH, Context, DclnoError, STATUS_NAMES, exported_symbols, load_library,
    find_mu_noalloc, measure_fp64_peaks, refine_eigenpairs,
)
