"""DC-LNO oracle: a plain, slow, FP64 CPU statement of the hot path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` import this package.  The product path (the
CUDA library and its Python binding) never imports, links or executes it, and
the two share no code; they share only the seeded inputs of ``tbsystems``.

What it computes follows the paper (Ozaki, Fukuda, Jiang, "Efficient O(N)
divide-conquer method with localized natural orbitals"), Sec. II:

* ``lambda_blocks``  Lambda_0i = sum_Rj rho_{0i,Rj} S_{Rj,0i}      Eq. (Lambda)
* ``lnos``           V^-1 Lambda V = lambda, keep the leading k     Eq. (eigendecomp), (apop_Lambda)
* ``cluster_members``/``assemble``  H^(i), S^(i) in the PAO/LNO basis  Eq. (Hi)
* ``solve_cluster``  H^(i) c = eps S^(i) c, central-atom weights     Eq. (Gi)
* ``find_mu``        common chemical potential                       Sec. II.C step (iv)
* ``density_rows``   rho_{0i,Rj} = sum_mu f(eps_mu) c c             Eq. (dm) with Eq. (Gi)
* ``full_diag``      conventional diagonalisation of a whole open system

Pins: see ``tests/test_oracle_*.py``.  Parity unpinned: the LNO vectors
themselves (only the span they define is fixed by the method; tests compare
cluster results, and vectors only when the selected eigenvalues are simple).
"""
from .dclno_oracle import *  # noqa: F401,F403
