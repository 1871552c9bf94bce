"""FP64 CPU oracle for the hybrid compressible LBM + FODIBM-R time step.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference that
the CUDA path is checked against.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may
import it.  It shares no code with the CUDA path and imports nothing from it.

Every function follows the paper (arXiv 2607.07432, "An improved fully
one-sided diffuse-interface immersed boundary method with target-value
reconstruction for compressible flows") step by step, in plain numpy FP64,
and cites the section / equation it implements.

Modules
-------
lattice   velocity sets, weights, Hermite polynomials, flux tables (App. A)
lbm       equilibrium, HRR collision, forcing, energy equation, streaming,
          far-field boundaries, the full time step (Sec. 2.2, 2.5, App. A)
ib        regularized delta, one-sided interpolation / spreading, scaling
          factor, Lagrangian weight, effective boundary, target-value
          reconstruction, Lagrangian forcing (Sec. 2.3, 2.4)

Parity status of the readings the paper leaves open is listed in each
function docstring; a^C (Eq. af2, "lattice-dependent component", only cited)
is "parity unpinned" against the paper and pinned only by physics tests.
"""
