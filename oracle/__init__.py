"""Plain FP64 CPU oracle of the coarse-grained Li-S model (arXiv 2511.05233).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or run
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
``cpu_baseline`` / ``--impl reference`` legs use it.  It shares no code, table or
constant with the CUDA library; both sides receive the same seeded inputs from
``paper_2511_05233_gb300.inputs``, a module that holds no model arithmetic.

Every function is written from the paper's equations in the paper's order, with
numpy as the only helper (scipy's SuperLU for exact linear solves).  All
arithmetic is complex-safe so that Jacobian-vector products can be taken by the
complex-step method (Im R(z + i*eps*v) / eps), an exact directional derivative
up to rounding that needs no hand-derived Jacobian.

Modules
  constants   parameters of Tabs. 1, 2, 5.1, 5.2 and Sec. 2
  chemistry   Tab. 3 reactions, Eqs. 2-3, 5-6, 18-24, Tab. 6 equilibrium
  dg          generic DG0 (Eq. 48) and DG1 interior-penalty (Eqs. 43-47, B1) operators
  lis         the Li-S residual of Tab. 4 on a masked voxel grid, cell voltage (Eq. A1)
  newton      complex-step JVP, coloured Jacobian, Newton with line search, implicit Euler (Eq. 50)
  control     naive controller (Fig. 4) and H211b + Richardson (Eqs. 51-54)
  init        Tab. 6 state and parabolic relaxation (Eq. 56)
  appendix    App. A 1D benchmarks (Eqs. B2-B9)

Parity status: every function above is pinned by tests in ``tests/test_oracle_*.py``
except the full discharge curve of the 3D Li-S model, which the paper gives only
as figures (parity unpinned against the paper; pinned only GPU vs oracle).
"""
