"""Plain FP64 CPU oracle of the IMEX HDG-DG method for planar shallow water.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code, table or
helper with the CUDA library; it is a slow, literal restatement of the paper
(Kang, Giraldo, Bui-Thanh, "IMEX HDG-DG", arXiv:1711.02751):

* ``gll``      -- Gauss-Lobatto-Legendre nodes, weights, nodal derivative matrix
                  (the tensor-product collocation the spatial discretisation uses).
* ``swe``      -- periodic quad mesh, the split shallow-water fluxes (Sec. 4.1,
                  eqs. psweFluxTensor / psweLinearFluxTensor), the DG residual
                  NL(q) (eq. WeakForm_DG with the Rusanov flux, eq. Full_russanov /
                  Linear_russanov), the HDG residual L(q, qhat) with the hybridised
                  Lax-Friedrichs flux (eq. linear_hdgflux3) and the conservation
                  residual (eq. HDGcont).
* ``hdg``      -- the implicit stage system of Sec. 6 (eq. linearizedHDGsystem):
                  direct solve of the unreduced (Q, Qhat) system, and the static
                  condensation route (eq. linearizedHDGsystem_schur, then
                  eq. recover_volume_unknowns).
* ``imex``     -- the ARS IMEX-RK tableaux (Sec. 2, eq. IMEXRKi) and Algorithm 1
                  (IMEX HDG-DG), plus diagnostics (mass, energy, relative L2).

Pins (closed forms, invariants, brute force, printed values) live in
``tests/test_oracle_*.py``.  Every function is FP64 numpy.
"""
from . import gll, swe, hdg, imex  # noqa: F401
