"""Plain FP64 CPU oracle for the HBPC two-derivative deferred-correction DGSEM
(Zeifang & Schuetz, "Two-derivative deferred correction time discretization for
the discontinuous Galerkin method").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the package
``paper_2109_04804_gb300`` and its CUDA library) may import, call or link this
package; only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s oracle
runs use it (the timed CPU baseline, the reference arm, and the reference
answers the bench's accuracy fields compare against, all in child processes or
the reference arm's own process).  The oracle shares no code with the CUDA path: it is written
from the paper, in numpy, in the order and notation of the paper, with library
primitives (tensordot, solve, expm) used only as single steps.

Modules
  basis   -- 1-D nodal basis, quadrature, differentiation matrices (Sec. 3.1.1)
  laws    -- physical fluxes and their Jacobian-vector products (Eq. 13, 21)
  dgsem   -- R^(1) (Eq. 12) and R^(2) (Eq. 16) on periodic Cartesian meshes
  newton  -- extended residual G (Sec. 3.2.1), matrix-free Jv (Eq. 23/24),
             GMRES, Newton (Eq. 17), BJ_ext preconditioner (Sec. 3.2.3)
  hbpc    -- Butcher tableaux (Eq. A.1-A.3) and Algorithm 1 (Sec. 2.1)
  exact   -- exact references for linear problems (dense / Fourier block)
"""
