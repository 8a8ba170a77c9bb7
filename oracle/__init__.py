"""Plain, slow, FP64 CPU oracle for the layered-media Nystrom BIE.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
It shares no code with the CUDA library in ``paper_2511_12450_gb300/``; the two
meet only through the seeded input generators in ``workloads/``.

What it computes is the plain definition of the operator that the fast
multipole method accelerates (Sec. 3.3, eqs. linearSystem, matrixelmemts):
the dense Nystrom matrix K with exactly evaluated layered Green's functions,
its product with a vector, the dense GMRES solution and the scattered field.

Modules
  core          ctypes wrapper of oracle_core.c: reaction Green's function G^r by
                a direct interface solve + adaptive Sommerfeld contour quadrature
  green         free-space kernel (i/4) H_0^(1) and the full layered G
  nystrom       elements, self term I^s, dense K, matvec, field evaluation
  combined      combined-field (double + single layer) operator and field, an
                opt-in second-kind form; needs the field-point gradient of G^r
                (core.gr_grad_block)
  background    plane incidence and the background field u^b (transfer solve)
  paper_forms   the paper's own recursions (R~, T~, sigma, A_l, B_l), used only
                to pin them against the direct solves
  gmres         dense GMRES (modified Gram-Schmidt, Givens)
  tree          plain quadtree, interaction lists and the overlapping
                domain-decomposition preconditioner (dense, per leaf)

Parity status: every function here is pinned by tests in tests/test_oracle_*.py
against closed forms, special cases, invariants or brute force.
"""
