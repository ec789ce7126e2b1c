"""Plain FP64 CPU oracle for the pyramid DG acoustic-wave method (Chan & Warburton).

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call or run
anything in this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` use it. It shares
no code with the CUDA library: it takes the same seeded mesh as input and
computes the same discrete solution by a different, deliberately plain route.

Route (all float64, numpy):
  * Gauss rules by Golub-Welsch (eigenvalues of the Jacobi matrix).
  * The rational orthonormal basis psi of Eq. (1) (Bergot-Cohen-Durufle), not
    the semi-nodal basis the GPU path uses. By Lemma 4 both span the same
    space, and with the same exact cubature both give the same discrete
    solution up to rounding.
  * Geometry from Bedrosian's vertex functions in (r,s,t) (Sec. 2).
  * Dense per-element mass, stiffness and face matrices, inverted densely
    (no use of the diagonal-mass result this work is checking).
  * The flux of Sec. 4.3 and the Carpenter-Kennedy 2N-storage RK4.

Parity status of each function is stated in its docstring; every function here
is pinned by a ``-m "not gpu"`` test against something other than itself.
"""
