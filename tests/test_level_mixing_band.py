"""Band structure of the c-direction level mixing (Lemma 3's c functions).

With the semi-nodal c functions G_k(c) = ((1-c)/2)^k P_{N-k}^{(2k+3,0)}(c) and the
(N+1)-point Gauss-Jacobi(2,0) volume rule in c, the projections onto level k' of
the weighted c-interpolated values and derivatives,

    MH[k'][k] = sum_r w_r/4 G_k'(c_r) H_k(c_r),   H_k = 2/(1-c) G_k,
    MG[k'][k] = sum_r w_r/4 G_k'(c_r) G_k'(c_r),

are banded: MH is symmetric tridiagonal and MG is lower Hessenberg. The off-band
integrands are (1-c)^{2k'+3} times a polynomial of degree below N-k', which
P_{N-k'}^{(2k'+3,0)} is orthogonal to, and the rule integrates them exactly.
The library stores the off-band entries as exact zeros (and refuses to set up if
its own sums leave more than rounding there); the kernels skip them. The check
below uses the oracle's recurrence and Golub-Welsch rule, not the library's."""

import numpy as np
import pytest

from oracle.rules import gauss_jacobi, jacobi, jacobi_deriv


def _mixing(N):
    c, w = gauss_jacobi(N + 1, 2.0, 0.0)
    wc = w / 4.0
    G = np.array([((1 - c) / 2) ** k * jacobi(N - k, 2 * k + 3, 0.0, c) for k in range(N + 1)])
    H = np.array([2.0 / (1 - c) * G[k] for k in range(N + 1)])
    dG = np.array([-k / 2 * ((1 - c) / 2) ** max(k - 1, 0) * jacobi(N - k, 2 * k + 3, 0.0, c)
                   + ((1 - c) / 2) ** k * jacobi_deriv(N - k, 2 * k + 3, 0.0, c) for k in range(N + 1)])
    MH = np.einsum("r,ar,br->ab", wc, G, H)
    MG = np.einsum("r,ar,br->ab", wc, G, dG)
    return MH, MG


@pytest.mark.parametrize("N", range(1, 8))
def test_mh_tridiagonal_mg_hessenberg(N):
    MH, MG = _mixing(N)
    scale = max(np.abs(MH).max(), np.abs(MG).max())
    for kp in range(N + 1):
        for k in range(N + 1):
            if abs(k - kp) >= 2:
                assert abs(MH[kp, k]) < 1e-13 * scale, (kp, k, MH[kp, k])
            else:
                assert abs(MH[kp, k]) > 1e-6 * scale, (kp, k)  # the band itself is full
            if k >= kp + 2:
                assert abs(MG[kp, k]) < 1e-13 * scale, (kp, k, MG[kp, k])
            else:
                assert abs(MG[kp, k]) > 1e-6 * scale, (kp, k)
    assert np.allclose(MH, MH.T, atol=1e-13 * scale)


def test_entries_closed_form_n1():
    """Two entries at N = 1 against exact integrals (both integrands are polynomials the
    2-point rule integrates exactly). G_1 = (1-c)/2, H_1 = 1, G_0' = d/dc P_1^{(3,0)} = 5/2:
    MH[1][1] = int (1-c)^3/8 dc = 1/2,  MG[1][0] = 5/16 int (1-c)^3 dc = 5/4."""
    MH, MG = _mixing(1)
    assert abs(MH[1, 1] - 0.5) < 1e-14
    assert abs(MG[1, 0] - 1.25) < 1e-14
