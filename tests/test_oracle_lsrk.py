"""Pins for the Carpenter-Kennedy 2N-storage RK4 in oracle/dg.py (cited in Sec. 4.1).

The 2N-storage scheme res = A_s res + dt f(u); u += B_s res is converted to
its Butcher tableau and the eight order conditions up to order 4 are checked;
then fourth-order convergence on scalar ODEs.
"""

import numpy as np

from oracle.dg import LSRK_A, LSRK_B, LSRK_C


def _butcher():
    s = 5
    # res_s = sum_j beta_{s,j} k_j with k_j = dt f(stage j input);
    # u_{s} (after stage s) = u_0 + sum_{i<=s} B_i res_i
    beta = np.zeros((s, s))
    for i in range(s):
        if i > 0:
            beta[i, :i] = LSRK_A[i] * beta[i - 1, :i]
        beta[i, i] = 1.0
    # stage j is evaluated at u_{j-1}; u_j = u_0 + sum_{i<=j} B_i sum_l beta[i,l] k_l
    cum = np.zeros((s + 1, s))
    for j in range(s):
        cum[j + 1] = cum[j] + LSRK_B[j] * beta[j]
    A = cum[:s]  # row j: coefficients of k_l in the input of stage j
    b = cum[s]
    return A, b


def test_order_conditions():
    A, b = _butcher()
    c = A.sum(axis=1)
    np.testing.assert_allclose(c, LSRK_C, atol=1e-15)
    assert abs(b.sum() - 1) < 1e-15
    assert abs(b @ c - 1 / 2) < 1e-15
    assert abs(b @ c ** 2 - 1 / 3) < 1e-15
    assert abs(b @ A @ c - 1 / 6) < 1e-15
    assert abs(b @ c ** 3 - 1 / 4) < 1e-15
    assert abs(b @ (c * (A @ c)) - 1 / 8) < 1e-15
    assert abs(b @ A @ c ** 2 - 1 / 12) < 1e-15
    assert abs(b @ A @ A @ c - 1 / 24) < 1e-15


def _integrate(f, y0, T, n):
    dt = T / n
    y = np.array(y0)
    res = np.zeros_like(y)
    t = 0.0
    for _ in range(n):
        for s in range(5):
            res = LSRK_A[s] * res + dt * f(t + LSRK_C[s] * dt, y)
            y = y + LSRK_B[s] * res
        t += dt
    return y


def test_fourth_order_linear_and_nonlinear():
    lam = -1.0 + 2.0j
    f = lambda t, y: lam * y
    errs = [abs(_integrate(f, [1.0 + 0j], 1.0, n)[0] - np.exp(lam)) for n in (10, 20, 40)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.8)
    # y' = -y^2 + cos(t), non-autonomous: reference by a much finer run
    g = lambda t, y: -y ** 2 + np.cos(t)
    ref = _integrate(g, [0.5], 2.0, 4000)[0]
    errs = [abs(_integrate(g, [0.5], 2.0, n)[0] - ref) for n in (10, 20, 40)]
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 3.7)
