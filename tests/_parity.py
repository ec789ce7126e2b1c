"""Parity check shared by the GPU tests: a CUDA-path state against the oracle's, compared by
their values at every element's volume cubature points, both mesh-wide (quadrature-weighted
relative L2 over the four fields) and on the worst element (that element's L2 difference over
the larger of its own norm and the root-mean-square element norm), each within the tolerance.
"""

import json
import os

TOL = {"f64": 1e-12, "f32": 1e-5}


def parity(dg, A, B, elems=None):
    """(mesh-wide relative L2, worst element) of point arrays A (CUDA path) and B (oracle)."""
    if elems is None:
        rel = dg.rel_l2_points(A, B)
    else:
        import numpy as np
        wJ = dg.w[None, :] * dg.J[np.asarray(elems)]
        rel = float(np.sqrt(np.einsum("kq,kqc->", wJ, (A - B) ** 2) / np.einsum("kq,kqc->", wJ, B ** 2)))
    return rel, dg.worst_element_rel(A, B, elems)


def check(dg, A, B, tol, ctx=None, elems=None):
    """Assert both parity measures are within tol; returns them. With PYRDG_PARITY_LOG set, each
    check appends one JSON line (test, context, both measures, tolerance) to that file, so the
    measured errors against the oracle can be reported as numbers."""
    rel, worst = parity(dg, A, B, elems)
    record(rel, worst, tol, ctx)
    return rel, worst


def record(rel, worst, tol, ctx=None):
    """Log (see check) and assert a pair of parity measures."""
    log = os.environ.get("PYRDG_PARITY_LOG")
    if log:
        with open(log, "a") as fh:
            fh.write(json.dumps({"test": os.environ.get("PYTEST_CURRENT_TEST", "").split(" ")[0],
                                 "ctx": repr(ctx), "rel_l2": float(rel), "worst_element": float(worst),
                                 "tol": tol}) + "\n")
    assert rel <= tol and worst <= tol, (ctx, "rel", rel, "worst element", worst, "tol", tol)
