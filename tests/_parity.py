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


def face_neighbours(EToV):
    """Element adjacency through shared faces (test-side, from vertex sets only)."""
    faces = ((0, 1, 2, 3), (0, 1, 4), (1, 2, 4), (3, 2, 4), (0, 3, 4))
    owner = {}
    nbrs = [[] for _ in range(len(EToV))]
    for k, row in enumerate(EToV):
        for f in faces:
            key = tuple(sorted(int(row[i]) for i in f))
            if key in owner:
                j = owner.pop(key)
                nbrs[k].append(j)
                nbrs[j].append(k)
            else:
                owner[key] = k
    return nbrs


def patch(nbrs, centre, radius):
    """Sorted element indices within `radius` face hops of `centre`."""
    seen = {centre: 0}
    frontier = [centre]
    for r in range(radius):
        nxt = []
        for k in frontier:
            for j in nbrs[k]:
                if j not in seen:
                    seen[j] = r + 1
                    nxt.append(j)
        frontier = nxt
    return sorted(seen)
