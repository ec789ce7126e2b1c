"""Seeded synthetic inputs: pyramid meshes and random coefficient states.

This module is the one place both the CUDA path and the CPU oracle take their
inputs from. It holds none of the method's arithmetic: it only lays out a box
of hexahedra, cuts each hexahedron into six pyramids that share the hex centre
as apex (Sec. 3.2 and Sec. 4.3 of the paper build their meshes this way), and
perturbs vertex positions with a seeded generator.

Vertex order of each pyramid (EToV row): v1..v4 are the base quadrilateral,
ordered so that (v2 - v1) x (v4 - v1) points toward the apex v5; v3 is the base
vertex opposite v1. This matches the reference pyramid of Sec. 2, whose base
vertices (-1,-1,-1), (1,-1,-1), (1,1,-1), (-1,1,-1) carry the apex (-1,-1,1)
above them, so the vertex map has a positive Jacobian.
"""

from __future__ import annotations

import numpy as np

# The six faces of a unit hex as (v1, v2, v3, v4) corner offsets (dx, dy, dz),
# each ordered so that (v2 - v1) x (v4 - v1) points into the hex (toward the
# centre, which becomes the apex).
_HEX_FACES = (
    ((0, 0, 0), (0, 1, 0), (0, 1, 1), (0, 0, 1)),  # x = 0, inward +x
    ((1, 0, 0), (1, 0, 1), (1, 1, 1), (1, 1, 0)),  # x = 1, inward -x
    ((0, 0, 0), (0, 0, 1), (1, 0, 1), (1, 0, 0)),  # y = 0, inward +y
    ((0, 1, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1)),  # y = 1, inward -y
    ((0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0)),  # z = 0, inward +z
    ((0, 0, 1), (0, 1, 1), (1, 1, 1), (1, 0, 1)),  # z = 1, inward -z
)


def make_pyramid_mesh(nx, ny=None, nz=None, delta=0.0, seed=0, domain=(0.0, 1.0)):
    """Box of nx*ny*nz hexahedra, each cut into 6 pyramids from its centre.

    Parameters
    ----------
    nx, ny, nz : hexahedra per axis (ny, nz default to nx).
    delta : relative perturbation. Every coordinate of every vertex that is
        not on the box boundary (interior grid vertices and all hex centres)
        moves by an independent U[-delta*h, delta*h], with h the hex size
        along that axis. Boundary vertices stay put, so the box is kept.
    seed : seed of numpy.random.default_rng. One (Nv, 3) array of U[-1, 1)
        draws is taken for all vertices in index order (grid vertices with x
        fastest, then hex centres in hex order); boundary rows are zeroed.
    domain : (lo, hi) of the cube on every axis.

    Returns
    -------
    vertices : float64 array (Nv, 3)
    EToV : int32 array (K, 5), K = 6*nx*ny*nz, hex-major (x fastest), the six
        pyramids of a hex in face order -x, +x, -y, +y, -z, +z.
    """
    ny = nx if ny is None else ny
    nz = nx if nz is None else nz
    lo, hi = float(domain[0]), float(domain[1])
    h = np.array([(hi - lo) / nx, (hi - lo) / ny, (hi - lo) / nz])

    gi, gj, gk = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1), np.arange(nz + 1), indexing="ij")
    # vertex id = i + (nx+1)*(j + (ny+1)*k): flatten with x fastest
    grid = np.stack([gi.ravel(order="F"), gj.ravel(order="F"), gk.ravel(order="F")], axis=1)
    ngrid = grid.shape[0]
    hi_idx, hj_idx, hk_idx = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    hexes = np.stack([hi_idx.ravel(order="F"), hj_idx.ravel(order="F"), hk_idx.ravel(order="F")], axis=1)
    nhex = hexes.shape[0]

    verts = np.empty((ngrid + nhex, 3))
    verts[:ngrid] = lo + grid * h
    verts[ngrid:] = lo + (hexes + 0.5) * h

    interior = np.ones(ngrid + nhex, dtype=bool)
    n = np.array([nx, ny, nz])
    on_bnd = np.any((grid == 0) | (grid == n), axis=1)
    interior[:ngrid] = ~on_bnd

    rng = np.random.default_rng(seed)
    draws = rng.uniform(-1.0, 1.0, size=(ngrid + nhex, 3))
    if delta != 0.0:
        verts += np.where(interior[:, None], draws * (delta * h), 0.0)

    def gid(i, j, k):
        return i + (nx + 1) * (j + (ny + 1) * k)

    etov = np.empty((nhex, 6, 5), dtype=np.int64)
    for f, quad in enumerate(_HEX_FACES):
        for v, (dx, dy, dz) in enumerate(quad):
            etov[:, f, v] = gid(hexes[:, 0] + dx, hexes[:, 1] + dy, hexes[:, 2] + dz)
        etov[:, f, 4] = ngrid + np.arange(nhex)
    return verts, etov.reshape(nhex * 6, 5).astype(np.int32)


def random_state(K, Np, seed, scale=1.0):
    """Seeded random coefficient array of shape (K, 4, Np), float64, U[-scale, scale)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-scale, scale, size=(K, 4, Np))


def num_modes(N):
    """Np = (N+1)(N+2)(2N+3)/6 coefficients per field on a pyramid of degree N."""
    return (N + 1) * (N + 2) * (2 * N + 3) // 6


def batch_mesh_shapes(count=256, kmin=48, kmax=49152, nmin=2, nmax=6, seed=2):
    """Box shapes and degrees for a batch of independent meshes.

    Hex counts H = K/6 are drawn log-uniformly so that K spans [kmin, kmax];
    n = max(2, round(H^(1/3))) hexes along x and y and nz = max(1, round(H/n^2))
    along z, all on the unit cube. Degrees are uniform integers in [nmin, nmax].
    Returns a list of (nx, ny, nz, N).
    """
    rng = np.random.default_rng(seed)
    logk = rng.uniform(np.log(kmin), np.log(kmax), size=count)
    degs = rng.integers(nmin, nmax + 1, size=count)
    out = []
    for lk, N in zip(logk, degs):
        H = np.exp(lk) / 6.0
        n = max(2, int(round(H ** (1.0 / 3.0))))
        nz = max(1, int(round(H / (n * n))))
        out.append((n, n, nz, int(N)))
    return out
