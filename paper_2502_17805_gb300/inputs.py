"""Seeded synthetic inputs shared by the CUDA path and the oracle.

This module holds no arithmetic of the spectral-difference method: only the
problem inputs, i.e. meshes (corner coordinates + hexahedral connectivity,
the input the paper's solver starts from, Sec. "Meshing") and random states.

* ``box_mesh``   -- periodic Cartesian box of n^3 straight hexahedra,
                    optionally with seeded vertex jitter (curved trilinear map).
* ``shell_mesh`` -- cubed-sphere shell: 6 patches x Nz x Nz zonal elements x
                    Nr radial layers, equiangular in (alpha, beta) per patch
                    (Sec. "Meshing": N_cells = 6 Nr Nz^2).
* ``reorient``   -- seeded per-element rotation of the local corner numbering,
                    so shared faces meet in all 8 orientations.
* ``random_state`` -- seeded conserved variables with positive density and
                    pressure by construction of their ranges.

Corner numbering of a hexahedron: corner (i, j, k) -> i + 2j + 4k, with the
parameter directions (xi, eta, zeta) forming a right-handed frame; in the
shell, zeta is the outward radial direction.
"""
from __future__ import annotations

import math
from typing import Tuple

import numpy as np


def box_mesh(n: int, L: float = 1.0, jitter: float = 0.0, seed: int = 0) -> Tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Periodic box [0, L)^3 with n^3 hexahedra.

    Vertex ids wrap around (vertex (i, j, k) == vertex (i mod n, ...)), so the
    connectivity itself is periodic; the geometry is unwrapped with the returned
    period lengths.  ``jitter`` displaces every vertex by a seeded uniform
    amount in [-jitter, jitter] * (L / n) per coordinate.
    Returns (vertices [n^3, 3], hexes [n^3, 8], periodic_lengths [3]).
    """
    if n < 3:
        raise ValueError("a periodic box needs at least 3 elements per direction")
    h = L / n
    idx = np.arange(n)
    I, J, K = np.meshgrid(idx, idx, idx, indexing="ij")
    verts = np.stack([I.ravel(order="F"), J.ravel(order="F"), K.ravel(order="F")], axis=1).astype(np.float64) * h
    if jitter > 0:
        rng = np.random.default_rng(seed)
        verts = verts + rng.uniform(-jitter, jitter, size=verts.shape) * h

    def vid(i, j, k):
        return (i % n) + n * ((j % n) + n * (k % n))

    hexes = np.zeros((n ** 3, 8), dtype=np.int64)
    e = 0
    for k in range(n):
        for j in range(n):
            for i in range(n):
                for c in range(8):
                    di, dj, dk = c & 1, (c >> 1) & 1, (c >> 2) & 1
                    hexes[e, c] = vid(i + di, j + dj, k + dk)
                e += 1
    return verts, hexes, np.array([L, L, L], dtype=np.float64)


# Cube faces of the cubed sphere: (normal axis, sign, first tangent axis, second tangent axis);
# each (t1, t2, outward normal) triple is right-handed.
_CUBE_FACES = [(0, +1, 1, 2), (0, -1, 2, 1), (1, +1, 2, 0), (1, -1, 0, 2), (2, +1, 0, 1), (2, -1, 1, 0)]


def _surface_lattice(nz: int):
    """Unique points of the cube surface lattice {-nz, -nz+2, ..., nz}^3 (max |coord| = nz)."""
    ids = -np.ones((nz + 1, nz + 1, nz + 1), dtype=np.int64)
    pts = []
    for a in range(nz + 1):
        for b in range(nz + 1):
            for c in range(nz + 1):
                if a in (0, nz) or b in (0, nz) or c in (0, nz):
                    ids[a, b, c] = len(pts)
                    pts.append((a, b, c))
    pts = np.array(pts, dtype=np.int64)
    # equiangular direction: on the patch x = +1 the point has y/x = tan(alpha), z/x = tan(beta),
    # alpha, beta = -pi/4 + i/nz * pi/2; the same tangent rule holds on every patch.
    lat = 2 * pts - nz  # in [-nz, nz]
    t = np.tan(lat * (math.pi / (4.0 * nz)))
    t[lat == nz] = 1.0
    t[lat == -nz] = -1.0
    d = t / np.linalg.norm(t, axis=1, keepdims=True)
    return ids, d


def shell_mesh(nz: int, nr: int, r_in: float = 0.70, r_out: float = 0.98) -> Tuple[np.ndarray, np.ndarray]:
    """Cubed-sphere shell of 6 * nz^2 * nr hexahedra between radii r_in and r_out.

    Radial layers are equally spaced in r.  Element order: patch, then the
    zonal index pair, then the radial layer (radial columns are contiguous).
    Returns (vertices [n_v, 3], hexes [6 nz^2 nr, 8]).
    """
    ids, dirs = _surface_lattice(nz)
    n_s = dirs.shape[0]
    radii = r_in + (r_out - r_in) * np.arange(nr + 1) / nr
    radii[-1] = r_out
    verts = (radii[:, None, None] * dirs[None, :, :]).reshape(-1, 3)
    blocks = []
    j, i, k = np.meshgrid(np.arange(nz), np.arange(nz), np.arange(nr), indexing="ij")
    j, i, k = j.ravel(), i.ravel(), k.ravel()  # element order within a patch: j, i, then k fastest
    for (ax, sg, t1, t2) in _CUBE_FACES:
        h = np.empty((j.size, 8), dtype=np.int64)
        for c in range(8):
            di, dj, dk = c & 1, (c >> 1) & 1, (c >> 2) & 1
            lat = [None, None, None]
            lat[ax] = np.full(j.size, nz if sg > 0 else 0)
            lat[t1] = i + di
            lat[t2] = j + dj
            h[:, c] = (k + dk) * n_s + ids[lat[0], lat[1], lat[2]]
        blocks.append(h)
    hexes = np.concatenate(blocks, axis=0)
    return verts, hexes


def _cube_rotations():
    """The 24 signed permutation matrices with determinant +1."""
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product((1, -1), repeat=3):
            R = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                R[r, perm[r]] = signs[r]
            if round(np.linalg.det(R)) == 1:
                out.append(R)
    return out


def reorient(hexes: np.ndarray, seed: int) -> np.ndarray:
    """Renumber each element's corners by a seeded proper rotation of its local frame.

    The element keeps its shape and right-handedness; only which corner is
    (0,0,0) and which directions are xi, eta, zeta change, so shared faces meet
    in every orientation a conforming hexahedral mesh allows.
    """
    rots = _cube_rotations()
    rng = np.random.default_rng(seed)
    choice = rng.integers(0, len(rots), size=hexes.shape[0])
    out = np.empty_like(hexes)
    for r, R in enumerate(rots):
        # new corner c (coordinates s in {-1,1}^3) takes the old corner at R s
        perm = np.zeros(8, dtype=np.int64)
        for c in range(8):
            s = np.array([2 * (c & 1) - 1, 2 * ((c >> 1) & 1) - 1, 2 * ((c >> 2) & 1) - 1])
            t = R @ s
            perm[c] = ((t[0] + 1) // 2) + 2 * ((t[1] + 1) // 2) + 4 * ((t[2] + 1) // 2)
        sel = choice == r
        out[sel] = hexes[sel][:, perm]
    return out


def random_state(n_e: int, N: int, seed: int = 0) -> np.ndarray:
    """Seeded conserved state (9, n_e, N^3) with positive density and pressure.

    rho in [0.8, 1.2], momentum in [-0.1, 0.1], B in [-0.3, 0.3], psi in
    [-0.02, 0.02] and E in [1.5, 2.5]: the kinetic, magnetic and psi energies
    are below 0.2, so the pressure stays positive for any gamma > 1.
    """
    rng = np.random.default_rng(seed)
    n3 = N ** 3
    q = np.empty((9, n_e, n3))
    q[0] = rng.uniform(0.8, 1.2, (n_e, n3))
    q[1:4] = rng.uniform(-0.1, 0.1, (3, n_e, n3))
    q[4] = rng.uniform(1.5, 2.5, (n_e, n3))
    q[5:8] = rng.uniform(-0.3, 0.3, (3, n_e, n3))
    q[8] = rng.uniform(-0.02, 0.02, (n_e, n3))
    return q


def n_elements_shell(nz: int, nr: int) -> int:
    return 6 * nz * nz * nr
