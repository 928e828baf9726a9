"""Checks of the synthetic input generators against the paper's mesh definitions."""
import os

import numpy as np

from paper_2502_17805_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_meshes.txt")


def _rows():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            yield [int(x) for x in line.split()]


def test_paper_mesh_counts():
    for nr, nz, order, cells, dof in _rows():
        assert inputs.n_elements_shell(nz, nr) == cells
        assert cells * order ** 3 == dof
    nr, nz, order, cells, dof = next(_rows())  # the mesh of the paper's figure is built in full
    v, h = inputs.shell_mesh(nz, nr)
    assert h.shape == (cells, 8)
    assert np.unique(h).size == v.shape[0]


def test_shell_elements_right_handed():
    v, h = inputs.shell_mesh(3, 2)
    X = v[h]  # [e][corner][3]
    a, b, c = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 4] - X[:, 0]
    assert np.all(np.einsum("ed,ed->e", a, np.cross(b, c)) > 0)
    rr = np.linalg.norm(X[:, 4] - X[:, 0], axis=1)
    assert np.all(rr > 0)


def test_reorient_preserves_elements_and_handedness():
    v, h = inputs.shell_mesh(2, 2)
    h2 = inputs.reorient(h, seed=9)
    assert np.array_equal(np.sort(h, axis=1), np.sort(h2, axis=1))
    X = v[h2]
    a, b, c = X[:, 1] - X[:, 0], X[:, 2] - X[:, 0], X[:, 4] - X[:, 0]
    assert np.all(np.einsum("ed,ed->e", a, np.cross(b, c)) > 0)


def test_box_mesh_periodic_ids():
    v, h, per = inputs.box_mesh(4)
    assert v.shape == (64, 3) and h.shape == (64, 8)
    assert h.max() == 63 and np.all(per == 1.0)


def test_random_state_positive_pressure():
    q = inputs.random_state(10, 4, seed=1)
    gam = 5.0 / 3.0
    p = (gam - 1) * (q[4] - 0.5 * (q[1:4] ** 2).sum(0) / q[0] - 0.5 * (q[5:8] ** 2).sum(0) - 0.5 * q[8] ** 2)
    assert p.min() > 0 and q[0].min() > 0
