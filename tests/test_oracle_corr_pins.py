"""Pins of the oracle's grid correction (CPU only): trilinear interpolation is
exact for linear fields and at nodes (textbook properties), and the grid built
from the distortion field undoes the field on true points pushed forward
through it (a forward evaluation, independent of the grid's inversion) to the
trilinear error bound h^2 |d''| / 8 ~ 0.03 cm."""
import math

import numpy as np
import pytest

import oracle
from paper_1910_12214_b300 import synth

TAN = math.tan(math.radians(10.0))


def _linear_grid(n=9):
    bounds = np.array([[80.0, 250.0, -1.2, 1.2, -10.0, 260.0]], np.float32)
    xs = np.linspace(80, 250, n)
    vs = np.linspace(-1.2, 1.2, n)
    zs = np.linspace(-10, 260, n)
    X, V, Z = np.meshgrid(xs, vs, zs, indexing="ij")
    g = np.zeros((1, n, n, n, 3), np.float32)
    g[0, ..., 1] = 0.25 + 0.01 * X - 0.5 * V + 0.002 * Z
    g[0, ..., 2] = -1.0 + 0.003 * X + 0.7 * V - 0.004 * Z
    return g, bounds


def test_trilinear_is_exact_for_linear_fields():
    g, b = _linear_grid()
    rng = np.random.default_rng(0)
    x = rng.uniform(85, 246, 500)
    v = rng.uniform(-1.0, 1.0, 500)
    z = rng.uniform(0, 250, 500)
    dy, dz = oracle.trilinear(g, b, np.zeros(500), x, v * x * TAN, z)
    assert np.max(np.abs(dy - (0.25 + 0.01 * x - 0.5 * v + 0.002 * z))) < 2e-6
    assert np.max(np.abs(dz - (-1.0 + 0.003 * x + 0.7 * v - 0.004 * z))) < 2e-6


def test_trilinear_reproduces_node_values_and_clamps():
    rng = np.random.default_rng(1)
    g = rng.normal(size=(2, 5, 6, 7, 3)).astype(np.float32)
    b = np.array([[80, 250, -1.2, 1.2, 0, 250], [70, 260, -1.3, 1.3, -250, 0]], np.float32)
    for s in (0, 1):
        for i, j, k in [(0, 0, 0), (4, 5, 6), (2, 3, 1), (1, 4, 5)]:
            x = b[s, 0] + i * (b[s, 1] - b[s, 0]) / 4
            v = b[s, 2] + j * (b[s, 3] - b[s, 2]) / 5
            z = b[s, 4] + k * (b[s, 5] - b[s, 4]) / 6
            dy, dz = oracle.trilinear(g, b, [s], [x], [v * x * TAN], [z])
            assert abs(dy[0] - g[s, i, j, k, 1]) < 1e-5 and abs(dz[0] - g[s, i, j, k, 2]) < 1e-5
    # beyond the last z node: the value of the clamped coordinate
    dy_far, _ = oracle.trilinear(g, b, [0], [150.0], [0.0], [1000.0])
    dy_edge, _ = oracle.trilinear(g, b, [0], [150.0], [0.0], [250.0])
    assert abs(dy_far[0] - dy_edge[0]) < 1e-12


@pytest.mark.slow
def test_grid_undoes_the_forward_distortion():
    d = synth.make_distortion(seed=2, n_sectors=1, single_sector=True)
    grid, bounds = synth.correction_grid(d)
    rng = np.random.default_rng(3)
    n = 4000
    x = rng.uniform(85, 246, n)
    y_true = rng.uniform(-0.95, 0.95, n) * x * TAN
    z_true = rng.uniform(-245, 245, n)
    dy, dz = d.field(0, x, y_true, z_true)  # forward: measured = true + d(true)
    ym, zm = y_true + dy, z_true + dz
    cy, cz = oracle.trilinear(grid, bounds, np.zeros(n), x, ym, zm)
    err = np.hypot(ym + cy - y_true, zm + cz - z_true)
    assert np.abs(dy).max() > 5.0  # the field is strong
    assert err.max() < 0.08 and np.median(err) < 0.01
