"""Pins of the k/q grids and their weights (step A1) from mathematics, not
from the generator's own formulas.

* Regular n1 x n2 x n3 grid (q running over the k-grid, uniform weights): the
  weighted sum of f(q) = cos 2 pi (m . q) is the discrete orthogonality
  relation, 1 when m is a multiple of the grid in every direction and 0
  otherwise (exactly, to rounding).
* Dual grid of Sec. 2.5 (regular q-grid without Gamma plus the 2^dim points
  +-d b_i around it, d = d_reg/10): with the near-Gamma points sharing
  Gamma's weight (the reading of the weights), the weighted sum of the same
  smooth periodic f equals the regular-grid sum with f(Gamma) = 1 replaced by
  the mean of f over the displaced points, cos(2 pi m1 d1) cos(2 pi m2 d2),
  so it differs from the regular-grid quadrature by O(d^2):
  |diff| <= 2 pi^2 (m1^2 d1^2 + m2^2 d2^2) / |Q_reg|.  A wrong share (a
  point weighted 1/|Q_reg| instead of 1/(2^dim |Q_reg|), a dropped point)
  breaks the sum rule by O(1/|Q_reg|).
* Every pair (q, k_j, k_j + q) has kpts[pair_kq] = kpts[pair_k] + q modulo the
  reciprocal lattice, each q runs over every k_j of K_reg once, and K_reg is
  the regular k-grid.
"""
import itertools
import math

import numpy as np
import pytest

from paper_2505_06021_gb300 import synth


def _wrap(x):
    return x - np.floor(x + 0.5)


def _cos_sum(grid, m):
    return float(np.sum(grid.w_q * np.cos(2 * math.pi * (grid.qpts @ np.asarray(m, float)))))


@pytest.mark.parametrize("dims", [(4, 4, 1), (3, 2, 1), (5, 1, 1)])
def test_regular_grid_discrete_orthogonality(dims):
    g = synth.regular_kq_grid(dims)
    for m in itertools.product(range(-6, 7), range(-6, 7), range(0, 2)):
        expect = 1.0 if all(mi % di == 0 for mi, di in zip(m, dims)) else 0.0
        assert _cos_sum(g, m) == pytest.approx(expect, abs=1e-13), m


@pytest.mark.parametrize("q_dims,k_dims", [((3, 3, 1), (6, 6, 1)), ((2, 2, 1), (4, 4, 1)), ((4, 2, 1), (4, 4, 1))])
def test_dual_grid_weights_smooth_functions(q_dims, k_dims):
    g = synth.dual_kq_grid(q_dims, k_dims, dim=2)
    n_reg = q_dims[0] * q_dims[1]
    d = np.array([0.1 / q_dims[0], 0.1 / q_dims[1]])
    assert np.sum(g.w_q) == pytest.approx(1.0, abs=1e-15)
    assert np.all(g.w_q > 0)
    for m in itertools.product(range(0, 4), range(0, 4)):
        m3 = (m[0], m[1], 0)
        reg = 1.0 if (m[0] % q_dims[0] == 0 and m[1] % q_dims[1] == 0) else 0.0
        got = _cos_sum(g, m3)
        # exact closed form of the dual-grid sum under the weight reading
        closed = reg + (math.cos(2 * math.pi * m[0] * d[0]) * math.cos(2 * math.pi * m[1] * d[1]) - 1.0) / n_reg
        assert got == pytest.approx(closed, abs=1e-13), m
        # and the O(d^2) closeness to the regular-grid quadrature
        bound = 2 * math.pi ** 2 * (m[0] ** 2 * d[0] ** 2 + m[1] ** 2 * d[1] ** 2) / n_reg
        assert abs(got - reg) <= bound + 1e-14, m


@pytest.mark.parametrize("make", [lambda: synth.regular_kq_grid((4, 4, 1)),
                                  lambda: synth.dual_kq_grid((3, 3, 1), (6, 6, 1), dim=2)])
def test_pairs_are_k_and_k_plus_q(make):
    g = make()
    kreg = g.kpts[: g.n_reg]
    # K_reg is the regular grid
    n = int(round(math.sqrt(g.n_reg)))
    expect = {(round(_wrap(i / n) * n), round(_wrap(j / n) * n)) for i in range(n) for j in range(n)}
    got = {(round(x * n), round(y * n)) for x, y, _ in kreg}
    assert got == expect
    assert g.zeta_k == pytest.approx(1.0 / g.n_reg, rel=1e-15)
    for iq in range(g.qpts.shape[0]):
        assert sorted(g.pair_k[iq].tolist()) == list(range(g.n_reg))
        dk = _wrap(g.kpts[g.pair_kq[iq]] - g.kpts[g.pair_k[iq]] - g.qpts[iq])
        assert np.abs(dk).max() < 1e-12


def test_dual_grid_near_gamma_points():
    g = synth.dual_kq_grid((3, 3, 1), (6, 6, 1), dim=2)
    near = g.qpts[g.near_gamma]
    assert near.shape[0] == 4
    # the four sign combinations of +-d b1 +- d b2, d = (1/3)/10
    signs = {tuple(np.sign(p[:2]).astype(int)) for p in near}
    assert signs == {(1, 1), (1, -1), (-1, 1), (-1, -1)}
    assert np.allclose(np.abs(near[:, :2]), 1.0 / 30.0, atol=1e-15)
    assert np.allclose(g.w_q[g.near_gamma], 1.0 / 36.0, rtol=1e-15)
    assert np.allclose(g.w_q[~g.near_gamma], 1.0 / 9.0, rtol=1e-15)
