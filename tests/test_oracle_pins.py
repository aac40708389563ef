"""Pins of the CPU oracle against results fixed by the paper and by
mathematics, independent of the oracle's own formulas.

* Casida plasmon formula (direct RPA, real Gamma-only): E_c = 1/2 sum_n
  (Omega_n - A_nn), Omega^2 = eig(Delta^(1/2) (Delta + 4K) Delta^(1/2)),
  A = Delta + 2K.
* direct MP2 (second order of the power series of Sec. 2.1, eq. 1):
  -(1/4pi) int Tr Pi^2 d omega = -2 zeta_k^2 sum_st |G_st|^2 / (Delta_s + Delta_t).
* single transition: closed-form frequency integral.
* Sylvester's determinant identity in the transition space (the metric
  independence of the appendix: det and trace do not depend on how V is
  factored).
* Hermitian, negative semidefinite chi0; eps <= 0; omega^-4 tail.
* V^(1/2) against the generator's closed form Q diag(sqrt lam) Q^H.
* determinants by permutation expansion on tiny matrices; pivoted LU.
* Gauss-Legendre frequency grid on integrals with closed forms.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

HERE = os.path.dirname(os.path.abspath(__file__))


def _rand_herm(n, rng, is_complex=True):
    a = rng.standard_normal((n, n)) + (1j * rng.standard_normal((n, n)) if is_complex else 0)
    return 0.5 * (a + a.conj().T)


def _small_problem(is_complex, n_aux=12, n_occ=3, n_virt=5, kdims=(2, 2, 1), n_w=8, seed=7, **kw):
    grid = synth.regular_kq_grid(kdims) if is_complex else synth.gamma_grid()
    return synth.make_problem("pin", is_complex=is_complex, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt, grid=grid,
                              n_w=n_w, seed=seed, **kw)


def _transition_data(p, q):
    """Stack the transitions s = (j, i, a) of all k-pairs of q: columns of C,
    their energies Delta_s, straight from the generator's arrays."""
    cols, deltas = [], []
    for j in range(p.n_k):
        eo, ev = p.eps_pair(q, j)
        cols.append(p.C(q, j))
        deltas.append((ev[None, :] - eo[:, None]).reshape(-1))
    return np.concatenate(cols, axis=1), np.concatenate(deltas)


# ----------------------------------------------------------------- Jacobi


@pytest.mark.parametrize("is_complex", [False, True])
def test_jacobi_against_numpy(is_complex):
    rng = np.random.default_rng(1)
    A = _rand_herm(23, rng, is_complex)
    lam, U, sweeps = oracle.jacobi_eigh(A)
    assert 0 < sweeps < 30
    ref = np.linalg.eigvalsh(A)
    assert np.allclose(np.sort(lam), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    assert np.allclose(U.conj().T @ U, np.eye(23), atol=1e-12)
    assert np.allclose(A @ U, U * lam[None, :], atol=1e-11)


@pytest.mark.parametrize("is_complex", [False, True])
def test_vhalf_closed_form(is_complex):
    p = _small_problem(is_complex, n_aux=40)
    q = 1 if is_complex else 0
    Qm, lam = p.V_eig(q)
    ref = (Qm * np.sqrt(lam)[None, :]) @ Qm.conj().T
    Vh = oracle.vhalf(p.V(q))
    assert np.abs(Vh - ref).max() < 1e-12 * np.abs(ref).max()
    assert np.abs(Vh - Vh.conj().T).max() < 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------- determinants


def _det_perm(M):
    n = M.shape[0]
    tot = 0j
    for perm in itertools.permutations(range(n)):
        sgn = 1
        for i in range(n):
            for j in range(i + 1, n):
                if perm[i] > perm[j]:
                    sgn = -sgn
        prod = 1 + 0j
        for i in range(n):
            prod *= M[i, perm[i]]
        tot += sgn * prod
    return tot


@pytest.mark.parametrize("n", [1, 2, 3, 4])
@pytest.mark.parametrize("is_complex", [False, True])
def test_logdet_bruteforce(n, is_complex):
    rng = np.random.default_rng(10 + n)
    B = rng.standard_normal((n, n + 2)) + (1j * rng.standard_normal((n, n + 2)) if is_complex else 0)
    Pi = -(B @ B.conj().T) * 0.7  # Pi <= 0, so 1 - Pi is positive definite
    ld, tr = oracle.logdet(Pi)
    M = np.eye(n) - Pi
    det = _det_perm(M)
    assert abs(det.imag) < 1e-12 * abs(det)
    assert ld == pytest.approx(math.log(det.real), rel=1e-13, abs=1e-14)
    assert tr == pytest.approx(np.trace(Pi).real, rel=1e-14)
    assert oracle.logabsdet_lu(M) == pytest.approx(math.log(abs(det)), rel=1e-13, abs=1e-14)


def test_logdet_not_pd_raises():
    Pi = np.diag([0.5, 2.0, 0.1])  # 1 - 2 < 0
    with pytest.raises(oracle.OracleError):
        oracle.logdet(Pi)


@pytest.mark.parametrize("is_complex", [False, True])
def test_logdet_vs_lu_medium(is_complex):
    rng = np.random.default_rng(3)
    n = 37
    B = rng.standard_normal((n, 50)) + (1j * rng.standard_normal((n, 50)) if is_complex else 0)
    Pi = -(B @ B.conj().T) / 20
    ld, _ = oracle.logdet(Pi)
    assert ld == pytest.approx(oracle.logabsdet_lu(np.eye(n) - Pi), rel=1e-12)
    sign, ref = np.linalg.slogdet(np.eye(n) - Pi)
    assert ld == pytest.approx(ref, rel=1e-12)


# -------------------------------------------------------- frequency grid


def test_frequency_grid_integrals():
    om, zw = synth.frequency_grid(32)
    assert np.all(om > 0) and np.all(zw > 0)
    for delta in (0.3, 1.0, 2.5):
        assert np.sum(zw / (delta ** 2 + om ** 2)) == pytest.approx(math.pi / (2 * delta), rel=1e-10)
    a, b = 0.4, 1.7
    assert np.sum(zw / ((a * a + om ** 2) * (b * b + om ** 2))) == pytest.approx(
        math.pi / (2 * a * b * (a + b)), rel=1e-10)


# ------------------------------------------------------------- dual grid


def test_dual_grid_counts_golden():
    g = json.load(open(os.path.join(HERE, "golden", "dual_grid_counts.json")))
    ex = g["worked_example"]
    grid = synth.dual_kq_grid(ex["q_reg"], ex["k_reg"], dim=ex["dim"], enhance=g["enhance_fraction"])
    assert grid.n_reg == ex["K_reg_size"]
    assert grid.kpts.shape[0] == ex["K_G_size"]
    n_add = g["added_points_per_dim"][str(ex["dim"])]
    assert int(grid.near_gamma.sum()) == n_add
    assert grid.pair_k.shape == (ex["q_reg"][0] * ex["q_reg"][1] - 1 + n_add, ex["K_reg_size"])
    assert grid.w_q.sum() == pytest.approx(1.0, abs=1e-14)
    for dim, cnt in g["added_points_per_dim"].items():
        d = int(dim)
        qd = [2] * d + [1] * (3 - d)
        gr = synth.dual_kq_grid(qd, [4] * d + [1] * (3 - d), dim=d)
        assert int(gr.near_gamma.sum()) == cnt
        assert gr.kpts.shape[0] == (cnt + 1) * gr.n_reg
        # near-Gamma points at +-d b_i with d = d_reg / 10
        near = gr.qpts[gr.near_gamma]
        assert np.allclose(np.abs(near[:, :d]), 0.1 / 2)
    # regular q keep k_j + q inside K_reg
    for iq in np.where(~grid.near_gamma)[0]:
        assert np.all(grid.pair_kq[iq] < grid.n_reg)


# ------------------------------------------------------------- invariants


@pytest.mark.parametrize("is_complex", [False, True])
def test_chi0_hermitian_negative(is_complex):
    p = _small_problem(is_complex, n_aux=20, n_occ=3, n_virt=7)
    q = p.n_q - 1
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    for om in (0.0, 0.7, 30.0):
        chi = oracle.chi0(C, eo, ev, p.grid.zeta_k, om)
        nrm = np.abs(chi).max()
        assert np.abs(chi - chi.conj().T).max() <= 1e-14 * nrm
        ev_chi = np.linalg.eigvalsh(0.5 * (chi + chi.conj().T))
        assert ev_chi.max() <= 1e-12 * nrm
        assert ev_chi.min() < 0


def test_eps_sign_and_tail():
    p = _small_problem(True, n_aux=16, n_occ=2, n_virt=6, kdims=(2, 1, 1))
    Vh = oracle.vhalf(p.V(1))
    C = [p.C(1, j) for j in range(p.n_k)]
    eo = [p.eps_pair(1, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(1, j)[1] for j in range(p.n_k)]
    vals = {}
    for om in (0.0, 1.0, 200.0, 400.0, 800.0):
        Pi = oracle.sandwich(Vh, oracle.chi0(C, eo, ev, p.grid.zeta_k, om))
        ld, tr = oracle.logdet(Pi)
        assert ld >= 0.0 and tr <= 0.0
        vals[om] = ld + tr
        assert vals[om] <= 0.0
    # eps ~ -1/2 Tr Pi^2 ~ omega^-4 at large omega
    r1 = vals[200.0] / vals[400.0]
    r2 = vals[400.0] / vals[800.0]
    assert r1 == pytest.approx(16.0, rel=2e-2)
    assert r2 == pytest.approx(16.0, rel=5e-3)


# ------------------------------------------------------- closed forms


def test_single_transition_closed_form():
    delta, c, v = 0.9, 0.8, 1.7
    K = c * v * c
    C = [np.array([[c]])]
    eo, ev = [np.array([-0.4])], [np.array([0.5])]
    Vh = oracle.vhalf(np.array([[v]]))
    # per frequency: eps(omega) = ln(1 + D K) - D K, D = 4 Delta / (Delta^2 + omega^2)
    for om in (0.0, 0.3, 5.0):
        Pi = oracle.sandwich(Vh, oracle.chi0(C, eo, ev, 1.0, om))
        ld, tr = oracle.logdet(Pi)
        D = 4 * delta / (delta ** 2 + om ** 2)
        assert ld + tr == pytest.approx(math.log1p(D * K) - D * K, rel=1e-13)
    # integrated: E = 1/2 (sqrt(Delta^2 + 4 Delta K) - Delta) - K
    om_all, zw = synth.frequency_grid(64)
    eps = np.zeros((1, len(om_all)))
    for w, om in enumerate(om_all):
        Pi = oracle.sandwich(Vh, oracle.chi0(C, eo, ev, 1.0, om))
        ld, tr = oracle.logdet(Pi)
        eps[0, w] = ld + tr
    Ec = oracle.energy_sum(np.ones(1), zw, eps)
    exact = 0.5 * (math.sqrt(delta ** 2 + 4 * delta * K) - delta) - K
    assert Ec == pytest.approx(exact, rel=1e-10)


def _casida(p):
    C, delta = _transition_data(p, 0)
    V = p.V(0)
    K = C.T @ V @ C
    sq = np.sqrt(delta)
    M = sq[:, None] * (np.diag(delta) + 4 * K) * sq[None, :]
    omega = np.sqrt(np.linalg.eigvalsh(M))
    return 0.5 * np.sum(omega) - 0.5 * np.sum(delta) - np.trace(K)


def test_casida_plasmon_formula():
    """Direct RPA at Gamma, real orbitals: the frequency integral of the
    oracle's integrand equals the plasmon formula; the quadrature error falls
    off exponentially with the number of Gauss-Legendre nodes."""
    base = synth.config0()
    exact = _casida(base)
    errs = []
    for n_w in (8, 16, 32, 64):
        p = synth.config0(n_w=n_w)
        Ec = oracle.energy(p)["Ec"]
        errs.append(abs(Ec - exact))
    assert errs[-1] < 1e-9 * abs(exact)
    assert errs[1] < errs[0] and errs[2] < errs[1]
    assert errs[2] < 1e-7 * abs(exact)


@pytest.mark.parametrize("is_complex", [False, True])
def test_direct_mp2(is_complex):
    """Second-order term of the power series: -(1/4pi) int Tr Pi^2 equals
    -2 zeta_k^2 sum_st |G_st|^2 / (Delta_s + Delta_t), G = C^T V conj(C);
    also eps(lambda V) -> -lambda^2/2 Tr Pi^2 for weak coupling."""
    p = _small_problem(is_complex, n_aux=14, n_occ=2, n_virt=5, n_w=48)
    q = p.n_q - 1
    C, delta = _transition_data(p, q)
    V = p.V(q)
    G = C.T @ V @ C.conj()
    zk = p.grid.zeta_k
    exact = -2 * zk * zk * np.sum(np.abs(G) ** 2 / (delta[:, None] + delta[None, :]))
    Vh = oracle.vhalf(V)
    Cb = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    tr2 = []
    for om in p.omega:
        Pi = oracle.sandwich(Vh, oracle.chi0(Cb, eo, ev, zk, om))
        tr2.append(np.sum(np.abs(Pi) ** 2))
    mp2 = -np.sum(p.zeta_w * np.array(tr2)) / (4 * math.pi)
    assert mp2 == pytest.approx(exact, rel=1e-10)
    # weak coupling: eps(lambda) / lambda^2 -> -1/2 Tr Pi^2
    lam = 1e-4
    Pi = oracle.sandwich(Vh * math.sqrt(lam), oracle.chi0(Cb, eo, ev, zk, p.omega[3]))
    ld, tr = oracle.logdet(Pi)
    assert (ld + tr) / (lam * lam) == pytest.approx(-0.5 * tr2[3], rel=1e-3)


@pytest.mark.parametrize("is_complex", [False, True])
def test_sylvester_transition_space(is_complex):
    """ln det(1 - V^(1/2) chi V^(1/2)) = ln det(1 + D^(1/2) G D^(1/2)) with
    D = zeta_k 4 Delta/(Delta^2 + omega^2) and G = C^T V conj(C) (n_trans x
    n_trans), per (q, omega); also Tr Pi = -sum_s D_s G_ss."""
    p = _small_problem(is_complex, n_aux=18, n_occ=2, n_virt=4, n_w=6)
    for q in range(p.n_q):
        C, delta = _transition_data(p, q)
        V = p.V(q)
        G = C.T @ V @ C.conj()
        Vh = oracle.vhalf(V)
        Cb = [p.C(q, j) for j in range(p.n_k)]
        eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
        ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
        for w in (0, 3, 5):
            om = p.omega[w]
            D = p.grid.zeta_k * 4 * delta / (delta ** 2 + om ** 2)
            sD = np.sqrt(D)
            M = np.eye(len(D)) + sD[:, None] * G * sD[None, :]
            sign, ref = np.linalg.slogdet(M)
            Pi = oracle.sandwich(Vh, oracle.chi0(Cb, eo, ev, p.grid.zeta_k, om))
            ld, tr = oracle.logdet(Pi)
            assert ld == pytest.approx(ref, rel=1e-12)
            assert tr == pytest.approx(-np.sum(D * np.diag(G).real), rel=1e-12)


def test_energy_sum_weights():
    """The q-sum is weighted by w_q and the frequency sum by zeta_w / 2pi:
    a separable table gives the product of the two one-dimensional sums."""
    wq = np.array([0.25, 0.5, 0.25])
    zw = np.array([0.1, 0.7, 1.3, 0.2])
    f = np.array([1.0, -2.0, 3.0])
    g = np.array([-0.5, 0.25, 2.0, 4.0])
    Ec = oracle.energy_sum(wq, zw, np.outer(f, g))
    assert Ec == pytest.approx(np.dot(wq, f) * np.dot(zw, g) / (2 * math.pi), rel=1e-15)
