"""Pins of the oracle's periodic projector (Sec. 2.3): S(k) = U D U^H,
R(k) = Theta(D(k) - eps_d), R~ = prod_k R(k), T(k) = U R~ U^H, c~ = T c.

Each property below is fixed by the definition, independently of how the
oracle evaluates it (numpy's eigvalsh / eigh serve as the independent route):

* T(k) is a Hermitian projector of rank N - m that commutes with S(k);
* m (the zeros of R~) is the largest number of eigenvalues below eps_d over
  the k-points, since the eigenvalues are in ascending order;
* a k-point with fewer small eigenvalues still loses its m lowest
  eigen-directions (the product over k removes the same positions everywhere);
* eps_d below every eigenvalue leaves c unchanged; c inside the kept span is
  unchanged;
* diagonal overlaps give the closed-form diagonal T.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth


def _prob(is_complex=True):
    grid = synth.regular_kq_grid((2, 2, 1)) if is_complex else synth.gamma_grid()
    return synth.make_ao_problem("proj", is_complex=is_complex, n_bas_atom=(12, 14), n_fit_atom=(6, 4), n_occ=3,
                                 n_virt=9, grid=grid, n_w=4, seed=41)


@pytest.mark.parametrize("is_complex", [True, False])
def test_projector_is_a_hermitian_projector_commuting_with_S(is_complex):
    p = _prob(is_complex)
    S = [p.overlap(k)[0] for k in range(p.n_kpts)]
    c = [p.mo(k) for k in range(p.n_kpts)]
    eps_d = 1e-4
    out, m, Ts, lams = oracle.projector(S, eps_d, c)
    counts = [int(np.sum(np.linalg.eigvalsh(s) < eps_d)) for s in S]
    assert m == max(counts)
    for s, T, lam, ct, c0 in zip(S, Ts, lams, out, c):
        assert np.allclose(lam, np.linalg.eigvalsh(s), rtol=0, atol=1e-13)
        assert np.allclose(T, T.conj().T, atol=1e-14)
        assert np.allclose(T @ T, T, atol=1e-13)
        assert abs(np.real(np.trace(T)) - (p.n_bas - m)) < 1e-12
        assert np.allclose(T @ s, s @ T, atol=1e-12)
        assert np.allclose(ct, T @ c0, atol=1e-14)


def test_fewer_small_eigenvalues_still_lose_m_directions():
    n = 10
    rng = np.random.default_rng(3)
    Q0, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    Q1, _ = np.linalg.qr(rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n)))
    lam0 = np.concatenate([[1e-6, 3e-6], np.linspace(0.5, 2.0, n - 2)])
    lam1 = np.linspace(0.4, 2.5, n)  # nothing below eps_d here
    S0 = (Q0 * lam0) @ Q0.conj().T
    S1 = (Q1 * lam1) @ Q1.conj().T
    c = [np.eye(n, dtype=complex)[:, :4]] * 2
    out, m, Ts, _ = oracle.projector([S0, S1], 1e-4, c)
    assert m == 2
    w, U = np.linalg.eigh(S1)
    assert abs(np.real(np.trace(Ts[1])) - (n - 2)) < 1e-12
    assert np.allclose(Ts[1] @ U[:, :2], 0.0, atol=1e-12)  # its two lowest directions are removed
    assert np.allclose(Ts[1] @ U[:, 2:], U[:, 2:], atol=1e-12)


def test_threshold_below_spectrum_and_kept_span_leave_c_unchanged():
    p = _prob()
    S = [p.overlap(k)[0] for k in range(p.n_kpts)]
    c = [p.mo(k) for k in range(p.n_kpts)]
    out, m, _, _ = oracle.projector(S, 1e-9, c)
    assert m == 0
    for a, b in zip(out, c):
        assert np.allclose(a, b, atol=1e-14)
    # c inside the kept span
    out, m, Ts, _ = oracle.projector(S, 1e-4, c)
    kept = [T @ x for T, x in zip(Ts, c)]
    again, _, _, _ = oracle.projector(S, 1e-4, kept)
    for a, b in zip(again, kept):
        assert np.allclose(a, b, atol=1e-13)


def test_diagonal_overlaps_closed_form():
    d0 = np.array([0.9, 2e-6, 1.4, 0.3, 5e-7, 2.2])
    d1 = np.array([3e-6, 1.1, 0.7, 1.9, 0.5, 2.5])
    c = [np.eye(6)] * 2
    out, m, Ts, _ = oracle.projector([np.diag(d0), np.diag(d1)], 1e-4, c)
    assert m == 2
    # positions 0, 1 of the ascending order are removed at both k-points
    keep0 = np.ones(6)
    keep0[np.argsort(d0)[:2]] = 0.0
    keep1 = np.ones(6)
    keep1[np.argsort(d1)[:2]] = 0.0
    assert np.allclose(Ts[0], np.diag(keep0), atol=1e-15)
    assert np.allclose(Ts[1], np.diag(keep1), atol=1e-15)
