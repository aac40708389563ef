"""Pins of the oracle's AO -> MO transform of the fit coefficients (Sec. 2.2:
PADF products in reciprocal space, k-dependent coefficients, KS states).

The oracle writes C_{gamma,ia}(q,k) = sum_{mu nu} conj(c_{mu i}(k)) c_{nu a}(k+q)
B^{mu nu}_gamma with B from the PADF arrays at k and k+q.  Each test below
fixes a property that a plausible slip (a dropped term, a conjugate on the
wrong factor, a swapped k-point, wrong atom offsets, wrong MO columns) breaks:

* identity MOs reduce the transform to a lookup of B's two PADF terms;
* diagonal phase MOs multiply each entry by e^{-i theta_i(k)} e^{i phi_a(k+q)};
* swapping the roles of (k, occupied) and (k+q, virtual) conjugates every
  entry (the two PADF terms map onto each other);
* a fit function's coefficients depend only on its own atom's PADF block;
* chi0 built from the transformed coefficients equals chi0 from the AO-space
  pair response contracted with B on both sides (another summation order).
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth


def _prob(is_complex=True, nb=(5, 7), nf=(6, 4), n_occ=3, n_virt=8, dims=(2, 1, 1), seed=11):
    return synth.make_ao_problem("pin", is_complex=is_complex, n_bas_atom=nb, n_fit_atom=nf, n_occ=n_occ,
                                 n_virt=n_virt, grid=synth.regular_kq_grid(dims) if dims else synth.gamma_grid(),
                                 n_w=4, seed=seed)


def _dense_B(p, Pk, Pkq):
    """B[gamma, mu, nu] from the two PADF terms, atom block by atom block."""
    nb, nf = p.n_bas_atom, p.n_fit_atom
    B = np.zeros((p.n_aux, p.n_bas, p.n_bas), np.complex128)
    b0 = np.cumsum((0,) + nb)
    f0 = np.cumsum((0,) + nf)
    s0 = np.cumsum((0,) + tuple(x * y for x, y in zip(nb, nf)))
    for A in range(p.n_atoms):
        for ml in range(nb[A]):
            for gl in range(nf[A]):
                s = s0[A] + ml * nf[A] + gl
                g = f0[A] + gl
                m = b0[A] + ml
                B[g, m, :] += Pkq[:, s]  # gamma and mu on A: C_{nu mu gamma}(k+q)
                B[g, :, m] += np.conj(Pk[:, s])  # gamma and nu on A: conj(C_{mu nu gamma}(k))
    return B


@pytest.mark.parametrize("is_complex", [True, False])
def test_identity_mos_read_the_padf_terms(is_complex):
    p = _prob(is_complex=is_complex, nb=(4, 6), nf=(5, 3), n_occ=4, n_virt=6, dims=(2, 1, 1) if is_complex else None)
    q, j = (1, 0) if is_complex else (0, 0)
    k, kq = p.grid.pair_k[q, j], p.grid.pair_kq[q, j]
    Pk, Pkq = p.padf(k), p.padf(kq)
    eye = np.eye(p.n_bas, dtype=p.dtype)
    C = oracle.ao2mo(is_complex, p.n_bas_atom, p.n_fit_atom, p.n_occ, p.n_virt, Pk, Pkq, eye, eye)
    B = _dense_B(p, Pk, Pkq)
    expect = B[:, :p.n_occ, p.n_occ:p.n_occ + p.n_virt].reshape(p.n_aux, -1)
    assert np.array_equal(C, expect if is_complex else expect.real)


def test_phase_mos_multiply_entries():
    p = _prob()
    q, j = 1, 1
    k, kq = p.grid.pair_k[q, j], p.grid.pair_kq[q, j]
    Pk, Pkq = p.padf(k), p.padf(kq)
    rng = np.random.default_rng(5)
    th = rng.uniform(-np.pi, np.pi, p.n_bas)
    ph = rng.uniform(-np.pi, np.pi, p.n_bas)
    eye = np.eye(p.n_bas, dtype=np.complex128)
    C0 = oracle.ao2mo(True, p.n_bas_atom, p.n_fit_atom, p.n_occ, p.n_virt, Pk, Pkq, eye, eye)
    C1 = oracle.ao2mo(True, p.n_bas_atom, p.n_fit_atom, p.n_occ, p.n_virt, Pk, Pkq, np.diag(np.exp(1j * th)),
                      np.diag(np.exp(1j * ph)))
    f = np.exp(-1j * th[:p.n_occ])[:, None] * np.exp(1j * ph[p.n_occ:p.n_occ + p.n_virt])[None, :]
    assert np.allclose(C1, C0 * f.reshape(1, -1), rtol=0, atol=1e-15)


def test_role_swap_conjugates():
    p = _prob(nb=(6, 3, 5), nf=(4, 5, 3), n_occ=3, n_virt=9)
    q, j = 1, 0
    k, kq = p.grid.pair_k[q, j], p.grid.pair_kq[q, j]
    Pk, Pkq, ck, ckq = p.padf(k), p.padf(kq), p.mo(k), p.mo(kq)
    no, nv = p.n_occ, p.n_virt
    C = oracle.ao2mo(True, p.n_bas_atom, p.n_fit_atom, no, nv, Pk, Pkq, ck, ckq)
    # k-side: (k+q) with its virtual states as the "occupied" set; k+q-side: k
    # with its occupied states as the "virtual" set
    side_a = np.ascontiguousarray(np.concatenate([ckq[:, no:no + nv], np.zeros((p.n_bas, no))], axis=1))
    side_b = np.ascontiguousarray(np.concatenate([np.zeros((p.n_bas, nv)), ck[:, :no]], axis=1))
    Cs = oracle.ao2mo(True, p.n_bas_atom, p.n_fit_atom, nv, no, Pkq, Pk, side_a, side_b)
    swapped = Cs.reshape(p.n_aux, nv, no).transpose(0, 2, 1).reshape(p.n_aux, -1)
    assert np.allclose(swapped, np.conj(C), rtol=0, atol=1e-14)


def test_fit_rows_depend_on_own_atom_block_only():
    p = _prob(nb=(5, 4, 6), nf=(3, 6, 4))
    q, j = 1, 1
    k, kq = p.grid.pair_k[q, j], p.grid.pair_kq[q, j]
    Pk, Pkq, ck, ckq = p.padf(k), p.padf(kq), p.mo(k), p.mo(kq)
    args = (True, p.n_bas_atom, p.n_fit_atom, p.n_occ, p.n_virt)
    C = oracle.ao2mo(*args, Pk, Pkq, ck, ckq)
    s0 = np.cumsum((0,) + tuple(x * y for x, y in zip(p.n_bas_atom, p.n_fit_atom)))
    f0 = np.cumsum((0,) + p.n_fit_atom)
    for A in range(p.n_atoms):
        Pk2, Pkq2 = Pk.copy(), Pkq.copy()
        Pk2[:, s0[A]:s0[A + 1]] *= 1.7
        Pkq2[:, s0[A]:s0[A + 1]] += 0.3
        C2 = oracle.ao2mo(*args, Pk2, Pkq2, ck, ckq)
        own = slice(f0[A], f0[A + 1])
        other = np.ones(p.n_aux, bool)
        other[own] = False
        assert np.array_equal(C2[other], C[other])
        assert np.min(np.abs(C2[own] - C[own]).max(axis=1)) > 1e-3


@pytest.mark.parametrize("is_complex", [True, False])
def test_chi0_matches_ao_space_pair_response(is_complex):
    p = _prob(is_complex=is_complex, nb=(4, 5), nf=(5, 4), n_occ=2, n_virt=5, dims=(2, 1, 1) if is_complex else None)
    q, w = (1, 2) if is_complex else (0, 2)
    om = float(p.omega[w])
    blocks = [oracle.ao2mo_block(p, q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    chi = oracle.chi0(blocks, eo, ev, p.grid.zeta_k, om)
    ref = np.zeros((p.n_aux, p.n_aux), np.complex128)
    for j in range(p.n_k):
        k, kq = p.grid.pair_k[q, j], p.grid.pair_kq[q, j]
        B = _dense_B(p, p.padf(k), p.padf(kq))
        co = p.mo(k)[:, :p.n_occ]
        cv = p.mo(kq)[:, p.n_occ:p.n_occ + p.n_virt]
        delta = ev[j][None, :] - eo[j][:, None]  # [i, a]
        d = -4.0 * delta / (delta ** 2 + om ** 2)
        # R[mu, nu, mu', nu'] = sum_ia d_ia c_mu,i conj(c_nu,a) conj(c_mu',i) c_nu',a
        R = np.einsum("ia,mi,na,pi,ra->mnpr", d, co, np.conj(cv), np.conj(co), cv)
        ref += p.grid.zeta_k * np.einsum("gmn,mnpr,hpr->gh", np.conj(B), R, B)
    scale = np.abs(ref).max()
    assert np.abs(chi - (ref if is_complex else ref.real)).max() <= 1e-13 * scale


# ---- k-dependent PADF coefficients: C(k) = sum_dR C^{0,dR} e^{i k.dR} ----

def test_padf_k_is_an_inverse_dft_on_the_supercell():
    """On a regular n1 x n2 k-grid with the lattice vectors of one n1 x n2
    supercell the lattice sum is n1 n2 times numpy's inverse 2-D DFT."""
    n1, n2, ne = 3, 4, 7
    rng = np.random.default_rng(21)
    C0 = rng.standard_normal((n1, n2, ne))
    R = np.array([(a, b, 0) for a in range(n1) for b in range(n2)])
    ref = n1 * n2 * np.fft.ifft2(C0, axes=(0, 1))
    for a in range(n1):
        for b in range(n2):
            got = oracle.padf_k([C0[x, y] for x in range(n1) for y in range(n2)], R, (a / n1, b / n2, 0.0))
            assert np.allclose(got, ref[a, b], rtol=0, atol=1e-14)


def test_padf_k_conjugate_at_minus_k_and_gamma_sum():
    rng = np.random.default_rng(22)
    R = synth.lattice_2d(2)
    C0 = [rng.standard_normal(11) for _ in range(len(R))]
    kf = (0.137, -0.291, 0.0)
    a = oracle.padf_k(C0, R, kf)
    b = oracle.padf_k(C0, R, tuple(-x for x in kf))
    assert np.allclose(b, np.conj(a), rtol=0, atol=1e-15)
    g = oracle.padf_k(C0, R, (0.0, 0.0, 0.0))
    assert np.allclose(g.real, np.sum(C0, axis=0), rtol=0, atol=1e-14) and np.all(g.imag == 0.0)


def test_padf_k_lattice_shift_is_a_phase():
    rng = np.random.default_rng(23)
    R = synth.lattice_2d(1)
    C0 = [rng.standard_normal(5) for _ in range(len(R))]
    kf = (0.25, 0.4, 0.0)
    n0 = np.array([2, -1, 0])
    a = oracle.padf_k(C0, R, kf)
    b = oracle.padf_k(C0, R + n0[None, :], kf)
    assert np.allclose(b, a * np.exp(2j * np.pi * np.dot(kf, n0)), rtol=0, atol=1e-14)
