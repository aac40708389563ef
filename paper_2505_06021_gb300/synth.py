"""Seeded synthetic inputs for the periodic RPA hot path.

This module only *generates inputs*: band energies, density-fitting
coefficients C_{P,ia}(q,k), Coulomb matrices V(q), the dual k/q grids with
their weights, and the imaginary-frequency quadrature nodes.  It performs none
of the method's arithmetic (no chi0, no sandwich, no log-det, no energy sum),
so both the CPU oracle and the GPU library can consume the same arrays.

The shapes and value distributions stand in for the paper's h-BN, fluoro-
polyacetylene and CO/MgO workloads (Sec. 4), whose basis sets, fit sets and
orbitals are not available:

* band energies: occupied band centres ~ U[-1.0, -0.3] Ha, virtual centres
  ~ U[0.1, 2.0] Ha, plus a 2-D dispersion 0.05 Ha * (cos 2pi k1 + cos 2pi k2)/2
  on periodic grids (the same shift for every band, so the gap stays >= 0.4 Ha
  minus 0.1 Ha of total dispersion);
* fit coefficients: real N(0, 1/N_ov) at Gamma-only, complex Gaussian with the
  variance 1/N_ov split equally between real and imaginary parts otherwise;
* Coulomb matrices: V = Q diag(lam) Q^H with Q Haar-random (QR of a Gaussian
  matrix with the phase of R's diagonal divided out) and lam ~ logU[0.1, 10];
  on periodic grids the leading eigenvalue is scaled by (q_min/|q|)^2 for
  q != Gamma, mimicking the 1/|q|^2 growth of the Coulomb kernel near Gamma
  (Sec. 2.4 damping and Sec. 2.5 divergence discussion);
* frequency grid: n-point Gauss-Legendre on (-1, 1) mapped to [0, inf) by
  omega = omega0 (1+x)/(1-x), weight zeta = w * 2 omega0/(1-x)^2 (the paper's
  "modified Gauss-Legendre" grid, Sec. 4 computational details; the exact
  mapping is not printed, this one is a standard choice);
* dual grids (Sec. 2.5): a regular q-grid without Gamma plus 2^dim points at
  sum_i +-d b_i, d = d_reg/10, and K_G = K_reg U {k_j + q}.

Every random draw comes from a numpy PCG64 stream keyed by (seed, tag,
indices), so any single C(q,k) block or V(q) can be regenerated on its own
without producing the rest of the job.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

BASE_SEED = 20250506

# ----------------------------------------------------------------------------
# random streams
# ----------------------------------------------------------------------------

_TAGS = {"eps": 1, "C": 2, "V": 3, "batch": 4, "serve": 5, "padf": 6, "mo": 7, "padfR": 8, "ovl": 9}


def _rng(seed: int, tag: str, *idx: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), _TAGS[tag], *map(int, idx)])))


# ----------------------------------------------------------------------------
# frequency grid
# ----------------------------------------------------------------------------


def frequency_grid(n: int, omega0: float = 1.0) -> Tuple[np.ndarray, np.ndarray]:
    """n-point Gauss-Legendre rule mapped from (-1, 1) to [0, inf).

    omega_j = omega0 (1 + x_j)/(1 - x_j),  zeta_j = w_j 2 omega0/(1 - x_j)^2,
    so that sum_j zeta_j f(omega_j) approximates int_0^inf f(omega) d omega.
    """
    x, w = np.polynomial.legendre.leggauss(int(n))
    omega = omega0 * (1.0 + x) / (1.0 - x)
    zeta = w * 2.0 * omega0 / (1.0 - x) ** 2
    return omega.astype(np.float64), zeta.astype(np.float64)


# ----------------------------------------------------------------------------
# k / q grids (Sec. 2.5, dual grids)
# ----------------------------------------------------------------------------


def _wrap(x: np.ndarray) -> np.ndarray:
    """Fractional coordinates wrapped into [-1/2, 1/2)."""
    return x - np.floor(x + 0.5)


def regular_grid(dims: Sequence[int]) -> np.ndarray:
    """Regular Monkhorst-Pack-style grid including Gamma, fractional coords."""
    n1, n2, n3 = (list(dims) + [1, 1, 1])[:3]
    pts = [(i / n1, j / n2, l / n3) for i in range(n1) for j in range(n2) for l in range(n3)]
    return _wrap(np.array(pts, dtype=np.float64))


@dataclasses.dataclass
class KQGrid:
    """Explicit q-points, k-points and (q, k_j, k_j+q) pairs with weights."""

    kpts: np.ndarray  # [n_kpts, 3] fractional coordinates of K_G
    qpts: np.ndarray  # [n_q, 3]
    pair_k: np.ndarray  # [n_q, n_k] int32 index into kpts of k_j
    pair_kq: np.ndarray  # [n_q, n_k] int32 index into kpts of k_j + q
    w_q: np.ndarray  # [n_q] q weights, sum 1
    zeta_k: float  # 1/|K_reg|
    n_reg: int  # |K_reg|
    near_gamma: np.ndarray  # [n_q] bool, True for the added points around Gamma
    q_min: float  # smallest nonzero |q| of the regular q-grid


def _index_of(pts: List[np.ndarray], p: np.ndarray, tol: float = 1e-9) -> int:
    for i, x in enumerate(pts):
        if np.all(np.abs(_wrap(x - p)) < tol):
            return i
    pts.append(_wrap(p.copy()))
    return len(pts) - 1


def regular_kq_grid(dims: Sequence[int]) -> KQGrid:
    """Regular k-grid with q running over the same grid (Gamma included),
    uniform q weights 1/|Q| and zeta_k = 1/|K_reg|."""
    kreg = regular_grid(dims)
    pts = [k for k in kreg]
    nk = len(kreg)
    pair_k = np.zeros((nk, nk), np.int32)
    pair_kq = np.zeros((nk, nk), np.int32)
    for iq, q in enumerate(kreg):
        for j in range(nk):
            pair_k[iq, j] = j
            pair_kq[iq, j] = _index_of(pts, kreg[j] + q)
    assert len(pts) == nk
    norms = np.linalg.norm(kreg, axis=1)
    q_min = float(np.min(norms[norms > 1e-12])) if nk > 1 else 1.0
    return KQGrid(np.array(pts), kreg.copy(), pair_k, pair_kq, np.full(nk, 1.0 / nk), 1.0 / nk, nk,
                  np.zeros(nk, bool), q_min)


def dual_kq_grid(q_dims: Sequence[int], k_dims: Sequence[int], dim: int, enhance: float = 0.1) -> KQGrid:
    """Dual grid of Sec. 2.5.

    Q_G = (regular q-grid q_dims) \\ {Gamma}  U  {sum_i +-d b_i, i < dim}
    with d = enhance * d_reg (d_reg = 1/q_dims[i] in fractional units), and
    K_G = K_reg U {k_j + q : k_j in K_reg, q in Q_G}.

    Weights (not printed in the paper; see the design notes): every regular
    q != Gamma carries 1/|Q_reg|; the 2^dim points near Gamma share Gamma's
    weight 1/|Q_reg| equally; zeta_k = 1/|K_reg|.  The q-grid must be a
    sub-lattice of the k-grid so that k_j + q stays in K_reg for regular q.
    """
    qd = (list(q_dims) + [1, 1, 1])[:3]
    kd = (list(k_dims) + [1, 1, 1])[:3]
    for a, b in zip(qd, kd):
        if b % a != 0:
            raise ValueError("q-grid must be a sub-lattice of the k-grid")
    kreg = regular_grid(kd)
    qreg = regular_grid(qd)
    nq_reg = len(qreg)
    qs, w, near = [], [], []
    for q in qreg:
        if np.linalg.norm(q) < 1e-12:
            continue
        qs.append(q)
        w.append(1.0 / nq_reg)
        near.append(False)
    signs = np.array(np.meshgrid(*[[-1.0, 1.0]] * dim, indexing="ij")).reshape(dim, -1).T
    for s in signs:
        q = np.zeros(3)
        for i in range(dim):
            q[i] = s[i] * enhance / qd[i]
        qs.append(q)
        w.append(1.0 / nq_reg / len(signs))
        near.append(True)
    qpts = np.array(qs)
    pts = [k for k in kreg]
    nk = len(kreg)
    pair_k = np.zeros((len(qpts), nk), np.int32)
    pair_kq = np.zeros((len(qpts), nk), np.int32)
    for iq, q in enumerate(qpts):
        for j in range(nk):
            pair_k[iq, j] = j
            pair_kq[iq, j] = _index_of(pts, kreg[j] + q)
    norms = np.linalg.norm(qreg, axis=1)
    q_min = float(np.min(norms[norms > 1e-12]))
    return KQGrid(np.array(pts), qpts, pair_k, pair_kq, np.array(w), 1.0 / nk, nk, np.array(near), q_min)


def gamma_grid() -> KQGrid:
    z = np.zeros((1, 3))
    return KQGrid(z, z.copy(), np.zeros((1, 1), np.int32), np.zeros((1, 1), np.int32), np.ones(1), 1.0, 1,
                  np.zeros(1, bool), 1.0)


# ----------------------------------------------------------------------------
# problem description
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Problem:
    """One RPA energy job: shapes, grids, energies, frequencies; C and V are
    generated lazily per block from seeded streams."""

    name: str
    is_complex: bool
    n_aux: int
    n_occ: int
    n_virt: int
    grid: KQGrid
    eps_occ: np.ndarray  # [n_kpts, n_occ]
    eps_virt: np.ndarray  # [n_kpts, n_virt]
    omega: np.ndarray  # [n_w]
    zeta_w: np.ndarray  # [n_w]
    seed: int
    lam_lo: float = 0.1
    lam_hi: float = 10.0
    scale_lead: bool = True

    @property
    def n_q(self) -> int:
        return int(self.grid.pair_k.shape[0])

    @property
    def n_k(self) -> int:
        return int(self.grid.pair_k.shape[1])

    @property
    def n_w(self) -> int:
        return int(self.omega.shape[0])

    @property
    def n_ov(self) -> int:
        return self.n_occ * self.n_virt

    @property
    def dtype(self):
        return np.complex128 if self.is_complex else np.float64

    def C(self, q: int, j: int, out: Optional[np.ndarray] = None) -> np.ndarray:
        """Fit coefficients C_{P,ia}(q, k_j): [n_aux, n_occ*n_virt], row-major
        with the pair index t = i*n_virt + a contiguous.  `out` (optional, C
        contiguous, right shape and dtype) receives the block in place."""
        rng = _rng(self.seed, "C", q, j)
        shape = (self.n_aux, self.n_ov)
        if out is None:
            out = np.empty(shape, self.dtype)
        assert out.shape == shape and out.dtype == self.dtype and out.flags.c_contiguous
        v = out.view(np.float64)
        rng.standard_normal(out=v, dtype=np.float64)
        v *= math.sqrt(0.5 / self.n_ov) if self.is_complex else 1.0 / math.sqrt(self.n_ov)
        return out

    def V_eig(self, q: int) -> Tuple[np.ndarray, np.ndarray]:
        """(Q, lam) with V(q) = Q diag(lam) Q^H, Q Haar-random."""
        rng = _rng(self.seed, "V", q)
        n = self.n_aux
        if self.is_complex:
            z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
        else:
            z = rng.standard_normal((n, n))
        Qm, R = np.linalg.qr(z)
        d = np.diagonal(R)
        ph = d / np.abs(d)
        Qm = Qm * ph[None, :]
        lam = np.exp(rng.uniform(math.log(self.lam_lo), math.log(self.lam_hi), n))
        if self.scale_lead and self.n_q > 1:
            qn = float(np.linalg.norm(self.grid.qpts[q]))
            if qn > 1e-12:
                i = int(np.argmax(lam))
                lam[i] *= (self.grid.q_min / qn) ** 2
        return Qm.astype(self.dtype), lam

    def V(self, q: int) -> np.ndarray:
        Qm, lam = self.V_eig(q)
        V = (Qm * lam[None, :]) @ Qm.conj().T
        V = 0.5 * (V + V.conj().T)
        return np.ascontiguousarray(V.astype(self.dtype))

    def eps_pair(self, q: int, j: int) -> Tuple[np.ndarray, np.ndarray]:
        """(eps_occ at k_j, eps_virt at k_j + q)."""
        return self.eps_occ[self.grid.pair_k[q, j]], self.eps_virt[self.grid.pair_kq[q, j]]

    def chi0_flops(self) -> float:
        """Algorithmic FP64 flops of the chi0 build for the whole job, counting
        the Hermitian lower triangle: 4 N (N+1) N_ov per (q, k, omega) for complex
        data (8 flops per complex multiply-add), N (N+1) N_ov for real data."""
        per = (4.0 if self.is_complex else 1.0) * self.n_aux * (self.n_aux + 1) * self.n_ov
        return per * self.n_q * self.n_k * self.n_w

    def c_bytes(self) -> int:
        return self.n_aux * self.n_ov * (16 if self.is_complex else 8) * self.n_q * self.n_k


class AOProblem(Problem):
    """An RPA job given in the atomic-orbital form of Sec. 2.2 instead of by
    its MO-basis fit coefficients C_{P,ia}(q, k).

    Atoms A = 0..n_atoms-1 carry n_bas_atom[A] primary basis functions and
    n_fit_atom[A] fit functions, both numbered atom by atom (n_aux = sum of
    n_fit_atom).  Per k-point kappa of K_G the job holds

    * the k-dependent pair-atomic fit coefficients C_{nu mu alpha}(kappa) of
      the PADF expansion (alpha a fit function on the atom of mu), stored as
      ``padf(kappa)``: [n_bas, S] with S = sum_A n_bas_atom[A] n_fit_atom[A]
      and column s = pf_off[A] + (mu - bas_off[A]) n_fit_atom[A] + alpha_loc;
    * the MO coefficients c_{mu n}(kappa), ``mo(kappa)``: [n_bas, n_mo],
      n_mo = n_occ + n_virt, occupied columns first.

    Draws: PADF entries Gaussian (complex: variance split between the real
    and imaginary parts) with variance n_atoms / (2 N_ov), so that for
    orthonormal MOs the MO-basis coefficients have the variance 1/N_ov of
    ``Problem.C``; MO coefficients are the first n_mo columns of a Haar-random
    unitary (orthogonal when real).  The MO-basis coefficients themselves are
    a result of the method and are not generated here.

    Lattice form (``lattice`` given, [n_R, 3] integer vectors): the job holds
    the real cell-pair coefficients C^{0,dR} per lattice vector instead,
    ``padf_R(r)`` [n_bas, S] with variance shares decaying as e^{-|dR|}
    (summing to the k-form variance), and the k-dependent arrays are the
    method's lattice sums, not generated here.
    """

    def __init__(self, base: Problem, n_bas_atom: Sequence[int], n_fit_atom: Sequence[int],
                 lattice: Optional[np.ndarray] = None, eps_d: Optional[float] = None):
        super().__init__(**{f.name: getattr(base, f.name) for f in dataclasses.fields(Problem)})
        self.n_bas_atom = tuple(int(x) for x in n_bas_atom)
        self.n_fit_atom = tuple(int(x) for x in n_fit_atom)
        if len(self.n_bas_atom) != len(self.n_fit_atom) or sum(self.n_fit_atom) != self.n_aux:
            raise ValueError("fit functions per atom must sum to n_aux")
        if self.n_occ + self.n_virt > self.n_bas:
            raise ValueError("n_occ + n_virt exceeds the basis size")
        self.lattice = None if lattice is None else np.ascontiguousarray(lattice, np.int32).reshape(-1, 3)
        # periodic projector threshold (None: the MO coefficients are used as they are)
        self.eps_d = eps_d

    @property
    def n_atoms(self) -> int:
        return len(self.n_bas_atom)

    @property
    def n_bas(self) -> int:
        return sum(self.n_bas_atom)

    @property
    def n_mo(self) -> int:
        return self.n_occ + self.n_virt

    @property
    def n_pf(self) -> int:
        return sum(b * f for b, f in zip(self.n_bas_atom, self.n_fit_atom))

    @property
    def n_kpts(self) -> int:
        return int(self.grid.kpts.shape[0])

    def C(self, q: int, j: int, out: Optional[np.ndarray] = None) -> np.ndarray:
        raise TypeError("an AO job has no stored MO-basis fit coefficients")

    def padf(self, kappa: int) -> np.ndarray:
        if self.lattice is not None:
            raise TypeError("a lattice-form AO job holds cell-pair coefficients, not k-dependent ones")
        rng = _rng(self.seed, "padf", kappa)
        out = np.empty((self.n_bas, self.n_pf), self.dtype)
        v = out.view(np.float64)
        rng.standard_normal(out=v, dtype=np.float64)
        var = self.n_atoms / (2.0 * self.n_ov)
        v *= math.sqrt(0.5 * var) if self.is_complex else math.sqrt(var)
        return out

    def mo(self, kappa: int) -> np.ndarray:
        rng = _rng(self.seed, "mo", kappa)
        n = self.n_bas
        if self.is_complex:
            z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
        else:
            z = rng.standard_normal((n, n))
        Qm, R = np.linalg.qr(z)
        d = np.diagonal(R)
        Qm = Qm * (d / np.abs(d))[None, :]
        return np.ascontiguousarray(Qm[:, :self.n_mo].astype(self.dtype))

    def padf_R(self, r: int) -> np.ndarray:
        """Real cell-pair coefficients of lattice vector lattice[r]: [n_bas, S]."""
        rng = _rng(self.seed, "padfR", r)
        w = np.exp(-np.linalg.norm(self.lattice.astype(np.float64), axis=1))
        var = self.n_atoms / (2.0 * self.n_ov) * w[r] / w.sum()
        out = rng.standard_normal((self.n_bas, self.n_pf))
        out *= math.sqrt(var)
        return out

    def overlap(self, kappa: int, n_small_max: int = 3) -> Tuple[np.ndarray, int]:
        """Basis-set overlap S(kappa) = Q diag(lam) Q^H (Q Haar) with near-linear
        dependencies: lam ~ U[0.3, 3] except 0..n_small_max of them (seeded per
        k-point) ~ logU[1e-7, 1e-5].  Returns (S, number of small eigenvalues)."""
        rng = _rng(self.seed, "ovl", kappa)
        n = self.n_bas
        if self.is_complex:
            z = (rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))) / math.sqrt(2.0)
        else:
            z = rng.standard_normal((n, n))
        Qm, R = np.linalg.qr(z)
        Qm = Qm * (np.diagonal(R) / np.abs(np.diagonal(R)))[None, :]
        lam = rng.uniform(0.3, 3.0, n)
        n_small = int(rng.integers(0, n_small_max + 1))
        lam[:n_small] = np.exp(rng.uniform(math.log(1e-7), math.log(1e-5), n_small))
        S = (Qm * lam[None, :]) @ Qm.conj().T
        S = 0.5 * (S + S.conj().T)
        return np.ascontiguousarray(S.astype(self.dtype)), n_small

    def padf_bytes(self) -> int:
        if self.lattice is not None:
            return self.n_bas * self.n_pf * 8 * len(self.lattice)
        return self.n_bas * self.n_pf * (16 if self.is_complex else 8) * self.n_kpts


def lattice_2d(radius: int) -> np.ndarray:
    """In-plane lattice vectors (a, b, 0) with |a|, |b| <= radius."""
    return np.array([(a, b, 0) for a in range(-radius, radius + 1) for b in range(-radius, radius + 1)], np.int32)


def make_ao_problem(name: str, *, is_complex: bool, n_bas_atom: Sequence[int], n_fit_atom: Sequence[int],
                    n_occ: int, n_virt: int, grid: KQGrid, n_w: int, seed: int, lattice=None, eps_d=None,
                    **kw) -> AOProblem:
    base = make_problem(name, is_complex=is_complex, n_aux=int(sum(n_fit_atom)), n_occ=n_occ, n_virt=n_virt,
                        grid=grid, n_w=n_w, seed=seed, **kw)
    return AOProblem(base, n_bas_atom, n_fit_atom, lattice, eps_d)


def _bands(seed: int, grid: KQGrid, n_occ: int, n_virt: int, dispersion: float) -> Tuple[np.ndarray, np.ndarray]:
    rng = _rng(seed, "eps")
    occ_c = np.sort(rng.uniform(-1.0, -0.3, n_occ))
    virt_c = np.sort(rng.uniform(0.1, 2.0, n_virt))
    k = grid.kpts
    shift = dispersion * 0.5 * (np.cos(2 * np.pi * k[:, 0]) + np.cos(2 * np.pi * k[:, 1]))
    return (occ_c[None, :] + shift[:, None]).copy(), (virt_c[None, :] + shift[:, None]).copy()


def make_problem(name: str, *, is_complex: bool, n_aux: int, n_occ: int, n_virt: int, grid: KQGrid, n_w: int,
                 seed: int, dispersion: Optional[float] = None, omega0: float = 1.0,
                 scale_lead: bool = True) -> Problem:
    if dispersion is None:
        dispersion = 0.0 if grid.n_reg == 1 else 0.05
    eo, ev = _bands(seed, grid, n_occ, n_virt, dispersion)
    om, zw = frequency_grid(n_w, omega0)
    return Problem(name, is_complex, n_aux, n_occ, n_virt, grid, eo, ev, om, zw, seed, scale_lead=scale_lead)


# ----------------------------------------------------------------------------
# the five workloads and scaled-down variants of them
# ----------------------------------------------------------------------------


def config0(n_w: int = 16, seed: Optional[int] = None) -> Problem:
    """Gamma-only, real: N_aux=64, N_occ=4, N_virt=28, 16 frequencies."""
    return make_problem("gamma-real-N64", is_complex=False, n_aux=64, n_occ=4, n_virt=28, grid=gamma_grid(),
                        n_w=n_w, seed=BASE_SEED + 0 if seed is None else seed)


def config1(n_w: int = 20, seed: Optional[int] = None, n_aux: int = 512, n_occ: int = 32, n_virt: int = 224,
            kdims=(4, 4, 1)) -> Problem:
    """2-D periodic, complex: 4x4x1 k and q grids (16 q incl. Gamma, uniform
    weights), N_aux=512, N_occ=32, N_virt=224, 20 frequencies."""
    return make_problem("periodic2d-c128-N%d" % n_aux, is_complex=True, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                        grid=regular_kq_grid(kdims), n_w=n_w, seed=BASE_SEED + 1 if seed is None else seed)


def config1_ao(n_w: int = 20, seed: Optional[int] = None, n_bas_atom=(128, 128), n_fit_atom=(256, 256),
               n_occ: int = 32, n_virt: int = 224, kdims=(4, 4, 1), lattice_radius: Optional[int] = None) -> AOProblem:
    """The 2-D periodic workload in AO form: two atoms with 128 basis and 256
    fit functions each (N_bas = 256 = N_occ + N_virt, N_aux = 512), PADF and
    MO coefficients per k-point of the 4x4x1 grid, 20 frequencies."""
    return make_ao_problem("periodic2d-ao-N%d" % sum(n_fit_atom), is_complex=True, n_bas_atom=n_bas_atom,
                           n_fit_atom=n_fit_atom, n_occ=n_occ, n_virt=n_virt, grid=regular_kq_grid(kdims), n_w=n_w,
                           seed=BASE_SEED + 5 if seed is None else seed,
                           lattice=None if lattice_radius is None else lattice_2d(lattice_radius))


def config2(n_w: int = 16, seed: Optional[int] = None, n_aux: int = 768, n_occ: int = 32, n_virt: int = 480,
            q_dims=(3, 3, 1), k_dims=(6, 6, 1)) -> Problem:
    """Slab dual grid: coarse 3x3x1 q-grid without Gamma plus 4 near-Gamma
    points (d = d_reg/10), dense 6x6x1 K_reg; N_aux=768, N_occ=32,
    N_virt=480, 16 frequencies."""
    return make_problem("slab-dual-c128-N%d" % n_aux, is_complex=True, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                        grid=dual_kq_grid(q_dims, k_dims, dim=2), n_w=n_w,
                        seed=BASE_SEED + 2 if seed is None else seed)


def config3_instances(n_inst: int = 64, seed: Optional[int] = None, n_w: int = 16,
                      aux_range=(128, 1024), occ_range=(8, 64), ratio_range=(4, 15)) -> List[Problem]:
    """Batched uneven: independent Gamma-real or 2x2x1-complex instances with
    N_aux ~ U{128..1024}, N_occ ~ U{8..64}, N_virt = r N_occ, r ~ U{4..15}."""
    s0 = BASE_SEED + 3 if seed is None else seed
    rng = _rng(s0, "batch")
    out = []
    for i in range(n_inst):
        n_aux = int(rng.integers(aux_range[0], aux_range[1] + 1))
        n_occ = int(rng.integers(occ_range[0], occ_range[1] + 1))
        r = int(rng.integers(ratio_range[0], ratio_range[1] + 1))
        periodic = bool(rng.integers(0, 2))
        grid = regular_kq_grid((2, 2, 1)) if periodic else gamma_grid()
        out.append(make_problem("inst%02d" % i, is_complex=periodic, n_aux=n_aux, n_occ=n_occ, n_virt=r * n_occ,
                                grid=grid, n_w=n_w, seed=s0 * 1000 + i))
    return out


def serving_stream(n_jobs: int = 200, rate_per_s: float = 1.0, seed: Optional[int] = None,
                   mix=(0.5, 0.3, 0.2), scale: float = 1.0) -> List[Tuple[float, Problem]]:
    """Poisson arrivals of jobs drawn 50/30/20 from config-0 / config-1 /
    config-3-style sizes with k-grids n x n x 1, n ~ U{1..4}.  `scale` shrinks
    N_aux and N_ov for small test streams.  Returns (arrival_time_s, problem)."""
    s0 = BASE_SEED + 4 if seed is None else seed
    rng = _rng(s0, "serve")
    t = 0.0
    out = []
    for i in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        u = float(rng.uniform())
        kind = 0 if u < mix[0] else (1 if u < mix[0] + mix[1] else 2)
        n = int(rng.integers(1, 5))
        if kind == 0:
            n_aux, n_occ, n_virt, n = 64, 4, 28, 1
        elif kind == 1:
            n_aux, n_occ, n_virt = 512, 32, 224
        else:
            n_aux = int(rng.integers(128, 1025))
            n_occ = int(rng.integers(8, 65))
            n_virt = int(rng.integers(4, 16)) * n_occ
        if scale != 1.0:
            n_aux = max(8, int(n_aux * scale))
            n_occ = max(1, int(n_occ * math.sqrt(scale)))
            n_virt = max(1, int(n_virt * math.sqrt(scale)))
        grid = gamma_grid() if n == 1 else regular_kq_grid((n, n, 1))
        n_w = 16 if kind != 1 else 20
        out.append((t, make_problem("job%03d" % i, is_complex=(n > 1), n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                                    grid=grid, n_w=n_w, seed=s0 * 1000 + i)))
    return out
