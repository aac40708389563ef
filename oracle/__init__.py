"""ctypes front-end of the plain FP64 CPU oracle (``rpa_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` use it.  The GPU library never imports, links
or calls anything here, and nothing here imports the GPU library.

Each function restates one step of the paper's method (arXiv 2505.06021):

* :func:`projector` - periodic projector T(k) and regularised MO coefficients, Sec. 2.3
* :func:`padf_k`    - k-dependent PADF coefficients from the cell-pair ones, Sec. 2.2
* :func:`ao2mo`     - MO-basis fit coefficients C_{gamma,ia}(q, k) from the
                      k-dependent PADF and MO coefficients, Sec. 2.2
* :func:`chi0`      - fit-basis response chi0_PQ(q, i omega), Sec. 2.2
* :func:`vhalf`     - V(q)^(1/2) by Hermitian Jacobi, Sec. 2.1 / Algorithm 1
* :func:`sandwich`  - Pi = V^(1/2) chi0 V^(1/2), Sec. 2.1 / Algorithm 1
* :func:`logdet`    - ln det(1 - Pi) (Cholesky) and Tr Pi, Algorithm 1
* :func:`logabsdet_lu` - cross-check of ln|det| by pivoted LU
* :func:`energy_sum`   - E_c = (1/2pi) sum_w zeta_w sum_q w_q eps_qw, Sec. 2.6
* :func:`energy`    - the whole job, composed from the above
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Dict, Optional, Sequence, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rpa_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, IEEE semantics, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", _SRC, "-o", _LIB + ".tmp",
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        i, d = ctypes.c_int, ctypes.c_double
        lib.oracle_chi0.argtypes = [i, i, i, i, i, ctypes.POINTER(_dp), ctypes.POINTER(_dp), ctypes.POINTER(_dp), d,
                                    d, _dp, i]
        lib.oracle_jacobi_eigh.argtypes = [i, i, _dp, _dp, _dp, i, d]
        ip = ctypes.POINTER(ctypes.c_int)
        lib.oracle_ao2mo.argtypes = [i, i, ip, ip, i, i, i, _dp, _dp, _dp, _dp, i, ip, _dp, i]
        lib.oracle_padf_k.argtypes = [i, ip, ctypes.POINTER(_dp), ctypes.c_long, _dp, _dp, i]
        lib.oracle_vhalf.argtypes = [i, i, _dp, _dp]
        lib.oracle_sandwich.argtypes = [i, i, _dp, _dp, _dp, i]
        lib.oracle_logdet_cholesky.argtypes = [i, i, _dp, _dp, _dp]
        lib.oracle_logabsdet_lu.argtypes = [i, i, _dp, _dp]
        lib.oracle_energy_sum.argtypes = [i, i, _dp, _dp, _dp, _dp]
        lib.oracle_max_threads.argtypes = []
        for f in (lib.oracle_chi0, lib.oracle_ao2mo, lib.oracle_padf_k, lib.oracle_jacobi_eigh, lib.oracle_vhalf,
                  lib.oracle_sandwich, lib.oracle_logdet_cholesky, lib.oracle_logabsdet_lu, lib.oracle_energy_sum,
                  lib.oracle_max_threads):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def _f64(a: np.ndarray, is_complex: bool) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.complex128 if is_complex else np.float64)
    return a


def chi0(C_blocks: Sequence[np.ndarray], eps_occ: Sequence[np.ndarray], eps_virt: Sequence[np.ndarray], zeta_k: float,
         omega: float, n_threads: Optional[int] = None) -> np.ndarray:
    """chi0_PQ at one q and one frequency from the n_k blocks C_j = C(q, k_j)
    ([n_aux, n_occ*n_virt]), eps_occ[j] at k_j and eps_virt[j] at k_j + q."""
    is_c = bool(np.iscomplexobj(C_blocks[0]))
    Cs = [_f64(c, is_c) for c in C_blocks]
    eo = [np.ascontiguousarray(e, np.float64) for e in eps_occ]
    ev = [np.ascontiguousarray(e, np.float64) for e in eps_virt]
    n_aux, n_ov = Cs[0].shape
    n_occ, n_virt = eo[0].shape[0], ev[0].shape[0]
    if n_occ * n_virt != n_ov:
        raise ValueError("C width must be n_occ * n_virt")
    out = np.zeros((n_aux, n_aux), np.complex128 if is_c else np.float64)
    cp = (_dp * len(Cs))(*[_ptr(c.view(np.float64)) for c in Cs])
    op = (_dp * len(eo))(*[_ptr(e) for e in eo])
    vp = (_dp * len(ev))(*[_ptr(e) for e in ev])
    rc = _load().oracle_chi0(int(is_c), n_aux, n_occ, n_virt, len(Cs), cp, op, vp, float(zeta_k), float(omega),
                             _ptr(out.view(np.float64)), int(n_threads or max_threads()))
    if rc != 0:
        raise OracleError("oracle_chi0 rc=%d" % rc)
    return out


def ao2mo(is_complex: bool, n_bas_atom: Sequence[int], n_fit_atom: Sequence[int], n_occ: int, n_virt: int,
          padf_k: np.ndarray, padf_kq: np.ndarray, mo_k: np.ndarray, mo_kq: np.ndarray,
          entries: Optional[np.ndarray] = None, n_threads: Optional[int] = None) -> np.ndarray:
    """MO-basis fit coefficients of one (q, k) pair from the PADF arrays at k
    and k+q and the MO coefficients at k (occupied side) and k+q (virtual
    side).  Returns [n_aux, n_occ*n_virt], or, with entries ([n, 2] int
    (gamma, t) rows), the n selected values."""
    nb = np.ascontiguousarray(n_bas_atom, np.int32)
    nf = np.ascontiguousarray(n_fit_atom, np.int32)
    arrs = [_f64(a, is_complex) for a in (padf_k, padf_kq, mo_k, mo_kq)]
    n_mo = arrs[2].shape[1]
    n_aux = int(nf.sum())
    ip = ctypes.POINTER(ctypes.c_int)
    if entries is None:
        out = np.zeros((n_aux, n_occ * n_virt), np.complex128 if is_complex else np.float64)
        ne, ep = 0, ctypes.cast(None, ip)
    else:
        entries = np.ascontiguousarray(entries, np.int32).reshape(-1, 2)
        out = np.zeros(entries.shape[0], np.complex128 if is_complex else np.float64)
        ne, ep = entries.shape[0], entries.ctypes.data_as(ip)
    rc = _load().oracle_ao2mo(int(is_complex), len(nb), nb.ctypes.data_as(ip), nf.ctypes.data_as(ip), int(n_occ),
                              int(n_virt), int(n_mo), *[_ptr(a.view(np.float64)) for a in arrs], ne, ep,
                              _ptr(out.view(np.float64)), int(n_threads or max_threads()))
    if rc != 0:
        raise OracleError("oracle_ao2mo rc=%d" % rc)
    return out


def padf_k(C0: Sequence[np.ndarray], R: np.ndarray, kfrac: Sequence[float],
           n_threads: Optional[int] = None) -> np.ndarray:
    """C(k) = sum_r C0[r] e^{2 pi i kfrac . R[r]} for real arrays C0[r] of one
    shape and integer lattice vectors R ([n_R, 3]); complex result."""
    arrs = [np.ascontiguousarray(a, np.float64) for a in C0]
    Ri = np.ascontiguousarray(R, np.int32).reshape(-1, 3)
    kf = np.ascontiguousarray(kfrac, np.float64).reshape(3)
    out = np.zeros(arrs[0].shape, np.complex128)
    ip = ctypes.POINTER(ctypes.c_int)
    pp = (_dp * len(arrs))(*[_ptr(a) for a in arrs])
    rc = _load().oracle_padf_k(len(arrs), Ri.ctypes.data_as(ip), pp, int(arrs[0].size), _ptr(kf),
                               _ptr(out.view(np.float64)), int(n_threads or max_threads()))
    if rc != 0:
        raise OracleError("oracle_padf_k rc=%d" % rc)
    return out


def padf_of(problem, kappa: int, n_threads: Optional[int] = None) -> np.ndarray:
    """The k-dependent PADF array of k-point kappa of an AO-form problem: given
    directly, or (lattice form) formed from the cell-pair coefficients."""
    if getattr(problem, "lattice", None) is None:
        return problem.padf(kappa)
    C = padf_k([problem.padf_R(r) for r in range(len(problem.lattice))], problem.lattice,
               problem.grid.kpts[kappa], n_threads)
    return C if problem.is_complex else np.ascontiguousarray(C.real)


_proj_cache: Dict[tuple, list] = {}


def mo_of(problem, kappa: int) -> np.ndarray:
    """MO coefficients of k-point kappa as the transform uses them: the
    problem's own, or (eps_d set) the periodic projector's c~."""
    if getattr(problem, "eps_d", None) is None:
        return problem.mo(kappa)
    key = (id(problem), problem.seed, problem.eps_d, problem.n_bas, problem.n_mo, problem.n_kpts)
    if key not in _proj_cache:
        S = [problem.overlap(k)[0] for k in range(problem.n_kpts)]
        _proj_cache.clear()
        _proj_cache[key] = projector(S, problem.eps_d, [problem.mo(k) for k in range(problem.n_kpts)])[0]
    return _proj_cache[key][kappa]


def ao2mo_block(problem, q: int, j: int, entries: Optional[np.ndarray] = None,
                n_threads: Optional[int] = None) -> np.ndarray:
    """C(q, k_j) of an AO-form problem (``synth.AOProblem``)."""
    k, kq = int(problem.grid.pair_k[q, j]), int(problem.grid.pair_kq[q, j])
    return ao2mo(problem.is_complex, problem.n_bas_atom, problem.n_fit_atom, problem.n_occ, problem.n_virt,
                 padf_of(problem, k, n_threads), padf_of(problem, kq, n_threads), mo_of(problem, k),
                 mo_of(problem, kq), entries, n_threads)


def _blocks(problem, q: int, n_threads: Optional[int] = None):
    if hasattr(problem, "padf"):
        return [ao2mo_block(problem, q, j, n_threads=n_threads) for j in range(problem.n_k)]
    return [problem.C(q, j) for j in range(problem.n_k)]


def jacobi_eigh(A: np.ndarray, max_sweeps: int = 100, tol: float = 1e-14) -> Tuple[np.ndarray, np.ndarray, int]:
    is_c = bool(np.iscomplexobj(A))
    A = _f64(A, is_c)
    n = A.shape[0]
    lam = np.zeros(n)
    U = np.zeros_like(A)
    rc = _load().oracle_jacobi_eigh(int(is_c), n, _ptr(A.view(np.float64)), _ptr(lam), _ptr(U.view(np.float64)),
                                    max_sweeps, tol)
    if rc < 0:
        raise OracleError("jacobi rc=%d" % rc)
    return lam, U, rc


def projector(S_list: Sequence[np.ndarray], eps_d: float, c_list: Sequence[np.ndarray]):
    """Periodic projector method (Sec. 2.3), step by step:

    1. S(k) = U(k) D(k) U(k)^H by the Jacobi eigendecomposition, eigenvalues in
       ascending order (the order a Hermitian eigensolver reports);
    2. R(k)_ii = Theta(D_ii(k) - eps_d), with Theta(0) = 1;
    3. R~ = prod_k R(k) (diagonal matrices, so element by element);
    4. T(k) = U(k) R~ U(k)^H;
    5. c~(k) = T(k) c(k).

    Returns (the list of c~(k), the number of diagonal zeros of R~, the list
    of T(k), the sorted eigenvalues per k)."""
    eigs = []
    for S in S_list:
        lam, U, _ = jacobi_eigh(S)
        order = np.argsort(lam, kind="stable")
        eigs.append((lam[order], U[:, order]))
    Rt = np.ones(len(eigs[0][0]))
    for lam, _ in eigs:
        Rt = Rt * (lam - eps_d >= 0.0).astype(np.float64)
    Ts, out = [], []
    for (lam, U), c in zip(eigs, c_list):
        T = (U * Rt[None, :]) @ U.conj().T
        Ts.append(T)
        out.append(T @ c)
    return out, int(np.sum(Rt == 0.0)), Ts, [lam for lam, _ in eigs]


def vhalf(V: np.ndarray) -> np.ndarray:
    is_c = bool(np.iscomplexobj(V))
    V = _f64(V, is_c)
    out = np.zeros_like(V)
    rc = _load().oracle_vhalf(int(is_c), V.shape[0], _ptr(V.view(np.float64)), _ptr(out.view(np.float64)))
    if rc != 0:
        raise OracleError("oracle_vhalf rc=%d" % rc)
    return out


def sandwich(Vh: np.ndarray, chi: np.ndarray, n_threads: Optional[int] = None) -> np.ndarray:
    is_c = bool(np.iscomplexobj(Vh) or np.iscomplexobj(chi))
    Vh, chi = _f64(Vh, is_c), _f64(chi, is_c)
    out = np.zeros_like(chi)
    rc = _load().oracle_sandwich(int(is_c), chi.shape[0], _ptr(Vh.view(np.float64)), _ptr(chi.view(np.float64)),
                                 _ptr(out.view(np.float64)), int(n_threads or max_threads()))
    if rc != 0:
        raise OracleError("oracle_sandwich rc=%d" % rc)
    return out


def logdet(Pi: np.ndarray) -> Tuple[float, float]:
    """(ln det(1 - Pi), Tr Pi) by unblocked Cholesky of 1 - Pi."""
    is_c = bool(np.iscomplexobj(Pi))
    Pi = _f64(Pi, is_c)
    ld, tr = ctypes.c_double(), ctypes.c_double()
    rc = _load().oracle_logdet_cholesky(int(is_c), Pi.shape[0], _ptr(Pi.view(np.float64)), ctypes.byref(ld),
                                        ctypes.byref(tr))
    if rc != 0:
        raise OracleError("oracle_logdet_cholesky rc=%d (not positive definite)" % rc)
    return float(ld.value), float(tr.value)


def logabsdet_lu(M: np.ndarray) -> float:
    is_c = bool(np.iscomplexobj(M))
    M = _f64(M, is_c)
    out = ctypes.c_double()
    rc = _load().oracle_logabsdet_lu(int(is_c), M.shape[0], _ptr(M.view(np.float64)), ctypes.byref(out))
    if rc != 0:
        raise OracleError("oracle_logabsdet_lu rc=%d" % rc)
    return float(out.value)


def energy_sum(w_q: np.ndarray, zeta_w: np.ndarray, eps_qw: np.ndarray) -> float:
    w_q = np.ascontiguousarray(w_q, np.float64)
    zeta_w = np.ascontiguousarray(zeta_w, np.float64)
    eps_qw = np.ascontiguousarray(eps_qw, np.float64)
    out = ctypes.c_double()
    rc = _load().oracle_energy_sum(eps_qw.shape[0], eps_qw.shape[1], _ptr(w_q), _ptr(zeta_w), _ptr(eps_qw),
                                   ctypes.byref(out))
    if rc != 0:
        raise OracleError("oracle_energy_sum rc=%d" % rc)
    return float(out.value)


def term(problem, q: int, w: int, Vh: Optional[np.ndarray] = None, n_threads: Optional[int] = None,
         C_blocks=None) -> Dict[str, float]:
    """One integrand term eps_{q,w} = ln det(1 - Pi) + Tr Pi of a synthetic
    problem (``paper_2505_06021_gb300.synth.Problem``)."""
    if C_blocks is None:
        C_blocks = _blocks(problem, q, n_threads)
    eo = [problem.eps_pair(q, j)[0] for j in range(problem.n_k)]
    ev = [problem.eps_pair(q, j)[1] for j in range(problem.n_k)]
    if Vh is None:
        Vh = vhalf(problem.V(q))
    chi = chi0(C_blocks, eo, ev, problem.grid.zeta_k, float(problem.omega[w]), n_threads)
    Pi = sandwich(Vh, chi, n_threads)
    ld, tr = logdet(Pi)
    return {"lndet": ld, "trPi": tr, "eps": ld + tr}


def energy(problem, n_threads: Optional[int] = None, qs: Optional[Sequence[int]] = None,
           ws: Optional[Sequence[int]] = None) -> Dict[str, object]:
    """Whole job (or a (q, w) subset): per-term table and E_c (E_c only when
    the full table is computed)."""
    qs = list(range(problem.n_q)) if qs is None else list(qs)
    ws = list(range(problem.n_w)) if ws is None else list(ws)
    lndet = np.full((problem.n_q, problem.n_w), np.nan)
    trpi = np.full((problem.n_q, problem.n_w), np.nan)
    for q in qs:
        Vh = vhalf(problem.V(q))
        C_blocks = _blocks(problem, q, n_threads)
        for w in ws:
            t = term(problem, q, w, Vh=Vh, n_threads=n_threads, C_blocks=C_blocks)
            lndet[q, w], trpi[q, w] = t["lndet"], t["trPi"]
    eps = lndet + trpi
    Ec = None
    if len(qs) == problem.n_q and len(ws) == problem.n_w:
        Ec = energy_sum(problem.grid.w_q, problem.zeta_w, eps)
    return {"lndet": lndet, "trPi": trpi, "eps": eps, "Ec": Ec}
