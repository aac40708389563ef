"""The GPU evaluates ln det(1 - Pi) + Tr Pi of the paper's Pi = V^(1/2) chi0
V^(1/2) in two algebraically equal forms (the metric independence of the
paper's appendix; Sylvester's determinant identity):

* sandwich form (FP64 path): Pi' = L^H chi0 L with V = L L^H;
* inverse form (split-precision path): ln det(1 - Pi) = ln det(V^-1 - chi0)
  + ln det V and Tr Pi = Tr(chi0 V) = sum_PQ Re(chi0_PQ conj(V_PQ)).

Both are checked here on the CPU against the oracle's V^(1/2) route on a small
problem; numpy's Cholesky and inverse serve as the independent route.  The
inverse form loses
digits only where ln det(1 - Pi) is tiny next to ln det V (large frequencies);
its absolute error stays at the rounding level of ln det V.
"""
import numpy as np

import oracle
from paper_2505_06021_gb300 import synth


def _problem():
    return synth.make_problem("id", is_complex=True, n_aux=40, n_occ=3, n_virt=9,
                              grid=synth.regular_kq_grid((2, 2, 1)), n_w=10, seed=17)


def _chi(p, q, w):
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    return oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))


def test_sandwich_and_inverse_forms_match_vhalf_route():
    p = _problem()
    for q in (0, p.n_q - 1):
        V = p.V(q)
        Vh = oracle.vhalf(V)
        L = np.linalg.cholesky(V)
        ldV = 2.0 * np.sum(np.log(np.real(np.diag(L))))
        W = np.linalg.inv(V)
        for w in range(p.n_w):
            chi = _chi(p, q, w)
            lndet, tr = oracle.logdet(oracle.sandwich(Vh, chi))
            eps = lndet + tr
            # sandwich form
            Pp = L.conj().T @ chi @ L
            s2, ld2 = np.linalg.slogdet(np.eye(p.n_aux) - Pp)
            assert s2 > 0
            assert abs(ld2 - lndet) <= 1e-12 * max(1.0, abs(lndet))
            assert abs(np.real(np.trace(Pp)) - tr) <= 1e-12 * max(1.0, abs(tr))
            # inverse form
            Lm = np.linalg.cholesky(W - chi)
            ld3 = 2.0 * np.sum(np.log(np.real(np.diag(Lm)))) + ldV
            tr3 = np.sum(np.real(chi * V.conj()))
            assert abs(ld3 - lndet) <= 1e-11 * max(1.0, abs(ldV))
            assert abs(tr3 - tr) <= 1e-12 * max(1.0, abs(tr))
            assert abs((ld3 + tr3) - eps) <= 1e-11 * max(1.0, abs(ldV))
