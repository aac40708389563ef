"""The frequency-batched chi0 plan (rpa_freq_plan, host-only) against the CPU
oracle.

The plan splits the transitions into bins of their energy D (interior edges,
ascending) and, inside bin b, writes every node's weight as a combination of
rank[b] skeleton nodes' weights.  Pins, none of which restates the plan's
own arithmetic:

* exactness at the skeleton nodes (coefficient rows are unit vectors there);
* the factorised chi0, sum_b sum_r coef[b][r][w] X_{b,r} with X_{b,r} the
  oracle's chi0 of bin b's transitions alone (columns of C outside the bin
  zeroed) at the skeleton frequency, equals the oracle's chi0 at every node w
  within the plan's error bound: every weight d_t(w) of one frequency has the
  same sign, so a relative error e of each weight moves chi0 by at most
  e |chi0| in the Loewner order, |d chi0_PQ| <= e max_P |chi0_PP|; within a
  bin whose ends differ by the factor rho, the residual err[b] (relative to
  the bin's largest weight) is at most err[b] rho relative to each weight;
* the modelled work is below n_w contractions for a 16-node grid over the
  band structure of the periodic workloads;
* a planted mistake (the coefficients of two skeletons swapped) breaks the
  equality by many orders of magnitude more than the bound.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def rpa():
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


def _host_job(rpa, p):
    t = rpa.upload_problem(p, device="cpu")
    return rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED, mem=rpa.MEM_HOST)


def _bins(edges, D):
    return np.searchsorted(np.asarray(edges), D, side="right")


def _factorised(p, plan, q, C, w_list):
    """sum_b sum_r coef X_{b,r} with X from the oracle on bin-masked C."""
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    D = [(ev[j][None, :] - eo[j][:, None]).reshape(-1) for j in range(p.n_k)]
    out = {w: 0.0 for w in w_list}
    for b in range(plan["n_bins"]):
        Cb = []
        for j in range(p.n_k):
            m = _bins(plan["edges"], D[j]) == b
            Cb.append(np.where(m[None, :], C[j], 0.0))
        for r in range(plan["rank"][b]):
            s = plan["skel"][b][r]
            X = oracle.chi0(Cb, eo, ev, p.grid.zeta_k, float(p.omega[s]))
            for w in w_list:
                out[w] = out[w] + plan["coef"][b][r][w] * X
    return out


@pytest.mark.parametrize("is_complex", [True, False])
def test_plan_factorised_chi0_matches_oracle(rpa, is_complex):
    if is_complex:
        p = synth.config1(n_w=16, n_aux=20, n_occ=6, n_virt=40, kdims=(2, 2, 1))
    else:
        p = synth.make_problem("fr", is_complex=False, n_aux=20, n_occ=6, n_virt=60, grid=synth.gamma_grid(), n_w=16,
                               seed=5)
    job = _host_job(rpa, p)
    plan = job.freq_plan(mode=2)
    assert plan["n_bins"] >= 2
    assert np.all(plan["rank"] < p.n_w)
    assert np.all(plan["err"] <= 1e-10)
    # exact at the skeleton nodes
    for b in range(plan["n_bins"]):
        for r in range(plan["rank"][b]):
            row = plan["coef"][b][:plan["rank"][b], plan["skel"][b][r]]
            assert np.allclose(row, np.eye(plan["rank"][b])[r], atol=1e-12)
    q = p.n_q - 1
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    ws = [0, 3, 7, 11, 15]
    fac = _factorised(p, plan, q, C, ws)
    edges = np.concatenate([[0.0], plan["edges"]])
    rho = max(plan["edges"][1:] / plan["edges"][:-1]) if len(plan["edges"]) > 1 else 10.0
    bound = 2.0 * plan["err"].max() * rho
    for w in ws:
        ref = oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))
        scale = np.abs(np.diag(ref)).max()
        err = np.abs(fac[w] - ref).max() / scale
        assert err <= bound + 1e-14, (w, err, bound)
    assert edges.size >= 2


def test_plan_saves_work_on_the_periodic_band_structure(rpa):
    for p in (synth.config1(n_aux=8, n_occ=32, n_virt=224), synth.config2(n_aux=8, n_occ=32, n_virt=480)):
        plan = _host_job(rpa, p).freq_plan(mode=0)
        assert plan["n_bins"] > 0
        assert plan["work_ratio"] < 0.6, plan["work_ratio"]


def test_plan_off_for_few_frequencies(rpa):
    p = synth.make_problem("f3", is_complex=True, n_aux=16, n_occ=3, n_virt=9, grid=synth.regular_kq_grid((2, 1, 1)),
                           n_w=3, seed=7)
    assert _host_job(rpa, p).freq_plan(mode=0)["n_bins"] == 0


def test_planted_coefficient_swap_is_caught(rpa):
    p = synth.config1(n_w=16, n_aux=12, n_occ=4, n_virt=30, kdims=(2, 1, 1))
    plan = _host_job(rpa, p).freq_plan(mode=2)
    b = int(np.argmax(plan["rank"]))
    bad = dict(plan)
    bad["coef"] = plan["coef"].copy()
    bad["coef"][b][[0, 1]] = bad["coef"][b][[1, 0]]
    q = 0
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    w = [i for i in range(p.n_w) if i not in plan["skel"][b][:plan["rank"][b]]][0]
    ref = oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))
    err = np.abs(_factorised(p, bad, q, C, [w])[w] - ref).max() / np.abs(np.diag(ref)).max()
    assert err > 1e-6
