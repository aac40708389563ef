"""GPU parity of the frequency-batched split-precision chi0 (rpa_config
chi0_freq = 2: contractions over energy bins at skeleton frequencies,
recombined per frequency in FP64) against the CPU oracle.

Tolerances (written here, derived from the arithmetic):
* chi0 elements: each X_{b,r} carries the split-precision error of a single
  contraction (below 5e-8 of its own largest diagonal entry, the bar of the
  per-frequency path); the recombination multiplies it by at most the
  plan's coefficient sum (<= 16 by construction, 2-6 in practice), and the
  factorisation adds 1e-10 relative.  Bar: 16 x 5e-8 = 8e-7 of max|chi|.
* E_c: |dE_c| <= 1 microhartree against the oracle (the mixed path's bar);
  against the per-frequency split path 1e-7 Ha here.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_CHI = 8e-7
TOL_EC = 1e-6  # Hartree


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


def _oracle_chi(p, q, w):
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    return oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))


def _periodic(n_aux=150, n_occ=5, n_virt=37, kdims=(2, 2, 1), n_w=16, seed=51):
    return synth.make_problem("fb", is_complex=True, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                              grid=synth.regular_kq_grid(kdims), n_w=n_w, seed=seed)


@pytest.mark.parametrize("kind", ["complex", "real"])
def test_binned_chi0_elementwise(rpa, kind):
    if kind == "complex":
        p = _periodic()
    else:
        p = synth.make_problem("fr", is_complex=False, n_aux=130, n_occ=6, n_virt=70, grid=synth.gamma_grid(),
                               n_w=16, seed=52)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=2) as c:
        for q in sorted({0, p.n_q - 1}):
            chi = c.chi0(job, q).cpu().numpy()
            for w in (0, 5, 10, 15):
                ref = _oracle_chi(p, q, w)
                err = np.abs(chi[w] - ref).max() / np.abs(ref).max()
                assert err <= TOL_CHI, (q, w, err)
                assert np.array_equal(chi[w], chi[w].conj().T)


def test_binned_energy_against_oracle_and_per_frequency(rpa):
    p = _periodic(n_aux=96, n_occ=4, n_virt=30, seed=53)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=2) as c:
        rb = c.energy(job)
        rb2 = c.energy(job)
    with rpa.Context(0, chi0_freq=1) as c:
        rf = c.energy(job)
    ref = oracle.energy(p)
    assert rb["Ec"] == rb2["Ec"]  # deterministic
    assert abs(rb["Ec"] - ref["Ec"]) <= TOL_EC
    assert abs(rb["Ec"] - rf["Ec"]) <= 1e-7
    assert np.max(np.abs(rb["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-6


def test_binned_several_rounds(rpa):
    """A workspace cap small enough that each q needs several rounds of
    skeleton slots (one workspace region, no in-launch slicing)."""
    p = _periodic(n_aux=100, n_occ=4, n_virt=40, seed=54)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=2, hbm_cap_bytes=6 << 20) as c:
        r = c.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC
    assert np.max(np.abs(r["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-6


def test_binned_host_staged_and_ragged(rpa):
    """Host-resident inputs (staged per q-batch) and shapes off the tile grid:
    n_aux not a multiple of 128, n_occ*n_virt not a multiple of 8."""
    p = _periodic(n_aux=131, n_occ=3, n_virt=29, kdims=(3, 1, 1), n_w=20, seed=55)
    th = rpa.upload_problem(p, device="cpu", pin=True)
    job = rpa.job_from_problem(p, th, prec=rpa.PREC_MIXED, mem=rpa.MEM_HOST)
    with rpa.Context(0, chi0_freq=2) as c:
        r = c.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC
    assert np.max(np.abs(r["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-6


def test_binned_is_default_when_it_saves_work(rpa):
    p = _periodic(n_aux=64, n_occ=4, n_virt=30, seed=56)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0) as c:
        c.profile(True)
        c.energy(job)
        flops_auto = c.profile_counters()["tensor_flops"]
    with rpa.Context(0, chi0_freq=1) as c:
        c.profile(True)
        c.energy(job)
        flops_full = c.profile_counters()["tensor_flops"]
    plan = rpa.job_from_problem(p, rpa.upload_problem(p, device="cpu"), prec=rpa.PREC_MIXED,
                                mem=rpa.MEM_HOST).freq_plan()
    assert plan["n_bins"] > 0 and flops_auto < 0.8 * flops_full


def test_binned_pipelined_launch_count_and_determinism(rpa):
    """Several q of one shape with all skeletons in one round: the weighted
    planes of each next q are written inside the current q's tensor-core
    launch, so a job has one standalone weighted-slicing launch, six
    preparation launches per q and one tensor-core launch per q."""
    p = synth.make_problem("pipeb", is_complex=True, n_aux=384, n_occ=4, n_virt=24,
                           grid=synth.regular_kq_grid((2, 2, 1)), n_w=16, seed=47)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=2) as c:
        c.profile(True)
        r = c.energy(job)
        prof = c.profile_read()
        r2 = c.energy(job)
    assert prof["slice"][1] == 1 + 6 * p.n_q, prof["slice"]
    assert prof["chi0"][1] == p.n_q
    assert r["Ec"] == r2["Ec"] and np.array_equal(r["eps"], r2["eps"])
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC, (r["Ec"], ref["Ec"])
    assert np.max(np.abs(r["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-6


def test_binned_wait_runs_out_and_context_recovers(rpa):
    """Failure path of the frequency-batched launch without a GPU fault: one
    work item's operand copies are never issued, the bounded wait runs out,
    the call reports a time-out, and the same context then gives the same
    energy as before."""
    import time

    p = _periodic(n_aux=96, n_occ=3, n_virt=30, kdims=(2, 1, 1), seed=57)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=2) as c:
        good = c.energy(job)["Ec"]
        c.test_drop_copy(0)
        t0 = time.perf_counter()
        with pytest.raises(rpa.RpaError) as e:
            c.energy(job)
        assert e.value.status == rpa.RPA_E_TIMEOUT
        assert time.perf_counter() - t0 < 60.0
        assert c.energy(job)["Ec"] == good


def test_binned_not_positive_definite_reported(rpa):
    """An indefinite V(q) planted on the host is reported with its q by the
    frequency-batched path as well, and the context keeps working."""
    p = _periodic(n_aux=80, n_occ=3, n_virt=24, kdims=(2, 1, 1), seed=58)
    t = rpa.upload_problem(p)
    Vbad = t["V"][1].clone()
    Vbad[5, 5] = -60.0
    t2 = dict(t)
    t2["V"] = [t["V"][0], Vbad]
    with rpa.Context(0, chi0_freq=2) as c:
        with pytest.raises(rpa.RpaError) as e:
            c.energy(rpa.job_from_problem(p, t2, prec=rpa.PREC_MIXED))
        assert e.value.status == rpa.RPA_E_NOTPD and "V(q=1)" in str(e.value)
        r = c.energy(rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED))
    assert abs(r["Ec"] - oracle.energy(p)["Ec"]) <= TOL_EC
