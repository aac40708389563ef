"""GPU tests of the serving runtime (rpa_submit / rpa_wait): continuous
batching of RPA energy jobs of different sizes.

Each result must be the same alone and in the mix: FP64 jobs bit for bit (the
same kernels run on the job's own lane, whatever else shares the device),
mixed-precision jobs within 1e-9 Ha (far inside the 1 microhartree bar; the
split-K plan of a q may differ between the synchronous and the lane
workspace).  The solo runs use the per-frequency chi0 of the served path
(chi0_freq = 1).  Every served result is also checked against the CPU
oracle: FP64 jobs at 1e-10 relative, mixed jobs within 1 microhartree.
Jobs submitted together must overlap on the device, admission must respect
the HBM cap, and the latency statistics must be filled in.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_MIX = 1e-9  # Hartree, served vs alone
TOL_ORACLE_FP64 = 1e-10  # relative
TOL_ORACLE_MIX = 1e-6  # Hartree


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


def _jobs(rpa, n=10, seed=91, problems=None):
    out = []
    for i, (_, p) in enumerate(synth.serving_stream(n_jobs=n, rate_per_s=1.0, seed=seed, scale=0.1)):
        prec = rpa.PREC_FP64 if i % 4 == 3 else rpa.PREC_MIXED
        out.append(rpa.job_from_problem(p, rpa.upload_problem(p), prec=prec))
        if problems is not None:
            problems.append(p)
    return out


def _check_oracle(rpa, job, p, Ec):
    ref = oracle.energy(p)["Ec"]
    if job.s.prec == rpa.PREC_FP64:
        assert abs(Ec - ref) <= TOL_ORACLE_FP64 * abs(ref), (p.name, Ec, ref)
    else:
        assert abs(Ec - ref) <= TOL_ORACLE_MIX, (p.name, Ec, ref)


def test_served_results_equal_alone(rpa):
    probs = []
    jobs = _jobs(rpa, problems=probs)
    with rpa.Context(0, chi0_freq=1) as c:
        alone = [c.energy(j)["Ec"] for j in jobs]
    with rpa.Context(0, max_inflight=8) as c:
        tickets = [c.submit(j) for j in jobs]
        served = [c.wait(t, 300.0)[0] for t in tickets]
        st = c.serving_stats()
        peak = c.serving_peak()
    for j, a, s, p in zip(jobs, alone, served, probs):
        if j.s.prec == rpa.PREC_FP64:
            assert s == a
        else:
            assert abs(s - a) <= TOL_MIX, (s, a)
        _check_oracle(rpa, j, p, s)
    assert st["jobs_done"] == len(jobs)
    assert 0.0 < st["lat_p50_s"] <= st["lat_p99_s"]
    assert peak["max_running"] >= 2  # submitted together: they overlap on the device
    assert peak["max_batch"] >= 2  # and waiting jobs share micro-batches


def test_admission_respects_hbm_cap(rpa):
    jobs = _jobs(rpa, n=6, seed=92)
    fp = [j.footprint() for j in jobs]
    cap = max(fp) + min(fp)  # room for the largest job and at most a small one besides
    with rpa.Context(0, hbm_cap_bytes=cap, max_inflight=8) as c:
        tickets = [c.submit(j) for j in jobs]
        for t in tickets:
            c.wait(t, 300.0)
        peak = c.serving_peak()
    assert peak["max_bytes"] <= cap
    assert peak["max_running"] >= 1


def test_poll_not_ready_then_done(rpa):
    jobs = _jobs(rpa, n=2, seed=93)
    with rpa.Context(0) as c:
        t = c.submit(jobs[0])
        r = c.poll(t)
        assert r is None or isinstance(r[0], float)
        Ec, _ = c.wait(t, 300.0)
        assert np.isfinite(Ec) and Ec < 0.0
        with pytest.raises(rpa.RpaError):
            c.poll(t)  # a ticket is retired once its result was read


def test_failed_job_does_not_disturb_the_others(rpa):
    """A job whose V(q) is indefinite fails alone (RPA_E_NOTPD with its q) while
    the jobs around it in the stream complete with their solo results."""
    jobs = _jobs(rpa, n=5, seed=94)
    with rpa.Context(0, chi0_freq=1) as c:
        alone = [c.energy(j)["Ec"] for j in jobs]
    p = synth.make_problem("bad", is_complex=True, n_aux=48, n_occ=2, n_virt=5, grid=synth.regular_kq_grid((2, 1, 1)),
                           n_w=4, seed=95)
    t = rpa.upload_problem(p)
    Vbad = t["V"][1].clone()
    Vbad[2, 2] = -40.0
    t["V"] = [t["V"][0], Vbad]
    bad = rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED)
    with rpa.Context(0, max_inflight=8) as c:
        tickets = [c.submit(j) for j in jobs[:2]] + [c.submit(bad)] + [c.submit(j) for j in jobs[2:]]
        results = []
        for k, tk in enumerate(tickets):
            if k == 2:
                with pytest.raises(rpa.RpaError) as e:
                    c.wait(tk, 300.0)
                assert e.value.status == rpa.RPA_E_NOTPD and "V(q=1)" in str(e.value)
            else:
                results.append(c.wait(tk, 300.0)[0])
    for j, a, s in zip(jobs, alone, results):
        if j.s.prec == rpa.PREC_FP64:
            assert s == a
        else:
            assert abs(s - a) <= TOL_MIX
