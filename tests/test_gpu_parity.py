"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Tolerances (written here, derived from the arithmetic):
* chi0 elements: |chi_gpu - chi_oracle| <= 1e-12 max|chi| -- both sides sum
  K <= 1e4 FP64 products in different orders, worst-case relative rounding
  K * 2^-53 ~ 1e-12 of the largest entry;
* every integrand term (ln det, Tr Pi, eps) and E_c: 1e-10 relative, the bar
  the plain FP64 path must meet.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_CHI = 1e-12
TOL_TERM = 1e-10


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


@pytest.fixture(scope="module")
def ctx(rpa):
    c = rpa.Context(0)
    yield c
    c.close()


def _small_complex(n_aux=77, n_occ=3, n_virt=11, kdims=(2, 2, 1), n_w=5, seed=21):
    return synth.make_problem("t", is_complex=True, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                              grid=synth.regular_kq_grid(kdims), n_w=n_w, seed=seed)


def _small_real(n_aux=45, n_occ=4, n_virt=13, n_w=7, seed=22):
    return synth.make_problem("t", is_complex=False, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                              grid=synth.gamma_grid(), n_w=n_w, seed=seed)


def _oracle_chi(p, q, w):
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    return oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))


def _rel(a, b):
    return np.abs(np.asarray(a) - np.asarray(b)) / np.abs(np.asarray(b))


@pytest.mark.parametrize("kind", ["complex", "real"])
def test_chi0_elementwise(rpa, ctx, kind):
    p = _small_complex() if kind == "complex" else _small_real()
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    for q in sorted({0, p.n_q - 1}):
        chi = ctx.chi0(job, q).cpu().numpy()
        for w in range(p.n_w):
            ref = _oracle_chi(p, q, w)
            err = np.abs(chi[w] - ref).max() / np.abs(ref).max()
            assert err <= TOL_CHI, (q, w, err)
            # exactly Hermitian (lower triangle mirrored)
            assert np.array_equal(chi[w], chi[w].conj().T)


def test_chi0_tile_edges(rpa, ctx):
    """n_aux on and around the 32-row tile edge, n_ov of 1 and not a multiple
    of the 16-wide chunk, a single k-pair."""
    for n_aux, n_occ, n_virt in ((32, 1, 1), (33, 1, 17), (64, 2, 9), (1, 1, 3), (95, 1, 1)):
        p = synth.make_problem("e", is_complex=True, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt,
                               grid=synth.regular_kq_grid((2, 1, 1)), n_w=3, seed=n_aux)
        job = rpa.job_from_problem(p, rpa.upload_problem(p))
        chi = ctx.chi0(job, 1).cpu().numpy()
        for w in range(p.n_w):
            ref = _oracle_chi(p, 1, w)
            assert np.abs(chi[w] - ref).max() <= TOL_CHI * np.abs(ref).max(), (n_aux, n_occ, n_virt, w)


@pytest.mark.parametrize("kind", ["complex", "real"])
def test_logdet_from_oracle_chi(rpa, ctx, kind):
    """Steps A4-A6 alone: the oracle's chi0 is handed to rpa_logdet."""
    p = _small_complex(n_aux=70) if kind == "complex" else _small_real(n_aux=50)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    q = p.n_q - 1
    chis = np.stack([_oracle_chi(p, q, w) for w in range(p.n_w)])
    out = ctx.logdet(job, q, torch.from_numpy(chis).cuda())
    Vh = oracle.vhalf(p.V(q))
    for w in range(p.n_w):
        ld, tr = oracle.logdet(oracle.sandwich(Vh, chis[w]))
        assert abs(out[w, 0] - ld) <= TOL_TERM * abs(ld)
        assert abs(out[w, 1] - tr) <= TOL_TERM * abs(tr)
        assert abs(out[w].sum() - (ld + tr)) <= TOL_TERM * abs(ld + tr)


def _check_energy(r, ref):
    for key in ("lndet", "trPi", "eps"):
        rel = _rel(r[key], ref[key])
        assert np.nanmax(rel) <= TOL_TERM, (key, np.nanmax(rel))
    if ref["Ec"] is not None:
        assert abs(r["Ec"] - ref["Ec"]) <= TOL_TERM * abs(ref["Ec"])


def test_energy_gamma_real_config(rpa, ctx):
    """Gamma-only real workload, full size (N_aux=64, 4 occ, 28 virt, 16 freq)."""
    p = synth.config0()
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    r = ctx.energy(job)
    _check_energy(r, oracle.energy(p))


def test_energy_small_periodic(rpa, ctx):
    p = _small_complex(n_aux=90, n_occ=2, n_virt=13, kdims=(3, 2, 1), n_w=6)
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    _check_energy(ctx.energy(job), oracle.energy(p))


def test_energy_small_dual_grid(rpa, ctx):
    """Dual k-grid (Sec. 2.5): 2x2x1 q-grid without Gamma + 4 near-Gamma
    points, 4x4x1 K_reg; k_j + q leaves K_reg for the near-Gamma points."""
    p = synth.config2(n_aux=40, n_occ=2, n_virt=5, q_dims=(2, 2, 1), k_dims=(4, 4, 1), n_w=4)
    assert p.grid.kpts.shape[0] == 5 * 16
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    _check_energy(ctx.energy(job), oracle.energy(p))


def test_host_memory_path_matches_device(rpa, ctx):
    p = _small_complex(n_aux=64, n_occ=2, n_virt=7, kdims=(2, 2, 1), n_w=4)
    jd = rpa.job_from_problem(p, rpa.upload_problem(p))
    jh = rpa.job_from_problem(p, rpa.upload_problem(p, device="cpu", pin=True), mem=rpa.MEM_HOST)
    a, b = ctx.energy(jd), ctx.energy(jh)
    assert a["Ec"] == b["Ec"]
    assert np.array_equal(a["eps"], b["eps"])


def test_deterministic(rpa, ctx):
    p = _small_complex(n_aux=50, n_occ=2, n_virt=6)
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    a, b = ctx.energy(job), ctx.energy(job)
    assert a["Ec"] == b["Ec"] and np.array_equal(a["eps"], b["eps"])


def test_not_positive_definite_reported(rpa, ctx):
    """Failures made on the host: an indefinite V(q) and a chi0 that makes
    1 - Pi indefinite come back as RPA_E_NOTPD with (q, w), no device trap."""
    p = _small_complex(n_aux=24, n_occ=2, n_virt=3, kdims=(2, 1, 1), n_w=3)
    t = rpa.upload_problem(p)
    Vbad = t["V"][1].clone()
    Vbad[3, 3] = -50.0
    t2 = dict(t)
    t2["V"] = [t["V"][0], Vbad]
    job = rpa.job_from_problem(p, t2)
    with pytest.raises(rpa.RpaError) as e:
        ctx.energy(job)
    assert e.value.status == rpa.RPA_E_NOTPD and "V(q=1)" in str(e.value)
    job = rpa.job_from_problem(p, t)
    chi = torch.zeros((p.n_w, 24, 24), dtype=torch.complex128, device="cuda")
    chi[2] = 100.0 * torch.eye(24, dtype=torch.complex128, device="cuda")  # chi > 0: 1 - Pi indefinite
    with pytest.raises(rpa.RpaError) as e:
        ctx.logdet(job, 0, chi)
    assert e.value.status == rpa.RPA_E_NOTPD and "w=2" in str(e.value)
    # the context stays usable
    r = ctx.energy(job)
    assert math.isfinite(r["Ec"])


def test_large_aux_cluster_cholesky(rpa, ctx):
    """N_aux >= 256 with few matrices per launch: the Cholesky factorisations
    run on thread-block clusters (8 CTAs per matrix); parity as everywhere,
    and an indefinite V is still reported with its q."""
    p = _small_complex(n_aux=300, n_occ=2, n_virt=6, kdims=(2, 1, 1), n_w=3)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    _check_energy(ctx.energy(job), oracle.energy(p))
    Vbad = t["V"][0].clone()
    Vbad[7, 7] = -80.0
    t2 = dict(t)
    t2["V"] = [Vbad, t["V"][1]]
    with pytest.raises(rpa.RpaError) as e:
        ctx.energy(rpa.job_from_problem(p, t2))
    assert e.value.status == rpa.RPA_E_NOTPD and "V(q=0)" in str(e.value)
    assert math.isfinite(ctx.energy(job)["Ec"])


def test_kernel_launch_count(rpa, ctx):
    p = _small_complex(n_aux=40, n_occ=2, n_virt=4)
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    n0 = ctx.launches
    ctx.energy(job)
    # d table, chi0, V factor, 2 sandwich passes, log-det, quadrature
    assert ctx.launches - n0 == 7


@pytest.mark.slow
def test_periodic_config_full_size_sampled(rpa):
    """The 2-D periodic workload at full size (N_aux=512, 32 occ, 224 virt,
    16 k x 16 q, 20 freq) through the same launch configuration as the
    benchmark; the oracle recomputes the six sampled (q, w) terms."""
    p = synth.config1()
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    with rpa.Context(0) as c:
        r = c.energy(job)
    del t
    torch.cuda.empty_cache()
    # the sampled subset: q in {Gamma, 5} x w in {0, 10, 19}
    qs, ws = [0, 5], [0, 10, 19]
    ref = oracle.energy(p, qs=qs, ws=ws)
    for q in qs:
        for w in ws:
            for key in ("eps", "lndet", "trPi"):
                assert abs(r[key][q, w] - ref[key][q, w]) <= TOL_TERM * abs(ref[key][q, w]), (q, w, key)
    # properties that hold at any size
    assert r["Ec"] < 0 and np.all(r["eps"] < 0)
    assert np.all(r["lndet"] > 0) and np.all(r["trPi"] < 0)
