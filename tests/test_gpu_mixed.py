"""GPU parity of the split-precision chi0 (BF16 digit slices on tcgen05 with
exact FP32 accumulation of the leading slice levels) against the FP64 oracle.

Tolerances (written here, derived from the arithmetic):
* chi0: every value is a 31-bit fixed-point number relative to a per-row power
  of two; all four 8-bit digits are kept, and the slice pairs of level >= 4
  that are dropped contribute up to 2^-30 of the squared row scale per term
  with random signs.  Typical entries sit ~2^-4 below the row maximum, so
  relative to max|chi| (the diagonal, ~K typical squares) the error is about
  2^-22 / sqrt(K), below 5e-8 for K >= 16 real terms.  Bar: 5e-8.
* E_c: the spec bar for the mixed path, |dE_c| <= 1 microhartree.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_CHI = 5e-8
TOL_EC = 1e-6  # Hartree


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


def _oracle_chi(p, q, w):
    C = [p.C(q, j) for j in range(p.n_k)]
    eo = [p.eps_pair(q, j)[0] for j in range(p.n_k)]
    ev = [p.eps_pair(q, j)[1] for j in range(p.n_k)]
    return oracle.chi0(C, eo, ev, p.grid.zeta_k, float(p.omega[w]))


@pytest.mark.parametrize("kind", ["complex", "real"])
def test_mixed_chi0_elementwise(rpa, ctx, kind):
    if kind == "complex":
        p = synth.make_problem("m", is_complex=True, n_aux=150, n_occ=4, n_virt=17,
                               grid=synth.regular_kq_grid((2, 2, 1)), n_w=4, seed=41)
    else:
        p = synth.make_problem("m", is_complex=False, n_aux=140, n_occ=5, n_virt=31, grid=synth.gamma_grid(),
                               n_w=4, seed=42)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    for q in sorted({0, p.n_q - 1}):
        chi = ctx.chi0(job, q).cpu().numpy()
        for w in range(p.n_w):
            ref = _oracle_chi(p, q, w)
            err = np.abs(chi[w] - ref).max() / np.abs(ref).max()
            assert err <= TOL_CHI, (q, w, err)
            assert np.array_equal(chi[w], chi[w].conj().T)


def test_mixed_tile_edges(rpa, ctx):
    """n_aux below, at and across the 128-row / 64-column tile edges; one
    transition; a K range far from the 1024-t chunk."""
    for n_aux, n_occ, n_virt, kd in ((1, 1, 1, (2, 1, 1)), (63, 1, 3, (2, 1, 1)), (64, 2, 5, (1, 1, 1)),
                                     (65, 1, 7, (2, 1, 1)), (129, 3, 3, (2, 1, 1)), (200, 2, 9, (2, 1, 1))):
        cplx = kd != (1, 1, 1)
        grid = synth.regular_kq_grid(kd) if cplx else synth.gamma_grid()
        p = synth.make_problem("e", is_complex=cplx, n_aux=n_aux, n_occ=n_occ, n_virt=n_virt, grid=grid, n_w=2,
                               seed=n_aux)
        job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
        q = p.n_q - 1
        chi = ctx.chi0(job, q).cpu().numpy()
        for w in range(p.n_w):
            ref = _oracle_chi(p, q, w)
            assert np.abs(chi[w] - ref).max() <= TOL_CHI * np.abs(ref).max(), (n_aux, n_occ, n_virt, w)


def test_mixed_energy_gamma_real_config(rpa, ctx):
    """Gamma-only real workload (N_aux=64, 4 occ, 28 virt, 16 frequencies)."""
    p = synth.config0()
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    r = ctx.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC


def test_mixed_energy_periodic(rpa, ctx):
    p = synth.make_problem("m", is_complex=True, n_aux=160, n_occ=6, n_virt=30,
                           grid=synth.regular_kq_grid((2, 2, 1)), n_w=6, seed=43)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    r = ctx.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC, (r["Ec"], ref["Ec"])
    assert np.max(np.abs(r["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-8


def test_mixed_energy_large_aux(rpa, ctx):
    """N_aux = 300: inverse-form tail with the cluster Cholesky (few, large
    matrices per launch)."""
    p = synth.make_problem("m", is_complex=True, n_aux=300, n_occ=2, n_virt=6,
                           grid=synth.regular_kq_grid((2, 1, 1)), n_w=3, seed=45)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    r = ctx.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC, (r["Ec"], ref["Ec"])
    assert np.max(np.abs(r["eps"] - ref["eps"]) / np.abs(ref["eps"])) <= 1e-8


def test_mixed_energy_at_frequency_limit(rpa, ctx):
    """32 frequencies (the split path's maximum: one persistent launch round
    carries up to 32 frequency groups of a q)."""
    p = synth.make_problem("m32", is_complex=True, n_aux=72, n_occ=2, n_virt=7,
                           grid=synth.regular_kq_grid((2, 1, 1)), n_w=32, seed=46)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    r = ctx.energy(job)
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC, (r["Ec"], ref["Ec"])
    # the largest nodes carry tiny terms: compare against the largest one
    assert np.max(np.abs(r["eps"] - ref["eps"])) <= 1e-8 * np.max(np.abs(ref["eps"]))


def test_mixed_energy_pipelined_slicing(rpa):
    """Several q of one shape whose tensor-core launches fill the GPU (4 q,
    N_aux 384: 12 tiles x 16 frequencies = 192 work items): the weighted digit
    planes of each next q are written by the slicer warps of the current q's
    launch, so the job has one standalone weighted-slicing launch plus the
    five preparation launches per q.  E_c and every term against the oracle,
    and bit-identical on a second run.  Per-frequency chi0 (chi0_freq = 1);
    the frequency-batched form of the same pipeline is tested in
    test_gpu_freq.py."""
    p = synth.make_problem("pipe", is_complex=True, n_aux=384, n_occ=4, n_virt=24,
                           grid=synth.regular_kq_grid((2, 2, 1)), n_w=16, seed=47)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0, chi0_freq=1) as c:
        c.profile(True)
        r = c.energy(job)
        prof = c.profile_read()
        r2 = c.energy(job)
    assert prof["slice"][1] == 6 + 5 * (p.n_q - 1), prof["slice"]
    assert prof["chi0"][1] == p.n_q
    assert r["Ec"] == r2["Ec"] and np.array_equal(r["eps"], r2["eps"])
    ref = oracle.energy(p)
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_EC, (r["Ec"], ref["Ec"])
    assert np.max(np.abs(r["eps"] - ref["eps"])) <= 1e-8 * np.max(np.abs(ref["eps"]))


def test_mixed_deterministic_and_slice_count(rpa):
    p = synth.make_problem("m", is_complex=True, n_aux=96, n_occ=3, n_virt=20, grid=synth.regular_kq_grid((2, 1, 1)),
                           n_w=3, seed=44)
    t = rpa.upload_problem(p)
    jf = rpa.job_from_problem(p, t)
    jm = rpa.job_from_problem(p, t, prec=rpa.PREC_MIXED)
    errs = {}
    for s in (2, 3, 4):
        with rpa.Context(0, n_slices=s) as c:
            a = c.energy(jm)
            b = c.energy(jm)
            assert a["Ec"] == b["Ec"] and np.array_equal(a["eps"], b["eps"])
            ref = c.energy(jf)
            errs[s] = abs(a["Ec"] - ref["Ec"])
    assert errs[4] < errs[3] < errs[2]
    assert errs[4] <= TOL_EC


@pytest.mark.slow
def test_slab_dual_grid_full_size_subset(rpa):
    """The slab dual-grid workload at full size (N_aux=768, 32 occ, 480 virt,
    36 k per q, 16 freq) on two of its q-points, the first regular one and the
    first near-Gamma one (the dual grid's displaced point, whose V has the
    scaled leading eigenvalue), both paths in the benchmark's launch
    configuration: every term of the sampled subset q x w in {0, 8, 15}
    against the oracle, the FP64 path at 1e-10 and the split-precision path at
    1e-8 relative per term; the split path against the FP64 path on all
    terms of the two q and on their weighted energy."""
    from paper_2505_06021_gb300 import shard

    p = synth.config2()
    ng = np.asarray(p.grid.near_gamma, bool)
    qs = [int(np.argmin(ng)), int(np.argmax(ng))]
    ws = [0, 8, 15]
    t = rpa.upload_problem(p, qs=qs)
    g = p.grid
    sel = [q * p.n_k + j for q in qs for j in range(p.n_k)]
    jf = rpa.Job(is_complex=True, n_aux=p.n_aux, n_occ=p.n_occ, n_virt=p.n_virt,
                 pair_k=g.pair_k[qs].reshape(-1), pair_kq=g.pair_kq[qs].reshape(-1), w_q=g.w_q[qs],
                 zeta_k=g.zeta_k, omega=p.omega, zeta_w=p.zeta_w, eps_occ=t["eps_occ"], eps_virt=t["eps_virt"],
                 C=t["C"], V=t["V"])
    assert len(sel) == len(t["C"])
    jm = jf.with_prec(rpa.PREC_MIXED)
    with rpa.Context(0) as c:
        rf = c.energy(jf)
        rm = c.energy(jm)
    del t
    torch.cuda.empty_cache()
    rel = np.abs(rm["eps"] - rf["eps"]) / np.abs(rf["eps"])
    assert rel.max() <= 1e-8, rel.max()
    assert abs(rm["Ec"] - rf["Ec"]) <= TOL_EC
    ref = oracle.energy(p, qs=qs, ws=ws)
    for i, q in enumerate(qs):
        for w in ws:
            for key in ("eps", "lndet", "trPi"):
                assert abs(rf[key][i, w] - ref[key][q, w]) <= 1e-10 * abs(ref[key][q, w]), (q, w, key)
            assert abs(rm["eps"][i, w] - ref["eps"][q, w]) <= 1e-8 * abs(ref["eps"][q, w]), (q, w)
    assert shard.quadrature(rf["eps"], g.w_q[qs], p.zeta_w) == pytest.approx(rf["Ec"], rel=1e-12)


def test_tensor_core_wait_runs_out_and_context_recovers(rpa):
    """Failure path without a GPU fault: one work item's operand copies are
    never issued, the MMA thread's bounded wait (2 s) runs out, the kernel
    raises its flag, drains and frees tensor memory, the call reports a
    time-out, and the same context then computes the right energy."""
    import time

    p = synth.make_problem("m", is_complex=True, n_aux=96, n_occ=3, n_virt=10, grid=synth.regular_kq_grid((2, 1, 1)),
                           n_w=3, seed=46)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    with rpa.Context(0) as c:
        good = c.energy(job)["Ec"]
        c.test_drop_copy(0)
        t0 = time.perf_counter()
        with pytest.raises(rpa.RpaError) as e:
            c.energy(job)
        assert e.value.status == rpa.RPA_E_TIMEOUT
        assert time.perf_counter() - t0 < 60.0
        assert c.energy(job)["Ec"] == good
