"""GPU parity of AO-form jobs (Sec. 2.2): the MO-basis fit coefficients formed
on the device from the k-dependent PADF and MO coefficients, and the whole
path run from them.

* rpa_ao2mo vs the oracle's double sum, element by element, on shapes with
  ragged 32-wide tiles in every dimension (several atoms of uneven sizes) and
  on Gamma-only real data: FP64, 1e-12 of the block's largest entry;
* rpa_energy of an AO job vs the oracle's whole job (FP64: 1e-10 relative per
  term and on E_c; split precision: |dE_c| <= 1 microhartree);
* rpa_chi0 of an AO job equals rpa_chi0 of the same job given the
  coefficients directly;
* at the benchmark's AO workload size: sampled entries of one q against the
  oracle, entry by entry;
* the batch and serving entry points refuse AO jobs.
"""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_C = 1e-12  # of max |C| per block
TOL_TERM = 1e-10  # relative, FP64 path
TOL_MIX = 1e-6  # Hartree


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


def _ragged():
    return synth.make_ao_problem("ao-ragged", is_complex=True, n_bas_atom=(40, 36, 34), n_fit_atom=(50, 40, 30),
                                 n_occ=37, n_virt=70, grid=synth.regular_kq_grid((2, 2, 1)), n_w=4, seed=61)


def _small(is_complex=True):
    grid = synth.regular_kq_grid((2, 2, 1)) if is_complex else synth.gamma_grid()
    return synth.make_ao_problem("ao-small", is_complex=is_complex, n_bas_atom=(10, 14, 8),
                                 n_fit_atom=(24, 30, 18), n_occ=5, n_virt=27, grid=grid, n_w=8, seed=62)


def _check_blocks(got, p, q):
    for j in range(p.n_k):
        ref = oracle.ao2mo_block(p, q, j)
        g = got[j].cpu().numpy()
        assert np.abs(g - ref).max() <= TOL_C * np.abs(ref).max(), (q, j)


def test_ao2mo_matches_oracle_ragged_tiles(rpa):
    p = _ragged()
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        for q in (0, 3):
            out = c.ao2mo(job, q)
            torch.cuda.synchronize()
            _check_blocks(out, p, q)


def test_ao2mo_matches_oracle_gamma_real(rpa):
    p = _small(is_complex=False)
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        out = c.ao2mo(job, 0)
        torch.cuda.synchronize()
    assert out.dtype == torch.float64
    _check_blocks(out, p, 0)


@pytest.mark.parametrize("is_complex", [True, False])
def test_ao_energy_matches_oracle_fp64(rpa, is_complex):
    p = _small(is_complex)
    ref = oracle.energy(p)
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t, prec=rpa.PREC_FP64)
    with rpa.Context(0) as c:
        r = c.energy(job)
    for key in ("lndet", "trPi", "eps"):
        a, b = np.asarray(r[key]), ref[key]
        assert np.all(np.abs(a - b) <= TOL_TERM * np.maximum(np.abs(b), 1e-300)), key
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_TERM * abs(ref["Ec"])


def test_ao_energy_mixed_within_microhartree(rpa):
    p = _small()
    ref = oracle.energy(p)
    t = rpa.upload_ao_problem(p)
    with rpa.Context(0) as c:
        r = c.energy(rpa.job_from_ao_problem(p, t, prec=rpa.PREC_MIXED))
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_MIX


def test_ao_chi0_equals_chi0_of_given_coefficients(rpa):
    p = _small()
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    q = 2
    with rpa.Context(0) as c:
        C = c.ao2mo(job, q)
        # the same job with the coefficients given directly (other q unused)
        blocks = [C[j] for j in range(p.n_k)] * p.n_q
        cjob = rpa.Job(is_complex=True, n_aux=p.n_aux, n_occ=p.n_occ, n_virt=p.n_virt, pair_k=p.grid.pair_k,
                       pair_kq=p.grid.pair_kq, w_q=p.grid.w_q, zeta_k=p.grid.zeta_k, omega=p.omega,
                       zeta_w=p.zeta_w, eps_occ=t["eps_occ"], eps_virt=t["eps_virt"], C=blocks, V=t["V"])
        a = c.chi0(job, q).cpu().numpy()
        b = c.chi0(cjob, q).cpu().numpy()
    assert np.array_equal(a, b)


def test_ao2mo_bench_size_sampled(rpa):
    """The benchmark's AO workload (two atoms of 128 basis / 256 fit functions,
    N_occ 32, N_virt 224, 4x4x1 grid): 160 sampled entries per pair of q = 5
    against the oracle, in the same launch configuration the benchmark uses."""
    p = synth.config1_ao()
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    q = 5
    with rpa.Context(0) as c:
        out = c.ao2mo(job, q)
        torch.cuda.synchronize()
    rng = np.random.default_rng(7)
    for j in (0, 7, 15):
        ent = np.stack([rng.integers(0, p.n_aux, 160), rng.integers(0, p.n_ov, 160)], axis=1)
        ent[0] = (p.n_aux - 1, p.n_ov - 1)
        ref = oracle.ao2mo_block(p, q, j, entries=ent)
        g = out[j].cpu().numpy()[ent[:, 0], ent[:, 1]]
        scale = out[j].abs().max().item()
        assert np.abs(g - ref).max() <= TOL_C * scale, j


def test_batch_and_serving_refuse_ao_jobs(rpa):
    p = _small()
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        with pytest.raises(rpa.RpaError) as e:
            c.energy_batch([job])
        assert e.value.status == rpa.RPA_E_INVAL
        with pytest.raises(rpa.RpaError) as e:
            c.submit(job)
        assert e.value.status == rpa.RPA_E_INVAL


# ---- lattice form: k-dependent PADF arrays as lattice sums on the device ----

def _lattice(is_complex=True):
    grid = synth.regular_kq_grid((2, 2, 1)) if is_complex else synth.gamma_grid()
    return synth.make_ao_problem("ao-lat", is_complex=is_complex, n_bas_atom=(20, 14, 9), n_fit_atom=(26, 30, 16),
                                 n_occ=7, n_virt=33, grid=grid, n_w=6, seed=63, lattice=synth.lattice_2d(2))


@pytest.mark.parametrize("is_complex", [True, False])
def test_lattice_form_ao2mo_matches_oracle(rpa, is_complex):
    p = _lattice(is_complex)
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        for q in range(p.n_q):
            out = c.ao2mo(job, q)
            torch.cuda.synchronize()
            _check_blocks(out, p, q)


def test_lattice_form_equals_k_form_given_the_lattice_sums(rpa):
    """Isolates the lattice-sum kernel: the k form fed with the oracle's lattice
    sums must give the lattice form's coefficients to rounding."""
    p = _lattice()
    t = rpa.upload_ao_problem(p)
    jl = rpa.job_from_ao_problem(p, t)
    tk = dict(t, padf=[torch.from_numpy(oracle.padf_of(p, k)).cuda() for k in range(p.n_kpts)], padf_R=None)
    jk = rpa.job_from_ao_problem(synth.AOProblem(p, p.n_bas_atom, p.n_fit_atom), tk)
    with rpa.Context(0) as c:
        for q in (0, 3):
            a = c.ao2mo(jl, q)
            b = c.ao2mo(jk, q)
            torch.cuda.synchronize()
            scale = b.abs().max().item()
            assert (a - b).abs().max().item() <= 1e-13 * scale, q


def test_lattice_form_energy_matches_oracle_fp64(rpa):
    p = _lattice()
    ref = oracle.energy(p)
    t = rpa.upload_ao_problem(p)
    with rpa.Context(0) as c:
        r = c.energy(rpa.job_from_ao_problem(p, t, prec=rpa.PREC_FP64))
    assert np.all(np.abs(r["eps"] - ref["eps"]) <= TOL_TERM * np.abs(ref["eps"]))
    assert abs(r["Ec"] - ref["Ec"]) <= TOL_TERM * abs(ref["Ec"])


# ---- degenerate shapes -------------------------------------------------------

@pytest.mark.parametrize("nb,nf,n_occ,n_virt", [
    ((9,), (13,), 2, 7),              # a single atom: both PADF terms on every fit function
    ((1, 12, 1), (3, 9, 1), 1, 13),   # one-function atoms, one occupied state
    ((6, 6), (5, 5), 11, 1),          # one virtual state
])
def test_ao2mo_degenerate_shapes(rpa, nb, nf, n_occ, n_virt):
    p = synth.make_ao_problem("ao-deg", is_complex=True, n_bas_atom=nb, n_fit_atom=nf, n_occ=n_occ, n_virt=n_virt,
                              grid=synth.regular_kq_grid((2, 1, 1)), n_w=4, seed=64)
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        for q in range(p.n_q):
            out = c.ao2mo(job, q)
            torch.cuda.synchronize()
            _check_blocks(out, p, q)


def test_lattice_form_single_vector(rpa):
    """One lattice vector dR = 0: every k-point's array is the cell-pair array."""
    p = synth.make_ao_problem("ao-lat1", is_complex=True, n_bas_atom=(7, 5), n_fit_atom=(8, 6), n_occ=3, n_virt=9,
                              grid=synth.regular_kq_grid((2, 2, 1)), n_w=4, seed=65,
                              lattice=np.zeros((1, 3), np.int32))
    t = rpa.upload_ao_problem(p)
    job = rpa.job_from_ao_problem(p, t)
    with rpa.Context(0) as c:
        out = c.ao2mo(job, 1)
        torch.cuda.synchronize()
    _check_blocks(out, p, 1)
