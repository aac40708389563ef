"""rpa_logdet_noalloc, the log-det entry point for callers that cannot
allocate device memory at call time (its scratch is a static device array),
must give the same results as rpa_logdet, call after call, and the CPU
oracle's results on the same chi0.  Kept in a file that pytest collects last.

Tolerance: 1e-10 relative per (ln det, Tr Pi), the per-term bar of the FP64
path.  Sizes: n_aux 150 (one CTA per factorisation) and 384, the documented
limit, where a single matrix is factorised on a thread-block cluster; both
complex and real data."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # relative, the per-term bar of the FP64 path


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build

    build.build()
    return m


def _problem(is_complex, n_aux):
    grid = synth.regular_kq_grid((2, 2, 1)) if is_complex else synth.gamma_grid()
    return synth.make_problem("na", is_complex=is_complex, n_aux=n_aux, n_occ=3, n_virt=9, grid=grid, n_w=4,
                              seed=33 + n_aux + int(is_complex))


@pytest.mark.parametrize("is_complex,n_aux", [(True, 150), (True, 384), (False, 384)])
def test_noalloc_matches_logdet_and_oracle_twice(rpa, is_complex, n_aux):
    p = _problem(is_complex, n_aux)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    q = p.n_q - 1
    with rpa.Context(0) as ctx:
        chi = ctx.chi0(job, q)
        ref = ctx.logdet(job, q, chi)
    # the oracle on the same chi0: V^1/2 by Jacobi, the sandwich, the Cholesky log-det
    Vh = oracle.vhalf(p.V(q))
    chi_h = chi.cpu().numpy()
    orc = np.array([oracle.logdet(oracle.sandwich(Vh, chi_h[w])) for w in range(p.n_w)])
    for _ in range(2):
        out = torch.full((p.n_w, 2), float("nan"), dtype=torch.float64, device="cuda")
        rpa.logdet_noalloc(is_complex, p.n_aux, p.n_w, t["V"][q], chi, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL * np.abs(ref)), (got, ref)
        assert np.all(np.abs(got - orc) <= TOL * np.abs(orc)), (got, orc)


def test_noalloc_allocates_nothing(rpa):
    p = _problem(True, 200)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    with rpa.Context(0) as ctx:
        chi = ctx.chi0(job, 0)
    out = torch.zeros((p.n_w, 2), dtype=torch.float64, device="cuda")
    rpa.logdet_noalloc(True, p.n_aux, p.n_w, t["V"][0], chi, out)  # warm-up: address lookup, module load
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        rpa.logdet_noalloc(True, p.n_aux, p.n_w, t["V"][0], chi, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_not_positive_definite_V(rpa):
    p = _problem(True, 300)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    with rpa.Context(0) as ctx:
        chi = ctx.chi0(job, 0)
    Vbad = t["V"][0].clone()
    Vbad[7, 7] = -80.0
    out = torch.zeros((p.n_w, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rpa.RpaError) as e:
        rpa.logdet_noalloc(True, p.n_aux, p.n_w, Vbad, chi, out)
    assert e.value.status == rpa.RPA_E_NOTPD and "V is not positive definite" in str(e.value)
    # and the next call on good inputs is right again
    rpa.logdet_noalloc(True, p.n_aux, p.n_w, t["V"][0], chi, out)
    torch.cuda.synchronize()
    assert np.all(np.isfinite(out.cpu().numpy()))


def test_noalloc_rejects_oversize_and_host_pointers(rpa):
    V = torch.eye(400, dtype=torch.complex128, device="cuda")
    chi = torch.zeros((1, 400, 400), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rpa.RpaError) as e:
        rpa.logdet_noalloc(True, 400, 1, V, chi, out)
    assert e.value.status == rpa.RPA_E_INVAL and "384" in str(e.value)
    # a host output array (rpa_logdet's convention) is refused by the C entry point itself
    lib = rpa.load_library()
    host_out = np.zeros(2)
    V8, chi8 = V[:8, :8].contiguous(), chi[:, :8, :8].contiguous()
    st = lib.rpa_logdet_noalloc(1, 8, 1, ctypes.c_void_p(V8.data_ptr()), ctypes.c_void_p(chi8.data_ptr()),
                                host_out.ctypes.data_as(ctypes.c_void_p), None)
    assert st == rpa.RPA_E_INVAL and b"out" in lib.rpa_noalloc_last_error()
