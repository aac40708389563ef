"""rpa_logdet_noalloc, the log-det entry point for callers that cannot
allocate device memory at call time (its scratch is a static device array),
must give the same results as rpa_logdet, call after call.  Kept in a file
that pytest collects last."""
import numpy as np
import pytest

from paper_2505_06021_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # relative, the per-term bar of the FP64 path


def test_noalloc_matches_context_logdet_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as rpa
    from paper_2505_06021_gb300 import build

    build.build()
    p = synth.make_problem("na", is_complex=True, n_aux=150, n_occ=3, n_virt=9,
                           grid=synth.regular_kq_grid((2, 2, 1)), n_w=5, seed=33)
    t = rpa.upload_problem(p)
    job = rpa.job_from_problem(p, t)
    q = 2
    with rpa.Context(0) as ctx:
        chi = ctx.chi0(job, q)
        ref = ctx.logdet(job, q, chi)
    for _ in range(2):
        out = torch.full((p.n_w, 2), float("nan"), dtype=torch.float64, device="cuda")
        rpa.logdet_noalloc(True, p.n_aux, p.n_w, t["V"][q], chi, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        assert np.all(np.abs(got - ref) <= TOL * np.abs(ref)), (got, ref)


def test_noalloc_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as rpa

    V = torch.eye(400, dtype=torch.complex128, device="cuda")
    chi = torch.zeros((1, 400, 400), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 2), dtype=torch.float64, device="cuda")
    with pytest.raises(rpa.RpaError) as e:
        rpa.logdet_noalloc(True, 400, 1, V, chi, out)
    assert e.value.status == rpa.RPA_E_INVAL and "384" in str(e.value)
