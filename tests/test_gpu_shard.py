"""The library-backed q-sharding on one GPU: the q-blocks of two ranks are
computed one after another through shard.gpu_rows over shard.sub_job, and the
assembled integrand table and E_c must equal the unsharded rpa_energy bit for
bit on the FP64 path (each (q, omega) term runs the same kernels on the same
inputs; the table is summed in a fixed order), and within the split path's
1e-9 Ha of it on the mixed path.  The multi-rank exchange itself is covered
by the gloo tests on CPU."""
import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import shard, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rpa():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import paper_2505_06021_gb300 as m
    from paper_2505_06021_gb300 import build as b

    b.build()
    return m


def _sharded(ctx, job, world):
    """Each rank's rows as energy_sharded computes them (its q-block through
    gpu_rows over sub_job), summed as the all-reduce of the ranks' tables
    would, then the fixed-order quadrature."""
    n_q, n_w = job.s.n_q, job.s.n_w
    rows = shard.gpu_rows(ctx, job)
    table = np.zeros((n_q, n_w))
    for qs in shard.q_blocks(n_q, world):
        part = np.zeros((n_q, n_w))
        if len(qs):
            part[qs[0]:qs[-1] + 1] = rows(list(qs))
        table += part
    return shard.quadrature(table, job.w_q, job.zeta_w), table


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_equals_unsharded_fp64(rpa, world):
    p = synth.make_problem("sh", is_complex=True, n_aux=72, n_occ=3, n_virt=10, grid=synth.regular_kq_grid((3, 2, 1)),
                           n_w=5, seed=71)
    job = rpa.job_from_problem(p, rpa.upload_problem(p))
    with rpa.Context(0) as c:
        full = c.energy(job)
        Ec, table = _sharded(c, job, world)
    assert np.array_equal(table, full["eps"])
    assert Ec == pytest.approx(full["Ec"], rel=1e-14)
    ref = oracle.energy(p)
    assert np.max(np.abs(table - ref["eps"]) / np.abs(ref["eps"])) <= 1e-10


def test_sharded_mixed_close_to_unsharded(rpa):
    p = synth.make_problem("shm", is_complex=True, n_aux=96, n_occ=3, n_virt=12,
                           grid=synth.regular_kq_grid((2, 2, 1)), n_w=4, seed=72)
    job = rpa.job_from_problem(p, rpa.upload_problem(p), prec=rpa.PREC_MIXED)
    # per-frequency chi0: the frequency-batched plan depends on the q-points of the (sub-)job
    with rpa.Context(0, chi0_freq=1) as c:
        full = c.energy(job)
        Ec, table = _sharded(c, job, 2)
    assert abs(Ec - full["Ec"]) <= 1e-9
    assert np.max(np.abs(table - full["eps"]) / np.abs(full["eps"])) <= 1e-8
