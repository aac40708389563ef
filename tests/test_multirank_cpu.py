"""Multi-rank host logic on CPU: q-block sharding of one job over world_size 2
gloo ranks, with the oracle standing in for each rank's GPU, must reproduce the
single-process energy; the final quadrature is identical on every rank."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2505_06021_gb300 import shard, synth


def _problem():
    return synth.make_problem("mr", is_complex=True, n_aux=14, n_occ=2, n_virt=4,
                              grid=synth.regular_kq_grid((3, 1, 1)), n_w=5, seed=61)


def _rows_oracle(p):
    def rows(qs):
        r = oracle.energy(p, qs=qs)
        return r["eps"][list(qs)]

    return rows


def test_q_blocks_cover_once():
    for n_q in (1, 2, 5, 16, 17):
        for world in (1, 2, 3, 8):
            blocks = shard.q_blocks(n_q, world)
            flat = [q for b in blocks for q in b]
            assert flat == list(range(n_q))
            sizes = [len(b) for b in blocks]
            assert max(sizes) - min(sizes) <= 1


def test_quadrature_matches_oracle_sum():
    p = _problem()
    ref = oracle.energy(p)
    assert shard.quadrature(ref["eps"], p.grid.w_q, p.zeta_w) == pytest.approx(ref["Ec"], rel=1e-14)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = _problem()
    Ec, table = shard.energy_sharded(p.n_q, p.n_w, p.grid.w_q, p.zeta_w, _rows_oracle(p), rank, world)
    out[rank] = (Ec, table)
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    import torch.multiprocessing as mp

    world = 2
    port = _free_port()
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    p = _problem()
    ref = oracle.energy(p)
    E0, t0 = out[0]
    E1, t1 = out[1]
    assert E0 == E1
    assert np.array_equal(t0, t1)
    assert np.allclose(t0, ref["eps"], rtol=1e-13, atol=0)
    assert E0 == pytest.approx(ref["Ec"], rel=1e-13)


def test_block_job_equals_sub_job_of_the_whole():
    """A rank's q-block job built from only its own uploaded blocks (the
    q-sharded benchmark mode) describes the same job as the whole job
    restricted to those q-points."""
    torch = pytest.importorskip("torch")
    import paper_2505_06021_gb300 as rpa

    p = synth.make_problem("bj", is_complex=True, n_aux=10, n_occ=2, n_virt=3,
                           grid=synth.regular_kq_grid((3, 2, 1)), n_w=4, seed=62)
    whole = rpa.job_from_problem(p, rpa.upload_problem(p, "cpu"), prec=rpa.PREC_FP64, mem=rpa.MEM_HOST)
    for world in (2, 4):
        for qs in shard.q_blocks(p.n_q, world):
            qs = list(qs)
            a = shard.sub_job(whole, qs)
            b = shard.block_job(p, rpa.upload_problem(p, "cpu", qs=qs), qs, rpa.PREC_FP64, rpa.MEM_HOST)
            assert np.array_equal(a.pair_k, b.pair_k) and np.array_equal(a.pair_kq, b.pair_kq)
            assert np.array_equal(a.w_q, b.w_q)
            assert len(a.C_t) == len(b.C_t) == len(qs) * p.n_k
            for x, y in zip(a.C_t + a.V_t, b.C_t + b.V_t):
                assert torch.equal(x, y)
    with pytest.raises(ValueError):
        shard.block_job(p, rpa.upload_problem(p, "cpu", qs=[0]), [0, 1], rpa.PREC_FP64, rpa.MEM_HOST)
