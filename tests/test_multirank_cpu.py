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
