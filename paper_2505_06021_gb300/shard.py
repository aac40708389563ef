"""Multi-GPU sharding of one RPA job over its q-points.

The (q, omega) terms of the RPA energy are independent (Sec. 2.6 of the paper:
process groups own (q, omega) pairs and the only communication is one gather
of e_omega).  Here each rank owns a contiguous block of q-points (q-major, so a
rank holds only its own C(q, k) blocks and V(q)), computes its rows of the
integrand table eps[q][w] with the library, and the full table is summed over
ranks on the host (one all-reduce of n_q * n_w doubles).  The final quadrature
E_c = (1/2 pi) sum_w zeta_w sum_q w_q eps[q][w] is done in a fixed order with
compensated sums, so every rank gets the same E_c bit for bit.
"""
from __future__ import annotations

import math
from typing import Callable, List, Optional, Sequence

import numpy as np


def q_blocks(n_q: int, world: int) -> List[range]:
    """Contiguous, balanced q-blocks, one per rank (first ranks get the extra)."""
    base, extra = divmod(n_q, world)
    out, start = [], 0
    for r in range(world):
        n = base + (1 if r < extra else 0)
        out.append(range(start, start + n))
        start += n
    return out


def _neumaier(values) -> float:
    s, c = 0.0, 0.0
    for x in values:
        t = s + x
        c += (s - t) + x if abs(s) >= abs(x) else (x - t) + s
        s = t
    return s + c


def quadrature(eps_qw: np.ndarray, w_q: Sequence[float], zeta_w: Sequence[float]) -> float:
    """E_c from the integrand table, q-sum inside, frequency sum outside."""
    n_q, n_w = eps_qw.shape
    e_w = [_neumaier(w_q[q] * eps_qw[q, w] for q in range(n_q)) for w in range(n_w)]
    return _neumaier(zeta_w[w] * e_w[w] for w in range(n_w)) / (2.0 * math.pi)


def energy_sharded(n_q: int, n_w: int, w_q, zeta_w, compute_rows: Callable[[Sequence[int]], np.ndarray],
                   rank: int, world: int, group=None):
    """Runs `compute_rows(qs)` (-> eps rows [len(qs), n_w]) for this rank's
    q-block, sums the table over ranks and returns (E_c, eps table)."""
    qs = list(q_blocks(n_q, world)[rank])
    table = np.zeros((n_q, n_w), np.float64)
    if qs:
        rows = np.asarray(compute_rows(qs), np.float64)
        table[qs[0]:qs[-1] + 1] = rows
    if world > 1:
        import torch
        import torch.distributed as dist

        t = torch.from_numpy(table)
        if dist.get_backend(group) == "nccl":
            t = t.cuda()
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        table = t.cpu().numpy()
    return quadrature(table, np.asarray(w_q, np.float64), np.asarray(zeta_w, np.float64)), table


def sub_job(job, qs: Sequence[int]):
    """The rpa_job restricted to the q-points `qs` (a contiguous block)."""
    from . import Job

    n_k = job.s.n_k
    sel = [q * n_k + j for q in qs for j in range(n_k)]
    return Job(is_complex=bool(job.s.is_complex), n_aux=job.s.n_aux, n_occ=job.s.n_occ, n_virt=job.s.n_virt,
               pair_k=job.pair_k[sel], pair_kq=job.pair_kq[sel], w_q=job.w_q[list(qs)], zeta_k=job.s.zeta_k,
               omega=job.omega, zeta_w=job.zeta_w, eps_occ=job.eps_occ_t, eps_virt=job.eps_virt_t,
               C=[job.C_t[i] for i in sel], V=[job.V_t[q] for q in qs], prec=job.s.prec, mem=job.s.mem)


def block_job(problem, tensors, qs: Sequence[int], prec: int, mem: int = 0):
    """The job of the q-points `qs` (a contiguous block) of a synthetic
    problem whose tensors hold those q only (``upload_problem(..., qs=qs)``):
    a rank materialises and keeps just its own C(q, k) blocks and V(q)."""
    from . import Job

    g = problem.grid
    n_k = problem.n_k
    sel = [q * n_k + j for q in qs for j in range(n_k)]
    if len(tensors["C"]) != len(sel) or len(tensors["V"]) != len(qs):
        raise ValueError("tensors must hold the C blocks and V of exactly the q-points qs")
    return Job(is_complex=problem.is_complex, n_aux=problem.n_aux, n_occ=problem.n_occ, n_virt=problem.n_virt,
               pair_k=np.asarray(g.pair_k).reshape(-1)[sel],
               pair_kq=np.asarray(g.pair_kq).reshape(-1)[sel], w_q=np.asarray(g.w_q)[list(qs)], zeta_k=g.zeta_k,
               omega=problem.omega, zeta_w=problem.zeta_w, eps_occ=tensors["eps_occ"], eps_virt=tensors["eps_virt"],
               C=tensors["C"], V=tensors["V"], prec=prec, mem=mem)


def gpu_rows(ctx, job) -> Callable[[Sequence[int]], np.ndarray]:
    """compute_rows for energy_sharded backed by the library on this rank's GPU."""

    def rows(qs):
        return ctx.energy(sub_job(job, qs))["eps"]

    return rows
