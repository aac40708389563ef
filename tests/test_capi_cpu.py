"""Host-side checks of the C-ABI library that need no GPU: it builds for
sm_103a, loads, exports every entry point include/rpa.h declares, validates
job descriptors, computes admission footprints, and fails cleanly (no crash)
when no device is present."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2505_06021_gb300 as rpa
from paper_2505_06021_gb300 import build as rbuild
from paper_2505_06021_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    rbuild.build()
    return rpa.load_library()


def _declared():
    txt = open(os.path.join(ROOT, "include", "rpa.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(rpa_[a-z0-9_]+)\s*\(", txt)))


def test_exports_every_declared_symbol(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) == set(rpa.EXPORTS)


class FakeTensor:
    """Stands in for a device tensor: only its address is passed on."""

    def __init__(self, addr, shape=(1,)):
        self.addr, self.shape = addr, shape

    def data_ptr(self):
        return self.addr


def _fake_job(p, **over):
    t = {"C": [FakeTensor(0x10000 + 0x100 * i) for i in range(p.n_q * p.n_k)],
         "V": [FakeTensor(0x90000 + 0x100 * i) for i in range(p.n_q)],
         "eps_occ": FakeTensor(0x1000, p.eps_occ.shape), "eps_virt": FakeTensor(0x2000, p.eps_virt.shape)}
    t.update(over)
    return rpa.job_from_problem(p, t)


def test_validate_accepts_good_jobs(lib):
    for p in (synth.config0(), synth.config1(n_aux=32, n_occ=2, n_virt=5), synth.config2(n_aux=16, n_occ=2,
                                                                                          n_virt=3)):
        st, msg = _fake_job(p).validate()
        assert st == rpa.RPA_OK, msg


def test_validate_rejects_bad_jobs(lib):
    p = synth.config1(n_aux=32, n_occ=2, n_virt=5)
    j = _fake_job(p)
    j.s.n_aux = 0
    assert j.validate()[0] == rpa.RPA_E_INVAL
    j = _fake_job(p)
    j.pair_kq[3] = 10 ** 6
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "out of range" in msg
    j = _fake_job(p)
    j._Cp[5] = None
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "C[5]" in msg
    j = _fake_job(p)
    j.s.prec = 9
    assert j.validate()[0] == rpa.RPA_E_INVAL
    j = _fake_job(p)
    j.omega[2] = float("nan")
    assert j.validate()[0] == rpa.RPA_E_INVAL
    # real data is Gamma-only
    j = _fake_job(p)
    j.s.is_complex = 0
    assert j.validate()[0] == rpa.RPA_E_INVAL


def test_validate_rejects_misaligned_device_pointers(lib):
    """Device-resident C and V are read as whole elements (16 bytes for
    complex128): a pointer off that alignment is refused on the host."""
    p = synth.config1(n_aux=32, n_occ=2, n_virt=5)
    j = _fake_job(p, C=[FakeTensor(0x10008 + 0x100 * i) for i in range(p.n_q * p.n_k)])
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "C[0]" in msg and "aligned" in msg
    j = _fake_job(p, V=[FakeTensor(0x90000 + 0x100 * i + (8 if i == 2 else 0)) for i in range(p.n_q)])
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "V[2]" in msg and "aligned" in msg
    # real (Gamma-only) data needs 8 bytes only
    g = synth.config0()
    j = _fake_job(g, C=[FakeTensor(0x10008 + 0x100 * i) for i in range(g.n_q * g.n_k)])
    assert j.validate()[0] == rpa.RPA_OK


def test_footprint_grows_with_size(lib):
    a = _fake_job(synth.config1(n_aux=64, n_occ=2, n_virt=5)).footprint()
    b = _fake_job(synth.config1(n_aux=128, n_occ=2, n_virt=5)).footprint()
    assert 0 < a < b
    c1 = _fake_job(synth.config1()).footprint()
    # device-resident C of the 2-D periodic workload alone is 15.0 GB
    assert c1 > 15.0e9


def test_create_without_device_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    cfg = rpa.rpa_config(0, 0, 0, 0.0, 0)
    st = lib.rpa_create(ctypes.byref(cfg), ctypes.byref(h))
    assert st == rpa.RPA_E_CUDA
    assert b"device" in lib.rpa_last_error(None)


def _fake_ao_job(p, **over):
    t = {"padf": [FakeTensor(0x200000 + 0x100 * k) for k in range(p.n_kpts)],
         "mo": [FakeTensor(0x300000 + 0x100 * k, (p.n_bas, p.n_mo)) for k in range(p.n_kpts)],
         "V": [FakeTensor(0x90000 + 0x100 * i) for i in range(p.n_q)],
         "eps_occ": FakeTensor(0x1000, p.eps_occ.shape), "eps_virt": FakeTensor(0x2000, p.eps_virt.shape)}
    t.update(over)
    return rpa.job_from_ao_problem(p, t)


def test_validate_ao_jobs(lib):
    p = synth.config1_ao(n_bas_atom=(8, 6), n_fit_atom=(10, 14), n_occ=3, n_virt=9)
    st, msg = _fake_ao_job(p).validate()
    assert st == rpa.RPA_OK, msg
    j = _fake_ao_job(p)
    j._nf[1] = 13  # fit functions no longer sum to n_aux
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "n_aux" in msg
    j = _fake_ao_job(p)
    j._Pp[4] = None
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "NULL" in msg
    j = _fake_ao_job(p)
    j._ao.n_mo = p.n_occ + p.n_virt - 1
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "n_mo" in msg
    j = _fake_ao_job(p)
    j.s.mem = rpa.MEM_HOST
    assert j.validate()[0] == rpa.RPA_E_INVAL


def test_ao_footprint_counts_padf_not_mo_basis_coefficients(lib):
    p = synth.config1_ao()
    fp = _fake_ao_job(p).footprint()
    # PADF arrays of the 16 k-points 4.3 GB + half-transforms 4.3 GB + the
    # MO-basis coefficients of one batch of 4 q (3.8 GB) + the tail's chi0 of
    # all q: the job's 15 GB of C never resides at once
    fc = _fake_job(synth.config1()).footprint()
    assert 9.0e9 < fp < fc
    assert p.padf_bytes() == 16 * 256 * 65536 * 16
    # lattice form: 25 real cell-pair arrays instead of 16 complex k-point arrays
    pl = synth.config1_ao(lattice_radius=2)
    R = [FakeTensor(0x400000 + 0x100 * r) for r in range(len(pl.lattice))]
    fl = _fake_ao_job(pl, padf=None, padf_R=R).footprint()
    assert fl < fp


def test_validate_lattice_form_ao_jobs(lib):
    p = synth.config1_ao(n_bas_atom=(8, 6), n_fit_atom=(10, 14), n_occ=3, n_virt=9, lattice_radius=1)
    R = [FakeTensor(0x400000 + 0x100 * r) for r in range(len(p.lattice))]
    st, msg = _fake_ao_job(p, padf=None, padf_R=R).validate()
    assert st == rpa.RPA_OK, msg
    # both forms at once
    j = _fake_ao_job(p, padf=[FakeTensor(0x200000 + 0x100 * k) for k in range(p.n_kpts)], padf_R=R)
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "not both" in msg
    j = _fake_ao_job(p, padf=None, padf_R=R)
    j._Rp[3] = None
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "padf_R" in msg
    # a real Gamma-only job needs integer k-point coordinates
    g = synth.make_ao_problem("g", is_complex=False, n_bas_atom=(4, 4), n_fit_atom=(6, 6), n_occ=2, n_virt=5,
                              grid=synth.gamma_grid(), n_w=4, seed=3, lattice=synth.lattice_2d(1))
    Rg = [FakeTensor(0x500000 + 0x100 * r) for r in range(len(g.lattice))]
    j = _fake_ao_job(g, padf=None, padf_R=Rg)
    assert j.validate()[0] == rpa.RPA_OK
    j._kf[0] = 0.5
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "integer kfrac" in msg


def test_validate_projector_ao_jobs(lib):
    p = synth.config1_ao(n_bas_atom=(8, 6), n_fit_atom=(10, 14), n_occ=3, n_virt=9)
    p.eps_d = 1e-4
    ovl = [FakeTensor(0x600000 + 0x100 * k) for k in range(p.n_kpts)]
    st, msg = _fake_ao_job(p, overlap=ovl).validate()
    assert st == rpa.RPA_OK, msg
    j = _fake_ao_job(p, overlap=ovl)
    j._Op[2] = None
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "overlap" in msg
    j = _fake_ao_job(p, overlap=ovl)
    j._ao.eps_d = float("nan")
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "eps_d" in msg


def test_mixed_frequency_limit(lib):
    p32 = synth.make_problem("f", is_complex=True, n_aux=16, n_occ=2, n_virt=3, grid=synth.regular_kq_grid((2, 1, 1)),
                             n_w=32, seed=1)
    j = _fake_job(p32)
    j.s.prec = rpa.PREC_MIXED
    assert j.validate()[0] == rpa.RPA_OK
    p33 = synth.make_problem("f", is_complex=True, n_aux=16, n_occ=2, n_virt=3, grid=synth.regular_kq_grid((2, 1, 1)),
                             n_w=33, seed=1)
    j = _fake_job(p33)
    j.s.prec = rpa.PREC_MIXED
    st, msg = j.validate()
    assert st == rpa.RPA_E_INVAL and "32" in msg
    j.s.prec = rpa.PREC_FP64  # the FP64 path has no such limit
    assert j.validate()[0] == rpa.RPA_OK
