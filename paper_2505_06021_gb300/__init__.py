"""Python binding of librpa (GB300 / sm_103a): argument marshalling only.

Every step of the RPA hot path runs in the library's CUDA kernels; this
module builds the ``rpa_job`` descriptors of ``include/rpa.h`` from device
(or pinned host) tensors and calls the C ABI through ctypes.  PyTorch is used
for device memory and streams.  If the compiled library is missing, importing
the binding's entry points raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "librpa.so")

RPA_OK, RPA_E_INVAL, RPA_E_NOMEM, RPA_E_CUDA, RPA_E_NOTPD, RPA_E_TIMEOUT, RPA_E_BUSY, RPA_E_NOTREADY = range(8)
PREC_FP64, PREC_MIXED = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
FREQ_MAX_BINS = 32  # RPA_FREQ_MAX_BINS: energy bins of the frequency-batched chi0 at most

STATUS_NAMES = {0: "OK", 1: "INVAL", 2: "NOMEM", 3: "CUDA", 4: "NOTPD", 5: "TIMEOUT", 6: "BUSY", 7: "NOTREADY"}

# Entry points declared in include/rpa.h
EXPORTS = ("rpa_create", "rpa_destroy", "rpa_last_error", "rpa_job_validate", "rpa_job_footprint", "rpa_freq_plan",
           "rpa_chi0",
           "rpa_ao2mo", "rpa_projector", "rpa_logdet", "rpa_energy", "rpa_energy_batch", "rpa_submit", "rpa_poll",
           "rpa_wait",
           "rpa_serving_stats", "rpa_serving_peak", "rpa_test_drop_copy", "rpa_kernel_launches", "rpa_stream",
           "rpa_profile", "rpa_profile_read", "rpa_profile_counters", "rpa_logdet_noalloc",
           "rpa_noalloc_last_error")

# kernel classes of rpa_profile_read
KERNEL_CLASSES = ("dtab", "chi0", "vfactor", "sandwich", "logdet", "reduce", "slice", "chi0_reduce", "ao2mo",
                  "proj", "h2d")


class RpaError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


class rpa_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_cap_bytes", ctypes.c_size_t), ("n_slices", ctypes.c_int),
                ("timeout_s", ctypes.c_double), ("max_inflight", ctypes.c_int), ("chi0_freq", ctypes.c_int)]


class rpa_ao(ctypes.Structure):
    _fields_ = [("n_atoms", ctypes.c_int), ("n_bas_atom", ctypes.POINTER(ctypes.c_int)),
                ("n_fit_atom", ctypes.POINTER(ctypes.c_int)), ("n_mo", ctypes.c_int),
                ("padf", ctypes.POINTER(ctypes.c_void_p)), ("mo", ctypes.POINTER(ctypes.c_void_p)),
                ("n_R", ctypes.c_int), ("lattice", ctypes.POINTER(ctypes.c_int)),
                ("kfrac", ctypes.POINTER(ctypes.c_double)), ("padf_R", ctypes.POINTER(ctypes.c_void_p)),
                ("overlap", ctypes.POINTER(ctypes.c_void_p)), ("eps_d", ctypes.c_double)]


class rpa_job(ctypes.Structure):
    _fields_ = [("is_complex", ctypes.c_int), ("n_aux", ctypes.c_int), ("n_occ", ctypes.c_int),
                ("n_virt", ctypes.c_int), ("n_q", ctypes.c_int), ("n_k", ctypes.c_int), ("n_w", ctypes.c_int),
                ("n_kpts", ctypes.c_int), ("pair_k", ctypes.POINTER(ctypes.c_int)),
                ("pair_kq", ctypes.POINTER(ctypes.c_int)), ("w_q", ctypes.POINTER(ctypes.c_double)),
                ("zeta_k", ctypes.c_double), ("omega", ctypes.POINTER(ctypes.c_double)),
                ("zeta_w", ctypes.POINTER(ctypes.c_double)), ("eps_occ", ctypes.c_void_p),
                ("eps_virt", ctypes.c_void_p), ("C", ctypes.POINTER(ctypes.c_void_p)),
                ("V", ctypes.POINTER(ctypes.c_void_p)), ("prec", ctypes.c_int), ("mem", ctypes.c_int),
                ("ao", ctypes.POINTER(rpa_ao))]


_lib = None


def load_library(path: str = LIB_PATH):
    """Load librpa.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("librpa.so not built at %s: run `python -c 'import __graft_entry__ as g; g.build()'`" % path)
    lib = ctypes.CDLL(path)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    J = ctypes.POINTER(rpa_job)
    u64 = ctypes.c_uint64
    sig = {
        "rpa_create": (I, [ctypes.POINTER(rpa_config), ctypes.POINTER(P)]),
        "rpa_destroy": (I, [P]),
        "rpa_last_error": (ctypes.c_char_p, [P]),
        "rpa_job_validate": (I, [J, ctypes.c_char_p, S]),
        "rpa_job_footprint": (I, [J, ctypes.POINTER(S)]),
        "rpa_freq_plan": (I, [J, I, ctypes.POINTER(I), ctypes.POINTER(D), ctypes.POINTER(I), ctypes.POINTER(I),
                              ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "rpa_chi0": (I, [P, J, I, P, P]),
        "rpa_ao2mo": (I, [P, J, I, P, P]),
        "rpa_projector": (I, [P, J, ctypes.POINTER(P), ctypes.POINTER(D), ctypes.POINTER(I), P]),
        "rpa_logdet": (I, [P, J, I, P, ctypes.POINTER(D), P]),
        "rpa_energy": (I, [P, J, ctypes.POINTER(D), ctypes.POINTER(D), ctypes.POINTER(D)]),
        "rpa_energy_batch": (I, [P, J, I, ctypes.POINTER(D)]),
        "rpa_submit": (I, [P, J, ctypes.POINTER(u64)]),
        "rpa_poll": (I, [P, u64, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "rpa_wait": (I, [P, u64, D, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "rpa_serving_stats": (I, [P, ctypes.POINTER(u64)] + [ctypes.POINTER(D)] * 5),
        "rpa_serving_peak": (I, [P, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(I)]),
        "rpa_test_drop_copy": (I, [P, I]),
        "rpa_kernel_launches": (u64, [P]),
        "rpa_stream": (P, [P]),
        "rpa_profile": (I, [P, I]),
        "rpa_profile_read": (I, [P, ctypes.POINTER(D), ctypes.POINTER(u64)]),
        "rpa_profile_counters": (I, [P, ctypes.POINTER(u64), ctypes.POINTER(u64)]),
        "rpa_logdet_noalloc": (I, [I, I, I, P, P, P, P]),
        "rpa_noalloc_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype, f.argtypes = res, args
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class Job:
    """An ``rpa_job`` plus the host arrays and tensors it points to (kept
    alive with the descriptor).

    ``C`` is a list (length n_q*n_k, q-major) of tensors [n_aux, n_occ*n_virt]
    and ``V`` a list of n_q tensors [n_aux, n_aux], complex128 or float64, all
    on the device (mem=MEM_DEVICE) or all in host memory (mem=MEM_HOST,
    pinned for speed).  ``eps_occ`` [n_kpts, n_occ], ``eps_virt`` [n_kpts,
    n_virt] float64 tensors in the same memory.

    AO form (``ao`` given, ``C`` None): ``ao`` is a dict with ``n_bas_atom``,
    ``n_fit_atom`` (per atom), and the per-k-point device tensors ``padf``
    [n_bas, S] and ``mo`` [n_bas, n_mo] (layouts of ``rpa_ao``); lattice form:
    ``padf`` None and ``padf_R`` (real [n_bas, S] per lattice vector),
    ``lattice`` [n_R, 3] integers and ``kfrac`` [n_kpts, 3]; projector:
    ``overlap`` (device [n_bas, n_bas] per k-point) and ``eps_d``."""

    def __init__(self, *, is_complex: bool, n_aux: int, n_occ: int, n_virt: int, pair_k, pair_kq, w_q, zeta_k: float,
                 omega, zeta_w, eps_occ, eps_virt, C: Optional[Sequence], V: Sequence, prec: int = PREC_FP64,
                 mem: int = MEM_DEVICE, ao: Optional[Dict[str, object]] = None):
        self.pair_k = np.array(pair_k, np.int32).reshape(-1)
        self.pair_kq = np.array(pair_kq, np.int32).reshape(-1)
        self.w_q = np.array(w_q, np.float64).reshape(-1)
        self.omega = np.array(omega, np.float64).reshape(-1)
        self.zeta_w = np.array(zeta_w, np.float64).reshape(-1)
        n_q = int(self.w_q.shape[0])
        n_k = int(self.pair_k.shape[0] // n_q)
        self.C_t, self.V_t = list(C or []), list(V)
        self.eps_occ_t, self.eps_virt_t = eps_occ, eps_virt
        self._Cp = (ctypes.c_void_p * len(self.C_t))(*[int(c.data_ptr()) for c in self.C_t])
        self._Vp = (ctypes.c_void_p * len(self.V_t))(*[int(v.data_ptr()) for v in self.V_t])
        s = rpa_job()
        s.is_complex, s.n_aux, s.n_occ, s.n_virt = int(is_complex), n_aux, n_occ, n_virt
        s.n_q, s.n_k, s.n_w, s.n_kpts = n_q, n_k, int(self.omega.shape[0]), int(eps_occ.shape[0])
        s.pair_k = self.pair_k.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        s.pair_kq = self.pair_kq.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        s.w_q, s.zeta_k = _dptr(self.w_q), float(zeta_k)
        s.omega, s.zeta_w = _dptr(self.omega), _dptr(self.zeta_w)
        s.eps_occ, s.eps_virt = int(eps_occ.data_ptr()), int(eps_virt.data_ptr())
        s.C = ctypes.cast(self._Cp, ctypes.POINTER(ctypes.c_void_p)) if self.C_t else None
        s.V = ctypes.cast(self._Vp, ctypes.POINTER(ctypes.c_void_p))
        s.prec, s.mem = int(prec), int(mem)
        self.ao_t = ao
        if ao is not None:
            self._nb = np.array(ao["n_bas_atom"], np.int32)
            self._nf = np.array(ao["n_fit_atom"], np.int32)
            padf = ao.get("padf") or []
            self._Pp = (ctypes.c_void_p * max(1, len(padf)))(*[int(t.data_ptr()) for t in padf])
            self._Mp = (ctypes.c_void_p * len(ao["mo"]))(*[int(t.data_ptr()) for t in ao["mo"]])
            a = rpa_ao()
            a.n_atoms = int(self._nb.shape[0])
            a.n_bas_atom = self._nb.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            a.n_fit_atom = self._nf.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
            a.n_mo = int(ao["mo"][0].shape[1])
            a.padf = ctypes.cast(self._Pp, ctypes.POINTER(ctypes.c_void_p)) if padf else None
            a.mo = ctypes.cast(self._Mp, ctypes.POINTER(ctypes.c_void_p))
            if ao.get("padf_R") is not None:
                self._lat = np.ascontiguousarray(ao["lattice"], np.int32).reshape(-1)
                self._kf = np.ascontiguousarray(ao["kfrac"], np.float64).reshape(-1)
                self._Rp = (ctypes.c_void_p * len(ao["padf_R"]))(*[int(t.data_ptr()) for t in ao["padf_R"]])
                a.n_R = len(ao["padf_R"])
                a.lattice = self._lat.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
                a.kfrac = _dptr(self._kf)
                a.padf_R = ctypes.cast(self._Rp, ctypes.POINTER(ctypes.c_void_p))
            if ao.get("overlap") is not None:
                self._Op = (ctypes.c_void_p * len(ao["overlap"]))(*[int(t.data_ptr()) for t in ao["overlap"]])
                a.overlap = ctypes.cast(self._Op, ctypes.POINTER(ctypes.c_void_p))
                a.eps_d = float(ao["eps_d"])
            self._ao = a
            s.ao = ctypes.pointer(a)
        self.s = s

    @property
    def n_q(self):
        return self.s.n_q

    @property
    def n_w(self):
        return self.s.n_w

    def with_prec(self, prec: int) -> "Job":
        j = Job.__new__(Job)
        j.__dict__.update(self.__dict__)
        s = rpa_job.from_buffer_copy(self.s)
        s.prec = int(prec)
        j.s = s
        return j

    def validate(self) -> Tuple[int, str]:
        buf = ctypes.create_string_buffer(512)
        st = load_library().rpa_job_validate(ctypes.byref(self.s), buf, 512)
        return st, buf.value.decode()

    def freq_plan(self, mode: int = 0) -> Dict[str, object]:
        """rpa_freq_plan (host-only; needs a MEM_HOST job): the frequency
        factorisation of the split-precision chi0."""
        nb = ctypes.c_int()
        nw = self.s.n_w
        edges = np.zeros(FREQ_MAX_BINS)
        rank = np.zeros(FREQ_MAX_BINS, np.int32)
        skel = np.zeros(FREQ_MAX_BINS * nw, np.int32)
        coef = np.zeros(FREQ_MAX_BINS * nw * nw)
        err = np.zeros(FREQ_MAX_BINS)
        wr = ctypes.c_double()
        ip = ctypes.POINTER(ctypes.c_int)
        st = load_library().rpa_freq_plan(ctypes.byref(self.s), int(mode), ctypes.byref(nb), _dptr(edges),
                                          rank.ctypes.data_as(ip), skel.ctypes.data_as(ip), _dptr(coef), _dptr(err),
                                          ctypes.byref(wr))
        if st:
            raise RpaError(st, "rpa_freq_plan failed")
        n = int(nb.value)
        return {"n_bins": n, "edges": edges[:max(0, n - 1)].copy(), "rank": rank[:n].copy(),
                "skel": skel.reshape(FREQ_MAX_BINS, nw)[:n].copy(), "coef": coef.reshape(FREQ_MAX_BINS, nw, nw)[:n].copy(),
                "err": err[:n].copy(), "work_ratio": float(wr.value)}

    def footprint(self) -> int:
        out = ctypes.c_size_t()
        st = load_library().rpa_job_footprint(ctypes.byref(self.s), ctypes.byref(out))
        if st:
            raise RpaError(st, self.validate()[1])
        return int(out.value)


def job_from_problem(problem, tensors: Dict[str, object], prec: int = PREC_FP64, mem: int = MEM_DEVICE) -> Job:
    g = problem.grid
    return Job(is_complex=problem.is_complex, n_aux=problem.n_aux, n_occ=problem.n_occ, n_virt=problem.n_virt,
               pair_k=g.pair_k, pair_kq=g.pair_kq, w_q=g.w_q, zeta_k=g.zeta_k, omega=problem.omega,
               zeta_w=problem.zeta_w, eps_occ=tensors["eps_occ"], eps_virt=tensors["eps_virt"], C=tensors["C"],
               V=tensors["V"], prec=prec, mem=mem)


def job_from_ao_problem(problem, tensors: Dict[str, object], prec: int = PREC_FP64) -> Job:
    """Job of an AO-form synthetic problem (``synth.AOProblem``) from
    :func:`upload_ao_problem`'s tensors."""
    g = problem.grid
    ao = {"n_bas_atom": problem.n_bas_atom, "n_fit_atom": problem.n_fit_atom, "padf": tensors.get("padf"),
          "mo": tensors["mo"]}
    if tensors.get("padf_R") is not None:
        ao.update(padf_R=tensors["padf_R"], lattice=problem.lattice, kfrac=problem.grid.kpts)
    if tensors.get("overlap") is not None:
        ao.update(overlap=tensors["overlap"], eps_d=problem.eps_d)
    return Job(is_complex=problem.is_complex, n_aux=problem.n_aux, n_occ=problem.n_occ, n_virt=problem.n_virt,
               pair_k=g.pair_k, pair_kq=g.pair_kq, w_q=g.w_q, zeta_k=g.zeta_k, omega=problem.omega,
               zeta_w=problem.zeta_w, eps_occ=tensors["eps_occ"], eps_virt=tensors["eps_virt"], C=None,
               V=tensors["V"], prec=prec, mem=MEM_DEVICE, ao=ao)


def upload_ao_problem(problem, device="cuda", threads: int = 0):
    """Device tensors of an AO-form problem: PADF (or, lattice form, cell-pair
    coefficients per lattice vector) and MO arrays per k-point, V per q, band
    energies."""
    import concurrent.futures as cf

    import torch

    dev = torch.device(device)
    if dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())

    def put(a):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dev)

    nthr = threads or min(16, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(nthr) as ex:
        lat = getattr(problem, "lattice", None) is not None
        padf = None if lat else list(ex.map(lambda k: put(problem.padf(k)), range(problem.n_kpts)))
        padf_R = list(ex.map(lambda r: put(problem.padf_R(r)), range(len(problem.lattice)))) if lat else None
        mo = list(ex.map(lambda k: put(problem.mo(k)), range(problem.n_kpts)))
        V = list(ex.map(lambda q: put(problem.V(q)), range(problem.n_q)))
        ovl = None
        if getattr(problem, "eps_d", None) is not None:
            ovl = list(ex.map(lambda k: put(problem.overlap(k)[0]), range(problem.n_kpts)))
    return {"padf": padf, "padf_R": padf_R, "mo": mo, "V": V, "overlap": ovl,
            "eps_occ": put(problem.eps_occ.astype(np.float64)), "eps_virt": put(problem.eps_virt.astype(np.float64))}


def upload_problem(problem, device="cuda", qs: Optional[Sequence[int]] = None, pin: bool = False,
                   threads: int = 0):
    """Materialise a synthetic problem's inputs as torch tensors on `device`
    (a CUDA device, or host memory with device='cpu'; pinned with pin=True).
    Blocks are generated by a thread pool (each block has its own seeded
    stream, so the result does not depend on the thread count)."""
    import concurrent.futures as cf

    import torch

    dt = torch.complex128 if problem.is_complex else torch.float64
    npdt = np.complex128 if problem.is_complex else np.float64
    qs = list(range(problem.n_q)) if qs is None else list(qs)
    on_host = str(device) == "cpu"
    dev = None if on_host else torch.device(device)
    if dev is not None and dev.index is None:
        dev = torch.device("cuda", torch.cuda.current_device())

    def put(a):
        t = torch.from_numpy(np.ascontiguousarray(a))
        if on_host:
            return t.pin_memory() if pin else t
        return t.to(dev)

    blocks = [(q, j) for q in qs for j in range(problem.n_k)]
    # host inputs: one allocation for all blocks (pinned once, contiguous),
    # the blocks are views of it
    big = torch.empty((len(blocks), problem.n_aux, problem.n_ov), dtype=dt, pin_memory=pin) if on_host else None
    index = {qj: i for i, qj in enumerate(blocks)}

    def make_c(qj):
        q, j = qj
        if on_host:
            t = big[index[qj]]
            problem.C(q, j, out=t.numpy())
            return t
        h = np.empty((problem.n_aux, problem.n_ov), npdt)
        problem.C(q, j, out=h)
        return torch.from_numpy(h).to(dev)

    nthr = threads or min(16, os.cpu_count() or 4)
    with cf.ThreadPoolExecutor(nthr) as ex:
        C = list(ex.map(make_c, blocks))
        V = list(ex.map(lambda q: put(problem.V(q)), qs))
    eo = put(problem.eps_occ.astype(np.float64))
    ev = put(problem.eps_virt.astype(np.float64))
    return {"C": C, "V": V, "eps_occ": eo, "eps_virt": ev}


def logdet_noalloc(is_complex: bool, n_aux: int, n_w: int, V, chi, out, stream=None) -> None:
    """rpa_logdet_noalloc: the log-det step with the library's static scratch
    (no device allocation).  V, chi and out are contiguous device tensors of
    the current device: V [n_aux, n_aux] and chi [n_w, n_aux, n_aux] in
    complex128 (is_complex) or float64, out float64 with 2 n_w elements."""
    import torch

    dt = torch.complex128 if is_complex else torch.float64
    dev = torch.cuda.current_device()
    for name, t, want, n in (("V", V, dt, n_aux * n_aux), ("chi", chi, dt, n_w * n_aux * n_aux),
                             ("out", out, torch.float64, 2 * n_w)):
        if not t.is_cuda or t.device.index != dev:
            raise ValueError("%s must be a tensor on the current CUDA device %d" % (name, dev))
        if t.dtype != want or not t.is_contiguous() or t.numel() < n:
            raise ValueError("%s must be a contiguous %s tensor of at least %d elements" % (name, want, n))
    lib = load_library()
    st_ptr = (stream or torch.cuda.current_stream()).cuda_stream
    st = lib.rpa_logdet_noalloc(int(is_complex), int(n_aux), int(n_w), ctypes.c_void_p(V.data_ptr()),
                                ctypes.c_void_p(chi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(st_ptr))
    if st:
        raise RpaError(st, lib.rpa_noalloc_last_error().decode())


class Context:
    """An ``rpa_ctx`` on one device."""

    def __init__(self, device: int = 0, hbm_cap_bytes: int = 0, n_slices: int = 0, timeout_s: float = 0.0,
                 max_inflight: int = 0, chi0_freq: int = 0):
        self.lib = load_library()
        cfg = rpa_config(device, hbm_cap_bytes, n_slices, timeout_s, max_inflight, chi0_freq)
        h = ctypes.c_void_p()
        st = self.lib.rpa_create(ctypes.byref(cfg), ctypes.byref(h))
        if st:
            raise RpaError(st, self.lib.rpa_last_error(None).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.rpa_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, st):
        if st:
            raise RpaError(st, self.lib.rpa_last_error(self.h).decode())

    @property
    def launches(self) -> int:
        return int(self.lib.rpa_kernel_launches(self.h))

    @property
    def stream_handle(self) -> int:
        """cudaStream_t of the context's compute stream (rpa_energy runs there)."""
        return int(self.lib.rpa_stream(self.h) or 0)

    def profile(self, enable: bool = True):
        self._check(self.lib.rpa_profile(self.h, int(enable)))

    def profile_read(self) -> Dict[str, Tuple[float, int]]:
        ms = (ctypes.c_double * len(KERNEL_CLASSES))()
        n = (ctypes.c_uint64 * len(KERNEL_CLASSES))()
        self._check(self.lib.rpa_profile_read(self.h, ms, n))
        return {k: (ms[i], int(n[i])) for i, k in enumerate(KERNEL_CLASSES)}

    def profile_counters(self) -> Dict[str, int]:
        """Tensor-core flops issued (process wide) and host -> device bytes
        staged by this context since profiling was switched on."""
        f = ctypes.c_uint64()
        h = ctypes.c_uint64()
        self._check(self.lib.rpa_profile_counters(self.h, ctypes.byref(f), ctypes.byref(h)))
        return {"tensor_flops": int(f.value), "h2d_bytes": int(h.value)}

    def chi0(self, job: Job, q: int, out=None, stream=None):
        import torch

        n = job.s.n_aux
        if out is None:
            dt = torch.complex128 if job.s.is_complex else torch.float64
            out = torch.empty((job.s.n_w, n, n), dtype=dt, device="cuda")
        st_ptr = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.rpa_chi0(self.h, ctypes.byref(job.s), int(q), ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(st_ptr)))
        return out

    def ao2mo(self, job: Job, q: int, out=None, stream=None):
        """MO-basis fit coefficients of q for an AO-form job: [n_k, n_aux,
        n_occ*n_virt] device tensor."""
        import torch

        if out is None:
            dt = torch.complex128 if job.s.is_complex else torch.float64
            out = torch.empty((job.s.n_k, job.s.n_aux, job.s.n_occ * job.s.n_virt), dtype=dt, device="cuda")
        st_ptr = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.rpa_ao2mo(self.h, ctypes.byref(job.s), int(q), ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(st_ptr)))
        return out

    def projector(self, job: Job, out=None, stream=None):
        """Periodic projector of an AO-form job with overlaps: (list of c~
        device tensors per k-point, removed directions m, eigenvalues [n_kpts,
        n_bas] ascending)."""
        import torch

        mo = job.ao_t["mo"]
        if out is None:
            out = [torch.empty_like(t) for t in mo]
        ptrs = (ctypes.c_void_p * len(out))(*[int(t.data_ptr()) for t in out])
        n_bas = int(mo[0].shape[0])
        eig = np.zeros((len(out), n_bas))
        m = ctypes.c_int()
        st_ptr = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.rpa_projector(self.h, ctypes.byref(job.s), ptrs, _dptr(eig), ctypes.byref(m),
                                           ctypes.c_void_p(st_ptr)))
        return out, int(m.value), eig

    def logdet(self, job: Job, q: int, chi, stream=None) -> np.ndarray:
        import torch

        out = np.zeros(2 * job.s.n_w)
        st_ptr = (stream or torch.cuda.current_stream()).cuda_stream
        self._check(self.lib.rpa_logdet(self.h, ctypes.byref(job.s), int(q), ctypes.c_void_p(chi.data_ptr()),
                                        _dptr(out), ctypes.c_void_p(st_ptr)))
        return out.reshape(job.s.n_w, 2)

    def energy(self, job: Job) -> Dict[str, object]:
        nqw = job.s.n_q * job.s.n_w
        Ec = ctypes.c_double()
        eps = np.zeros(nqw)
        parts = np.zeros(2 * nqw)
        self._check(self.lib.rpa_energy(self.h, ctypes.byref(job.s), ctypes.byref(Ec), _dptr(eps), _dptr(parts)))
        parts = parts.reshape(job.s.n_q, job.s.n_w, 2)
        return {"Ec": Ec.value, "eps": eps.reshape(job.s.n_q, job.s.n_w), "lndet": parts[..., 0],
                "trPi": parts[..., 1]}

    def energy_batch(self, jobs: Sequence[Job]) -> np.ndarray:
        arr = (rpa_job * len(jobs))(*[j.s for j in jobs])
        out = np.zeros(len(jobs))
        self._check(self.lib.rpa_energy_batch(self.h, arr, len(jobs), _dptr(out)))
        return out

    def submit(self, job: Job) -> int:
        t = ctypes.c_uint64()
        self._check(self.lib.rpa_submit(self.h, ctypes.byref(job.s), ctypes.byref(t)))
        return int(t.value)

    def poll(self, ticket: int, job: Optional[Job] = None):
        Ec = ctypes.c_double()
        eps = np.zeros(job.s.n_q * job.s.n_w) if job is not None else None
        st = self.lib.rpa_poll(self.h, ctypes.c_uint64(ticket), ctypes.byref(Ec),
                               _dptr(eps) if eps is not None else None)
        if st == RPA_E_NOTREADY:
            return None
        self._check(st)
        return Ec.value, eps

    def wait(self, ticket: int, timeout_s: float = 60.0, job: Optional[Job] = None):
        Ec = ctypes.c_double()
        eps = np.zeros(job.s.n_q * job.s.n_w) if job is not None else None
        self._check(self.lib.rpa_wait(self.h, ctypes.c_uint64(ticket), float(timeout_s), ctypes.byref(Ec),
                                      _dptr(eps) if eps is not None else None))
        return Ec.value, eps

    def serving_stats(self) -> Dict[str, float]:
        n = ctypes.c_uint64()
        v = [ctypes.c_double() for _ in range(5)]
        self._check(self.lib.rpa_serving_stats(self.h, ctypes.byref(n), *[ctypes.byref(x) for x in v]))
        return {"jobs_done": int(n.value), "lat_mean_s": v[0].value, "lat_p50_s": v[1].value,
                "lat_p99_s": v[2].value, "wait_p50_s": v[3].value, "wait_p99_s": v[4].value}

    def test_drop_copy(self, item: int) -> None:
        """Test hook: the next split-precision chi0 launch leaves work item
        `item`'s operand copies unissued; the call then reports a time-out."""
        self._check(self.lib.rpa_test_drop_copy(self.h, int(item)))

    def serving_peak(self) -> Dict[str, int]:
        r = ctypes.c_int()
        b = ctypes.c_size_t()
        m = ctypes.c_int()
        self._check(self.lib.rpa_serving_peak(self.h, ctypes.byref(r), ctypes.byref(b), ctypes.byref(m)))
        return {"max_running": int(r.value), "max_bytes": int(b.value), "max_batch": int(m.value)}
