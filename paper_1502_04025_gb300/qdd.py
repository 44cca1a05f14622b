"""Thin ctypes binding of libqdd (include/qdd.h): argument marshalling only.

Every function keeps the name of its C entry point.  Arrays are accepted as
numpy arrays (host memory) or torch CUDA tensors (device memory, with the
caller's current stream); both use the host layouts of ``qdd.h``:
links (V, 4, 3, 3) complex128 and spinors (V, 4, 3) / (nrhs, V, 4, 3)
complex128.  Every step of the computation runs in the library's CUDA
kernels; there is no fallback: importing this module fails if libqdd.so is
missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# QDD_CHECKED=1 loads the range-checked build of the same library (tests)
LIB_PATH = os.path.join(HERE, "libqdd_check.so" if os.environ.get("QDD_CHECKED") == "1" else "libqdd.so")

(QDD_OK, QDD_EINVAL, QDD_ENOMEM, QDD_EBUDGET, QDD_ENOCONV, QDD_ENAN, QDD_ETIMEOUT, QDD_ECUDA, QDD_ENOTREADY,
 QDD_ECOMM) = range(10)
QDD_PREC_F64, QDD_PREC_F32, QDD_PREC_F16S, QDD_PREC_BF16S, QDD_PREC_DF64, QDD_PREC_H16 = range(6)
PRECS = {"f64": QDD_PREC_F64, "f32": QDD_PREC_F32, "f16": QDD_PREC_F16S, "bf16": QDD_PREC_BF16S,
         "df64": QDD_PREC_DF64, "h16": QDD_PREC_H16}
STATUS_NAMES = ["QDD_OK", "QDD_EINVAL", "QDD_ENOMEM", "QDD_EBUDGET", "QDD_ENOCONV", "QDD_ENAN", "QDD_ETIMEOUT",
                "QDD_ECUDA", "QDD_ENOTREADY", "QDD_ECOMM"]

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{os.path.basename(LIB_PATH)} is not built ({LIB_PATH}); run __graft_entry__.build()")


class qdd_solve_params(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart_m", ctypes.c_int), ("max_restarts", ctypes.c_int),
                ("nmr", ctypes.c_int), ("ncy", ctypes.c_int), ("sap_prec", ctypes.c_int),
                ("arnoldi_prec", ctypes.c_int), ("use_sap", ctypes.c_int), ("nrhs", ctypes.c_int),
                ("reorth", ctypes.c_int), ("relax_eta", ctypes.c_double), ("dr_k", ctypes.c_int)]


class qdd_report(ctypes.Structure):
    _fields_ = [("converged", ctypes.c_int), ("iters", ctypes.c_int), ("restarts", ctypes.c_int),
                ("true_rel_res", ctypes.c_double), ("est_rel_res", ctypes.c_double), ("seconds", ctypes.c_double),
                ("ms_sap", ctypes.c_double), ("ms_dslash", ctypes.c_double), ("ms_blas", ctypes.c_double),
                ("sap_launches", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("deflated_restarts", ctypes.c_int),
                ("n_history", ctypes.c_int), ("res_history", ctypes.POINTER(ctypes.c_double))]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "res_history"}
        d["history"] = [self.res_history[i] for i in range(self.n_history)] if self.res_history else []
        return d


class qdd_mg_params(ctypes.Structure):
    _fields_ = [("nv", ctypes.c_int), ("setup_iters", ctypes.c_int), ("setup_ncy", ctypes.c_int),
                ("nmr", ctypes.c_int), ("post_ncy", ctypes.c_int), ("coarse_iters", ctypes.c_int),
                ("sap_prec", ctypes.c_int), ("bootstrap", ctypes.c_int)]


class qdd_tune_result(ctypes.Structure):
    _fields_ = [("dom", ctypes.c_int * 4), ("nmr", ctypes.c_int),
                ("iters", ctypes.c_int), ("n_tried", ctypes.c_int), ("ms", ctypes.c_double),
                ("wave_load", ctypes.c_double)]


_vp = ctypes.c_void_p

# communication hooks of a sharded lattice (qdd_comm)
ALLREDUCE_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_size_t)
SHIFT_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_void_p, ctypes.c_size_t)


class qdd_comm(ctypes.Structure):
    _fields_ = [("user", ctypes.c_void_p), ("rank", ctypes.c_int), ("size", ctypes.c_int),
                ("allreduce_sum", ALLREDUCE_FN), ("shift", SHIFT_FN)]
_ip = ctypes.POINTER(ctypes.c_int)
_dp = ctypes.POINTER(ctypes.c_double)

_lib = ctypes.CDLL(LIB_PATH)
_SIGS = {
    "qdd_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_size_t]),
    "qdd_destroy": (None, [_vp]),
    "qdd_last_error": (ctypes.c_char_p, []),
    "qdd_set_profiling": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qdd_get_kernel_times": (ctypes.c_int, [_vp, _dp, ctypes.c_int]),
    "qdd_get_kernel_work": (ctypes.c_int, [_vp, _dp]),
    "qdd_memory": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_size_t), ctypes.POINTER(ctypes.c_size_t)]),
    "qdd_measure_fma_peak": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp]),
    "qdd_create_gauge_field": (ctypes.c_int, [_vp, _ip, _ip, _vp, ctypes.c_int, ctypes.POINTER(_vp)]),
    "qdd_destroy_gauge": (None, [_vp]),
    "qdd_create_gauge_field_slab": (ctypes.c_int, [_vp, _ip, _ip, _vp, ctypes.c_int, ctypes.POINTER(qdd_comm),
                                                   ctypes.POINTER(_vp)]),
    "qdd_slab_regions": (ctypes.c_int, [_ip, _ip, ctypes.c_int, _ip]),
    "qdd_layout_faces": (ctypes.c_int, [_ip, _ip, _ip, _vp]),
    "qdd_set_link_compression": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qdd_link_compression": (ctypes.c_int, [_vp, _ip, _ip]),
    "qdd_check_hits": (ctypes.c_int, [ctypes.POINTER(ctypes.c_ulonglong)]),
    "qdd_check_set_wait_limit": (ctypes.c_int, [ctypes.c_int, ctypes.c_uint]),
    "qdd_set_schwarz_variant": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qdd_set_clover": (ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double]),
    "qdd_get_clover": (ctypes.c_int, [_vp, ctypes.c_int, _vp]),
    "qdd_apply_D": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "qdd_sap_apply": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, _vp]),
    "qdd_default_params": (None, [ctypes.POINTER(qdd_solve_params)]),
    "qdd_solve": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, ctypes.POINTER(qdd_solve_params),
                                 ctypes.POINTER(qdd_report), _vp]),
    "qdd_cdot_multi": (ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int64, _vp, ctypes.c_int64, _vp, _vp]),
    "qdd_cdot_multi_noalloc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int64, _vp, ctypes.c_int64, _vp, _vp]),
    "qdd_load_model": (ctypes.c_double, [ctypes.c_double, ctypes.c_double]),
    "qdd_domain_working_set": (ctypes.c_double, [_ip, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "qdd_layout": (ctypes.c_int, [_ip, _ip, _vp, _vp, _vp]),
    "qdd_autotune": (ctypes.c_int, [_vp, _ip, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_int,
                                    ctypes.POINTER(qdd_solve_params), _ip, ctypes.c_int, _ip, ctypes.c_int,
                                    ctypes.POINTER(qdd_tune_result), ctypes.c_char_p, ctypes.c_size_t]),
    "qdd_submit": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.POINTER(qdd_solve_params),
                                  ctypes.POINTER(ctypes.c_uint64)]),
    "qdd_poll": (ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(qdd_report), ctypes.c_double]),
    "qdd_serve_config": (ctypes.c_int, [_vp, ctypes.c_int]),
    "qdd_mg_default_params": (None, [ctypes.POINTER(qdd_mg_params)]),
    "qdd_mg_setup": (ctypes.c_int, [_vp, ctypes.POINTER(qdd_mg_params), _vp, ctypes.c_int]),
    "qdd_mg_vcycle": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_int, _vp]),
    "qdd_mg_get_basis": (ctypes.c_int, [_vp, _vp]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class QddError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.qdd_last_error().decode(errors="replace")
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


def _check(status: int, where: str, ok=(QDD_OK,)):
    if status not in ok:
        raise QddError(status, where)
    return status


def _ivec(v):
    return (ctypes.c_int * 4)(*[int(a) for a in v])


def _prec(p) -> int:
    return PRECS[p] if isinstance(p, str) else int(p)


def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """(pointer, on_device) of a numpy array or a torch CUDA tensor."""
    if _is_torch(a):
        import torch

        assert a.is_contiguous()
        if a.dtype == torch.complex128 or a.dtype == torch.float64:
            return a.data_ptr(), 1 if a.is_cuda else 0
        raise TypeError("torch tensors must be complex128 or float64")
    assert isinstance(a, np.ndarray) and a.flags["C_CONTIGUOUS"], "numpy arrays must be C-contiguous"
    assert a.dtype in (np.complex128, np.float64)
    return a.ctypes.data, 0


def _stream(a=None):
    if a is not None and _is_torch(a) and a.is_cuda:
        import torch

        return torch.cuda.current_stream(a.device).cuda_stream
    return None


def _like(a, shape=None):
    if _is_torch(a):
        import torch

        return torch.empty(a.shape if shape is None else shape, dtype=a.dtype, device=a.device)
    return np.empty(a.shape if shape is None else shape, dtype=np.complex128)


# ---------------------------------------------------------------- context

def qdd_create(device: int = 0, hbm_budget_bytes: int = 0):
    h = _vp()
    _check(_lib.qdd_create(ctypes.byref(h), device, hbm_budget_bytes), "qdd_create")
    return h


def qdd_destroy(ctx):
    _lib.qdd_destroy(ctx)


def qdd_last_error() -> str:
    return _lib.qdd_last_error().decode(errors="replace")


QDD_PROF_SAP, QDD_PROF_DSLASH, QDD_PROF_BLAS, QDD_PROF_OTHER, QDD_PROF_ALL = 1, 2, 4, 8, 15


def qdd_set_profiling(ctx, classes=QDD_PROF_ALL):
    """Event-time the selected kernel classes (bit mask; True = all, False/0 = off)."""
    if classes is True:
        classes = QDD_PROF_ALL
    _check(_lib.qdd_set_profiling(ctx, int(classes)), "qdd_set_profiling")


def qdd_get_kernel_times(ctx, reset: bool = False) -> dict:
    out = (ctypes.c_double * 6)()
    _check(_lib.qdd_get_kernel_times(ctx, out, 1 if reset else 0), "qdd_get_kernel_times")
    return {"sap": (out[0], int(out[1])), "dslash": (out[2], int(out[3])), "blas": (out[4], int(out[5]))}


def qdd_get_kernel_work(ctx) -> dict:
    """Algorithmic (flop, bytes) per kernel class since the last reset of
    qdd_get_kernel_times (only the FP64 vector kernels count theirs)."""
    out = (ctypes.c_double * 6)()
    _check(_lib.qdd_get_kernel_work(ctx, out), "qdd_get_kernel_work")
    return {"sap": (out[0], out[1]), "dslash": (out[2], out[3]), "blas": (out[4], out[5])}


def qdd_memory(ctx):
    u, b = ctypes.c_size_t(), ctypes.c_size_t()
    _check(_lib.qdd_memory(ctx, ctypes.byref(u), ctypes.byref(b)), "qdd_memory")
    return u.value, b.value


def qdd_measure_fma_peak(device: int = 0, fp64: bool = True, target_ms: float = 200.0):
    """(TFLOP/s, ms) of the FMA-chain kernel in FP64 or FP32 on `device`."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(_lib.qdd_measure_fma_peak(device, 1 if fp64 else 0, float(target_ms), ctypes.byref(t), ctypes.byref(ms)),
           "qdd_measure_fma_peak")
    return t.value, ms.value


# ------------------------------------------------------------ gauge field

def qdd_create_gauge_field(ctx, L, dom, links):
    h = _vp()
    p, dev = _ptr(links)
    _check(_lib.qdd_create_gauge_field(ctx, _ivec(L), _ivec(dom), p, dev, ctypes.byref(h)), "qdd_create_gauge_field")
    return h


# the hooks of each sharded gauge field, kept alive until it is destroyed
_slab_hooks = {}


def qdd_create_gauge_field_slab(ctx, Lloc, dom, links_ext, comm):
    """A gauge field sharded in t: this rank's local lattice Lloc, the links of
    the extended local lattice (one domain block of halo on each side) and
    the communication hooks (an object with a ``struct`` qdd_comm field, kept
    alive here until the field is destroyed)."""
    h = _vp()
    p, dev = _ptr(links_ext)
    _check(_lib.qdd_create_gauge_field_slab(ctx, _ivec(Lloc), _ivec(dom), p, dev, ctypes.byref(comm.struct),
                                            ctypes.byref(h)), "qdd_create_gauge_field_slab")
    _slab_hooks[h.value] = comm
    return h


def qdd_slab_regions(Lloc, dom, colour: int):
    """((first domain slot, domains, direction) sent up, (...) sent down) of the
    face slots exchanged after a half-sweep of `colour` (host logic)."""
    out = (ctypes.c_int * 6)()
    _check(_lib.qdd_slab_regions(_ivec(Lloc), _ivec(dom), int(colour), out), "qdd_slab_regions")
    return tuple(out[0:3]), tuple(out[3:6])


def qdd_layout_faces(L, dom):
    """(foff[8], fcoord[Vd]) of the face-slot layout of a domain shape (host logic)."""
    Vd = int(np.prod(dom))
    foff = (ctypes.c_int * 8)()
    fcoord = np.zeros(Vd, dtype=np.uint32)
    _check(_lib.qdd_layout_faces(_ivec(L), _ivec(dom), foff, fcoord.ctypes.data), "qdd_layout_faces")
    return list(foff), fcoord


def qdd_destroy_gauge(g):
    _lib.qdd_destroy_gauge(g)
    _slab_hooks.pop(g.value if isinstance(g, _vp) else g, None)


def qdd_set_link_compression(g, two_rows: bool):
    _check(_lib.qdd_set_link_compression(g, int(bool(two_rows))), "qdd_set_link_compression")


def qdd_link_compression(g):
    """(two_rows, is_su3): whether the FP32/16-bit operator reads two rows
    per link, and whether every link passed the SU(3) check."""
    t, u = ctypes.c_int(), ctypes.c_int()
    _check(_lib.qdd_link_compression(g, ctypes.byref(t), ctypes.byref(u)), "qdd_link_compression")
    return bool(t.value), bool(u.value)


def qdd_check_hits() -> int:
    """Out-of-range indices the range-checked build has skipped (raises
    QddError with the normal build)."""
    h = ctypes.c_ulonglong()
    _check(_lib.qdd_check_hits(ctypes.byref(h)), "qdd_check_hits")
    return h.value


def qdd_set_schwarz_variant(g, variant: int):
    """0: links and clover staged when they fit (domain size fixed at compile
    time for 16-bit 4^4 domains; form 3 with FP32 links); 1: links staged,
    clover through the cache, three CTAs per SM; 2: the one-thread form with
    the size taken at run time; 3: two threads per site pair (FP32
    arithmetic; agrees with the one-thread form to rounding)."""
    _check(_lib.qdd_set_schwarz_variant(g, int(variant)), "qdd_set_schwarz_variant")


def qdd_check_set_wait_limit(device: int, spins: int):
    """Range-checked build only: poll limit of the Schwarz kernel's first
    bounded wait (raises QddError with the normal build)."""
    _check(_lib.qdd_check_set_wait_limit(device, int(spins)), "qdd_check_set_wait_limit")


def qdd_set_clover(g, c_sw: float, kappa: float):
    _check(_lib.qdd_set_clover(g, float(c_sw), float(kappa)), "qdd_set_clover")


def qdd_get_clover(g, V: int, which: int = 0) -> np.ndarray:
    out = np.zeros((V, 2, 6, 6), dtype=np.complex128)
    _check(_lib.qdd_get_clover(g, which, out.ctypes.data), "qdd_get_clover")
    return out


# --------------------------------------------------------------- operators

def qdd_apply_D(g, x, prec="f64", nrhs: int = 1, out=None):
    out = _like(x) if out is None else out
    pi, dev = _ptr(x)
    po, dev2 = _ptr(out)
    assert dev == dev2
    _check(_lib.qdd_apply_D(g, pi, po, nrhs, _prec(prec), dev, _stream(x)), "qdd_apply_D")
    return out


def qdd_sap_apply(g, eta, nmr: int, n_half: int, prec="f64", nrhs: int = 1, want_rho: bool = False):
    psi = _like(eta)
    rho = _like(eta) if want_rho else None
    pe, dev = _ptr(eta)
    pp, _ = _ptr(psi)
    pr = _ptr(rho)[0] if want_rho else None
    _check(_lib.qdd_sap_apply(g, pe, pp, pr, nrhs, nmr, n_half, _prec(prec), dev, _stream(eta)), "qdd_sap_apply")
    return (psi, rho) if want_rho else psi


def qdd_default_params(**kw) -> qdd_solve_params:
    p = qdd_solve_params()
    _lib.qdd_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("sap_prec", "arnoldi_prec"):
            v = _prec(v)
        setattr(p, k, v)
    return p


def qdd_solve(g, b, params: qdd_solve_params | None = None, x=None, allow_noconv: bool = False, **kw):
    """Solve D x = b; returns (x, report dict)."""
    p = params if params is not None else qdd_default_params(**kw)
    x = _like(b) if x is None else x
    pb, dev = _ptr(b)
    px, _ = _ptr(x)
    rep = qdd_report()
    st = _lib.qdd_solve(g, pb, px, dev, ctypes.byref(p), ctypes.byref(rep), _stream(b))
    _check(st, "qdd_solve", ok=(QDD_OK, QDD_ENOCONV) if allow_noconv else (QDD_OK,))
    return x, rep.as_dict()


def qdd_cdot_multi(ctx, v, w):
    """<v_i, w> for the rows of v (torch CUDA complex128 tensors); returns a CUDA tensor."""
    import torch

    assert v.is_cuda and w.is_cuda and v.dtype == torch.complex128 and w.dtype == torch.complex128
    assert v.dim() == 2 and v.stride(1) == 1 and w.is_contiguous(), "rows of v and w must be contiguous"
    nvec, n = v.shape
    out = torch.empty(nvec, dtype=torch.complex128, device=v.device)
    _check(_lib.qdd_cdot_multi(ctx, v.data_ptr(), nvec, v.stride(0), w.data_ptr(), n, out.data_ptr(),
                               _stream(v)), "qdd_cdot_multi")
    return out


def qdd_cdot_multi_noalloc(v, w, out=None):
    """<v_i, w> without any device allocation inside the library (torch CUDA
    complex128 tensors; out, if given, is a CUDA tensor of nvec elements).
    The call does not wait: out is ready in the order of torch's current
    stream, which every later torch operation on that stream respects."""
    import torch

    assert v.is_cuda and w.is_cuda and v.dtype == torch.complex128 and w.dtype == torch.complex128
    assert v.dim() == 2 and v.stride(1) == 1 and w.is_contiguous(), "rows of v and w must be contiguous"
    nvec, n = v.shape
    if out is None:
        out = torch.empty(nvec, dtype=torch.complex128, device=v.device)
    _check(_lib.qdd_cdot_multi_noalloc(v.data_ptr(), nvec, v.stride(0), w.data_ptr(), n, out.data_ptr(),
                                       _stream(v)), "qdd_cdot_multi_noalloc")
    return out


# -------------------------------------------------------------- host logic

def qdd_load_model(n_domains_per_colour: float, n_slots: float) -> float:
    return _lib.qdd_load_model(float(n_domains_per_colour), float(n_slots))


def qdd_domain_working_set(dom, link_bytes: int, n_full: int, n_even: int) -> float:
    return _lib.qdd_domain_working_set(_ivec(dom), link_bytes, n_full, n_even)


def qdd_layout(L, dom):
    """(site_of, nbl, nbd) arrays of the device layout (host logic)."""
    V = int(np.prod(L))
    Vd = int(np.prod(dom))
    Nd = V // Vd
    site_of = np.zeros(V, dtype=np.int32)
    nbl = np.zeros(Vd * 8, dtype=np.uint16)
    nbd = np.zeros(Nd * 8, dtype=np.int32)
    _check(_lib.qdd_layout(_ivec(L), _ivec(dom), site_of.ctypes.data, nbl.ctypes.data, nbd.ctypes.data),
           "qdd_layout")
    return site_of, nbl.reshape(Vd, 8), nbd.reshape(Nd, 8)


def qdd_autotune(ctx, L, links, c_sw: float, kappa: float, b, params: qdd_solve_params, dom_candidates,
                 nmr_candidates=()):
    """Fastest (dom, nmr) for this problem; returns (result dict, per-candidate log)."""
    import json

    pl, ldev = _ptr(links)
    pb, bdev = _ptr(b)
    doms = (ctypes.c_int * (4 * len(dom_candidates)))(*[int(v) for d in dom_candidates for v in d])
    nmrs = (ctypes.c_int * max(1, len(nmr_candidates)))(*[int(v) for v in nmr_candidates])
    res = qdd_tune_result()
    buf = ctypes.create_string_buffer(1 << 16)
    _check(_lib.qdd_autotune(ctx, _ivec(L), pl, ldev, float(c_sw), float(kappa), pb, bdev, ctypes.byref(params),
                             doms, len(dom_candidates), nmrs, len(nmr_candidates), ctypes.byref(res), buf,
                             len(buf)), "qdd_autotune")
    out = {"dom": tuple(res.dom), "nmr": res.nmr, "iters": res.iters,
           "n_tried": res.n_tried, "ms": res.ms, "wave_load": res.wave_load}
    return out, json.loads(buf.value.decode())


# ---------------------------------------------------------------- serving

def qdd_serve_config(ctx, max_slots: int):
    _check(_lib.qdd_serve_config(ctx, max_slots), "qdd_serve_config")


def qdd_submit(ctx, g, b: np.ndarray, x: np.ndarray, params: qdd_solve_params) -> int:
    t = ctypes.c_uint64()
    assert isinstance(b, np.ndarray) and isinstance(x, np.ndarray), "serving takes host arrays"
    _check(_lib.qdd_submit(ctx, g, b.ctypes.data, x.ctypes.data, ctypes.byref(params), ctypes.byref(t)),
           "qdd_submit")
    return t.value


def qdd_poll(ctx, ticket: int, timeout_s: float = 0.0):
    """(status, report dict or None); status QDD_ENOTREADY while in flight."""
    rep = qdd_report()
    st = _lib.qdd_poll(ctx, ticket, ctypes.byref(rep), timeout_s)
    if st == QDD_ENOTREADY:
        return st, None
    return st, rep.as_dict()


# ------------------------------------------------------------------ multigrid

def qdd_mg_default_params(**kw) -> qdd_mg_params:
    p = qdd_mg_params()
    _lib.qdd_mg_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k not in dict(qdd_mg_params._fields_):
            raise TypeError(f"unknown multigrid parameter {k!r}")
        setattr(p, k, _prec(v) if k == "sap_prec" else v)
    return p


def qdd_mg_setup(g, w0, params: qdd_mg_params | None = None, **kw):
    """Build the two-level multigrid preconditioner from the nv random fields w0 (nv, V, 4, 3)."""
    p = params if params is not None else qdd_mg_default_params(**kw)
    pw, dev = _ptr(w0)
    _check(_lib.qdd_mg_setup(g, ctypes.byref(p), pw, dev), "qdd_mg_setup")


def qdd_mg_vcycle(g, v):
    z = _like(v)
    pv, dev = _ptr(v)
    pz, _ = _ptr(z)
    _check(_lib.qdd_mg_vcycle(g, pv, pz, dev, _stream(v)), "qdd_mg_vcycle")
    return z


def qdd_mg_get_basis(g, nv: int, V: int) -> np.ndarray:
    out = np.empty((nv, V, 4, 3), dtype=np.complex128)
    _check(_lib.qdd_mg_get_basis(g, out.ctypes.data_as(_vp)), "qdd_mg_get_basis")
    return out
