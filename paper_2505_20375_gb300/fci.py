"""Python binding of libfci (include/fci.h): argument marshalling only.

Every step of the sigma build and of Davidson runs in the CUDA library; this module
turns numpy/torch objects into pointers and sizes, allocates caller-owned device
buffers with torch, and raises on error codes.  If libfci.so is missing it raises at
import: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfci.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(
        f"{LIB_PATH} is missing: build it with `python -c 'import __graft_entry__ as g; g.build()'` "
        "(the CUDA library is the only implementation)")

_lib = ctypes.CDLL(LIB_PATH)

FCI_OK, FCI_ERR_ARG, FCI_ERR_OOM, FCI_ERR_CUDA, FCI_ERR_NOT_CONVERGED, FCI_ERR_TIMEOUT, \
    FCI_ERR_UNSUPPORTED, FCI_ERR_STATE = range(8)
FCI_R64, FCI_C128 = 0, 1
FCI_MODE_NONE, FCI_MODE_FCI, FCI_MODE_SPINOR, FCI_MODE_DAS = range(4)
FCI_PREC_FP64, FCI_PREC_OZ_BF16 = 0, 1
PRECISIONS = {"fp64": FCI_PREC_FP64, "oz_bf16": FCI_PREC_OZ_BF16}
TABLES = {"strings_alpha": 0, "strings_beta": 1, "repl_alpha": 2, "repl_beta": 3,
          "das_categories": 4, "das_address": 5}

_vp, _i32, _i64, _dbl, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t


class fci_info(ctypes.Structure):
    _fields_ = [("mode", _i32), ("dtype", _i32), ("n_orb", _i32), ("n_alpha", _i32), ("n_beta", _i32),
                ("n_pair", _i32), ("n_ent_alpha", _i32), ("n_ent_beta", _i32),
                ("n_str_alpha", _i64), ("n_str_beta", _i64), ("n_det", _i64),
                ("n_det_intermediate", _i64), ("n_categories", _i32), ("n_categories_intermediate", _i32)]


class fci_davidson_opts(ctypes.Structure):
    _fields_ = [("max_iter", _i32), ("max_subspace", _i32), ("tol_residual", _dbl), ("tol_energy", _dbl),
                ("eps", _dbl), ("precision", _i32), ("n_slices", _i32), ("switch_residual", _dbl),
                ("use_guess", _i32), ("final_precision", _i32), ("final_slices", _i32), ("gap_bound", _i32),
                ("staged_sigma", _i32), ("start_mix", _dbl)]


class fci_davidson_iter(ctypes.Structure):
    _fields_ = [("iteration", _i32), ("precision", _i32), ("energy", _dbl), ("delta_energy", _dbl),
                ("max_delta_c", _dbl), ("residual_norm", _dbl), ("seconds", _dbl)]


class fci_davidson_log(ctypes.Structure):
    _fields_ = [("n_iter", _i32), ("converged", _i32), ("n_sigma", _i32), ("capacity", _i32),
                ("iters", ctypes.POINTER(fci_davidson_iter)), ("e1", _dbl), ("r1_norm", _dbl), ("r0_norm", _dbl),
                ("gap_lower", _dbl), ("error_bound", _dbl), ("gap_iterations", _i32)]


def _sig(name, args, res=_i32):
    f = getattr(_lib, name)
    f.argtypes = args
    f.restype = res
    return f


_create = _sig("fci_create", [ctypes.POINTER(_vp), _i32])
_destroy = _sig("fci_destroy", [_vp])
_last_error = _sig("fci_last_error", [_vp], ctypes.c_char_p)
_get_info = _sig("fci_get_info", [_vp, ctypes.POINTER(fci_info)])
_count = _sig("fci_count_determinants", [_i32, _i32, _i32], _i64)
_setup = _sig("fci_setup_integrals", [_vp, _i32, _i32, _vp, _vp, _dbl, _vp])
_strings = _sig("fci_build_strings", [_vp, _i32, _i32, _vp])
_das = _sig("das_build_categories", [_vp, _i32, _vp, _vp, _vp, _i32, _vp])
_diag = _sig("fci_diagonal", [_vp, _vp, _vp])
_ws = _sig("fci_sigma_workspace_bytes", [_vp, _i32, _i32, _i32, ctypes.POINTER(_sz)])
_sigma = _sig("fci_sigma", [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _sz, _vp])
_host_ws = _sig("fci_sigma_host_workspace_bytes", [_vp, _i32, _i32, _i32, ctypes.POINTER(_sz)])
_sigma_host = _sig("fci_sigma_host", [_vp, _vp, _vp, _i32, _i32, _i32, _vp, _sz, _vp])
_dav_defaults = _sig("fci_davidson_default_opts", [ctypes.POINTER(fci_davidson_opts)], None)
_dav_ws = _sig("fci_davidson_workspace_bytes", [_vp, ctypes.POINTER(fci_davidson_opts), ctypes.POINTER(_sz)])
_davidson = _sig("davidson_solve", [_vp, ctypes.POINTER(fci_davidson_opts), _vp, ctypes.POINTER(_dbl),
                                    ctypes.POINTER(fci_davidson_log), _vp, _sz, _vp])
_tbytes = _sig("fci_table_bytes", [_vp, _i32, ctypes.POINTER(_sz)])
_tcopy = _sig("fci_copy_table", [_vp, _i32, _vp, _sz, _vp])
_set_timing = _sig("fci_set_phase_timing", [_vp, _i32])
_get_times = _sig("fci_get_phase_times", [_vp, ctypes.POINTER(_dbl), ctypes.POINTER(_i64), _i32])
_sync_status = _sig("fci_sync_status", [_vp, _vp])
_sigma_graph = _sig("fci_sigma_graph", [_vp, _vp, _vp, _i32, _i32, _vp, _sz, _vp])
_clear_graphs = _sig("fci_clear_graphs", [_vp])


class fci_tune_report(ctypes.Structure):
    _fields_ = [("n_candidates", _i32), ("chosen", _i32), ("param_a", _i32 * 8), ("param_b", _i32 * 8),
                ("ms", _dbl * 8)]


_tune = _sig("fci_tune_sigma", [_vp, _i32, _vp, _vp, _vp, _sz, _i32, _vp, ctypes.POINTER(fci_tune_report)])


class fci_sigma_job(ctypes.Structure):
    _fields_ = [("handle", _vp), ("C", _vp), ("sigma", _vp), ("precision", _i32), ("n_slices", _i32),
                ("workspace", _vp), ("workspace_bytes", _sz)]


_sigma_grouped = _sig("fci_sigma_grouped", [ctypes.POINTER(fci_sigma_job), _i32, _vp])
_sigma_grouped_graph = _sig("fci_sigma_grouped_graph", [ctypes.POINTER(fci_sigma_job), _i32, _vp])
_clear_grouped_graphs = _sig("fci_clear_grouped_graphs", [])
_dav_begin = _sig("davidson_begin", [_vp, ctypes.POINTER(fci_davidson_opts), _vp, _vp, _sz, _vp, ctypes.POINTER(_vp)])
_dav_request = _sig("davidson_request", [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i32),
                                         ctypes.POINTER(_i32), ctypes.POINTER(_vp), ctypes.POINTER(_sz)])
_dav_advance = _sig("davidson_advance", [_vp, ctypes.POINTER(_i32)])
_dav_finish = _sig("davidson_finish", [_vp, _vp, ctypes.POINTER(_dbl), ctypes.POINTER(fci_davidson_log)])
_cs_ws = _sig("fci_sigma_compressed_workspace_bytes", [_vp, _i64, ctypes.POINTER(_sz)])
_cs_sigma = _sig("fci_sigma_compressed", [_vp, _vp, _vp, _i64, _vp, _vp, _i64, ctypes.POINTER(_i64), _vp, _sz, _vp])
PHASES = ("gather", "contract", "scatter", "other")


class FCIError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libfci error {code}: {msg}")
        self.code = code


def count_determinants(n_orb: int, n_alpha: int, n_beta: int) -> int:
    return int(_count(n_orb, n_alpha, n_beta))


def last_error(h=None) -> str:
    return (_last_error(h) or b"").decode()


def _gap_of(log) -> dict:
    if log.gap_iterations <= 0 and log.e1 != log.e1:  # NaN: no gap phase
        return None
    return {k: getattr(log, k) for k in ("e1", "r1_norm", "r0_norm", "gap_lower", "error_bound", "gap_iterations")}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return _vp(s.cuda_stream)


def _alloc(nbytes: int, device) -> torch.Tensor:
    """Caller-owned device buffer (torch allocator), 256-byte aligned."""
    return torch.empty(max(int(nbytes), 1) + 256, dtype=torch.uint8, device=device)


def _aligned_ptr(buf: torch.Tensor) -> int:
    p = buf.data_ptr()
    return (p + 255) & ~255


@dataclass
class DavidsonResult:
    energy: float
    vector: torch.Tensor
    converged: bool
    n_sigma: int
    iterations: list
    gap: dict = None  # gap_bound: e1, r1_norm, r0_norm, gap_lower, error_bound, gap_iterations


class FCI:
    """One problem on one GPU: integrals, strings (FCI, spinor or DAS layout)."""

    def __init__(self, device: int = 0):
        self.device = torch.device("cuda", device)
        h = _vp()
        rc = _create(ctypes.byref(h), device)
        if rc:
            raise FCIError(rc, last_error(None))
        self._h = h
        self._ws = None
        self._ws_ptr = 0
        self._ws_bytes = 0

    def close(self):
        if getattr(self, "_h", None):
            _destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc:
            raise FCIError(rc, last_error(self._h))

    # -------------------------------------------------------------- setup
    def setup_integrals(self, h1: np.ndarray, g2: np.ndarray, e_core: float = 0.0):
        cplx = np.iscomplexobj(h1) or np.iscomplexobj(g2)
        dt = np.complex128 if cplx else np.float64
        self._h1 = np.ascontiguousarray(h1, dt)
        self._g2 = np.ascontiguousarray(g2, dt)
        n = self._h1.shape[0]
        self._check(_setup(self._h, n, FCI_C128 if cplx else FCI_R64, self._h1.ctypes.data,
                           self._g2.ctypes.data, float(e_core), _stream()))
        return self

    def build_strings(self, n_alpha: int, n_beta: int = -1):
        self._check(_strings(self._h, n_alpha, n_beta, _stream()))
        return self

    def build_das(self, orbs_per_space, ref_alpha, ref_beta, max_transfer: int):
        S = len(orbs_per_space)
        o = (ctypes.c_int * S)(*orbs_per_space)
        a = (ctypes.c_int * S)(*ref_alpha)
        b = (ctypes.c_int * S)(*ref_beta)
        self._check(_das(self._h, S, o, a, b, max_transfer, _stream()))
        return self

    @property
    def info(self) -> dict:
        inf = fci_info()
        self._check(_get_info(self._h, ctypes.byref(inf)))
        return {k: getattr(inf, k) for k, _ in fci_info._fields_}

    @property
    def is_complex(self) -> bool:
        return self.info["dtype"] == FCI_C128

    @property
    def n_det(self) -> int:
        return self.info["n_det"]

    def vector_dtype(self):
        return torch.complex128 if self.is_complex else torch.float64

    # ------------------------------------------------------------ compute
    def diagonal(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.n_det, dtype=torch.float64, device=self.device)
        self._check(_diag(self._h, out.data_ptr(), _stream(stream)))
        return out

    def sigma_workspace_bytes(self, precision="fp64", n_slices=0, n_vec=1) -> int:
        b = _sz()
        self._check(_ws(self._h, n_vec, PRECISIONS[precision], n_slices, ctypes.byref(b)))
        return b.value

    def _workspace(self, nbytes: int):
        if self._ws is None or self._ws_bytes < nbytes:
            if self._ws is not None:
                _clear_graphs(self._h)  # cached graphs name the old buffer
            self._ws = None
            self._ws = _alloc(nbytes, self.device)
            self._ws_ptr = _aligned_ptr(self._ws)
            self._ws_bytes = nbytes
        return self._ws_ptr, self._ws_bytes

    def sigma(self, C: torch.Tensor, precision: str = "fp64", n_slices: int = 0, out: torch.Tensor = None,
              stream=None) -> torch.Tensor:
        """sigma = H C.  C: (n_det,) or (n_vec, n_det) on the device (fci_sigma), or on the
        host (fci_sigma_host: the library copies C in and sigma back inside the call)."""
        if C.dtype != self.vector_dtype():
            raise TypeError(f"C must be {self.vector_dtype()}")
        n_vec = 1 if C.dim() == 1 else C.shape[0]
        if C.shape[-1] != self.n_det:
            raise ValueError("C has the wrong length")
        if C.device.type == "cpu":
            Ch = C.contiguous()
            dst = out if out is not None else torch.empty_like(Ch, pin_memory=Ch.is_pinned())
            if dst.device.type != "cpu" or not dst.is_contiguous() or dst.shape != Ch.shape:
                raise ValueError("out must be a contiguous host tensor of C's shape")
            b = _sz()
            self._check(_host_ws(self._h, n_vec, PRECISIONS[precision], n_slices, ctypes.byref(b)))
            p, nb = self._workspace(b.value)
            self._check(_sigma_host(self._h, Ch.data_ptr(), dst.data_ptr(), n_vec, PRECISIONS[precision], n_slices,
                                    p, nb, _stream(stream)))
            return dst
        Cd = C.contiguous()
        if Cd.device != self.device:
            raise ValueError(f"C must be on the handle's device ({self.device}) or on the host")
        if out is None:
            res = torch.empty_like(Cd)
        elif out.device != self.device or out.dtype != Cd.dtype or out.shape != Cd.shape or not out.is_contiguous():
            raise ValueError("out must be a contiguous tensor of C's shape and dtype on the handle's device")
        else:
            res = out
        p, nb = self._workspace(self.sigma_workspace_bytes(precision, n_slices, n_vec))
        self._check(_sigma(self._h, Cd.data_ptr(), res.data_ptr(), n_vec, PRECISIONS[precision], n_slices,
                           p, nb, _stream(stream)))
        return res

    def sigma_graph(self, C: torch.Tensor, out: torch.Tensor, precision: str = "fp64", n_slices: int = 0,
                    stream=None) -> torch.Tensor:
        """sigma = H C for one device vector through a cached CUDA graph (fci_sigma_graph)."""
        p, nb = self._workspace(self.sigma_workspace_bytes(precision, n_slices))
        self._check(_sigma_graph(self._h, C.data_ptr(), out.data_ptr(), PRECISIONS[precision], n_slices, p, nb,
                                 _stream(stream)))
        return out

    def sigma_graph_into(self, x: int, y: int, precision, n_slices: int, ws: int, ws_bytes: int, stream=None):
        """fci_sigma_graph on caller pointers: y = H x (DEVICE addresses) with the caller's
        workspace, e.g. the sigma request of a step-wise Davidson solve."""
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        self._check(_sigma_graph(self._h, _vp(x), _vp(y), prec, n_slices, _vp(ws), ws_bytes, _stream(stream)))

    def clear_graphs(self):
        self._check(_clear_graphs(self._h))

    def tune(self, C: torch.Tensor, n_slices: int, reps: int = 3, stream=None) -> dict:
        """Time every tile shape of the split-precision contraction on this problem and keep
        the fastest for later split sigma builds with n_slices slices (fci_tune_sigma)."""
        Cd = C.to(self.device).contiguous()
        out = torch.empty_like(Cd)
        p, nb = self._workspace(self.sigma_workspace_bytes("oz_bf16", n_slices))
        r = fci_tune_report()
        self._check(_tune(self._h, n_slices, Cd.data_ptr(), out.data_ptr(), p, nb, reps, _stream(stream),
                          ctypes.byref(r)))
        das = bool(self.info["n_categories"])
        cands = [({"k_chunk_cores": r.param_a[i], "producer_warps": r.param_b[i]} if das
                  else {"dets_per_tile": r.param_a[i], "path": "two-pass gemm" if r.param_b[i] else "fused"})
                 | {"ms": r.ms[i]} for i in range(r.n_candidates)]
        return {"n_slices": n_slices, "candidates": cands, "chosen": cands[r.chosen]}

    def davidson_opts(self, max_iter=100, max_subspace=32, tol_residual=1e-6, tol_energy=1e-10, eps=0.0,
                      precision="fp64", n_slices=6, switch_residual=1e-5, final_precision="fp64", final_slices=0,
                      use_guess=False, staged_sigma=False, gap_bound=False, start_mix=None) -> fci_davidson_opts:
        o = fci_davidson_opts()
        _dav_defaults(ctypes.byref(o))
        if start_mix is not None:
            o.start_mix = start_mix
        o.max_iter, o.max_subspace = max_iter, max_subspace
        o.tol_residual, o.tol_energy, o.eps = tol_residual, tol_energy, eps
        o.precision, o.n_slices, o.switch_residual = PRECISIONS[precision], n_slices, switch_residual
        o.final_precision, o.final_slices = PRECISIONS[final_precision], final_slices
        o.use_guess = 1 if use_guess else 0
        o.staged_sigma = 1 if staged_sigma else 0
        o.gap_bound = 1 if gap_bound else 0
        return o

    def davidson_workspace_bytes(self, opts: fci_davidson_opts) -> int:
        b = _sz()
        self._check(_dav_ws(self._h, ctypes.byref(opts), ctypes.byref(b)))
        return b.value

    def davidson(self, max_iter=100, max_subspace=32, tol_residual=1e-6, tol_energy=1e-10, eps=0.0,
                 precision="fp64", n_slices=6, switch_residual=1e-5, guess: torch.Tensor = None,
                 final_precision="fp64", final_slices=0, gap_bound=False, start_mix=None,
                 stream=None) -> DavidsonResult:
        o = fci_davidson_opts()
        _dav_defaults(ctypes.byref(o))
        if start_mix is not None:
            o.start_mix = start_mix
        o.max_iter, o.max_subspace = max_iter, max_subspace
        o.tol_residual, o.tol_energy, o.eps = tol_residual, tol_energy, eps
        o.precision, o.n_slices, o.switch_residual = PRECISIONS[precision], n_slices, switch_residual
        o.use_guess = 1 if guess is not None else 0
        o.final_precision, o.final_slices = PRECISIONS[final_precision], final_slices
        o.gap_bound = 1 if gap_bound else 0
        b = _sz()
        self._check(_dav_ws(self._h, ctypes.byref(o), ctypes.byref(b)))
        p, nb = self._workspace(b.value)
        C = (guess.to(self.device).clone() if guess is not None
             else torch.zeros(self.n_det, dtype=self.vector_dtype(), device=self.device))
        cap = max_iter + 2
        iters = (fci_davidson_iter * cap)()
        log = fci_davidson_log(0, 0, 0, cap, ctypes.cast(iters, ctypes.POINTER(fci_davidson_iter)))
        E = _dbl()
        rc = _davidson(self._h, ctypes.byref(o), C.data_ptr(), ctypes.byref(E), ctypes.byref(log), p, nb,
                       _stream(stream))
        if rc not in (FCI_OK, FCI_ERR_NOT_CONVERGED):
            self._check(rc)
        its = [{k: getattr(iters[i], k) for k, _ in fci_davidson_iter._fields_} for i in range(log.n_iter)]
        return DavidsonResult(E.value, C, bool(log.converged), log.n_sigma, its, _gap_of(log))

    def sigma_compressed(self, addr: torch.Tensor, val: torch.Tensor, capacity: int = None, stream=None):
        """sigma = H C for a categorically compressed C on the DAS layout
        (fci_sigma_compressed): addr (int64, ascending DAS target addresses) and val
        (float64) on the device; returns sigma's support (ascending addresses) and values."""
        if addr.dim() != 1 or val.shape != addr.shape:
            raise ValueError("addr and val must be 1-D and of the same length")
        addr = addr.to(self.device, torch.int64).contiguous()
        val = val.to(self.device, torch.float64).contiguous()
        nnz = addr.numel()
        b = _sz()
        self._check(_cs_ws(self._h, nnz, ctypes.byref(b)))
        p, nb = self._workspace(b.value)
        if capacity is None:
            nm = self.info["n_ent_alpha"] + self.info["n_ent_beta"]
            capacity = max(1, nnz * nm * nm)
        out_a = torch.empty(capacity, dtype=torch.int64, device=self.device)
        out_v = torch.empty(capacity, dtype=torch.float64, device=self.device)
        n = _i64()
        self._check(_cs_sigma(self._h, addr.data_ptr(), val.data_ptr(), nnz, out_a.data_ptr(), out_v.data_ptr(),
                              capacity, ctypes.byref(n), p, nb, _stream(stream)))
        return out_a[:n.value], out_v[:n.value]

    def sync_status(self, stream=None):
        """Synchronise and raise FCIError(FCI_ERR_TIMEOUT) if a device wait expired."""
        self._check(_sync_status(self._h, _stream(stream)))

    # ------------------------------------------------------------- timing
    def set_phase_timing(self, enable: bool = True):
        self._check(_set_timing(self._h, 1 if enable else 0))

    def phase_times(self, reset: bool = True) -> dict:
        ms = (_dbl * 4)()
        nl = (_i64 * 4)()
        self._check(_get_times(self._h, ms, nl, 1 if reset else 0))
        return {p: {"ms": ms[i], "launches": nl[i]} for i, p in enumerate(PHASES)}

    # ------------------------------------------------------------- tables
    def table(self, name: str) -> torch.Tensor:
        t = TABLES[name]
        b = _sz()
        self._check(_tbytes(self._h, t, ctypes.byref(b)))
        if b.value == 0:
            raise FCIError(FCI_ERR_STATE, f"table {name} does not exist in this layout")
        dt = {0: torch.int64, 1: torch.int64, 2: torch.int32, 3: torch.int32, 4: torch.int64, 5: torch.int64}[t]
        out = torch.empty(b.value // torch.tensor([], dtype=dt).element_size(), dtype=dt, device=self.device)
        self._check(_tcopy(self._h, t, out.data_ptr(), b.value, _stream()))
        torch.cuda.current_stream().synchronize()
        return out


# ---------------------------------------------------------------- batched steps

def _job_array(jobs):
    arr = (fci_sigma_job * len(jobs))()
    for i, (f, C, out, prec, sl, ws, wsb) in enumerate(jobs):
        arr[i] = fci_sigma_job(f._h, _vp(C if isinstance(C, int) else C.data_ptr()),
                               _vp(out if isinstance(out, int) else out.data_ptr()),
                               PRECISIONS[prec] if isinstance(prec, str) else prec, sl, _vp(ws), wsb)
    return arr


def sigma_grouped(jobs, stream=None, graph=False):
    """jobs: list of (FCI, C, sigma, precision, n_slices, workspace_ptr, workspace_bytes);
    one fci_sigma_grouped call (split-precision jobs share one contraction launch), or with
    graph=True fci_sigma_grouped_graph (replayed from a cached CUDA graph for a repeated
    job list)."""
    arr = _job_array(jobs)
    rc = (_sigma_grouped_graph if graph else _sigma_grouped)(arr, len(jobs), _stream(stream))
    if rc:
        raise FCIError(rc, last_error(None) or last_error(jobs[0][0]._h))


def clear_grouped_graphs():
    _clear_grouped_graphs()


class DavidsonStepper:
    """Step-wise Davidson over the C ABI (davidson_begin/request/advance/finish): the
    caller computes y = H x for each request, e.g. for many solves with one grouped call."""

    def __init__(self, f: FCI, opts: fci_davidson_opts, guess: torch.Tensor = None, stream=None):
        self.f = f
        self.stream = stream
        nbytes = f.davidson_workspace_bytes(opts)
        self._ws = _alloc(nbytes, f.device)  # caller-owned, kept alive by this object
        self._ws_ptr = _aligned_ptr(self._ws)
        self._nbytes = nbytes
        self.opts = opts
        st = _vp()
        g = _vp(guess.data_ptr()) if guess is not None else None
        f._check(_dav_begin(f._h, ctypes.byref(opts), g, _vp(self._ws_ptr), nbytes, _stream(stream), ctypes.byref(st)))
        self._st = st
        self.done = False

    def request(self):
        x, y, ws = _vp(), _vp(), _vp()
        prec, sl = _i32(), _i32()
        wsb = _sz()
        self.f._check(_dav_request(self._st, ctypes.byref(x), ctypes.byref(y), ctypes.byref(prec), ctypes.byref(sl),
                                   ctypes.byref(ws), ctypes.byref(wsb)))
        return x.value, y.value, prec.value, sl.value, ws.value, wsb.value

    def advance(self):
        d = _i32()
        self.f._check(_dav_advance(self._st, ctypes.byref(d)))
        self.done = bool(d.value)
        return self.done

    def finish(self, max_log=400):
        C = torch.empty(self.f.n_det, dtype=self.f.vector_dtype(), device=self.f.device)
        iters = (fci_davidson_iter * max_log)()
        log = fci_davidson_log(0, 0, 0, max_log, ctypes.cast(iters, ctypes.POINTER(fci_davidson_iter)))
        E = _dbl()
        rc = _dav_finish(self._st, C.data_ptr(), ctypes.byref(E), ctypes.byref(log))
        self._st = None
        if rc not in (FCI_OK, FCI_ERR_NOT_CONVERGED):
            self.f._check(rc)
        its = [{k: getattr(iters[i], k) for k, _ in fci_davidson_iter._fields_} for i in range(log.n_iter)]
        return DavidsonResult(E.value, C, bool(log.converged), log.n_sigma, its, _gap_of(log))
