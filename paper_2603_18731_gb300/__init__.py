"""Python binding of the GB300 subspace Hamiltonian library (``libqsd.so``).

Argument marshalling only: every step of the computation runs in the CUDA
library behind the C ABI declared in ``include/qsd.h``; the names here are the
ABI's names without the ``qsd_`` prefix.  PyTorch supplies device memory and
streams.  There is no CPU fallback: when the library is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqsd.so")

QSD_OK = 0
QSD_FP64 = 0
QSD_FP32_MIXED = 1
QSD_FP32_DOT2 = 2
STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "QUBIT_RANGE", 3: "REPEATED_INDEX", 4: "NOT_HERMITIAN",
    5: "COMPLEX_UNSUPPORTED", 6: "OOM", 7: "NOT_CONVERGED", 8: "TIMEOUT", 9: "CUDA", 10: "CAPACITY",
    11: "CANCELLED", 12: "PENDING", 13: "INTERNAL",
}


class QsdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code
        self.status = STATUS.get(code, str(code))


class OpInfo(C.Structure):
    _fields_ = [("n_qubits", C.c_int32), ("n_words", C.c_int32), ("n_terms_in", C.c_int64),
                ("n_terms", C.c_int64), ("n_diag_terms", C.c_int64), ("n_groups", C.c_int64),
                ("n_ladder_groups", C.c_int64), ("n_excitation_groups", C.c_int64),
                ("n_excitation_shapes", C.c_int32), ("excitation_rank_index", C.c_int32),
                ("max_group_terms", C.c_int64), ("is_real", C.c_int32),
                ("is_hermitian", C.c_int32), ("identity_coef", C.c_double), ("n_linear_ranges", C.c_int64)]


class LanczosParams(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_steps", C.c_int32), ("tol", C.c_double),
                ("refine_tol", C.c_double), ("check_every", C.c_int32), ("refine_steps", C.c_int32),
                ("max_refine", C.c_int32), ("use_graphs", C.c_int32), ("seed", C.c_uint64),
                ("v0", C.c_void_p), ("time_limit_s", C.c_double)]


class LanczosInfo(C.Structure):
    _fields_ = [("steps", C.c_int32), ("refine_restarts", C.c_int32), ("residual", C.c_double),
                ("energy_unrefined", C.c_double), ("status", C.c_int32), ("applies", C.c_int32)]


class LobpcgParams(C.Structure):
    _fields_ = [("k", C.c_int32), ("max_iters", C.c_int32), ("tol", C.c_double), ("seed", C.c_uint64),
                ("x0", C.c_void_p), ("precondition", C.c_int32), ("start", C.c_int32)]


class LobpcgInfo(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("max_residual", C.c_double),
                ("status", C.c_int32), ("reserved", C.c_int32)]


class TrimInfo(C.Structure):
    _fields_ = [("groups_in", C.c_int64), ("groups_kept", C.c_int64), ("terms_in", C.c_int64),
                ("terms_kept", C.c_int64), ("d_min", C.c_double), ("splitting", C.c_double)]


class RampsInfo(C.Structure):
    _fields_ = [("levels", C.c_int32), ("stopped_by_limit", C.c_int32), ("truncated", C.c_int32),
                ("reserved", C.c_int32), ("rows_out", C.c_int64), ("candidates", C.c_int64),
                ("level_rows", C.c_int64 * 64)]


class ServerStats(C.Structure):
    _fields_ = [("queued", C.c_int64), ("active", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("admitted", C.c_int64), ("bytes_in_use", C.c_uint64), ("peak_bytes", C.c_uint64),
                ("budget_bytes", C.c_uint64), ("packed_requests", C.c_int64), ("packed_chunks", C.c_int64)]


_lib = None
_lock = threading.Lock()

# (name, restype, argtypes) of every exported entry point
_P, _I32, _I64, _U64, _D = C.c_void_p, C.c_int32, C.c_int64, C.c_uint64, C.c_double
SIGNATURES = [
    ("qsd_create", C.c_int, [C.c_int, _P, C.POINTER(_P)]),
    ("qsd_destroy", C.c_int, [_P]),
    ("qsd_last_error", C.c_char_p, [_P]),
    ("qsd_load_operator", C.c_int, [_P, _I32, _I64, _P, _P, _P, _P, _P, C.POINTER(_P)]),
    ("qsd_op_get_info", C.c_int, [_P, C.POINTER(OpInfo)]),
    ("qsd_op_groups", C.c_int, [_P, _P]),
    ("qsd_free_op", C.c_int, [_P]),
    ("qsd_build_subspace", C.c_int, [_P, _I32, _I64, _P, C.c_int, C.POINTER(_P), C.POINTER(_I64)]),
    ("qsd_subspace_info", C.c_int, [_P, C.POINTER(_I64), C.POINTER(_I32), C.POINTER(_I64)]),
    ("qsd_inject_alloc_failures", C.c_int, [_I64]),
    ("qsd_subspace_factored", C.c_int, [_P, C.POINTER(_I32), C.POINTER(_I32), C.POINTER(_I64), C.POINTER(_I64),
                                        C.POINTER(_I64)]),
    ("qsd_subspace_keys", C.c_int, [_P, _P, _P, C.c_int]),
    ("qsd_subspace_index", C.c_int, [_P, _P, _I64, _P, _P]),
    ("qsd_free_sub", C.c_int, [_P]),
    ("qsd_set_tuning", C.c_int, [_P, _I32, _I64]),
    ("qsd_apply_H_batch", C.c_int, [_P, _I32, _P, _P, _I32, _I32, _P, _P]),
    ("qsd_apply_H_complex", C.c_int, [_P, _P, _P, _I32, _P, _P]),
    ("qsd_to_csr", C.c_int, [_P, _P, _P, _I32, C.POINTER(C.c_int64), _P, _P, _I32, _P, _P]),
    ("qsd_trim_operator", C.c_int, [_P, _P, _P, _D, C.POINTER(_P), C.POINTER(TrimInfo)]),
    ("qsd_lobpcg_default_params", None, [C.POINTER(LobpcgParams)]),
    ("qsd_lobpcg", C.c_int, [_P, _P, _P, C.POINTER(LobpcgParams), _P, _P, C.POINTER(LobpcgInfo)]),
    ("qsd_ramps", C.c_int, [_P, _P, _P, _D, _D, _I32, _P, _I64, C.POINTER(_P), C.POINTER(RampsInfo)]),
    ("qsd_product_path", C.c_int, [_P, _P, _P, _I32, _I64, C.POINTER(C.c_int32)]),
    ("qsd_apply_H", C.c_int, [_P, _P, _P, C.c_int, _I32, _P, _P]),
    ("qsd_apply_H_host", C.c_int, [_P, _P, _P, C.c_int, _I32, _P, _P]),
    ("qsd_diagonal", C.c_int, [_P, _P, _P, _P]),
    ("qsd_target_table", C.c_int, [_P, _P, _P, _I64, _I64, _P]),
    ("qsd_term_table", C.c_int, [_P, _P, _P, _I64, _I64, _P]),
    ("qsd_rayleigh_quotient", C.c_int, [_P, _P, _P, _P, _P]),
    ("qsd_rayleigh_quotient_noalloc", C.c_int, [_P, _P, _P, _P, _P]),
    ("qsd_lanczos_default_params", None, [C.POINTER(LanczosParams)]),
    ("qsd_lanczos_ground_state", C.c_int, [_P, _P, _P, C.POINTER(LanczosParams), C.POINTER(_D), _P,
                                          C.POINTER(LanczosInfo)]),
    ("qsd_server_create", C.c_int, [_P, C.c_size_t, _I32, C.POINTER(_P)]),
    ("qsd_server_submit", C.c_int, [_P, _P, _P, C.POINTER(LanczosParams), C.POINTER(_U64)]),
    ("qsd_server_poll", C.c_int, [_P, _U64, C.POINTER(_D), C.POINTER(LanczosInfo), _P]),
    ("qsd_server_wait", C.c_int, [_P, _U64, _D, C.POINTER(_D), C.POINTER(LanczosInfo), _P]),
    ("qsd_server_cancel", C.c_int, [_P, _U64]),
    ("qsd_server_release", C.c_int, [_P, _U64]),
    ("qsd_server_get_stats", C.c_int, [_P, C.POINTER(ServerStats)]),
    ("qsd_server_set_pack_rows", C.c_int, [_P, _I64]),
    ("qsd_server_last_error", C.c_char_p, [_P]),
    ("qsd_server_destroy", C.c_int, [_P]),
]


def lib(build_if_missing: bool = True):
    """Load ``libqsd.so`` (building it first when absent)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                if not build_if_missing:
                    raise ImportError(f"{LIB_PATH} is not built")
                from . import build as _build
                _build.build()
            L = C.CDLL(LIB_PATH)
            for name, res, args in SIGNATURES:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _t_ptr(t):
    return C.c_void_p(t.data_ptr())


def W_of(n_qubits: int) -> int:
    return 1 if n_qubits <= 64 else (n_qubits + 63) // 64


class Operator:
    def __init__(self, ctx: "Context", handle, n_qubits: int):
        self.ctx, self.handle, self.n_qubits = ctx, handle, n_qubits

    def info(self) -> dict:
        i = OpInfo()
        self.ctx._check(lib().qsd_op_get_info(self.handle, C.byref(i)))
        return {f: getattr(i, f) for f, _ in OpInfo._fields_}

    def groups(self) -> np.ndarray:
        g = self.info()["n_groups"]
        out = np.zeros((max(g, 1), W_of(self.n_qubits)), np.uint64)
        self.ctx._check(lib().qsd_op_groups(self.handle, _np_ptr(out)))
        return out[:g]

    def free(self):
        if self.handle:
            lib().qsd_free_op(self.handle)
            self.handle = None


class Subspace:
    def __init__(self, ctx: "Context", handle, n_qubits: int, dim: int):
        self.ctx, self.handle, self.n_qubits, self.dim = ctx, handle, n_qubits, dim

    @property
    def W(self) -> int:
        return W_of(self.n_qubits)

    def capacity(self) -> int:
        d, n, cap = C.c_int64(), C.c_int32(), C.c_int64()
        self.ctx._check(lib().qsd_subspace_info(self.handle, C.byref(d), C.byref(n), C.byref(cap)))
        return cap.value

    def factored(self) -> dict:
        """The sector-factored index: is_product, split, n_a, n_b, neighbours."""
        ip, sp = C.c_int32(), C.c_int32()
        na, nb, nn = C.c_int64(), C.c_int64(), C.c_int64()
        self.ctx._check(lib().qsd_subspace_factored(self.handle, C.byref(ip), C.byref(sp), C.byref(na),
                                                    C.byref(nb), C.byref(nn)))
        return {"is_product": bool(ip.value), "split": sp.value, "n_a": na.value, "n_b": nb.value,
                "neighbours": nn.value}

    def free(self):
        if self.handle:
            lib().qsd_free_sub(self.handle)
            self.handle = None


class Context:
    """A library context on one CUDA device and one CUDA stream (a dedicated
    ``torch.cuda.Stream`` unless one is given)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("paper_2603_18731_gb300 needs a CUDA GPU; none is visible")
        self.torch = torch
        self.device = torch.device("cuda", device)
        self.stream = stream if stream is not None else torch.cuda.Stream(device=self.device)
        h = C.c_void_p()
        rc = lib().qsd_create(device, C.c_void_p(self.stream.cuda_stream), C.byref(h))
        if rc != QSD_OK:
            raise QsdError(rc, lib().qsd_last_error(None).decode())
        self.handle = h

    # -- plumbing
    def _check(self, rc: int):
        if rc != QSD_OK:
            raise QsdError(rc, lib().qsd_last_error(self.handle).decode())

    def synchronize(self):
        self.stream.synchronize()

    def empty(self, shape, dtype):
        with self.torch.cuda.stream(self.stream):
            return self.torch.empty(shape, dtype=dtype, device=self.device)

    def close(self):
        if getattr(self, "handle", None):
            lib().qsd_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- ABI calls
    def set_tuning(self, knob: int, value: int):
        """knob 1: product path (0 auto, 1 group scan, 2 excitation index,
        3 half evaluation, 4 factored, 5 filter/verify); knob 2: lanes per
        row of the group scan (0 auto, 1, 8); knob 3: autotuning of the
        product path on first use (1 on, 0 off); knob 4: the autotuner may
        pick the half evaluation; knob 5: row order of the lane-per-row scans
        (0 auto, 1 index, 2 hash); knob 6: half-sum tables of the factored
        product's linear ranges (1 on, 0 off).  See QSD_TUNE_* in qsd.h."""
        self._check(lib().qsd_set_tuning(self.handle, int(knob), int(value)))

    def product_path(self, op: "Operator", sub: "Subspace", precision: int = 0, k: int = 1) -> int:
        """Path of the next product (0: scan, one lane per row; 1: scan, 8
        lanes per row; 2: excitation index), without timing anything."""
        out = C.c_int32(0)
        self._check(lib().qsd_product_path(self.handle, op.handle, sub.handle, int(precision), int(k), C.byref(out)))
        return int(out.value)

    def load_operator(self, op) -> Operator:
        """``op``: any object with n_qubits, term_ptr, op_qubit, op_code, coef
        (complex) as numpy arrays (e.g. ``workloads.QubitOperator``)."""
        tp = np.ascontiguousarray(op.term_ptr, np.int64)
        oq = np.ascontiguousarray(op.op_qubit, np.int32)
        oc = np.ascontiguousarray(op.op_code, np.uint8)
        cr = np.ascontiguousarray(np.real(op.coef), np.float64)
        ci = np.ascontiguousarray(np.imag(op.coef), np.float64)
        h = C.c_void_p()
        self._check(lib().qsd_load_operator(self.handle, int(op.n_qubits), int(cr.shape[0]), _np_ptr(tp),
                                            _np_ptr(oq), _np_ptr(oc), _np_ptr(cr), _np_ptr(ci), C.byref(h)))
        return Operator(self, h, int(op.n_qubits))

    def build_subspace(self, n_qubits: int, words) -> Subspace:
        """``words``: [n, W] uint64 numpy array (host) or int64/uint64 CUDA tensor."""
        h = C.c_void_p()
        dim = C.c_int64()
        if isinstance(words, np.ndarray):
            w = np.ascontiguousarray(words, np.uint64)
            self._check(lib().qsd_build_subspace(self.handle, n_qubits, int(w.shape[0]), _np_ptr(w), 0,
                                                 C.byref(h), C.byref(dim)))
        else:
            w = words.contiguous()
            self._check(lib().qsd_build_subspace(self.handle, n_qubits, int(w.shape[0]), _t_ptr(w), 1,
                                                 C.byref(h), C.byref(dim)))
        return Subspace(self, h, n_qubits, dim.value)

    def subspace_keys(self, sub: Subspace) -> np.ndarray:
        out = np.zeros((max(sub.dim, 1), sub.W), np.uint64)
        self._check(lib().qsd_subspace_keys(self.handle, sub.handle, _np_ptr(out), 0))
        return out[:sub.dim]

    def subspace_index(self, sub: Subspace, keys):
        """``keys``: CUDA int64 tensor [n, W] (bit patterns); returns int64 [n]."""
        keys = keys.contiguous()
        out = self.empty((keys.shape[0],), self.torch.int64)
        self._check(lib().qsd_subspace_index(self.handle, sub.handle, int(keys.shape[0]), _t_ptr(keys),
                                             _t_ptr(out)))
        return out

    def apply_H(self, op: Operator, sub: Subspace, x, y=None, precision: int = QSD_FP64):
        """y = H_S x for CUDA tensors x of shape [D] or [D, k]."""
        dt = self.torch.float64 if precision == QSD_FP64 else self.torch.float32
        if x.dtype != dt or not x.is_contiguous():
            raise ValueError(f"x must be a contiguous {dt} tensor")
        k = 1 if x.dim() == 1 else int(x.shape[1])
        if y is None:
            y = self.empty(tuple(x.shape), dt)
        self._check(lib().qsd_apply_H(self.handle, op.handle, sub.handle, precision, k, _t_ptr(x), _t_ptr(y)))
        return y

    def apply_H_complex(self, op: Operator, sub: Subspace, x, y=None):
        """y = H_S x for CUDA complex128 tensors of shape [D] or [D, k] (any
        operator, complex elements allowed)."""
        if x.dtype != self.torch.complex128 or not x.is_contiguous():
            raise ValueError("x must be a contiguous complex128 tensor")
        k = 1 if x.dim() == 1 else int(x.shape[1])
        if y is None:
            y = self.empty(tuple(x.shape), self.torch.complex128)
        self._check(lib().qsd_apply_H_complex(self.handle, op.handle, sub.handle, k, _t_ptr(x), _t_ptr(y)))
        return y

    def apply_H_batch(self, ops, subs, xs, ys=None, precision: int = QSD_FP64):
        """Packed products y_i = H_S(ops[i], subs[i]) x_i in one launch (per key
        width); xs: CUDA tensors [D_i] or [D_i, k] with a common k."""
        dt = self.torch.float64 if precision == QSD_FP64 else self.torch.float32
        n = len(ops)
        if not (len(subs) == len(xs) == n):
            raise ValueError("ops, subs and xs must have the same length")
        ks = {1 if x.dim() == 1 else int(x.shape[1]) for x in xs}
        if len(ks) > 1 or any(x.dtype != dt or not x.is_contiguous() for x in xs):
            raise ValueError(f"xs must be contiguous {dt} tensors with one column count")
        k = ks.pop() if ks else 1
        if ys is None:
            ys = [self.empty(tuple(x.shape), dt) for x in xs]
        arr = C.c_void_p * max(n, 1)
        self._check(lib().qsd_apply_H_batch(self.handle, n, arr(*[o.handle for o in ops]),
                                            arr(*[s_.handle for s_ in subs]), precision, k,
                                            arr(*[_t_ptr(x) for x in xs]), arr(*[_t_ptr(y) for y in ys])))
        return ys

    def apply_H_host(self, op: Operator, sub: Subspace, x: np.ndarray, precision: int = QSD_FP64,
                     out: np.ndarray | None = None) -> np.ndarray:
        dt = np.float64 if precision == QSD_FP64 else np.float32
        if x.dtype != dt or not x.flags["C_CONTIGUOUS"]:
            raise ValueError(f"x must be a contiguous {dt} array")
        k = 1 if x.ndim == 1 else int(x.shape[1])
        y = np.empty_like(x) if out is None else out
        self._check(lib().qsd_apply_H_host(self.handle, op.handle, sub.handle, precision, k, _np_ptr(x),
                                           _np_ptr(y)))
        return y

    def diagonal(self, op: Operator, sub: Subspace):
        out = self.empty((sub.dim,), self.torch.float64)
        self._check(lib().qsd_diagonal(self.handle, op.handle, sub.handle, _t_ptr(out)))
        return out

    def target_table(self, op: Operator, sub: Subspace, row0: int = 0, nrows: int | None = None):
        nrows = sub.dim - row0 if nrows is None else nrows
        G = op.info()["n_groups"]
        out = self.empty((nrows, G), self.torch.int64)
        self._check(lib().qsd_target_table(self.handle, op.handle, sub.handle, row0, nrows, _t_ptr(out)))
        return out

    def term_table(self, op: Operator, sub: Subspace, row0: int = 0, nrows: int | None = None):
        nrows = sub.dim - row0 if nrows is None else nrows
        T = op.info()["n_terms_in"]
        out = self.empty((nrows, T), self.torch.int8)
        self._check(lib().qsd_term_table(self.handle, op.handle, sub.handle, row0, nrows, _t_ptr(out)))
        return out

    def rayleigh_quotient(self, op: Operator, sub: Subspace, u):
        """(u^T H u / u^T u, |H u - theta u| / |u|, u^T u) for a CUDA float64 vector u."""
        out = np.zeros(3)
        self._check(lib().qsd_rayleigh_quotient(self.handle, op.handle, sub.handle, _t_ptr(u), _np_ptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def rayleigh_quotient_noalloc(self, op: Operator, sub: Subspace, u):
        """As rayleigh_quotient with no device allocation (fixed library scratch,
        at most 2^20 rows; overlapping calls race)."""
        out = np.zeros(3)
        self._check(lib().qsd_rayleigh_quotient_noalloc(self.handle, op.handle, sub.handle, _t_ptr(u),
                                                        _np_ptr(out)))
        return float(out[0]), float(out[1]), float(out[2])

    def trim_operator(self, op: Operator, sub: Subspace, tol: float):
        """Operator without the groups whose element bound over the subspace's
        smallest diagonal splitting is below ``tol``: (Operator, info dict)."""
        h = C.c_void_p()
        info = TrimInfo()
        self._check(lib().qsd_trim_operator(self.handle, op.handle, sub.handle, float(tol), C.byref(h),
                                            C.byref(info)))
        return Operator(self, h, op.n_qubits), {f: getattr(info, f) for f, _ in TrimInfo._fields_}

    def lobpcg(self, op: Operator, sub: Subspace, k: int = 1, want_vectors: bool = False, check: bool = True,
               **params):
        """The k lowest eigenpairs: (evals numpy [k], info dict[, vectors tensor
        [D, k]]).  Keyword arguments set fields of qsd_lobpcg_params."""
        p = LobpcgParams()
        lib().qsd_lobpcg_default_params(C.byref(p))
        p.k = int(k)
        x0 = params.pop("x0", None)
        for key, v in params.items():
            setattr(p, key, v)
        if x0 is not None:
            p.x0 = C.c_void_p(x0.data_ptr())
        ev = np.zeros(k)
        info = LobpcgInfo()
        vec = self.empty((sub.dim, k), self.torch.float64) if want_vectors else None
        rc = lib().qsd_lobpcg(self.handle, op.handle, sub.handle, C.byref(p), _np_ptr(ev),
                              _t_ptr(vec) if vec is not None else None, C.byref(info))
        d = {f: getattr(info, f) for f, _ in LobpcgInfo._fields_ if f != "reserved"}
        if check and rc not in (QSD_OK, 7):
            self._check(rc)
        d["status"] = STATUS.get(rc, rc)
        return (ev, d, vec) if want_vectors else (ev, d)

    def ramps(self, op: Operator, start: Subspace, E: float, tau: float, max_levels: int = 16,
              restrict: Subspace | None = None, max_rows: int = 0):
        """RAMPS refinement from the rows of ``start``: (new Subspace, info)."""
        h = C.c_void_p()
        info = RampsInfo()
        self._check(lib().qsd_ramps(self.handle, op.handle, start.handle, float(E), float(tau), int(max_levels),
                                    restrict.handle if restrict is not None else None, int(max_rows), C.byref(h),
                                    C.byref(info)))
        d = {f: getattr(info, f) for f, _ in RampsInfo._fields_ if f not in ("level_rows", "reserved")}
        d["level_rows"] = [int(info.level_rows[i]) for i in range(min(info.levels, 64))]
        return Subspace(self, h, start.n_qubits, int(info.rows_out)), d

    def csr_size(self, op: Operator, sub: Subspace, full: bool = False) -> int:
        """Pass 1 of the CSR build: the number of stored entries (the counts
        are kept in the context for the next ``to_csr`` of the same pair)."""
        nnz = C.c_int64(0)
        self._check(lib().qsd_to_csr(self.handle, op.handle, sub.handle, 1 if full else 0, C.byref(nnz), None,
                                     None, 32, None, None))
        return int(nnz.value)

    def to_csr(self, op: Operator, sub: Subspace, full: bool = False, index_bits: int = 32,
               complex_data: bool = False):
        """CSR arrays of H_S as CUDA tensors (indptr int64, indices int32/64,
        data float64[, data_im float64]).  ``full``: evaluate every group of
        every row instead of the lower triangle and its mirror."""
        flags = 1 if full else 0
        nnz = C.c_int64(0)
        self._check(lib().qsd_to_csr(self.handle, op.handle, sub.handle, flags, C.byref(nnz), None, None,
                                     int(index_bits), None, None))
        t = self.torch
        n = int(nnz.value)
        indptr = self.empty((sub.dim + 1,), t.int64)
        indices = self.empty((max(n, 1),), t.int32 if index_bits == 32 else t.int64)
        data = self.empty((max(n, 1),), t.float64)
        data_im = self.empty((max(n, 1),), t.float64) if complex_data else None
        self._check(lib().qsd_to_csr(self.handle, op.handle, sub.handle, flags, C.byref(nnz), _t_ptr(indptr),
                                     _t_ptr(indices), int(index_bits), _t_ptr(data),
                                     _t_ptr(data_im) if data_im is not None else None))
        out = (indptr, indices[:n], data[:n])
        return out + (data_im[:n],) if complex_data else out

    def lanczos_ground_state(self, op: Operator, sub: Subspace, want_vector: bool = False,
                             check: bool = True, **params):
        """Returns (energy, info dict[, vector tensor]).  Keyword arguments set
        fields of qsd_lanczos_params (precision, max_steps, tol, ...)."""
        p = LanczosParams()
        lib().qsd_lanczos_default_params(C.byref(p))
        v0 = params.pop("v0", None)
        for k, v in params.items():
            setattr(p, k, v)
        if v0 is not None:
            p.v0 = C.c_void_p(v0.data_ptr())
        e = C.c_double()
        info = LanczosInfo()
        vec = self.empty((sub.dim,), self.torch.float64) if want_vector else None
        rc = lib().qsd_lanczos_ground_state(self.handle, op.handle, sub.handle, C.byref(p), C.byref(e),
                                            _t_ptr(vec) if vec is not None else None, C.byref(info))
        d = {f: getattr(info, f) for f, _ in LanczosInfo._fields_}
        if check and rc not in (QSD_OK,):
            raise QsdError(rc, lib().qsd_last_error(self.handle).decode())
        return (e.value, d, vec) if want_vector else (e.value, d)


def lanczos_params(**params) -> LanczosParams:
    """qsd_lanczos_params with the library defaults, overridden by keywords
    (``v0`` takes a CUDA float64 tensor)."""
    p = LanczosParams()
    lib().qsd_lanczos_default_params(C.byref(p))
    v0 = params.pop("v0", None)
    for k, v in params.items():
        setattr(p, k, v)
    if v0 is not None:
        p.v0 = C.c_void_p(v0.data_ptr())
    return p


class Server:
    """Continuous-batching ground-state server (qsd_server_*)."""

    def __init__(self, ctx: Context, budget_bytes: int, max_active: int = 8):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(lib().qsd_server_create(ctx.handle, int(budget_bytes), int(max_active), C.byref(h)))
        self.handle = h

    def _err(self, rc):
        raise QsdError(rc, (lib().qsd_server_last_error(self.handle) or b"").decode())

    def submit(self, op: Operator, sub: Subspace, **params) -> int:
        t = C.c_uint64()
        rc = lib().qsd_server_submit(self.handle, op.handle, sub.handle, C.byref(lanczos_params(**params)),
                                     C.byref(t))
        if rc != QSD_OK:
            self._err(rc)
        return t.value

    def _result(self, rc, e, info, times):
        d = {f: getattr(info, f) for f, _ in LanczosInfo._fields_}
        return {"status": STATUS.get(rc, rc), "code": rc, "energy": e.value, "info": d,
                "t_submit": times[0], "t_admit": times[1], "t_done": times[2]}

    def poll(self, ticket: int):
        e, info, times = C.c_double(), LanczosInfo(), np.zeros(3)
        rc = lib().qsd_server_poll(self.handle, ticket, C.byref(e), C.byref(info), _np_ptr(times))
        return None if rc == 12 else self._result(rc, e, info, times)

    def wait(self, ticket: int, timeout_s: float = 0.0):
        e, info, times = C.c_double(), LanczosInfo(), np.zeros(3)
        rc = lib().qsd_server_wait(self.handle, ticket, timeout_s, C.byref(e), C.byref(info), _np_ptr(times))
        return self._result(rc, e, info, times)

    def cancel(self, ticket: int):
        lib().qsd_server_cancel(self.handle, ticket)

    def release(self, ticket: int) -> bool:
        return lib().qsd_server_release(self.handle, ticket) == QSD_OK

    def set_pack_rows(self, rows: int):
        """Requests with at most ``rows`` rows join the packs of small requests
        (packed launches); 0 disables packing."""
        rc = lib().qsd_server_set_pack_rows(self.handle, int(rows))
        if rc != QSD_OK:
            self._err(rc)

    def stats(self) -> dict:
        st = ServerStats()
        lib().qsd_server_get_stats(self.handle, C.byref(st))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().qsd_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)
