"""CPU oracle of the subspace Hamiltonian-vector product.

TEST INFRASTRUCTURE ONLY: this package may be imported, called or built only
by ``tests/``, ``__graft_entry__`` (its ``smoke()`` check and ``build()``,
which compiles the C part) and the CPU-baseline leg of ``bench.py``.  The
library never imports it, and it imports nothing from the library; the only
code both sides share is the seeded input generator ``workloads``.

Three independent layers, each written from the paper's definitions:

* ``qsd_oracle.c`` (loaded here through ctypes): the plain definition of
  ``H_S`` evaluated word by word from single-qubit matrix elements, with binary
  search in the integer-sorted subspace, FP64 complex; plus a plain FP64
  Lanczos with full reorthogonalisation and a Sturm-bisection tridiagonal
  solve.
* ``brute.py``: dense Kronecker products of 2x2 matrices for n <= 12 qubits.
* ``fermion.py``: second quantisation on occupation-number bit-strings, with
  no qubit alphabet at all, to check the Jordan-Wigner input generator.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "qsd_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into ``oracle/_build``."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            p = C.c_void_p
            i64 = C.c_int64
            i32 = C.c_int
            L.orc_sort_unique.restype = i64
            L.orc_sort_unique.argtypes = [i32, i64, p, p]
            L.orc_find.restype = i64
            L.orc_find.argtypes = [i32, i64, p, p]
            L.orc_check_operator.argtypes = [i32, i64, p, p, p]
            L.orc_apply.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, i32, p, p, p, p]
            L.orc_apply_rows.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, i32, p, i64, p, p, p]
            L.orc_diagonal.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, p, p]
            L.orc_term_table.argtypes = [i32, i32, i64, p, p, p, i64, p, i64, i64, p]
            L.orc_groups.restype = i64
            L.orc_groups.argtypes = [i32, i64, p, p, p, p, p, i64, p]
            L.orc_target_table.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, i64, p, i64, i64, p]
            L.orc_row_elements.restype = i64
            L.orc_row_elements.argtypes = [i32, i32, i64, p, p, p, p, p, p, p, p, p]
            L.orc_csr_count.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, p]
            L.orc_csr_fill.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, p, p, p, p]
            L.orc_tridiag_min.restype = C.c_double
            L.orc_tridiag_min.argtypes = [i32, p, p]
            L.orc_lanczos.argtypes = [i32, i32, i64, p, p, p, p, p, i64, p, i32, C.c_double,
                                      C.c_uint64, p, p, p]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _W(n):
    return max(1, (n + 63) // 64)


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError({1: "invalid argument", 2: "qubit index out of range",
                           3: "repeated qubit index in a word"}.get(rc, f"error {rc}"))


def _op_arrays(op):
    return (np.ascontiguousarray(op.term_ptr, np.int64), np.ascontiguousarray(op.op_qubit, np.int32),
            np.ascontiguousarray(op.op_code, np.uint8), np.ascontiguousarray(op.coef.real, np.float64),
            np.ascontiguousarray(op.coef.imag, np.float64))


def sort_unique(words: np.ndarray) -> np.ndarray:
    """Distinct bit-strings of ``words`` ([n, W] uint64) in integer order."""
    words = np.ascontiguousarray(words, np.uint64)
    n, W = words.shape
    out = np.zeros((max(n, 1), W), np.uint64)
    d = lib().orc_sort_unique(W, n, _ptr(words), _ptr(out))
    return out[:d].copy()


def find(keys: np.ndarray, queries: np.ndarray) -> np.ndarray:
    """Index of each query string in the sorted ``keys`` (-1 when absent)."""
    keys = np.ascontiguousarray(keys, np.uint64)
    queries = np.ascontiguousarray(queries, np.uint64)
    L = lib()
    W = keys.shape[1]
    return np.asarray([L.orc_find(W, keys.shape[0], _ptr(keys), _ptr(queries[i]))
                       for i in range(queries.shape[0])], np.int64)


def check_operator(op) -> None:
    tp, oq, oc, _, _ = _op_arrays(op)
    _check(lib().orc_check_operator(op.n_qubits, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc)))


def apply(op, keys: np.ndarray, x: np.ndarray) -> np.ndarray:
    """y = H_S x.  ``keys``: sorted unique [D, W]; ``x``: [D] or [D, k],
    real or complex.  Returns complex128 of x's shape."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    x = np.asarray(x)
    shape = x.shape
    x2 = x.reshape(D, 1) if x.ndim == 1 else x.reshape(D, x.shape[1])
    k = x2.shape[1]
    xr = np.ascontiguousarray(x2.real, np.float64)
    xi = np.ascontiguousarray(x2.imag, np.float64) if np.iscomplexobj(x2) else None
    yr = np.zeros((D, k))
    yi = np.zeros((D, k))
    tp, oq, oc, cr, ci = _op_arrays(op)
    _check(lib().orc_apply(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                           D, _ptr(keys), k, _ptr(xr), _ptr(xi), _ptr(yr), _ptr(yi)))
    return (yr + 1j * yi).reshape(shape)


def apply_rows(op, keys: np.ndarray, x: np.ndarray, rows) -> np.ndarray:
    """(H_S x)[rows] for a real ``x`` ([D] or [D, k]); complex result (the
    coefficients may be complex).  A complex ``x`` raises TypeError: the C
    routine reads real x only.  ``rows`` may repeat and come in any order."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    if np.iscomplexobj(x):
        raise TypeError("apply_rows takes a real x")
    x = np.asarray(x, np.float64)
    x2 = np.ascontiguousarray(x.reshape(D, 1) if x.ndim == 1 else x)
    k = x2.shape[1]
    rows = np.ascontiguousarray(rows, np.int64)
    yr = np.zeros((rows.shape[0], k))
    yi = np.zeros((rows.shape[0], k))
    tp, oq, oc, cr, ci = _op_arrays(op)
    _check(lib().orc_apply_rows(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                                D, _ptr(keys), k, _ptr(x2), rows.shape[0], _ptr(rows), _ptr(yr), _ptr(yi)))
    y = yr + 1j * yi
    return y[:, 0] if x.ndim == 1 else y


def diagonal(op, keys: np.ndarray) -> np.ndarray:
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    dr, di = np.zeros(D), np.zeros(D)
    tp, oq, oc, cr, ci = _op_arrays(op)
    _check(lib().orc_diagonal(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                              D, _ptr(keys), _ptr(dr), _ptr(di)))
    return dr + 1j * di


def term_table(op, keys: np.ndarray, row0: int = 0, nrows: int | None = None) -> np.ndarray:
    """int8 [nrows, T]: 0 if <r|W_t|.> is zero, else 1+p with factor i^p."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    nrows = D - row0 if nrows is None else nrows
    out = np.zeros((nrows, op.n_terms), np.int8)
    tp, oq, oc, _, _ = _op_arrays(op)
    _check(lib().orc_term_table(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc),
                                D, _ptr(keys), row0, nrows, _ptr(out)))
    return out


def groups(op) -> np.ndarray:
    """Distinct nonempty flip sets ([G, W]) ordered by (weight, value)."""
    tp, oq, oc, cr, ci = _op_arrays(op)
    W = _W(op.n_qubits)
    out = np.zeros((max(op.n_terms, 1), W), np.uint64)
    g = lib().orc_groups(W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                         op.n_terms, _ptr(out))
    return out[:g].copy()


def target_table(op, keys: np.ndarray, row0: int = 0, nrows: int | None = None) -> np.ndarray:
    """int64 [nrows, G]: per row and group (``groups`` order) -2 when no
    term of the group is nonzero at the row, -1 when the column is absent,
    else the column index."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    nrows = D - row0 if nrows is None else nrows
    g = np.ascontiguousarray(groups(op))
    out = np.zeros((nrows, g.shape[0]), np.int64)
    tp, oq, oc, cr, ci = _op_arrays(op)
    _check(lib().orc_target_table(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr),
                                  _ptr(ci), D, _ptr(keys), g.shape[0], _ptr(g), row0, nrows, _ptr(out)))
    return out


def row_elements(op, row: np.ndarray):
    """Row ``row`` ([W] uint64, any bit-string) of H over the whole Hilbert
    space: (cols [m, W] ascending, elements [m] complex); the diagonal is
    always listed."""
    row = np.ascontiguousarray(row, np.uint64)
    W = row.shape[0]
    tp, oq, oc, cr, ci = _op_arrays(op)
    T = op.n_terms
    cols = np.zeros((T + 1, W), np.uint64)
    re, im = np.zeros(T + 1), np.zeros(T + 1)
    m = lib().orc_row_elements(op.n_qubits, W, T, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci), _ptr(row),
                               _ptr(cols), _ptr(re), _ptr(im))
    if m < 0:
        _check(int(-m))
    return cols[:m].copy(), re[:m] + 1j * im[:m]


def csr(op, keys: np.ndarray):
    """(indptr, indices, data) of H_S: diagonal always stored, columns
    ascending, numeric zeros kept."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    tp, oq, oc, cr, ci = _op_arrays(op)
    L = lib()
    cnt = np.zeros(D, np.int64)
    _check(L.orc_csr_count(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                           D, _ptr(keys), _ptr(cnt)))
    indptr = np.zeros(D + 1, np.int64)
    np.cumsum(cnt, out=indptr[1:])
    nnz = int(indptr[-1])
    indices = np.zeros(nnz, np.int64)
    dr, di = np.zeros(nnz), np.zeros(nnz)
    _check(L.orc_csr_fill(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                          D, _ptr(keys), _ptr(indptr), _ptr(indices), _ptr(dr), _ptr(di)))
    return indptr, indices, dr + 1j * di


def dense(op, keys: np.ndarray) -> np.ndarray:
    """Dense H_S (small D) from the CSR form."""
    indptr, indices, data = csr(op, keys)
    D = keys.shape[0]
    H = np.zeros((D, D), np.complex128)
    for a in range(D):
        H[a, indices[indptr[a]:indptr[a + 1]]] = data[indptr[a]:indptr[a + 1]]
    return H


def tridiag_min(alpha: np.ndarray, beta: np.ndarray) -> float:
    """Smallest eigenvalue of the symmetric tridiagonal matrix with diagonal
    alpha[m] and off-diagonal beta[1..m-1] (beta[0] unused)."""
    a = np.ascontiguousarray(alpha, np.float64)
    b = np.ascontiguousarray(beta, np.float64)
    return float(lib().orc_tridiag_min(a.shape[0], _ptr(a), _ptr(b)))


def lanczos(op, keys: np.ndarray, m_max: int = 300, tol: float = 1e-13, seed: int = 0,
            v0: np.ndarray | None = None):
    """(energy, steps) of the plain FP64 Lanczos on the real symmetric H_S."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D, W = keys.shape
    tp, oq, oc, cr, ci = _op_arrays(op)
    e = np.zeros(1)
    s = np.zeros(1, np.int32)
    v = None if v0 is None else np.ascontiguousarray(v0, np.float64)
    _check(lib().orc_lanczos(op.n_qubits, W, op.n_terms, _ptr(tp), _ptr(oq), _ptr(oc), _ptr(cr), _ptr(ci),
                             D, _ptr(keys), m_max, tol, seed, _ptr(v), _ptr(e), _ptr(s)))
    return float(e[0]), int(s[0])


def ground_energy(op, keys: np.ndarray, tol: float = 1e-12) -> float:
    """Lowest eigenvalue of the real symmetric H_S: dense ``eigh`` for
    D <= 3000, else SciPy's ARPACK (``eigsh``) on the oracle product."""
    keys = np.ascontiguousarray(keys, np.uint64)
    D = keys.shape[0]
    if D <= 3000:
        H = dense(op, keys)
        return float(np.linalg.eigvalsh(H.real if np.allclose(H.imag, 0) else H)[0])
    import scipy.sparse.linalg as sla
    A = sla.LinearOperator((D, D), matvec=lambda v: apply(op, keys, v.reshape(-1)).real, dtype=np.float64)
    vals = sla.eigsh(A, k=1, which="SA", tol=tol, return_eigenvectors=False)
    return float(vals[0])
