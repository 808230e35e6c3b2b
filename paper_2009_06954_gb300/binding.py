"""ctypes binding of ``libasss.so`` (C ABI in ``include/asss.h``).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host memory) or torch tensors (host or CUDA
memory); the library detects device pointers itself.  If ``libasss.so`` has not
been built, importing names from here works but the first call raises
``ImportError`` - there is no fallback implementation.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import sys
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libasss.so")

ASSS_PREC_FP64, ASSS_PREC_MIXED = 0, 1
ASSS_OUTER_TFQMR, ASSS_OUTER_FGMRES = 0, 1
STATUS = {0: "ok", 1: "invalid argument", 2: "malformed pattern", 3: "zero pivot",
          4: "breakdown", 5: "not converged", 6: "stagnation", 7: "rank above r_max",
          8: "device wait timed out", 9: "out of device memory", 10: "CUDA error",
          11: "unsupported input"}
SOFT = {4, 5, 6}


class AsssError(RuntimeError):
    def __init__(self, where, status, msg):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status}): {msg}")
        self.status = status


class CSR(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("gamma", C.c_double), ("k_lanczos", C.c_int), ("reorth", C.c_int),
                ("s_pattern", C.POINTER(CSR)), ("row_perm", C.c_void_p), ("dr", C.c_void_p),
                ("dc", C.c_void_p), ("inner_tol", C.c_double), ("setup_tol", C.c_double),
                ("outer_tol", C.c_double), ("inner_maxit", C.c_int), ("outer_maxit", C.c_int),
                ("restart", C.c_int), ("precision", C.c_int), ("outer", C.c_int), ("r_max", C.c_int),
                ("seed", C.c_uint64), ("lls_tol", C.c_double), ("lls_maxit", C.c_int),
                ("zero_tol", C.c_double), ("wait_timeout_ms", C.c_double), ("stream", C.c_void_p),
                ("inner_format", C.c_int), ("q_bf16", C.c_int), ("s_values", C.c_void_p),
                ("scaling", C.c_int), ("rhs_block", C.c_int), ("sell_sigma", C.c_int), ("sell_split", C.c_int),
                ("factor", C.c_int)]

FORMATS = {"auto": 0, "sell": 1, "diag": 2}
SCALINGS = {"maxes": 0, "matching": 1}
FACTORS = {"diag": 0, "ildl0": 1, "ildl0_bk": 2}


class Stats(C.Structure):
    _fields_ = [("status", C.c_int), ("outer_its", C.c_int), ("cycles", C.c_int),
                ("inner_its_total", C.c_longlong), ("inner_solves", C.c_int),
                ("inner_its_avg", C.c_double), ("relres", C.c_double), ("r", C.c_int),
                ("k_eff", C.c_int), ("prec2", C.c_int), ("lls_its", C.c_int),
                ("lls_relgrad", C.c_double), ("nnz_pattern", C.c_longlong),
                ("t_setup_ms", C.c_double), ("t_solve_ms", C.c_double), ("t_inner_ms", C.c_double),
                ("inner_bytes", C.c_longlong), ("inner_launches", C.c_int), ("sell_sigma", C.c_int),
                ("sell_split", C.c_int), ("factor_colours", C.c_int), ("t_op_ms", C.c_double),
                ("op_calls", C.c_int), ("op_bytes", C.c_longlong), ("op_flops", C.c_longlong), ("t_orth_ms", C.c_double),
                ("orth_calls", C.c_int), ("orth_bytes", C.c_longlong), ("orth_flops", C.c_longlong),
                ("factor_pairs", C.c_int)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTED = ["asss_default_options", "asss_setup", "asss_solve", "asss_solve_adjoint",
            "asss_apply_operator", "asss_apply_preconditioner", "asss_export", "asss_destroy",
            "asss_status_str", "asss_last_error", "asss_skew_symmetrizer", "asss_skew_lanczos",
            "asss_mrs", "asss_mrs_multi", "asss_kernel_launches", "asss_mrs_noalloc", "asss_export_permutation",
            "asss_matching_scaling", "asss_export_factor", "asss_export_pivots", "asss_setup_batched",
            "asss_solve_batched", "asss_destroy_batched", "asss_batch_cta_threads", "asss_batch_cta_registers"]

_lib = None
_live = weakref.WeakSet()   # open handles, closed at exit while CUDA is still up


@atexit.register
def _close_all():
    for s in list(_live):
        try:
            s.close()
        except Exception:
            pass


def lib():
    """Load libasss.so once and declare the C signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run __graft_entry__.build() "
                          "(or python -m paper_2009_06954_gb300.build)")
    L = C.CDLL(LIB_PATH)
    P = C.c_void_p
    pS = C.POINTER(Stats)
    pCSR = C.POINTER(CSR)
    pO = C.POINTER(Options)
    L.asss_default_options.argtypes = [pO]
    L.asss_default_options.restype = None
    L.asss_setup.argtypes = [pCSR, pO, C.POINTER(P), pS]
    L.asss_solve.argtypes = [P, C.c_int, P, C.c_int64, P, C.c_int64, pS]
    L.asss_solve_adjoint.argtypes = [P, C.c_int, P, C.c_int64, P, C.c_int64, P, C.c_int64, P, pS]
    L.asss_apply_operator.argtypes = [P, C.c_int, P, P]
    L.asss_apply_preconditioner.argtypes = [P, C.c_int, P, P, pS]
    L.asss_export.argtypes = [P, P, P, P, P, P, P, P, P]
    L.asss_destroy.argtypes = [P]
    L.asss_destroy.restype = None
    L.asss_status_str.argtypes = [C.c_int]
    L.asss_status_str.restype = C.c_char_p
    L.asss_last_error.argtypes = []
    L.asss_last_error.restype = C.c_char_p
    L.asss_skew_symmetrizer.argtypes = [pCSR, pCSR, pO, P, pS]
    L.asss_skew_lanczos.argtypes = [pCSR, P, C.c_int, C.c_int, P, P, C.POINTER(C.c_int), P]
    L.asss_mrs.argtypes = [pCSR, C.c_int, P, P, C.c_double, C.c_double, P, P, C.c_double, C.c_int,
                           C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double), P]
    L.asss_export_permutation.argtypes = [P, P]
    L.asss_export_factor.argtypes = [P, P, P, P, P, C.c_int64, C.POINTER(C.c_int64)]
    L.asss_export_pivots.argtypes = [P, P, P, P, P, P, P, C.POINTER(C.c_int)]
    L.asss_matching_scaling.argtypes = [pCSR, P, P, P, C.POINTER(C.c_int), P]
    L.asss_mrs_multi.argtypes = [pCSR, C.c_int, P, P, C.c_double, C.c_double, C.c_int, P, C.c_int64, P, C.c_int64,
                                 C.c_double, C.c_int, C.c_int, C.c_int, P, P, P]
    L.asss_mrs_noalloc.argtypes = [C.c_int64, C.c_int64, P, P, P, C.c_int, C.c_int, P, P, C.c_double,
                                   C.c_double, P, P, C.c_double, C.c_int, C.POINTER(C.c_int),
                                   C.POINTER(C.c_double), P]
    L.asss_mrs_noalloc.restype = C.c_int
    L.asss_setup_batched.argtypes = [C.c_int, C.POINTER(pCSR), pO, C.POINTER(P), pS]
    L.asss_solve_batched.argtypes = [P, C.c_int, P, P, pS]
    L.asss_destroy_batched.argtypes = [P]
    L.asss_destroy_batched.restype = None
    L.asss_batch_cta_threads.argtypes = [P]
    L.asss_batch_cta_threads.restype = C.c_int
    L.asss_batch_cta_registers.argtypes = [P]
    L.asss_batch_cta_registers.restype = C.c_int
    L.asss_kernel_launches.argtypes = []
    L.asss_kernel_launches.restype = C.c_ulonglong
    for f in ("asss_setup", "asss_solve", "asss_solve_adjoint", "asss_apply_operator",
              "asss_apply_preconditioner", "asss_export", "asss_skew_symmetrizer",
              "asss_skew_lanczos", "asss_mrs", "asss_mrs_multi", "asss_setup_batched", "asss_solve_batched",
              "asss_export_permutation", "asss_matching_scaling", "asss_export_factor", "asss_export_pivots"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _check(where, status, soft_ok=False):
    if status == 0 or (soft_ok and status in SOFT):
        return
    raise AsssError(where, status, lib().asss_last_error().decode(errors="replace"))


# ----------------------------------------------------------------------------
# array plumbing
# ----------------------------------------------------------------------------
def _is_torch(a):
    return type(a).__module__.startswith("torch")


def _ptr(a, keep):
    """Raw pointer of a contiguous numpy array / torch tensor (kept alive in keep)."""
    if a is None:
        return None
    if _is_torch(a):
        if not a.is_contiguous():
            a = a.contiguous()
        keep.append(a)
        return a.data_ptr()
    a = np.ascontiguousarray(a)
    keep.append(a)
    return a.ctypes.data


def _host(a, dtype):
    if _is_torch(a):
        a = a.detach().cpu().numpy()
    return np.ascontiguousarray(np.asarray(a, dtype=dtype))


def _csr_struct(A, keep, values=True):
    """scipy.sparse matrix (or (indptr, indices, data, n)) -> CSR struct."""
    if isinstance(A, tuple):
        indptr, indices, data, n = A
    else:
        import scipy.sparse as sp
        A = sp.csr_matrix(A)
        A.sort_indices()
        indptr, indices, data, n = A.indptr, A.indices, A.data, A.shape[0]
    rp = _host(indptr, np.int64)
    ci = _host(indices, np.int32)
    keep += [rp, ci]
    vp = None
    if values and data is not None:
        v = _host(data, np.float64) if not _is_torch(data) or not data.is_cuda else data
        vp = _ptr(v, keep)
    s = CSR(int(n), int(ci.size), rp.ctypes.data, ci.ctypes.data, vp)
    keep.append(s)
    return s


def default_options():
    o = Options()
    lib().asss_default_options(C.byref(o))
    return o


def _options(keep, **kw):
    o = default_options()
    prec = kw.pop("precision", None)
    if prec is not None:
        o.precision = {"fp64": ASSS_PREC_FP64, "mixed": ASSS_PREC_MIXED}.get(prec, prec)
    outer = kw.pop("outer", None)
    if outer is not None:
        o.outer = {"tfqmr": ASSS_OUTER_TFQMR, "fgmres": ASSS_OUTER_FGMRES}.get(outer, outer)
    sp_ = kw.pop("s_pattern", None)
    if sp_ is not None:
        s = _csr_struct(sp_, keep, values=False)
        o.s_pattern = C.pointer(s)
    for name in ("row_perm", "dr", "dc", "s_values"):
        v = kw.pop(name, None)
        if v is not None:
            arr = _host(v, np.int32 if name == "row_perm" else np.float64)
            keep.append(arr)
            setattr(o, name, arr.ctypes.data)
    fmt = kw.pop("inner_format", None)
    if fmt is not None:
        o.inner_format = FORMATS.get(fmt, fmt)
    scl = kw.pop("scaling", None)
    if scl is not None:
        o.scaling = SCALINGS.get(scl, scl)
    fac = kw.pop("factor", None)
    if fac is not None:
        o.factor = FACTORS.get(fac, fac)
    stream = kw.pop("stream", None)
    if stream is not None:
        o.stream = stream if isinstance(stream, int) else stream.cuda_stream
    if "k" in kw:
        kw["k_lanczos"] = kw.pop("k")
    for key, val in kw.items():
        if val is None:
            continue
        if key in ("reorth", "q_bf16", "rhs_block"):
            val = int(bool(val))
        setattr(o, key, val)
    return o


# ----------------------------------------------------------------------------
# whole-method API
# ----------------------------------------------------------------------------
class Solver:
    """Set-up once (§4.1 pre-processing), then solve for any number of b.

    A: scipy.sparse matrix (host).  Options follow ``asss_options``: precision
    ('fp64' | 'mixed'), outer ('tfqmr' | 'fgmres'), gamma, k, reorth, s_pattern,
    inner_tol, setup_tol, outer_tol, inner_maxit, outer_maxit, restart, r_max,
    seed, lls_tol, lls_maxit, zero_tol, wait_timeout_ms, row_perm, dr, dc, stream, s_values,
    scaling ('maxes' | 'matching': how Eq. mc64's P, D_r, D_c are found when none is given),
    rhs_block (several right-hand sides in lockstep blocks sharing multi-column mrs launches),
    factor ('diag' | 'ildl0': the no-fill incomplete L D L^T of M^, §3 / §4.1 ~ildl(0)),
    sell_sigma, sell_split (SELL-C storage of J~: sorting window and work-unit width; 0 = tuned)
    (saved S values to resume the set-up from, e.g. ``export(nnz)["s_val"]`` of an
    earlier solver for the same matrix).
    """

    def __init__(self, A, **opts):
        self._keep = []
        self.n = int(A.shape[0])
        self.nnz = int(A.nnz)
        csr = _csr_struct(A, self._keep)
        self._opts = _options(self._keep, **opts)
        h = C.c_void_p()
        st = Stats()
        status = lib().asss_setup(C.byref(csr), C.byref(self._opts), C.byref(h), C.byref(st))
        _check("asss_setup", status)
        self._h = h
        self.setup_stats = st.as_dict()
        _live.add(self)

    def close(self):
        if getattr(self, "_h", None):
            lib().asss_destroy(self._h)
            self._h = None

    def __del__(self):
        # during interpreter shutdown the process exit releases device memory; no
        # CUDA call is made then
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def _out_like(self, b, cols):
        if _is_torch(b):
            import torch
            return torch.empty((cols, self.n), dtype=torch.float64, device=b.device).T if cols > 1 \
                else torch.empty(self.n, dtype=torch.float64, device=b.device)
        return np.empty((self.n, cols), order="F") if cols > 1 else np.empty(self.n)

    def solve(self, b, x=None):
        """x with ||b - A x|| <= outer_tol ||b||; b is n or n x nrhs (column-major)."""
        keep = []
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        if not _is_torch(b):
            b = np.asfortranarray(np.asarray(b, dtype=np.float64))
        if x is None:
            x = self._out_like(b, nrhs)
        st = Stats()
        status = lib().asss_solve(self._h, nrhs, _ptr_f(b, keep), self.n, _ptr_f(x, keep), self.n,
                                  C.byref(st))
        _check("asss_solve", status, soft_ok=True)
        return x, st.as_dict()

    def solve_adjoint(self, g, x=None, lam=None, dA=None):
        """lambda with A^T lambda = g; with x also dA_e = -lambda_i x_j on A's nonzeros.
        lam (n) and dA (nnz), when given, receive the results (host or device, e.g.
        pinned host buffers kept across calls); otherwise they are allocated like g."""
        keep = []
        if lam is None:
            lam = self._out_like(g, 1)
        _check_out("lam", lam, self.n)
        xp = None
        if x is not None:
            if dA is None:
                if _is_torch(g):
                    import torch
                    dA = torch.empty(self.nnz, dtype=torch.float64, device=g.device)
                else:
                    dA = np.empty(self.nnz)
            _check_out("dA", dA, self.nnz)
            xp = _ptr_f(x, keep)
        else:
            dA = None
        st = Stats()
        status = lib().asss_solve_adjoint(self._h, 1, _ptr_f(g, keep), self.n, _ptr_f(lam, keep),
                                          self.n, xp, self.n, _ptr_f(dA, keep), C.byref(st))
        _check("asss_solve_adjoint", status, soft_ok=True)
        return lam, dA, st.as_dict()

    def apply_operator(self, v, transpose=False):
        keep = []
        out = self._out_like(v, 1)
        _check("asss_apply_operator",
               lib().asss_apply_operator(self._h, int(transpose), _ptr_f(v, keep), _ptr_f(out, keep)))
        return out

    def apply_preconditioner(self, u, transpose=False):
        keep = []
        out = self._out_like(u, 1)
        st = Stats()
        _check("asss_apply_preconditioner",
               lib().asss_apply_preconditioner(self._h, int(transpose), _ptr_f(u, keep),
                                               _ptr_f(out, keep), C.byref(st)))
        return out, int(st.inner_its_total)

    def export_permutation(self):
        """Row permutation of Eq. mc64: row i of Abar is row perm[i] of D_r A D_c."""
        out = np.empty(self.n, dtype=np.int32)
        _check("asss_export_permutation", lib().asss_export_permutation(self._h, out.ctypes.data))
        return out

    def export_factor(self):
        """The incomplete factor (factor='ildl0'): colour of each row and L (strictly
        lower in the (colour, index) order, original indexing) as scipy CSR."""
        import scipy.sparse as sp
        n = self.n
        nl = C.c_int64(0)
        _check("asss_export_factor", lib().asss_export_factor(self._h, None, None, None, None, 0, C.byref(nl)))
        colour = np.empty(n, dtype=np.int32)
        rp = np.empty(n + 1, dtype=np.int64)
        ci = np.empty(max(nl.value, 1), dtype=np.int32)
        lv = np.empty(max(nl.value, 1))
        _check("asss_export_factor", lib().asss_export_factor(self._h, colour.ctypes.data, rp.ctypes.data,
                                                              ci.ctypes.data, lv.ctypes.data, nl.value,
                                                              C.byref(nl)))
        L = sp.csr_matrix((lv[:nl.value], ci[:nl.value], rp), shape=(n, n))
        return colour, L

    def export_pivots(self):
        """The 2x2 pivots (factor='ildl0_bk'): partner of each row (-1: 1x1), the
        off-diagonal D entries, and U_r (n x r dense) of M~_r = -2 U_r U_r^T; None when
        no 2x2 block was formed."""
        n = self.n
        r = int(self.setup_stats["r"])
        npairs = C.c_int(0)
        part = np.empty(n, dtype=np.int32)
        doff = np.empty(n)
        i1 = np.empty(max(r, 1), dtype=np.int32)
        i2 = np.empty(max(r, 1), dtype=np.int32)
        c1 = np.empty(max(r, 1))
        c2 = np.empty(max(r, 1))
        _check("asss_export_pivots", lib().asss_export_pivots(self._h, part.ctypes.data, doff.ctypes.data,
                                                              i1.ctypes.data, i2.ctypes.data, c1.ctypes.data,
                                                              c2.ctypes.data, C.byref(npairs)))
        if npairs.value == 0:
            return None
        U = np.zeros((n, r))
        for a in range(r):
            U[i1[a], a] += c1[a]
            if i2[a] >= 0:
                U[i2[a], a] += c2[a]
        return {"npairs": npairs.value, "partner": part.astype(np.int64), "d_off": doff, "Ur": U}

    def export(self, s_nnz):
        n = self.n
        k = int(self.setup_stats["k_eff"])
        r = int(self.setup_stats["r"])
        out = {"dr": np.empty(n), "dc": np.empty(n), "w": np.empty(n), "d": np.empty(n),
               "s_val": np.empty(s_nnz), "Q": np.empty((n, k), order="F"),
               "alpha": np.empty(max(k - 1, 0)), "neg": np.empty(r, dtype=np.int32)}
        keep = []
        _check("asss_export", lib().asss_export(
            self._h, *[_ptr_f(out[key], keep) for key in ("dr", "dc", "w", "d", "s_val", "Q", "alpha", "neg")]))
        return out


class BatchSolver:
    """Many systems of uneven size, each set up once, solved together by one
    persistent launch (replayed CUDA graph) for nrhs right-hand sides each.

    mats: list of scipy.sparse matrices.  Options as for ``Solver``; precision,
    outer method and J~ storage are fixed (mixed, flexible GMRES, skew-diagonal),
    restart is capped at 24.  ``solve`` takes b as one concatenated vector: system m
    occupies [off_m * nrhs, (off_m + n_m) * nrhs), column-major n_m x nrhs, with
    off_m the sum of the sizes before it (``offsets``).
    """

    def __init__(self, mats, **opts):
        self._keep = []
        self.sizes = [int(A.shape[0]) for A in mats]
        self.offsets = np.concatenate([[0], np.cumsum(self.sizes)]).astype(np.int64)
        self.total = int(self.offsets[-1])
        structs = [_csr_struct(A, self._keep) for A in mats]
        arr = (C.POINTER(CSR) * len(structs))(*[C.pointer(c) for c in structs])
        self._keep.append(arr)
        self._opts = _options(self._keep, **opts)
        h = C.c_void_p()
        st = Stats()
        status = lib().asss_setup_batched(len(structs), arr, C.byref(self._opts), C.byref(h), C.byref(st))
        _check("asss_setup_batched", status)
        self._h = h
        self.setup_stats = st.as_dict()
        _live.add(self)

    @property
    def cta_threads(self):
        """CTA size picked by the tuner on the first solve (0 before it)."""
        return int(lib().asss_batch_cta_threads(self._h)) if getattr(self, "_h", None) else 0

    @property
    def cta_registers(self):
        """Registers a thread of the CTA shape picked by the tuner (64, 80 or 128; 0 before it)."""
        return int(lib().asss_batch_cta_registers(self._h)) if getattr(self, "_h", None) else 0

    def close(self):
        if getattr(self, "_h", None):
            lib().asss_destroy_batched(self._h)
            self._h = None

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def pack(self, blocks):
        """List of n_m x nrhs (or n_m) arrays -> concatenated numpy vector."""
        return np.concatenate([np.asarray(b, dtype=np.float64).reshape(len(b), -1).ravel(order="F")
                               for b in blocks])

    def unpack(self, v, nrhs):
        v = np.asarray(v)
        return [v[o * nrhs:(o + n) * nrhs].reshape((n, nrhs), order="F")
                for o, n in zip(self.offsets[:-1], self.sizes)]

    def solve(self, b, nrhs=1, x=None):
        """x for every (system, column); b host or device, length total * nrhs."""
        keep = []
        if not _is_torch(b):
            b = np.ascontiguousarray(b, dtype=np.float64)
        if b.shape[0] != self.total * nrhs:
            raise ValueError(f"b must have {self.total * nrhs} entries")
        if x is None:
            if _is_torch(b):
                import torch
                x = torch.empty_like(b)
            else:
                x = np.empty_like(b)
        st = Stats()
        status = lib().asss_solve_batched(self._h, int(nrhs), _ptr_f(b, keep), _ptr_f(x, keep), C.byref(st))
        _check("asss_solve_batched", status, soft_ok=True)
        return x, st.as_dict()


def _check_out(name, a, size):
    """An output buffer: float64, contiguous, size entries."""
    if _is_torch(a):
        ok = a.dtype.is_floating_point and a.element_size() == 8 and a.is_contiguous() and a.numel() == size
    else:
        ok = a.dtype == np.float64 and a.flags.c_contiguous and a.size == size
    if not ok:
        raise ValueError(f"{name} must be a contiguous float64 buffer of {size} entries")


def _ptr_f(a, keep):
    if a is None:
        return None
    if _is_torch(a):
        keep.append(a)
        return a.data_ptr()
    if not (a.flags.f_contiguous or a.flags.c_contiguous):
        raise ValueError("array must be contiguous")
    keep.append(a)
    return a.ctypes.data


# ----------------------------------------------------------------------------
# single steps
# ----------------------------------------------------------------------------
def skew_symmetrizer(Abar, s_pattern, gamma=1.0, lls_tol=1e-13, lls_maxit=20000):
    """S values (pattern CSR order) minimising the §2 least-squares objective."""
    keep = []
    a = _csr_struct(Abar, keep)
    p = _csr_struct(s_pattern, keep, values=False)
    o = _options(keep, gamma=gamma, lls_tol=lls_tol, lls_maxit=lls_maxit)
    out = np.empty(p.nnz)
    st = Stats()
    _check("asss_skew_symmetrizer",
           lib().asss_skew_symmetrizer(C.byref(a), C.byref(p), C.byref(o), out.ctypes.data, C.byref(st)))
    return out, st.as_dict()


def skew_lanczos(J, q1, k, reorth=True):
    """(Q n x k_eff, alpha) from k steps of Fig. 2 on the skew matrix J."""
    keep = []
    a = _csr_struct(J, keep)
    n = int(a.n)
    q1 = np.ascontiguousarray(q1, dtype=np.float64)
    Q = np.empty((n, max(k, 1)), order="F")
    alpha = np.empty(max(k - 1, 1))
    ke = C.c_int(0)
    _check("asss_skew_lanczos", lib().asss_skew_lanczos(C.byref(a), q1.ctypes.data, int(k), int(bool(reorth)),
                                                          Q.ctypes.data, alpha.ctypes.data, C.byref(ke), None))
    ke = ke.value
    return np.asfortranarray(Q[:, :ke]), alpha[:max(ke - 1, 0)].copy()


def mrs(J, b, Q=None, alpha=None, shift=1.0, sign=1.0, tol=1e-10, maxit=1000, precision="fp64",
        fmt="auto"):
    """mrs (App. B) on (shift I + sign (J - Q S_k Q^T)) x = b; returns (x, its, ratio)."""
    keep = []
    a = _csr_struct(J, keep)
    n = int(a.n)
    k = 0 if Q is None else Q.shape[1]
    qp = None
    ap = None
    if k:
        Qf = np.asfortranarray(Q, dtype=np.float64)
        keep.append(Qf)
        qp = Qf.ctypes.data
        if k > 1:
            al = np.ascontiguousarray(alpha, dtype=np.float64)
            keep.append(al)
            ap = al.ctypes.data
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.empty(n)
    its = C.c_int(0)
    ratio = C.c_double(0.0)
    prec = {"fp64": ASSS_PREC_FP64, "mixed": ASSS_PREC_MIXED, "fp32": ASSS_PREC_MIXED}[precision]
    _check("asss_mrs", lib().asss_mrs(C.byref(a), k, qp, ap, float(shift), float(sign), b.ctypes.data,
                                      x.ctypes.data, float(tol), int(maxit), prec, FORMATS[fmt], C.byref(its),
                                      C.byref(ratio), None))
    return x, its.value, ratio.value


def matching_scaling(A):
    """(row_perm, dr, dc, rounds): maximum-product matching and dual scalings (Eq. mc64)."""
    keep = []
    a = _csr_struct(A, keep)
    n = int(a.n)
    perm = np.empty(n, dtype=np.int32)
    dr = np.empty(n)
    dc = np.empty(n)
    rounds = C.c_int(0)
    _check("asss_matching_scaling", lib().asss_matching_scaling(C.byref(a), perm.ctypes.data, dr.ctypes.data,
                                                                dc.ctypes.data, C.byref(rounds), None))
    return perm, dr, dc, rounds.value


def mrs_multi(J, B, Q=None, alpha=None, shift=1.0, sign=1.0, tol=1e-10, maxit=1000, precision="fp64",
              fmt="auto"):
    """App. B's simultaneous mrs iterations for the columns of B (n x nrhs); returns
    (X, its[nrhs], ratio[nrhs])."""
    keep = []
    a = _csr_struct(J, keep)
    n = int(a.n)
    k = 0 if Q is None else Q.shape[1]
    qp = ap = None
    if k:
        Qf = np.asfortranarray(Q, dtype=np.float64)
        keep.append(Qf)
        qp = Qf.ctypes.data
        if k > 1:
            al = np.ascontiguousarray(alpha, dtype=np.float64)
            keep.append(al)
            ap = al.ctypes.data
    B = np.asfortranarray(np.asarray(B, dtype=np.float64).reshape(n, -1))
    nrhs = B.shape[1]
    X = np.empty((n, nrhs), order="F")
    its = np.zeros(nrhs, dtype=np.int32)
    ratio = np.zeros(nrhs)
    prec = {"fp64": ASSS_PREC_FP64, "mixed": ASSS_PREC_MIXED, "fp32": ASSS_PREC_MIXED}[precision]
    _check("asss_mrs_multi", lib().asss_mrs_multi(C.byref(a), k, qp, ap, float(shift), float(sign), nrhs,
                                                  B.ctypes.data, n, X.ctypes.data, n, float(tol), int(maxit), prec,
                                                  FORMATS[fmt], its.ctypes.data, ratio.ctypes.data, None))
    return X, its, ratio


def kernel_launches() -> int:
    """Kernels launched by libasss.so in this process so far."""
    return int(lib().asss_kernel_launches())
