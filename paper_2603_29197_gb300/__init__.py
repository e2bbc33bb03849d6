"""Python binding of the GB300 QOCO-style interior-point solver.

Thin layer over the C ABI (include/qoco_gpu.h): it converts CSC matrices and numpy
arrays to the ABI's plain pointers, passes torch CUDA tensors by data pointer and
the current torch stream as the cudaStream_t.  Every step of the method runs in
libqoco_gpu.so; nothing here computes.

Use (a problem is any object with n, m, p, P, c, A, b, G, h, l, q; P upper CSC):

    import paper_2603_29197_gb300 as q
    S = q.Solver(prob)                      # validation, ordering, symbolic analysis, upload
    status = S.solve()                      # 0 = solved to 1e-7
    sol = S.solution()                      # x, s, y, z (numpy) and the info dict
    grads = S.backward(dx=gx)               # gx = dL/dx as a CUDA float64 tensor → dP, dc, dA, db, dG, dh
    S.update_data(c=new_c); S.solve()       # same pattern, new numbers: no new analysis
    B = q.BatchSolver(list_of_problems)     # one interior-point loop over many instances
    S.close(); B.close()

`solve_function()` wraps solve + backward as a torch.autograd.Function.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (ORDER_AMD, ORDER_AUTO, ORDER_ND, ORDER_NATURAL, STATUS_NAMES,  # noqa: F401
                   Info, Settings)

__all__ = ["Solver", "BatchSolver", "Cones", "analyze", "default_settings", "load", "STATUS_NAMES",
           "solve_function"]


def load():
    return _lib.load()


def default_settings(**kw) -> Settings:
    st = Settings()
    load().qoco_gpu_default_settings(C.byref(st))
    for k, v in kw.items():
        if not hasattr(st, k):
            raise TypeError(f"unknown setting {k!r}")
        setattr(st, k, v)
    return st


class _CSCHold:
    """Keeps the int32/float64 copies of one CSC matrix alive for a call."""

    def __init__(self, M, rows, cols):
        if M is None:
            self.ptr = None
            return
        M = M.tocsc() if hasattr(M, "tocsc") else M
        self.colptr = np.ascontiguousarray(M.indptr, dtype=np.int32)
        self.rowidx = np.ascontiguousarray(M.indices, dtype=np.int32)
        self.val = np.ascontiguousarray(M.data, dtype=np.float64)
        self.s = _lib.CSC(int(M.shape[0]), int(M.shape[1]), int(self.rowidx.size),
                          self.colptr.ctypes.data_as(C.POINTER(C.c_int)),
                          self.rowidx.ctypes.data_as(C.POINTER(C.c_int)),
                          self.val.ctypes.data_as(C.POINTER(C.c_double)))
        self.ptr = C.byref(self.s)


# numpy mirror of qoco_csc (same field offsets), for tables of many matrices
_CSC_DTYPE = np.dtype({"names": [f for f, _ in _lib.CSC._fields_],
                       "formats": [np.int32, np.int32, np.int32, np.uintp, np.uintp, np.uintp],
                       "offsets": [getattr(_lib.CSC, f).offset for f, _ in _lib.CSC._fields_],
                       "itemsize": C.sizeof(_lib.CSC)})


def _csc_row(tab, i, M, rows, cols):
    """Fills tab[i] (a _CSC_DTYPE table) from the CSC matrix M; returns the int32/float64
    copies that must stay alive for the call."""
    M = M.tocsc() if hasattr(M, "tocsc") else M
    colptr = np.ascontiguousarray(M.indptr, dtype=np.int32)
    rowidx = np.ascontiguousarray(M.indices, dtype=np.int32)
    val = np.ascontiguousarray(M.data, dtype=np.float64)
    tab[i] = (rows, cols, rowidx.size, colptr.ctypes.data, rowidx.ctypes.data, val.ctypes.data)
    return colptr, rowidx, val


def _dptr(a):
    return None if a is None else a.ctypes.data_as(C.POINTER(C.c_double))


def _vec(a, n):
    if a is None or n == 0:
        return None
    return np.ascontiguousarray(a, dtype=np.float64)


def _settings(settings, kw):
    if settings is None:
        return default_settings(**kw)
    for k, v in kw.items():
        setattr(settings, k, v)
    return settings


def _problem_args(prob):
    n, m, p = int(prob.n), int(prob.m), int(prob.p)
    P = _CSCHold(prob.P if getattr(prob, "P", None) is not None and prob.P.nnz else None, n, n)
    A = _CSCHold(prob.A if p else None, p, n)
    G = _CSCHold(prob.G if m else None, m, n)
    q = np.ascontiguousarray(list(prob.q), dtype=np.int32)
    return n, m, p, P, A, G, q


def _torch_stream(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _tptr(t):
    return C.c_void_p(0 if t is None else t.data_ptr())


def _batch_tables(probs):
    """The per-instance arguments of qoco_gpu_setup_batch / qoco_gpu_analyze_batch: the
    arrays to keep alive, the size lists (n, m, p, l, nsoc) and the tables (P, c, A, b, G,
    h, q).  The qoco_csc structs and pointer tables are filled as numpy arrays of
    addresses (one ctypes conversion per table, not one per instance)."""
    nb = len(probs)
    holds = []
    ns, ms, ps, ls, nsocs = [], [], [], [], []
    Ps, As, Gs = (np.zeros(nb, dtype=_CSC_DTYPE) for _ in range(3))
    cs, bs, hs, qs = (np.zeros(nb, dtype=np.uintp) for _ in range(4))
    for i, pr in enumerate(probs):
        n, m, p = int(pr.n), int(pr.m), int(pr.p)
        q = np.ascontiguousarray(list(pr.q), dtype=np.int32)
        Pm = pr.P if getattr(pr, "P", None) is not None and pr.P.nnz else None
        for M, rows, tab in ((Pm, n, Ps), (pr.A if p else None, p, As), (pr.G if m else None, m, Gs)):
            if M is not None:
                holds.append(_csc_row(tab, i, M, rows, n))
        for v, k, tab in ((pr.c, n, cs), (pr.b, p, bs), (pr.h, m, hs)):
            a = _vec(v, k)
            if a is not None:
                holds.append(a)
                tab[i] = a.ctypes.data
        holds.append(q)
        if len(q):
            qs[i] = q.ctypes.data
        ns.append(n); ms.append(m); ps.append(p); ls.append(int(pr.l)); nsocs.append(len(q))
    dp = C.POINTER(C.POINTER(C.c_double))
    tables = (Ps.ctypes.data_as(C.POINTER(_lib.CSC)), cs.ctypes.data_as(dp), As.ctypes.data_as(C.POINTER(_lib.CSC)),
              bs.ctypes.data_as(dp), Gs.ctypes.data_as(C.POINTER(_lib.CSC)), hs.ctypes.data_as(dp),
              qs.ctypes.data_as(C.POINTER(C.POINTER(C.c_int))))
    return holds, (ns, ms, ps, ls, nsocs), tables


def analyze_batch(probs, settings=None, **kw):
    """Host-only analysis of a batch as qoco_gpu_setup_batch makes it (no GPU needed):
    returns (info, perm, sn_ptr, f_s, level_s) in the stack's numbering."""
    lib = load()
    st = _settings(settings, kw)
    nb = len(probs)
    holds, (ns, ms, ps, ls, nsocs), (Ps, _, As, _, Gs, _, qs) = _batch_tables(probs)
    arr = lambda v: (C.c_int * nb)(*v)  # noqa: E731
    args = (nb, arr(ns), arr(ms), arr(ps), Ps, As, Gs, arr(ls), arr(nsocs), qs, C.byref(st))
    info = Info()
    N = sum(ns) + sum(ms) + sum(ps)
    perm = np.zeros(N, dtype=np.int32)
    ip = C.POINTER(C.c_int)
    rc = lib.qoco_gpu_analyze_batch(*args, C.byref(info), perm.ctypes.data_as(ip), None, None, None)
    if rc != 0:
        raise ValueError(f"batch analysis failed: {STATUS_NAMES.get(rc, rc)}: {info.message.decode()}")
    ns_ = info.n_supernodes
    sn = np.zeros(ns_ + 1, dtype=np.int32)
    fs = np.zeros(max(1, ns_), dtype=np.int32)
    lv = np.zeros(max(1, ns_), dtype=np.int32)
    lib.qoco_gpu_analyze_batch(*args, None, None, sn.ctypes.data_as(ip), fs.ctypes.data_as(ip), lv.ctypes.data_as(ip))
    del holds
    return info.as_dict(), perm, sn, fs[:ns_], lv[:ns_]


def analyze(prob, settings=None, structure=False, **kw):
    """Host-only ordering + symbolic analysis (no GPU needed): returns (info, perm, sn_ptr),
    plus (f_s, level_s) per supernode when structure=True."""
    lib = load()
    st = _settings(settings, kw)
    n, m, p, P, A, G, q = _problem_args(prob)
    info = Info()
    N = n + p + m
    perm = np.zeros(N, dtype=np.int32)
    rc = lib.qoco_gpu_analyze(n, m, p, P.ptr, A.ptr, G.ptr, int(prob.l), len(q),
                              q.ctypes.data_as(C.POINTER(C.c_int)), C.byref(st), C.byref(info),
                              perm.ctypes.data_as(C.POINTER(C.c_int)), None, None, None)
    if rc != 0:
        raise ValueError(f"analysis failed: {STATUS_NAMES.get(rc, rc)}: {info.message.decode()}")
    sn = np.zeros(info.n_supernodes + 1, dtype=np.int32)
    fs = np.zeros(max(1, info.n_supernodes), dtype=np.int32)
    lv = np.zeros(max(1, info.n_supernodes), dtype=np.int32)
    ip = C.POINTER(C.c_int)
    lib.qoco_gpu_analyze(n, m, p, P.ptr, A.ptr, G.ptr, int(prob.l), len(q),
                         q.ctypes.data_as(ip), C.byref(st), None, None, sn.ctypes.data_as(ip),
                         fs.ctypes.data_as(ip), lv.ctypes.data_as(ip))
    if structure:
        return info.as_dict(), perm, sn, fs[:info.n_supernodes], lv[:info.n_supernodes]
    return info.as_dict(), perm, sn


def fp64_peaks(stream=None):
    """(DFMA, DMMA) GFLOP/s of the current GPU, measured by the library's own kernels
    (qoco_gpu_fp64_peaks)."""
    lib = load()
    a, b = C.c_double(), C.c_double()
    rc = lib.qoco_gpu_fp64_peaks(C.byref(a), C.byref(b), _torch_stream(stream))
    if rc != 0:
        raise SolverError(rc, "fp64_peaks")
    return a.value, b.value


class SolverError(RuntimeError):
    def __init__(self, code, msg=""):
        super().__init__(f"{STATUS_NAMES.get(code, code)} ({code}) {msg}")
        self.code = code


class Solver:
    """setup(n, m, p, P, c, A, b, G, h, l, nsoc, q) on construction, then solve()
    (the paper's interface, §2.1).  `prob` is any object with those attributes
    (P upper-triangular CSC)."""

    def __init__(self, prob, settings=None, **kw):
        self.lib = load()
        self.st = _settings(settings, kw)
        n, m, p, P, A, G, q = _problem_args(prob)
        self.n, self.m, self.p = n, m, p
        self.N = n + m + p
        c = _vec(prob.c, n)
        b = _vec(prob.b, p)
        h = _vec(prob.h, m)
        self._h = C.c_void_p()
        rc = self.lib.qoco_gpu_setup(C.byref(self._h), n, m, p, P.ptr, _dptr(c), A.ptr, _dptr(b),
                                     G.ptr, _dptr(h), int(prob.l), len(q),
                                     q.ctypes.data_as(C.POINTER(C.c_int)) if len(q) else None,
                                     C.byref(self.st))
        if rc != 0:
            self._h = None
            raise SolverError(rc, "setup")
        self._nnz = (P.s.nnz if P.ptr is not None else 0, A.s.nnz if A.ptr is not None else 0,
                     G.s.nnz if G.ptr is not None else 0)

    def solve(self, stream=None) -> int:
        return int(self.lib.qoco_gpu_solve(self._h, _torch_stream(stream) if stream is not None else None))

    def info(self) -> dict:
        info = Info()
        self.lib.qoco_gpu_get_info(self._h, C.byref(info))
        return info.as_dict()

    def solution(self):
        x = np.zeros(self.n)
        s = np.zeros(self.m)
        y = np.zeros(self.p)
        z = np.zeros(self.m)
        info = Info()
        rc = self.lib.qoco_gpu_get_solution(self._h, _dptr(x), _dptr(s), _dptr(y), _dptr(z),
                                            C.byref(info))
        if rc != 0:
            raise SolverError(rc, "get_solution")
        return dict(x=x, s=s, y=y, z=z, info=info.as_dict())

    def device_solution(self):
        """(x, s, y, z) as device addresses (ints) owned by the solver."""
        ptrs = [C.c_void_p() for _ in range(4)]
        self.lib.qoco_gpu_solution_device(self._h, *[C.byref(v) for v in ptrs])
        return tuple(v.value for v in ptrs)

    # ---- shared-iterate entry points (torch CUDA float64 tensors) ----
    def kkt_factor_at(self, s, z, stream=None):
        rc = self.lib.qoco_gpu_kkt_factor_at(self._h, _tptr(s), _tptr(z), _torch_stream(stream))
        if rc != 0:
            raise SolverError(rc, "kkt_factor_at")

    def kkt_solve(self, r, x, stream=None):
        steps = C.c_int()
        be = C.c_double()
        rc = self.lib.qoco_gpu_kkt_solve(self._h, _tptr(r), _tptr(x), C.byref(steps), C.byref(be),
                                         _torch_stream(stream))
        if rc != 0:
            raise SolverError(rc, "kkt_solve")
        return steps.value, be.value

    def get_kkt(self):
        info = self.info()
        N, nnz = int(info["kkt_dim"]), int(info["kkt_nnz"])
        rowptr = np.zeros(N + 1, dtype=np.int64)
        col = np.zeros(nnz, dtype=np.int32)
        val = np.zeros(nnz)
        rc = self.lib.qoco_gpu_get_kkt(self._h, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
                                       col.ctypes.data_as(C.POINTER(C.c_int)), _dptr(val))
        if rc != 0:
            raise SolverError(rc, "get_kkt")
        return rowptr, col, val

    def factor_dense(self):
        N = self.N
        perm = np.zeros(N, dtype=np.int32)
        L = np.zeros((N, N))
        D = np.zeros(N)
        rc = self.lib.qoco_gpu_get_factor_dense(self._h, perm.ctypes.data_as(C.POINTER(C.c_int)),
                                                _dptr(L), _dptr(D))
        if rc != 0:
            raise SolverError(rc, "get_factor_dense")
        return perm, L, D

    def pivot_reciprocals(self):
        out = np.zeros(self.N)
        rc = self.lib.qoco_gpu_get_pivot_reciprocals(self._h, _dptr(out))
        if rc != 0:
            raise SolverError(rc, "get_pivot_reciprocals")
        return out

    def set_profiling(self, on=True):
        """True/1: every phase; 2: the factorisation phase alone; False/0: off."""
        rc = self.lib.qoco_gpu_set_profiling(self._h, 2 if on == 2 else (1 if on else 0))
        if rc != 0:
            raise SolverError(rc, "set_profiling")

    def profile(self) -> dict:
        pr = _lib.Profile()
        self.lib.qoco_gpu_get_profile(self._h, C.byref(pr))
        return pr.as_dict()

    def solution_tensors(self, stream=None):
        """Copies of x, y, z in new torch CUDA float64 tensors (device-to-device)."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        x, y, z = (torch.empty(k, dtype=torch.float64, device=dev) for k in (self.n, self.p, self.m))
        rc = self.lib.qoco_gpu_copy_solution(self._h, _tptr(x), None, _tptr(y), _tptr(z), _torch_stream(stream))
        if rc != 0:
            raise SolverError(rc, "copy_solution")
        return x, y, z

    # ---- adjoint and parametric update -------------------------------------------
    def nnz(self):
        """Stored entries of P (upper), A and G as given at setup."""
        return self._nnz

    def backward(self, dx=None, dy=None, dz=None, stream=None):
        """Gradients of a loss with respect to (P values, c, A values, b, G values, h)
        given its gradients with respect to x, y, z (torch CUDA float64 tensors or None).
        Returns a dict of torch CUDA tensors dP, dc, dA, db, dG, dh."""
        import torch
        dev = torch.device("cuda", torch.cuda.current_device())
        nP, nA, nG = self._nnz
        out = {k: torch.empty(sz, dtype=torch.float64, device=dev)
               for k, sz in (("dP", nP), ("dc", self.n), ("dA", nA), ("db", self.p), ("dG", nG), ("dh", self.m))}
        rc = self.lib.qoco_gpu_backward(self._h, _tptr(dx), _tptr(dy), _tptr(dz), _tptr(out["dP"]),
                                        _tptr(out["dc"]), _tptr(out["dA"]), _tptr(out["db"]),
                                        _tptr(out["dG"]), _tptr(out["dh"]), _torch_stream(stream))
        if rc != 0:
            raise SolverError(rc, "backward")
        return out

    def backward_info(self):
        steps = C.c_int()
        be = C.c_double()
        rf = C.c_int()
        self.lib.qoco_gpu_backward_info(self._h, C.byref(steps), C.byref(be), C.byref(rf))
        return dict(refine_steps=steps.value, backward_error=be.value, refactored=bool(rf.value))

    def update_data(self, P=None, c=None, A=None, b=None, G=None, h=None, stream=None):
        """New values on the setup's sparsity patterns (P, A, G: value arrays in CSC
        order).  All given arrays are numpy (host) or all torch CUDA tensors (device)."""
        given = [a for a in (P, c, A, b, G, h) if a is not None]
        on_device = bool(given) and hasattr(given[0], "data_ptr")
        if on_device:
            args = [_tptr(a) for a in (P, c, A, b, G, h)]
        else:
            keep = [None if a is None else np.ascontiguousarray(a, dtype=np.float64) for a in (P, c, A, b, G, h)]
            args = [C.c_void_p(0) if a is None else C.c_void_p(a.ctypes.data) for a in keep]
        rc = self.lib.qoco_gpu_update_data(self._h, *args, 1 if on_device else 0, _torch_stream(stream))
        if rc != 0:
            raise SolverError(rc, "update_data")

    def close(self):
        if self._h:
            self.lib.qoco_gpu_cleanup(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class BatchSolver(Solver):
    """Independent instances (objects with the attributes Solver takes) solved together
    by one interior-point loop with per-instance scalars (qoco_gpu_setup_batch)."""

    def __init__(self, probs, settings=None, **kw):  # noqa: D401  (own set-up)
        self.lib = load()
        self.st = _settings(settings, kw)
        nb = len(probs)
        holds, (ns, ms, ps, ls, nsocs), (Ps, cs, As, bs, Gs, hs, qs) = _batch_tables(probs)
        arr = lambda v: (C.c_int * nb)(*v)  # noqa: E731
        self.n, self.m, self.p = sum(ns), sum(ms), sum(ps)
        self.N = self.n + self.m + self.p
        self.batch = nb
        self._sizes = (ns, ms, ps)
        self._h = C.c_void_p()
        rc = self.lib.qoco_gpu_setup_batch(C.byref(self._h), nb, arr(ns), arr(ms), arr(ps), Ps, cs, As, bs, Gs,
                                           hs, arr(ls), arr(nsocs), qs, C.byref(self.st))
        if rc != 0:
            self._h = None
            raise SolverError(rc, "setup_batch")
        self._nnz = (sum(int(pr.P.nnz) for pr in probs if getattr(pr, "P", None) is not None),
                     sum(int(pr.A.nnz) for pr, p in zip(probs, ps) if p),
                     sum(int(pr.G.nnz) for pr in probs))
        k = nb + 1
        self.offsets = {key: np.zeros(k, dtype=np.int32) for key in ("xo", "yo", "lo", "ko", "so")}
        self.lib.qoco_gpu_batch_offsets(self._h, *[self.offsets[key].ctypes.data_as(C.POINTER(C.c_int))
                                                   for key in ("xo", "yo", "lo", "ko", "so")])

    def batch_info(self):
        nb = self.batch
        st = np.zeros(nb, dtype=np.int32)
        it = np.zeros(nb, dtype=np.int32)
        po, do, gp = np.zeros(nb), np.zeros(nb), np.zeros(nb)
        rc = self.lib.qoco_gpu_batch_info(self._h, st.ctypes.data_as(C.POINTER(C.c_int)),
                                          it.ctypes.data_as(C.POINTER(C.c_int)), _dptr(po), _dptr(do), _dptr(gp))
        if rc != 0:
            raise SolverError(rc, "batch_info")
        return dict(status=st, iters=it, pobj=po, dobj=do, gap=gp)

    def instance_solutions(self):
        """Per-instance x, s, y, z sliced from the stacked iterate."""
        sol = self.solution()
        o = self.offsets
        L = int(o["lo"][-1])
        out = []
        for i in range(self.batch):
            def cone(v):
                return np.concatenate([v[o["lo"][i]:o["lo"][i + 1]], v[L + o["so"][i]:L + o["so"][i + 1]]])
            out.append(dict(x=sol["x"][o["xo"][i]:o["xo"][i + 1]], y=sol["y"][o["yo"][i]:o["yo"][i + 1]],
                            s=cone(sol["s"]), z=cone(sol["z"])))
        return out


def _solve_function():
    import torch

    class SolveFunction(torch.autograd.Function):
        """(P values, c, A values, b, G values, h) ↦ (x, y, z) through a Solver whose
        sparsity patterns are fixed: forward is update_data + solve, backward is the
        adjoint (qoco_gpu_backward).  Inputs are torch CUDA float64 tensors."""

        @staticmethod
        def forward(ctx, solver, P_val, c, A_val, b, G_val, h):
            solver.update_data(P=P_val, c=c, A=A_val, b=b, G=G_val, h=h)
            st = solver.solve(torch.cuda.current_stream().cuda_stream)
            if st != 0:
                raise SolverError(st, "solve")
            ctx.solver = solver
            return solver.solution_tensors()

        @staticmethod
        def backward(ctx, gx, gy, gz):
            g = ctx.solver.backward(gx.contiguous() if gx is not None else None,
                                    gy.contiguous() if gy is not None else None,
                                    gz.contiguous() if gz is not None else None)
            return None, g["dP"], g["dc"], g["dA"], g["db"], g["dG"], g["dh"]

    return SolveFunction


def solve_function():
    """The torch.autograd.Function class wrapping solve + adjoint."""
    return _solve_function()


class Cones:
    """Device descriptor of K = R^l_+ × Q^{q_0} × … for the stand-alone cone kernels."""

    def __init__(self, l, q):
        self.lib = load()
        self.l = int(l)
        self.q = np.ascontiguousarray(list(q), dtype=np.int32)
        self.m = self.l + int(self.q.sum())
        self._h = C.c_void_p()
        rc = self.lib.qoco_gpu_cones_create(C.byref(self._h), self.l, len(self.q),
                                            self.q.ctypes.data_as(C.POINTER(C.c_int)) if len(self.q) else None)
        if rc != 0:
            self._h = None
            raise SolverError(rc, "cones_create")

    def _check(self, rc, what):
        if rc != 0:
            raise SolverError(rc, what)

    def nt_scaling(self, s, z, stream=None):
        import torch
        w = torch.empty_like(s)
        lam = torch.empty_like(s)
        eta = torch.empty(max(1, len(self.q)), dtype=s.dtype, device=s.device)
        self._check(self.lib.qoco_gpu_cone_nt_scaling(self._h, _tptr(s), _tptr(z), _tptr(w), _tptr(eta),
                                                      _tptr(lam), _torch_stream(stream)), "nt_scaling")
        return w, eta[:len(self.q)], lam

    def product(self, u, v, stream=None):
        import torch
        out = torch.empty_like(u)
        self._check(self.lib.qoco_gpu_cone_product(self._h, _tptr(u), _tptr(v), _tptr(out),
                                                   _torch_stream(stream)), "product")
        return out

    def division(self, lam, v, stream=None):
        import torch
        out = torch.empty_like(v)
        self._check(self.lib.qoco_gpu_cone_division(self._h, _tptr(lam), _tptr(v), _tptr(out),
                                                    _torch_stream(stream)), "division")
        return out

    def max_step_scratch_bytes(self):
        return int(self.lib.qoco_gpu_cone_max_step_scratch_bytes(self._h))

    def max_step(self, u, du, cap=float("inf"), scratch=None, stream=None):
        import torch
        if scratch is None:
            scratch = torch.empty(self.max_step_scratch_bytes() // 8 + 1, dtype=torch.float64,
                                  device=u.device)
        out = torch.empty(1, dtype=torch.float64, device=u.device)
        self._check(self.lib.qoco_gpu_cone_max_step(self._h, _tptr(u), _tptr(du), float(cap), _tptr(out),
                                                    _tptr(scratch), _torch_stream(stream)), "max_step")
        return out

    def max_step_noalloc(self, u, du, out, cap=float("inf"), stream=None):
        """Allocation-free max step: writes the step into `out` (a 1-element float64 CUDA
        tensor the caller owns) using the library's fixed device scratch; returns the C
        status code instead of raising, so callers can see TOO_LARGE."""
        return int(self.lib.qoco_gpu_cone_max_step_noalloc(self._h, _tptr(u), _tptr(du), float(cap),
                                                           _tptr(out), _torch_stream(stream)))

    def close(self):
        if self._h:
            self.lib.qoco_gpu_cones_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
