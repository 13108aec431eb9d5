"""GB300 direct domain-decomposition solver: Python binding of include/dd.h.

A thin ctypes layer over libdd_gb300.so: it marshals arrays into the C ABI
(dd_setup / dd_factor / dd_solve / dd_get_schur / dd_get_stats / dd_free) and
does no arithmetic of its own.  There is no CPU fallback: if the CUDA library
is missing or no GPU is visible the calls raise.

    from paper_2002_05019_gb300 import Solver
    s = Solver.from_problem(problem, precision="mixed")
    s.factor()
    u, lam = s.solve(f)          # f: (sum n_i, nrhs) complex128, host or CUDA tensor
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libdd_gb300.so")
_lib = None

DD_OK = 0
STATUS = {0: "DD_OK", 1: "DD_ERR_INVALID_ARG", 2: "DD_ERR_NOT_SYMMETRIC", 3: "DD_ERR_SINGULAR_PIVOT",
          4: "DD_ERR_OOM", 5: "DD_ERR_CUDA", 6: "DD_ERR_NOT_FACTORED", 7: "DD_ERR_NOT_CONVERGED",
          8: "DD_ERR_TIMEOUT", 9: "DD_ERR_NO_DEVICE"}
PRECISION = {"fp64": 0, "mixed": 1}


class DDError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.dd_strerror(code).decode() if _lib is not None else STATUS.get(code, "?")
        super().__init__(f"{where}: {STATUS.get(code, code)} ({msg})")


class c128(C.Structure):
    _fields_ = [("re", C.c_double), ("im", C.c_double)]


class Subdomain(C.Structure):
    _fields_ = [("n", C.c_int32), ("rowptr", C.POINTER(C.c_int32)), ("colind", C.POINTER(C.c_int32)),
                ("val", C.c_void_p), ("nb", C.c_int32), ("b_dual", C.POINTER(C.c_int32)),
                ("b_local", C.POINTER(C.c_int32)), ("b_sign", C.POINTER(C.c_int8))]


class Options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("refine_tol", C.c_double), ("max_refine", C.c_int32),
                ("pivoting", C.c_int32), ("tree_parent", C.POINTER(C.c_int32)),
                ("centroids", C.POINTER(C.c_double)), ("cuda_stream", C.c_void_p), ("device", C.c_int32),
                ("time_kernels", C.c_int32), ("simt_update", C.c_int32), ("update_panels", C.c_int32),
                ("sparse_min", C.c_int32), ("sparse_leaf", C.c_int32), ("tune_cache", C.c_char_p)]

KERNEL_CLASSES = ["diag", "trsm", "update", "assemble", "init"]


class Stats(C.Structure):
    _fields_ = [("n_sub", C.c_int32), ("n_dual", C.c_int32), ("n_fronts", C.c_int32), ("n_levels", C.c_int32),
                ("n_primal", C.c_int64), ("max_front", C.c_int32), ("flops_factor", C.c_double),
                ("flops_solve", C.c_double), ("bytes_factor", C.c_int64), ("bytes_device", C.c_int64),
                ("t_setup_ms", C.c_double), ("t_factor_ms", C.c_double), ("t_solve_ms", C.c_double),
                ("growth", C.c_double), ("min_pivot", C.c_double), ("refine_iters", C.c_int32),
                ("refine_last", C.c_double), ("launches_factor", C.c_int32), ("launches_solve", C.c_int32),
                ("kernel_ms", C.c_double * 5), ("kernel_launches", C.c_int32 * 5), ("kernel_flops", C.c_double * 5),
                ("interchanges", C.c_int64), ("pivots_2x2", C.c_int64)]


class Schedule(C.Structure):
    _fields_ = [("update_panels", C.c_int32), ("ahead_fronts", C.c_int32), ("reserve_sms", C.c_int32),
                ("factor_ms", C.c_double), ("configs_tried", C.c_int32), ("split_sms", C.c_int32)]


EXPORTS = ["dd_default_options", "dd_setup", "dd_set_values", "dd_factor", "dd_solve", "dd_solve_subset", "dd_get_schur",
           "dd_set_schedule", "dd_autotune",
           "dd_get_stats", "dd_strerror", "dd_free", "dd_dense_solve_noalloc", "dd_selftest_wait_timeout",
           "dd_symbolic", "dd_domain_symbolic", "dd_domain_assembly", "dd_shard_plan", "dd_selftest_pivot_tile",
           "dd_tune_key", "dd_tune_cache_lookup", "dd_tune_cache_store"]


def library_path() -> str:
    return _LIB_PATH


def load(build_if_missing: bool = True):
    """Load libdd_gb300.so (building it with nvcc first if it is absent or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        from .build import build
        build()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"{_LIB_PATH} is missing: build it with paper_2002_05019_gb300.build.build()")
    lib = C.CDLL(_LIB_PATH)
    lib.dd_default_options.argtypes = [C.POINTER(Options)]
    lib.dd_setup.argtypes = [C.POINTER(C.c_void_p), C.c_int32, C.POINTER(Subdomain), C.c_int32, C.POINTER(Options)]
    lib.dd_set_values.argtypes = [C.c_void_p, C.c_void_p]
    lib.dd_factor.argtypes = [C.c_void_p]
    lib.dd_solve.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_void_p, C.c_int64, C.c_void_p,
                             C.c_int64]
    lib.dd_solve_subset.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_int32),
                                    C.c_void_p, C.c_int64, C.c_void_p, C.c_int64]
    lib.dd_get_schur.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.dd_get_stats.argtypes = [C.c_void_p, C.POINTER(Stats)]
    lib.dd_set_schedule.argtypes = [C.c_void_p, C.POINTER(Schedule)]
    lib.dd_autotune.argtypes = [C.c_void_p, C.c_int32, C.POINTER(Schedule)]
    lib.dd_strerror.argtypes = [C.c_int]
    lib.dd_strerror.restype = C.c_char_p
    lib.dd_free.argtypes = [C.c_void_p]
    lib.dd_free.restype = None
    lib.dd_selftest_wait_timeout.argtypes = [C.c_void_p]
    lib.dd_selftest_pivot_tile.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dd_domain_symbolic.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.dd_domain_assembly.argtypes = [C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.dd_symbolic.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]
    lib.dd_shard_plan.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p,
                                  C.c_void_p, C.c_void_p]
    lib.dd_tune_key.argtypes = [C.c_int32, C.c_void_p, C.c_int32, C.c_void_p, C.POINTER(C.c_uint64)]
    lib.dd_tune_cache_lookup.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(Schedule), C.POINTER(C.c_int32)]
    lib.dd_tune_cache_store.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(Schedule)]
    lib.dd_dense_solve_noalloc.argtypes = [C.c_int32, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, C.c_int64,
                                           C.c_void_p, C.c_int64, C.c_void_p]
    _lib = lib
    return lib


def _ptr(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _check(code: int, where: str, ok=(DD_OK,)):
    if code not in ok:
        raise DDError(code, where)
    return code


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _marshal(subdomains, tree_parent=None, centroids=None):
    """dd_subdomain array and default dd_options for a list of domain dicts;
    returns (subs, opt, keep), keep holding the arrays the pointers refer to."""
    lib = load()
    keep = []
    subs = (Subdomain * len(subdomains))()
    for k, s in enumerate(subdomains):
        rp = np.ascontiguousarray(s["indptr"], dtype=np.int32)
        ci = np.ascontiguousarray(s["indices"], dtype=np.int32)
        va = np.ascontiguousarray(s["data"], dtype=np.complex128)
        bd = np.ascontiguousarray(s["b_dual"], dtype=np.int32)
        bl = np.ascontiguousarray(s["b_local"], dtype=np.int32)
        bs = np.ascontiguousarray(s["b_sign"], dtype=np.int8)
        keep += [rp, ci, va, bd, bl, bs]
        subs[k] = Subdomain(int(s["n"]), _ptr(rp, C.c_int32), _ptr(ci, C.c_int32), va.ctypes.data, bd.size,
                            _ptr(bd, C.c_int32), _ptr(bl, C.c_int32), _ptr(bs, C.c_int8))
    opt = Options()
    lib.dd_default_options(C.byref(opt))
    if tree_parent is not None:
        tp = np.ascontiguousarray(tree_parent, dtype=np.int32)
        keep.append(tp)
        opt.tree_parent = _ptr(tp, C.c_int32)
    if centroids is not None:
        ce = np.ascontiguousarray(centroids, dtype=np.float64).ravel()
        keep.append(ce)
        opt.centroids = _ptr(ce, C.c_double)
    return subs, opt, keep


def _problem_subs(p):
    return [dict(n=s.n, indptr=s.indptr, indices=s.indices, data=s.data, b_dual=s.b_dual,
                 b_local=s.b_local, b_sign=s.b_sign) for s in p.subs]


def symbolic(subdomains, n_dual: int, tree_parent=None, centroids=None) -> dict:
    """The front tree of the library's symbolic analysis (dd_symbolic; host only,
    no GPU): parent, ne, nu per front (domains first, then separator fronts in
    post-order), the front of every dual, and each front's update-row duals."""
    lib = load()
    subs, opt, keep = _marshal(subdomains, tree_parent, centroids)
    n_sub = len(subdomains)
    cap = 2 * n_sub + 1
    nf = C.c_int32(0)
    parent, ne, nu = (np.zeros(cap, np.int32) for _ in range(3))
    dual_front = np.zeros(max(n_dual, 1), np.int32)
    upd_ptr = np.zeros(cap + 1, np.int64)
    st = lib.dd_symbolic(n_sub, subs, int(n_dual), C.byref(opt), cap, C.byref(nf), parent.ctypes.data,
                         ne.ctypes.data, nu.ctypes.data, dual_front.ctypes.data, 0, upd_ptr.ctypes.data, None)
    _check(st, "dd_symbolic")
    n = nf.value
    upd_idx = np.zeros(max(int(upd_ptr[n]), 1), np.int32)
    st = lib.dd_symbolic(n_sub, subs, int(n_dual), C.byref(opt), cap, C.byref(nf), parent.ctypes.data,
                         ne.ctypes.data, nu.ctypes.data, dual_front.ctypes.data, upd_idx.size, upd_ptr.ctypes.data,
                         upd_idx.ctypes.data)
    _check(st, "dd_symbolic")
    del keep
    return {"n_front": n, "parent": parent[:n].copy(), "ne": ne[:n].copy(), "nu": nu[:n].copy(),
            "dual_front": dual_front[:n_dual].copy(),
            "upd": [upd_idx[upd_ptr[x]:upd_ptr[x + 1]].copy() for x in range(n)]}


def domain_symbolic(indptr, indices, is_last=None, leaf_max: int = 256) -> dict:
    """Nested-dissection front tree of one domain matrix (dd_domain_symbolic;
    host only): rows flagged in is_last are eliminated last, in the root."""
    lib = load()
    rp = np.ascontiguousarray(indptr, dtype=np.int32)
    ci = np.ascontiguousarray(indices, dtype=np.int32)
    n = rp.size - 1
    il = None if is_last is None else np.ascontiguousarray(is_last, dtype=np.int8)
    cap = max(2 * n + 1, 1)
    nf = C.c_int32(0)
    stored = C.c_int64(0)
    parent, ne, nu = (np.zeros(cap, np.int32) for _ in range(3))
    order, front_of = np.zeros(max(n, 1), np.int32), np.zeros(max(n, 1), np.int32)
    upd_ptr = np.zeros(cap + 1, np.int64)
    args = (n, rp.ctypes.data, ci.ctypes.data, None if il is None else il.ctypes.data, int(leaf_max), cap,
            C.byref(nf), parent.ctypes.data, ne.ctypes.data, nu.ctypes.data, order.ctypes.data,
            front_of.ctypes.data, C.byref(stored))
    _check(lib.dd_domain_symbolic(*args, 0, upd_ptr.ctypes.data, None), "dd_domain_symbolic")
    k = nf.value
    upd_idx = np.zeros(max(int(upd_ptr[k]), 1), np.int32)
    _check(lib.dd_domain_symbolic(*args, upd_idx.size, upd_ptr.ctypes.data, upd_idx.ctypes.data), "dd_domain_symbolic")
    return {"n_front": k, "parent": parent[:k].copy(), "ne": ne[:k].copy(), "nu": nu[:k].copy(),
            "order": order[:n].copy(), "front_of": front_of[:n].copy(), "stored": stored.value,
            "upd": [upd_idx[upd_ptr[x]:upd_ptr[x + 1]].copy() for x in range(k)]}


def domain_assembly(indptr, indices, is_last=None, leaf_max: int = 256) -> dict:
    """Assembly maps of the domain's front tree (dd_domain_assembly; host only):
    every front's rows, the extend-add map of its update rows into its parent,
    and the front position of every CSR entry of A_i."""
    lib = load()
    rp = np.ascontiguousarray(indptr, dtype=np.int32)
    ci = np.ascontiguousarray(indices, dtype=np.int32)
    n = rp.size - 1
    il = None if is_last is None else np.ascontiguousarray(is_last, dtype=np.int8)
    cap = max(2 * n + 1, 1)
    nf = C.c_int32(0)
    parent, ne = np.zeros(cap, np.int32), np.zeros(cap, np.int32)
    rows_ptr = np.zeros(cap + 1, np.int64)
    head = (n, rp.ctypes.data, ci.ctypes.data, None if il is None else il.ctypes.data, int(leaf_max), cap,
            C.byref(nf), parent.ctypes.data, ne.ctypes.data)
    _check(lib.dd_domain_assembly(*head, 0, rows_ptr.ctypes.data, None, None, None, None, None), "dd_domain_assembly")
    k = nf.value
    m = int(rows_ptr[k])
    rows, ea = np.zeros(max(m, 1), np.int32), np.zeros(max(m, 1), np.int32)
    nnz = int(rp[-1]) if n else 0
    af, ar, ac = (np.zeros(max(nnz, 1), np.int32) for _ in range(3))
    _check(lib.dd_domain_assembly(*head, rows.size, rows_ptr.ctypes.data, rows.ctypes.data, ea.ctypes.data,
                                  af.ctypes.data, ar.ctypes.data, ac.ctypes.data), "dd_domain_assembly")
    return {"n_front": k, "parent": parent[:k].copy(), "ne": ne[:k].copy(), "rows_ptr": rows_ptr[:k + 1].copy(),
            "rows": rows[:m].copy(), "ea_map": ea[:m].copy(), "a_front": af[:nnz].copy(), "a_row": ar[:nnz].copy(),
            "a_col": ac[:nnz].copy()}


def pivot_tile(tile, precision: str = "dfloat"):
    """One 64 x 64 complex diagonal tile through the mixed form's diagonal
    kernel (dd_selftest_pivot_tile; needs a GPU): pivot blocks in "fp32",
    "dfloat" (double-float) or "fp64".  Returns (factor, L^-1) as complex64
    arrays: D on the factor's diagonal, L strictly below."""
    lib = load()
    a = np.ascontiguousarray(tile, dtype=np.complex64)
    if a.shape != (64, 64):
        raise ValueError("a 64 x 64 tile")
    out = a.copy()
    linv = np.zeros_like(a)
    code = {"fp32": 0, "dfloat": 1, "fp64": 2}[precision]
    _check(lib.dd_selftest_pivot_tile(a.ctypes.data, code, out.ctypes.data, linv.ctypes.data, None),
           "dd_selftest_pivot_tile")
    return out, linv


def tune_key(subdomains, n_dual: int, precision: str = "mixed", pivoting: int = 0, tree_parent=None,
             centroids=None) -> int:
    """The autotuner cache's problem key of a decomposition (dd_tune_key; host only)."""
    lib = load()
    subs, opt, keep = _marshal(subdomains, tree_parent, centroids)
    opt.precision = PRECISION[precision]
    opt.pivoting = int(pivoting)
    key = C.c_uint64(0)
    _check(lib.dd_tune_key(len(subdomains), subs, int(n_dual), C.byref(opt), C.byref(key)), "dd_tune_key")
    del keep
    return key.value


def tune_key_problem(p, precision: str = "mixed", pivoting: int = 0) -> int:
    """tune_key() for a femgen.Problem, with its domain tree."""
    return tune_key(_problem_subs(p), p.n_dual, precision, pivoting, tree_parent=p.rcb.parent)


def tune_cache_lookup(path: str, key: str):
    """The schedule cached under `key` in the cache file (dd_tune_cache_lookup), or None."""
    lib = load()
    sc = Schedule()
    found = C.c_int32(0)
    _check(lib.dd_tune_cache_lookup(os.fsencode(path), key.encode(), C.byref(sc), C.byref(found)),
           "dd_tune_cache_lookup")
    return {k: getattr(sc, k) for k, _ in Schedule._fields_} if found.value else None


def tune_cache_store(path: str, key: str, schedule: dict):
    """Append one schedule line under `key` (dd_tune_cache_store)."""
    lib = load()
    sc = Schedule(int(schedule["update_panels"]), int(schedule["ahead_fronts"]), int(schedule["reserve_sms"]),
                  float(schedule.get("factor_ms", 0.0)), 0, int(schedule.get("split_sms", 0)))
    _check(lib.dd_tune_cache_store(os.fsencode(path), key.encode(), C.byref(sc)), "dd_tune_cache_store")


def shard_plan(subdomains, n_dual: int, n_ranks: int, tree_parent=None, centroids=None) -> dict:
    """Cut of the front tree into n_ranks subtrees (dd_shard_plan; host only):
    the owner rank of every front and the root front of every rank's subtree."""
    lib = load()
    subs, opt, keep = _marshal(subdomains, tree_parent, centroids)
    cap = 2 * len(subdomains) + 1
    nf = C.c_int32(0)
    front_rank = np.zeros(cap, np.int32)
    rank_root = np.zeros(max(int(n_ranks), 1), np.int32)
    _check(lib.dd_shard_plan(len(subdomains), subs, int(n_dual), C.byref(opt), int(n_ranks), cap, C.byref(nf),
                             front_rank.ctypes.data, rank_root.ctypes.data), "dd_shard_plan")
    del keep
    return {"n_front": nf.value, "front_rank": front_rank[:nf.value].copy(), "rank_root": rank_root.copy()}


def symbolic_problem(p) -> dict:
    """symbolic() for a femgen.Problem, with its domain tree."""
    return symbolic(_problem_subs(p), p.n_dual, tree_parent=p.rcb.parent)


def shard_plan_problem(p, n_ranks: int) -> dict:
    """shard_plan() for a femgen.Problem, with its domain tree."""
    return shard_plan(_problem_subs(p), p.n_dual, n_ranks, tree_parent=p.rcb.parent)


class Solver:
    """One factorization of an arrowhead system on one GPU."""

    def __init__(self, subdomains, n_dual: int, precision: str = "fp64", refine_tol: float = 1e-13,
                 max_refine: int | None = None, tree_parent=None, centroids=None, stream=None, device: int = 0,
                 time_kernels: bool | int = False, simt_update: bool = False, pivoting: int | None = None,
                 update_panels: int | None = None, sparse_min: int | None = None, sparse_leaf: int | None = None,
                 tune_cache: str | None = None):
        lib = load()
        subs, opt, self._keep = _marshal(subdomains, tree_parent, centroids)
        self.n = [int(s["n"]) for s in subdomains]
        self.n_loc = int(sum(self.n))
        self.n_dual = int(n_dual)
        self.nnz = [int(np.size(s["indices"])) for s in subdomains]
        opt.precision = PRECISION[precision]
        opt.refine_tol = refine_tol
        if max_refine is not None:
            opt.max_refine = int(max_refine)
        if stream is not None:
            opt.cuda_stream = C.c_void_p(int(stream))
        opt.device = device
        # True / 1: every launch; 2: the trailing-update launches only
        opt.time_kernels = 2 if (not isinstance(time_kernels, bool) and time_kernels == 2) else (1 if time_kernels else 0)
        opt.simt_update = 1 if simt_update else 0
        if update_panels is not None:
            opt.update_panels = int(update_panels)   # tensor-core update: 1 or 2 panels per pass
        if pivoting is not None:
            opt.pivoting = int(pivoting)   # 0 none, 1 auxiliary fronts, 2 every front (restricted Bunch-Kaufman)
        if sparse_min is not None:
            opt.sparse_min = int(sparse_min)   # domains of >= sparse_min unknowns: nested-dissection front trees
        if sparse_leaf is not None:
            opt.sparse_leaf = int(sparse_leaf)
        if tune_cache is not None:
            opt.tune_cache = os.fsencode(tune_cache)   # schedule cache file (copied by dd_setup)
        self.precision = precision
        h = C.c_void_p()
        _check(lib.dd_setup(C.byref(h), len(subdomains), subs, self.n_dual, C.byref(opt)), "dd_setup")
        self._h = h
        self._keep = []   # dd_setup deep-copied every input

    @classmethod
    def from_problem(cls, p, **kw):
        """Build from a femgen.Problem (domain CSRs, B entries and the domain tree)."""
        kw.setdefault("tree_parent", p.rcb.parent)
        return cls(_problem_subs(p), p.n_dual, **kw)

    def set_values(self, vals):
        """New values for every A_i (same patterns), domain after domain: host array or CUDA tensor."""
        if _is_torch(vals):
            _check(_lib.dd_set_values(self._h, C.c_void_p(vals.data_ptr())), "dd_set_values")
        else:
            v = np.ascontiguousarray(vals, dtype=np.complex128)
            _check(_lib.dd_set_values(self._h, C.c_void_p(v.ctypes.data)), "dd_set_values")

    def factor(self):
        _check(_lib.dd_factor(self._h), "dd_factor")

    def solve(self, f, allow_not_converged: bool = False):
        """Solve for the stacked local loads f (n_loc x nrhs, column-major).

        numpy in -> numpy out; a CUDA torch tensor in -> CUDA tensors out.
        Returns (u, lambda).
        """
        ok = (DD_OK, 7) if allow_not_converged else (DD_OK,)
        if _is_torch(f):
            import torch
            ff = f if f.dim() == 2 else f[:, None]
            nrhs = ff.shape[1]
            ft = ff.t().contiguous()                  # (nrhs, n_loc): column-major f
            ut = torch.empty((nrhs, self.n_loc), dtype=torch.complex128, device=f.device)
            lt = torch.empty((nrhs, max(self.n_dual, 1)), dtype=torch.complex128, device=f.device)
            code = _lib.dd_solve(self._h, nrhs, C.c_void_p(ft.data_ptr()), self.n_loc, C.c_void_p(ut.data_ptr()),
                                 self.n_loc, C.c_void_p(lt.data_ptr()) if self.n_dual else None,
                                 max(self.n_dual, 1))
            _check(code, "dd_solve", ok)
            self.last_status = code
            uo, lo = ut.t(), lt[:, :self.n_dual].t()
            return (uo[:, 0], lo[:, 0]) if f.dim() == 1 else (uo, lo)
        fa = np.asarray(f, dtype=np.complex128)
        vec = fa.ndim == 1
        fa = np.asfortranarray(fa[:, None] if vec else fa)
        nrhs = fa.shape[1]
        uo = np.zeros((self.n_loc, nrhs), dtype=np.complex128, order="F")
        lo = np.zeros((self.n_dual, nrhs), dtype=np.complex128, order="F")
        code = _lib.dd_solve(self._h, nrhs, C.c_void_p(fa.ctypes.data), self.n_loc, C.c_void_p(uo.ctypes.data),
                             self.n_loc, C.c_void_p(lo.ctypes.data) if self.n_dual else None, max(self.n_dual, 1))
        _check(code, "dd_solve", ok)
        self.last_status = code
        return (uo[:, 0], lo[:, 0]) if vec else (uo, lo)

    def autotune(self, repeats: int = 2) -> dict:
        """Time dd_factor under each schedule of the tensor-core path, keep the fastest
        (the handle is left factored with it); returns the chosen schedule."""
        sc = Schedule()
        _check(_lib.dd_autotune(self._h, int(repeats), C.byref(sc)), "dd_autotune")
        return {k: getattr(sc, k) for k, _ in Schedule._fields_}

    def set_schedule(self, update_panels: int, ahead_fronts: int, reserve_sms: int, split_sms: int = 0):
        sc = Schedule(int(update_panels), int(ahead_fronts), int(reserve_sms), 0.0, 0, int(split_sms))
        _check(_lib.dd_set_schedule(self._h, C.byref(sc)), "dd_set_schedule")

    def solve_subset(self, f, domains, allow_not_converged: bool = False):
        """Solve for the stacked local loads f (numpy, n_loc x nrhs) and recover only
        the listed domains: returns (u of those domains stacked in the given order, lambda)."""
        ok = (DD_OK, 7) if allow_not_converged else (DD_OK,)
        req = np.ascontiguousarray(domains, dtype=np.int32)
        fa = np.asarray(f, dtype=np.complex128)
        vec = fa.ndim == 1
        fa = np.asfortranarray(fa[:, None] if vec else fa)
        nrhs = fa.shape[1]
        rows = int(sum(self.n[int(i)] for i in req)) if all(0 <= int(i) < len(self.n) for i in req) else 1
        uo = np.zeros((max(rows, 1), nrhs), dtype=np.complex128, order="F")
        lo = np.zeros((self.n_dual, nrhs), dtype=np.complex128, order="F")
        code = _lib.dd_solve_subset(self._h, nrhs, C.c_void_p(fa.ctypes.data), self.n_loc, req.size,
                                    _ptr(req, C.c_int32), C.c_void_p(uo.ctypes.data), max(rows, 1),
                                    C.c_void_p(lo.ctypes.data) if self.n_dual else None, max(self.n_dual, 1))
        _check(code, "dd_solve_subset", ok)
        uo = uo[:rows]
        return (uo[:, 0], lo[:, 0]) if vec else (uo, lo)

    def schur(self, i: int):
        """F_i = B_i A_i^{-1} B_i^T of domain i (m_i x m_i) and its ascending dual ids."""
        m = C.c_int32()
        _check(_lib.dd_get_schur(self._h, i, None, None, C.byref(m)), "dd_get_schur")
        out = np.zeros((m.value, m.value), dtype=np.complex128, order="F")
        duals = np.zeros(m.value, dtype=np.int32)
        _check(_lib.dd_get_schur(self._h, i, C.c_void_p(out.ctypes.data), _ptr(duals, C.c_int32), C.byref(m)),
               "dd_get_schur")
        return out, duals

    def stats(self) -> dict:
        st = Stats()
        _check(_lib.dd_get_stats(self._h, C.byref(st)), "dd_get_stats")
        out = {}
        for name, _ in Stats._fields_:
            v = getattr(st, name)
            out[name] = dict(zip(KERNEL_CLASSES, list(v))) if name.startswith("kernel_") else v
        return out

    def free(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.dd_free(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def stacked_loads(problem) -> np.ndarray:
    """The local loads f_i of a femgen.Problem stacked domain after domain: (n_loc, nrhs)."""
    return np.concatenate([s.f for s in problem.subs], axis=0)


def unstack(problem, u: np.ndarray):
    """Split a stacked (n_loc, nrhs) array back into per-domain blocks."""
    offs = np.cumsum([0] + [s.n for s in problem.subs])
    return [u[offs[k]:offs[k + 1]] for k in range(problem.n_sub)]


__all__ = ["Solver", "DDError", "load", "library_path", "stacked_loads", "unstack", "symbolic", "symbolic_problem",
           "domain_symbolic", "domain_assembly", "shard_plan", "shard_plan_problem", "pivot_tile",
           "tune_key", "tune_key_problem", "tune_cache_lookup", "tune_cache_store",
           "EXPORTS", "PRECISION"]
