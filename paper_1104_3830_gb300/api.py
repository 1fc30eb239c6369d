"""Python face of libsa: the C entry points under the same names, taking torch CUDA
tensors for device buffers and numpy arrays for host buffers.  Marshalling only.

Weights: a 2-D int16 or int32 CUDA tensor whose rows are contiguous (stride(1) == 1);
its leading dimension is stride(0).  :func:`to_device` builds one with a 16-byte row
pitch, the layout the fused kernel reads.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from ._lib import SaError, check, lib, make_opts  # noqa: F401


class Context:
    """An sa_ctx bound to one device and CUDA stream (torch's current stream by default)."""

    def __init__(self, device: int = 0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        h = ctypes.c_void_p()
        check(lib().sa_create(ctypes.byref(h), int(device), ctypes.c_void_p(int(stream))))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            lib().sa_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sa_create(device: int = 0, stream=None) -> Context:
    return Context(device, stream)


def sa_destroy(ctx: Context) -> None:
    ctx.close()


def sa_set_batch_plan(ctx: Context, buckets=None) -> None:
    """sa_set_batch_plan from a list of (n_hi, path, warps, per_block) with path "group", "regs",
    "krows" or "block" (warps and per_block: warps per instance and groups per block);
    None restores the library's default plan."""
    if buckets is None:
        check(lib().sa_set_batch_plan(ctx.handle, None))
        return
    plan = L.sa_batch_plan()
    plan.count = len(buckets)
    for b, (n_hi, path, warps, per_block) in enumerate(buckets):
        plan.n_hi[b] = int(n_hi)
        plan.path[b] = {"group": L.SA_BATCH_GROUP, "regs": L.SA_BATCH_REGS, "krows": L.SA_BATCH_KROWS}.get(
            path, L.SA_BATCH_BLOCK)
        plan.warps[b] = int(warps)
        plan.per_block[b] = int(per_block)
    check(lib().sa_set_batch_plan(ctx.handle, ctypes.byref(plan)))


def sa_set_option(ctx: Context, name: str, value: int) -> None:
    """sa_set_option by name: wait_limit_ns, solve_gpu, step_sparse, max_grid, fused_threads,
    step_l2_bytes, test_unreachable_barrier."""
    check(lib().sa_set_option(ctx.handle, L.OPTION[name], int(value)))


def sa_last_error() -> str:
    return lib().sa_last_error().decode(errors="replace")


def sa_version() -> str:
    return lib().sa_version().decode()


def _wtype(t):
    import torch
    if t.dtype == torch.int16:
        return L.SA_I16
    if t.dtype == torch.int32:
        return L.SA_I32
    raise TypeError("weights must be int16 or int32")


def matrix(w) -> L.sa_matrix:
    """sa_matrix view of a 2-D CUDA tensor with unit column stride."""
    if not w.is_cuda or w.dim() != 2 or w.stride(1) != 1 or w.size(0) != w.size(1):
        raise ValueError("need a square 2-D CUDA tensor with contiguous rows")
    return L.sa_matrix(w.data_ptr(), _wtype(w), w.size(0), w.stride(0))


def to_device(w_host: np.ndarray, device: int = 0, align_bytes: int = 16):
    """Copy an n x n numpy int16/int32 matrix to the GPU with a padded row pitch."""
    import torch
    n = w_host.shape[0]
    esz = w_host.dtype.itemsize
    ld = -(-n * esz // align_bytes) * align_bytes // esz
    buf = torch.zeros((n, ld), dtype=torch.int16 if esz == 2 else torch.int32, device=f"cuda:{device}")
    buf[:, :n].copy_(torch.from_numpy(np.ascontiguousarray(w_host)))
    return buf[:, :n]


def sa_scale(ctx: Context, w, p, tol=1e-6, max_sweeps=20000, prec="mixed", kernel="auto", warm_keep_v=False,
             resume_from=0, u=None, v=None, allow_not_converged=True):
    """Log-domain Sinkhorn over the schedule p; returns (u, v, info) with u, v CUDA FP64."""
    import torch
    n = w.size(0)
    if u is None:
        u = torch.zeros(n, dtype=torch.float64, device=w.device)
    if v is None:
        v = torch.zeros(n, dtype=torch.float64, device=w.device)
    m = matrix(w)
    o = make_opts(p, tol, max_sweeps, prec, kernel, warm_keep_v, resume_from)
    info = L.sa_scale_info()
    st = lib().sa_scale(ctx.handle, ctypes.byref(m), ctypes.byref(o), ctypes.c_void_p(u.data_ptr()),
                        ctypes.c_void_p(v.data_ptr()), ctypes.byref(info))
    if not (allow_not_converged and st == L.SA_E_NOT_CONVERGED):
        check(st)
    d = L.info_dict(info)
    d["status"] = st
    return u, v, d


def sa_verify(ctx: Context, w, p, u, v, want_sums=False):
    """FP64 row/column sums of X(p): (max row err, max col err[, rows, cols])."""
    import torch
    m = matrix(w)
    n = w.size(0)
    rows = torch.empty(n, dtype=torch.float64, device=w.device) if want_sums else None
    cols = torch.empty(n, dtype=torch.float64, device=w.device) if want_sums else None
    er, ec = ctypes.c_double(), ctypes.c_double()
    check(lib().sa_verify(ctx.handle, ctypes.byref(m), float(p), ctypes.c_void_p(u.data_ptr()),
                          ctypes.c_void_p(v.data_ptr()), ctypes.c_void_p(rows.data_ptr() if rows is not None else 0),
                          ctypes.c_void_p(cols.data_ptr() if cols is not None else 0), ctypes.byref(er), ctypes.byref(ec)))
    if want_sums:
        return er.value, ec.value, rows, cols
    return er.value, ec.value


def _csr_to_numpy(c: L.sa_csr):
    n, nnz = c.n, c.nnz
    rp = np.ctypeslib.as_array(c.row_ptr, shape=(n + 1,)).copy()
    col = np.ctypeslib.as_array(c.col, shape=(max(nnz, 1),))[:nnz].copy()
    w = np.ctypeslib.as_array(c.w, shape=(max(nnz, 1),))[:nnz].copy()
    return rp, col, w


def sa_prune(ctx: Context, w, p, u, v, t=0.0, guard=True):
    """Reduced instance B as numpy CSR (row_ptr, col, w) and the certificate log_ub."""
    m = matrix(w)
    c = L.sa_csr()
    ub = ctypes.c_double()
    check(lib().sa_prune(ctx.handle, ctypes.byref(m), float(p), ctypes.c_void_p(u.data_ptr()),
                         ctypes.c_void_p(v.data_ptr()), float(t), int(bool(guard)), ctypes.byref(c), ctypes.byref(ub)))
    try:
        rp, col, wv = _csr_to_numpy(c)
    finally:
        lib().sa_csr_free(ctypes.byref(c))
    return rp, col, wv, ub.value


def sa_solve_reduced(row_ptr, col, w, n=None, beta0=None, near=None):
    """Exact solve of a CSR instance: (perm, sum_log_w, alpha, beta).  beta0: starting
    column duals in maximisation form, else the column minima.  near: solve from the column
    minima, then return the optimal duals with the largest beta <= near (e.g. the
    scaling's v/p)."""
    if beta0 is not None and near is not None:
        raise ValueError("give beta0 or near, not both")
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    n = len(row_ptr) - 1 if n is None else n
    c = L.sa_csr(n, len(col), row_ptr.ctypes.data_as(L._I64P), col.ctypes.data_as(L._I32P),
                 w.ctypes.data_as(L._I32P))
    perm = np.zeros(n, dtype=np.int32)
    s = ctypes.c_double()
    al = np.zeros(n)
    be = np.zeros(n)
    if near is not None:
        b0 = np.ascontiguousarray(near, dtype=np.float64)
        if b0.shape != (n,):
            raise ValueError("near must have n entries")
        check(lib().sa_solve_reduced_near(ctypes.byref(c), b0.ctypes.data_as(L._DP), perm.ctypes.data_as(L._I32P),
                                          ctypes.byref(s), al.ctypes.data_as(L._DP), be.ctypes.data_as(L._DP)))
    elif beta0 is None:
        check(lib().sa_solve_reduced(ctypes.byref(c), perm.ctypes.data_as(L._I32P), ctypes.byref(s),
                                     al.ctypes.data_as(L._DP), be.ctypes.data_as(L._DP)))
    else:
        b0 = np.ascontiguousarray(beta0, dtype=np.float64)
        if b0.shape != (n,):
            raise ValueError("beta0 must have n entries")
        check(lib().sa_solve_reduced_warm(ctypes.byref(c), b0.ctypes.data_as(L._DP), perm.ctypes.data_as(L._I32P),
                                          ctypes.byref(s), al.ctypes.data_as(L._DP), be.ctypes.data_as(L._DP)))
    return perm, s.value, al, be


def sa_solve_reduced_gpu(ctx: Context, row_ptr, col, w, price0=None, n=None):
    """Exact solve of a CSR instance with GPU-auction prices first: (perm, sum_log_w, alpha,
    beta, info)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    w = np.ascontiguousarray(w, dtype=np.int32)
    n = len(row_ptr) - 1 if n is None else n
    c = L.sa_csr(n, len(col), row_ptr.ctypes.data_as(L._I64P), col.ctypes.data_as(L._I32P),
                 w.ctypes.data_as(L._I32P))
    perm = np.zeros(n, dtype=np.int32)
    s = ctypes.c_double()
    al = np.zeros(n)
    be = np.zeros(n)
    info = L.sa_auction_info()
    p0 = None if price0 is None else np.ascontiguousarray(price0, dtype=np.float64)
    check(lib().sa_solve_reduced_gpu(ctx.handle, ctypes.byref(c), None if p0 is None else p0.ctypes.data_as(L._DP),
                                     perm.ctypes.data_as(L._I32P), ctypes.byref(s), al.ctypes.data_as(L._DP),
                                     be.ctypes.data_as(L._DP), ctypes.byref(info)))
    d = {k: getattr(info, k) for k, _ in info._fields_}
    return perm, s.value, al, be, d


def sa_certify(ctx: Context, w, alpha, beta, tau=1e-9, max_add=1 << 16):
    """(number of dual violations on A, CSR of up to max_add of them)."""
    m = matrix(w)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    nv = ctypes.c_int64()
    c = L.sa_csr()
    check(lib().sa_certify(ctx.handle, ctypes.byref(m), al.ctypes.data_as(L._DP), be.ctypes.data_as(L._DP),
                           float(tau), ctypes.byref(nv), int(max_add), ctypes.byref(c)))
    try:
        add = _csr_to_numpy(c)
    finally:
        lib().sa_csr_free(ctypes.byref(c))
    return nv.value, add


def _result_dict(r: L.sa_assign_result, perm):
    d = {k: getattr(r, k) for k, _ in L.sa_assign_result._fields_ if k not in ("perm", "scale")}
    d["scale"] = L.info_dict(r.scale)
    d["perm"] = perm
    return d


def sa_assign(ctx: Context, w, p, tol=1e-6, max_sweeps=20000, prec="mixed", kernel="auto", t=0.0):
    """Scale, prune, solve and certify: the optimal permutation of A and statistics."""
    m = matrix(w)
    n = w.size(0)
    perm = np.zeros(n, dtype=np.int32)
    r = L.sa_assign_result()
    r.perm = perm.ctypes.data_as(L._I32P)
    o = make_opts(p, tol, max_sweeps, prec, kernel)
    check(lib().sa_assign(ctx.handle, ctypes.byref(m), ctypes.byref(o), float(t), ctypes.byref(r)))
    return _result_dict(r, perm)


def sa_algorithm1(ctx: Context, w, opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=20, eps=0.0, t=0.0,
                  max_sweeps=20000, prec="mixed", kernel="auto", allow_not_converged=False):
    """The paper's preprocessing loop with adaptive p (prescaled scale); returns a dict."""
    m = matrix(w)
    n = w.size(0)
    perm = np.full(n, -1, dtype=np.int32)
    r = L.sa_alg1_result()
    r.perm = perm.ctypes.data_as(L._I32P)
    o = L.sa_alg1_opts(float(opt_ratio), float(p0), float(dp), int(max_rounds), float(eps), float(t), int(max_sweeps),
                       L.PREC[prec], L.KERNEL[kernel])
    st = lib().sa_algorithm1(ctx.handle, ctypes.byref(m), ctypes.byref(o), ctypes.byref(r))
    if not (allow_not_converged and st == L.SA_E_NOT_CONVERGED):
        check(st)
    return {"status": st, "perm": perm, "sum_log_w": r.sum_log_w, "gamma": r.gamma, "p_final": r.p_final,
            "p_raw": r.p_raw, "rounds": r.rounds, "sweeps_total": r.sweeps_total, "nnz": r.nnz}


def sa_assign_host(ctx: Context, w_host: np.ndarray, p, tol=1e-6, max_sweeps=20000, prec="mixed", kernel="auto",
                   t=0.0):
    """sa_assign on a host (numpy, ideally pinned) matrix: the copy is part of the call."""
    w_host = np.ascontiguousarray(w_host)
    n = w_host.shape[0]
    wt = L.SA_I16 if w_host.dtype == np.int16 else L.SA_I32
    perm = np.zeros(n, dtype=np.int32)
    r = L.sa_assign_result()
    r.perm = perm.ctypes.data_as(L._I32P)
    o = make_opts(p, tol, max_sweeps, prec, kernel)
    check(lib().sa_assign_host(ctx.handle, ctypes.c_void_p(w_host.ctypes.data), wt, n, w_host.strides[0] //
                               w_host.dtype.itemsize, ctypes.byref(o), float(t), ctypes.byref(r)))
    return _result_dict(r, perm)


def sa_narrow_i32_to_i16(ctx: Context, src, dst):
    n = src.size(0)
    bad = ctypes.c_int64()
    check(lib().sa_narrow_i32_to_i16(ctx.handle, ctypes.c_void_p(src.data_ptr()), src.stride(0),
                                     ctypes.c_void_p(dst.data_ptr()), dst.stride(0), n, ctypes.byref(bad)))
    return bad.value
