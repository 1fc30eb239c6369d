"""FP64 CPU oracle for the Sinkhorn preprocessing of the optimal assignment problem.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The product library never links
or calls it, and it shares no code with the CUDA path: the C core ``orc.c`` is compiled
on its own by :func:`build` and reached through ctypes.

Every function follows a passage of Sharify, Gaubert and Grigori, arXiv:1104.3830:

* :func:`log_weights`     b = log a (Eq. pentropyopt), b = -inf where a = 0
* :func:`sinkhorn`        log-domain p-Sinkhorn (Sec. 4.1.2) per p of a schedule,
                          stopped at an eps-bistochastic matrix (Sec. 4.2)
* :func:`xmatrix`, :func:`sums`   X(p) = D_r A^(p) D_c from the potentials
* :func:`prune_mask`, :func:`prune_csr`   reduced matrix B (Eq. matrixred)
* :func:`log_ub`          approximate optimality certificate (Prop. aoc)
* :func:`gamma`           ratio gamma (Eq. optratio)
* :func:`prescale`        prescaling into [1, e] (Sec. 4.1.1)
* :func:`hungarian`, :func:`lapjv`, :func:`bruteforce`   exact optimal assignment
                          (the LP of Sec. 2.2), two independent O(n^3) solvers and
                          exhaustive search for n <= 10
* :func:`dual_violations` LP-duality optimality check for (alpha, beta)
* :func:`preprocess`      Algorithm 1 with a fixed p schedule: scale, prune, solve B
* :func:`algorithm1`      Algorithm 1 with the adaptive p of Sec. 5 (gamma <= opt_ratio)
* :func:`newton`          the Newton scaling of Sec. 5.3 (Knight-Ruiz iteration on the
                          symmetric embedding of A^(p)), dense FP64 solves

Parity pins live in ``tests/test_oracle_*.py``.  Nothing is "parity unpinned" except
the paper's Tables 1-3 (their test matrices are not available here) and the printed
digits of the 5x5 X(50) (p = 50 amplifies the rounding of the printed 3-decimal A beyond
the printed digits).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "orc.c")
_LIB_PATH = os.path.join(_HERE, "liborc.so")
_lib = None
_lock = threading.Lock()

OK, NOT_CONVERGED, E_INVALID, E_NO_SUPPORT, E_INFEASIBLE = 0, 1, -1, -2, -3


def build(force: bool = False) -> str:
    """Compile orc.c into liborc.so next to it (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
           _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        i, d = ctypes.c_int, ctypes.c_double
        sig = {
            "orc_num_threads": (i, []),
            "orc_set_num_threads": (None, [i]),
            "orc_sinkhorn": (i, [i, dp, dp, i, d, i, i, dp, dp, ip, dp]),
            "orc_sinkhorn_from": (i, [i, dp, d, d, i, dp, dp, ip, dp]),
            "orc_xmatrix": (i, [i, dp, d, dp, dp, dp]),
            "orc_sums": (i, [i, dp, d, dp, dp, dp, dp]),
            "orc_prune_mask": (i, [i, dp, d, dp, dp, d, i, u8p]),
            "orc_log_ub": (d, [i, dp, d, dp]),
            "orc_prescale": (d, [i, dp, dp, dp]),
            "orc_hungarian": (i, [i, dp, ip, dp, dp]),
            "orc_lapjv": (i, [i, dp, ip]),
            "orc_bruteforce": (i, [i, dp, ip, dp]),
            "orc_dual_violations": (ctypes.c_int64, [i, dp, dp, dp, d, dp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype, f.argtypes = res, args
        _lib = lib
        return lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def _square(b):
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.ndim != 2 or b.shape[0] != b.shape[1]:
        raise ValueError("expected a square matrix")
    return b


def num_threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(_load().orc_num_threads())


def set_num_threads(k: int) -> None:
    """Threads of the oracle's later parallel loops (timing only: each loop splits
    independent rows or columns, so the results do not depend on it)."""
    _load().orc_set_num_threads(int(k))


def log_weights(a) -> np.ndarray:
    """b_ij = log a_ij in FP64, -inf where a_ij = 0 (Eq. pentropyopt; 0*(-inf) = 0)."""
    a = np.asarray(a)
    if np.any(a < 0):
        raise ValueError("weights must be non-negative")
    with np.errstate(divide="ignore"):
        return np.log(a.astype(np.float64))


def sinkhorn(b, p_sched, tol=1e-6, max_sweeps=20000, warm_keep_v=False):
    """Log-domain Sinkhorn at each p of an increasing schedule (Sec. 4.1.2, Sec. 4.2).

    Returns (u, v, sweeps_per_p, resid_per_p, status) with x_ij = exp(p b_ij - u_i - v_j)
    at the last p.  status: 0 converged, 1 some step hit max_sweeps, < 0 invalid input.
    """
    b = _square(b)
    n = b.shape[0]
    p = np.ascontiguousarray(np.atleast_1d(p_sched), dtype=np.float64)
    u = np.zeros(n)
    v = np.zeros(n)
    sw = np.zeros(len(p), dtype=np.int32)
    rs = np.zeros(len(p))
    st = _load().orc_sinkhorn(n, _dp(b), _dp(p), len(p), float(tol), int(max_sweeps),
                              int(bool(warm_keep_v)), _dp(u), _dp(v), _ip(sw), _dp(rs))
    return u, v, sw, rs, int(st)


def sinkhorn_from(b, p, u, v, tol=1e-6, max_sweeps=20000):
    """Continue the iteration at one p from the given potentials (copies are returned)."""
    b = _square(b)
    n = b.shape[0]
    u = np.array(u, dtype=np.float64, copy=True)
    v = np.array(v, dtype=np.float64, copy=True)
    sw = np.zeros(1, dtype=np.int32)
    rs = np.zeros(1)
    st = _load().orc_sinkhorn_from(n, _dp(b), float(p), float(tol), int(max_sweeps),
                                   _dp(u), _dp(v), _ip(sw), _dp(rs))
    return u, v, int(sw[0]), float(rs[0]), int(st)


def xmatrix(b, p, u, v) -> np.ndarray:
    """X(p) with x_ij = exp(p b_ij - u_i - v_j) (Thm. prop-borweinlewisnussbaum)."""
    b = _square(b)
    n = b.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    x = np.empty((n, n))
    _load().orc_xmatrix(n, _dp(b), float(p), _dp(u), _dp(v), _dp(x))
    return x


def sums(b, p, u, v):
    """(row sums, column sums) of X(p) in FP64."""
    b = _square(b)
    n = b.shape[0]
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    r = np.empty(n)
    c = np.empty(n)
    _load().orc_sums(n, _dp(b), float(p), _dp(u), _dp(v), _dp(r), _dp(c))
    return r, c


def prune_mask(b, p, u, v, t=None, guard=True) -> np.ndarray:
    """Boolean mask of B (Eq. matrixred): keep x_ij(p) >= t, t = 1/n by default (Sec. 4.2).

    guard keeps every row's and column's largest entry as well (our reading for empty
    rows or columns, which the paper leaves open)."""
    b = _square(b)
    n = b.shape[0]
    if t is None:
        t = 1.0 / n
    log_t = np.log(t) if t > 0 else -np.inf
    u = np.ascontiguousarray(u, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    m = np.zeros((n, n), dtype=np.uint8)
    _load().orc_prune_mask(n, _dp(b), float(p), _dp(u), _dp(v), float(log_t), int(bool(guard)),
                           m.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)))
    return m.astype(bool)


def prune_csr(mask: np.ndarray):
    """CSR (row_ptr int64, col int32) of a boolean mask, columns ascending per row."""
    rows, cols = np.nonzero(mask)
    counts = np.bincount(rows, minlength=mask.shape[0])
    row_ptr = np.zeros(mask.shape[0] + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return row_ptr, cols.astype(np.int32)


def log_ub(b, p, v) -> float:
    """Right side of Eq. e-certificate: an upper bound on log w_opt(A) for any v."""
    b = _square(b)
    v = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().orc_log_ub(b.shape[0], _dp(b), float(p), _dp(v)))


def gamma(log_ub_value: float, log_w_opt_b: float) -> float:
    """gamma = exp(certificate) / w_opt(B) (Eq. optratio), in log form."""
    return float(np.exp(log_ub_value - log_w_opt_b))


def prescale(a):
    """Prescaling of Sec. 4.1.1; returns (scaled matrix, m, c)."""
    a = _square(a)
    out = np.empty_like(a)
    c = np.zeros(1)
    m = _load().orc_prescale(a.shape[0], _dp(a), _dp(out), _dp(c))
    return out, float(m), float(c[0])


def hungarian(b):
    """Exact max sum_i b_{i,sigma(i)} by the O(n^3) Hungarian method.

    Returns (perm, alpha, beta, status); alpha_i + beta_j >= b_ij with equality on the
    assignment.  status E_INFEASIBLE if the allowed entries hold no permutation."""
    b = _square(b)
    n = b.shape[0]
    perm = np.full(n, -1, dtype=np.int32)
    al = np.zeros(n)
    be = np.zeros(n)
    st = _load().orc_hungarian(n, _dp(b), _ip(perm), _dp(al), _dp(be))
    return perm, al, be, int(st)


def lapjv(b):
    """Exact max sum_i b_{i,sigma(i)} by dense Jonker-Volgenant (all entries allowed)."""
    b = _square(b)
    n = b.shape[0]
    perm = np.full(n, -1, dtype=np.int32)
    st = _load().orc_lapjv(n, _dp(b), _ip(perm))
    return perm, int(st)


def bruteforce(b):
    """Exhaustive optimum over all n! permutations, n <= 10: (perm, best, status)."""
    b = _square(b)
    n = b.shape[0]
    perm = np.full(n, -1, dtype=np.int32)
    best = np.zeros(1)
    st = _load().orc_bruteforce(n, _dp(b), _ip(perm), _dp(best))
    return perm, float(best[0]), int(st)


def dual_violations(b, alpha, beta, tau=1e-9):
    """(count, max gap) of allowed entries with alpha_i + beta_j < b_ij - tau."""
    b = _square(b)
    al = np.ascontiguousarray(alpha, dtype=np.float64)
    be = np.ascontiguousarray(beta, dtype=np.float64)
    gap = np.zeros(1)
    c = _load().orc_dual_violations(b.shape[0], _dp(b), _dp(al), _dp(be), float(tau), _dp(gap))
    return int(c), float(gap[0])


def perm_weight_exact(w, perm) -> int:
    """prod_i w_{i, perm(i)} as an exact Python integer (integer weights only)."""
    w = np.asarray(w)
    out = 1
    for i, j in enumerate(perm):
        out *= int(w[i, int(j)])
    return out


def preprocess(w, p_sched, tol=1e-6, max_sweeps=20000, t=None, guard=True):
    """Algorithm 1 with the fixed schedule p_sched: Sinkhorn at each p, prune at t (1/n),
    solve B exactly, and report the certificate and gamma (Eq. optratio).

    Returns a dict with u, v, sweeps, mask, perm (optimal on B), log_w_B, log_ub, gamma."""
    b = log_weights(w)
    u, v, sw, rs, st = sinkhorn(b, p_sched, tol, max_sweeps)
    p = float(np.atleast_1d(p_sched)[-1])
    mask = prune_mask(b, p, u, v, t, guard)
    bb = np.where(mask, b, -np.inf)
    perm, al, be, st_h = hungarian(bb)
    log_w_b = float(sum(b[i, perm[i]] for i in range(len(perm)))) if st_h == 0 else -np.inf
    ub = log_ub(b, p, v)
    return {"u": u, "v": v, "sweeps": sw, "resid": rs, "status": st, "mask": mask,
            "perm": perm, "solve_status": st_h, "log_w_B": log_w_b, "log_ub": ub,
            "gamma": gamma(ub, log_w_b) if st_h == 0 else np.inf}


def algorithm1(w, opt_ratio=2.0, p0=100.0, dp=50.0, max_rounds=20, eps=None, t=None, max_sweeps=20000,
               guard=True):
    """Algorithm 1 of the paper with adaptive p: prescale (Sec. 4.1.1), then for p = p0,
    p0 + dp, ... scale to an eps-bistochastic X (eps = 1/n by default), prune at t (1/n),
    solve B exactly and stop when gamma (Eq. optratio) <= opt_ratio.  p is on the prescaled
    scale; the scaling runs on the raw log weights at p * m (the prescaling identity), with
    each round warm-started from the last (potentials scaled by the ratio of the p values).

    Returns a dict with perm, log_w_B, gamma, p_final, p_raw, rounds, sweeps, status
    (0 success, 1 max_rounds reached)."""
    b = log_weights(w)
    n = b.shape[0]
    wpos = np.asarray(w)[np.asarray(w) > 0]
    ratio = float(wpos.max()) / float(wpos.min())
    m = 1.0 / np.log(ratio) if ratio > np.e else 1.0
    eps = 1.0 / n if eps is None else eps
    t = 1.0 / n if t is None else t
    u = v = None
    p, p_prev = p0, None
    sweeps = 0
    out = None
    for r in range(max_rounds):
        p_raw = p * m
        if u is None:
            u, v, sw, rs, st = sinkhorn(b, [p_raw], eps, max_sweeps)
            sweeps += int(sw.sum())
        else:
            f = p_raw / p_prev
            u, v, sw, rs, st = sinkhorn_from(b, p_raw, u * f, v * f, eps, max_sweeps)
            sweeps += sw
        mask = prune_mask(b, p_raw, u, v, t, guard)
        perm, al, be, st_h = hungarian(np.where(mask, b, -np.inf))
        if st_h == 0:
            log_w_b = float(sum(b[i, perm[i]] for i in range(n)))
            g = gamma(log_ub(b, p_raw, v), log_w_b)
        else:
            log_w_b, g = -np.inf, np.inf
        out = {"perm": perm, "log_w_B": log_w_b, "gamma": g, "p_final": p, "p_raw": p_raw, "rounds": r + 1,
               "sweeps": sweeps, "nnz": int(mask.sum()), "status": 1}
        if g <= opt_ratio:
            out["status"] = 0
            return out
        p_prev = p_raw
        p += dp
    return out



def newton(b, p, tol=1e-12, max_newton=200, delta=0.1):
    """Diagonal scaling of A^(p) by Newton iteration (Sec. 5.3, after Knight and Ruiz).

    The nonsymmetric A^(p) enters through its symmetric embedding S = [[0, A], [A^T, 0]];
    the scaling x = (x_r, x_c) > 0 solves f(x) = D(x) S x - 1 = 0, and Newton's method
    on f reads A_k x_{k+1} = S x_k + D(x_k)^{-1} 1 with A_k = S + D(x_k)^{-1} D(S x_k).
    Each A_k is singular along the scaling gauge (x_r t, x_c / t) but the system is
    consistent, so it is solved densely by least squares (numpy) after the change of
    variables x_{k+1} = D(x_k) y that makes it symmetric.  The iteration starts from the
    max-normalised point (rows, then columns, divided by their largest entry).  A step
    whose new
    x_{k+1} / x_k falls below delta anywhere is shortened so that its smallest ratio is
    delta (keeps x positive; the paper defers such safeguards to Knight and Ruiz).

    A^(p) is formed explicitly, scaled by exp(-p max b): this is the paper's remark that
    a non-logarithmic scaling needs p (b_max - b_min) within the exponent range of the
    arithmetic (Sec. 4.1.1); beyond 700 this raises ValueError.

    Returns (u, v, iterations, residuals, status) with x_ij = exp(p b_ij - u_i - v_j);
    residuals[k] = max |f(x_k)| (rows and columns); status 0 converged, 1 not.
    """
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    fin = np.isfinite(b)
    bmax, bmin = float(b[fin].max()), float(b[fin].min())
    if p * (bmax - bmin) > 700.0:
        raise ValueError("p (b_max - b_min) > 700: A^(p) leaves the FP64 range")
    shift = p * bmax
    with np.errstate(invalid="ignore"):
        a = np.where(fin, np.exp(p * b - shift), 0.0)
    s = np.zeros((2 * n, 2 * n))
    s[:n, n:] = a
    s[n:, :n] = a.T
    # starting point: rows, then columns, divided by their largest entry (a diagonal
    # scaling, so X(p) is unchanged); from x = 1 the Newton systems of a wide-range
    # A^(p) are numerically singular and the damped steps stall
    x = np.ones(2 * n)
    x[:n] = 1.0 / a.max(axis=1)
    x[n:] = 1.0 / (x[:n, None] * a).max(axis=0)
    res = []
    status = 1
    for k in range(max_newton + 1):
        sx = s @ x
        f = x * sx - 1.0
        res.append(float(np.max(np.abs(f))))
        if res[-1] <= tol:
            status = 0
            break
        if k == max_newton:
            break
        # the same equation multiplied by D(x_k) on the left, in y = x_{k+1} / x_k:
        # (D(x_k) S D(x_k) + D(v)) y = v + 1 with v = D(x_k) S x_k, which is symmetric
        # and well scaled whatever the spread of x_k
        vk = x * sx
        mk = x[:, None] * s * x[None, :] + np.diag(vk)
        y = np.linalg.lstsq(mk, vk + 1.0, rcond=None)[0]
        if y.min() < delta:
            tau = (1.0 - delta) / (1.0 - y.min())
            y = 1.0 + tau * (y - 1.0)
        x = x * y
    u = shift - np.log(x[:n])
    v = -np.log(x[n:])
    return u, v, len(res) - 1, np.array(res), status
