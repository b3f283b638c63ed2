"""ctypes binding of libiccg (include/iccg.h): argument marshalling only.

Every function here has the name of the C entry point it calls.  Arrays may be
numpy arrays (host) or torch tensors (host or CUDA); their data pointers are
passed straight through, so all compute runs in the library's CUDA kernels.
The library is loaded from this package directory; if it is missing the
import of any function raises (there is no fallback path).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiccg.so")

STATUS = {0: "ICCG_OK", 1: "ICCG_ERR_ARG", 2: "ICCG_ERR_COLORING", 3: "ICCG_ERR_BREAKDOWN",
          4: "ICCG_NOT_CONVERGED", 5: "ICCG_ERR_CUDA", 6: "ICCG_ERR_TIMEOUT", 7: "ICCG_ERR_NONFINITE",
          8: "ICCG_ERR_UNIMPLEMENTED", 9: "ICCG_ERR_STATE"}
ICCG_OK, ICCG_ERR_ARG, ICCG_NOT_CONVERGED = 0, 1, 4


class IccgError(RuntimeError):
    def __init__(self, status, where, index=-1, msg=""):
        self.status = status
        self.index = index
        super().__init__(f"{where}: {STATUS.get(status, status)} (index {index}) {msg}".strip())


class iccg_opts(ctypes.Structure):
    _fields_ = [("precond_fp32", ctypes.c_int32), ("warps_per_cta", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("no_graph", ctypes.c_int32),
                ("no_pdl", ctypes.c_int32), ("solver", ctypes.c_int32), ("lane_block_max", ctypes.c_int32),
                ("tile_mapping", ctypes.c_int32), ("fuse_sweep", ctypes.c_int32)]


SOLVERS = {"auto": 0, "persistent": 1, "phased": 2}
TILE_MAPPINGS = {"auto": 0, "cta": 1, "warp": 2, "pair": 3, "units": 4}


class iccg_batch_opts(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32), ("autotune", ctypes.c_int32),
                ("rows_per_thread", ctypes.c_int32), ("reserved", ctypes.c_int32 * 4)]


_lib = None


def load():
    """Load libiccg.so (raises when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} not built; run paper_2609_00561_gb300.build.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i32, i64, d, u64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double, ctypes.c_uint64
    P = ctypes.POINTER
    sig = {
        "iccg_setup": [P(vp), i32, i64, vp, vp, vp, vp, vp, vp, i32, i32, P(iccg_opts), vp],
        "iccg_factor": [vp],
        "iccg_solve": [vp, vp, vp, d, i32, P(i32), vp],
        "iccg_precond": [vp, vp, vp],
        "iccg_spmv": [vp, vp, vp],
        "iccg_get_factor": [vp, vp, P(i64)],
        "iccg_profile_solve": [vp, vp, vp, d, i32, P(i32), vp, vp],
        "iccg_info": [vp, vp],
        "iccg_time_spmv_phase": [vp, i32, P(d)],
        "iccg_last_error": [vp, P(i64), P(ctypes.c_char_p)],
        "iccg_set_wait_limit": [vp, u64],
        "iccg_graph": [i32, vp, vp, vp, vp, P(i64)],
        "iccg_block_abmc": [i32, vp, vp, i32, vp, P(i32)],
        "iccg_block_leiden": [i32, vp, vp, i32, d, i32, d, u64, vp, P(i32)],
        "iccg_sort_blocks_desc": [i32, i32, vp],
        "iccg_color_order": [i32, vp, vp, i32, vp, vp, P(i32), vp, vp, vp],
        "iccg_level_order": [i32, vp, vp, vp, P(i32), vp, vp, vp],
        "iccg_dev_graph": [i32, vp, vp, i64, vp, vp, P(i64), vp],
        "iccg_dev_color_order": [i32, vp, vp, i64, i32, vp, vp, P(i32), vp, vp, vp, vp],
        "iccg_dev_sort_blocks_desc": [i32, i32, vp, vp],
        "iccg_dev_block_leiden": [i32, vp, vp, i64, i32, d, i32, vp, P(i32), vp],
        "iccg_split_levels": [i32, vp, vp, vp, vp, vp, i32, i32, i32, vp, vp, vp, P(i32), P(i32)],
        "iccg_spmv_dot_noalloc": [i32, vp, vp, vp, vp, vp, vp, vp],
        "iccg_batch_create": [P(vp), vp, i32, i32, P(iccg_batch_opts)],
        "iccg_features": [i32, vp, vp, vp, vp],
        "iccg_check_layout": [i32, i64, vp, vp, vp, vp, vp, vp, i32, i32, i32, i32, i32, vp, P(ctypes.c_char_p)],
        "iccg_mlp_forward": [vp, i32, i32, i32, vp, i32, vp, vp, vp],
        "iccg_mlp_grad": [vp, i32, i32, i32, vp, vp, vp, ctypes.c_float, i32, vp, vp, vp, vp],
        "iccg_mlp_adam": [vp, vp, vp, vp, i64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, i32,
                          vp],
        "iccg_batch_solve": [vp, vp, vp, d, i32, vp, vp, vp],
        "iccg_batch_tune": [vp, vp, d, i32, P(d)],
        "iccg_batch_info": [vp, vp],
        "iccg_batch_set_wait_limit": [vp, u64],
        "iccg_batch_last_error": [vp, P(ctypes.c_char_p)],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.iccg_destroy.argtypes = [vp]
    L.iccg_destroy.restype = None
    L.iccg_batch_destroy.argtypes = [vp]
    L.iccg_batch_destroy.restype = None
    L.iccg_mlp_nparams.argtypes = [i32, i32, i32]
    L.iccg_mlp_nparams.restype = ctypes.c_int64
    _lib = L
    return L


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(st, where, ctx=None):
    if st in (ICCG_OK, ICCG_NOT_CONVERGED):
        return st
    idx, msg = -1, ""
    if ctx is not None:
        i = ctypes.c_int64(-1)
        m = ctypes.c_char_p()
        load().iccg_last_error(ctx, ctypes.byref(i), ctypes.byref(m))
        idx, msg = i.value, (m.value or b"").decode()
    raise IccgError(st, where, idx, msg)


def _as(a, dt):
    if hasattr(a, "data_ptr"):
        return a
    return np.ascontiguousarray(a, dtype=dt)


def make_opts(precond_fp32=0, warps_per_cta=0, rows_per_thread=0, no_graph=0, no_pdl=0, solver="auto",
              lane_block_max=0, tile_mapping="auto", fuse_sweep=0):
    o = iccg_opts()
    o.precond_fp32, o.warps_per_cta, o.rows_per_thread, o.no_graph, o.no_pdl = (
        int(precond_fp32), int(warps_per_cta), int(rows_per_thread), int(no_graph), int(no_pdl))
    o.solver = SOLVERS[solver] if isinstance(solver, str) else int(solver)
    o.lane_block_max = int(lane_block_max)
    o.tile_mapping = TILE_MAPPINGS[tile_mapping] if isinstance(tile_mapping, str) else int(tile_mapping)
    o.fuse_sweep = int(fuse_sweep)
    return o


# ---------------------------------------------------------------------------
# C entry points
# ---------------------------------------------------------------------------
def iccg_setup(n, nnz, rowptr, colind, val, perm, block_ptr, color_ptr, n_b, n_c, opts=None, stream=None):
    """Returns a context handle (ctypes.c_void_p)."""
    L = load()
    ctx = ctypes.c_void_p()
    keep = [_as(rowptr, np.int64), _as(colind, np.int32), _as(val, np.float64), _as(perm, np.int32),
            _as(block_ptr, np.int32), _as(color_ptr, np.int32)]
    o = opts if opts is not None else make_opts()
    st = L.iccg_setup(ctypes.byref(ctx), int(n), int(nnz), *[_ptr(k) for k in keep], int(n_b), int(n_c),
                      ctypes.byref(o), ctypes.c_void_p(stream or 0))
    if st != ICCG_OK:
        err = IccgError(st, "iccg_setup")
        if ctx.value:
            i = ctypes.c_int64(-1)
            m = ctypes.c_char_p()
            L.iccg_last_error(ctx, ctypes.byref(i), ctypes.byref(m))
            err = IccgError(st, "iccg_setup", i.value, (m.value or b"").decode())
            L.iccg_destroy(ctx)
        raise err
    return ctx


def iccg_factor(ctx):
    return _check(load().iccg_factor(ctx), "iccg_factor", ctx)


def iccg_solve(ctx, b, x, tol=1e-8, maxit=10000, want_hist=True):
    """x is updated in place (in: x0).  Returns (status, iterations, history)."""
    it = ctypes.c_int32(0)
    hist = np.zeros(maxit + 1) if want_hist else None
    st = load().iccg_solve(ctx, _ptr(b), _ptr(x), float(tol), int(maxit), ctypes.byref(it), _ptr(hist))
    _check(st, "iccg_solve", ctx)
    return st, it.value, (hist[: it.value + 1].copy() if want_hist else None)


def iccg_precond(ctx, r, z):
    return _check(load().iccg_precond(ctx, _ptr(r), _ptr(z)), "iccg_precond", ctx)


def iccg_spmv(ctx, p, q):
    return _check(load().iccg_spmv(ctx, _ptr(p), _ptr(q)), "iccg_spmv", ctx)


def iccg_get_factor(ctx):
    """IC(0) factor as values on tril(A_hat) in CSR order (diagonal last)."""
    cnt = ctypes.c_int64(0)
    _check(load().iccg_get_factor(ctx, None, ctypes.byref(cnt)), "iccg_get_factor", ctx)
    out = np.zeros(cnt.value)
    _check(load().iccg_get_factor(ctx, _ptr(out), ctypes.byref(cnt)), "iccg_get_factor", ctx)
    return out


PHASES = ("init", "spmv", "fwd", "fused", "bwd", "all")


def iccg_profile_solve(ctx, b, x, tol=1e-8, maxit=10000):
    """Returns (status, iterations, {phase: ms}, {phase: launches})."""
    it = ctypes.c_int32(0)
    ms = np.zeros(6)
    ln = np.zeros(6, dtype=np.int64)
    st = load().iccg_profile_solve(ctx, _ptr(b), _ptr(x), float(tol), int(maxit), ctypes.byref(it),
                                   _ptr(ms), _ptr(ln))
    _check(st, "iccg_profile_solve", ctx)
    return st, it.value, dict(zip(PHASES, ms.tolist())), dict(zip(PHASES, ln.tolist()))


def iccg_time_spmv_phase(ctx, reps=50):
    """Milliseconds of one SpMV phase (p update + SpMV with <p,q>) of a PCG
    iteration, averaged over `reps` back-to-back launches."""
    ms = ctypes.c_double(0.0)
    _check(load().iccg_time_spmv_phase(ctx, int(reps), ctypes.byref(ms)), "iccg_time_spmv_phase", ctx)
    return ms.value


INFO_KEYS = ("n", "nnz", "n_b", "n_c", "groups", "global_groups", "nL", "max_levels", "max_group_rows", "tiles",
             "tile_colors", "warp_tile_colors", "pair_tile_colors", "unit_colors", "fused_sweep",
             "factor_launches", "launches_per_iteration", "solve_fixed_launches")


def iccg_info(ctx):
    out = np.zeros(len(INFO_KEYS), dtype=np.int64)
    _check(load().iccg_info(ctx, _ptr(out)), "iccg_info", ctx)
    return dict(zip(INFO_KEYS, out.tolist()))


def iccg_last_error(ctx):
    i = ctypes.c_int64(-1)
    m = ctypes.c_char_p()
    load().iccg_last_error(ctx, ctypes.byref(i), ctypes.byref(m))
    return i.value, (m.value or b"").decode()


def iccg_set_wait_limit(ctx, wait_ns):
    """Device-side wait limit (ns) of the persistent solver; 0 = default."""
    return _check(load().iccg_set_wait_limit(ctx, int(wait_ns)), "iccg_set_wait_limit", ctx)


def iccg_destroy(ctx):
    if ctx is not None and ctx.value:
        load().iccg_destroy(ctx)


def iccg_graph(n, rowptr, colind):
    rowptr = _as(rowptr, np.int64)
    colind = _as(colind, np.int32)
    gptr = np.zeros(n + 1, dtype=np.int64)
    m = ctypes.c_int64(0)
    _check(load().iccg_graph(int(n), _ptr(rowptr), _ptr(colind), _ptr(gptr), None, ctypes.byref(m)), "iccg_graph")
    gadj = np.zeros(max(m.value, 1), dtype=np.int32)
    _check(load().iccg_graph(int(n), _ptr(rowptr), _ptr(colind), _ptr(gptr), _ptr(gadj), ctypes.byref(m)), "iccg_graph")
    return gptr, gadj[: m.value]


def iccg_block_abmc(n, gptr, gadj, s):
    gptr, gadj = _as(gptr, np.int64), _as(gadj, np.int32)
    block_of = np.zeros(max(n, 1), dtype=np.int32)
    nb = ctypes.c_int32(0)
    _check(load().iccg_block_abmc(int(n), _ptr(gptr), _ptr(gadj), int(s), _ptr(block_of), ctypes.byref(nb)),
           "iccg_block_abmc")
    return block_of[:n], nb.value


def iccg_block_leiden(n, gptr, gadj, quality, gamma, n_iter=2, beta=0.01, seed=42):
    q = {"modularity": 0, "md": 0, "cpm": 1, "cp": 1}[quality] if isinstance(quality, str) else int(quality)
    gptr, gadj = _as(gptr, np.int64), _as(gadj, np.int32)
    block_of = np.zeros(max(n, 1), dtype=np.int32)
    nb = ctypes.c_int32(0)
    _check(load().iccg_block_leiden(int(n), _ptr(gptr), _ptr(gadj), q, float(gamma), int(n_iter), float(beta),
                                    int(seed), _ptr(block_of), ctypes.byref(nb)), "iccg_block_leiden")
    return block_of[:n], nb.value


def iccg_sort_blocks_desc(n, n_b, block_of):
    b = np.array(block_of, dtype=np.int32, copy=True)
    _check(load().iccg_sort_blocks_desc(int(n), int(n_b), _ptr(b)), "iccg_sort_blocks_desc")
    return b


def iccg_color_order(n, gptr, gadj, n_b, block_of):
    """Returns (color_of, n_c, perm, block_ptr, color_ptr)."""
    gptr, gadj, block_of = _as(gptr, np.int64), _as(gadj, np.int32), _as(block_of, np.int32)
    color_of = np.zeros(max(n_b, 1), dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    bptr = np.zeros(n_b + 1, dtype=np.int32)
    cptr = np.zeros(n_b + 1, dtype=np.int32)
    nc = ctypes.c_int32(0)
    _check(load().iccg_color_order(int(n), _ptr(gptr), _ptr(gadj), int(n_b), _ptr(block_of), _ptr(color_of),
                                   ctypes.byref(nc), _ptr(perm), _ptr(bptr), _ptr(cptr)), "iccg_color_order")
    return color_of[:n_b], nc.value, perm[:n], bptr, cptr[: nc.value + 1]


def iccg_dev_graph(rowptr, colind, stream=None):
    """Device graph: rowptr int64[n+1], colind int32[nnz] CUDA tensors ->
    (gptr int64[n+1], gadj int32[m]) CUDA tensors."""
    import torch
    n, nnz = rowptr.numel() - 1, colind.numel()
    gptr = torch.empty(n + 1, dtype=torch.int64, device=rowptr.device)
    gadj = torch.empty(max(2 * nnz, 1), dtype=torch.int32, device=rowptr.device)
    m = ctypes.c_int64(0)
    _check(load().iccg_dev_graph(int(n), _ptr(rowptr), _ptr(colind), int(nnz), _ptr(gptr), _ptr(gadj),
                                 ctypes.byref(m), ctypes.c_void_p(stream or 0)), "iccg_dev_graph")
    return gptr, gadj[: m.value]


def iccg_dev_color_order(gptr, gadj, n_b, block_of, stream=None):
    """Device greedy block coloring + ordering (CUDA tensors in and out).
    Returns (color_of, n_c, perm, block_ptr, color_ptr)."""
    import torch
    n, dev = gptr.numel() - 1, gptr.device
    color_of = torch.empty(max(n_b, 1), dtype=torch.int32, device=dev)
    perm = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    bptr = torch.empty(n_b + 1, dtype=torch.int32, device=dev)
    cptr = torch.empty(n_b + 1, dtype=torch.int32, device=dev)
    nc = ctypes.c_int32(0)
    _check(load().iccg_dev_color_order(int(n), _ptr(gptr), _ptr(gadj), int(gadj.numel()), int(n_b), _ptr(block_of),
                                       _ptr(color_of), ctypes.byref(nc), _ptr(perm), _ptr(bptr), _ptr(cptr),
                                       ctypes.c_void_p(stream or 0)), "iccg_dev_color_order")
    return color_of[:n_b], nc.value, perm[:n], bptr, cptr[: nc.value + 1]


def iccg_dev_sort_blocks_desc(n_b, block_of, stream=None):
    """Relabels the CUDA tensor block_of in place (Leiden block order)."""
    _check(load().iccg_dev_sort_blocks_desc(int(block_of.numel()), int(n_b), _ptr(block_of),
                                            ctypes.c_void_p(stream or 0)), "iccg_dev_sort_blocks_desc")
    return block_of


def iccg_dev_block_leiden(gptr, gadj, quality, gamma, n_iter=2, stream=None):
    """Device Leiden blocking (CUDA tensors).  Returns (block_of, n_b)."""
    import torch
    q = {"modularity": 0, "md": 0, "cpm": 1, "cp": 1}[quality] if isinstance(quality, str) else int(quality)
    n = gptr.numel() - 1
    block_of = torch.empty(max(n, 1), dtype=torch.int32, device=gptr.device)
    nb = ctypes.c_int32(0)
    _check(load().iccg_dev_block_leiden(int(n), _ptr(gptr), _ptr(gadj), int(gadj.numel()), q, float(gamma),
                                        int(n_iter), _ptr(block_of), ctypes.byref(nb), ctypes.c_void_p(stream or 0)),
           "iccg_dev_block_leiden")
    return block_of[:n], nb.value


def dev_blocking(a, method="leiden_cpm", gamma=0.5, n_iter=2, block_size=32, stream=None):
    """The blocking pipeline on the device (graph -> Leiden -> size order ->
    greedy coloring -> ordering); returns the host dict of `blocking`.
    method "abmc": the graph and the coloring / ordering on the device, the
    ABMC blocks themselves by the host code (a sequential breadth-first
    construction by its definition)."""
    import torch
    rp = torch.as_tensor(np.asarray(a.rowptr, dtype=np.int64)).cuda()
    ci = torch.as_tensor(np.asarray(a.colind, dtype=np.int32)).cuda()
    gptr, gadj = iccg_dev_graph(rp, ci, stream)
    if method == "abmc":
        bo, nb = iccg_block_abmc(a.n, gptr.cpu().numpy(), gadj.cpu().numpy(), block_size)
        block_of = torch.as_tensor(bo).cuda()
    else:
        q = {"leiden_md": "modularity", "leiden_cpm": "cpm"}[method]
        block_of, nb = iccg_dev_block_leiden(gptr, gadj, q, gamma, n_iter, stream)
        iccg_dev_sort_blocks_desc(nb, block_of, stream)
    color_of, nc, perm, bptr, cptr = iccg_dev_color_order(gptr, gadj, nb, block_of, stream)
    return {"perm": perm.cpu().numpy(), "block_ptr": bptr.cpu().numpy(), "color_ptr": cptr.cpu().numpy(),
            "n_b": nb, "n_c": nc, "block_of": block_of.cpu().numpy(), "color_of": color_of.cpu().numpy()}


def iccg_level_order(n, gptr, gadj):
    """Returns (level_of, n_lev, perm, block_ptr, color_ptr)."""
    gptr, gadj = _as(gptr, np.int64), _as(gadj, np.int32)
    lev = np.zeros(max(n, 1), dtype=np.int32)
    perm = np.zeros(max(n, 1), dtype=np.int32)
    bptr = np.zeros(n + 1, dtype=np.int32)
    cptr = np.zeros(n + 1, dtype=np.int32)
    nl = ctypes.c_int32(0)
    _check(load().iccg_level_order(int(n), _ptr(gptr), _ptr(gadj), _ptr(lev), ctypes.byref(nl), _ptr(perm),
                                   _ptr(bptr), _ptr(cptr)), "iccg_level_order")
    return lev[:n], nl.value, perm[:n], bptr, cptr[: nl.value + 1]


def iccg_split_levels(a, bl, max_rows=32):
    """Refines a blocking dict (perm, block_ptr, color_ptr, n_b, n_c): blocks
    above max_rows rows become their in-block levels, one color of one-row
    blocks per level.  Returns a blocking dict of the same form."""
    n = a.n
    keep = [_as(a.rowptr, np.int64), _as(a.colind, np.int32), _as(bl["perm"], np.int32),
            _as(bl["block_ptr"], np.int32), _as(np.asarray(bl["color_ptr"])[:bl["n_c"] + 1], np.int32)]
    perm = np.zeros(max(n, 1), dtype=np.int32)
    bptr = np.zeros(n + 1, dtype=np.int32)
    cptr = np.zeros(n + 1, dtype=np.int32)
    nb, nc = ctypes.c_int32(0), ctypes.c_int32(0)
    _check(load().iccg_split_levels(int(n), *[_ptr(k) for k in keep], int(bl["n_b"]), int(bl["n_c"]), int(max_rows),
                                    _ptr(perm), _ptr(bptr), _ptr(cptr), ctypes.byref(nb), ctypes.byref(nc)),
           "iccg_split_levels")
    return {"perm": perm[:n], "block_ptr": bptr[:nb.value + 1], "color_ptr": cptr[:nc.value + 1], "n_b": nb.value,
            "n_c": nc.value}


NOALLOC_MAX_ROWS = 4194304


def iccg_spmv_dot_noalloc(n, rowptr, colind, val, p, q, pq, stream=None):
    """q = A p and pq[0] = <p, q> through the allocation-free entry point.
    All arrays are device tensors owned by the caller (rowptr int64, colind
    int32, val / p / q / pq float64); returns the status code."""
    return load().iccg_spmv_dot_noalloc(int(n), _ptr(rowptr), _ptr(colind), _ptr(val), _ptr(p), _ptr(q),
                                        _ptr(pq), ctypes.c_void_p(stream or 0))


# ---------------------------------------------------------------------------
# conveniences built only from the entry points above
# ---------------------------------------------------------------------------
def blocking(a, method="abmc", block_size=32, gamma=1.0, n_iter=2, beta=0.01, seed=42):
    """graph -> ABMC or Leiden (+ size sort) -> greedy coloring -> ordering,
    or the level-set ordering of the natural order ("levels": one-row blocks,
    colors = levels).  `a` has fields n, rowptr, colind.  Returns a dict like
    the oracle's."""
    gptr, gadj = iccg_graph(a.n, a.rowptr, a.colind)
    if method == "levels":
        lev, nl, perm, bptr, cptr = iccg_level_order(a.n, gptr, gadj)
        return {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": a.n, "n_c": nl,
                "block_of": np.arange(a.n, dtype=np.int32), "color_of": lev}
    if method == "abmc":
        block_of, nb = iccg_block_abmc(a.n, gptr, gadj, block_size)
    elif method in ("leiden_md", "leiden_cpm"):
        q = 0 if method == "leiden_md" else 1
        block_of, nb = iccg_block_leiden(a.n, gptr, gadj, q, gamma, n_iter, beta, seed)
        block_of = iccg_sort_blocks_desc(a.n, nb, block_of)
    else:
        raise ValueError(method)
    color_of, nc, perm, bptr, cptr = iccg_color_order(a.n, gptr, gadj, nb, block_of)
    return {"perm": perm, "block_ptr": bptr, "color_ptr": cptr, "n_b": nb, "n_c": nc,
            "block_of": block_of, "color_of": color_of}


class Solver:
    """Owns one iccg context: setup + factor at construction."""

    def __init__(self, a, bl, precond_fp32=False, warps_per_cta=0, rows_per_thread=0, no_graph=False,
                 no_pdl=False, stream=None, factor=True, solver="auto", lane_block_max=0, tile_mapping="auto",
                 fuse_sweep=0):
        self.n = a.n
        self.ctx = iccg_setup(a.n, a.nnz, a.rowptr, a.colind, a.val, bl["perm"], bl["block_ptr"],
                              bl["color_ptr"], bl["n_b"], bl["n_c"],
                              make_opts(precond_fp32, warps_per_cta, rows_per_thread, no_graph, no_pdl, solver,
                                        lane_block_max, tile_mapping, fuse_sweep),
                              stream)
        if factor:
            iccg_factor(self.ctx)

    def solve(self, b, x=None, tol=1e-8, maxit=10000):
        if x is None:
            x = np.zeros(self.n) if isinstance(b, np.ndarray) else b.new_zeros(b.shape)
        st, it, hist = iccg_solve(self.ctx, b, x, tol, maxit)
        return x, it, hist, st

    def info(self):
        return iccg_info(self.ctx)

    def close(self):
        iccg_destroy(self.ctx)
        self.ctx = None

    def __del__(self):
        try:
            if getattr(self, "ctx", None) is not None:
                self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# batched solve (many systems, several right-hand sides each, one launch)
# ---------------------------------------------------------------------------
def _batch_check(st, where, h):
    if st in (ICCG_OK, ICCG_NOT_CONVERGED):
        return st
    m = ctypes.c_char_p()
    if h:
        load().iccg_batch_last_error(h, ctypes.byref(m))
    raise IccgError(st, where, -1, (m.value or b"").decode())


class BatchSolver:
    """iccg_batch over factored Solvers (set up with lane_block_max=-1)."""

    def __init__(self, solvers, nrhs, warps_per_cta=0, ctas_per_sm=0, autotune=False, rows_per_thread=0):
        self.solvers = list(solvers)
        self.nrhs = int(nrhs)
        self.ns = [s.n for s in self.solvers]
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        o = iccg_batch_opts()
        o.warps_per_cta, o.ctas_per_sm, o.autotune = int(warps_per_cta), int(ctas_per_sm), int(bool(autotune))
        o.rows_per_thread = int(rows_per_thread)
        h = ctypes.c_void_p()
        st = load().iccg_batch_create(ctypes.byref(h), arr, len(self.solvers), self.nrhs, ctypes.byref(o))
        self.h = h
        if st != ICCG_OK:
            err = None
            try:
                _batch_check(st, "iccg_batch_create", h)
            except IccgError as e:
                err = e
            if h.value:
                load().iccg_batch_destroy(h)
                self.h = None
            raise err

    def info(self):
        out = np.zeros(7, dtype=np.int32)
        _batch_check(load().iccg_batch_info(self.h, _ptr(out)), "iccg_batch_info", self.h)
        return dict(zip(("warps_per_cta", "ctas_per_sm", "grid", "kp", "smax", "split_exp_x3", "rows_per_thread"),
                        out.tolist()))

    def set_wait_limit(self, wait_ns):
        """iccg_batch_set_wait_limit: barrier wait limit (ns); 0 = default."""
        _batch_check(load().iccg_batch_set_wait_limit(self.h, int(wait_ns)), "iccg_batch_set_wait_limit", self.h)

    def tune(self, B=None, tol=1e-8, maxit=10000):
        """Shape search on B (x0 = 0, to tol) or, without B, a random probe."""
        ms = ctypes.c_double(0.0)
        bp = None if B is None else (ctypes.c_void_p * len(B))(*[_ptr(b) for b in B])
        _batch_check(load().iccg_batch_tune(self.h, bp, float(tol), int(maxit), ctypes.byref(ms)),
                     "iccg_batch_tune", self.h)
        return ms.value

    def solve(self, B, X, tol=1e-8, maxit=10000, want_hist=False):
        """B[s], X[s]: (nrhs, n_s) C-contiguous float64 (numpy or torch, host or
        device); X holds x0 and receives x.  Returns (status, iters, per-RHS
        status, histories)."""
        ns = len(self.solvers)
        bp = (ctypes.c_void_p * ns)(*[_ptr(b) for b in B])
        xp = (ctypes.c_void_p * ns)(*[_ptr(x) for x in X])
        it = np.zeros(ns * self.nrhs, dtype=np.int32)
        stv = np.zeros(ns * self.nrhs, dtype=np.int32)
        hists = None
        hp = None
        if want_hist:
            hists = [np.zeros((maxit + 1, self.nrhs)) for _ in range(ns)]
            hp = (ctypes.c_void_p * ns)(*[h.ctypes.data for h in hists])
        st = load().iccg_batch_solve(self.h, bp, xp, float(tol), int(maxit), _ptr(it), _ptr(stv), hp)
        if st not in (ICCG_OK, ICCG_NOT_CONVERGED, 7):
            _batch_check(st, "iccg_batch_solve", self.h)
        return st, it.reshape(ns, self.nrhs), stv.reshape(ns, self.nrhs), hists

    def close(self):
        if getattr(self, "h", None):
            load().iccg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned blocking: features and the MLP kernels
# ---------------------------------------------------------------------------
NFEATURES = 20


def features(a):
    """The 20 matrix statistics of iccg_features (host)."""
    out = np.zeros(NFEATURES)
    keep = [_as(a.rowptr, np.int64), _as(a.colind, np.int32), _as(a.val, np.float64)]
    _check(load().iccg_features(int(a.n), *[_ptr(k) for k in keep], _ptr(out)), "iccg_features")
    return out


def mlp_nparams(nf, hidden, ncls):
    return int(load().iccg_mlp_nparams(int(nf), int(hidden), int(ncls)))


def mlp_forward(params, nf, hidden, ncls, X, out, act=None, stream=None):
    _check(load().iccg_mlp_forward(_ptr(params), int(nf), int(hidden), int(ncls), _ptr(X), int(X.shape[0]),
                                   _ptr(out), _ptr(act), ctypes.c_void_p(stream or 0)), "iccg_mlp_forward")


def mlp_grad(params, nf, hidden, ncls, X, ycls, yreg, wreg, grad, loss, work, stream=None):
    _check(load().iccg_mlp_grad(_ptr(params), int(nf), int(hidden), int(ncls), _ptr(X), _ptr(ycls), _ptr(yreg),
                                float(wreg), int(X.shape[0]), _ptr(grad), _ptr(loss), _ptr(work),
                                ctypes.c_void_p(stream or 0)), "iccg_mlp_grad")


def mlp_adam(params, grad, m, v, lr, beta1, beta2, eps, step, stream=None):
    _check(load().iccg_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(params.numel()), float(lr),
                                float(beta1), float(beta2), float(eps), int(step), ctypes.c_void_p(stream or 0)),
           "iccg_mlp_adam")


def check_layout(a, bl, group_rows=256, lane_max=32, use_units=False):
    """Host-only check of the device layout (iccg_check_layout): returns
    (status, tiles + warp units, groups, failed checks, first failure, message)."""
    keep = [_as(a.rowptr, np.int64), _as(a.colind, np.int32), _as(a.val, np.float64), _as(bl["perm"], np.int32),
            _as(bl["block_ptr"], np.int32), _as(np.asarray(bl["color_ptr"])[:bl["n_c"] + 1], np.int32)]
    rep = np.zeros(4, dtype=np.int64)
    m = ctypes.c_char_p()
    st = load().iccg_check_layout(int(a.n), int(a.nnz), *[_ptr(k) for k in keep], int(bl["n_b"]), int(bl["n_c"]),
                                  int(group_rows), int(lane_max), int(bool(use_units)), _ptr(rep), ctypes.byref(m))
    return st, int(rep[0]), int(rep[1]), int(rep[2]), int(rep[3]), (m.value or b"").decode()

