"""Thin ctypes binding of libdmrg.so (include/dmrg.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. Buffers may be numpy arrays (host) or torch tensors
(host or CUDA); they are passed to the library as raw pointers. If the
library is not built, every call raises RuntimeError - there is no fallback.
"""

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdmrg.so")

DMRG_OK, DMRG_EINVAL, DMRG_ENOMEM, DMRG_ECUDA, DMRG_ENOCONV, DMRG_ETIMEOUT, DMRG_ESTATE = range(7)
STATUS_NAMES = ["DMRG_OK", "DMRG_EINVAL", "DMRG_ENOMEM", "DMRG_ECUDA", "DMRG_ENOCONV",
                "DMRG_ETIMEOUT", "DMRG_ESTATE"]
DMRG_FP64, DMRG_BF16X2, DMRG_BF16X3, DMRG_FP16X2 = 0, 1, 2, 3


class dmrg_opts(ctypes.Structure):
    _fields_ = [("sigma_prec", ctypes.c_int), ("dav_max_space", ctypes.c_int),
                ("dav_max_iter", ctypes.c_int), ("keep_one_per_q", ctypes.c_int),
                ("noise", ctypes.c_double), ("seed", ctypes.c_ulonglong), ("device", ctypes.c_int),
                ("graphs", ctypes.c_int), ("mixed_cut", ctypes.c_int), ("tc_chain", ctypes.c_int),
                ("tc_producers", ctypes.c_int)]


class dmrg_sigma_info(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_longlong), ("n_products", ctypes.c_longlong),
                ("flops", ctypes.c_double), ("op_elements", ctypes.c_longlong),
                ("op_bytes_read", ctypes.c_double), ("psi_size", ctypes.c_longlong),
                ("tc_items_per_sm", ctypes.c_int), ("tc_producers", ctypes.c_int),
                ("tc_unit_cost", ctypes.c_double)]


class DMRGError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 7 else status}: {msg}")
        self.status = status


class dmrg_request(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("n_left_modes", ctypes.c_int), ("n_modes", ctypes.c_int),
                ("N", ctypes.c_int), ("two_sz", ctypes.c_int), ("n_sec_left", ctypes.c_int),
                ("sec_left", ctypes.c_void_p), ("n_sec_right", ctypes.c_int), ("sec_right", ctypes.c_void_p),
                ("seed", ctypes.c_ulonglong), ("sigma_prec", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double)]


class dmrg_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("converged", ctypes.c_int), ("slot", ctypes.c_int), ("energy", ctypes.c_double),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double), ("t_loaded", ctypes.c_double),
                ("t_done", ctypes.c_double),
                ("bytes", ctypes.c_longlong)]


_lib = None

# C signatures: name -> (restype, argtypes)
_P, _I, _D, _LL, _ULL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_ulonglong
SIGNATURES = {
    "dmrg_default_opts": (None, [ctypes.POINTER(dmrg_opts)]),
    "dmrg_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(dmrg_opts)]),
    "dmrg_destroy": (None, [_P]),
    "dmrg_last_error": (ctypes.c_char_p, [_P]),
    "dmrg_stream": (_P, [_P]),
    "dmrg_set_precision": (_I, [_P, _I]),
    "dmrg_load_synthetic": (_I, [_P, _I, _I, _I, _I, _I, _P, _I, _P, _ULL]),
    "dmrg_load_synthetic_part": (_I, [_P, _I, _I, _I, _I, _I, _P, _I, _P, _ULL, _I, _I]),
    "dmrg_partition_info": (_I, [_I, _I, _I, _I, _I, _P, _I, _P, _I, _I, ctypes.POINTER(_LL),
                                 ctypes.POINTER(_LL), ctypes.POINTER(_LL), _P, _I]),
    "dmrg_psi_layout": (_I, [_P, _I, ctypes.POINTER(_I), _P, _P, _P, _P, ctypes.POINTER(_LL)]),
    "dmrg_get_sigma_info": (_I, [_P, _I, ctypes.POINTER(dmrg_sigma_info)]),
    "dmrg_sigma": (_I, [_P, _I, _P, _P]),
    "dmrg_sigma_noalloc": (_I, [_P, _I, _P, _P]),
    "dmrg_davidson": (_I, [_P, _I, _P, _D, ctypes.POINTER(_D), _P, ctypes.POINTER(_I)]),
    "dmrg_build_blocks": (_I, [_P, _P, _P, _I, _I, _I, _I]),
    "dmrg_sweep": (_I, [_P, _P, _I, _D, _P, _P]),
    "dmrg_sweep_log": (_I, [_P, _P, _I, _P]),
    "dmrg_sigma_part": (_I, [_P, _I, _I, _I, _P, _P]),
    "dmrg_autotune": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_D), ctypes.POINTER(_D)]),
    "dmrg_block_info": (_I, [_P, _I, _I, _P, _P, _P, _P]),
    "dmrg_block_read": (_I, [_P, _I, _I, _I, _P]),
    "dmrg_sync": (_I, [_P]),
    "dmrg_profile": (_I, [_P, _I]),
    "dmrg_profile_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_LL)]),
    "dmrg_profile_waits": (_I, [_P, _P, _I]),
    "dmrg_server_create": (_I, [ctypes.POINTER(_P), _I, _I, _LL]),
    "dmrg_server_submit": (_I, [_P, ctypes.POINTER(dmrg_request)]),
    "dmrg_server_poll": (_I, [_P, _P, _I, _I]),
    "dmrg_server_pending": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I), ctypes.POINTER(_LL)]),
    "dmrg_server_last_error": (ctypes.c_char_p, [_P]),
    "dmrg_server_destroy": (None, [_P]),
}


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built; run paper_2103_09976_gb300.build.build() "
                               "(the CUDA library is required, there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(x):
    """Raw pointer of a numpy array, torch tensor or None."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    if isinstance(x, int):
        return x
    raise TypeError(f"unsupported buffer type {type(x)}")


def _check(ctx, st):
    if st != DMRG_OK:
        raise DMRGError(st, lib().dmrg_last_error(ctx).decode())


def dmrg_default_opts():
    o = dmrg_opts()
    lib().dmrg_default_opts(ctypes.byref(o))
    return o


def dmrg_create(opts=None, **kw):
    o = opts if opts is not None else dmrg_default_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    h = ctypes.c_void_p()
    st = lib().dmrg_create(ctypes.byref(h), ctypes.byref(o))
    _check(None, st)
    return h.value


def dmrg_destroy(ctx):
    lib().dmrg_destroy(ctx)


def dmrg_last_error(ctx):
    return lib().dmrg_last_error(ctx).decode()


def dmrg_stream(ctx):
    return lib().dmrg_stream(ctx)


def dmrg_set_precision(ctx, prec):
    _check(ctx, lib().dmrg_set_precision(ctx, int(prec)))


def dmrg_sync(ctx):
    _check(ctx, lib().dmrg_sync(ctx))


def _sec_array(secs):
    a = np.ascontiguousarray(np.array(secs, dtype=np.int32).reshape(-1, 3))
    return a


def dmrg_load_synthetic(ctx, n_left_modes, n_modes, N, two_sz, sec_left, sec_right, seed):
    L = _sec_array(sec_left)
    R = _sec_array(sec_right)
    _check(ctx, lib().dmrg_load_synthetic(ctx, n_left_modes, n_modes, N, two_sz, len(L), _ptr(L),
                                          len(R), _ptr(R), int(seed)))


def dmrg_load_synthetic_part(ctx, n_left_modes, n_modes, N, two_sz, sec_left, sec_right, seed, rank, n_ranks):
    L = _sec_array(sec_left)
    R = _sec_array(sec_right)
    _check(ctx, lib().dmrg_load_synthetic_part(ctx, n_left_modes, n_modes, N, two_sz, len(L), _ptr(L),
                                               len(R), _ptr(R), int(seed), int(rank), int(n_ranks)))


def dmrg_partition_info(n_left_modes, n_modes, N, two_sz, sec_left, sec_right, rank, n_ranks, max_ids=0):
    """Host-only: dict(n_terms, op_elements, total_elements, term_ids) of sub-Hamiltonian rank."""
    L = _sec_array(sec_left)
    R = _sec_array(sec_right)
    nt, oe, te = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    ids = np.zeros(max(1, max_ids), dtype=np.int32)
    _check(None, lib().dmrg_partition_info(n_left_modes, n_modes, N, two_sz, len(L), _ptr(L), len(R), _ptr(R),
                                           int(rank), int(n_ranks), ctypes.byref(nt), ctypes.byref(oe),
                                           ctypes.byref(te), _ptr(ids), int(max_ids)))
    return {"n_terms": nt.value, "op_elements": oe.value, "total_elements": te.value,
            "term_ids": ids[:min(max_ids, nt.value)]}


def dmrg_psi_layout(ctx, site=-1):
    """Returns dict with q_l (nblk x 2), m_l, m_r, offset, size."""
    nb = ctypes.c_int()
    size = ctypes.c_longlong()
    _check(ctx, lib().dmrg_psi_layout(ctx, site, ctypes.byref(nb), None, None, None, None,
                                      ctypes.byref(size)))
    n = nb.value
    q = np.zeros((n, 2), dtype=np.int32)
    ml = np.zeros(n, dtype=np.int32)
    mr = np.zeros(n, dtype=np.int32)
    off = np.zeros(n, dtype=np.int64)
    _check(ctx, lib().dmrg_psi_layout(ctx, site, ctypes.byref(nb), _ptr(q), _ptr(ml), _ptr(mr),
                                      _ptr(off), ctypes.byref(size)))
    return {"q_l": q, "m_l": ml, "m_r": mr, "offset": off, "size": size.value}


def dmrg_get_sigma_info(ctx, site=-1):
    info = dmrg_sigma_info()
    _check(ctx, lib().dmrg_get_sigma_info(ctx, site, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in dmrg_sigma_info._fields_}


def dmrg_sigma(ctx, site, psi, sigma):
    _check(ctx, lib().dmrg_sigma(ctx, site, _ptr(psi), _ptr(sigma)))


def dmrg_sigma_part(ctx, site, rank, n_ranks, psi, sigma):
    """FP64 sigma of the NC terms owned by sub-Hamiltonian `rank` of `n_ranks`."""
    _check(ctx, lib().dmrg_sigma_part(ctx, site, rank, n_ranks, _ptr(psi), _ptr(sigma)))


def dmrg_autotune(ctx, site=-1):
    """Tune the sigma work list of the context's precision (FP64, or the
    tensor-core plan and its producer setting); returns (items_per_sm,
    per_task_cost, best_ms)."""
    w, c, ms = ctypes.c_int(), ctypes.c_double(), ctypes.c_double()
    _check(ctx, lib().dmrg_autotune(ctx, site, ctypes.byref(w), ctypes.byref(c), ctypes.byref(ms)))
    return w.value, c.value, ms.value


def dmrg_sigma_noalloc(ctx, site, psi, sigma):
    """FP64 sigma with the library's fixed 32 MiB device scratch (no allocation;
    device pointers only; calls on one device must not overlap)."""
    _check(ctx, lib().dmrg_sigma_noalloc(ctx, site, _ptr(psi), _ptr(sigma)))


def dmrg_davidson(ctx, site, psi0, tol, psi_out=None):
    e = ctypes.c_double()
    it = ctypes.c_int()
    st = lib().dmrg_davidson(ctx, site, _ptr(psi0), float(tol), ctypes.byref(e), _ptr(psi_out),
                             ctypes.byref(it))
    if st not in (DMRG_OK, DMRG_ENOCONV):
        _check(ctx, st)
    return e.value, it.value, st == DMRG_OK


def dmrg_build_blocks(ctx, t, v, K, N, two_sz, M_init):
    t = np.ascontiguousarray(t, dtype=np.float64)
    v = np.ascontiguousarray(v, dtype=np.float64)
    _check(ctx, lib().dmrg_build_blocks(ctx, _ptr(t), _ptr(v), K, N, two_sz, M_init))


def dmrg_sweep(ctx, M_schedule, tol):
    Ms = np.ascontiguousarray(np.array(M_schedule, dtype=np.int32))
    e = np.zeros(len(Ms))
    d = np.zeros(len(Ms))
    _check(ctx, lib().dmrg_sweep(ctx, _ptr(Ms), len(Ms), float(tol), _ptr(e), _ptr(d)))
    return e, d


def dmrg_block_info(ctx, side, j):
    """Returns (sectors as an (n, 2) int array, dims, number of operators)."""
    ns, nops = ctypes.c_int(), ctypes.c_int()
    _check(ctx, lib().dmrg_block_info(ctx, side, j, ctypes.byref(ns), None, None, ctypes.byref(nops)))
    q = np.zeros((ns.value, 2), dtype=np.int32)
    d = np.zeros(ns.value, dtype=np.int32)
    _check(ctx, lib().dmrg_block_info(ctx, side, j, ctypes.byref(ns), _ptr(q), _ptr(d), ctypes.byref(nops)))
    return q, d, nops.value


def dmrg_block_read(ctx, side, j, op):
    """Dense matrix of operator `op` of block (side, j) over its basis."""
    _, d, _ = dmrg_block_info(ctx, side, j)
    tot = int(d.sum())
    out = np.zeros((tot, tot))
    _check(ctx, lib().dmrg_block_read(ctx, side, j, op, _ptr(out)))
    return out


class dmrg_step_log(ctypes.Structure):
    _fields_ = [("sweep", ctypes.c_int), ("site", ctypes.c_int), ("forward", ctypes.c_int),
                ("iters", ctypes.c_int), ("converged", ctypes.c_int), ("kept", ctypes.c_int),
                ("psi_size", ctypes.c_longlong), ("energy", ctypes.c_double),
                ("discarded", ctypes.c_double), ("t_block", ctypes.c_double), ("t_solve", ctypes.c_double),
                ("t_decimate", ctypes.c_double), ("t_transform", ctypes.c_double)]


def dmrg_sweep_log(ctx):
    """Per-step records of the last dmrg_sweep call, as a list of dicts."""
    n = ctypes.c_int()
    _check(ctx, lib().dmrg_sweep_log(ctx, None, 0, ctypes.byref(n)))
    buf = (dmrg_step_log * max(1, n.value))()
    _check(ctx, lib().dmrg_sweep_log(ctx, buf, n.value, ctypes.byref(n)))
    return [{f: getattr(buf[k], f) for f, _ in dmrg_step_log._fields_} for k in range(n.value)]


KERNEL_SIGMA, KERNEL_REDUCE, KERNEL_DAVIDSON, KERNEL_BLOCKING, KERNEL_SIGMA_SMALL = 0, 1, 2, 3, 4


def dmrg_profile(ctx, enable, waits=False):
    """Per-kernel CUDA-event timing on (enable) / off; waits=True also runs the
    tensor-core kernel's wait accounting (slower kernel)."""
    _check(ctx, lib().dmrg_profile(ctx, (2 if waits else 1) if enable else 0))


def dmrg_profile_read(ctx, kernel):
    ms = ctypes.c_double()
    n = ctypes.c_longlong()
    _check(ctx, lib().dmrg_profile_read(ctx, kernel, ctypes.byref(ms), ctypes.byref(n)))
    return ms.value, n.value


WAIT_KINDS = {1: "stage free", 2: "sigma tile free", 3: "X tile free", 4: "stage loaded",
              5: "second operand written", 6: "X tile computed", 7: "second operand free",
              8: "sigma tile computed", 9: "record slot free", 10: "record loaded (producer)",
              11: "terminator slot", 12: "record loaded (MMA)", 13: "record loaded (epilogue)",
              14: "MMA thread issuing MMAs", 15: "MMA thread committing"}


def dmrg_profile_waits(ctx):
    buf = np.zeros(17)
    _check(ctx, lib().dmrg_profile_waits(ctx, _ptr(buf), 17))
    return buf


# ------------------------------------------------------------------ serving
def _scheck(srv, st):
    if st != DMRG_OK:
        raise DMRGError(st, lib().dmrg_server_last_error(srv).decode())


def dmrg_server_create(device=0, n_slots=4, budget_bytes=200 << 30):
    h = ctypes.c_void_p()
    st = lib().dmrg_server_create(ctypes.byref(h), device, n_slots, int(budget_bytes))
    if st != DMRG_OK:
        raise DMRGError(st, "dmrg_server_create failed")
    return h.value


def dmrg_server_submit(srv, req_id, n_left_modes, n_modes, N, two_sz, left, right, seed,
                       sigma_prec=DMRG_FP64, max_iter=200, tol=1e-8):
    """Queue one Davidson solve; left/right are (N, 2Sz, dim) sector lists."""
    L = np.ascontiguousarray(np.array(left, dtype=np.int32).reshape(-1, 3))
    R = np.ascontiguousarray(np.array(right, dtype=np.int32).reshape(-1, 3))
    r = dmrg_request(req_id, n_left_modes, n_modes, N, two_sz, len(L), L.ctypes.data, len(R), R.ctypes.data,
                     seed, sigma_prec, max_iter, float(tol))
    _scheck(srv, lib().dmrg_server_submit(srv, ctypes.byref(r)))


def dmrg_server_poll(srv, max_results=64, wait_ms=0):
    """Finished results as a list of dicts."""
    buf = (dmrg_result * max_results)()
    n = lib().dmrg_server_poll(srv, buf, max_results, int(wait_ms))
    return [{f: getattr(buf[k], f) for f, _ in dmrg_result._fields_} for k in range(n)]


def dmrg_server_pending(srv):
    q, r, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_longlong()
    _scheck(srv, lib().dmrg_server_pending(srv, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b)))
    return q.value, r.value, b.value


def dmrg_server_last_error(srv):
    return lib().dmrg_server_last_error(srv).decode()


def dmrg_server_destroy(srv):
    lib().dmrg_server_destroy(srv)
