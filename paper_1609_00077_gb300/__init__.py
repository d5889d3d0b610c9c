"""GB300 PQ amplitude solver: Python binding of the C ABI in include/ppq.h.

The binding only marshals arguments (pointers, sizes, the CUDA stream); every
step of the residual, the energy and the Jacobi/DIIS update runs in the CUDA
kernels of libppq.so.  There is no CPU fallback: importing the binding without
the compiled library raises.  Build it with ``python -m
paper_1609_00077_gb300.build`` (or ``__graft_entry__.build()``).
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libppq.so")

N_CHANNELS_1 = 3
N_CHANNELS_2 = 29


class PPQError(RuntimeError):
    pass


class Opts(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int), ("K_H", ctypes.c_int), ("precision", ctypes.c_int),
                ("switch_tol", ctypes.c_double), ("r_tol", ctypes.c_double),
                ("e_tol", ctypes.c_double), ("max_iter", ctypes.c_int),
                ("diis_dim", ctypes.c_int), ("diis_start", ctypes.c_int),
                ("level_shift", ctypes.c_double), ("guess", ctypes.c_int),
                ("profile", ctypes.c_int), ("polish", ctypes.c_int), ("max_rank", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("polish_iters", ctypes.c_int), ("switched_at", ctypes.c_int),
                ("res_norm", ctypes.c_double), ("e_corr", ctypes.c_double),
                ("e_total", ctypes.c_double), ("t_residual_ms", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("residual_flops", ctypes.c_double),
                ("quartic_flops", ctypes.c_double), ("t_quartic_ms", ctypes.c_double),
                ("n_quartic", ctypes.c_int), ("n_launches", ctypes.c_int),
                ("evals_fp32", ctypes.c_int), ("evals_fp64", ctypes.c_int),
                ("t_quartic32_ms", ctypes.c_double), ("n_quartic32", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libppq.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise PPQError(f"{LIB_PATH} is missing: build the CUDA library first "
                           "(python -m paper_1609_00077_gb300.build)")
        L = ctypes.CDLL(LIB_PATH)
        P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        L.ppq_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.ppq_amp_count.argtypes = [I, I, ctypes.POINTER(S)]
        L.ppq_amp_layout.argtypes = [I, P]
        L.pq_residual.argtypes = [I, P, P, P, P, P, P, P, I, P]
        L.pq_residual_static.argtypes = [I, P, P, P, P, P, P, P, I, P]
        L.pq_solve.argtypes = [I, P, P, P, P, D, ctypes.POINTER(Opts), P, P, P, P,
                               ctypes.POINTER(Info), P]
        L.ph_solve.argtypes = L.pq_solve.argtypes
        L.ph_residual.argtypes = [I, P, P, P, P, P, P, P, I, I, P]
        L.ppq_subset_residual.argtypes = [I, I, I, P, P, P, P, P, P, P, I, P]
        L.pq_solve_cd.argtypes = [I, P, P, P, P, I, D, ctypes.POINTER(Opts), P, P, P, P, ctypes.POINTER(Info), P]
        L.ph_solve_cd.argtypes = L.pq_solve_cd.argtypes
        L.ppq_natural_occupations.argtypes = [I, P, P, P, P]
        L.ppq_wait_selftest.argtypes = [ctypes.c_longlong, P, P]
        L.ph_tables_counts.argtypes = [I, I, I, P]
        L.ph_tables_copy.argtypes = [I, I, I, I, P]
        L.ppq_profile_count.argtypes = []
        L.ppq_profile_entry.argtypes = [I, ctypes.c_char_p, I, P, P, P, P]
        L.pq_solve_batched.argtypes = [I, P, P, P, P, P, P, ctypes.POINTER(Opts), P, P, P, P, P]
        L.pq_lagrangian_gradient.argtypes = [I, P, P, P, P, P, P, P, P, P]
        L.pq_lambda.argtypes = [I, P, P, P, P, P, ctypes.POINTER(Opts), P, ctypes.POINTER(Info), P]
        L.pq_gradient.argtypes = [I, P, P, P, P, D, ctypes.POINTER(Opts), P, P, P, P, P, P,
                                  ctypes.POINTER(Info), P]
        L.ph_gradient.argtypes = L.pq_gradient.argtypes
        L.ph_lagrangian_gradient.argtypes = [I, P, P, P, P, P, P, I, P, P, P]
        L.ppq_tc_plan.argtypes = [I, P, I, P, I, ctypes.POINTER(I), ctypes.POINTER(I)]
        L.ppq_last_error.restype = ctypes.c_char_p
        for f in (L.ppq_default_opts, L.ppq_amp_count, L.ppq_amp_layout, L.pq_residual,
                  L.pq_residual_static, L.pq_solve, L.ph_solve, L.pq_solve_batched,
                  L.pq_lagrangian_gradient,
                  L.pq_lambda, L.pq_gradient, L.ppq_release, L.ppq_tc_plan, L.ph_residual,
                  L.ph_tables_counts, L.ph_tables_copy, L.ppq_profile_count, L.ppq_profile_entry,
                  L.ppq_subset_residual, L.pq_solve_cd, L.ph_solve_cd, L.ppq_natural_occupations,
                  L.ppq_wait_selftest, L.ph_gradient, L.ph_lagrangian_gradient):
            f.restype = ctypes.c_int
        _lib = L
    return _lib


EXPORTED = ["ppq_default_opts", "ppq_amp_count", "ppq_amp_layout", "pq_residual",
            "pq_residual_static", "pq_solve", "ph_solve", "ph_residual", "pq_solve_batched",
            "pq_lagrangian_gradient", "pq_lambda", "pq_gradient", "ppq_release", "ppq_last_error",
            "ppq_tc_plan", "ph_tables_counts", "ph_tables_copy", "ppq_profile_count",
            "ppq_profile_entry", "ppq_subset_residual", "pq_solve_cd", "ph_solve_cd",
            "ppq_natural_occupations", "ppq_wait_selftest", "ph_gradient", "ph_lagrangian_gradient"]


def _ptr(x):
    """Device pointer of a torch tensor or host pointer of a numpy array."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags['C_CONTIGUOUS']
        return x.ctypes.data
    return x.data_ptr()


def _stream(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:
        pass
    return None


def _check_buf(x, n, name, device=None):
    """Argument check before any launch: x must be FP64, C-contiguous and hold
    at least n elements; with device set, a CUDA tensor on that device."""
    if isinstance(x, np.ndarray):
        if device is not None:
            raise PPQError(f"{name} must be a CUDA tensor (device memory)")
        ok = x.dtype == np.float64 and x.flags['C_CONTIGUOUS']
        size = x.size
    else:
        ok = str(getattr(x, "dtype", "")) == "torch.float64" and x.is_contiguous()
        size = x.numel()
        if device is not None and (not x.is_cuda or x.device != device):
            raise PPQError(f"{name} must be a CUDA tensor on {device}")
    if not ok:
        raise PPQError(f"{name} must be a contiguous float64 array")
    if size < n:
        raise PPQError(f"{name} holds {size} elements, {n} needed")


def _device_of(x):
    return x.device if hasattr(x, "is_cuda") and x.is_cuda else None


def _check(rc, what):
    if rc < 0:
        raise PPQError(f"{what} failed ({rc}): {lib().ppq_last_error().decode()}")
    return rc


def amp_count(n_pairs, K=2):
    n = ctypes.c_size_t()
    _check(lib().ppq_amp_count(K, n_pairs, ctypes.byref(n)), "ppq_amp_count")
    return n.value


def amp_layout(K=2):
    """(number of pairs, monomials...) per channel: 32 rows of 3 for K = 2,
    335 rows of 4 for K = 3."""
    rows = 32 if K == 2 else 32 + 303
    d = np.zeros(rows * (K + 1), dtype=np.int32)
    _check(lib().ppq_amp_layout(K, d.ctypes.data), "ppq_amp_layout")
    return d.reshape(rows, K + 1)


def tc_plan(n_pairs):
    """Work list of the tensor-core quartic kernel (host only): chunks as an
    (n, 12) int16 array (c1, c2, n_g, n_cols, g[4], q[4]) and CTAs as an (m, 3)
    int32 array (row tile, first chunk, end chunk)."""
    nc, nt = ctypes.c_int(), ctypes.c_int()
    _check(lib().ppq_tc_plan(n_pairs, None, 0, None, 0, ctypes.byref(nc), ctypes.byref(nt)), "ppq_tc_plan")
    ch = np.zeros((nc.value, 12), dtype=np.int16)
    ct = np.zeros((nt.value, 3), dtype=np.int32)
    _check(lib().ppq_tc_plan(n_pairs, ch.ctypes.data, nc.value, ct.ctypes.data, nt.value,
                             ctypes.byref(nc), ctypes.byref(nt)), "ppq_tc_plan")
    return ch, ct


def profile_table():
    """Per-kernel classes of the last call made with profile=1: list of dicts
    (name, ms, launches, bytes, flops), largest time first."""
    L = lib()
    out = []
    for i in range(L.ppq_profile_count()):
        name = ctypes.create_string_buffer(256)
        ms, by, fl = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        n = ctypes.c_int()
        _check(L.ppq_profile_entry(i, name, 256, ctypes.cast(ctypes.pointer(ms), ctypes.c_void_p),
                                   ctypes.cast(ctypes.pointer(n), ctypes.c_void_p),
                                   ctypes.cast(ctypes.pointer(by), ctypes.c_void_p),
                                   ctypes.cast(ctypes.pointer(fl), ctypes.c_void_p)), "ppq_profile_entry")
        out.append({"name": name.value.decode(), "ms": ms.value, "launches": n.value,
                    "bytes": by.value, "flops": fl.value})
    return sorted(out, key=lambda d: -d["ms"])


def default_opts(**kw):
    o = Opts()
    lib().ppq_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _pairs(occ, vir):
    occ = np.ascontiguousarray(occ, dtype=np.int32)
    vir = np.ascontiguousarray(vir, dtype=np.int32)
    return occ, vir


def pq_residual(occ_of_pair, vir_of_pair, h, eri, t, r=None, precision=0, stream=None):
    """R(T) and E_c at amplitudes t (layout of include/ppq.h).  h, eri, t, r may
    be torch CUDA tensors or numpy arrays (FP64, contiguous).  Returns (r, e_corr)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    if r is None:
        r = np.zeros(amp_count(N)) if isinstance(t, np.ndarray) else t.new_zeros(amp_count(N))
    n = 2 * N
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t, amp_count(N), "t"), (r, amp_count(N), "r")):
        _check_buf(x, cnt, name)
    e = ctypes.c_double()
    rc = lib().pq_residual(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), _ptr(t),
                           _ptr(r), ctypes.cast(ctypes.pointer(e), ctypes.c_void_p),
                           precision, _stream(stream))
    _check(rc, "pq_residual")
    return r, e.value


def pq_residual_static(occ_of_pair, vir_of_pair, h, eri, t, r, precision=0, stream=None):
    """pq_residual without device allocation (scratch in a fixed 8 MiB device
    array, n_pairs <= 12).  For callers that cannot call cudaMalloc: h, eri, t
    and r must already be device tensors (torch CUDA).  Returns e_corr."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    n = 2 * N
    dev = _device_of(t)
    if dev is None:
        raise PPQError("pq_residual_static needs device pointers: t must be a CUDA tensor")
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t, amp_count(N), "t"), (r, amp_count(N), "r")):
        _check_buf(x, cnt, name, device=dev)
    e = ctypes.c_double()
    rc = lib().pq_residual_static(len(occ), occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri),
                                  _ptr(t), _ptr(r), ctypes.cast(ctypes.pointer(e), ctypes.c_void_p),
                                  precision, _stream(stream))
    _check(rc, "pq_residual_static")
    return e.value


def pq_solve(occ_of_pair, vir_of_pair, h, eri, e_const=0.0, t_in=None, t_out=None,
             stream=None, **opts):
    """Solve the PQ equations.  Returns (status, e_total, t_out, info dict)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    o = default_opts(**opts)
    if t_in is not None and 'guess' not in opts:
        o.guess = 1
    if t_out is None:
        t_out = np.zeros(amp_count(N))
    ec, et = ctypes.c_double(), ctypes.c_double()
    info = Info()
    rc = lib().pq_solve(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), float(e_const),
                        ctypes.byref(o), _ptr(t_in), _ptr(t_out),
                        ctypes.cast(ctypes.pointer(ec), ctypes.c_void_p),
                        ctypes.cast(ctypes.pointer(et), ctypes.c_void_p),
                        ctypes.byref(info), _stream(stream))
    _check(rc, "pq_solve")
    return rc, et.value, t_out, info.as_dict()


def ph_residual(occ_of_pair, vir_of_pair, h, eri, t, r=None, precision=0, K_H=3, stream=None):
    """R(T) and E_c of the three-pair (PH) model at amplitudes t (the K = 3
    layout of include/ppq.h; only the sorted-label entries are read).  h, eri,
    t, r may be torch CUDA tensors or numpy arrays (FP64, contiguous).
    Returns (r, e_corr), r with every stored order filled."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    L = amp_count(N, 3)
    if r is None:
        r = np.zeros(L) if isinstance(t, np.ndarray) else t.new_zeros(L)
    n = 2 * N
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t, L, "t"), (r, L, "r")):
        _check_buf(x, cnt, name)
    e = ctypes.c_double()
    rc = lib().ph_residual(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), _ptr(t), _ptr(r),
                           ctypes.cast(ctypes.pointer(e), ctypes.c_void_p), precision, K_H, _stream(stream))
    _check(rc, "ph_residual")
    return r, e.value


def subset_residual(K, K_H, occ_of_pair, vir_of_pair, h, eri, t, r=None, precision=0, stream=None):
    """R(T) and E_c by the label-subset expansion for amplitudes over K = 2 or
    3 labels and integrals over K_H labels (0 = K, -1 = untruncated with
    K = 2), in the layout of include/ppq.h for K.  Returns (r, e_corr)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    L = amp_count(N, K)
    if r is None:
        r = np.zeros(L) if isinstance(t, np.ndarray) else t.new_zeros(L)
    n = 2 * N
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t, L, "t"), (r, L, "r")):
        _check_buf(x, cnt, name)
    e = ctypes.c_double()
    rc = lib().ppq_subset_residual(K, K_H, N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), _ptr(t),
                                   _ptr(r), ctypes.cast(ctypes.pointer(e), ctypes.c_void_p), precision,
                                   _stream(stream))
    _check(rc, "ppq_subset_residual")
    return r, e.value


def ph_solve(occ_of_pair, vir_of_pair, h, eri, e_const=0.0, t_in=None, t_out=None, stream=None, **opts):
    """Solve the three-pair (PH) equations.  Returns (status, e_total, t_out,
    info dict); t_out uses the K = 3 layout."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    L = amp_count(N, 3)
    o = default_opts(**opts)
    if t_in is not None and 'guess' not in opts:
        o.guess = 1
    if t_out is None:
        t_out = np.zeros(L)
    n = 2 * N
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t_out, L, "t_out")):
        _check_buf(x, cnt, name)
    if t_in is not None:
        _check_buf(t_in, L, "t_in")
    ec, et = ctypes.c_double(), ctypes.c_double()
    info = Info()
    rc = lib().ph_solve(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), float(e_const),
                        ctypes.byref(o), _ptr(t_in), _ptr(t_out),
                        ctypes.cast(ctypes.pointer(ec), ctypes.c_void_p),
                        ctypes.cast(ctypes.pointer(et), ctypes.c_void_p),
                        ctypes.byref(info), _stream(stream))
    _check(rc, "ph_solve")
    return rc, et.value, t_out, info.as_dict()


def _solve_cd(fn, K, occ_of_pair, vir_of_pair, h, B, e_const, t_in, t_out, stream, opts):
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    L = amp_count(N, K)
    o = default_opts(**opts)
    if t_in is not None and 'guess' not in opts:
        o.guess = 1
    if t_out is None:
        t_out = np.zeros(L)
    n = 2 * N
    naux = (B.shape[0] if hasattr(B, "shape") else 0)
    for x, cnt, name in ((h, n * n, "h"), (B, naux * n * n, "B"), (t_out, L, "t_out")):
        _check_buf(x, cnt, name)
    if t_in is not None:
        _check_buf(t_in, L, "t_in")
    ec, et = ctypes.c_double(), ctypes.c_double()
    info = Info()
    rc = fn(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(B), int(naux), float(e_const), ctypes.byref(o),
            _ptr(t_in), _ptr(t_out), ctypes.cast(ctypes.pointer(ec), ctypes.c_void_p),
            ctypes.cast(ctypes.pointer(et), ctypes.c_void_p), ctypes.byref(info), _stream(stream))
    _check(rc, fn.__name__)
    return rc, et.value, t_out, info.as_dict()


def pq_solve_cd(occ_of_pair, vir_of_pair, h, B, e_const=0.0, t_in=None, t_out=None, stream=None, **opts):
    """pq_solve with the integrals as factors B[Q][p][q] ((pq|rs) = sum_Q
    B[Q,p,q] B[Q,r,s]; shape (naux, n, n)).  Returns (status, e_total, t_out,
    info dict)."""
    return _solve_cd(lib().pq_solve_cd, 2, occ_of_pair, vir_of_pair, h, B, e_const, t_in, t_out, stream, opts)


def ph_solve_cd(occ_of_pair, vir_of_pair, h, B, e_const=0.0, t_in=None, t_out=None, stream=None, **opts):
    """ph_solve with the integrals as factors B[Q][p][q]."""
    return _solve_cd(lib().ph_solve_cd, 3, occ_of_pair, vir_of_pair, h, B, e_const, t_in, t_out, stream, opts)


def natural_occupations(gamma, vectors=False, stream=None):
    """Eigenvalues (descending) of a symmetric density matrix gamma (torch CUDA
    tensor or numpy array, n x n FP64), and the natural orbitals as columns
    when vectors=True.  Returns numpy arrays."""
    n = gamma.shape[0]
    _check_buf(gamma, n * n, "gamma")
    occ = np.zeros(n)
    vec = np.zeros((n, n)) if vectors else None
    _check(lib().ppq_natural_occupations(n, _ptr(gamma), occ.ctypes.data, None if vec is None else vec.ctypes.data,
                                         _stream(stream)), "ppq_natural_occupations")
    return (occ, vec) if vectors else occ


def wait_selftest(cycles=100000, stream=None):
    """Run the bounded-wait self-test (a barrier nothing arrives on); True when
    the wait ran out after `cycles` clock cycles, as it must."""
    flag = ctypes.c_int(0)
    _check(lib().ppq_wait_selftest(int(cycles), ctypes.cast(ctypes.pointer(flag), ctypes.c_void_p),
                                   _stream(stream)), "ppq_wait_selftest")
    return bool(flag.value)


def pq_solve_batched(systems, stream=None, with_amplitudes=False, **opts):
    """Solve many Hamiltonians in one call.  systems: list of (occ_of_pair,
    vir_of_pair, h, eri, e_const) with h / eri torch CUDA tensors or numpy
    arrays.  Returns (status, e_total array, info list[, amplitude list])."""
    n = len(systems)
    occs = [_pairs(o, v)[0] for o, v, *_ in systems]
    virs = [_pairs(o, v)[1] for o, v, *_ in systems]
    NP = np.array([len(o) for o in occs], dtype=np.int32)
    occ_p = (ctypes.c_void_p * n)(*[o.ctypes.data for o in occs])
    vir_p = (ctypes.c_void_p * n)(*[v.ctypes.data for v in virs])
    h_p = (ctypes.c_void_p * n)(*[_ptr(s[2]) for s in systems])
    e_p = (ctypes.c_void_p * n)(*[_ptr(s[3]) for s in systems])
    ec = np.array([float(s[4]) for s in systems])
    amps = [np.zeros(amp_count(int(k))) for k in NP] if with_amplitudes else None
    t_p = (ctypes.c_void_p * n)(*[a.ctypes.data for a in amps]) if with_amplitudes else None
    e_corr = np.zeros(n); e_total = np.zeros(n)
    infos = (Info * n)()
    o = default_opts(**opts)
    rc = lib().pq_solve_batched(n, NP.ctypes.data, ctypes.cast(occ_p, ctypes.c_void_p),
                                ctypes.cast(vir_p, ctypes.c_void_p), ctypes.cast(h_p, ctypes.c_void_p),
                                ctypes.cast(e_p, ctypes.c_void_p), ec.ctypes.data, ctypes.byref(o),
                                ctypes.cast(t_p, ctypes.c_void_p) if t_p is not None else None,
                                e_corr.ctypes.data, e_total.ctypes.data,
                                ctypes.cast(infos, ctypes.c_void_p), _stream(stream))
    _check(rc, "pq_solve_batched")
    out = (rc, e_total, [i.as_dict() for i in infos])
    return out + (amps,) if with_amplitudes else out


def pq_lagrangian_gradient(occ_of_pair, vir_of_pair, h, eri, t, lam, grad=None, stream=None):
    """grad_t L(t, lambda) = dE_c/dt + J^T lambda (FP64, adjoint kernels).
    Returns (grad, e_corr)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    if grad is None:
        grad = np.zeros(amp_count(len(occ))) if isinstance(t, np.ndarray) else t.new_zeros(amp_count(len(occ)))
    e = ctypes.c_double()
    rc = lib().pq_lagrangian_gradient(len(occ), occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri),
                                      _ptr(t), _ptr(lam), _ptr(grad),
                                      ctypes.cast(ctypes.pointer(e), ctypes.c_void_p), _stream(stream))
    _check(rc, "pq_lagrangian_gradient")
    return grad, e.value


def pq_lambda(occ_of_pair, vir_of_pair, h, eri, t, lam_out=None, stream=None, **opts):
    """Lambda amplitudes at converged t.  Returns (status, lambda, info)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    if lam_out is None:
        lam_out = np.zeros(amp_count(len(occ)))
    o = default_opts(**opts)
    info = Info()
    rc = lib().pq_lambda(len(occ), occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), _ptr(t),
                         ctypes.byref(o), _ptr(lam_out), ctypes.byref(info), _stream(stream))
    _check(rc, "pq_lambda")
    return rc, lam_out, info.as_dict()


def pq_gradient(occ_of_pair, vir_of_pair, h, eri, e_const=0.0, stream=None, want_eri=True,
                **opts):
    """Solve PQ, then Lambda, then return (status, e_total, dE/dh, dE/d(pq|rs) or None,
    dE/dkappa, info).  Outputs are torch CUDA tensors when h is one, else numpy."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    n = 2 * len(occ)
    if isinstance(h, np.ndarray):
        dh = np.zeros((n, n)); dk = np.zeros((n, n))
        dv = np.zeros((n, n, n, n)) if want_eri else None
    else:
        dh = h.new_zeros((n, n)); dk = h.new_zeros((n, n))
        dv = h.new_zeros((n, n, n, n)) if want_eri else None
    et = ctypes.c_double()
    info = Info()
    o = default_opts(**opts)
    rc = lib().pq_gradient(len(occ), occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri),
                           float(e_const), ctypes.byref(o), None, None, _ptr(dh),
                           _ptr(dv) if dv is not None else None, _ptr(dk),
                           ctypes.cast(ctypes.pointer(et), ctypes.c_void_p), ctypes.byref(info),
                           _stream(stream))
    _check(rc, "pq_gradient")
    return rc, et.value, dh, dv, dk, info.as_dict()


def ph_lagrangian_gradient(occ_of_pair, vir_of_pair, h, eri, t, lam, K_H=3, grad=None, stream=None):
    """grad_t L(t, lambda) of the PH model (K = 3 layout; FP64 reverse pass of
    the label-subset expansion).  Returns (grad, e_corr)."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    L = amp_count(N, 3)
    if grad is None:
        grad = np.zeros(L) if isinstance(t, np.ndarray) else t.new_zeros(L)
    n = 2 * N
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri"), (t, L, "t"), (lam, L, "lam"), (grad, L, "grad")):
        _check_buf(x, cnt, name)
    e = ctypes.c_double()
    rc = lib().ph_lagrangian_gradient(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), _ptr(t), _ptr(lam),
                                      K_H, _ptr(grad), ctypes.cast(ctypes.pointer(e), ctypes.c_void_p),
                                      _stream(stream))
    _check(rc, "ph_lagrangian_gradient")
    return grad, e.value


def ph_gradient(occ_of_pair, vir_of_pair, h, eri, e_const=0.0, stream=None, want_eri=True, t_out=None,
                lam_out=None, **opts):
    """Solve PH, then Lambda, then return (status, e_total, dE/dh, dE/d(pq|rs)
    or None, dE/dkappa, info).  Outputs are torch CUDA tensors when h is one,
    else numpy; t_out / lam_out (K = 3 layout) are filled when given."""
    occ, vir = _pairs(occ_of_pair, vir_of_pair)
    N = len(occ)
    n = 2 * N
    L = amp_count(N, 3)
    if isinstance(h, np.ndarray):
        dh = np.zeros((n, n)); dk = np.zeros((n, n))
        dv = np.zeros((n, n, n, n)) if want_eri else None
    else:
        dh = h.new_zeros((n, n)); dk = h.new_zeros((n, n))
        dv = h.new_zeros((n, n, n, n)) if want_eri else None
    for x, cnt, name in ((h, n * n, "h"), (eri, n ** 4, "eri")):
        _check_buf(x, cnt, name)
    for x, name in ((t_out, "t_out"), (lam_out, "lam_out")):
        if x is not None:
            _check_buf(x, L, name)
    et = ctypes.c_double()
    info = Info()
    o = default_opts(**opts)
    rc = lib().ph_gradient(N, occ.ctypes.data, vir.ctypes.data, _ptr(h), _ptr(eri), float(e_const),
                           ctypes.byref(o), _ptr(t_out), _ptr(lam_out), _ptr(dh),
                           _ptr(dv) if dv is not None else None, _ptr(dk),
                           ctypes.cast(ctypes.pointer(et), ctypes.c_void_p), ctypes.byref(info), _stream(stream))
    _check(rc, "ph_gradient")
    return rc, et.value, dh, dv, dk, info.as_dict()


_FUNCTIONS = {}


def _autograd_function(model="pq"):
    """torch.autograd.Function of the PQ or PH total energy of (h, (pq|rs)):
    forward solves the amplitudes and the Lambda equations (pq_gradient /
    ph_gradient), backward returns the relaxed densities dE/dh and
    dE/d(pq|rs) scaled by the incoming gradient."""
    if model in _FUNCTIONS:
        return _FUNCTIONS[model]
    import torch
    grad_fn = pq_gradient if model == "pq" else ph_gradient

    class Energy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, h, eri, occ_of_pair, vir_of_pair, e_const, opts):
            rc, e, dh, dv, dk, info = grad_fn(occ_of_pair, vir_of_pair, h.contiguous(), eri.contiguous(), e_const,
                                              **(opts or {}))
            if rc != 0:
                raise PPQError(f"{model}_gradient status {rc}")
            ctx.save_for_backward(dh, dv)
            return h.new_tensor(e)

        @staticmethod
        def backward(ctx, g):
            dh, dv = ctx.saved_tensors
            return g * dh, g * dv, None, None, None, None

    Energy.__name__ = "PQEnergy" if model == "pq" else "PHEnergy"
    _FUNCTIONS[model] = Energy
    return Energy


def _rotated(h, eri, kappa):
    """(U^T h U, (pq|rs) in the rotated orbitals), U = exp(kappa - kappa^T):
    the orbital rotation C -> C U as torch operations, so that autograd
    carries dE/dh and dE/d(pq|rs) on to kappa."""
    import torch
    U = torch.linalg.matrix_exp(kappa - kappa.transpose(0, 1))
    h2 = U.transpose(0, 1) @ h @ U
    v2 = torch.einsum('pqrs,pi,qj,rk,sl->ijkl', eri, U, U, U, U)
    return h2, v2


def pq_energy(h, eri, occ_of_pair, vir_of_pair, e_const=0.0, kappa=None, **opts):
    """Differentiable PQ total energy (torch.autograd): gradients w.r.t. h and
    (pq|rs) come from the Lambda equations (pq_gradient).  With kappa (an
    n_orb x n_orb tensor; only its antisymmetric part acts) the integrals are
    first rotated by U = exp(kappa - kappa^T), so that the energy is also
    differentiable in the orbitals: at kappa = 0 the gradient with respect to
    kappa is the orbital-rotation gradient dE/dkappa of pq_gradient."""
    if kappa is not None:
        h, eri = _rotated(h, eri, kappa)
    return _autograd_function("pq").apply(h, eri, occ_of_pair, vir_of_pair, e_const, opts)


def ph_energy(h, eri, occ_of_pair, vir_of_pair, e_const=0.0, kappa=None, **opts):
    """Differentiable PH total energy (torch.autograd) through ph_gradient;
    kappa as in pq_energy."""
    if kappa is not None:
        h, eri = _rotated(h, eri, kappa)
    return _autograd_function("ph").apply(h, eri, occ_of_pair, vir_of_pair, e_const, opts)


def release():
    return lib().ppq_release()
