"""GB300-native Sakurai-Sugiura eigensolver with shifted CG for the Hermitian
Wilson fermion matrix (arXiv:1004.0292), Python binding.

This module only marshals arguments to the C ABI of ``lib/libssqcd.so``
(declared in ``include/ssqcd.h``); every step of the computation runs in the
library's CUDA kernels.  Arrays may be numpy (host) or torch CUDA tensors
(device); complex data are complex128.  If the library has not been built,
importing works but every call raises ``RuntimeError`` -- there is no CPU
fallback.

Names follow the C ABI without the ``ssqcd_`` prefix:
``create_lattice``, ``upload_gauge``, ``apply_H``, ``apply_H_mixed``,
``contour``, ``shifted_cg``, ``moments``, ``ss_solve``, ``ss_eigpairs``,
``small_eigh``, ``kernel_launches``.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "OK", "ERR_ARG", "ERR_OOM", "ERR_BREAKDOWN", "ERR_NOCONV", "ERR_CUDA",
    "FP64", "MIXED", "MIXED_F32LINKS", "FP64_SHIFT32", "FP64_DFSHIFT", "DF", "EXTRACT_RR", "EXTRACT_HANKEL", "PATH_LINES", "PATH_CIRCLE", "SsqcdError",
    "library_path", "lib", "Server", "time_stencil", "create_lattice", "upload_gauge", "apply_H", "apply_H_mixed",
    "contour", "shifted_cg", "moments", "moments_noalloc", "ss_solve", "ss_solve_windows", "ss_eigpairs", "small_eigh",
    "kernel_launches", "set_kernel_timing", "set_stencil_variant", "stencil_tuning", "Lattice", "Result", "Opts", "Stats",
]

OK, ERR_ARG, ERR_OOM, ERR_BREAKDOWN, ERR_NOCONV, ERR_CUDA = 0, 1, 2, 3, 4, 5
FP64, MIXED, MIXED_F32LINKS, FP64_SHIFT32, FP64_DFSHIFT, DF = 0, 1, 2, 3, 4, 5
EXTRACT_RR, EXTRACT_HANKEL = 0, 1
PATH_LINES, PATH_CIRCLE = 0, 1

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "lib", "libssqcd.so")


class SsqcdError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"ssqcd error {code}: {msg}")
        self.code = code


class Opts(C.Structure):
    _fields_ = [
        ("path", C.c_int), ("beta", C.c_double), ("nprime", C.c_int), ("tol", C.c_double),
        ("sigma", C.c_double), ("max_iter", C.c_int), ("rank_tol", C.c_double),
        ("sources", C.c_void_p), ("sources_on_device", C.c_int), ("reliable_every", C.c_int),
        ("windows", C.c_int), ("extract", C.c_int), ("hankel_tol", C.c_double), ("refine", C.c_int),
        ("basis", C.c_int), ("basis_max_bytes", C.c_double), ("source_block", C.c_int),
        ("converged_tol", C.c_double), ("block_streams", C.c_int),
    ]


class Stats(C.Structure):
    _fields_ = [
        ("iterations", C.c_int), ("max_shift_iters", C.c_int), ("matvecs_rr", C.c_int),
        ("rank", C.c_int), ("n_ritz", C.c_int), ("n_accepted", C.c_int), ("reliable_updates", C.c_int),
        ("ms_cg", C.c_double), ("ms_moments", C.c_double), ("ms_rr", C.c_double),
        ("gamma", C.c_double), ("rho", C.c_double), ("points", C.c_int), ("shift_updates", C.c_longlong),
        ("timed", C.c_int), ("launches_update", C.c_int), ("ms_k_stencil", C.c_double),
        ("ms_k_seed", C.c_double), ("ms_k_scalars", C.c_double), ("ms_k_update", C.c_double),
        ("timed_shift_updates", C.c_longlong), ("basis", C.c_int), ("basis_bytes", C.c_double),
        ("n_converged", C.c_int), ("real_moments", C.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    """The loaded shared library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_1004_0292_gb300.build` "
                           "(no CPU fallback exists)")
    L = C.CDLL(path)
    vp, i, d = C.c_void_p, C.c_int, C.c_double
    sig = {
        "ssqcd_create_lattice": (i, [vp, d, i, i, vp, vp]),
        "ssqcd_upload_gauge": (i, [vp, vp, i]),
        "ssqcd_apply_H": (i, [vp, vp, vp, i, i]),
        "ssqcd_apply_H_mixed": (i, [vp, vp, vp, i, i]),
        "ssqcd_server_create": (i, [C.c_size_t, vp]),
        "ssqcd_server_submit": (i, [vp, vp, vp, i, i, i, vp, vp]),
        "ssqcd_server_submit_windows": (i, [vp, vp, i, vp, i, i, i, vp, vp]),
        "ssqcd_server_progress": (i, [vp, i, vp]),
        "ssqcd_server_status": (i, [vp, C.c_longlong, vp, vp]),
        "ssqcd_server_take": (i, [vp, C.c_longlong, vp]),
        "ssqcd_server_counts": (i, [vp, vp, vp, vp]),
        "ssqcd_server_deferred": (i, [vp, vp]),
        "ssqcd_server_request_bytes": (i, [vp, C.c_longlong, vp]),
        "ssqcd_server_destroy": (None, [vp]),
        "ssqcd_lattice_destroy": (None, [vp]),
        "ssqcd_contour": (i, [i, d, d, d, i, vp, vp]),
        "ssqcd_shifted_cg": (i, [vp, i, vp, i, vp, i, d, d, i, i, i, vp, vp, vp, vp]),
        "ssqcd_moments": (i, [vp, i, i, i, vp, vp, vp, vp, i]),
        "ssqcd_default_opts": (None, [vp]),
        "ssqcd_ss_solve": (i, [vp, vp, i, i, i, vp, vp]),
        "ssqcd_ss_solve_windows": (i, [vp, i, vp, i, i, i, vp, vp]),
        "ssqcd_ss_moments": (i, [vp, vp, i, i, i, vp, vp, i, vp]),
        "ssqcd_ss_eigpairs": (i, [vp, vp, vp, vp, vp, vp]),
        "ssqcd_result_destroy": (None, [vp]),
        "ssqcd_small_eigh": (i, [i, vp, vp, vp]),
        "ssqcd_last_error": (C.c_char_p, []),
        "ssqcd_kernel_launches": (C.c_longlong, []),
        "ssqcd_time_stencil": (i, [vp, i, i, vp]),
        "ssqcd_set_kernel_timing": (i, [i]),
        "ssqcd_set_stencil_variant": (i, [i]),
        "ssqcd_stencil_tuning": (i, [vp, i, vp, vp]),
        "ssqcd_moments_noalloc": (i, [i, i, i, C.c_longlong, vp, vp, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def _check(code):
    if code != OK:
        raise SsqcdError(code, lib().ssqcd_last_error().decode())


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype=np.complex128):
    """(pointer, on_device, keepalive) for a numpy array or torch CUDA tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        if not x.is_cuda or not x.is_contiguous():
            raise ValueError("torch tensors must be contiguous CUDA tensors")
        return x.data_ptr(), 1, x
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream  # torch.cuda.Stream


class Lattice:
    """Owning handle of a ``ssqcd_lattice``."""

    def __init__(self, handle, dims, kappa, bc_t, precision):
        self.handle = handle
        self.dims = tuple(dims)
        self.kappa = kappa
        self.bc_t = bc_t
        self.precision = precision
        self.V = int(np.prod(dims))
        self.n = 12 * self.V

    def __del__(self):
        if getattr(self, "handle", None):
            lib().ssqcd_lattice_destroy(self.handle)
            self.handle = None


class Result:
    """Owning handle of a ``ssqcd_result`` plus the status of the solve."""

    def __init__(self, handle, status, lattice, error=""):
        self.handle = handle
        self.status = status
        self.lattice = lattice
        self.error = error

    def __del__(self):
        if getattr(self, "handle", None):
            lib().ssqcd_result_destroy(self.handle)
            self.handle = None


def create_lattice(dims, kappa, bc_t=-1, precision=FP64, stream=None) -> Lattice:
    d = (C.c_int * 4)(*[int(x) for x in dims])
    h = C.c_void_p()
    _check(lib().ssqcd_create_lattice(d, float(kappa), int(bc_t), int(precision), _stream_handle(stream), C.byref(h)))
    return Lattice(h, dims, kappa, bc_t, precision)


def upload_gauge(lat: Lattice, U):
    p, dev, keep = _ptr(U)
    _check(lib().ssqcd_upload_gauge(lat.handle, p, dev))


def _apply(fn, lat, psi):
    nrhs = int(np.prod(psi.shape)) // lat.n
    if _is_torch(psi):
        import torch
        out = torch.empty_like(psi)
    else:
        out = np.empty(psi.shape, dtype=np.complex128)
    pi, dev, keep = _ptr(psi)
    po, _, keep2 = _ptr(out)
    _check(fn(lat.handle, pi, po, nrhs, dev))
    return out if _is_torch(psi) else keep2.reshape(psi.shape)


def apply_H(lat: Lattice, psi):
    """A psi for psi of shape (..., V, 4, 3), complex128 (numpy or CUDA tensor)."""
    return _apply(lib().ssqcd_apply_H, lat, psi)


def apply_H_mixed(lat: Lattice, psi):
    """A psi with the mixed path's FP32 / FP16-link stencil."""
    return _apply(lib().ssqcd_apply_H_mixed, lat, psi)


def contour(path, gamma, rho, beta, N):
    z = np.empty(N, dtype=np.complex128)
    w = np.empty(N, dtype=np.complex128)
    _check(lib().ssqcd_contour(int(path), float(gamma), float(rho), float(beta), int(N), z.ctypes.data, w.ctypes.data))
    return z, w


def shifted_cg(lat: Lattice, z, v, sigma=0.0, tol=1e-12, max_iter=100000, precision=FP64, reliable_every=0,
               want_y=True):
    """Solve (z_j I - A) y = v_l for all shifts z (N,) and sources v (L, V, 4, 3).

    Returns (status, y (L, N, V, 4, 3) or None, iters (L, N), xi (L, N), seed_iters)."""
    z = np.ascontiguousarray(z, dtype=np.complex128)
    N = len(z)
    L = int(np.prod(v.shape)) // lat.n
    pv, dev, keep = _ptr(v)
    if dev:
        import torch
        y = torch.empty((L, N, lat.V, 4, 3), dtype=torch.complex128, device=v.device) if want_y else None
        iters = torch.empty((L, N), dtype=torch.int32, device=v.device)
        xi = torch.empty((L, N), dtype=torch.complex128, device=v.device)
    else:
        y = np.empty((L, N, lat.V, 4, 3), dtype=np.complex128) if want_y else None
        iters = np.empty((L, N), dtype=np.int32)
        xi = np.empty((L, N), dtype=np.complex128)
    si = C.c_int(0)
    py = None if y is None else (y.data_ptr() if dev else y.ctypes.data)
    pit = iters.data_ptr() if dev else iters.ctypes.data
    pxi = xi.data_ptr() if dev else xi.ctypes.data
    code = lib().ssqcd_shifted_cg(lat.handle, N, z.ctypes.data, L, pv, dev, float(sigma), float(tol), int(max_iter),
                                  int(precision), int(reliable_every), py, pit, pxi, C.byref(si))
    if code not in (OK, ERR_BREAKDOWN, ERR_NOCONV):
        _check(code)
    return code, y, iters, xi, si.value


def moments(lat: Lattice, w, zeta, y, M):
    """s_hat (L, M, V, 4, 3) from y (L, N, V, 4, 3) (Eq. 2)."""
    w = np.ascontiguousarray(w, dtype=np.complex128)
    zeta = np.ascontiguousarray(zeta, dtype=np.complex128)
    N = len(w)
    L = int(np.prod(y.shape)) // (lat.n * N)
    py, dev, keep = _ptr(y)
    if dev:
        import torch
        s = torch.empty((L, M, lat.V, 4, 3), dtype=torch.complex128, device=y.device)
        ps = s.data_ptr()
    else:
        s = np.empty((L, M, lat.V, 4, 3), dtype=np.complex128)
        ps = s.ctypes.data
    _check(lib().ssqcd_moments(lat.handle, N, int(M), L, w.ctypes.data, zeta.ctypes.data, py, ps, dev))
    return s


def moments_noalloc(w, zeta, y, M, stream=None):
    """Allocation-free moments: y (L, N, ...) complex128 CUDA tensor ->
    s_hat (L, M, ...) (Eq. 2).  Uses the library's fixed device scratch
    (N * M <= 4096); returns a new tensor allocated here by torch, the
    library itself allocates nothing.  Raises ValueError when y, w and zeta
    do not agree on N."""
    import torch
    w = np.ascontiguousarray(w, dtype=np.complex128)
    zeta = np.ascontiguousarray(zeta, dtype=np.complex128)
    N = len(w)
    if not (_is_torch(y) and y.is_cuda and y.is_contiguous() and y.dtype == torch.complex128):
        raise ValueError("y must be a contiguous complex128 CUDA tensor")
    if zeta.shape != (N,) or w.shape != (N,):
        raise ValueError("w and zeta must be 1-D arrays of the same length N")
    if y.dim() < 3 or y.shape[1] != N:
        raise ValueError("y must have shape (L, N, ...) with N = len(w)")
    L = y.shape[0]
    n = int(np.prod(y.shape[2:]))
    if L < 1 or n < 1 or y.numel() != L * N * n:
        raise ValueError("y must be a non-empty (L, N, ...) tensor")
    s = torch.empty((L, M) + tuple(y.shape[2:]), dtype=torch.complex128, device=y.device)
    st = _stream_handle(stream if stream is not None else torch.cuda.current_stream())
    _check(lib().ssqcd_moments_noalloc(N, int(M), L, n, w.ctypes.data, zeta.ctypes.data, y.data_ptr(),
                                       s.data_ptr(), st))
    return s


def _solve_opts(lat, sources, beta, nprime, tol, sigma, max_iter, rank_tol, path, reliable_every, windows, extract,
                hankel_tol, refine, basis, basis_max_bytes, source_block, block_streams=1):
    L = int(np.prod(sources.shape)) // lat.n
    o = Opts()
    lib().ssqcd_default_opts(C.byref(o))
    ps, dev, keep = _ptr(sources)
    o.path, o.beta, o.nprime, o.tol, o.sigma = int(path), float(beta), int(nprime), float(tol), float(sigma)
    o.max_iter, o.rank_tol, o.sources, o.sources_on_device = int(max_iter), float(rank_tol), ps, dev
    o.reliable_every = int(reliable_every)
    o.windows = int(windows)
    o.extract, o.hankel_tol, o.refine = int(extract), float(hankel_tol), int(refine)
    o.basis, o.basis_max_bytes = int(basis), float(basis_max_bytes)
    o.source_block = int(source_block)
    o.block_streams = int(block_streams)
    return L, o, keep


def ss_solve(lat: Lattice, interval, N, M, sources, beta=0.3, nprime=0, tol=1e-12, sigma=0.0, max_iter=100000,
             rank_tol=1e-14, path=PATH_LINES, reliable_every=0, windows=1, extract=0,
             hankel_tol=1e-12, refine=0, basis=1, basis_max_bytes=0.0, source_block=0, block_streams=1) -> Result:
    """Run the solver; returns a Result (check ``status``).  ``basis`` / ``basis_max_bytes``: moments
    from the stored seed residuals (FP64 and DF lattices; see ssqcd_opts); ``source_block``: sources
    per shifted-CG run; ``block_streams``: source blocks whose runs proceed at once."""
    L, o, keep = _solve_opts(lat, sources, beta, nprime, tol, sigma, max_iter, rank_tol, path, reliable_every,
                             windows, extract, hankel_tol, refine, basis, basis_max_bytes, source_block,
                             block_streams)
    iv = (C.c_double * 2)(float(interval[0]), float(interval[1]))
    h = C.c_void_p()
    code = lib().ssqcd_ss_solve(lat.handle, iv, int(N), int(M), L, C.byref(o), C.byref(h))
    if not h.value:
        _check(code)
    err = lib().ssqcd_last_error().decode() if code != OK else ""
    return Result(h, code, lat, err)


def ss_solve_windows(lat: Lattice, intervals, N, M, sources, beta=0.3, nprime=0, tol=1e-12, sigma=0.0,
                     max_iter=100000, rank_tol=1e-14, path=PATH_LINES, extract=0, hankel_tol=1e-12, refine=0,
                     basis=1, basis_max_bytes=0.0, source_block=0, block_streams=1) -> Result:
    """Several windows [(a_k, b_k), ...] out of one shifted-CG run (ssqcd_ss_solve_windows)."""
    iv_list = [float(x) for ab in intervals for x in ab]
    K = len(iv_list) // 2
    L, o, keep = _solve_opts(lat, sources, beta, nprime, tol, sigma, max_iter, rank_tol, path, 0, 1, extract,
                             hankel_tol, refine, basis, basis_max_bytes, source_block, block_streams)
    iv = (C.c_double * (2 * K))(*iv_list)
    h = C.c_void_p()
    code = lib().ssqcd_ss_solve_windows(lat.handle, K, iv, int(N), int(M), L, C.byref(o), C.byref(h))
    if not h.value:
        _check(code)
    err = lib().ssqcd_last_error().decode() if code != OK else ""
    return Result(h, code, lat, err)


def ss_moments(lat: Lattice, interval, N, M, sources, beta=0.3, nprime=0, tol=1e-12, sigma=0.0, max_iter=100000,
               path=PATH_LINES, basis=1, basis_max_bytes=0.0):
    """The moments s_hat (L, M, V, 4, 3) of the first window of ss_solve with these options (Eq. 2) and the
    shifted-CG stats dict."""
    L = int(np.prod(sources.shape)) // lat.n
    o = Opts()
    lib().ssqcd_default_opts(C.byref(o))
    ps, dev, keep = _ptr(sources)
    o.path, o.beta, o.nprime, o.tol, o.sigma = int(path), float(beta), int(nprime), float(tol), float(sigma)
    o.max_iter, o.sources, o.sources_on_device = int(max_iter), ps, dev
    o.basis, o.basis_max_bytes = int(basis), float(basis_max_bytes)
    iv = (C.c_double * 2)(float(interval[0]), float(interval[1]))
    s = np.empty((L, int(M), lat.V, 4, 3), dtype=np.complex128)
    st = Stats()
    _check(lib().ssqcd_ss_moments(lat.handle, iv, int(N), int(M), L, C.byref(o), s.ctypes.data, 0, C.byref(st)))
    return s, st.as_dict()


def ss_eigpairs(res: Result, want_vectors=True):
    """(evals, evecs (count, V, 4, 3) or None, residuals, stats dict)."""
    cnt = C.c_int(0)
    st = Stats()
    _check(lib().ssqcd_ss_eigpairs(res.handle, C.byref(cnt), None, None, None, C.byref(st)))
    k = cnt.value
    ev = np.empty(k, dtype=np.float64)
    rs = np.empty(k, dtype=np.float64)
    vec = np.empty((k, res.lattice.V, 4, 3), dtype=np.complex128) if want_vectors else None
    _check(lib().ssqcd_ss_eigpairs(res.handle, C.byref(cnt), ev.ctypes.data if k else None,
                                   vec.ctypes.data if (want_vectors and k) else None,
                                   rs.ctypes.data if k else None, C.byref(st)))
    if k == 0:
        # still fill stats
        pass
    return ev, vec, rs, st.as_dict()


class Server:
    """Request scheduler (ssqcd_server_*): continuous batching of solves."""

    QUEUED, RUNNING, DONE, FAILED = 0, 1, 2, 3

    def __init__(self, memory_budget=0):
        h = C.c_void_p()
        _check(lib().ssqcd_server_create(C.c_size_t(int(memory_budget)), C.byref(h)))
        self.handle = h
        self._lats = {}

    def submit(self, lat: Lattice, interval, N, M, sources, beta=0.3, nprime=0, tol=1e-12, sigma=0.0,
               max_iter=100000, rank_tol=1e-14, path=PATH_LINES, windows=1, extract=0, hankel_tol=1e-12, refine=0,
               basis=1, basis_max_bytes=0.0):
        L = int(np.prod(sources.shape)) // lat.n
        o = Opts()
        lib().ssqcd_default_opts(C.byref(o))
        ps, dev, keep = _ptr(sources)
        o.path, o.beta, o.nprime, o.tol, o.sigma = int(path), float(beta), int(nprime), float(tol), float(sigma)
        o.max_iter, o.rank_tol, o.sources, o.sources_on_device = int(max_iter), float(rank_tol), ps, dev
        o.windows, o.extract, o.hankel_tol, o.refine = int(windows), int(extract), float(hankel_tol), int(refine)
        o.basis, o.basis_max_bytes = int(basis), float(basis_max_bytes)
        iv = (C.c_double * 2)(float(interval[0]), float(interval[1]))
        rid = C.c_longlong(0)
        _check(lib().ssqcd_server_submit(self.handle, lat.handle, iv, int(N), int(M), L, C.byref(o), C.byref(rid)))
        self._lats[rid.value] = lat
        return rid.value

    def submit_windows(self, lat: Lattice, intervals, N, M, sources, beta=0.3, nprime=0, tol=1e-12, sigma=0.0,
                       max_iter=100000, rank_tol=1e-14, path=PATH_LINES, extract=0, hankel_tol=1e-12, refine=0,
                       basis=1, basis_max_bytes=0.0, source_block=0):
        iv_list = [float(x) for ab in intervals for x in ab]
        K = len(iv_list) // 2
        L, o, keep = _solve_opts(lat, sources, beta, nprime, tol, sigma, max_iter, rank_tol, path, 0, 1, extract,
                                 hankel_tol, refine, basis, basis_max_bytes, source_block)
        iv = (C.c_double * (2 * K))(*iv_list)
        rid = C.c_longlong(0)
        _check(lib().ssqcd_server_submit_windows(self.handle, lat.handle, K, iv, int(N), int(M), L, C.byref(o),
                                                 C.byref(rid)))
        self._lats[rid.value] = lat
        return rid.value

    def progress(self, wait=False) -> int:
        n = C.c_int(0)
        _check(lib().ssqcd_server_progress(self.handle, 1 if wait else 0, C.byref(n)))
        return n.value

    def status(self, rid):
        st = C.c_int(0)
        ms = C.c_double(0.0)
        _check(lib().ssqcd_server_status(self.handle, C.c_longlong(rid), C.byref(st), C.byref(ms)))
        return st.value, ms.value

    def request_bytes(self, rid) -> int:
        b = C.c_size_t(0)
        _check(lib().ssqcd_server_request_bytes(self.handle, C.c_longlong(rid), C.byref(b)))
        return b.value

    def counts(self):
        q, r, f = C.c_int(0), C.c_int(0), C.c_int(0)
        _check(lib().ssqcd_server_counts(self.handle, C.byref(q), C.byref(r), C.byref(f)))
        return q.value, r.value, f.value

    def deferred(self) -> int:
        """Requests that waited at the head of the queue for memory."""
        n = C.c_longlong(0)
        _check(lib().ssqcd_server_deferred(self.handle, C.byref(n)))
        return n.value

    def take(self, rid) -> "Result":
        h = C.c_void_p()
        code = lib().ssqcd_server_take(self.handle, C.c_longlong(rid), C.byref(h))
        lat = self._lats.pop(rid, None)
        err = lib().ssqcd_last_error().decode() if code != OK else ""
        if not h.value:
            _check(code)
        return Result(h, code, lat, err)

    def close(self):
        if self.handle is not None and self.handle.value:
            lib().ssqcd_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def small_eigh(a):
    """Eigen-decomposition of a small complex Hermitian matrix (host C++)."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    m = a.shape[0]
    ev = np.empty(m, dtype=np.float64)
    vec = np.empty((m, m), dtype=np.complex128)
    _check(lib().ssqcd_small_eigh(m, a.ctypes.data, ev.ctypes.data, vec.ctypes.data))
    return ev, vec


def time_stencil(lat: Lattice, nrhs: int, reps: int = 20) -> float:
    """Mean device ms of one stencil application to nrhs fields (the lattice's precision)."""
    ms = C.c_double(0.0)
    _check(lib().ssqcd_time_stencil(lat.handle, int(nrhs), int(reps), C.byref(ms)))
    return ms.value


def set_stencil_variant(variant: int):
    """Force FP32 stencil variant 0..7, or -1 to tune per lattice size and rhs count."""
    _check(lib().ssqcd_set_stencil_variant(int(variant)))


def stencil_tuning(lat: Lattice, nrhs: int):
    """(chosen variant, microseconds per application of each variant) recorded for lat and nrhs."""
    v = C.c_int(0)
    us = (C.c_double * 8)()
    _check(lib().ssqcd_stencil_tuning(lat.handle, int(nrhs), C.byref(v), us))
    return v.value, list(us)


def kernel_launches() -> int:
    return int(lib().ssqcd_kernel_launches())


def set_kernel_timing(enable: bool):
    _check(lib().ssqcd_set_kernel_timing(1 if enable else 0))
