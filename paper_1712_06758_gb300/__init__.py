"""Python binding of the GB300 SPDE sampler (libspde.so, C ABI in include/spde.h).

Argument marshalling only: every step of the sampling path runs in the CUDA
library.  Functions keep the C names (spde_grid_create, spde_mesh_attach,
spde_sample, ...); `Sampler` is a thin convenience wrapper over them.
Device buffers are torch CUDA tensors (their data_ptr is passed), host
buffers are NumPy arrays.  Importing this package does not build anything:
if libspde.so is missing it raises, so no path can silently fall back to a
CPU implementation.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libspde.so")

SPDE_OK, SPDE_EINVAL, SPDE_ENOMEM, SPDE_EMESH, SPDE_ENOCONV, SPDE_ETIMEOUT, SPDE_ECUDA, SPDE_EBUSY, SPDE_ECANCELED = range(9)
SPDE_PREC_MIXED, SPDE_PREC_FP64 = 0, 1
SPDE_SOLVER_MINRES, SPDE_SOLVER_SCHUR_CG = 0, 1
SPDE_OUT_LOGNORMAL, SPDE_OUT_GAUSSIAN, SPDE_OUT_GRID_GAUSSIAN, SPDE_OUT_F64 = 0, 1, 2, 16
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "EMESH", 4: "ENOCONV", 5: "ETIMEOUT", 6: "ECUDA", 7: "EBUSY",
                8: "ECANCELED"}


class spde_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_outer", ctypes.c_int), ("max_iter", ctypes.c_int), ("omega", ctypes.c_double),
                ("schur_c", ctypes.c_double), ("flux_diag", ctypes.c_double), ("check_every", ctypes.c_int),
                ("device", ctypes.c_int), ("use_graphs", ctypes.c_int), ("serve_budget_bytes", ctypes.c_int64),
                ("serve_max_batch", ctypes.c_int), ("solver", ctypes.c_int), ("sweep_planes", ctypes.c_int),
                ("coarse_fp16", ctypes.c_int), ("sweep_rows", ctypes.c_int)]


class spde_stats(ctypes.Structure):
    _fields_ = [("outer_iters", ctypes.c_int), ("inner_iters", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("setup_ms", ctypes.c_double), ("nnz", ctypes.c_int64)]


class spde_tuning(ctypes.Structure):
    _fields_ = [("omega", ctypes.c_double), ("inner_tol", ctypes.c_double), ("flux_diag", ctypes.c_double),
                ("sweep_planes", ctypes.c_int), ("ms_per_call", ctypes.c_double), ("default_ms", ctypes.c_double),
                ("evaluated", ctypes.c_int)]


class SpdeError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "spde_opts_init": [ctypes.POINTER(spde_opts)],
    "spde_grid_create": [ctypes.POINTER(_P), ctypes.POINTER(spde_opts)],
    "spde_level_add": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "spde_level_add_box": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)],
    "spde_mesh_attach": [_P, ctypes.c_int, ctypes.c_int64, _P, ctypes.c_int64, _P],
    "spde_sample": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                    ctypes.c_uint64, ctypes.c_int, _P, _P],
    "spde_check_wait_limit": [ctypes.c_int, _P],
    "spde_level_set_fields": [_P, ctypes.c_int, _P, _P],
    "spde_sample_fields": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _P, _P],
    "spde_sample_coupled": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                            ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int, _P, _P, _P],
    "spde_submit": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                    ctypes.c_uint64, ctypes.c_int, _P, ctypes.POINTER(ctypes.c_int64)],
    "spde_poll": [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                  ctypes.POINTER(ctypes.c_int)],
    "spde_cancel": [_P, ctypes.c_int64],
    "spde_query_footprint": [_P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "spde_get_stats": [_P, ctypes.POINTER(spde_stats)],
    "spde_wait": [_P],
    "spde_autotune": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.POINTER(spde_tuning)],
    "spde_level_set_tuning": [_P, ctypes.c_int, ctypes.POINTER(spde_tuning)],
    "spde_mesh_info": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)],
    "spde_mesh_copy_csr": [_P, ctypes.c_int, _P, _P, _P, _P],
    "spde_destroy": [_P],
    "spde_noise": [ctypes.c_int64, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double, _P, _P],
    "spde_noise_words": [ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint64, _P, _P],
    "spde_profile_enable": [_P, ctypes.c_int],
    "spde_profile_read": [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_int64),
                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)],
    "spde_apply": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P],
    "spde_apply_box": [ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                       _P, _P, _P],
    "spde_precond": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                     ctypes.POINTER(spde_opts), _P, _P, _P],
    "spde_precond_box": [ctypes.POINTER(ctypes.c_int), ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                         ctypes.POINTER(spde_opts), _P, _P, _P],
    "spde_precond_noalloc": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                             ctypes.POINTER(spde_opts), _P, _P, _P],
    "spde_precond_status": [_P],
    "spde_schur_apply": [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, _P, _P, _P],
    "spde_solve": [_P, ctypes.c_int, ctypes.c_int, ctypes.c_double, _P, _P, _P],
    "spde_project": [_P, ctypes.c_int, ctypes.c_int, _P, ctypes.c_int, _P, _P],
}
EXPORTED = sorted(list(_SIGS) + ["spde_last_error"])


def lib():
    """Load libspde.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libspde.so is not built: run `python -m paper_1712_06758_gb300.build` "
                              "(nvcc, sm_103a); there is no CPU fallback")
        lb = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(lb, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        lb.spde_last_error.argtypes = []
        lb.spde_last_error.restype = ctypes.c_char_p
        _lib = lb
    return _lib


def _check(status):
    if status != SPDE_OK:
        raise SpdeError(status, lib().spde_last_error().decode())
    return status


def _ptr(buf):
    """Raw pointer of a torch tensor (device) or a NumPy array (host)."""
    if buf is None:
        return None
    if isinstance(buf, np.ndarray):
        if not buf.flags.c_contiguous:
            raise ValueError("host array must be C-contiguous")
        return buf.ctypes.data
    if hasattr(buf, "data_ptr"):
        if not buf.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return buf.data_ptr()
    return int(buf)


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


# ---- C functions, same names -------------------------------------------------
def spde_opts_init():
    o = spde_opts()
    _check(lib().spde_opts_init(ctypes.byref(o)))
    return o


def spde_grid_create(opts=None):
    h = _P()
    _check(lib().spde_grid_create(ctypes.byref(h), ctypes.byref(opts) if opts is not None else None))
    return h


def spde_level_add(ctx, level, n, lo, hi):
    lo = (ctypes.c_double * 3)(*lo)
    hi = (ctypes.c_double * 3)(*hi)
    _check(lib().spde_level_add(ctx, level, n, lo, hi))


def spde_level_add_box(ctx, level, n, lo, hi):
    """n: cells per axis (three ints)."""
    n = (ctypes.c_int * 3)(*[int(v) for v in n])
    lo = (ctypes.c_double * 3)(*lo)
    hi = (ctypes.c_double * 3)(*hi)
    _check(lib().spde_level_add_box(ctx, level, n, lo, hi))


def spde_mesh_attach(ctx, level, xyz, tets):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    _check(lib().spde_mesh_attach(ctx, level, xyz.shape[0], _ptr(xyz), tets.shape[0], _ptr(tets)))


def spde_sample(ctx, level, nsamples, kappa, sigma, seed, first_sample, out_kind, out, stream=None):
    _check(lib().spde_sample(ctx, level, nsamples, kappa, sigma, seed, first_sample, out_kind, _ptr(out),
                             _stream(stream)))


def spde_level_set_fields(ctx, level, kappa_cells, sigma_cells):
    """kappa_cells, sigma_cells: the level's n^3 cell values (x fastest) on the host,
    or both None to clear.  The library reads n^3 values from each: pass arrays of
    exactly that length (Sampler.set_fields checks it)."""
    import numpy as np
    k = None if kappa_cells is None else np.ascontiguousarray(kappa_cells, dtype=np.float64).ravel()
    s = None if sigma_cells is None else np.ascontiguousarray(sigma_cells, dtype=np.float64).ravel()
    _check(lib().spde_level_set_fields(ctx, level, None if k is None else k.ctypes.data,
                                       None if s is None else s.ctypes.data))


def spde_check_wait_limit(device=0):
    """Runs the bounded-wait self-check; returns the time the probe's wait took (ms)."""
    ms = ctypes.c_double(0.0)
    _check(lib().spde_check_wait_limit(device, ctypes.byref(ms)))
    return ms.value


def spde_sample_fields(ctx, level, nsamples, seed, first_sample, out_kind, out, stream=None):
    _check(lib().spde_sample_fields(ctx, level, nsamples, seed, first_sample, out_kind, _ptr(out), _stream(stream)))


def spde_sample_coupled(ctx, fine_level, coarse_level, nsamples, kappa, sigma, seed, first_sample, out_kind,
                        out_fine, out_coarse, stream=None):
    _check(lib().spde_sample_coupled(ctx, fine_level, coarse_level, nsamples, kappa, sigma, seed, first_sample,
                                     out_kind, _ptr(out_fine), _ptr(out_coarse), _stream(stream)))


def spde_submit(ctx, level, nsamples, kappa, sigma, seed, first_sample, out_kind, out):
    rid = ctypes.c_int64()
    _check(lib().spde_submit(ctx, level, nsamples, kappa, sigma, seed, first_sample, out_kind, _ptr(out),
                             ctypes.byref(rid)))
    return rid.value


def spde_poll(ctx, request):
    """(done, latency_ms, status) of a request; a done request is forgotten."""
    done, lat, res = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    _check(lib().spde_poll(ctx, request, ctypes.byref(done), ctypes.byref(lat), ctypes.byref(res)))
    return bool(done.value), lat.value, res.value


def spde_cancel(ctx, request):
    _check(lib().spde_cancel(ctx, request))


def spde_query_footprint(ctx, level, nsamples):
    b = ctypes.c_int64()
    _check(lib().spde_query_footprint(ctx, level, nsamples, ctypes.byref(b)))
    return b.value


def spde_get_stats(ctx):
    s = spde_stats()
    _check(lib().spde_get_stats(ctx, ctypes.byref(s)))
    return {k: getattr(s, k) for k, _ in spde_stats._fields_}


def spde_wait(ctx):
    """Waits for the context's calls; raises SpdeError with their worst outcome."""
    _check(lib().spde_wait(ctx))


def spde_autotune(ctx, level, nsamples, kappa, sigma):
    """Runs the autotuner on `level`; returns the chosen schedule as a dict (kept on the level)."""
    t = spde_tuning()
    _check(lib().spde_autotune(ctx, level, nsamples, kappa, sigma, ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in spde_tuning._fields_}


def spde_level_set_tuning(ctx, level, tuning):
    """Puts a schedule (a dict with omega, inner_tol, flux_diag, sweep_planes) on `level`; None clears it."""
    if tuning is None:
        _check(lib().spde_level_set_tuning(ctx, level, None))
        return
    t = spde_tuning()
    for k in ("omega", "inner_tol", "flux_diag", "sweep_planes"):
        setattr(t, k, tuning[k])
    _check(lib().spde_level_set_tuning(ctx, level, ctypes.byref(t)))


def spde_mesh_info(ctx, level):
    nt, nz = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().spde_mesh_info(ctx, level, ctypes.byref(nt), ctypes.byref(nz)))
    return nt.value, nz.value


def spde_mesh_copy_csr(ctx, level):
    nt, nz = spde_mesh_info(ctx, level)
    rowptr = np.zeros(nt + 1, dtype=np.int64)
    col = np.zeros(max(nz, 1), dtype=np.int32)
    g = np.zeros(max(nz, 1), dtype=np.float64)
    vol = np.zeros(nt, dtype=np.float64)
    _check(lib().spde_mesh_copy_csr(ctx, level, _ptr(rowptr), _ptr(col), _ptr(g), _ptr(vol)))
    return rowptr, col[:nz], g[:nz], vol


def spde_profile_enable(ctx, enable=True):
    _check(lib().spde_profile_enable(ctx, 1 if enable else 0))


PROF_CLASSES = 18


def spde_profile_read(ctx, k):
    name = ctypes.c_char_p()
    nl, ms, by = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(lib().spde_profile_read(ctx, k, ctypes.byref(name), ctypes.byref(nl), ctypes.byref(ms), ctypes.byref(by)))
    return {"name": name.value.decode(), "launches": nl.value, "ms": ms.value, "bytes": by.value}


def spde_profile(ctx):
    """All kernel classes' counters as a list of dicts."""
    return [spde_profile_read(ctx, k) for k in range(PROF_CLASSES)]


def spde_last_error():
    return lib().spde_last_error().decode()


def spde_destroy(ctx):
    _check(lib().spde_destroy(ctx))


def spde_noise(ncells, nsamples, seed, first_sample, scale, out, stream=None):
    _check(lib().spde_noise(ncells, nsamples, seed, first_sample, scale, _ptr(out), _stream(stream)))


def spde_noise_words(npairs, seed, sample, out, stream=None):
    _check(lib().spde_noise_words(npairs, seed, sample, _ptr(out), _stream(stream)))


def spde_apply(n, h, kappa, nsamples, prec, x, y, stream=None):
    _check(lib().spde_apply(n, h, kappa, nsamples, prec, _ptr(x), _ptr(y), _stream(stream)))


def spde_apply_box(n, h, kappa, nsamples, prec, x, y, stream=None):
    n = (ctypes.c_int * 3)(*[int(v) for v in n])
    _check(lib().spde_apply_box(n, h, kappa, nsamples, prec, _ptr(x), _ptr(y), _stream(stream)))


def spde_precond_box(n, h, kappa, nsamples, prec, r, z, opts=None, stream=None):
    n = (ctypes.c_int * 3)(*[int(v) for v in n])
    _check(lib().spde_precond_box(n, h, kappa, nsamples, prec, ctypes.byref(opts) if opts is not None else None,
                                  _ptr(r), _ptr(z), _stream(stream)))


def spde_precond(n, h, kappa, nsamples, prec, r, z, opts=None, stream=None):
    _check(lib().spde_precond(n, h, kappa, nsamples, prec, ctypes.byref(opts) if opts is not None else None,
                              _ptr(r), _ptr(z), _stream(stream)))


def spde_precond_noalloc(n, h, kappa, nsamples, prec, r, z, opts=None, stream=None):
    """spde_precond without any device allocation (static 16 MiB scratch).

    For callers that may not allocate device memory: see include/spde.h.
    """
    _check(lib().spde_precond_noalloc(n, h, kappa, nsamples, prec,
                                      ctypes.byref(opts) if opts is not None else None, _ptr(r), _ptr(z),
                                      _stream(stream)))


def spde_precond_status(stream=None):
    """Raises SpdeError(SPDE_ETIMEOUT) when the last step-level preconditioner call timed out."""
    _check(lib().spde_precond_status(_stream(stream)))


def spde_schur_apply(n, h, kappa, nsamples, prec, x, y, stream=None):
    _check(lib().spde_schur_apply(n, h, kappa, nsamples, prec, _ptr(x), _ptr(y), _stream(stream)))


def spde_solve(ctx, level, nsamples, kappa, rhs, x, stream=None):
    _check(lib().spde_solve(ctx, level, nsamples, kappa, _ptr(rhs), _ptr(x), _stream(stream)))


def spde_project(ctx, level, nsamples, theta, out_kind, out, stream=None):
    _check(lib().spde_project(ctx, level, nsamples, _ptr(theta), out_kind, _ptr(out), _stream(stream)))


class Sampler:
    """One context: embedding grids by level, their meshes, and sampling."""

    def __init__(self, precision=SPDE_PREC_MIXED, **opts):
        o = spde_opts_init()
        o.precision = precision
        for k, v in opts.items():
            setattr(o, k, v)
        self.opts = o
        self.ctx = spde_grid_create(o)
        self.levels = {}

    def add_level(self, level, n, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0)):
        """n: cells per axis, one int (a cube) or three (a box of cubic cells)."""
        if isinstance(n, (int, np.integer)):
            spde_level_add(self.ctx, level, int(n), lo, hi)
            cells = int(n) ** 3
        else:
            spde_level_add_box(self.ctx, level, n, lo, hi)
            cells = int(n[0]) * int(n[1]) * int(n[2])
        self.levels[level] = (cells, tuple(lo), tuple(hi))

    def attach_mesh(self, level, xyz, tets):
        spde_mesh_attach(self.ctx, level, xyz, tets)

    def ntets(self, level):
        return spde_mesh_info(self.ctx, level)[0]

    def sample(self, level, nsamples, kappa, sigma, seed, first_sample=0, out_kind=SPDE_OUT_LOGNORMAL, out=None,
               stream=None, wait=True):
        """spde_sample; with wait (the default) also spde_wait, so the outcome is raised here."""
        import torch
        if out is None:
            cells = self.levels[level][0]
            per = cells if (out_kind & 15) == SPDE_OUT_GRID_GAUSSIAN else self.ntets(level)
            dt = torch.float64 if out_kind & SPDE_OUT_F64 else torch.float32
            out = torch.empty((nsamples, per), dtype=dt, device="cuda")
        spde_sample(self.ctx, level, nsamples, kappa, sigma, seed, first_sample, out_kind, out, stream)
        if wait:
            spde_wait(self.ctx)
        return out

    def set_fields(self, level, kappa_cells, sigma_cells):
        import numpy as np
        cells = self.levels[level][0]
        for a in (kappa_cells, sigma_cells):
            if a is not None and np.size(a) != cells:
                raise ValueError("fields of level %d need %d cell values" % (level, cells))
        spde_level_set_fields(self.ctx, level, kappa_cells, sigma_cells)

    def sample_fields(self, level, nsamples, seed, first_sample=0, out_kind=SPDE_OUT_LOGNORMAL, out=None,
                      stream=None, wait=True):
        import torch
        if out is None:
            cells = self.levels[level][0]
            per = cells if (out_kind & 15) == SPDE_OUT_GRID_GAUSSIAN else self.ntets(level)
            dt = torch.float64 if out_kind & SPDE_OUT_F64 else torch.float32
            out = torch.empty((nsamples, per), dtype=dt, device="cuda")
        spde_sample_fields(self.ctx, level, nsamples, seed, first_sample, out_kind, out, stream)
        if wait:
            spde_wait(self.ctx)
        return out

    def stats(self):
        return spde_get_stats(self.ctx)

    def close(self):
        if self.ctx:
            spde_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
