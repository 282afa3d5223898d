"""ctypes binding of the C-ABI in include/hdg.h (argument marshalling only).

Every function of the C-ABI has a Python counterpart of the same name. Array arguments are
torch CUDA float64 tensors in the exchange layouts of hdg.h (nodal values on the canonical
mesh); they are passed by device pointer, on the context's stream. Failures raise HdgError
with the library's status and message. Nothing here computes any part of the method.
"""
import ctypes
import os

from .build import LIB, build_library

_lib = None


class HdgError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        msg = _lib.hdg_status_string(status).decode() if _lib else str(status)
        detail = _lib.hdg_last_error().decode() if _lib else ''
        super().__init__(f'{where}: {msg} ({detail})' if detail else f'{where}: {msg}')


HDG_OK, HDG_ERR_INVALID_ARG, HDG_ERR_CUDA, HDG_ERR_OOM, HDG_ERR_NOT_CONVERGED, HDG_ERR_NUMERIC, \
    HDG_ERR_UNSUPPORTED, HDG_ERR_TIMEOUT = range(8)
TABLEAUS = {'ARS222': 0, 'ARS343': 1, 'IMEX_EULER': 2, 'SSP2_332': 3, 'SSP3_433': 4}
PRECISIONS = {'FP64': 0, 'MIXED': 1}


class hdg_mesh_desc(ctypes.Structure):
    _fields_ = [('n', ctypes.c_int), ('Lx', ctypes.c_double), ('Ly', ctypes.c_double),
                ('periodic_x', ctypes.c_int), ('periodic_y', ctypes.c_int)]


class hdg_params(ctypes.Structure):
    _fields_ = [('k', ctypes.c_int), ('alpha', ctypes.c_double), ('tau', ctypes.c_double),
                ('delta_up', ctypes.c_double), ('tableau', ctypes.c_int), ('dt', ctypes.c_double),
                ('n_richardson', ctypes.c_int), ('richardson_rtol', ctypes.c_double),
                ('richardson_max', ctypes.c_int), ('trace_rtol', ctypes.c_double),
                ('stepI_rtol', ctypes.c_double), ('max_iters', ctypes.c_int),
                ('stage_krylov', ctypes.c_int), ('inner_stepI_rtol', ctypes.c_double),
                ('inner_trace_rtol', ctypes.c_double), ('trace_mg', ctypes.c_int),
                ('device_loops', ctypes.c_int), ('inner_trace_vcycles', ctypes.c_int),
                ('precision', ctypes.c_int), ('inner_trace_fp32', ctypes.c_int),
                ('trace_fp32_vcycle', ctypes.c_int), ('inner_gs', ctypes.c_int), ('timeout_ms', ctypes.c_double),
                ('relax_eta', ctypes.c_double)]


class hdg_stats(ctypes.Structure):
    _fields_ = [('richardson_iters', ctypes.c_int), ('trace_solves', ctypes.c_int),
                ('trace_iters', ctypes.c_int), ('stepI_solves', ctypes.c_int),
                ('stepI_iters', ctypes.c_int), ('stage_solves', ctypes.c_int),
                ('last_update_norm', ctypes.c_double), ('last_trace_relres', ctypes.c_double),
                ('ms_total', ctypes.c_double), ('ms_trace', ctypes.c_double), ('ms_stepI', ctypes.c_double),
                ('ms_assembly', ctypes.c_double), ('ms_bdm', ctypes.c_double),
                ('graph_kernels', ctypes.c_longlong), ('stage_products32', ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hdg_server_stats(ctypes.Structure):
    _fields_ = [('submitted', ctypes.c_int), ('admitted', ctypes.c_int), ('completed', ctypes.c_int),
                ('active', ctypes.c_int), ('queued', ctypes.c_int), ('contexts_created', ctypes.c_int),
                ('contexts_reused', ctypes.c_int), ('contexts_released', ctypes.c_int),
                ('bytes_in_use', ctypes.c_double), ('steps', ctypes.c_longlong), ('stage_solves', ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


PHI = ctypes.CFUNCTYPE(ctypes.c_double, ctypes.c_double, ctypes.c_void_p)
_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_I64P = ctypes.POINTER(ctypes.c_int64)
_DP = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    'hdg_default_params': (None, [ctypes.POINTER(hdg_params)]),
    'hdg_status_string': (ctypes.c_char_p, [_I]),
    'hdg_last_error': (ctypes.c_char_p, []),
    'hdg_mesh_counts': (_I, [ctypes.POINTER(hdg_mesh_desc), _I, _I64P, _I64P]),
    'hdg_reference_rule': (_I, [_I, _I, _DP, _DP, ctypes.POINTER(_I)]),
    'hdg_reference_basis': (_I, [_I, _I, _DP, _DP]),
    'hdg_setup_mesh': (_I, [ctypes.POINTER(_P), ctypes.POINTER(hdg_mesh_desc), ctypes.POINTER(hdg_params), _P]),
    'hdg_destroy': (None, [_P]),
    'hdg_dof_sizes': (_I, [_P, _I64P, _I64P, _I64P]),
    'hdg_set_state': (_I, [_P, _P, _P, _P, _D]),
    'hdg_get_state': (_I, [_P, _P, _P, _P, _DP]),
    'hdg_project': (_I, [_P, _I, _P, _P]),
    'hdg_batch_step': (_I, [ctypes.POINTER(_P), _I, _I, ctypes.POINTER(hdg_stats)]),
    'hdg_ctx_bytes': (ctypes.c_size_t, [_P]),
    'hdg_estimate_bytes': (ctypes.c_double, [ctypes.POINTER(hdg_mesh_desc), ctypes.POINTER(hdg_params)]),
    'hdg_server_create': (_I, [ctypes.POINTER(_P), _I, _D, _I]),
    'hdg_server_submit': (_I, [_P, ctypes.POINTER(hdg_mesh_desc), ctypes.POINTER(hdg_params), _DP, _I,
                              ctypes.POINTER(ctypes.c_longlong)]),
    'hdg_server_progress': (_I, [_P, ctypes.POINTER(hdg_server_stats)]),
    'hdg_server_result': (_I, [_P, ctypes.c_longlong, _DP, _DP, _DP, _DP]),
    'hdg_server_destroy': (None, [_P]),
    'hdg_set_tracer': (_I, [_P, _P]),
    'hdg_get_tracer': (_I, [_P, _P]),
    'hdg_cg_project': (_I, [_P, _P, _P]),
    'hdg_tracer_rhs': (_I, [_P, _P, _P, _P]),
    'hdg_set_forcing': (_I, [_P, _P, PHI, _P]),
    'hdg_imex_step': (_I, [_P, _I, ctypes.POINTER(hdg_stats)]),
    'hdg_solve_stage': (_I, [_P, _D, _P, _P, _P, _P, _P, ctypes.POINTER(hdg_stats)]),
    'hdg_bdm_project': (_I, [_P, _P, _P]),
    'hdg_fimpl_apply': (_I, [_P, _P, _P, _P]),
    'hdg_tentative_solve': (_I, [_P, _D, _P, _P, _P, ctypes.POINTER(hdg_stats)]),
    'hdg_mixed_solve': (_I, [_P, _D, _P, _P, _P, _P, _P, ctypes.POINTER(hdg_stats)]),
    'hdg_trace_apply': (_I, [_P, _D, _P, _P]),
    'hdg_div_free_project': (_I, [_P, ctypes.POINTER(hdg_stats)]),
    'hdg_reconstruct_pressure': (_I, [_P, ctypes.POINTER(hdg_stats)]),
    'hdg_time_kernel': (_I, [_P, _I, _D, _I, _DP, _DP]),
    'hdg_trace_apply_noalloc': (_I, [_P, _D, _P, _P]),
}


def load(build=True):
    """Load (building if needed) the in-tree CUDA library. Raises if it cannot be loaded:
    there is no fallback path."""
    global _lib
    if _lib is not None:
        return _lib
    path = build_library() if build else LIB
    if not os.path.exists(path):
        raise RuntimeError(f'CUDA library missing: {path}')
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status, where):
    if status != HDG_OK:
        raise HdgError(status, where)


def _ptr(t):
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError('expected a contiguous CUDA float64 tensor')
    return ctypes.c_void_p(t.data_ptr())


# ------------------------------------------------------------------ host-only functions
def hdg_default_params():
    p = hdg_params()
    load().hdg_default_params(ctypes.byref(p))
    return p


def hdg_mesh_counts(n, k, periodic_x=False, periodic_y=False, Lx=1.0, Ly=1.0):
    d = hdg_mesh_desc(n, Lx, Ly, int(periodic_x), int(periodic_y))
    nc, nf = ctypes.c_int64(), ctypes.c_int64()
    _check(load().hdg_mesh_counts(ctypes.byref(d), k, ctypes.byref(nc), ctypes.byref(nf)), 'hdg_mesh_counts')
    return nc.value, nf.value


def hdg_reference_rule(k, which):
    import numpy as np
    n = _I(0)
    _check(load().hdg_reference_rule(k, which, None, None, ctypes.byref(n)), 'hdg_reference_rule')
    dim = 2 if which == 0 else 1
    pts = np.zeros(n.value * dim)
    wts = np.zeros(n.value)
    _check(load().hdg_reference_rule(k, which, pts.ctypes.data_as(_DP), wts.ctypes.data_as(_DP),
                                     ctypes.byref(n)), 'hdg_reference_rule')
    return pts.reshape(n.value, dim), wts


def hdg_reference_basis(m, pts):
    import numpy as np
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 2)
    d = (m + 1) * (m + 2) // 2
    vals = np.zeros((len(pts), d))
    _check(load().hdg_reference_basis(m, len(pts), pts.ctypes.data_as(_DP), vals.ctypes.data_as(_DP)),
           'hdg_reference_basis')
    return vals


# ------------------------------------------------------------------ context
class Context:
    """An hdg_ctx: mesh, operators and state on the current CUDA device."""

    def __init__(self, n, k, periodic_x=False, periodic_y=False, Lx=1.0, Ly=1.0, stream=None, **params):
        import torch
        lib = load()
        p = hdg_default_params()
        p.k = k
        for key, val in params.items():
            if key == 'tableau' and isinstance(val, str):
                val = TABLEAUS[val]
            if key == 'precision' and isinstance(val, str):
                val = PRECISIONS[val]
            if not hasattr(p, key):
                raise KeyError(key)
            setattr(p, key, val)
        self.params = p
        self.mesh = hdg_mesh_desc(n, Lx, Ly, int(periodic_x), int(periodic_y))
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        self._ctx = ctypes.c_void_p()
        _check(lib.hdg_setup_mesh(ctypes.byref(self._ctx), ctypes.byref(self.mesh), ctypes.byref(p),
                                  ctypes.c_void_p(stream.cuda_stream)), 'hdg_setup_mesh')
        nQ, nP, nL = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(lib.hdg_dof_sizes(self._ctx, ctypes.byref(nQ), ctypes.byref(nP), ctypes.byref(nL)), 'hdg_dof_sizes')
        self.nQ, self.nP, self.nL = nQ.value, nP.value, nL.value
        self.k, self.n = k, n
        self.ncells = 2 * n * n
        self._phi = None

    def close(self):
        if self._ctx:
            load().hdg_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # shapes of the exchange arrays
    def shapes(self):
        mu = (self.k + 2) * (self.k + 3) // 2
        npn = (self.k + 1) * (self.k + 2) // 2
        return (self.ncells, 2, mu), (self.ncells, npn), (self.nL // (self.k + 1), self.k + 1)

    def zeros(self):
        import torch
        sQ, sP, sL = self.shapes()
        z = lambda s: torch.zeros(s, dtype=torch.float64, device='cuda')
        return z(sQ), z(sP), z(sL)

    def hdg_set_state(self, Q, p=None, lam=None, t=0.0):
        _check(load().hdg_set_state(self._ctx, _ptr(Q), _ptr(p), _ptr(lam), t), 'hdg_set_state')

    def hdg_get_state(self):
        Q, p, lam = self.zeros()
        t = ctypes.c_double()
        _check(load().hdg_get_state(self._ctx, _ptr(Q), _ptr(p), _ptr(lam), ctypes.byref(t)), 'hdg_get_state')
        return Q, p, lam, t.value

    def hdg_project(self, field, values_at_qp):
        """L2 projection of samples at the volume quadrature points (field 0: velocity, values
        [ncells][2][nq]; field 1: pressure, values [ncells][nq]) -> nodal Q or p."""
        out = self.zeros()[field]
        _check(load().hdg_project(self._ctx, field, _ptr(values_at_qp), _ptr(out)), 'hdg_project')
        return out

    def hdg_set_tracer(self, q):
        _check(load().hdg_set_tracer(self._ctx, _ptr(q)), 'hdg_set_tracer')

    def hdg_get_tracer(self):
        out = self.zeros()[1]
        _check(load().hdg_get_tracer(self._ctx, _ptr(out)), 'hdg_get_tracer')
        return out

    def hdg_cg_project(self, Q):
        out = self.zeros()[0]
        _check(load().hdg_cg_project(self._ctx, _ptr(Q), _ptr(out)), 'hdg_cg_project')
        return out

    def hdg_tracer_rhs(self, q, U):
        out = self.zeros()[1]
        _check(load().hdg_tracer_rhs(self._ctx, _ptr(q), _ptr(U), _ptr(out)), 'hdg_tracer_rhs')
        return out

    def hdg_set_forcing(self, F, phi=None):
        if F is None:
            _check(load().hdg_set_forcing(self._ctx, None, PHI(), None), 'hdg_set_forcing')
            self._phi = None
            return
        cb = PHI(lambda t, user: float(phi(t))) if phi is not None else PHI()
        self._phi = cb                                   # keep the callback alive
        _check(load().hdg_set_forcing(self._ctx, _ptr(F), cb, None), 'hdg_set_forcing')

    def hdg_imex_step(self, nsteps=1, check=True):
        st = hdg_stats()
        s = load().hdg_imex_step(self._ctx, nsteps, ctypes.byref(st))
        if check:
            _check(s, 'hdg_imex_step')
        return st.as_dict() | {'status': s}

    def hdg_solve_stage(self, c, R, Qstar, Q, p, lam, check=True):
        st = hdg_stats()
        s = load().hdg_solve_stage(self._ctx, c, _ptr(R), _ptr(Qstar), _ptr(Q), _ptr(p), _ptr(lam), ctypes.byref(st))
        if check:
            _check(s, 'hdg_solve_stage')
        return st.as_dict() | {'status': s}

    def hdg_bdm_project(self, Q):
        out = self.zeros()[0]
        _check(load().hdg_bdm_project(self._ctx, _ptr(Q), _ptr(out)), 'hdg_bdm_project')
        return out

    def hdg_fimpl_apply(self, Qstar, Q):
        out = self.zeros()[0]
        _check(load().hdg_fimpl_apply(self._ctx, _ptr(Qstar), _ptr(Q), _ptr(out)), 'hdg_fimpl_apply')
        return out

    def hdg_tentative_solve(self, c, Qstar, R):
        out = self.zeros()[0]
        st = hdg_stats()
        _check(load().hdg_tentative_solve(self._ctx, c, _ptr(Qstar), _ptr(R), _ptr(out), ctypes.byref(st)),
               'hdg_tentative_solve')
        return out, st.as_dict()

    def hdg_mixed_solve(self, c, R=None, X=None):
        U, p, lam = self.zeros()
        st = hdg_stats()
        _check(load().hdg_mixed_solve(self._ctx, c, _ptr(R), _ptr(X), _ptr(U), _ptr(p), _ptr(lam), ctypes.byref(st)),
               'hdg_mixed_solve')
        return U, p, lam, st.as_dict()

    def hdg_trace_apply(self, c, lam):
        out = self.zeros()[2]
        _check(load().hdg_trace_apply(self._ctx, c, _ptr(lam), _ptr(out)), 'hdg_trace_apply')
        return out

    def hdg_div_free_project(self):
        st = hdg_stats()
        _check(load().hdg_div_free_project(self._ctx, ctypes.byref(st)), 'hdg_div_free_project')
        return st.as_dict()

    def hdg_reconstruct_pressure(self):
        st = hdg_stats()
        _check(load().hdg_reconstruct_pressure(self._ctx, ctypes.byref(st)), 'hdg_reconstruct_pressure')
        return st.as_dict()

    def hdg_time_kernel(self, which, c=1.0, reps=20):
        ms, b = ctypes.c_double(), ctypes.c_double()
        _check(load().hdg_time_kernel(self._ctx, which, c, reps, ctypes.byref(ms), ctypes.byref(b)), 'hdg_time_kernel')
        return ms.value, b.value

    def hdg_trace_apply_noalloc(self, c, lam, out):
        """hdg_trace_apply without device allocation; out is a caller-owned trace-shaped tensor.
        lam and out must hold nlambda doubles each, on the context's device."""
        import torch
        dev = torch.cuda.current_device()
        for name, t in (('lam', lam), ('out', out)):
            if t is None or t.numel() != self.nL:
                raise ValueError(f'{name} must hold {self.nL} doubles')
            if t.is_cuda and t.device.index != dev:
                raise ValueError(f'{name} is on cuda:{t.device.index}, the current device is cuda:{dev}')
        _check(load().hdg_trace_apply_noalloc(self._ctx, c, _ptr(lam), _ptr(out)), 'hdg_trace_apply_noalloc')
        return out

    def hdg_ctx_bytes(self):
        return int(load().hdg_ctx_bytes(self._ctx))


def make_params(k, **params):
    """hdg_params with the library's defaults, degree k and the given fields."""
    p = hdg_default_params()
    p.k = k
    for key, val in params.items():
        if key == 'tableau' and isinstance(val, str):
            val = TABLEAUS[val]
        if key == 'precision' and isinstance(val, str):
            val = PRECISIONS[val]
        if not hasattr(p, key):
            raise KeyError(key)
        setattr(p, key, val)
    return p


def hdg_batch_step(contexts, nsteps=1, check=True):
    """hdg_batch_step over Context objects: every context's step enqueued before any is waited for."""
    n = len(contexts)
    arr = (_P * n)(*[c._ctx.value for c in contexts])
    st = (hdg_stats * n)()
    s = load().hdg_batch_step(arr, n, nsteps, st)
    if check:
        _check(s, 'hdg_batch_step')
    return [x.as_dict() for x in st], s


def hdg_estimate_bytes(n, k, periodic_x=False, periodic_y=False, Lx=1.0, Ly=1.0, **params):
    d = hdg_mesh_desc(n, Lx, Ly, int(periodic_x), int(periodic_y))
    p = make_params(k, **params)
    return float(load().hdg_estimate_bytes(ctypes.byref(d), ctypes.byref(p)))


class Server:
    """An hdg_server: requests (mesh, parameters, initial velocity, steps) served with admission by
    device-memory budget and continuous batching."""

    def __init__(self, mem_budget_bytes, max_active, device=None):
        import torch
        lib = load()
        self._srv = ctypes.c_void_p()
        dev = torch.cuda.current_device() if device is None else device
        _check(lib.hdg_server_create(ctypes.byref(self._srv), dev, float(mem_budget_bytes), int(max_active)),
               'hdg_server_create')
        self._sizes = {}

    def submit(self, n, k, Q0, nsteps, periodic_x=False, periodic_y=False, Lx=1.0, Ly=1.0, **params):
        """Q0: host numpy array of the initial nodal velocity ((ncells, 2, mu) or flat). Returns the id."""
        import numpy as np
        d = hdg_mesh_desc(n, Lx, Ly, int(periodic_x), int(periodic_y))
        p = make_params(k, **params)
        q = np.ascontiguousarray(Q0, dtype=np.float64).reshape(-1)
        rid = ctypes.c_longlong()
        _check(load().hdg_server_submit(self._srv, ctypes.byref(d), ctypes.byref(p), q.ctypes.data_as(_DP), int(nsteps),
                                        ctypes.byref(rid)), 'hdg_server_submit')
        nc, nf = hdg_mesh_counts(n, k, periodic_x, periodic_y, Lx, Ly)
        mu, npn = (k + 2) * (k + 3) // 2, (k + 1) * (k + 2) // 2
        self._sizes[rid.value] = (nc * 2 * mu, nc * npn, nf * (k + 1))
        return rid.value

    def progress(self):
        st = hdg_server_stats()
        _check(load().hdg_server_progress(self._srv, ctypes.byref(st)), 'hdg_server_progress')
        return st.as_dict()

    def result(self, rid):
        """(Q, p, lambda, latency_ms) of a completed request (host numpy), or None if not complete."""
        import numpy as np
        nQ, nP, nL = self._sizes[rid]
        Q, p, lam, lat = np.empty(nQ), np.empty(nP), np.empty(nL), ctypes.c_double()
        s = load().hdg_server_result(self._srv, rid, Q.ctypes.data_as(_DP), p.ctypes.data_as(_DP),
                                     lam.ctypes.data_as(_DP), ctypes.byref(lat))
        if s != HDG_OK:
            return None
        del self._sizes[rid]
        return Q, p, lam, lat.value

    def close(self):
        if self._srv:
            load().hdg_server_destroy(self._srv)
            self._srv = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
