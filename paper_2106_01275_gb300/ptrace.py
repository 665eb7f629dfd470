"""Thin ctypes binding of libptrace (include/ptrace.h).

Argument marshalling only: every step of the estimator runs in the CUDA
library.  PyTorch provides device memory and the stream.  There is no CPU
fallback: if the library is missing or no GPU is present the calls raise.
The `*_host` functions are separate host-only twins of some device entry
points (the same site arithmetic and steps, run by host loops) that the
CPU tests use to check that code; no device entry point ever calls them.
Field layouts are those of the C ABI (see include/ptrace.h):
  scalar fields  torch.float64    [nrhs, N]
  spinor fields  torch.complex128 [nrhs, N, 4, 3]
  links          torch.complex128 [N, 4, 3, 3]
"""
import atexit
import ctypes
import os
import sys
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libptrace.so")

PT_OK, PT_ERR_ARG, PT_ERR_CUDA, PT_ERR_NOCONV, PT_ERR_TIMEOUT, PT_ERR_NUMERIC, PT_ERR_OOM = 0, -1, -2, -3, -4, -5, -6
PREC = {"fp64": 0, "mixed_fp32": 1, "mixed_bf16": 2}
NOISE = {"z2": 0, "z4": 1}
ORDER = {"natural": 0, "redblack": 1}
_ERRNAMES = {-1: "PT_ERR_ARG", -2: "PT_ERR_CUDA", -3: "PT_ERR_NOCONV", -4: "PT_ERR_TIMEOUT",
             -5: "PT_ERR_NUMERIC", -6: "PT_ERR_OOM"}


class PtraceError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (_ERRNAMES.get(code, str(code)), msg))
        self.code = code


class Stats(ctypes.Structure):
    _fields_ = [("n_rhs", ctypes.c_int64), ("inner_iters", ctypes.c_int64), ("outer_iters", ctypes.c_int64),
                ("site_rhs_applies", ctypes.c_int64), ("engine_iters", ctypes.c_int64),
                ("graph_launches", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("max_relres", ctypes.c_double), ("n_slots", ctypes.c_int32), ("n_noconv", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Tune(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_double), ("group", ctypes.c_int32), ("graph_iters", ctypes.c_int32),
                ("rhs_block", ctypes.c_int32), ("overlap", ctypes.c_int32), ("evenodd", ctypes.c_int32),
                ("cta_threads", ctypes.c_int32), ("sites_per_thread", ctypes.c_int32),
                ("seconds_per_rhs", ctypes.c_double)]

    def as_dict(self):
        return {"delta": self.delta, "group": self.group, "graph_iters": self.graph_iters,
                "rhs_block": self.rhs_block, "overlap": self.overlap, "evenodd": self.evenodd,
                "cta_threads": self.cta_threads, "sites_per_thread": self.sites_per_thread,
                "seconds_per_rhs": self.seconds_per_rhs}


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SIGS = {
    "pt_version": ([], _I),
    "pt_last_error": ([ctypes.c_char_p, ctypes.c_size_t], _I),
    "pt_create": ([ctypes.POINTER(_P), _I, _P], _I),
    "pt_destroy": ([_P], _I),
    "pt_synchronize": ([_P], _I),
    "pt_set_memory_budget": ([_P, ctypes.c_size_t], _I),
    "pt_set_max_slots": ([_P, _I], _I),
    "pt_set_launch_limit": ([_P, ctypes.c_int64], _I),
    "pt_autotune": ([_P, _P, _P, _I, _I, _I, ctypes.c_uint64, _I, _D, _I, _I, ctypes.POINTER(Tune)], _I),
    "pt_set_tuning": ([_P, _P, _I, ctypes.POINTER(Tune)], _I),
    "pt_get_tuning": ([_P, _P, _I, ctypes.POINTER(Tune)], _I),
    "pt_profile_enable": ([_P, _I], _I),
    "pt_profile_read": ([_P, _I, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(_D), _I], _I),
    "pt_op_laplacian": ([_P, ctypes.POINTER(_I), _D, ctypes.POINTER(_P)], _I),
    "pt_op_wilson": ([_P, ctypes.POINTER(_I), _P, _D, _I, ctypes.POINTER(_P)], _I),
    "pt_op_dof": ([_P], _I),
    "pt_op_set_clover": ([_P, _D], _I),
    "pt_op_destroy": ([_P], _I),
    "pt_apply": ([_P, _P, _P, _P, _I, _I], _I),
    "pt_stencil": ([_I, ctypes.POINTER(_I), _I, _I, ctypes.POINTER(_I), _I, ctypes.POINTER(_I)], _I),
    "pt_colour": ([_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, _I, _P, ctypes.POINTER(_I)], _I),
    "pt_colour_nested": ([_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, _I, _P, _I, _P,
                          ctypes.POINTER(_I)], _I),
    "pt_colour_conflicts": ([_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, _P,
                             ctypes.POINTER(ctypes.c_int64)], _I),
    "pt_colour_conflicts_noalloc": ([_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, _P,
                                     ctypes.POINTER(ctypes.c_int64)], _I),
    "pt_tile_dims": ([ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, ctypes.POINTER(_I)], _I),
    "pt_tile_replicate": ([_P, ctypes.POINTER(_I), _P, ctypes.POINTER(_I), _P], _I),
    "pt_colour_tiled": ([_P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, _I, _P, ctypes.POINTER(_I),
                         ctypes.POINTER(_I)], _I),
    "pt_clearance": ([_P, ctypes.POINTER(_I), _I, _P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _P, _P], _I),
    "pt_make_probes": ([_P, _P, ctypes.c_int64, _I, _I, ctypes.c_uint64, _I, _I, _I, _P], _I),
    "pt_solve": ([_P, _P, _P, _P, _I, _I, _D, _I, _P, _P, ctypes.POINTER(Stats)], _I),
    "pt_trace_PAinv": ([_P, _P, _P, _I, _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64, _I, _I, _I, _I, _D, _I,
                        _P, _P, _P, ctypes.POINTER(Stats)], _I),
    "pt_trace_PAinv_multi": ([_P, _P, _I, _P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64,
                              _I, _I, _I, _I, _D, _I, _P, ctypes.POINTER(Stats)], _I),
    "pt_trace_PAinv_nested": ([_P, _P, _I, _P, ctypes.POINTER(_I), _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64,
                               _I, _I, _I, _I, _D, _I, _P, ctypes.POINTER(Stats)], _I),
    "pt_deflation_terms": ([_P, _P, _P, _I, _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64, _I, _I, _I, _P, _P, _P,
                            _P, _P], _I),
    "pt_hermitian_eig": ([_I, _P, _I, _P, _P], _I),
    "pt_singular_triplets": ([_P, _P, _I, _I, _I, _P, _P, _P, _P], _I),
    "pt_eo_layout": ([ctypes.POINTER(_I), _I, _P, _P], _I),
    "pt_eo_host": ([_I, ctypes.POINTER(_I), _D, _D, _P, _I, _P, _P, _I, _P, _P, _P, _I], _I),
    "pt_eo_schur": ([_P, _P, _P, _P, _P, _P, _I], _I),
    "pt_eo_prepare": ([_P, _P, _P, _P, _P, _I], _I),
    "pt_eo_reconstruct": ([_P, _P, _P, _P, _P, _P, _I], _I),
    "pt_eo_clover_blocks": ([_P, _P, _D, _P, _P], _I),
    "pt_wmg_solve": ([_P, _P, _D, _I, _I, _I, _I, _D, _I, ctypes.c_uint64, _P, _P, _I, _D, _I, _P, _P], _I),
    "pt_wmg_solve_host": ([ctypes.POINTER(_I), _P, _D, _D, _I, _I, _I, _I, _I, _D, _I, ctypes.c_uint64, _P, _P, _I,
                           _D, _I, _P, _P], _I),
    "pt_wmg_setup_host": ([ctypes.POINTER(_I), _P, _D, _D, _I, _I, _I, _I, _D, ctypes.c_uint64, _P, _P], _I),
    "pt_mg_solve": ([_P, _P, _I, _I, _D, _P, _P, _I, _D, _I, _P, _P], _I),
    "pt_mg_solve_host": ([ctypes.POINTER(_I), _D, _I, _I, _D, _P, _P, _I, _D, _I, _P, _P], _I),
    "pt_mg_cycle_host": ([ctypes.POINTER(_I), _D, _I, _I, _D, _P, _P], _I),
    "pt_trace_PAinv_eo": ([_P, _P, _P, _I, _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64, _I, _I, _D, _I, _D, _P,
                           ctypes.POINTER(Stats)], _I),
    "pt_trace_PAinv_eo_host": ([ctypes.POINTER(_I), _D, _P, _I, _I, ctypes.POINTER(_I), _I, _I, ctypes.c_uint64, _I,
                                _I, _D, _I, _D, _P, ctypes.POINTER(Stats)], _I),
    "pt_eo_solve": ([_P, _P, _P, _P, _P, _P, _I, _D, _I, _P, _P], _I),
    "pt_eo_solve_host": ([_I, ctypes.POINTER(_I), _D, _D, _P, _I, _P, _P, _P, _P, _I, _D, _I, _P, _P], _I),
    "pt_clover_blocks_host": ([ctypes.POINTER(_I), _P, _D, _D, _P], _I),
    "pt_clover_blocks": ([_P, _P, _D, _P], _I),
    "pt_site_blocks_apply": ([_P, _I, _P, _P, _D, _P, _I], _I),
    "pt_site_blocks_invert_host": ([_I, _P, _D, _P], _I),
    "pt_site_blocks_invert": ([_P, _I, _P, _D, _P], _I),
    "pt_grad": ([_P, _P, _P, _I, _I, _I, _I, ctypes.c_uint64, _I, _I, _I, _I, _D, _I, _P, _P, _P, _P,
                 ctypes.POINTER(Stats)], _I),
}


def lib():
    """Load libptrace.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libptrace.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(code, ok=(PT_OK,)):
    if code not in ok:
        buf = ctypes.create_string_buffer(512)
        lib().pt_last_error(buf, 512)
        raise PtraceError(code, buf.value.decode(errors="replace"))
    return code


def _ints(vals):
    vals = [int(v) for v in vals]
    return (_I * len(vals))(*vals)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# Live handles, destroyed operators-first at interpreter exit while the CUDA
# runtime is still up (a destructor running after it has shut down may crash).
_LIVE = weakref.WeakValueDictionary()
_LIVE_ID = [0]


def _register(obj):
    _LIVE_ID[0] += 1
    _LIVE[_LIVE_ID[0]] = obj


@atexit.register
def _close_all():
    objs = list(_LIVE.values())
    for o in objs:
        if isinstance(o, Operator):
            o.close()
    for o in objs:
        if isinstance(o, Context):
            o.close()


def exported_symbols():
    """Names the binding expects the library to export."""
    return sorted(_SIGS)


class Context:
    """A library context bound to one CUDA device and stream.

    stream: a torch.cuda.Stream, an integer cudaStream_t, or None for torch's
    current stream (so torch CUDA events bracket the library's kernels)."""

    def __init__(self, device=0, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the ptrace library has no CPU path")
        self.device = int(device)
        torch.cuda.set_device(self.device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
        if handle == 0:
            handle = 1          # torch's default stream is the legacy stream: cudaStreamLegacy
        self.stream = stream
        self._h = ctypes.c_void_p()
        _check(lib().pt_create(ctypes.byref(self._h), self.device, ctypes.c_void_p(handle)))
        _register(self)

    @property
    def handle(self):
        return self._h

    def close(self):
        if self._h:
            # operators first: one finalised from a reference cycle after its
            # context must find nothing left to free
            for o in list(_LIVE.values()):
                if isinstance(o, Operator) and o.ctx is self:
                    o.close()
            lib().pt_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def synchronize(self):
        _check(lib().pt_synchronize(self._h))

    def set_memory_budget(self, nbytes):
        _check(lib().pt_set_memory_budget(self._h, int(nbytes)))

    def set_max_slots(self, n):
        _check(lib().pt_set_max_slots(self._h, int(n)))

    def set_launch_limit(self, n):
        _check(lib().pt_set_launch_limit(self._h, int(n)))

    def profile(self, on=True):
        _check(lib().pt_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, which=0, reset=True):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(lib().pt_profile_read(self._h, which, ctypes.byref(n), ctypes.byref(ms), 1 if reset else 0))
        return n.value, ms.value


class Operator:
    def __init__(self, ctx, handle, dims, dof, keep=None):
        self.ctx, self._h, self.dims, self.dof, self._keep = ctx, handle, list(dims), dof, keep
        self.N = int(np.prod(dims))
        _register(self)

    def close(self):
        if self._h:
            lib().pt_op_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def field_shape(self, nrhs):
        return (nrhs, self.N) if self.dof == 1 else (nrhs, self.N, 4, 3)

    def field_dtype(self):
        import torch
        return torch.float64 if self.dof == 1 else torch.complex128


def laplacian(ctx, dims, m2):
    h = ctypes.c_void_p()
    _check(lib().pt_op_laplacian(ctx.handle, _ints(dims), float(m2), ctypes.byref(h)))
    op = Operator(ctx, h, dims, 1)
    op.m2 = float(m2)
    return op


def wilson(ctx, dims, U, kappa, antiperiodic_t=True):
    """U: torch.complex128 tensor [N, 4, 3, 3] on the context's device."""
    import torch
    assert U.dtype == torch.complex128 and U.is_cuda and U.is_contiguous()
    h = ctypes.c_void_p()
    _check(lib().pt_op_wilson(ctx.handle, _ints(dims), _ptr(U), float(kappa), 1 if antiperiodic_t else 0,
                              ctypes.byref(h)))
    op = Operator(ctx, h, dims, 12)
    op.kappa = float(kappa)
    ctx.synchronize()
    return op


def set_clover(op, csw):
    """Give the Wilson operator op the clover term with coefficient csw (0
    removes it): pt_apply then applies A_W + C and the batched solves and
    traces use the clover operator on the even Schur complement."""
    _check(lib().pt_op_set_clover(op._h, float(csw)))
    op.csw = float(csw)
    return op


def apply(op, x, prec="fp64"):
    import torch
    x = x.contiguous()
    y = torch.empty_like(x)
    nrhs = x.shape[0]
    _check(lib().pt_apply(op.ctx.handle, op._h, _ptr(x), _ptr(y), nrhs, PREC[prec]))
    return y


def stencil(mu, p_list, k):
    p = _ints(p_list)
    n = _I()
    lib().pt_stencil(mu, p, len(p_list), k, None, 0, ctypes.byref(n))
    out = (_I * (4 * max(n.value, 1)))()
    _check(lib().pt_stencil(mu, p, len(p_list), k, out, n.value, ctypes.byref(n)))
    return np.array(out[:4 * n.value], dtype=np.int64).reshape(-1, 4)


def colour(ctx, dims, mu, p_list, k, order="natural", out=None):
    import torch
    N = int(np.prod(dims))
    col = out if out is not None else torch.empty(N, dtype=torch.int32, device="cuda:%d" % ctx.device)
    m = _I()
    _check(lib().pt_colour(ctx.handle, _ints(dims), mu, _ints(p_list), len(p_list), k,
                           ORDER[order] if isinstance(order, str) else int(order), _ptr(col), ctypes.byref(m)))
    return col, m.value


def colour_nested(ctx, dims, mu, p_list, k, parent, n_parent, order="natural", out=None):
    """Colouring at distance k nested in the coarser colouring `parent`
    (pt_colour_nested): (col, m)."""
    import torch
    N = int(np.prod(dims))
    col = out if out is not None else torch.empty(N, dtype=torch.int32, device="cuda:%d" % ctx.device)
    m = _I()
    _check(lib().pt_colour_nested(ctx.handle, _ints(dims), int(mu), _ints(p_list), len(p_list), int(k),
                                  ORDER[order] if isinstance(order, str) else int(order), _ptr(parent),
                                  int(n_parent), _ptr(col), ctypes.byref(m)))
    return col, m.value


def conflicts(ctx, dims, mu, p_list, k, col):
    n = ctypes.c_int64()
    _check(lib().pt_colour_conflicts(ctx.handle, _ints(dims), mu, _ints(p_list), len(p_list), k, _ptr(col),
                                     ctypes.byref(n)))
    return n.value


def conflicts_noalloc(dims, mu, p_list, k, col, stream=None):
    """Allocation-free conflict count (pt_colour_conflicts_noalloc): no context,
    no device allocation; runs on the current device and `stream` (default:
    torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    n = ctypes.c_int64()
    _check(lib().pt_colour_conflicts_noalloc(ctypes.c_void_p(handle), _ints(dims), int(mu), _ints(p_list),
                                             len(p_list), int(k), _ptr(col), ctypes.byref(n)))
    return n.value


def tile_dims(dims, mu, p_list, k):
    """Tile of Sec. 3.5 (pt_tile_dims; host only)."""
    out = (_I * 4)()
    _check(lib().pt_tile_dims(_ints(dims), int(mu), _ints(p_list), len(p_list), int(k), out))
    return list(out)


def tile_replicate(ctx, tile, tile_col, dims, out=None):
    """Repeat a tile's colouring over the lattice (pt_tile_replicate)."""
    import torch
    N = int(np.prod(dims))
    col = out if out is not None else torch.empty(N, dtype=torch.int32, device="cuda:%d" % ctx.device)
    _check(lib().pt_tile_replicate(ctx.handle, _ints(tile), _ptr(tile_col), _ints(dims), _ptr(col)))
    return col


def colour_tiled(ctx, dims, mu, p_list, k, order="natural", out=None):
    """Colour the Sec. 3.5 tile and repeat it (pt_colour_tiled): (col, m, tile)."""
    import torch
    N = int(np.prod(dims))
    col = out if out is not None else torch.empty(N, dtype=torch.int32, device="cuda:%d" % ctx.device)
    m = _I()
    tile = (_I * 4)()
    _check(lib().pt_colour_tiled(ctx.handle, _ints(dims), int(mu), _ints(p_list), len(p_list), int(k),
                                 ORDER[order] if isinstance(order, str) else int(order), _ptr(col), ctypes.byref(m),
                                 tile))
    return col, m.value, list(tile)


def clearance(ctx, dims, mu, col, p_list, k_list):
    """Table 5 statistic (pt_clearance): (matches, shell_sizes), int64 arrays
    [len(p_list), len(k_list)]; percentage = 100 matches / (N shell_size)."""
    m = np.zeros((len(p_list), len(k_list)), dtype=np.int64)
    s = np.zeros_like(m)
    _check(lib().pt_clearance(ctx.handle, _ints(dims), int(mu), _ptr(col), _ints(p_list), len(p_list),
                              _ints(k_list), len(k_list), _np_ptr(m), _np_ptr(s)))
    return m, s


def make_probe(ctx, col, colour_index, noise, seed, set_index, dof, component):
    """One probe in the user layout; component -1 = undiluted (independent noise per component)."""
    import torch
    N = col.numel()
    if dof == 1:
        v = torch.empty(N, dtype=torch.float64, device=col.device)
    else:
        v = torch.empty((N, 4, 3), dtype=torch.complex128, device=col.device)
    _check(lib().pt_make_probes(ctx.handle, _ptr(col), N, int(colour_index), NOISE[noise] if isinstance(noise, str)
                                else int(noise), int(seed), int(set_index), int(dof), int(component), _ptr(v)))
    return v


def solve(op, B, prec="mixed_fp32", tol=1e-10, maxit=10000, allow_noconv=False):
    import torch
    B = B.contiguous()
    X = torch.empty_like(B)
    nrhs = B.shape[0]
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs, dtype=np.float64)
    st = Stats()
    rc = lib().pt_solve(op.ctx.handle, op._h, _ptr(B), _ptr(X), nrhs, PREC[prec], float(tol), int(maxit),
                        _np_ptr(iters), _np_ptr(relres), ctypes.byref(st))
    _check(rc, (PT_OK, PT_ERR_NOCONV) if allow_noconv else (PT_OK,))
    return X, iters, relres, st.as_dict()


def trace(op, col, n_colours, mu, p_list, noise="z2", seed=0, set0=0, n_sets=1, dilute=True,
          prec="mixed_fp32", tol=1e-10, maxit=20000):
    """Probed estimates est[s, n] of Tr(P_{p_n} A^{-1}); returns (est, mean, var, stats)."""
    n_p = len(p_list)
    est = np.zeros((n_sets, n_p), dtype=np.complex128)
    mean = np.zeros(n_p, dtype=np.complex128)
    var = np.zeros(n_p, dtype=np.float64)
    st = Stats()
    rc = lib().pt_trace_PAinv(op.ctx.handle, op._h, _ptr(col), int(n_colours), int(mu), _ints(p_list), n_p,
                              NOISE[noise] if isinstance(noise, str) else int(noise), int(seed), int(set0),
                              int(n_sets), 1 if dilute else 0, PREC[prec], float(tol), int(maxit),
                              _np_ptr(est), _np_ptr(mean), _np_ptr(var), ctypes.byref(st))
    _check(rc)
    return est, mean, var, st.as_dict()


def autotune(op, col, n_colours, mu, noise="z2", seed=0, prec="mixed_fp32", tol=1e-10, maxit=20000,
             trial_rhs=64):
    """Run the library's autotuner on trial probes of `col`; returns the chosen
    parameters (also stored in the context for this operator/precision/lattice)."""
    t = Tune()
    _check(lib().pt_autotune(op.ctx.handle, op._h, _ptr(col), int(n_colours), int(mu),
                             NOISE[noise] if isinstance(noise, str) else int(noise), int(seed), PREC[prec],
                             float(tol), int(maxit), int(trial_rhs), ctypes.byref(t)))
    return t.as_dict()


def set_tuning(op, prec, delta=None, group=None, graph_iters=None, rhs_block=None, overlap=None, evenodd=None,
               cta_threads=None, sites_per_thread=None, reset=False):
    if reset:
        _check(lib().pt_set_tuning(op.ctx.handle, op._h, PREC[prec], None))
        return
    cur = get_tuning(op, prec)
    spt = cur["sites_per_thread"] if sites_per_thread is None else int(sites_per_thread)
    t = Tune(cur["delta"] if delta is None else float(delta), cur["group"] if group is None else int(group),
             cur["graph_iters"] if graph_iters is None else int(graph_iters),
             cur["rhs_block"] if rhs_block is None else int(rhs_block),
             cur["overlap"] if overlap is None else int(overlap),
             cur["evenodd"] if evenodd is None else int(evenodd),
             cur["cta_threads"] if cta_threads is None else int(cta_threads),
             0 if op.dof == 12 else spt, 0.0)
    _check(lib().pt_set_tuning(op.ctx.handle, op._h, PREC[prec], ctypes.byref(t)))


def get_tuning(op, prec):
    t = Tune()
    _check(lib().pt_get_tuning(op.ctx.handle, op._h, PREC[prec], ctypes.byref(t)))
    return t.as_dict()


def trace_multi(op, cols, n_colours, mu, p_list, noise="z2", seed=0, set0=0, n_sets=1, dilute=True,
                prec="mixed_fp32", tol=1e-10, maxit=20000):
    """Several colourings in one batched solve.  cols: torch.int32 [n_col, N] on the
    device; n_colours: list of ints.  Returns (est[n_col, n_sets, n_p], stats)."""
    n_col = len(n_colours)
    assert cols.shape[0] == n_col and cols.is_contiguous()
    n_p = len(p_list)
    est = np.zeros((n_col, n_sets, n_p), dtype=np.complex128)
    st = Stats()
    rc = lib().pt_trace_PAinv_multi(op.ctx.handle, op._h, n_col, _ptr(cols), _ints(n_colours), int(mu),
                                    _ints(p_list), n_p, NOISE[noise] if isinstance(noise, str) else int(noise),
                                    int(seed), int(set0), int(n_sets), 1 if dilute else 0, PREC[prec], float(tol),
                                    int(maxit), _np_ptr(est), ctypes.byref(st))
    _check(rc)
    return est, st.as_dict()


def trace_nested(op, cols, n_colours, mu, p_list, noise="z2", seed=0, set0=0, n_sets=1, dilute=True,
                 prec="mixed_fp32", tol=1e-10, maxit=20000):
    """Estimates at every level of nested colourings cols [n_lev, N] (coarsest
    first) from the finest level's solves.  Returns (est[n_lev, n_sets, n_p], stats)."""
    n_lev = len(n_colours)
    assert cols.shape[0] == n_lev and cols.is_contiguous()
    n_p = len(p_list)
    est = np.zeros((n_lev, n_sets, n_p), dtype=np.complex128)
    st = Stats()
    rc = lib().pt_trace_PAinv_nested(op.ctx.handle, op._h, n_lev, _ptr(cols), _ints(n_colours), int(mu),
                                     _ints(p_list), n_p, NOISE[noise] if isinstance(noise, str) else int(noise),
                                     int(seed), int(set0), int(n_sets), 1 if dilute else 0, PREC[prec], float(tol),
                                     int(maxit), _np_ptr(est), ctypes.byref(st))
    _check(rc)
    return est, st.as_dict()


def deflation_terms(op, col, n_colours, mu, p_list, noise, seed, set0, n_sets, U, V, M):
    """pt_deflation_terms: (corr[n_sets, n_p], exact[n_p]) complex; U, V:
    torch complex128 [n_ev, N, dof] on the device, M: numpy [n_ev, n_ev]."""
    import torch
    n_p = len(p_list)
    U = torch.view_as_real(U.contiguous()).contiguous()
    V = torch.view_as_real(V.contiguous()).contiguous()
    Mh = np.ascontiguousarray(np.asarray(M, dtype=np.complex128))
    corr = np.zeros((n_sets, n_p), dtype=np.complex128)
    exact = np.zeros(n_p, dtype=np.complex128)
    _check(lib().pt_deflation_terms(op.ctx.handle, op._h, _ptr(col), int(n_colours), int(mu), _ints(p_list), n_p,
                                    NOISE[noise] if isinstance(noise, str) else int(noise), int(seed), int(set0),
                                    int(n_sets), int(Mh.shape[0]), _ptr(U), _ptr(V), _np_ptr(Mh), _np_ptr(corr),
                                    _np_ptr(exact)))
    return corr, exact


def hermitian_eig(T, n_vec):
    """pt_hermitian_eig (host only): (w[m] ascending, X[m, n_vec]) for a
    Hermitian numpy matrix T; the columns of X are the lowest eigenvectors."""
    T = np.ascontiguousarray(np.asarray(T, dtype=np.complex128))
    m = T.shape[0]
    w = np.zeros(m, dtype=np.float64)
    X = np.zeros((max(n_vec, 1), m), dtype=np.complex128)
    _check(lib().pt_hermitian_eig(int(m), _np_ptr(T), int(n_vec), _np_ptr(w), _np_ptr(X)))
    return w, X[:n_vec].T


def singular_triplets(op, n_ev, block, n_iter, start):
    """pt_singular_triplets: (U, s, V) with U, V torch complex128 [n_ev, N, dof]
    on the device and s numpy float64 [n_ev] ascending; start: torch
    complex128 [block, N, dof] on the device."""
    import torch
    if start.dtype != torch.complex128 or not start.is_cuda or start.numel() < int(block) * op.N * op.dof:
        raise ValueError("start: torch complex128 [block, N, dof] on the device")
    S = torch.view_as_real(start.contiguous()).contiguous()
    U = torch.empty((n_ev, op.N, op.dof), dtype=torch.complex128, device=start.device)
    V = torch.empty_like(U)
    s = np.zeros(n_ev, dtype=np.float64)
    _check(lib().pt_singular_triplets(op.ctx.handle, op._h, int(n_ev), int(block), int(n_iter), _ptr(S),
                                      _ptr(torch.view_as_real(U)), _ptr(torch.view_as_real(V)), _np_ptr(s)))
    return U, s, V


def eo_layout(dims, parity):
    """pt_eo_layout (host only): (site[N/2], nbr[N/2, 8]) int32."""
    Nh = int(np.prod(dims)) // 2
    site = np.zeros(Nh, dtype=np.int32)
    nbr = np.zeros((Nh, 8), dtype=np.int32)
    _check(lib().pt_eo_layout(_ints(dims), int(parity), _np_ptr(site), _np_ptr(nbr)))
    return site, nbr


def eo_host(kind, dims, step, in1, in2=None, m2=0.0, kappa=0.0, U=None, antiperiodic_t=True, blocks=None):
    """pt_eo_host (host only): step 0 S in1, 1 b'_e from in1, 2 full x from
    (in1 = x_e, in2 = b); numpy arrays [nrhs, sites] (Laplacian) or
    [nrhs, sites, 4, 3] complex (Wilson); blocks: None or the clover
    (Aee, Aoo_inv), numpy complex128 [N/2, 12, 12] each."""
    N = int(np.prod(dims))
    dt = np.float64 if kind == 0 else np.complex128
    tail = () if kind == 0 else (4, 3)
    in1 = np.ascontiguousarray(np.asarray(in1, dtype=dt))
    nrhs = in1.shape[0]
    out_sites = N if step == 2 else N // 2
    out = np.zeros((nrhs, out_sites) + tail, dtype=dt)
    U = None if U is None else np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    if in2 is not None:
        in2 = np.ascontiguousarray(np.asarray(in2, dtype=dt))
    Aee = Aoo = None
    if blocks is not None:
        Aee = np.ascontiguousarray(np.asarray(blocks[0], dtype=np.complex128)).reshape(N // 2, 12, 12)
        Aoo = np.ascontiguousarray(np.asarray(blocks[1], dtype=np.complex128)).reshape(N // 2, 12, 12)
    _check(lib().pt_eo_host(int(kind), _ints(dims), float(m2), float(kappa),
                            _np_ptr(U) if U is not None else None, 1 if antiperiodic_t else 0,
                            _np_ptr(Aee) if Aee is not None else None, _np_ptr(Aoo) if Aoo is not None else None,
                            int(step),
                            _np_ptr(in1), _np_ptr(in2) if in2 is not None else None, _np_ptr(out), int(nrhs)))
    return out


def eo_solve_host(kind, dims, b, tol=1e-10, maxit=10000, m2=0.0, kappa=0.0, U=None, antiperiodic_t=True,
                  blocks=None):
    """pt_eo_solve_host (host only): (x, iters, relres) for numpy b
    [nrhs, N] (Laplacian) or [nrhs, N, 4, 3] complex (Wilson)."""
    dt = np.float64 if kind == 0 else np.complex128
    b = np.ascontiguousarray(np.asarray(b, dtype=dt))
    nrhs, N = b.shape[0], int(np.prod(dims))
    x = np.zeros_like(b)
    iters = np.zeros(nrhs, dtype=np.int32)
    relres = np.zeros(nrhs, dtype=np.float64)
    U = None if U is None else np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    Aee = Aoo = None
    if blocks is not None:
        Aee = np.ascontiguousarray(np.asarray(blocks[0], dtype=np.complex128)).reshape(N // 2, 12, 12)
        Aoo = np.ascontiguousarray(np.asarray(blocks[1], dtype=np.complex128)).reshape(N // 2, 12, 12)
    _check(lib().pt_eo_solve_host(int(kind), _ints(dims), float(m2), float(kappa),
                                  _np_ptr(U) if U is not None else None, 1 if antiperiodic_t else 0,
                                  _np_ptr(Aee) if Aee is not None else None, _np_ptr(Aoo) if Aoo is not None else None,
                                  _np_ptr(b), _np_ptr(x), int(nrhs), float(tol), int(maxit), _np_ptr(iters),
                                  _np_ptr(relres)))
    return x, iters, relres


def eo_solve(op, b, tol=1e-10, maxit=10000, blocks=None):
    """pt_eo_solve: (x, iters, relres) for full fields b [nrhs, N(, 4, 3)] on the device."""
    import torch
    b = _eo_field(op, b, op.N, "b")
    x = torch.empty_like(b)
    iters = np.zeros(b.shape[0], dtype=np.int32)
    relres = np.zeros(b.shape[0], dtype=np.float64)
    ae, ao = _eo_blocks(op, blocks)
    _check(lib().pt_eo_solve(op.ctx.handle, op._h, ae, ao, _eo_ptr(b), _eo_ptr(x), int(b.shape[0]), float(tol),
                             int(maxit), _np_ptr(iters), _np_ptr(relres)))
    return x, iters, relres


def trace_eo(op, col, n_colours, mu, p_list, noise="z2", seed=0, set0=0, n_sets=1, tol=1e-10, maxit=20000,
             delta=1e-5):
    """pt_trace_PAinv_eo (Laplacian, even-odd): (est[n_sets, n_p] complex, stats)."""
    est = np.zeros((n_sets, len(p_list)), dtype=np.complex128)
    st = Stats()
    _check(lib().pt_trace_PAinv_eo(op.ctx.handle, op._h, _ptr(col), int(n_colours), int(mu), _ints(p_list),
                                   len(p_list), NOISE[noise] if isinstance(noise, str) else int(noise), int(seed),
                                   int(set0), int(n_sets), float(tol), int(maxit), float(delta), _np_ptr(est),
                                   ctypes.byref(st)))
    return est, st.as_dict()


def trace_eo_host(dims, m2, col, n_colours, mu, p_list, noise="z2", seed=0, set0=0, n_sets=1, tol=1e-10,
                  maxit=20000, delta=1e-5):
    """pt_trace_PAinv_eo_host (no GPU): (est[n_sets, n_p] complex, stats)."""
    col = np.ascontiguousarray(np.asarray(col, dtype=np.int32))
    est = np.zeros((n_sets, len(p_list)), dtype=np.complex128)
    st = Stats()
    _check(lib().pt_trace_PAinv_eo_host(_ints(dims), float(m2), _np_ptr(col), int(n_colours), int(mu), _ints(p_list),
                                        len(p_list), NOISE[noise] if isinstance(noise, str) else int(noise),
                                        int(seed), int(set0), int(n_sets), float(tol), int(maxit), float(delta),
                                        _np_ptr(est), ctypes.byref(st)))
    return est, st.as_dict()


def wmg_solve(op, b, block=2, nv=4, sweeps=20, nu=2, omega=0.8, restart=30, seed=0, tol=1e-10, maxit=5000, csw=0.0):
    """pt_wmg_solve (Wilson): (x, iters, relres) for b torch complex128 [nrhs, N, 4, 3] on the device."""
    import torch
    b = _eo_field(op, b, op.N, "b")
    x = torch.empty_like(b)
    iters = np.zeros(b.shape[0], dtype=np.int32)
    relres = np.zeros(b.shape[0], dtype=np.float64)
    _check(lib().pt_wmg_solve(op.ctx.handle, op._h, float(csw), int(block), int(nv), int(sweeps), int(nu), float(omega),
                              int(restart), int(seed), _eo_ptr(b), _eo_ptr(x), int(b.shape[0]), float(tol),
                              int(maxit), _np_ptr(iters), _np_ptr(relres)))
    return x, iters, relres


def _wmg_links(dims, U):
    U = np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    if U.shape != (int(np.prod(dims)), 4, 3, 3):
        raise ValueError("links: complex128 [N, 4, 3, 3]")
    return U


def wmg_solve_host(dims, U, kappa, b, block=2, nv=4, sweeps=20, nu=2, omega=0.8, restart=30, seed=0, tol=1e-10,
                   maxit=5000, antiperiodic_t=True, csw=0.0):
    """pt_wmg_solve_host (no GPU): (x, iters, relres) for numpy b [nrhs, N, 4, 3] complex."""
    U = _wmg_links(dims, U)
    b = np.ascontiguousarray(np.asarray(b, dtype=np.complex128))
    x = np.zeros_like(b)
    iters = np.zeros(b.shape[0], dtype=np.int32)
    relres = np.zeros(b.shape[0], dtype=np.float64)
    _check(lib().pt_wmg_solve_host(_ints(dims), _np_ptr(U), float(kappa), float(csw), 1 if antiperiodic_t else 0,
                                   int(block),
                                   int(nv), int(sweeps), int(nu), float(omega), int(restart), int(seed), _np_ptr(b),
                                   _np_ptr(x), int(b.shape[0]), float(tol), int(maxit), _np_ptr(iters),
                                   _np_ptr(relres)))
    return x, iters, relres


def wmg_setup_host(dims, U, kappa, block=2, nv=4, sweeps=20, omega=0.8, seed=0, antiperiodic_t=True, csw=0.0):
    """pt_wmg_setup_host (no GPU): (P [Nc, 2, nv, block^4, 6], Ac [Nc, 9, 2 nv, 2 nv]) complex."""
    U = _wmg_links(dims, U)
    Nc = int(np.prod([d // block for d in dims]))
    P = np.zeros((Nc, 2, nv, block ** 4, 6), dtype=np.complex128)
    Ac = np.zeros((Nc, 9, 2 * nv, 2 * nv), dtype=np.complex128)
    _check(lib().pt_wmg_setup_host(_ints(dims), _np_ptr(U), float(kappa), float(csw), 1 if antiperiodic_t else 0,
                                   int(block),
                                   int(nv), int(sweeps), float(omega), int(seed), _np_ptr(P), _np_ptr(Ac)))
    return P, Ac


def mg_solve(op, b, block=2, nu=2, omega=0.8, tol=1e-10, maxit=10000):
    """pt_mg_solve (Laplacian): (x, iters, relres) for b torch float64 [nrhs, N] on the device."""
    import torch
    b = _eo_field(op, b, op.N, "b")
    x = torch.empty_like(b)
    iters = np.zeros(b.shape[0], dtype=np.int32)
    relres = np.zeros(b.shape[0], dtype=np.float64)
    _check(lib().pt_mg_solve(op.ctx.handle, op._h, int(block), int(nu), float(omega), _ptr(b), _ptr(x),
                             int(b.shape[0]), float(tol), int(maxit), _np_ptr(iters), _np_ptr(relres)))
    return x, iters, relres


def mg_solve_host(dims, m2, b, block=2, nu=2, omega=0.8, tol=1e-10, maxit=10000):
    """pt_mg_solve_host (no GPU): (x, iters, relres) for numpy b [nrhs, N]."""
    b = np.ascontiguousarray(np.asarray(b, dtype=np.float64))
    x = np.zeros_like(b)
    iters = np.zeros(b.shape[0], dtype=np.int32)
    relres = np.zeros(b.shape[0], dtype=np.float64)
    _check(lib().pt_mg_solve_host(_ints(dims), float(m2), int(block), int(nu), float(omega), _np_ptr(b), _np_ptr(x),
                                  int(b.shape[0]), float(tol), int(maxit), _np_ptr(iters), _np_ptr(relres)))
    return x, iters, relres


def mg_cycle_host(dims, m2, r, block=2, nu=2, omega=0.8):
    """pt_mg_cycle_host (no GPU): M r for one numpy vector r [N]."""
    r = np.ascontiguousarray(np.asarray(r, dtype=np.float64).reshape(-1))
    out = np.zeros_like(r)
    _check(lib().pt_mg_cycle_host(_ints(dims), float(m2), int(block), int(nu), float(omega), _np_ptr(r),
                                  _np_ptr(out)))
    return out


def _eo_field(op, x, sites, name):
    import torch
    want = (sites,) if op.dof == 1 else (sites, 4, 3)
    dt = torch.float64 if op.dof == 1 else torch.complex128
    if x.dtype != dt or not x.is_cuda or tuple(x.shape[1:]) != want:
        raise ValueError("%s: %s [nrhs, %s] on the device" % (name, dt, ", ".join(map(str, want))))
    return x.contiguous()


def _eo_ptr(t):
    import torch
    return _ptr(torch.view_as_real(t) if t.is_complex() else t)


def _eo_blocks(op, blocks):
    """(Aee, Aoo_inv) device pointers, or NULLs"""
    import torch
    if blocks is None:
        return _ptr(None), _ptr(None)
    out = []
    for B in blocks:
        if B.dtype != torch.complex128 or not B.is_cuda or tuple(B.shape) != (op.N // 2, 12, 12) or \
                not B.is_contiguous():
            raise ValueError("blocks: contiguous torch complex128 [N/2, 12, 12] on the device")
        out.append(_ptr(torch.view_as_real(B)))
    return out[0], out[1]


def eo_clover_blocks(op, csw):
    """pt_eo_clover_blocks: (Aee, Aoo_inv), torch complex128 [N/2, 12, 12] on the device."""
    import torch
    Aee = torch.empty((op.N // 2, 12, 12), dtype=torch.complex128, device="cuda:%d" % op.ctx.device)
    Aoo = torch.empty_like(Aee)
    _check(lib().pt_eo_clover_blocks(op.ctx.handle, op._h, float(csw), _ptr(torch.view_as_real(Aee)),
                                     _ptr(torch.view_as_real(Aoo))))
    return Aee, Aoo


def eo_schur(op, xe, blocks=None):
    """pt_eo_schur: S xe for even half fields xe [nrhs, N/2(, 4, 3)]; blocks:
    the clover (Aee, Aoo_inv) or None."""
    import torch
    xe = _eo_field(op, xe, op.N // 2, "xe")
    ye = torch.empty_like(xe)
    ae, ao = _eo_blocks(op, blocks)
    _check(lib().pt_eo_schur(op.ctx.handle, op._h, ae, ao, _eo_ptr(xe), _eo_ptr(ye), int(xe.shape[0])))
    return ye


def eo_prepare(op, b, blocks=None):
    """pt_eo_prepare: b'_e [nrhs, N/2(, 4, 3)] from full fields b [nrhs, N(, 4, 3)]."""
    import torch
    b = _eo_field(op, b, op.N, "b")
    be = torch.empty((b.shape[0], op.N // 2) + tuple(b.shape[2:]), dtype=b.dtype, device=b.device)
    _, ao = _eo_blocks(op, blocks)
    _check(lib().pt_eo_prepare(op.ctx.handle, op._h, ao, _eo_ptr(b), _eo_ptr(be), int(b.shape[0])))
    return be


def eo_reconstruct(op, xe, b, blocks=None):
    """pt_eo_reconstruct: full solutions x [nrhs, N(, 4, 3)] from xe and b."""
    import torch
    xe = _eo_field(op, xe, op.N // 2, "xe")
    b = _eo_field(op, b, op.N, "b")
    if xe.shape[0] != b.shape[0]:
        raise ValueError("xe and b hold different numbers of right-hand sides")
    x = torch.empty_like(b)
    _, ao = _eo_blocks(op, blocks)
    _check(lib().pt_eo_reconstruct(op.ctx.handle, op._h, ao, _eo_ptr(xe), _eo_ptr(b), _eo_ptr(x),
                                   int(b.shape[0])))
    return x


def clover_blocks_host(dims, U, kappa, csw):
    """pt_clover_blocks_host: C(x) as numpy complex128 [N, 12, 12] from numpy
    links [N, 4, 3, 3] (host only)."""
    U = np.ascontiguousarray(np.asarray(U, dtype=np.complex128))
    N = int(np.prod(dims))
    if U.shape != (N, 4, 3, 3):
        raise ValueError("links: complex128 [N, 4, 3, 3]")
    out = np.zeros((N, 12, 12), dtype=np.complex128)
    _check(lib().pt_clover_blocks_host(_ints(dims), _np_ptr(U), float(kappa), float(csw), _np_ptr(out)))
    return out


def site_blocks_invert_host(B, shift=1.0):
    """pt_site_blocks_invert_host: (shift 1 + B)^{-1} per block, numpy [n, 12, 12]."""
    B = np.ascontiguousarray(np.asarray(B, dtype=np.complex128))
    if B.ndim != 3 or B.shape[1:] != (12, 12):
        raise ValueError("blocks: complex128 [n, 12, 12]")
    out = np.zeros_like(B)
    _check(lib().pt_site_blocks_invert_host(int(B.shape[0]), _np_ptr(B), float(shift), _np_ptr(out)))
    return out


def clover_blocks(op, csw):
    """pt_clover_blocks: C(x) as torch complex128 [N, 12, 12] on the device."""
    import torch
    if op.dof != 12:
        raise ValueError("a Wilson-Dirac operator is required")
    out = torch.empty((op.N, 12, 12), dtype=torch.complex128, device="cuda:%d" % op.ctx.device)
    _check(lib().pt_clover_blocks(op.ctx.handle, op._h, float(csw), _ptr(torch.view_as_real(out))))
    return out


def site_blocks_apply(ctx, B, x, y=None, beta=0.0):
    """pt_site_blocks_apply: beta y + B x per site; B [N, 12, 12], x [nrhs, N, 4, 3]
    (torch complex128 on the device)."""
    import torch
    N = B.shape[0]
    if B.shape != (N, 12, 12) or x.dim() != 4 or tuple(x.shape[1:]) != (N, 4, 3) or \
            B.dtype != torch.complex128 or x.dtype != torch.complex128:
        raise ValueError("B: complex128 [N, 12, 12], x: complex128 [nrhs, N, 4, 3]")
    B, x = B.contiguous(), x.contiguous()
    if y is None:
        y, beta = torch.zeros_like(x), 0.0
    elif y.shape != x.shape or y.dtype != x.dtype or not y.is_contiguous():
        raise ValueError("y: contiguous, the shape and type of x")
    _check(lib().pt_site_blocks_apply(ctx.handle, int(N), _ptr(torch.view_as_real(B)), _ptr(torch.view_as_real(x)),
                                      float(beta), _ptr(torch.view_as_real(y)), int(x.shape[0])))
    return y


def site_blocks_invert(ctx, B, shift=1.0):
    """pt_site_blocks_invert: (shift 1 + B)^{-1} per site, torch [N, 12, 12] on the device."""
    import torch
    B = B.contiguous()
    out = torch.empty_like(B)
    _check(lib().pt_site_blocks_invert(ctx.handle, int(B.shape[0]), _ptr(torch.view_as_real(B)), float(shift),
                                       _ptr(torch.view_as_real(out))))
    return out


def grad(op, col, n_colours, mu, p, noise="z2", seed=0, set0=0, n_sets=1, dilute=True, prec="mixed_fp32",
         tol=1e-10, maxit=20000, links=False):
    """Adjoint gradient: returns (est[n_sets], dparam, G, Gbar, stats); G/Gbar are
    torch complex128 [N, 4, 3, 3] when links=True (Wilson only), else None."""
    import torch
    est = np.zeros(n_sets, dtype=np.complex128)
    dp = np.zeros(1, dtype=np.complex128)
    G = Gb = None
    if links:
        G = torch.empty((op.N, 4, 3, 3), dtype=torch.complex128, device=col.device)
        Gb = torch.empty_like(G)
    st = Stats()
    rc = lib().pt_grad(op.ctx.handle, op._h, _ptr(col), int(n_colours), int(mu), int(p),
                       NOISE[noise] if isinstance(noise, str) else int(noise), int(seed), int(set0), int(n_sets),
                       1 if dilute else 0, PREC[prec], float(tol), int(maxit), _np_ptr(est), _np_ptr(dp),
                       _ptr(G), _ptr(Gb), ctypes.byref(st))
    _check(rc)
    return est, complex(dp[0]), G, Gb, st.as_dict()
