"""ctypes binding of the C ABI in include/lsm.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Device
buffers are torch tensors (contiguous, on the handle's device); their
``data_ptr()`` is passed through unchanged.  No step of the method runs in
Python: when ``_lib/liblsm.so`` is missing, loading fails with an error.
"""
from __future__ import annotations

import ctypes as ct
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "liblsm.so")

LSM_OK = 0
LSM_ERR_ARG = -1
LSM_ERR_CUDA = -2
LSM_ERR_OOM = -3
LSM_ERR_BREAKDOWN = -4
LSM_ERR_NOCONV = -5
LSM_ERR_TIMEOUT = -6
LSM_WARN_SOURCE_ON_NODE = 1
LSM_FP64 = 0
LSM_MIXED = 1
LSM_GREEN_EXACT = 0
LSM_GREEN_PAPER = 1
LSM_KERNEL_DIFF, LSM_KERNEL_H = 0, 1
LSM_RESIDUAL_DFLOAT, LSM_RESIDUAL_FP64 = 0, 1

STATUS_NAMES = {0: "LSM_OK", -1: "LSM_ERR_ARG", -2: "LSM_ERR_CUDA", -3: "LSM_ERR_OOM", -4: "LSM_ERR_BREAKDOWN",
                -5: "LSM_ERR_NOCONV", -6: "LSM_ERR_TIMEOUT", 1: "LSM_WARN_SOURCE_ON_NODE"}

# every symbol the header declares, in declaration order
EXPORTS = ("lsm_default_opts", "lsm_create", "lsm_create_shared", "lsm_source", "lsm_source_moments", "lsm_apply", "lsm_apply_c64",
           "lsm_apply_df", "lsm_adjoint", "lsm_solve", "lsm_solve_batched", "lsm_solve_adjoint", "lsm_set_contrast", "lsm_gradient",
           "lsm_source_gradient", "lsm_time_traces", "lsm_seismograms", "lsm_set_schedule", "lsm_get_schedule", "lsm_autotune", "lsm_dot_c64", "lsm_launch_count", "lsm_timer_start", "lsm_timer_read",
           "lsm_apply_static", "lsm_destroy", "lsm_last_error")


class lsm_opts(ct.Structure):
    _fields_ = [("precision", ct.c_int), ("green", ct.c_int), ("tol", ct.c_double), ("maxit", ct.c_int),
                ("inner_tol", ct.c_double), ("max_outer", ct.c_int), ("taper", ct.c_int), ("graph", ct.c_int),
                ("kernel", ct.c_int), ("residual", ct.c_int), ("fused_dots", ct.c_int)]


class LSMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_lib = None


def load(path: str = LIB_PATH):
    """Load liblsm.so (once) and declare the prototypes."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"liblsm.so not found at {path}: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    lib = ct.CDLL(path)
    vp, i, d = ct.c_void_p, ct.c_int, ct.c_double
    lib.lsm_default_opts.argtypes = [ct.POINTER(lsm_opts)]
    lib.lsm_default_opts.restype = None
    lib.lsm_create.argtypes = [ct.POINTER(vp), ct.POINTER(i), d, d, d, d, vp, vp, d, ct.POINTER(lsm_opts), vp]
    lib.lsm_create.restype = i
    lib.lsm_create_shared.argtypes = [ct.POINTER(vp), vp, d]
    lib.lsm_create_shared.restype = i
    lib.lsm_source.argtypes = [vp, ct.POINTER(d), ct.POINTER(d), vp]
    lib.lsm_source.restype = i
    lib.lsm_source_moments.argtypes = [vp, i, ct.POINTER(d), ct.POINTER(d), ct.POINTER(vp)]
    lib.lsm_source_moments.restype = i
    lib.lsm_dot_c64.argtypes = [vp, ct.c_longlong, vp, vp, ct.POINTER(d)]
    lib.lsm_dot_c64.restype = i
    lib.lsm_set_schedule.argtypes = [vp, i, ct.POINTER(i)]
    lib.lsm_set_schedule.restype = i
    lib.lsm_get_schedule.argtypes = [vp, i, ct.POINTER(i)]
    lib.lsm_get_schedule.restype = i
    lib.lsm_autotune.argtypes = [vp, i, i, ct.POINTER(i), ct.POINTER(i)]
    lib.lsm_autotune.restype = i
    for name in ("lsm_apply", "lsm_apply_c64", "lsm_apply_df", "lsm_adjoint"):
        getattr(lib, name).argtypes = [vp, vp, vp]
        getattr(lib, name).restype = i
    lib.lsm_solve.argtypes = [vp, vp, vp, ct.POINTER(i), ct.POINTER(d)]
    lib.lsm_solve.restype = i
    lib.lsm_solve_batched.argtypes = [i, ct.POINTER(vp), ct.POINTER(vp), ct.POINTER(vp), ct.POINTER(i),
                                      ct.POINTER(d), ct.POINTER(i)]
    lib.lsm_solve_batched.restype = i
    lib.lsm_solve_adjoint.argtypes = [vp, vp, vp, ct.POINTER(i), ct.POINTER(d)]
    lib.lsm_solve_adjoint.restype = i
    lib.lsm_set_contrast.argtypes = [vp, vp, vp]
    lib.lsm_set_contrast.restype = i
    lib.lsm_gradient.argtypes = [vp, vp, vp, vp, vp, i]
    lib.lsm_gradient.restype = i
    lib.lsm_source_gradient.argtypes = [vp, ct.POINTER(d), vp, ct.POINTER(d)]
    lib.lsm_source_gradient.restype = i
    lib.lsm_time_traces.argtypes = [i, d, i, vp, i, d, d, d, vp, vp]
    lib.lsm_time_traces.restype = i
    lib.lsm_seismograms.argtypes = [vp, i, d, ct.POINTER(d), ct.POINTER(d), i, ct.POINTER(i), i, d, d, d, vp, i,
                                     ct.POINTER(i), ct.POINTER(d)]
    lib.lsm_seismograms.restype = i
    lib.lsm_launch_count.argtypes = [vp]
    lib.lsm_launch_count.restype = ct.c_longlong
    lib.lsm_timer_start.argtypes = [vp, i]
    lib.lsm_timer_start.restype = i
    lib.lsm_timer_read.argtypes = [vp, ct.POINTER(d), ct.POINTER(ct.c_longlong), ct.POINTER(ct.c_longlong)]
    lib.lsm_timer_read.restype = i
    lib.lsm_apply_static.argtypes = [vp, vp, vp]
    lib.lsm_apply_static.restype = i
    lib.lsm_destroy.argtypes = [vp]
    lib.lsm_destroy.restype = None
    lib.lsm_last_error.argtypes = [vp]
    lib.lsm_last_error.restype = ct.c_char_p
    _lib = lib
    return lib


def _ptr(t: torch.Tensor, dtype, numel):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != numel:
        raise TypeError(f"expected a contiguous {dtype} tensor of {numel} elements, got {t.dtype} {tuple(t.shape)}")
    return ct.c_void_p(t.data_ptr())


def _check(code, h=None, allow=()):
    if code != LSM_OK and code not in allow:
        msg = load().lsm_last_error(h)
        raise LSMError(code, msg.decode() if msg else "")
    return code


def lsm_default_opts(**kw) -> lsm_opts:
    o = lsm_opts()
    load().lsm_default_opts(ct.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def lsm_last_error(h=None) -> str:
    m = load().lsm_last_error(h)
    return m.decode() if m else ""


class Handle:
    """Owner of one lsm_t.  Fields are the grid n = (nx, ny, nz) and N = nx ny nz."""

    def __init__(self, ptr, n, precision, device):
        self.ptr = ptr
        self.n = tuple(n)
        self.N = n[0] * n[1] * n[2]
        self.precision = precision
        self.device = device

    def __del__(self):
        try:
            if self.ptr:
                load().lsm_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass


def lsm_create(n, dx, lambda0, mu0, rho0, dC: torch.Tensor, drho: torch.Tensor, omega, opts: lsm_opts | None = None,
               stream: torch.cuda.Stream | None = None) -> Handle:
    lib = load()
    nx, ny, nz = (int(v) for v in n)
    N = nx * ny * nz
    arr = (ct.c_int * 3)(nx, ny, nz)
    st = (stream or torch.cuda.current_stream(dC.device)).cuda_stream
    out = ct.c_void_p()
    o = opts if opts is not None else lsm_default_opts()
    code = lib.lsm_create(ct.byref(out), arr, float(dx), float(lambda0), float(mu0), float(rho0),
                          _ptr(dC, torch.float64, 21 * N), _ptr(drho, torch.float64, N), float(omega), ct.byref(o),
                          ct.c_void_p(st))
    _check(code, None)
    return Handle(out, (nx, ny, nz), o.precision, dC.device)


def lsm_create_shared(base: Handle, omega) -> Handle:
    out = ct.c_void_p()
    _check(load().lsm_create_shared(ct.byref(out), base.ptr, float(omega)), None)
    return Handle(out, base.n, base.precision, base.device)


def lsm_source(h: Handle, M6, xs, u0: torch.Tensor) -> int:
    M = (ct.c_double * 6)(*[float(v) for v in M6])
    x = (ct.c_double * 3)(*[float(v) for v in xs])
    return _check(load().lsm_source(h.ptr, M, x, _ptr(u0, torch.complex128, 3 * h.N)), h.ptr,
                  allow=(LSM_WARN_SOURCE_ON_NODE,))


def lsm_source_moments(h: Handle, Ms, xs, u0s) -> int:
    """Background fields of several moment tensors (rows of Ms, Voigt order) at one position."""
    Ms = [[float(v) for v in m] for m in Ms]
    nm = len(Ms)
    if len(u0s) != nm:
        raise ValueError("lsm_source_moments: one output per moment tensor")
    M = (ct.c_double * (6 * nm))(*[v for m in Ms for v in m])
    x = (ct.c_double * 3)(*[float(v) for v in xs])
    outs = (ct.c_void_p * nm)(*[_ptr(u, torch.complex128, 3 * h.N) for u in u0s])
    return _check(load().lsm_source_moments(h.ptr, nm, M, x, outs), h.ptr, allow=(LSM_WARN_SOURCE_ON_NODE,))


def lsm_apply(h: Handle, u: torch.Tensor, Au: torch.Tensor) -> None:
    _check(load().lsm_apply(h.ptr, _ptr(u, torch.complex128, 3 * h.N), _ptr(Au, torch.complex128, 3 * h.N)), h.ptr)


def lsm_apply_c64(h: Handle, u: torch.Tensor, Au: torch.Tensor) -> None:
    _check(load().lsm_apply_c64(h.ptr, _ptr(u, torch.complex64, 3 * h.N), _ptr(Au, torch.complex64, 3 * h.N)), h.ptr)


def lsm_apply_df(h: Handle, u: torch.Tensor, Au: torch.Tensor) -> None:
    _check(load().lsm_apply_df(h.ptr, _ptr(u, torch.complex128, 3 * h.N), _ptr(Au, torch.complex128, 3 * h.N)), h.ptr)


def lsm_adjoint(h: Handle, v: torch.Tensor, AHv: torch.Tensor) -> None:
    _check(load().lsm_adjoint(h.ptr, _ptr(v, torch.complex128, 3 * h.N), _ptr(AHv, torch.complex128, 3 * h.N)), h.ptr)


def lsm_solve(h: Handle, b: torch.Tensor, x: torch.Tensor, check=True):
    """Returns (status, iterations, relres)."""
    it = ct.c_int(0)
    rr = ct.c_double(0.0)
    code = load().lsm_solve(h.ptr, _ptr(b, torch.complex128, 3 * h.N), _ptr(x, torch.complex128, 3 * h.N),
                            ct.byref(it), ct.byref(rr))
    if check:
        _check(code, h.ptr)
    return code, it.value, rr.value


def lsm_solve_batched(hs, bs, xs, check=True):
    """Returns (status, [iterations], [relres], [per-system status])."""
    k = len(hs)
    H = (ct.c_void_p * k)(*[h.ptr.value if isinstance(h.ptr, ct.c_void_p) else h.ptr for h in hs])
    B = (ct.c_void_p * k)(*[_ptr(b, torch.complex128, 3 * h.N).value for b, h in zip(bs, hs)])
    X = (ct.c_void_p * k)(*[_ptr(x, torch.complex128, 3 * h.N).value for x, h in zip(xs, hs)])
    it = (ct.c_int * k)()
    rr = (ct.c_double * k)()
    stt = (ct.c_int * k)()
    code = load().lsm_solve_batched(k, H, B, X, it, rr, stt)
    if check:
        _check(code, hs[0].ptr)
    return code, list(it), list(rr), list(stt)


def lsm_solve_adjoint(h: Handle, b: torch.Tensor, x: torch.Tensor, check=True):
    """Solve A^H x = b.  Returns (status, iterations, relres)."""
    it = ct.c_int(0)
    rr = ct.c_double(0.0)
    code = load().lsm_solve_adjoint(h.ptr, _ptr(b, torch.complex128, 3 * h.N), _ptr(x, torch.complex128, 3 * h.N),
                                    ct.byref(it), ct.byref(rr))
    if check:
        _check(code, h.ptr)
    return code, it.value, rr.value


def lsm_set_contrast(h: Handle, dC: torch.Tensor, drho: torch.Tensor) -> None:
    _check(load().lsm_set_contrast(h.ptr, _ptr(dC, torch.float64, 21 * h.N), _ptr(drho, torch.float64, h.N)), h.ptr)


def lsm_gradient(h: Handle, u: torch.Tensor, lam: torch.Tensor, gC: torch.Tensor, grho: torch.Tensor,
                 accumulate: bool = False) -> None:
    _check(load().lsm_gradient(h.ptr, _ptr(u, torch.complex128, 3 * h.N), _ptr(lam, torch.complex128, 3 * h.N),
                               _ptr(gC, torch.float64, 21 * h.N), _ptr(grho, torch.float64, h.N),
                               1 if accumulate else 0), h.ptr)


def lsm_source_gradient(h: Handle, xs, lam: torch.Tensor):
    x = (ct.c_double * 3)(*[float(v) for v in xs])
    g = (ct.c_double * 6)()
    _check(load().lsm_source_gradient(h.ptr, x, _ptr(lam, torch.complex128, 3 * h.N), g), h.ptr)
    return list(g)


def lsm_time_traces(spectra: torch.Tensor, df, nt, dt, fp, t0, stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """spectra: device complex128 (nf, ntr) at f_k = k df -> device float64 traces (ntr, nt)."""
    nf, ntr = spectra.shape
    out = torch.empty((ntr, nt), dtype=torch.float64, device=spectra.device)
    st = (stream or torch.cuda.current_stream(spectra.device)).cuda_stream
    _check(load().lsm_time_traces(int(nf), float(df), int(ntr), _ptr(spectra, torch.complex128, nf * ntr), int(nt),
                                  float(dt), float(fp), float(t0), _ptr(out, torch.float64, ntr * nt), ct.c_void_p(st)))
    return out


def lsm_seismograms(base: Handle, nf, df, M6, xs, receivers, nt, dt, fp, t0, wave=32):
    """Receiver traces of one source over f_k = k df (k < nf): returns (status, traces (nrec, 3, nt)
    device float64, iterations [nf], relres [nf]).  receivers: (nrec, 3) node indices (ix, iy, iz)."""
    rec = [int(v) for r in receivers for v in r]
    nrec = len(rec) // 3
    out = torch.empty((nrec, 3, int(nt)), dtype=torch.float64, device=base.device)
    M = (ct.c_double * 6)(*[float(v) for v in M6])
    x = (ct.c_double * 3)(*[float(v) for v in xs])
    R = (ct.c_int * len(rec))(*rec)
    it = (ct.c_int * int(nf))()
    rr = (ct.c_double * int(nf))()
    code = load().lsm_seismograms(base.ptr, int(nf), float(df), M, x, nrec, R, int(nt), float(dt), float(fp), float(t0),
                                  _ptr(out, torch.float64, nrec * 3 * int(nt)), int(wave), it, rr)
    _check(code, base.ptr, allow=(LSM_WARN_SOURCE_ON_NODE,))
    return code, out, list(it), list(rr)


def lsm_launch_count(h: Handle) -> int:
    return int(load().lsm_launch_count(h.ptr))


def lsm_set_schedule(h: Handle, precision: int, v) -> None:
    arr = (ct.c_int * 6)(*[int(x) for x in v])
    _check(load().lsm_set_schedule(h.ptr, int(precision), arr), h.ptr)


def lsm_get_schedule(h: Handle, precision: int):
    arr = (ct.c_int * 6)()
    _check(load().lsm_get_schedule(h.ptr, int(precision), arr), h.ptr)
    return list(arr)


def lsm_autotune(h: Handle, nsys: int = 1, reps: int = 2):
    """Time every FFT schedule variant per stage on batches of nsys systems and keep the fastest;
    returns (v64, v32)."""
    a = (ct.c_int * 6)()
    b = (ct.c_int * 6)()
    _check(load().lsm_autotune(h.ptr, int(nsys), int(reps), a, b), h.ptr)
    return list(a), list(b)


def lsm_dot_c64(h: Handle, a: torch.Tensor, b: torch.Tensor) -> complex:
    """conj(a) . b of two complex64 device vectors with the mixed solver's inner-product accumulation."""
    if a.numel() != b.numel():
        raise ValueError("lsm_dot_c64: vectors of different lengths")
    out = (ct.c_double * 2)()
    n = a.numel()
    _check(load().lsm_dot_c64(h.ptr, n, _ptr(a, torch.complex64, n), _ptr(b, torch.complex64, n), out), h.ptr)
    return complex(out[0], out[1])


def lsm_timer_start(h: Handle, enable: bool = True) -> None:
    _check(load().lsm_timer_start(h.ptr, 1 if enable else 0), h.ptr)


def lsm_timer_read(h: Handle):
    """Returns (ms[12], launches[12], applies[2]) since lsm_timer_start; slot = 6 * p + stage, p = 1 for FP32."""
    ms = (ct.c_double * 12)()
    nl = (ct.c_longlong * 12)()
    ap = (ct.c_longlong * 2)()
    _check(load().lsm_timer_read(h.ptr, ms, nl, ap), h.ptr)
    return list(ms), list(nl), list(ap)


def lsm_apply_static(h: Handle, u: torch.Tensor, Au: torch.Tensor) -> None:
    """FP64 apply whose workspace is the library's static device array (no device allocation)."""
    _check(load().lsm_apply_static(h.ptr, _ptr(u, torch.complex128, 3 * h.N), _ptr(Au, torch.complex128, 3 * h.N)),
           h.ptr)
