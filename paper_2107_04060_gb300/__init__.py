"""Python binding of libbiotmg.so, the GB300 (sm_103a) monolithic-multigrid solver for the
reduced-quadrature three-field Biot system (arXiv 2107.04060).

The binding only marshals arguments: every step of assembly, relaxation, transfer, coarse
solve and Krylov iteration runs in the library's CUDA kernels.  PyTorch provides device
memory and streams.  There is no CPU fallback: importing this package fails if the shared
library has not been built (``python paper_2107_04060_gb300/build.py``), and every call
fails if no CUDA device is usable.

Names follow the C ABI of ``include/biotmg.h``: ``assemble``, ``setup_hierarchy``,
``vcycle``, ``apply``, ``residual``, ``fgmres_solve`` (see that header for the vector layout).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbiotmg.so")
if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python paper_2107_04060_gb300/build.py` "
                      "(there is no CPU fallback)")
lib = C.CDLL(LIB_PATH)

TYPES = ("ux", "uy", "bh", "bv", "bd", "wh", "wv", "wd", "pL", "pU")
VANKA, BSR, BSR_EXACT = 0, 1, 2
FP64, FP32 = 0, 1
STATUS = {0: "converged", 1: "maxit", 2: "breakdown", 3: "diverged"}


class MgOpts(C.Structure):
    _fields_ = [("smoother", C.c_int), ("nu1", C.c_int), ("nu2", C.c_int), ("omega", C.c_double),
                ("omega_J", C.c_double), ("n_coarse", C.c_int), ("precision", C.c_int),
                ("p_shift", C.c_double), ("gamma", C.c_int), ("coarse_op", C.c_int),
                ("patch_solve", C.c_int)]


class KrylovOpts(C.Structure):
    _fields_ = [("rtol", C.c_double), ("restart", C.c_int), ("maxit", C.c_int),
                ("x0_is_zero", C.c_int), ("arnoldi", C.c_int)]


ARNOLDI = {"fp64": 0, "mixed": 1}


class SolveInfo(C.Structure):
    _fields_ = [("iters", C.c_int), ("restarts", C.c_int), ("status", C.c_int),
                ("relres", C.c_double), ("relres_est", C.c_double), ("solve_ms", C.c_double)]


_vp = C.c_void_p
_sig = {
    "bmg_pitch": (C.c_int, [C.c_int]),
    "bmg_block_len": (C.c_size_t, [C.c_int]),
    "bmg_vector_len": (C.c_size_t, [C.c_int]),
    "bmg_free_dofs": (C.c_size_t, [C.c_int]),
    "bmg_assemble": (C.c_int, [C.c_int, C.c_double, C.c_double, _vp, C.c_double, C.c_double,
                               C.c_double, C.c_double, _vp, C.POINTER(_vp)]),
    "bmg_assemble_divdiv": (C.c_int, [C.c_int, C.c_double, C.c_double, _vp, C.c_double, C.c_double,
                                      C.c_double, C.c_double, C.c_int, _vp, C.POINTER(_vp)]),
    "bmg_assemble_logk": (C.c_int, [C.c_int, C.c_double, C.c_double, _vp, C.c_double, C.c_double,
                                    C.c_double, _vp, C.POINTER(_vp)]),
    "bmg_adjoint_gradient": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "bmg_backward_euler_rhs": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "bmg_apply": (C.c_int, [_vp, _vp, _vp, _vp]),
    "bmg_residual": (C.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "bmg_setup_hierarchy": (C.c_int, [_vp, C.POINTER(MgOpts), _vp, C.POINTER(_vp)]),
    "bmg_vcycle": (C.c_int, [_vp, _vp, _vp, _vp]),
    "bmg_fgmres_solve": (C.c_int, [_vp, _vp, _vp, C.POINTER(KrylovOpts), C.POINTER(SolveInfo), _vp]),
    "bmg_fgmres_solve_host": (C.c_int, [_vp, _vp, _vp, C.POINTER(KrylovOpts), C.POINTER(SolveInfo), _vp]),
    "bmg_fgmres_solve_noalloc": (C.c_int, [_vp, _vp, _vp, C.POINTER(KrylovOpts), C.POINTER(SolveInfo), _vp]),
    "bmg_noalloc_capacity": (C.c_size_t, []),
    "bmg_system_n": (C.c_int, [_vp]),
    "bmg_hierarchy_levels": (C.c_int, [_vp]),
    "bmg_hierarchy_tile": (C.c_int, [_vp, C.c_int, C.c_int]),
    "bmg_hierarchy_schur_iters": (C.c_int, [_vp]),
    "bmg_destroy_system": (None, [_vp]),
    "bmg_destroy_hierarchy": (None, [_vp]),
    "bmg_status_string": (C.c_char_p, [C.c_int]),
    "bmg_profile_start": (C.c_int, [C.c_int, C.c_int]),
    "bmg_launch_count": (C.c_longlong, []),
    "bmg_use_graphs": (C.c_int, [C.c_int]),
    "bmg_profile_stop": (C.c_int, [C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_double)]),
    "bmg_last_error": (C.c_char_p, []),
    "bmg_batch_create": (C.c_int, [C.POINTER(_vp), C.c_int, C.POINTER(KrylovOpts), C.c_int, _vp,
                                   C.POINTER(_vp)]),
    "bmg_batch_solve": (C.c_int, [_vp, C.POINTER(_vp), C.POINTER(_vp), C.POINTER(SolveInfo), _vp]),
    "bmg_batch_tile": (C.c_int, [_vp, C.c_int, C.c_int]),
    "bmg_batch_trips": (C.c_int, [_vp]),
    "bmg_batch_kernels_per_trip": (C.c_longlong, [_vp]),
    "bmg_batch_destroy": (None, [_vp]),
}
for _name, (_res, _args) in _sig.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class BmgError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise BmgError(f"{what}: {lib.bmg_status_string(rc).decode()} ({rc}): "
                       f"{lib.bmg_last_error().decode()}")


# ---- layout ------------------------------------------------------------------------------
def pitch(n: int) -> int:
    return lib.bmg_pitch(n)


def block_len(n: int) -> int:
    return lib.bmg_block_len(n)


def vector_len(n: int) -> int:
    return lib.bmg_vector_len(n)


def free_dofs(n: int) -> int:
    return lib.bmg_free_dofs(n)


def pack(n: int, fields: dict, dtype=np.float64) -> np.ndarray:
    """dict of ``[j, i]`` arrays (shapes of ``synthetic.shapes``) -> flat vector in the
    library's layout (10 blocks of (n+1) x pitch; unused slots zero)."""
    P = pitch(n)
    out = np.zeros((10, n + 1, P), dtype=dtype)
    for k, t in enumerate(TYPES):
        a = np.asarray(fields[t])
        out[k, :a.shape[0], :a.shape[1]] = a
    return out.reshape(-1)


def unpack(n: int, x) -> dict:
    """Inverse of ``pack``."""
    x = np.asarray(x).reshape(10, n + 1, pitch(n))
    shp = {"ux": (n + 1, n + 1), "uy": (n + 1, n + 1), "bh": (n + 1, n), "bv": (n, n + 1),
           "bd": (n, n), "wh": (n + 1, n), "wv": (n, n + 1), "wd": (n, n), "pL": (n, n), "pU": (n, n)}
    return {t: np.array(x[k, :shp[t][0], :shp[t][1]]) for k, t in enumerate(TYPES)}


def pack_k(n: int, K_L, K_U, dtype=np.float64) -> np.ndarray:
    """Per-triangle permeability ``(n, n)`` arrays -> the two-block field ``bmg_assemble`` reads."""
    P = pitch(n)
    out = np.zeros((2, n + 1, P), dtype=dtype)
    out[0, :n, :n] = K_L
    out[1, :n, :n] = K_U
    return out.reshape(-1)


def _ptr(t) -> int:
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise BmgError("expected a contiguous CUDA tensor")
    return t.data_ptr()


def _stream(stream) -> int:
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ---- handles -----------------------------------------------------------------------------
class System:
    """An assembled operator (``bmg_assemble``)."""

    def __init__(self, handle, n: int, params: dict):
        self._h = handle
        self.n = n
        self.params = params

    @property
    def handle(self):
        return self._h

    def apply(self, x, y, stream=None):
        import torch
        if x.dtype != torch.float64 or y.dtype != torch.float64:
            raise BmgError("apply: float64 vectors required")
        _check(lib.bmg_apply(self._h, _ptr(x), _ptr(y), _stream(stream)), "bmg_apply")

    def residual(self, b, x, r, stream=None):
        _check(lib.bmg_residual(self._h, _ptr(b), _ptr(x), _ptr(r), _stream(stream)), "bmg_residual")

    def backward_euler_rhs(self, x_prev, load, b, stream=None):
        """``bmg_backward_euler_rhs``: b = load + the pressure-row history term of x_prev."""
        _check(lib.bmg_backward_euler_rhs(self._h, _ptr(x_prev), _ptr(load), _ptr(b), _stream(stream)),
               "bmg_backward_euler_rhs")

    def adjoint_gradient(self, x, xi, dtheta, dlame, stream=None):
        """``bmg_adjoint_gradient``: dtheta (2 blocks, layout of K) and dlame = (dL/dlambda,
        dL/dmu), float64 CUDA tensors written by the library."""
        _check(lib.bmg_adjoint_gradient(self._h, _ptr(x), _ptr(xi), _ptr(dtheta), _ptr(dlame),
                                        _stream(stream)), "bmg_adjoint_gradient")

    def close(self):
        if self._h:
            lib.bmg_destroy_system(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def assemble(n: int, lam: float, mu: float, K=None, K_const: float = 1.0, tau: float = 1.0,
             alpha: float = 1.0, inv_M: float = 0.0, stream=None, divdiv: str = "reduced") -> System:
    """``bmg_assemble`` (``divdiv="reduced"``) or ``bmg_assemble_divdiv`` (``"exact"``: the
    original discretisation with exactly integrated grad-div term).  K is None (uniform
    ``K_const``) or a float64 CUDA tensor laid out as ``pack_k`` produces."""
    h = _vp()
    kp = None if K is None else _ptr(K)
    if divdiv == "reduced":
        _check(lib.bmg_assemble(n, lam, mu, kp, K_const, tau, alpha, inv_M, _stream(stream), C.byref(h)),
               "bmg_assemble")
    else:
        _check(lib.bmg_assemble_divdiv(n, lam, mu, kp, K_const, tau, alpha, inv_M,
                                       {"reduced": 0, "exact": 1}[divdiv], _stream(stream), C.byref(h)),
               "bmg_assemble_divdiv")
    return System(h, n, dict(lam=lam, mu=mu, K_const=K_const, tau=tau, alpha=alpha, inv_M=inv_M,
                             K_field=K is not None, divdiv=divdiv))


def assemble_logk(n: int, lam: float, mu: float, logK, tau: float = 1.0, alpha: float = 1.0,
                  inv_M: float = 0.0, stream=None) -> System:
    """``bmg_assemble_logk``: logK is a float32 CUDA tensor laid out as ``pack_k`` produces."""
    import torch
    if logK.dtype != torch.float32:
        raise BmgError("assemble_logk: float32 log-permeability required")
    h = _vp()
    _check(lib.bmg_assemble_logk(n, lam, mu, _ptr(logK), tau, alpha, inv_M, _stream(stream), C.byref(h)),
           "bmg_assemble_logk")
    return System(h, n, dict(lam=lam, mu=mu, tau=tau, alpha=alpha, inv_M=inv_M, K_field=True))


class Hierarchy:
    """A multigrid preconditioner (``bmg_setup_hierarchy``)."""

    def __init__(self, handle, system: System, opts: MgOpts):
        self._h = handle
        self.system = system     # keeps the system alive
        self.opts = opts
        self.n = system.n

    @property
    def levels(self) -> int:
        return lib.bmg_hierarchy_levels(self._h)

    def vcycle(self, r, z, stream=None):
        _check(lib.bmg_vcycle(self._h, _ptr(r), _ptr(z), _stream(stream)), "bmg_vcycle")

    def tile(self, level: int, kernel: str) -> int:
        """Tile index chosen at setup for a kernel family on a level (``bmg_hierarchy_tile``)."""
        return lib.bmg_hierarchy_tile(self._h, level, PROF[kernel])

    def schur_iters(self) -> int:
        """Exact BSR: most CG iterations one pressure step took so far (``bmg_hierarchy_schur_iters``)."""
        return lib.bmg_hierarchy_schur_iters(self._h)

    def fgmres_solve(self, b, x, rtol=1e-8, restart=50, maxit=500, x0_is_zero=True, stream=None,
                     arnoldi="fp64"):
        """``bmg_fgmres_solve``; ``arnoldi`` is "fp64" (default) or "mixed"."""
        ko = KrylovOpts(rtol, restart, maxit, 1 if x0_is_zero else 0, ARNOLDI[arnoldi])
        info = SolveInfo()
        _check(lib.bmg_fgmres_solve(self._h, _ptr(b), _ptr(x), C.byref(ko), C.byref(info),
                                    _stream(stream)), "bmg_fgmres_solve")
        return _info(info)

    def fgmres_solve_noalloc(self, b, x, rtol=1e-8, restart=30, maxit=500, x0_is_zero=True,
                             stream=None):
        """The allocation-free variant: the Krylov workspace is the library's fixed device
        array (``noalloc_capacity()`` doubles); see ``bmg_fgmres_solve_noalloc``."""
        ko = KrylovOpts(rtol, restart, maxit, 1 if x0_is_zero else 0, 0)
        info = SolveInfo()
        _check(lib.bmg_fgmres_solve_noalloc(self._h, _ptr(b), _ptr(x), C.byref(ko), C.byref(info),
                                            _stream(stream)), "bmg_fgmres_solve_noalloc")
        return _info(info)

    def fgmres_solve_host(self, b: np.ndarray, x: np.ndarray, rtol=1e-8, restart=50, maxit=500,
                          x0_is_zero=True, stream=None, arnoldi="fp64"):
        """Host-buffer variant: ``b`` and ``x`` are float64 numpy arrays (pinned or not)."""
        assert b.dtype == np.float64 and x.dtype == np.float64
        assert b.flags.c_contiguous and x.flags.c_contiguous
        ko = KrylovOpts(rtol, restart, maxit, 1 if x0_is_zero else 0, ARNOLDI[arnoldi])
        info = SolveInfo()
        _check(lib.bmg_fgmres_solve_host(self._h, b.ctypes.data, x.ctypes.data, C.byref(ko),
                                         C.byref(info), _stream(stream)), "bmg_fgmres_solve_host")
        return _info(info)

    def close(self):
        if self._h:
            lib.bmg_destroy_hierarchy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _info(info: SolveInfo) -> dict:
    return dict(iters=info.iters, restarts=info.restarts, status=STATUS.get(info.status, info.status),
                relres=info.relres, relres_est=info.relres_est, solve_ms=info.solve_ms)


def setup_hierarchy(system: System, smoother: str = "vanka", nu1: int = 1, nu2: int = 1,
                    omega: float = 0.8, omega_J: float = 1.0, n_coarse: int = 8,
                    precision: str = "fp64", p_shift: float = 0.0, cycle: str = "V",
                    coarse_op: str = "redisc", patch_solve: str = "cycle", stream=None) -> Hierarchy:
    """``bmg_setup_hierarchy``; ``smoother`` is "vanka", "bsr" (inexact Braess-Sarazin) or
    "bsr_exact" (exact Braess-Sarazin, FP64 only); ``cycle`` is "V" or "W" (gamma = 1 or 2), ``coarse_op``
    "redisc" (the paper's) or "galerkin", ``patch_solve`` "cycle" or "fp64" (FP64 Vanka
    patch solves inside an FP32 V-cycle)."""
    o = MgOpts({"vanka": VANKA, "bsr": BSR, "bsr_exact": BSR_EXACT}[smoother], nu1, nu2, omega, omega_J, n_coarse,
               FP64 if precision == "fp64" else FP32, p_shift, {"V": 1, "W": 2}[cycle],
               {"redisc": 0, "galerkin": 1}[coarse_op], {"cycle": 0, "fp64": 1}[patch_solve])
    h = _vp()
    _check(lib.bmg_setup_hierarchy(system.handle, C.byref(o), _stream(stream), C.byref(h)),
           "bmg_setup_hierarchy")
    return Hierarchy(h, system, o)


def vcycle(h: Hierarchy, r, z, stream=None):
    h.vcycle(r, z, stream)


class Batch:
    """Batched FGMRES over independent systems (``bmg_batch_create`` / ``bmg_batch_solve``):
    one graph launch per solve, the FGMRES state of every instance on the device."""

    def __init__(self, hierarchies, rtol=1e-8, restart=50, maxit=500, x0_is_zero=True,
                 autotune=True, stream=None, arnoldi="fp64"):
        self.hierarchies = list(hierarchies)      # keeps them alive
        self.count = len(self.hierarchies)
        arr = (_vp * self.count)(*[h._h for h in self.hierarchies])
        ko = KrylovOpts(rtol, restart, maxit, 1 if x0_is_zero else 0, ARNOLDI[arnoldi])
        self._b = _vp()
        _check(lib.bmg_batch_create(arr, self.count, C.byref(ko), 1 if autotune else 0,
                                    _stream(stream), C.byref(self._b)), "bmg_batch_create")

    def solve(self, bs, xs, stream=None):
        """Solve A_i x_i = b_i for every instance; returns the per-instance info dicts."""
        assert len(bs) == self.count and len(xs) == self.count
        pb = (_vp * self.count)(*[_ptr(b) for b in bs])
        px = (_vp * self.count)(*[_ptr(x) for x in xs])
        infos = (SolveInfo * self.count)()
        _check(lib.bmg_batch_solve(self._b, pb, px, infos, _stream(stream)), "bmg_batch_solve")
        return [_info(i) for i in infos]

    def tile(self, kernel: str, n: int) -> int:
        return lib.bmg_batch_tile(self._b, PROF[kernel], n)

    @property
    def trips(self) -> int:
        return lib.bmg_batch_trips(self._b)

    @property
    def kernels_per_trip(self) -> int:
        return lib.bmg_batch_kernels_per_trip(self._b)

    def close(self):
        if self._b:
            lib.bmg_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


PROF = {"apply": 1, "vanka": 2, "vanka_u": 3, "restrict": 4, "prolong": 5, "coarse": 6, "krylov": 7,
        "schur": 8}


def noalloc_capacity() -> int:
    """Doubles in the fixed device workspace of ``fgmres_solve_noalloc``."""
    return lib.bmg_noalloc_capacity()


def launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return lib.bmg_launch_count()


def use_graphs(enable: bool) -> bool:
    """``bmg_use_graphs``: V-cycles replayed as CUDA graphs (True by default); returns the
    previous setting."""
    return bool(lib.bmg_use_graphs(1 if enable else 0))


def profile_start(kernel: str, n: int = 0):
    """Time every later launch of a kernel family (on n-cell grids; 0 = any) with CUDA events."""
    _check(lib.bmg_profile_start(PROF[kernel], n), "bmg_profile_start")


def profile_stop() -> dict:
    """Stop timing: summed device milliseconds, launch count and processed grid cells."""
    ms, cnt, cells = C.c_double(), C.c_longlong(), C.c_double()
    _check(lib.bmg_profile_stop(C.byref(ms), C.byref(cnt), C.byref(cells)), "bmg_profile_stop")
    return dict(ms=ms.value, launches=cnt.value, cells=cells.value)


def apply(s: System, x, y, stream=None):
    s.apply(x, y, stream)


def residual(s: System, b, x, r, stream=None):
    s.residual(b, x, r, stream)


def fgmres_solve(h: Hierarchy, b, x, **kw) -> dict:
    return h.fgmres_solve(b, x, **kw)
