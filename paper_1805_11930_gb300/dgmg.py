"""Thin ctypes binding of the C ABI in include/dgmg.h.

Every function here only marshals arguments (torch tensors -> device
pointers, numpy arrays -> host pointers) and checks the returned status; all
computation happens in libdgmg.so.  There is no fallback: if the library
cannot be loaded, or a call fails, a DgmgError is raised.

The function names are those of the C ABI (dgmg_create, dgmg_apply, ...);
`Context` bundles them for convenience.
"""
import ctypes
import os

import numpy as np

from . import build as _build

DGMG_OK = 0
STATUS = {0: "DGMG_OK", 1: "DGMG_ERR_ARG", 2: "DGMG_ERR_OOM", 3: "DGMG_ERR_CUDA", 4: "DGMG_ERR_STATE",
          5: "DGMG_ERR_NOT_CONVERGED", 6: "DGMG_ERR_BREAKDOWN", 7: "DGMG_ERR_TIMEOUT"}
FP64, FP32, DF64 = 0, 1, 2
LAYOUT_AUTO, LAYOUT_LINE, LAYOUT_ELEMENT, LAYOUT_PLANE = 0, 1, 2, 3
LAYOUT_NAMES = {LAYOUT_LINE: "line", LAYOUT_ELEMENT: "element", LAYOUT_PLANE: "plane"}
KRYLOV_CG, KRYLOV_FCG, KRYLOV_FGMRES = 0, 1, 2
INNER_PCG, INNER_GMRES, INNER_DIRECT, INNER_GMRES_TRIDIAG = 0, 1, 2, 3
COARSE_AMG, COARSE_NONE, COARSE_P0 = 0, 1, 2
STOP_RESIDUAL, STOP_ENERGY = 0, 1
SMOOTHER_JACOBI, SMOOTHER_SSOR = 0, 1


class DgmgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(ctypes.Structure):
    _fields_ = [("krylov", ctypes.c_int), ("restart", ctypes.c_int), ("rtol", ctypes.c_double),
                ("maxit", ctypes.c_int), ("smoother_prec", ctypes.c_int), ("omega", ctypes.c_double),
                ("npre", ctypes.c_int), ("npost", ctypes.c_int), ("eps_inner", ctypes.c_double),
                ("maxit_inner", ctypes.c_int), ("inner", ctypes.c_int), ("inner_restart", ctypes.c_int),
                ("coarse", ctypes.c_int), ("timing", ctypes.c_int), ("coarse_cycles", ctypes.c_int),
                ("smoother", ctypes.c_int), ("apply_prec", ctypes.c_int), ("graph", ctypes.c_int),
                ("stop", ctypes.c_int), ("delay", ctypes.c_int)]


class SolveStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("converged", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("inner_mean", ctypes.c_double), ("inner_max", ctypes.c_int), ("ms_total", ctypes.c_double),
                ("inner_its_total", ctypes.c_longlong), ("sweeps", ctypes.c_longlong),
                ("zero_sweeps", ctypes.c_longlong),
                ("applies", ctypes.c_longlong), ("kernel_launches", ctypes.c_longlong),
                ("ms_smooth", ctypes.c_double), ("ms_apply", ctypes.c_double),
                ("energy_estimate", ctypes.c_double), ("iterations_run", ctypes.c_int),
                ("ms_transfer", ctypes.c_double), ("ms_coarse", ctypes.c_double), ("ms_krylov", ctypes.c_double),
                ("ms_device", ctypes.c_double), ("inner_std", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_LL = ctypes.c_longlong
_SIG = {
    "dgmg_default_opts": (None, [ctypes.POINTER(SolveOpts)]),
    "dgmg_create": (_I, [ctypes.POINTER(_P), _I, _P]),
    "dgmg_destroy": (_I, [_P]),
    "dgmg_last_error": (ctypes.c_char_p, [_P]),
    "dgmg_set_mesh": (_I, [_P, _I, _I, _I, _D, _D, _D, _I, _P]),
    "dgmg_set_penalty": (_I, [_P, _D]),
    "dgmg_set_coefficients": (_I, [_P, _P, _I, _P, _P]),
    "dgmg_sizes": (_I, [_P] + [ctypes.POINTER(_LL)] * 5),
    "dgmg_quadrature_points": (_I, [_P, _P, _P]),
    "dgmg_assemble_rhs": (_I, [_P, _P, _P, _P, _P]),
    "dgmg_apply": (_I, [_P, _P, _P, _I]),
    "dgmg_block_apply": (_I, [_P, _P, _P, _I]),
    "dgmg_block_diagonal": (_I, [_P, _P, _I]),
    "dgmg_block_smooth": (_I, [_P, _P, _P, _I, _D, _D, _I, _I, _I, _I, _P]),
    "dgmg_block_sor": (_I, [_P, _P, _P, _I, _D, _D, _I, _I, _I, _I, _I, _P]),
    "dgmg_restrict": (_I, [_P, _P, _P, _I]),
    "dgmg_prolong_add": (_I, [_P, _P, _P, _I]),
    "dgmg_coarse_matrix": (_I, [_P, _P]),
    "dgmg_coarse_cycle": (_I, [_P, _P, _P]),
    "dgmg_vcycle": (_I, [_P, _P, _P, ctypes.POINTER(SolveOpts)]),
    "dgmg_solve": (_I, [_P, _P, _P, ctypes.POINTER(SolveOpts), ctypes.POINTER(SolveStats)]),
    "dgmg_restrict_noalloc": (_I, [_I, _I, _I, _I, _P, _P, _I, _P]),
    "dgmg_set_launch_shape": (_I, [_P, _I, _I, _I]),
    "dgmg_block_inverse": (_I, [_P, _I, _P]),
    "dgmg_set_variable_coefficients": (_I, [_P, _P, _P, _P, _D]),
    "dgmg_restrict_p0": (_I, [_P, _P, _P, _I]),
    "dgmg_prolong_add_p0": (_I, [_P, _P, _P, _I]),
    "dgmg_coarse_matrix_p0": (_I, [_P, _P]),
    "dgmg_coarse_cycle_p0": (_I, [_P, _P, _P]),
    "dgmg_autotune": (_I, [_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dgmg_set_layout": (_I, [_P, _I, _I, _I]),
    "dgmg_get_layout": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "dgmg_batch_create": (_I, [ctypes.POINTER(_P), _I, _P, ctypes.POINTER(SolveOpts)]),
    "dgmg_batch_destroy": (_I, [_P]),
    "dgmg_batch_last_error": (ctypes.c_char_p, [_P]),
    "dgmg_batch_add": (_I, [_P, _P, _P, _P, _D, _I, ctypes.POINTER(_I)]),
    "dgmg_batch_step": (_I, [_P, _I, ctypes.POINTER(_I)]),
    "dgmg_batch_poll": (_I, [_P, _I, ctypes.POINTER(_I), ctypes.POINTER(SolveStats)]),
    "dgmg_batch_remove": (_I, [_P, _I]),
    "dgmg_batch_prime": (_I, [_P, _P, _P, ctypes.POINTER(SolveOpts)]),
}

BATCH_MAX = 16

NOALLOC_MAX_CELLS = 131072


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libdgmg.so (building it first if it is missing and nvcc exists)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path) or (build_if_missing and not _build.up_to_date()):
        if not build_if_missing:
            raise DgmgError(3, f"{path} not built; run paper_1805_11930_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIG.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    """Device pointer of a torch tensor (or an int), None -> NULL."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if not x.is_cuda:
        raise DgmgError(1, "expected a CUDA tensor")
    if not x.is_contiguous():
        raise DgmgError(1, "expected a contiguous tensor")
    return x.data_ptr()


def _host(a, dtype=np.float64):
    if a is None:
        return None, None
    arr = np.ascontiguousarray(a, dtype=dtype)
    return arr, arr.ctypes.data


def _prec(t, df64=False):
    import torch
    if t.dtype == torch.float64:
        return DF64 if df64 else FP64
    if t.dtype == torch.float32:
        return FP32
    raise DgmgError(1, f"unsupported dtype {t.dtype}")


def default_opts(**kw):
    o = SolveOpts()
    load().dgmg_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Context:
    """A dgmg_ctx bound to one device and stream (default: torch's current
    stream on that device)."""

    def __init__(self, device=0, stream=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        self.stream = stream
        self.device = device
        h = _P()
        st = self.lib.dgmg_create(ctypes.byref(h), device, stream)
        if st != DGMG_OK:
            raise DgmgError(st, "dgmg_create failed")
        self.h = h
        self.mesh = None

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgmg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, st):
        if st != DGMG_OK:
            raise DgmgError(st, self.lib.dgmg_last_error(self.h).decode())
        return st

    # ------------------------------------------------------------ setup
    def set_mesh(self, nx, ny, nz, lx, ly, lz, p, bc):
        bca = (ctypes.c_int * 6)(*[int(b) for b in bc])
        self._check(self.lib.dgmg_set_mesh(self.h, nx, ny, nz, lx, ly, lz, p, bca))
        self.mesh = (nx, ny, nz, lx, ly, lz, p, list(bc))

    def set_penalty(self, alpha):
        self._check(self.lib.dgmg_set_penalty(self.h, float(alpha)))

    def set_coefficients(self, K, b_vertex=None, c_cell=None):
        K = np.asarray(K, dtype=np.float64)
        kdim = 1 if K.ndim == 1 else K.shape[1]
        Ka, Kp = _host(K)
        ba, bp = _host(b_vertex)
        ca, cp = _host(c_cell)
        self._check(self.lib.dgmg_set_coefficients(self.h, Kp, kdim, bp, cp))

    def set_variable_coefficients(self, basis, p0, p2, gamma):
        """K(x) = sum_k (p0_k + p2_k x_k^2) n_k n_k^T (rows of `basis` are n_k),
        c(x) = gamma |x|^2 for the outer operator; cell-centre values for the
        preconditioner."""
        b, bp = _host(np.asarray(basis, dtype=np.float64).reshape(9))
        a0, p0p = _host(p0)
        a2, p2p = _host(p2)
        self._check(self.lib.dgmg_set_variable_coefficients(self.h, bp, p0p, p2p, float(gamma)))

    def sizes(self):
        v = [_LL() for _ in range(5)]
        self._check(self.lib.dgmg_sizes(self.h, *[ctypes.byref(x) for x in v]))
        return dict(zip(("ndof", "nvert", "ncell", "nvol_qp", "nface_qp"), [x.value for x in v]))

    def quadrature_points(self):
        s = self.sizes()
        vol = np.zeros((s["nvol_qp"], 3))
        face = np.zeros((s["nface_qp"], 3))
        self._check(self.lib.dgmg_quadrature_points(self.h, vol.ctypes.data, face.ctypes.data))
        return vol, face

    def assemble_rhs(self, f_qp, rhs, g_qp=None, j_qp=None):
        fa, fp = _host(f_qp)
        ga, gp = _host(g_qp)
        ja, jp = _host(j_qp)
        self._check(self.lib.dgmg_assemble_rhs(self.h, fp, gp, jp, _ptr(rhs)))

    # ------------------------------------------------------------ operators
    def apply(self, u, v, df64=False):
        """v = A u; df64=True: FP64 vectors, double-float arithmetic."""
        self._check(self.lib.dgmg_apply(self.h, _ptr(u), _ptr(v), _prec(u, df64)))

    def block_apply(self, u, v, df64=False):
        self._check(self.lib.dgmg_block_apply(self.h, _ptr(u), _ptr(v), _prec(u, df64)))

    def block_diagonal(self, diag):
        self._check(self.lib.dgmg_block_diagonal(self.h, _ptr(diag), _prec(diag)))

    def block_smooth(self, f, u, nsweep=1, omega=1.0, eps=1e-2, maxit=0, inner=INNER_PCG, inner_restart=12,
                     inner_its=None, df64=False):
        self._check(self.lib.dgmg_block_smooth(self.h, _ptr(f), _ptr(u), nsweep, omega, eps, maxit, inner,
                                               inner_restart, _prec(u, df64), _ptr(inner_its)))

    def block_sor(self, f, u, nsweep=1, omega=1.0, eps=1e-2, maxit=0, inner=INNER_PCG, inner_restart=12,
                  symmetric=True, inner_its=None, df64=False):
        self._check(self.lib.dgmg_block_sor(self.h, _ptr(f), _ptr(u), nsweep, omega, eps, maxit, inner,
                                            inner_restart, 1 if symmetric else 0, _prec(u, df64),
                                            _ptr(inner_its)))

    def block_inverse(self, prec=FP64, out=None):
        """Build the stored D_T^-1 of every cell (inner = INNER_DIRECT) in FP64
        or FP32; `out` (device tensor of ncell n^6 values) receives a copy,
        column-major per block."""
        self._check(self.lib.dgmg_block_inverse(self.h, prec, _ptr(out)))

    def restrict(self, r, r_hat):
        self._check(self.lib.dgmg_restrict(self.h, _ptr(r), _ptr(r_hat), _prec(r)))

    def prolong_add(self, u_hat, u):
        self._check(self.lib.dgmg_prolong_add(self.h, _ptr(u_hat), _ptr(u), _prec(u)))

    def coarse_matrix(self):
        s = self.sizes()
        st = np.zeros(27 * s["nvert"])
        self._check(self.lib.dgmg_coarse_matrix(self.h, st.ctypes.data))
        return st.reshape(s["nvert"], 27)

    def coarse_cycle(self, r_hat, u_hat):
        self._check(self.lib.dgmg_coarse_cycle(self.h, _ptr(r_hat), _ptr(u_hat)))

    # ------------------------------------------------------------ P0 subspace
    def restrict_p0(self, r, r_hat):
        self._check(self.lib.dgmg_restrict_p0(self.h, _ptr(r), _ptr(r_hat), _prec(r)))

    def prolong_add_p0(self, u_hat, u):
        self._check(self.lib.dgmg_prolong_add_p0(self.h, _ptr(u_hat), _ptr(u), _prec(u)))

    def coarse_matrix_p0(self):
        s = self.sizes()
        st = np.zeros(27 * s["ncell"])
        self._check(self.lib.dgmg_coarse_matrix_p0(self.h, st.ctypes.data))
        return st.reshape(s["ncell"], 27)

    def coarse_cycle_p0(self, r_hat, u_hat):
        self._check(self.lib.dgmg_coarse_cycle_p0(self.h, _ptr(r_hat), _ptr(u_hat)))

    def vcycle(self, f, u, opts=None):
        o = opts if opts is not None else default_opts()
        self._check(self.lib.dgmg_vcycle(self.h, _ptr(f), _ptr(u), ctypes.byref(o)))

    # ------------------------------------------------------------ launch shapes
    def set_launch_shape(self, prec, wpb_apply=0, wpb_smooth=0):
        """Warps per block of the operator / smoother kernels for FP64, FP32 or
        DF64 arithmetic (0 = default)."""
        self._check(self.lib.dgmg_set_launch_shape(self.h, prec, wpb_apply, wpb_smooth))

    def set_layout(self, prec, layout_apply=LAYOUT_AUTO, layout_smooth=LAYOUT_AUTO):
        """Work layouts (LAYOUT_LINE / ELEMENT / PLANE, or AUTO) of the
        operator and inner-PCG smoother kernels for FP64, FP32 or DF64."""
        self._check(self.lib.dgmg_set_layout(self.h, prec, layout_apply, layout_smooth))

    def get_layout(self, prec):
        """The layouts in use for a precision: (layout_apply, layout_smooth)."""
        a, s = _I(0), _I(0)
        self._check(self.lib.dgmg_get_layout(self.h, prec, ctypes.byref(a), ctypes.byref(s)))
        return a.value, s.value

    def autotune(self, prec=FP64, reps=3):
        """Time the layout and launch-shape candidates on the current mesh and
        keep the fastest; returns (wpb_apply, wpb_smooth) (get_layout gives the
        layouts)."""
        a, s = _I(0), _I(0)
        self._check(self.lib.dgmg_autotune(self.h, prec, reps, ctypes.byref(a), ctypes.byref(s)))
        return a.value, s.value

    def batch_prime(self, f, u, opts=None):
        """dgmg_batch_prime: the initial Krylov state of a batched solve of
        (f, u) with `opts`, on this context's stream."""
        o = opts if opts is not None else default_opts()
        self._check(self.lib.dgmg_batch_prime(self.h, _ptr(f), _ptr(u), ctypes.byref(o)))

    def solve(self, f, u, opts=None, check=True):
        o = opts if opts is not None else default_opts()
        stats = SolveStats()
        st = self.lib.dgmg_solve(self.h, _ptr(f), _ptr(u), ctypes.byref(o), ctypes.byref(stats))
        if check:
            self._check(st)
        return stats.as_dict() | {"status": STATUS.get(st, st)}


class Batch:
    """A dgmg_batch: the outer solves of several prepared contexts of one order
    in lockstep, each step one launch over all members (see include/dgmg.h).
    `opts`: the shared solve options (SolveOpts, default_opts() if None)."""

    def __init__(self, device=0, stream=None, opts=None):
        import torch
        self.lib = load()
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        elif not isinstance(stream, int):
            stream = stream.cuda_stream
        self.stream = stream
        self.device = device
        o = opts if opts is not None else default_opts()
        h = _P()
        st = self.lib.dgmg_batch_create(ctypes.byref(h), device, stream, ctypes.byref(o))
        if st != DGMG_OK:
            raise DgmgError(st, "dgmg_batch_create failed (unsupported options or no device)")
        self.h = h

    def _check(self, st):
        if st != DGMG_OK:
            msg = self.lib.dgmg_batch_last_error(self.h)
            raise DgmgError(st, msg.decode() if msg else "")

    def add(self, ctx, f, u, rtol=1e-8, maxit=500):
        """Add a prepared context with its right-hand side f and iterate u
        (device FP64 tensors); returns the member's slot."""
        slot = _I(-1)
        self._check(self.lib.dgmg_batch_add(self.h, ctx.h, _ptr(f), _ptr(u), rtol, maxit, ctypes.byref(slot)))
        return slot.value

    def step(self, iterations=1):
        """Run `iterations` outer iterations of every running member; returns
        how many still run."""
        left = _I(0)
        self._check(self.lib.dgmg_batch_step(self.h, iterations, ctypes.byref(left)))
        return left.value

    def poll(self, slot):
        """None while the member runs, else its statistics (dict with
        "status")."""
        done = _I(0)
        stats = SolveStats()
        st = self.lib.dgmg_batch_poll(self.h, slot, ctypes.byref(done), ctypes.byref(stats))
        if st not in (DGMG_OK, 5, 6):
            self._check(st)
        if not done.value:
            return None
        return stats.as_dict() | {"status": STATUS.get(st, st)}

    def remove(self, slot):
        self._check(self.lib.dgmg_batch_remove(self.h, slot))

    def close(self):
        if getattr(self, "h", None):
            self.lib.dgmg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def restrict_noalloc(nx, ny, nz, p, r, r_hat, stream=None):
    """dgmg_restrict_noalloc: R r into r_hat without a context or any device
    allocation (the scratch is a fixed array inside the library).  `stream`:
    a torch.cuda.Stream, a raw cudaStream_t or None (torch's current stream)."""
    import torch
    lib = load()
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    elif not isinstance(stream, int):
        stream = stream.cuda_stream
    st = lib.dgmg_restrict_noalloc(nx, ny, nz, p, _ptr(r), _ptr(r_hat), _prec(r), stream)
    if st != DGMG_OK:
        raise DgmgError(st, "dgmg_restrict_noalloc failed (sizes beyond "
                            f"{NOALLOC_MAX_CELLS} cells, bad arguments or a CUDA error)")


def exported_symbols(header_path=None):
    """Names of the functions declared in include/dgmg.h."""
    import re
    header_path = header_path or os.path.join(_build.INCLUDE, "dgmg.h")
    text = open(header_path).read()
    return sorted(set(re.findall(r"\b(dgmg_[a-z0-9_]+)\s*\(", text)))
