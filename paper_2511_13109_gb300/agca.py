"""ctypes binding of libagca (include/agca.h): argument marshalling only.

PyTorch provides device memory (the workspace and Galerkin store are uint8
CUDA tensors bound to the context) and the CUDA stream; every numerical step
runs in the library's CUDA kernels.  There is no CPU fallback: importing the
binding without the built library raises.
"""
from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libagca.so")

FP64, MIXED = 0, 1
F64, F32 = 0, 1
PROJ_ARITHMETIC, PROJ_HARMONIC, PROJ_GEOMETRIC = 0, 1, 2
(FIELD_MEAN, FIELD_MAX, FIELD_MIN, FIELD_FLAGS, FIELD_LIST, FIELD_GCA, FIELD_DIAG, FIELD_COARSE, FIELD_PMASS,
 FIELD_SIDX, FIELD_STENCIL) = range(11)

STATUS = {0: "AGCA_OK", 1: "AGCA_EINVAL", 2: "AGCA_ENOMEM", 3: "AGCA_ECUDA", 4: "AGCA_ENOTCONV",
          5: "AGCA_ETIMEOUT", 6: "AGCA_EINTERNAL", 7: "AGCA_ESTATE"}


class AgcaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class LevelInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("vertices", ctypes.c_int64), ("elements", ctypes.c_int64),
                ("n_flag", ctypes.c_int64), ("lambda_", ctypes.c_double), ("n_stencil", ctypes.c_int64)]


_lib = None
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_SZ = ctypes.c_size_t

_SIGS = {
    "agca_status_string": ([_I], ctypes.c_char_p),
    "agca_create": ([_I, _I, _I, _P, ctypes.POINTER(_P)], _I),
    "agca_destroy": ([_P], None),
    "agca_last_error": ([_P], ctypes.c_char_p),
    "agca_set_smoother": ([_P, _I, _D, _D, _I], _I),
    "agca_set_solver_options": ([_P, _D, _I], _I),
    "agca_workspace_size": ([_P, ctypes.POINTER(_SZ)], _I),
    "agca_bind_workspace": ([_P, _P, _SZ], _I),
    "agca_set_viscosity": ([_P, _P], _I),
    "agca_flag": ([_P, _D, ctypes.POINTER(_SZ)], _I),
    "agca_bind_gca_store": ([_P, _P, _SZ], _I),
    "agca_setup": ([_P], _I),
    "agca_apply": ([_P, _I, _I, _P, _P], _I),
    "agca_restrict": ([_P, _I, _I, _P, _P], _I),
    "agca_prolong_add": ([_P, _I, _I, _P, _P], _I),
    "agca_vcycle": ([_P, _P, _P], _I),
    "agca_stokes_apply": ([_P, _P, _P], _I),
    "agca_precondition": ([_P, _P, _P], _I),
    "agca_load_vector": ([_P, _P, _P], _I),
    "agca_solve": ([_P, _P, _P, _D, _I, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "agca_fgmres_workspace_size": ([_P, _I, ctypes.POINTER(_SZ)], _I),
    "agca_solve_fgmres": ([_P, _P, _P, _D, _I, _I, _I, _I, _P, _SZ, ctypes.POINTER(_I), ctypes.POINTER(_D)], _I),
    "agca_element_sensitivity": ([_P, _P, _P, _P], _I),
    "agca_adjoint_gradient": ([_P, _P, _P, _P, _D, _I, ctypes.POINTER(_I)], _I),
    "agca_stokes_apply_static": ([_I, _P, _P, _P, _P], _I),
    "agca_autotune": ([_P, _I, ctypes.c_char_p], _I),
    "agca_tile_config": ([_P, _I, _I, ctypes.POINTER(_I), ctypes.POINTER(_I)], _I),
    "agca_set_tile_config": ([_P, _I, _I, _I, _I], _I),
    "agca_stencil_tiles": ([_I, _I, _I, ctypes.POINTER(_I)], _I),
    "agca_set_coarse_projection": ([_P, _I], _I),
    "agca_set_level_coefficient": ([_P, _I, _P], _I),
    "agca_flag_gradient": ([_P, _P, _D, ctypes.POINTER(_SZ)], _I),
    "agca_launch_count": ([_P, ctypes.POINTER(ctypes.c_int64)], _I),
    "agca_profile_fine": ([_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_D), ctypes.POINTER(_D),
                           ctypes.POINTER(ctypes.c_int64)], _I),
    "agca_batch_create": ([_I, ctypes.POINTER(_I), _I, _P, ctypes.POINTER(_P)], _I),
    "agca_batch_destroy": ([_P], None),
    "agca_batch_last_error": ([_P], ctypes.c_char_p),
    "agca_batch_workspace_size": ([_P, ctypes.POINTER(_SZ)], _I),
    "agca_batch_bind_workspace": ([_P, _P, _SZ], _I),
    "agca_batch_set_viscosity": ([_P, _I, _P], _I),
    "agca_batch_flag": ([_P, _D, ctypes.POINTER(_SZ)], _I),
    "agca_batch_bind_gca_store": ([_P, _P, _SZ], _I),
    "agca_batch_setup": ([_P], _I),
    "agca_batch_load_vector": ([_P, _I, _P, _P], _I),
    "agca_batch_vcycle": ([_P, ctypes.POINTER(_P), ctypes.POINTER(_P)], _I),
    "agca_batch_solve": ([_P, ctypes.POINTER(_P), ctypes.POINTER(_P), _D, _I, ctypes.POINTER(_I),
                          ctypes.POINTER(_D)], _I),
    "agca_batch_context": ([_P, _I], _P),
    "agca_level_info": ([_P, _I, ctypes.POINTER(LevelInfo)], _I),
    "agca_get_level_data": ([_P, _I, _I, _P], _I),
}


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libagca is not built ({LIB_PATH} missing); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in _SIGS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def stencil_tiles(n: int, block_rows: int = 8, z_chunk: int = 0) -> dict:
    """Tile grid of the stencil kernels on a grid of n cubes per axis (see
    agca_stencil_tiles in include/agca.h)."""
    out = (_I * 7)()
    st = lib().agca_stencil_tiles(int(n), int(block_rows), int(z_chunk), out)
    if st != 0:
        raise AgcaError(st, f"agca_stencil_tiles(n={n}, by={block_rows}, zch={z_chunk})")
    keys = ("gxw", "gyw", "gxn", "gyn", "x0n", "gz", "zch")
    return dict(zip(keys, list(out)))


def default_levels(N: int) -> int:
    """Coarsen the 2N velocity grid while it stays even with >= 4 cubes."""
    n, L = 2 * N, 1
    while n % 2 == 0 and n // 2 >= 4:
        n //= 2
        L += 1
    return L


STATIC_MAX_N = 32


def stokes_apply_static(N: int, eta: torch.Tensor, x: torch.Tensor, y: torch.Tensor | None = None,
                        stream: torch.cuda.Stream | None = None) -> torch.Tensor:
    """y = K x without a context or any library allocation (N <= 32), for
    callers that cannot allocate device memory; see agca_stokes_apply_static.
    The output tensor y must be provided by such callers."""
    nL = 2 * N
    nt = 3 * (nL + 1) ** 3 + (N + 1) ** 3
    _need(eta, 6 * nL ** 3, torch.float64, "eta")
    _need(x, nt, torch.float64, "x")
    y = torch.empty_like(x) if y is None else y
    _need(y, nt, torch.float64, "y")
    if not (eta.device == x.device == y.device):
        raise ValueError(f"eta, x and y must be on one device (got {eta.device}, {x.device}, {y.device})")
    s = stream if stream is not None else torch.cuda.current_stream(x.device)
    if s.device != x.device:
        raise ValueError(f"the stream is on {s.device}, the tensors on {x.device}")
    with torch.cuda.device(x.device):  # the library works on the current device
        st = lib().agca_stokes_apply_static(N, _ptr(eta), _ptr(x), _ptr(y), _P(s.cuda_stream))
    if st != 0:
        raise AgcaError(st, f"agca_stokes_apply_static(N={N})")
    return y


def _ptr(t: torch.Tensor):
    return ctypes.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, n: int, dtype, name: str):
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous() or t.numel() != n:
        raise ValueError(f"{name}: expected contiguous {dtype} with {n} elements, got {t.dtype} {tuple(t.shape)}")


class Context:
    """One AGCA hierarchy on one GPU (see include/agca.h)."""

    def __init__(self, N: int, levels: int | None = None, precision: int = FP64, device="cuda",
                 stream: torch.cuda.Stream | None = None):
        self.N = N
        self.L = default_levels(N) if levels is None else levels
        self.precision = precision
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = _P()
        st = lib().agca_create(N, self.L, precision, _P(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise AgcaError(st, f"agca_create(N={N}, levels={self.L}, precision={precision})")
        self._h = h
        sz = _SZ()
        self._check(lib().agca_workspace_size(self._h, ctypes.byref(sz)), "workspace_size")
        self.workspace = torch.empty(int(sz.value), dtype=torch.uint8, device=self.device)
        self._check(lib().agca_bind_workspace(self._h, _ptr(self.workspace), sz.value), "bind_workspace")
        self.gca_store = None
        self.nL = 2 * N
        self.V = {l: (((self.nL >> (self.L - l)) + 1) ** 3) for l in range(1, self.L + 1)}
        self.E = {l: 6 * (self.nL >> (self.L - l)) ** 3 for l in range(1, self.L + 1)}
        self.Vp = (N + 1) ** 3
        self.nt = 3 * self.V[self.L] + self.Vp

    @classmethod
    def _borrowed(cls, handle, N, levels, precision, device, stream, owner):
        """View of a context owned by a batch (not destroyed by this object)."""
        self = cls.__new__(cls)
        self.N, self.L, self.precision = N, levels, precision
        self.device, self.stream = torch.device(device), stream
        self._h = handle
        self._owner = owner
        self.workspace = self.gca_store = None
        self.nL = 2 * N
        self.V = {l: (((self.nL >> (self.L - l)) + 1) ** 3) for l in range(1, self.L + 1)}
        self.E = {l: 6 * (self.nL >> (self.L - l)) ** 3 for l in range(1, self.L + 1)}
        self.Vp = (N + 1) ** 3
        self.nt = 3 * self.V[self.L] + self.Vp
        return self

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None and getattr(self, "_owner", None) is None:
            _lib.agca_destroy(h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            msg = lib().agca_last_error(self._h).decode()
            raise AgcaError(st, f"{what}: {msg}")

    def _cycle_dtype(self, dtype):
        return torch.float64 if dtype == F64 else torch.float32

    # ---- setup ---------------------------------------------------------------
    def set_smoother(self, degree=2, lo=0.1, hi=1.1, power_iters=20):
        self._check(lib().agca_set_smoother(self._h, degree, lo, hi, power_iters), "set_smoother")

    def set_solver_options(self, mixed_inner_rtol: float = 1e-4, check_every: int = 4):
        self._check(lib().agca_set_solver_options(self._h, float(mixed_inner_rtol), int(check_every)),
                    "set_solver_options")

    def set_coarse_projection(self, kind: int):
        """Coarse coefficient as the children's arithmetic (PROJ_ARITHMETIC),
        harmonic (PROJ_HARMONIC) or geometric (PROJ_GEOMETRIC) mean; before flag()."""
        self._check(lib().agca_set_coarse_projection(self._h, int(kind)), "set_coarse_projection")

    def set_viscosity(self, eta: torch.Tensor):
        _need(eta, self.E[self.L], torch.float64, "eta")
        self._check(lib().agca_set_viscosity(self._h, _ptr(eta)), "set_viscosity")

    def flag(self, nu: float) -> int:
        b = _SZ()
        self._check(lib().agca_flag(self._h, float(nu), ctypes.byref(b)), "flag")
        self.gca_store = torch.empty(int(b.value), dtype=torch.uint8, device=self.device)
        self._check(lib().agca_bind_gca_store(self._h, _ptr(self.gca_store), b.value), "bind_gca_store")
        return int(b.value)

    def flag_gradient(self, eta_vertex: torch.Tensor, nu: float) -> int:
        """Flags by the gradient rule of Eq. 2.8 from the finest nodal
        viscosity (see agca_flag_gradient); binds the Galerkin store."""
        _need(eta_vertex, self.V[self.L], torch.float64, "eta_vertex")
        b = _SZ()
        self._check(lib().agca_flag_gradient(self._h, _ptr(eta_vertex), float(nu), ctypes.byref(b)), "flag_gradient")
        self.gca_store = torch.empty(int(b.value), dtype=torch.uint8, device=self.device)
        self._check(lib().agca_bind_gca_store(self._h, _ptr(self.gca_store), b.value), "bind_gca_store")
        return int(b.value)

    def set_level_coefficient(self, level: int, coef: torch.Tensor):
        """DCA coefficient of a coarse level evaluated on that level (see
        agca_set_level_coefficient); after flag(), before setup()."""
        _need(coef, self.E[level] if 1 <= level < self.L else -1, torch.float64, "coef")
        self._check(lib().agca_set_level_coefficient(self._h, int(level), _ptr(coef)), "set_level_coefficient")

    def setup(self):
        self._check(lib().agca_setup(self._h), "setup")

    def prepare(self, eta: torch.Tensor, nu: float = 10.0):
        self.set_viscosity(eta)
        self.flag(nu)
        self.setup()

    # ---- level operators -----------------------------------------------------
    def apply(self, level: int, x: torch.Tensor, y: torch.Tensor | None = None, dtype=F64):
        td = self._cycle_dtype(dtype)
        n = 3 * self.V[level]
        _need(x, n, td, "x")
        y = torch.empty_like(x) if y is None else y
        _need(y, n, td, "y")
        self._check(lib().agca_apply(self._h, level, dtype, _ptr(x), _ptr(y)), "apply")
        return y

    def restrict(self, level: int, rf: torch.Tensor, dtype=F64):
        td = self._cycle_dtype(dtype)
        _need(rf, 3 * self.V[level], td, "rf")
        rc = torch.empty(3 * self.V[level - 1], dtype=td, device=self.device)
        self._check(lib().agca_restrict(self._h, level, dtype, _ptr(rf), _ptr(rc)), "restrict")
        return rc

    def prolong_add(self, level: int, ec: torch.Tensor, xf: torch.Tensor, dtype=F64):
        td = self._cycle_dtype(dtype)
        _need(ec, 3 * self.V[level - 1], td, "ec")
        _need(xf, 3 * self.V[level], td, "xf")
        self._check(lib().agca_prolong_add(self._h, level, dtype, _ptr(ec), _ptr(xf)), "prolong_add")
        return xf

    def vcycle(self, r: torch.Tensor, z: torch.Tensor | None = None):
        n = 3 * self.V[self.L]
        _need(r, n, torch.float64, "r")
        z = torch.empty_like(r) if z is None else z
        _need(z, n, torch.float64, "z")
        self._check(lib().agca_vcycle(self._h, _ptr(r), _ptr(z)), "vcycle")
        return z

    # ---- Stokes ----------------------------------------------------------------
    def stokes_apply(self, x: torch.Tensor, y: torch.Tensor | None = None):
        _need(x, self.nt, torch.float64, "x")
        y = torch.empty_like(x) if y is None else y
        _need(y, self.nt, torch.float64, "y")
        self._check(lib().agca_stokes_apply(self._h, _ptr(x), _ptr(y)), "stokes_apply")
        return y

    def precondition(self, r: torch.Tensor, z: torch.Tensor | None = None):
        _need(r, self.nt, torch.float64, "r")
        z = torch.empty_like(r) if z is None else z
        self._check(lib().agca_precondition(self._h, _ptr(r), _ptr(z)), "precondition")
        return z

    def load_vector(self, fbar: torch.Tensor):
        _need(fbar, 3 * self.E[self.L], torch.float64, "fbar")
        b = torch.empty(self.nt, dtype=torch.float64, device=self.device)
        self._check(lib().agca_load_vector(self._h, _ptr(fbar), _ptr(b)), "load_vector")
        return b

    def solve(self, b: torch.Tensor, rtol: float = 1e-8, maxit: int = 5000, x: torch.Tensor | None = None):
        _need(b, self.nt, torch.float64, "b")
        x = torch.empty_like(b) if x is None else x
        its, rel = _I(), _D()
        st = lib().agca_solve(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(its),
                              ctypes.byref(rel))
        self._check(st, "solve")
        return x, its.value, rel.value

    def solve_fgmres(self, b: torch.Tensor, rtol: float = 1e-8, maxit: int = 5000, restart: int = 50,
                     schur: str = "mass", z_iters: int = 30, x: torch.Tensor | None = None):
        """The paper's outer solver: FGMRES with the block-triangular
        preconditioner of Eq. 4.1 and S~^-1 = the lumped 1/eta mass ("mass")
        or the diag(A)-BFBT of Eq. 4.2 ("bfbt"); see agca_solve_fgmres."""
        _need(b, self.nt, torch.float64, "b")
        x = torch.empty_like(b) if x is None else x
        sz = _SZ()
        self._check(lib().agca_fgmres_workspace_size(self._h, int(restart), ctypes.byref(sz)), "fgmres_workspace_size")
        work = torch.empty(int(sz.value), dtype=torch.uint8, device=self.device)
        its, rel = _I(), _D()
        st = lib().agca_solve_fgmres(self._h, _ptr(b), _ptr(x), float(rtol), int(maxit), int(restart),
                                     {"mass": 0, "bfbt": 1}[schur], int(z_iters), _ptr(work), sz.value,
                                     ctypes.byref(its), ctypes.byref(rel))
        self._check(st, "solve_fgmres")
        return x, its.value, rel.value

    def element_sensitivity(self, lam_u: torch.Tensor, u: torch.Tensor):
        n = 3 * self.V[self.L]
        _need(lam_u, n, torch.float64, "lam_u")
        _need(u, n, torch.float64, "u")
        g = torch.empty(self.E[self.L], dtype=torch.float64, device=self.device)
        self._check(lib().agca_element_sensitivity(self._h, _ptr(lam_u), _ptr(u), _ptr(g)), "element_sensitivity")
        return g

    def adjoint_gradient(self, x: torch.Tensor, dJdu: torch.Tensor, rtol: float = 1e-10, maxit: int = 5000):
        _need(x, self.nt, torch.float64, "x")
        _need(dJdu, 3 * self.V[self.L], torch.float64, "dJdu")
        g = torch.empty(self.E[self.L], dtype=torch.float64, device=self.device)
        its = _I()
        self._check(lib().agca_adjoint_gradient(self._h, _ptr(x), _ptr(dJdu), _ptr(g), float(rtol), int(maxit),
                                                ctypes.byref(its)), "adjoint_gradient")
        return g, its.value

    # ---- introspection ---------------------------------------------------------
    def set_tile_config(self, level: int, mode: int, block_rows: int = 8, z_chunk: int = 0):
        """Fix the tile shape of one (level, stencil mode) launch by hand."""
        self._check(lib().agca_set_tile_config(self._h, int(level), int(mode), int(block_rows), int(z_chunk)),
                    "set_tile_config")

    def autotune(self, reps: int = 10, cache: str | None = None) -> dict:
        """Pick the tile shape of every V-cycle stencil launch by timing
        (agca_autotune); returns {(level, mode): (block_rows, z_chunk)}."""
        self._check(lib().agca_autotune(self._h, int(reps), cache.encode() if cache else None), "autotune")
        out = {}
        for l in range(2, self.L + 1):
            for mode in (1, 2, 3, 4):
                by, zc = _I(), _I()
                self._check(lib().agca_tile_config(self._h, l, mode, ctypes.byref(by), ctypes.byref(zc)), "tile_config")
                out[(l, mode)] = (by.value, zc.value)
        return out

    def launch_count(self) -> int:
        n = ctypes.c_int64()
        self._check(lib().agca_launch_count(self._h, ctypes.byref(n)), "launch_count")
        return n.value

    def profile_fine(self, enable: bool):
        """enable=True starts per-launch timing of the finest-level stencil
        kernels; enable=False stops and returns (ms, bytes, flops, launches)."""
        ms, by, fl, n = _D(), _D(), _D(), ctypes.c_int64()
        self._check(lib().agca_profile_fine(self._h, 1 if enable else 0, ctypes.byref(ms), ctypes.byref(by),
                                            ctypes.byref(fl), ctypes.byref(n)), "profile_fine")
        return ms.value, by.value, fl.value, n.value

    def level_info(self, level: int) -> LevelInfo:
        info = LevelInfo()
        self._check(lib().agca_level_info(self._h, level, ctypes.byref(info)), "level_info")
        return info

    def level_data(self, level: int, field: int) -> torch.Tensor:
        info = self.level_info(level)
        E, V = info.elements, info.vertices
        shape = {FIELD_MEAN: (E, torch.float64), FIELD_MAX: (E, torch.float64), FIELD_MIN: (E, torch.float64),
                 FIELD_FLAGS: (E, torch.uint8), FIELD_LIST: (info.n_flag, torch.int32),
                 FIELD_GCA: (info.n_flag * 144, torch.float64), FIELD_DIAG: (3 * V, torch.float64),
                 FIELD_COARSE: ((3 * (info.n - 1) ** 3) ** 2, torch.float64),
                 FIELD_PMASS: (self.Vp, torch.float64), FIELD_SIDX: (V, torch.int32),
                 FIELD_STENCIL: (info.n_stencil * 135, torch.float64)}[field]
        out = torch.empty(max(1, shape[0]), dtype=shape[1], device=self.device)
        self._check(lib().agca_get_level_data(self._h, level, field, _ptr(out)), "get_level_data")
        return out[:shape[0]]


class Batch:
    """Many independent problems solved in lockstep (agca_batch_*)."""

    def __init__(self, Ns, precision: int = MIXED, device="cuda", stream: torch.cuda.Stream | None = None):
        self.Ns = [int(n) for n in Ns]
        self.n = len(self.Ns)
        self.precision = precision
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        h = _P()
        arr = (_I * self.n)(*self.Ns)
        st = lib().agca_batch_create(self.n, arr, precision, _P(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise AgcaError(st, f"agca_batch_create({self.Ns})")
        self._h = h
        sz = _SZ()
        self._check(lib().agca_batch_workspace_size(self._h, ctypes.byref(sz)), "workspace_size")
        self.workspace = torch.empty(int(sz.value), dtype=torch.uint8, device=self.device)
        self._check(lib().agca_batch_bind_workspace(self._h, _ptr(self.workspace), sz.value), "bind_workspace")
        self.gca_store = None
        self.contexts = [Context._borrowed(lib().agca_batch_context(self._h, i), N, default_levels(N), precision,
                                           self.device, self.stream, self) for i, N in enumerate(self.Ns)]

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            for c in getattr(self, "contexts", []):
                c._h = None
            _lib.agca_batch_destroy(h)
            self._h = None

    def _check(self, st, what):
        if st != 0:
            raise AgcaError(st, f"{what}: {lib().agca_batch_last_error(self._h).decode()}")

    def prepare(self, etas, nu: float = 10.0):
        for i, eta in enumerate(etas):
            _need(eta, self.contexts[i].E[self.contexts[i].L], torch.float64, f"eta[{i}]")
            self._check(lib().agca_batch_set_viscosity(self._h, i, _ptr(eta)), "set_viscosity")
        b = _SZ()
        self._check(lib().agca_batch_flag(self._h, float(nu), ctypes.byref(b)), "flag")
        self.gca_store = torch.empty(max(256, int(b.value)), dtype=torch.uint8, device=self.device)
        self._check(lib().agca_batch_bind_gca_store(self._h, _ptr(self.gca_store), b.value), "bind_gca_store")
        self._check(lib().agca_batch_setup(self._h), "setup")

    def load_vector(self, i: int, fbar: torch.Tensor):
        c = self.contexts[i]
        _need(fbar, 3 * c.E[c.L], torch.float64, "fbar")
        b = torch.empty(c.nt, dtype=torch.float64, device=self.device)
        self._check(lib().agca_batch_load_vector(self._h, i, _ptr(fbar), _ptr(b)), "load_vector")
        return b

    def vcycle(self, rs, zs=None):
        zs = [torch.empty_like(r) for r in rs] if zs is None else zs
        for i, (r, z) in enumerate(zip(rs, zs)):
            n = 3 * self.contexts[i].V[self.contexts[i].L]
            _need(r, n, torch.float64, f"r[{i}]")
            _need(z, n, torch.float64, f"z[{i}]")
        ra = (_P * self.n)(*[r.data_ptr() for r in rs])
        za = (_P * self.n)(*[z.data_ptr() for z in zs])
        self._check(lib().agca_batch_vcycle(self._h, ra, za), "vcycle")
        return zs

    def solve(self, bs, rtol: float = 1e-8, maxit: int = 20000, xs=None):
        xs = [torch.empty_like(b) for b in bs] if xs is None else xs
        for i, (b, x) in enumerate(zip(bs, xs)):
            _need(b, self.contexts[i].nt, torch.float64, f"b[{i}]")
            _need(x, self.contexts[i].nt, torch.float64, f"x[{i}]")
        ba = (_P * self.n)(*[b.data_ptr() for b in bs])
        xa = (_P * self.n)(*[x.data_ptr() for x in xs])
        its = (_I * self.n)()
        rel = (_D * self.n)()
        self._check(lib().agca_batch_solve(self._h, ba, xa, float(rtol), int(maxit), its, rel), "solve")
        return xs, list(its), list(rel)
