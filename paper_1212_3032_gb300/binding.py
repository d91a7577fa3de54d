"""Thin Python binding of the libbem C-ABI (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts numpy
arrays and torch tensors to pointers and sizes and turns negative return
codes into ``BemError``. The library must have been built (``build.build()``);
importing fails loudly if it is missing.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libbem.so")

BEM_OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "NO_MESH", -3: "OOM", -4: "CUDA", -5: "NOT_CONVERGED", -6: "TIMEOUT",
          -7: "STATE"}
BC_TRACTION, BC_DISPLACEMENT = 0, 1
WIN_NONE, WIN_HANNING, WIN_BLACKMAN = 0, 1, 2
PREC_C64_MIXED, PREC_C128 = 0, 1
GUESS_ZERO, GUESS_SEM, GUESS_MLP = 0, 1, 2
FAR_AUTO, FAR_FULL, FAR_COMPACT = 0, 1, 2
FIELD_DISPLACEMENT, FIELD_STRAIN = 0, 1
PRECOND_BLOCK3, PRECOND_LEAF, PRECOND_AUTO = 0, 1, 2

EXPORTED = [
    "bem_default_opts", "bem_create", "bem_destroy", "bem_last_error", "bem_mesh", "bem_mesh_dev",
    "bem_set_material", "bem_set_window", "bem_solve_sweep", "bem_solve_sweep_dev",
    "bem_get_frequency_solution", "bem_time_response", "bem_time_response_dev", "bem_load_dft", "bem_idft",
    "bem_assemble", "bem_operator_rows", "bem_apply", "bem_rhs", "bem_solve_assembled", "bem_sem_guess",
    "bem_set_profiling", "bem_get_profile", "bem_apply_noalloc",
    "bem_mlp_num_params", "bem_mlp_init", "bem_mlp_set_training", "bem_mlp_set_weights", "bem_mlp_get_weights",
    "bem_mlp_forward", "bem_mlp_gradient", "bem_mlp_train_step", "bem_set_aca_reuse",
    "bem_far_block_info", "bem_set_far_storage", "bem_get_far_storage",
    "bem_add_mesh", "bem_mesh_count", "bem_solve_sweep_batched", "bem_mesh_frequency_solution",
    "bem_mesh_time_response", "bem_block_tree", "bem_interior_field", "bem_interior_strain",
    "bem_interior_time_response", "bem_apply_preconditioner",
]


class BemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("restart", ctypes.c_int32), ("max_iters", ctypes.c_int32),
                ("aca_tol", ctypes.c_double), ("leaf_size", ctypes.c_int32), ("eta_adm", ctypes.c_double),
                ("precision", ctypes.c_int32), ("guess", ctypes.c_int32), ("sem_k", ctypes.c_int32),
                ("dense", ctypes.c_int32), ("precond", ctypes.c_int32)]


class FreqStats(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int32), ("iters", ctypes.c_int32), ("cycles", ctypes.c_int32),
                ("converged", ctypes.c_int32), ("s_re", ctypes.c_double), ("s_im", ctypes.c_double),
                ("rel_residual", ctypes.c_double), ("guess_residual", ctypes.c_double),
                ("assemble_ms", ctypes.c_double), ("guess_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("near_bytes", ctypes.c_int64), ("far_bytes", ctypes.c_int64), ("max_rank", ctypes.c_int32),
                ("aca_failures", ctypes.c_int32), ("sem_residual", ctypes.c_double),
                ("precond", ctypes.c_int32), ("trial_iters", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class Profile(ctypes.Structure):
    _fields_ = [("hmv_launches", ctypes.c_int64), ("hmv_ms", ctypes.c_double), ("hmv_bytes", ctypes.c_double),
                ("assemble_calls", ctypes.c_int64), ("assemble_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_int64), ("aca_blocks", ctypes.c_int64),
                ("aca_stepped", ctypes.c_int64), ("aca_failures", ctypes.c_int64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class FarStorage(ctypes.Structure):
    _fields_ = [("compact", ctypes.c_int32), ("batches", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("factor_bytes", ctypes.c_int64), ("used_bytes", ctypes.c_int64), ("regrows", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_ if name != "reserved"}


_lib = None


def block_tree(centroid, h, leaf_size=64, eta_adm=1.0, dense=False):
    """The block partition of the operator (host only): (perm, near (n, 4), far (m, 4)) int32 arrays,
    blocks as (row begin, rows, column begin, columns) in tree positions."""
    lib = load_library()
    c = np.ascontiguousarray(centroid, dtype=np.float64).reshape(-1, 3)
    hh = np.ascontiguousarray(h, dtype=np.float64).ravel()
    ne = c.shape[0]
    nn, nf = ctypes.c_int64(), ctypes.c_int64()
    perm = np.zeros(ne, dtype=np.int32)
    rc = lib.bem_block_tree(_ptr(c), _ptr(hh), ne, int(leaf_size), float(eta_adm), 1 if dense else 0, _ptr(perm), 0,
                            None, None, ctypes.byref(nn), ctypes.byref(nf))
    if rc != 0:
        raise BemError(rc, "bem_block_tree")
    near = np.zeros((nn.value, 4), dtype=np.int32)
    far = np.zeros((nf.value, 4), dtype=np.int32)
    n = max(nn.value, nf.value)
    nb = np.zeros((n, 4), dtype=np.int32)
    fb = np.zeros((n, 4), dtype=np.int32)
    rc = lib.bem_block_tree(_ptr(c), _ptr(hh), ne, int(leaf_size), float(eta_adm), 1 if dense else 0, _ptr(perm), n,
                            _ptr(nb), _ptr(fb), ctypes.byref(nn), ctypes.byref(nf))
    if rc != 0:
        raise BemError(rc, "bem_block_tree")
    near[:] = nb[:nn.value]
    far[:] = fb[:nf.value]
    return perm, near, far


def load_library(path: str = LIB_PATH):
    """Loads libbem.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libbem.so not built at {path}; run paper_1212_3032_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P, I32, I64, D = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
    sig = {
        "bem_default_opts": (None, [ctypes.POINTER(Opts)]),
        "bem_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, P]),
        "bem_destroy": (None, [P]),
        "bem_last_error": (ctypes.c_char_p, [P]),
        "bem_mesh": (ctypes.c_int, [P, P, I64, P, I64, P, ctypes.POINTER(Opts)]),
        "bem_mesh_dev": (ctypes.c_int, [P, P, I64, P, I64, P, ctypes.POINTER(Opts)]),
        "bem_set_material": (ctypes.c_int, [P, D, D, D]),
        "bem_set_window": (ctypes.c_int, [P, D, ctypes.c_int]),
        "bem_solve_sweep": (ctypes.c_int, [P, D, I32, P, P, ctypes.POINTER(Opts), P]),
        "bem_solve_sweep_dev": (ctypes.c_int, [P, D, I32, P, P, ctypes.POINTER(Opts), P]),
        "bem_get_frequency_solution": (ctypes.c_int, [P, I32, P]),
        "bem_time_response": (ctypes.c_int, [P, P, I64, P]),
        "bem_time_response_dev": (ctypes.c_int, [P, P, I64, P]),
        "bem_load_dft": (ctypes.c_int, [P, D, I32, D, P, P]),
        "bem_idft": (ctypes.c_int, [P, D, I32, D, ctypes.c_int, P, I64, P]),
        "bem_assemble": (ctypes.c_int, [P, D, D, ctypes.POINTER(Opts)]),
        "bem_operator_rows": (ctypes.c_int, [P, P, I64, P]),
        "bem_apply": (ctypes.c_int, [P, P, P]),
        "bem_rhs": (ctypes.c_int, [P, D, D, P, P]),
        "bem_solve_assembled": (ctypes.c_int, [P, P, P, P, ctypes.POINTER(Opts), P]),
        "bem_sem_guess": (ctypes.c_int, [P, I32, P, P, P]),
        "bem_set_profiling": (ctypes.c_int, [P, ctypes.c_int]),
        "bem_apply_noalloc": (ctypes.c_int, [P, P, P]),
        "bem_get_profile": (ctypes.c_int, [P, ctypes.POINTER(Profile)]),
        "bem_set_aca_reuse": (ctypes.c_int, [P, ctypes.c_int]),
        "bem_far_block_info": (ctypes.c_int, [P, I64, P, P]),
        "bem_set_far_storage": (ctypes.c_int, [P, ctypes.c_int32, I64]),
        "bem_block_tree": (ctypes.c_int, [P, P, I64, ctypes.c_int32, ctypes.c_double, ctypes.c_int32, P, I64, P, P,
                                          P, P]),
        "bem_add_mesh": (ctypes.c_int, [P, P, I64, P, I64, P, P, P]),
        "bem_mesh_count": (ctypes.c_int, [P]),
        "bem_solve_sweep_batched": (ctypes.c_int, [P, ctypes.c_double, ctypes.c_int32, P, P, P, P]),
        "bem_mesh_frequency_solution": (ctypes.c_int, [P, ctypes.c_int32, ctypes.c_int32, P]),
        "bem_mesh_time_response": (ctypes.c_int, [P, ctypes.c_int32, P, I64, P]),
        "bem_get_far_storage": (ctypes.c_int, [P, P]),
        "bem_interior_field": (ctypes.c_int, [P, I32, P, I64, P]),
        "bem_apply_preconditioner": (ctypes.c_int, [P, I32, P, P]),
        "bem_interior_strain": (ctypes.c_int, [P, I32, P, I64, D, P]),
        "bem_interior_time_response": (ctypes.c_int, [P, P, I64, I32, D, P]),
        "bem_mlp_num_params": (I64, []),
        "bem_mlp_init": (ctypes.c_int, [P, ctypes.c_uint64]),
        "bem_mlp_set_training": (ctypes.c_int, [P, I32, D]),
        "bem_mlp_set_weights": (ctypes.c_int, [P, P, I64]),
        "bem_mlp_get_weights": (ctypes.c_int, [P, P, I64]),
        "bem_mlp_forward": (ctypes.c_int, [P, P, I64, P]),
        "bem_mlp_gradient": (ctypes.c_int, [P, P, P, I64, P, P]),
        "bem_mlp_train_step": (ctypes.c_int, [P, P, P, I64, D, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def default_opts(**kw) -> Opts:
    lib = load_library()
    o = Opts()
    lib.bem_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _tptr(t, dtype=None):
    """Device pointer of a contiguous CUDA tensor (checked: layout and dtype)."""
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and str(t.dtype) != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(int(t.data_ptr()))


class Context:
    """One libbem context on one CUDA device and stream."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load_library()
        if stream is None:
            try:
                import torch
                stream = torch.cuda.current_stream(device).cuda_stream
            except Exception:
                stream = 0
        h = ctypes.c_void_p()
        rc = self.lib.bem_create(ctypes.byref(h), int(device), ctypes.c_void_p(int(stream)))
        if rc != BEM_OK:
            raise BemError(rc, "bem_create failed")
        self.h = h
        self.ne = 0
        self.n_omega = 0

    def close(self):
        if getattr(self, "h", None):
            self.lib.bem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc, allow=()):
        if rc != BEM_OK and rc not in allow:
            raise BemError(rc, self.lib.bem_last_error(self.h).decode())
        return rc

    # --- problem definition -------------------------------------------------
    def mesh(self, xyz, tri, bc_type, opts: Opts | None = None):
        xyz = _f64(xyz)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        bc = np.ascontiguousarray(bc_type, dtype=np.int8)
        self._check(self.lib.bem_mesh(self.h, _ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], _ptr(bc),
                                      ctypes.byref(opts) if opts else None))
        self.ne = tri.shape[0]

    def mesh_dev(self, xyz_t, tri_t, bc_t, opts: Opts | None = None):
        if xyz_t.dim() != 2 or xyz_t.shape[1] != 3 or tri_t.dim() != 2 or tri_t.shape[1] != 3:
            raise ValueError("xyz and tri must be (n, 3)")
        self._check(self.lib.bem_mesh_dev(self.h, _tptr(xyz_t, "torch.float64"), xyz_t.shape[0],
                                          _tptr(tri_t, "torch.int32"), tri_t.shape[0], _tptr(bc_t, "torch.int8"),
                                          ctypes.byref(opts) if opts else None))
        self.ne = int(tri_t.shape[0])

    def set_material(self, E, nu, rho):
        self._check(self.lib.bem_set_material(self.h, float(E), float(nu), float(rho)))

    def set_window(self, eta, window=WIN_NONE):
        self._check(self.lib.bem_set_window(self.h, float(eta), int(window)))

    # --- sweep ----------------------------------------------------------------
    def solve_sweep(self, T, n_omega, load_hist, pattern, opts: Opts | None = None, allow_unconverged=False):
        load = _f64(load_hist)
        pat = _f64(pattern)
        stats = (FreqStats * (n_omega // 2 + 1))()
        rc = self.lib.bem_solve_sweep(self.h, float(T), int(n_omega), _ptr(load), _ptr(pat),
                                      ctypes.byref(opts) if opts else None, stats)
        self._check(rc, allow=(-5,) if allow_unconverged else ())
        self.n_omega = n_omega
        return [s.as_dict() for s in stats]

    def solve_sweep_dev(self, T, n_omega, load_t, pattern_t, opts: Opts | None = None, allow_unconverged=False):
        stats = (FreqStats * (n_omega // 2 + 1))()
        rc = self.lib.bem_solve_sweep_dev(self.h, float(T), int(n_omega), _tptr(load_t, "torch.float64"),
                                          _tptr(pattern_t, "torch.float64"),
                                          ctypes.byref(opts) if opts else None, stats)
        self._check(rc, allow=(-5,) if allow_unconverged else ())
        self.n_omega = n_omega
        return [s.as_dict() for s in stats]

    def get_frequency_solution(self, k):
        out = np.zeros(3 * self.ne, dtype=np.complex128)
        self._check(self.lib.bem_get_frequency_solution(self.h, int(k), _ptr(out)))
        return out

    def time_response(self, dofs):
        dofs = np.ascontiguousarray(dofs, dtype=np.int64)
        out = np.zeros((self.n_omega, dofs.size), dtype=np.float64)
        self._check(self.lib.bem_time_response(self.h, _ptr(dofs), dofs.size, _ptr(out)))
        return out

    def time_response_dev(self, dofs_t, out_t):
        if out_t.numel() != self.n_omega * dofs_t.numel():
            raise ValueError("out must hold n_omega x ndof values")
        self._check(self.lib.bem_time_response_dev(self.h, _tptr(dofs_t, "torch.int64"), dofs_t.numel(),
                                                   _tptr(out_t, "torch.float64")))

    # --- interior field (representation formula) --------------------------
    def interior_field(self, k, points):
        """(npts, 3) complex displacement at interior points, solved frequency k."""
        pts = _f64(points).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 3), dtype=np.complex128)
        self._check(self.lib.bem_interior_field(self.h, int(k), _ptr(pts), pts.shape[0], _ptr(out)))
        return out

    def interior_strain(self, k, points, h):
        """(npts, 6) complex strain (xx, yy, zz, xy, yz, xz), central differences with step h."""
        pts = _f64(points).reshape(-1, 3)
        out = np.zeros((pts.shape[0], 6), dtype=np.complex128)
        self._check(self.lib.bem_interior_strain(self.h, int(k), _ptr(pts), pts.shape[0], float(h), _ptr(out)))
        return out

    def interior_time_response(self, points, quantity=FIELD_DISPLACEMENT, h=0.0):
        """(n_omega, npts, 3 or 6) float64 time histories at interior points."""
        pts = _f64(points).reshape(-1, 3)
        nc = 6 if quantity == FIELD_STRAIN else 3
        out = np.zeros((self.n_omega, pts.shape[0], nc), dtype=np.float64)
        self._check(self.lib.bem_interior_time_response(self.h, _ptr(pts), pts.shape[0], int(quantity), float(h),
                                                        _ptr(out)))
        return out

    # --- several meshes (batched sweeps) -----------------------------------
    def add_mesh(self, xyz, tri, bc_type, opts: Opts | None = None) -> int:
        xyz = _f64(xyz)
        tri = np.ascontiguousarray(tri, dtype=np.int32)
        bc = np.ascontiguousarray(bc_type, dtype=np.int8)
        mid = ctypes.c_int32(-1)
        self._check(self.lib.bem_add_mesh(self.h, _ptr(xyz), xyz.shape[0], _ptr(tri), tri.shape[0], _ptr(bc),
                                          ctypes.byref(opts) if opts else None, ctypes.byref(mid)))
        if not hasattr(self, "batch_ne"):
            self.batch_ne = []
        self.batch_ne.append(int(tri.shape[0]))
        return mid.value

    def mesh_count(self) -> int:
        n = self.lib.bem_mesh_count(self.h)
        self._check(min(n, 0))
        return n

    def solve_sweep_batched(self, T, n_omega, load_hist, patterns, opts: Opts | None = None,
                            allow_unconverged=False):
        """Sweeps every added mesh; returns one list of per-frequency stats per mesh."""
        load = _f64(load_hist)
        pats = [_f64(p) for p in patterns]
        arr = (ctypes.c_void_p * len(pats))(*[p.ctypes.data for p in pats])
        nf = n_omega // 2 + 1
        stats = (FreqStats * (nf * len(pats)))()
        rc = self.lib.bem_solve_sweep_batched(self.h, float(T), int(n_omega), _ptr(load), arr,
                                              ctypes.byref(opts) if opts else None, stats)
        self._check(rc, allow=(-5,) if allow_unconverged else ())
        self.batch_n_omega = n_omega
        return [[stats[m * nf + k].as_dict() for k in range(nf)] for m in range(len(pats))]

    def _batch_ne(self, mesh_id):
        ne = getattr(self, "batch_ne", [])
        return ne[mesh_id] if 0 <= mesh_id < len(ne) else 0  # unknown ids: the library reports the error

    def mesh_frequency_solution(self, mesh_id, k):
        out = np.zeros(3 * self._batch_ne(mesh_id), dtype=np.complex128)
        self._check(self.lib.bem_mesh_frequency_solution(self.h, int(mesh_id), int(k), _ptr(out)))
        return out

    def mesh_time_response(self, mesh_id, dofs):
        dofs = np.ascontiguousarray(dofs, dtype=np.int64)
        out = np.zeros((getattr(self, "batch_n_omega", 0), dofs.size), dtype=np.float64)
        self._check(self.lib.bem_mesh_time_response(self.h, int(mesh_id), _ptr(dofs), dofs.size, _ptr(out)))
        return out

    # --- step-level entry points -------------------------------------------
    def load_dft(self, T, n_omega, eta, load_hist):
        load = _f64(load_hist)
        out = np.zeros(n_omega // 2 + 1, dtype=np.complex128)
        self._check(self.lib.bem_load_dft(self.h, float(T), int(n_omega), float(eta), _ptr(load), _ptr(out)))
        return out

    def idft(self, T, n_omega, eta, window, Rk):
        Rk = _c128(Rk)
        if Rk.ndim == 1:
            Rk = Rk[:, None]
        ndof = Rk.shape[1]
        out = np.zeros((n_omega, ndof), dtype=np.float64)
        self._check(self.lib.bem_idft(self.h, float(T), int(n_omega), float(eta), int(window), _ptr(Rk), ndof,
                                      _ptr(out)))
        return out

    def assemble(self, s, opts: Opts | None = None):
        s = complex(s)
        self._check(self.lib.bem_assemble(self.h, s.real, s.imag, ctypes.byref(opts) if opts else None))

    def operator_rows(self, rows):
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        out = np.zeros((rows.size, 3 * self.ne), dtype=np.complex128)
        self._check(self.lib.bem_operator_rows(self.h, _ptr(rows), rows.size, _ptr(out)))
        return out

    def apply(self, x):
        x = _c128(x)
        y = np.zeros_like(x)
        self._check(self.lib.bem_apply(self.h, _ptr(x), _ptr(y)))
        return y

    def apply_preconditioner(self, x, precond=PRECOND_BLOCK3):
        """M^-1 x with the assembled operator's 3 x 3 or leaf-block preconditioner."""
        x = _c128(x)
        y = np.zeros_like(x)
        self._check(self.lib.bem_apply_preconditioner(self.h, int(precond), _ptr(x), _ptr(y)))
        return y

    def rhs(self, p, pattern):
        p = complex(p)
        pat = _f64(pattern)
        b = np.zeros(3 * self.ne, dtype=np.complex128)
        self._check(self.lib.bem_rhs(self.h, p.real, p.imag, _ptr(pat), _ptr(b)))
        return b

    def solve_assembled(self, b, x0=None, opts: Opts | None = None, allow_unconverged=False):
        b = _c128(b)
        x = np.zeros_like(b)
        st = FreqStats()
        x0p = _ptr(_c128(x0)) if x0 is not None else None
        x0keep = _c128(x0) if x0 is not None else None
        if x0keep is not None:
            x0p = _ptr(x0keep)
        rc = self.lib.bem_solve_assembled(self.h, _ptr(b), x0p, _ptr(x), ctypes.byref(opts) if opts else None,
                                          ctypes.byref(st))
        self._check(rc, allow=(-5,) if allow_unconverged else ())
        return x, st.as_dict()

    def sem_guess(self, X, b):
        X = _c128(X)
        if X.ndim == 1:
            X = X[None, :]
        b = _c128(b)
        a0 = np.zeros_like(b)
        self._check(self.lib.bem_sem_guess(self.h, X.shape[0], _ptr(X) if X.size else None, _ptr(b), _ptr(a0)))
        return a0

    def apply_noalloc(self, x_t, y_t):
        """y = A x on device tensors (complex64, caller dof order); allocates nothing."""
        for t in (x_t, y_t):
            if str(t.dtype) != "torch.complex64" or t.numel() != 3 * self.ne:
                raise ValueError("x and y must be complex64 tensors of 3 ne values")
        self._check(self.lib.bem_apply_noalloc(self.h, _tptr(x_t), _tptr(y_t)))

    # --- learned initial guess ----------------------------------------------
    def mlp_num_params(self) -> int:
        return int(self.lib.bem_mlp_num_params())

    def mlp_init(self, seed: int):
        self._check(self.lib.bem_mlp_init(self.h, int(seed)))

    def mlp_set_training(self, steps_per_frequency: int, lr: float):
        self._check(self.lib.bem_mlp_set_training(self.h, int(steps_per_frequency), float(lr)))

    def mlp_set_weights(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float32)
        self._check(self.lib.bem_mlp_set_weights(self.h, _ptr(th), th.size))

    def mlp_get_weights(self):
        th = np.zeros(self.mlp_num_params(), dtype=np.float32)
        self._check(self.lib.bem_mlp_get_weights(self.h, _ptr(th), th.size))
        return th

    def mlp_forward(self, x):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.zeros((x.shape[0], 2), dtype=np.float32)
        self._check(self.lib.bem_mlp_forward(self.h, _ptr(x), x.shape[0], _ptr(y)))
        return y

    def mlp_gradient(self, x, t):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        g = np.zeros(self.mlp_num_params(), dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.bem_mlp_gradient(self.h, _ptr(x), _ptr(t), x.shape[0], _ptr(g), ctypes.byref(loss)))
        return loss.value, g

    def mlp_train_step(self, x, t, lr):
        x = np.ascontiguousarray(x, dtype=np.float32)
        t = np.ascontiguousarray(t, dtype=np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.bem_mlp_train_step(self.h, _ptr(x), _ptr(t), x.shape[0], float(lr), ctypes.byref(loss)))
        return loss.value

    # --- measurement -------------------------------------------------------
    def set_profiling(self, on: bool):
        self._check(self.lib.bem_set_profiling(self.h, 1 if on else 0))

    def set_aca_reuse(self, on: bool):
        self._check(self.lib.bem_set_aca_reuse(self.h, 1 if on else 0))

    def far_block_info(self):
        """(nblocks, 4) int32: rows, cols (elements), rank, rank settled by reused pivots (-1: no reuse)."""
        n = ctypes.c_int64()
        self._check(self.lib.bem_far_block_info(self.h, 0, None, ctypes.byref(n)))
        info = np.zeros((n.value, 4), dtype=np.int32)
        if n.value:
            self._check(self.lib.bem_far_block_info(self.h, n.value, _ptr(info), ctypes.byref(n)))
        return info

    def set_far_storage(self, mode: int, workspace_bytes: int = 0):
        """Factor storage (FAR_AUTO / FAR_FULL / FAR_COMPACT) of the meshes set after this call."""
        self._check(self.lib.bem_set_far_storage(self.h, int(mode), int(workspace_bytes)))

    def far_storage(self):
        f = FarStorage()
        self._check(self.lib.bem_get_far_storage(self.h, ctypes.byref(f)))
        return f.as_dict()

    def get_profile(self):
        p = Profile()
        self._check(self.lib.bem_get_profile(self.h, ctypes.byref(p)))
        return p.as_dict()
