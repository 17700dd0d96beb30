"""ctypes binding of libsem_gb300.so (include/sem.h): argument marshalling only.

Device memory comes from PyTorch tensors (their data pointers are passed
through), streams from torch.cuda.current_stream().  Every computation runs in
the library's CUDA kernels; there is no CPU or PyTorch fallback -- if the
library is missing, lib() raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_lib", "libsem_gb300.so")

SEM_OK = 0
SEM_ERR_INVALID_ARG = -1
SEM_ERR_CUDA = -2
SEM_ERR_MESH = -3
SEM_ERR_WORKSPACE = -4
SEM_ERR_NAN = -5
SEM_ERR_NOT_CONVERGED = -6
SEM_ERR_TIMEOUT = -7
SEM_ERR_UNSUPPORTED = -8
SEM_F64, SEM_F32, SEM_F64_PAIR = 0, 1, 2
SEM_GEOM_F32 = 1
SEM_GEOM_RX = 2
SEM_GEOM_PAIR = 4
SEM_GEOM_AFFINE = 8
SEM_GEOM_BF16 = 16
SEM_PCG_F64, SEM_PCG_MIXED, SEM_PCG_F64_PAIR = 0, 1, 2
SEM_KRYLOV_CG, SEM_KRYLOV_FGMRES = 0, 1

FIELD_MASS, FIELD_MULT, FIELD_DINV = 0, 1, 2


class MeshDesc(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("nel", ctypes.c_int * 3), ("periodic", ctypes.c_int * 3),
                ("dirichlet_faces", ctypes.c_int), ("vertices", ctypes.POINTER(ctypes.c_double)),
                ("geom_flags", ctypes.c_int)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("E", ctypes.c_int64), ("nloc", ctypes.c_int64),
                ("nglob", ctypes.c_int64), ("n_paper", ctypes.c_int64),
                ("n_shared_groups", ctypes.c_int64), ("n_shared_points", ctypes.c_int64),
                ("workspace_bytes", ctypes.c_size_t)]


class PcgOpts(ctypes.Structure):
    _fields_ = [("tol", ctypes.c_double), ("tol_is_relative", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("precision", ctypes.c_int), ("inner_tol", ctypes.c_double), ("h1", ctypes.c_double),
                ("h2", ctypes.c_double), ("check_every", ctypes.c_int), ("use_initial_guess", ctypes.c_int),
                ("profile", ctypes.c_int), ("dinv", ctypes.c_void_p), ("mixed_restart", ctypes.c_int),
                ("schwarz", ctypes.c_void_p), ("coarse_iters", ctypes.c_int), ("coarse_tol", ctypes.c_double),
                ("outer_pair", ctypes.c_int), ("schwarz_mid", ctypes.c_void_p), ("mid_weight", ctypes.c_double),
                ("inner_adapt", ctypes.c_double), ("krylov", ctypes.c_int), ("gmres_restart", ctypes.c_int)]


class PcgStats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("outer_iters", ctypes.c_int), ("status", ctypes.c_int),
                ("rel_res", ctypes.c_double), ("abs_res", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("wall_ms", ctypes.c_double), ("ax_ms", ctypes.c_double), ("gs_ms", ctypes.c_double),
                ("ax_launches", ctypes.c_int), ("kernel_launches", ctypes.c_int),
                ("outer_ax_ms", ctypes.c_double), ("outer_ax_launches", ctypes.c_int),
                ("init_rel_res", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SEM_TUNE_MAX_CONFIGS = 48


class TuneResult(ctypes.Structure):
    _fields_ = [("best_stages", ctypes.c_int), ("best_cap", ctypes.c_int), ("best_epc", ctypes.c_int),
                ("best_ms", ctypes.c_float), ("configs", ctypes.c_int),
                ("stages", ctypes.c_int * SEM_TUNE_MAX_CONFIGS), ("caps", ctypes.c_int * SEM_TUNE_MAX_CONFIGS),
                ("epcs", ctypes.c_int * SEM_TUNE_MAX_CONFIGS), ("ms", ctypes.c_float * SEM_TUNE_MAX_CONFIGS)]


_VP = ctypes.c_void_p
_SIGS = {
    "sem_version": ([], ctypes.c_char_p),
    "sem_last_error": ([], ctypes.c_char_p),
    "sem_status_string": ([ctypes.c_int], ctypes.c_char_p),
    "sem_mesh_workspace_bytes": ([ctypes.POINTER(MeshDesc)], ctypes.c_size_t),
    "sem_mesh_create": ([ctypes.POINTER(MeshDesc), _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "sem_mesh_destroy": ([_VP], ctypes.c_int),
    "sem_mesh_get_info": ([_VP, ctypes.POINTER(MeshInfo)], ctypes.c_int),
    "sem_mesh_coords": ([_VP, _VP, _VP], ctypes.c_int),
    "sem_mesh_field": ([_VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "sem_ax": ([_VP, _VP, _VP, ctypes.c_int, _VP], ctypes.c_int),
    "sem_helmholtz": ([_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP], ctypes.c_int),
    "sem_dssum": ([_VP, _VP, ctypes.c_int, ctypes.c_int, _VP], ctypes.c_int),
    "sem_scatter": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_glsc3": ([_VP, _VP, _VP, _VP, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_glsc3_noalloc": ([_VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_pcg_scratch_bytes": ([_VP, ctypes.POINTER(PcgOpts)], ctypes.c_size_t),
    "sem_pcg_solve": ([_VP, _VP, _VP, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgStats), _VP, ctypes.c_size_t,
                       _VP], ctypes.c_int),
    "sem_pcg_host_scratch_bytes": ([_VP, ctypes.POINTER(PcgOpts)], ctypes.c_size_t),
    "sem_pcg_solve_host": ([_VP, _VP, _VP, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgStats), _VP,
                            ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_mesh_check_device_error": ([_VP, ctypes.POINTER(ctypes.c_int), _VP], ctypes.c_int),
    "sem_wait_selftest": ([_VP, ctypes.c_int, ctypes.c_double, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_gemm_bf16_splitk_work_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "sem_gemm_bf16_splitk": ([_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                              ctypes.c_int, _VP, ctypes.c_size_t, _VP, _VP], ctypes.c_int),
    "sem_gemm_bf16": ([_VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_int, _VP, _VP,
                       ctypes.c_int, _VP, _VP], ctypes.c_int),
    "sem_mlp_workspace_bytes": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_size_t),
    "sem_mlp_create": ([ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t,
                        ctypes.POINTER(_VP)], ctypes.c_int),
    "sem_mlp_destroy": ([_VP], ctypes.c_int),
    "sem_mlp_num_params": ([_VP], ctypes.c_size_t),
    "sem_mlp_set_params": ([_VP, _VP, _VP], ctypes.c_int),
    "sem_mlp_get_params": ([_VP, _VP, _VP], ctypes.c_int),
    "sem_mlp_get_grads": ([_VP, _VP, _VP], ctypes.c_int),
    "sem_mlp_forward": ([_VP, _VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "sem_mlp_grad": ([_VP, _VP, _VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                      _VP], ctypes.c_int),
    "sem_mlp_grad_energy": ([_VP, _VP, _VP, _VP, ctypes.c_int, ctypes.c_double, ctypes.c_int, _VP, ctypes.c_size_t,
                             ctypes.POINTER(ctypes.c_double), _VP], ctypes.c_int),
    "sem_mlp_adam": ([_VP, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_double, _VP], ctypes.c_int),
    "sem_guess_residual": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_guess_residual_pair": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_guess_features": ([_VP, _VP, _VP, _VP, _VP, _VP, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                            _VP, ctypes.c_int, _VP], ctypes.c_int),
    "sem_ns_step_begin": ([_VP, ctypes.c_double, _VP], ctypes.c_int),
    "sem_ns_step_finish": ([_VP, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgOpts), _VP, ctypes.POINTER(PcgStats),
                            ctypes.POINTER(PcgStats), _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_ns_set": ([_VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "sem_ns_get_steps": ([_VP], ctypes.c_int),
    "sem_ns_set_steps": ([_VP, ctypes.c_int], ctypes.c_int),
    "sem_guess_target": ([_VP, _VP, _VP, _VP, _VP, ctypes.c_double, _VP, ctypes.c_int, _VP], ctypes.c_int),
    "sem_guess_apply": ([_VP, _VP, ctypes.c_int, _VP, _VP, _VP, ctypes.c_double, _VP, _VP], ctypes.c_int),
    "sem_pcg_batched_scratch_bytes": ([_VP, ctypes.c_int, ctypes.POINTER(PcgOpts)], ctypes.c_size_t),
    "sem_pcg_solve_batched_schwarz": ([_VP, _VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(PcgOpts), _VP, _VP,
                                       ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_pcg_solve_batched": ([_VP, ctypes.c_int, _VP, _VP, ctypes.POINTER(PcgOpts), _VP, _VP, ctypes.c_size_t, _VP],
                              ctypes.c_int),
    "sem_autotune_scratch_bytes": ([_VP], ctypes.c_size_t),
    "sem_autotune_operator": ([_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(TuneResult)],
                              ctypes.c_int),
    "sem_autotune_set": ([_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
    "sem_autotune_reset": ([], ctypes.c_int),
    "sem_gradient": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_advect": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_weak_div": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_ns_workspace_bytes": ([_VP], ctypes.c_size_t),
    "sem_ns_create": ([_VP, ctypes.c_double, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "sem_ns_destroy": ([_VP], ctypes.c_int),
    "sem_ns_set_velocity": ([_VP, _VP, _VP], ctypes.c_int),
    "sem_ns_get": ([_VP, ctypes.c_int, _VP, _VP], ctypes.c_int),
    "sem_ns_scratch_bytes": ([_VP, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgOpts)], ctypes.c_size_t),
    "sem_ns_step": ([_VP, ctypes.c_double, ctypes.POINTER(PcgOpts), ctypes.POINTER(PcgOpts), _VP,
                     ctypes.POINTER(PcgStats), ctypes.POINTER(PcgStats), _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_ns_kinetic_energy": ([_VP, ctypes.POINTER(ctypes.c_double), _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_ns_dealias_bytes": ([_VP], ctypes.c_size_t),
    "sem_ns_set_scheme": ([_VP, ctypes.c_int, ctypes.c_int, _VP, ctypes.c_size_t, _VP], ctypes.c_int),
    "sem_ns_advect": ([_VP, _VP, _VP, _VP], ctypes.c_int),
    "sem_schwarz_workspace_bytes": ([_VP, _VP], ctypes.c_size_t),
    "sem_schwarz_create": ([_VP, _VP, _VP, ctypes.c_size_t, _VP, ctypes.POINTER(_VP)], ctypes.c_int),
    "sem_schwarz_destroy": ([_VP], ctypes.c_int),
    "sem_schwarz_problems": ([_VP], ctypes.c_int),
    "sem_schwarz_fdm_1d": ([ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, _VP, _VP],
                           ctypes.c_int),
    "sem_schwarz_line_table": ([ctypes.c_int, _VP, ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
    "sem_schwarz_coarse_operator": ([_VP, _VP, ctypes.c_int, _VP, _VP, _VP], ctypes.c_int),
    "sem_schwarz_mid_work_bytes": ([_VP], ctypes.c_size_t),
    "sem_schwarz_apply3": ([_VP, _VP, ctypes.c_double, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP, ctypes.c_size_t,
                            _VP], ctypes.c_int),
    "sem_schwarz_apply": ([_VP, _VP, _VP, ctypes.c_int, ctypes.c_double, _VP], ctypes.c_int),
    "sem_perf_model": ([ctypes.c_int, _VP, _VP, ctypes.c_double, ctypes.POINTER(ctypes.c_double), _VP],
                       ctypes.c_int),
}

_lib = None
_lock = threading.Lock()


def exported_names() -> list[str]:
    return list(_SIGS)


def lib() -> ctypes.CDLL:
    """Load the library (raises if it has not been built: no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(SO):
                raise RuntimeError(f"{SO} not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
            L = ctypes.CDLL(SO)
            for name, (args, res) in _SIGS.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


class SemError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().sem_last_error().decode()
        super().__init__(f"{where}: status {status} ({lib().sem_status_string(status).decode()}): {msg}")
        self.status = status


def check(status: int, where: str) -> int:
    if status != SEM_OK:
        raise SemError(status, where)
    return status


def _stream():
    import torch
    return _VP(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return _VP(t.data_ptr())


class Mesh:
    """A box mesh living in a caller-owned (PyTorch) device workspace."""

    def __init__(self, N, nel, periodic, faces, vertices, geom_f32: bool = False, geom_rx: bool = False,
                 geom_pair: bool = False, geom_affine: bool = False, geom_bf16: bool = False):
        import numpy as np
        import torch
        self._verts = np.ascontiguousarray(vertices, dtype=np.float64).reshape(-1, 8, 3)
        d = MeshDesc()
        d.N = int(N)
        d.nel[:] = [int(a) for a in nel]
        d.periodic[:] = [int(bool(a)) for a in periodic]
        d.dirichlet_faces = int(faces)
        d.vertices = self._verts.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.geom_flags = ((SEM_GEOM_F32 if geom_f32 else 0) | (SEM_GEOM_RX if geom_rx else 0)
                        | (SEM_GEOM_PAIR if geom_pair else 0) | (SEM_GEOM_AFFINE if geom_affine else 0)
                        | (SEM_GEOM_BF16 if geom_bf16 else 0))
        self.desc = d
        nbytes = lib().sem_mesh_workspace_bytes(ctypes.byref(d))
        if nbytes == 0:
            raise SemError(SEM_ERR_INVALID_ARG, "sem_mesh_workspace_bytes")
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
        base = self.workspace.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        h = _VP()
        check(lib().sem_mesh_create(ctypes.byref(d), _VP(self._ws_ptr), nbytes, _stream(), ctypes.byref(h)),
              "sem_mesh_create")
        self.handle = h
        info = MeshInfo()
        check(lib().sem_mesh_get_info(h, ctypes.byref(info)), "sem_mesh_get_info")
        self.info = info
        self.N, self.E, self.nloc, self.nglob = info.N, info.E, info.nloc, info.nglob
        self.npt = (self.N + 1) ** 3
        self._red = torch.empty(1024 * 8 + 256, dtype=torch.uint8, device="cuda")
        self._res = torch.empty(1, dtype=torch.float64, device="cuda")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.sem_mesh_destroy(h)
            self.handle = None

    # ---- mesh data
    def coords(self):
        import torch
        xyz = torch.empty((3, self.E, self.npt), dtype=torch.float64, device="cuda")
        check(lib().sem_mesh_coords(self.handle, _ptr(xyz), _stream()), "sem_mesh_coords")
        return xyz

    def field(self, which: int):
        import torch
        out = torch.empty(self.nloc, dtype=torch.float64, device="cuda")
        check(lib().sem_mesh_field(self.handle, int(which), _ptr(out), _stream()), "sem_mesh_field")
        return out

    # ---- operators
    def ax(self, u, w=None, pair: bool = False):
        """w = A_L u; FP64 or FP32 by u's dtype; pair=True: FP64 fields with the
        operator evaluated in FP32-pair arithmetic (SEM_F64_PAIR)."""
        import torch
        if w is None:
            w = torch.empty_like(u)
        dt = SEM_F64 if u.dtype == torch.float64 else SEM_F32
        if pair:
            dt = SEM_F64_PAIR
        check(lib().sem_ax(self.handle, _ptr(u), _ptr(w), dt, _stream()), "sem_ax")
        return w

    def helmholtz(self, h1, h2, u, w=None):
        import torch
        if w is None:
            w = torch.empty_like(u)
        check(lib().sem_helmholtz(self.handle, float(h1), float(h2), _ptr(u), _ptr(w), _stream()), "sem_helmholtz")
        return w

    def dssum(self, u, mask: bool = True):
        import torch
        dt = SEM_F64 if u.dtype == torch.float64 else SEM_F32
        check(lib().sem_dssum(self.handle, _ptr(u), dt, int(bool(mask)), _stream()), "sem_dssum")
        return u

    def scatter(self, u_glob):
        import torch
        out = torch.empty(self.nloc, dtype=torch.float64, device="cuda")
        check(lib().sem_scatter(self.handle, _ptr(u_glob), _ptr(out), _stream()), "sem_scatter")
        return out

    def glsc3(self, a, b) -> float:
        base = (self._red.data_ptr() + 255) // 256 * 256
        check(lib().sem_glsc3(self.handle, _ptr(a), _ptr(b), _ptr(self._res), _VP(base), 1024 * 8 + 64,
                              _stream()), "sem_glsc3")
        return float(self._res.item())

    def glsc3_noalloc(self, a, b) -> float:
        """sem_glsc3_noalloc: the same product with the library's static scratch."""
        check(lib().sem_glsc3_noalloc(self.handle, _ptr(a), _ptr(b), _ptr(self._res), _stream()),
              "sem_glsc3_noalloc")
        return float(self._res.item())

    def pcg_opts(self, tol=1e-10, max_iter=10000, precision=SEM_PCG_F64, inner_tol=1e-4, h1=1.0, h2=0.0,
                 check_every=16, use_initial_guess=False, relative=True, profile=False,
                 mixed_restart=False, schwarz=None, coarse_iters=3, coarse_tol=1e-2,
                 outer_pair=False, schwarz_mid=None, mid_weight=0.15, inner_adapt=0.0, krylov=0,
                 gmres_restart=0) -> PcgOpts:
        """Solver options; schwarz: a Schwarz object (hybrid Schwarz inner
        preconditioner of the mixed solver), its coarse level solved by
        coarse_iters Jacobi-CG iterations (3: on the 32^3 channel, N = 7, more
        do not lower the outer iteration count) to coarse_tol; inner_adapt:
        theta of the adaptive inner tolerance (0: inner_tol every round);
        krylov: SEM_KRYLOV_CG or SEM_KRYLOV_FGMRES (gmres_restart: cycle
        length, 0 = 30)."""
        o = PcgOpts()
        o.inner_adapt = float(inner_adapt)
        o.krylov, o.gmres_restart = int(krylov), int(gmres_restart)
        o.schwarz = schwarz.handle.value if schwarz is not None else None
        o.schwarz_mid = schwarz_mid.handle.value if schwarz_mid is not None else None
        o.mid_weight = float(mid_weight)
        o.coarse_iters, o.coarse_tol = int(coarse_iters), float(coarse_tol)
        o.outer_pair = int(bool(outer_pair))
        o.profile = int(bool(profile))
        o.mixed_restart = int(bool(mixed_restart))
        o.tol, o.tol_is_relative, o.max_iter, o.precision = float(tol), int(relative), int(max_iter), int(precision)
        o.inner_tol, o.h1, o.h2 = float(inner_tol), float(h1), float(h2)
        o.check_every, o.use_initial_guess = int(check_every), int(bool(use_initial_guess))
        return o

    def pcg_scratch(self, opts: PcgOpts):
        import torch
        n = lib().sem_pcg_scratch_bytes(self.handle, ctypes.byref(opts))
        return torch.empty(n + 256, dtype=torch.uint8, device="cuda")

    def pcg(self, b, x=None, scratch=None, raise_on_error=True, **kw):
        """Solve with sem_pcg_solve; returns (x, stats dict)."""
        import torch
        opts = self.pcg_opts(use_initial_guess=x is not None, **kw)
        if x is None:
            x = torch.zeros_like(b)
        if scratch is None:
            scratch = self.pcg_scratch(opts)
        base = (scratch.data_ptr() + 255) // 256 * 256
        nbytes = scratch.numel() - (base - scratch.data_ptr())
        st = PcgStats()
        status = lib().sem_pcg_solve(self.handle, _ptr(b), _ptr(x), ctypes.byref(opts), ctypes.byref(st),
                                     _VP(base), nbytes, _stream())
        if raise_on_error and status not in (SEM_OK,):
            raise SemError(status, "sem_pcg_solve")
        return x, st.as_dict()

    def pcg_host_scratch(self, opts: PcgOpts):
        import torch
        n = lib().sem_pcg_host_scratch_bytes(self.handle, ctypes.byref(opts))
        return torch.empty(n + 256, dtype=torch.uint8, device="cuda")

    def pcg_host(self, b_host, x_host, scratch=None, raise_on_error=True, use_initial_guess=False, **kw):
        """sem_pcg_solve_host: b_host / x_host are CPU float64 tensors (pinned
        for asynchronous copies); the solution is written into x_host."""
        opts = self.pcg_opts(use_initial_guess=use_initial_guess, **kw)
        if scratch is None:
            scratch = self.pcg_host_scratch(opts)
        base = (scratch.data_ptr() + 255) // 256 * 256
        nbytes = scratch.numel() - (base - scratch.data_ptr())
        st = PcgStats()
        status = lib().sem_pcg_solve_host(self.handle, _ptr(b_host), _ptr(x_host), ctypes.byref(opts),
                                          ctypes.byref(st), _VP(base), nbytes, _stream())
        if raise_on_error and status != SEM_OK:
            raise SemError(status, "sem_pcg_solve_host")
        return x_host, st.as_dict()

    def autotune_set(self, dtype=SEM_F32, fused_cg=True, stages=2, cap=0, epc=1):
        """sem_autotune_set: this order's launch shape, without timing."""
        check(lib().sem_autotune_set(self.handle, int(dtype), int(bool(fused_cg)), int(stages), int(cap), int(epc)),
              "sem_autotune_set")

    def autotune(self, dtype=SEM_F32, fused_cg=True):
        """sem_autotune_operator for this mesh's order; returns the result dict."""
        import torch
        n = lib().sem_autotune_scratch_bytes(self.handle)
        scr = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        base = (scr.data_ptr() + 255) // 256 * 256
        r = TuneResult()
        check(lib().sem_autotune_operator(self.handle, int(dtype), int(bool(fused_cg)), _VP(base), n, _stream(),
                                          ctypes.byref(r)), "sem_autotune_operator")
        k = min(r.configs, SEM_TUNE_MAX_CONFIGS)
        return {"best_stages": r.best_stages, "best_cap": r.best_cap, "best_epc": r.best_epc, "best_ms": r.best_ms,
                "table": [(r.stages[i], r.caps[i], r.epcs[i], r.ms[i]) for i in range(k)]}

    # ---- Navier-Stokes building blocks
    def gradient(self, f):
        import torch
        g = torch.empty((3, self.nloc), dtype=torch.float64, device="cuda")
        check(lib().sem_gradient(self.handle, _ptr(f), _ptr(g), _stream()), "sem_gradient")
        return g

    def advect(self, u):
        import torch
        nl = torch.empty((3, self.nloc), dtype=torch.float64, device="cuda")
        check(lib().sem_advect(self.handle, _ptr(u), _ptr(nl), _stream()), "sem_advect")
        return nl

    def weak_div(self, F):
        import torch
        w = torch.empty(self.nloc, dtype=torch.float64, device="cuda")
        check(lib().sem_weak_div(self.handle, _ptr(F), _ptr(w), _stream()), "sem_weak_div")
        return w

    def check_device_error(self) -> int:
        c = ctypes.c_int()
        check(lib().sem_mesh_check_device_error(self.handle, ctypes.byref(c), _stream()), "check_device_error")
        return c.value

    def wait_selftest(self, kind: int, limit_s: float):
        """sem_wait_selftest: a bounded wait on something nothing completes
        (kind 0 mbarrier, 1 grid barrier); its code lands in the error word."""
        import torch
        scr = torch.empty(16 + 256, dtype=torch.uint8, device="cuda")
        base = (scr.data_ptr() + 255) // 256 * 256
        check(lib().sem_wait_selftest(self.handle, int(kind), float(limit_s), _VP(base), 16, _stream()),
              "sem_wait_selftest")
        return scr


class NSState:
    """sem_ns_* time stepper on a fully periodic mesh (built with geom_rx)."""

    def __init__(self, mesh: Mesh, Re: float):
        import torch
        self.mesh = mesh
        n = lib().sem_ns_workspace_bytes(mesh.handle)
        self.workspace = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = _VP()
        check(lib().sem_ns_create(mesh.handle, float(Re), _VP(base), n, _stream(), ctypes.byref(h)), "sem_ns_create")
        self.handle = h
        self._scratch = None
        self._scratch_key = None
        self._red = torch.empty(32768 + 256, dtype=torch.uint8, device="cuda")

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.sem_ns_destroy(h)
            self.handle = None

    def set_velocity(self, u):
        check(lib().sem_ns_set_velocity(self.handle, _ptr(u), _stream()), "sem_ns_set_velocity")

    def set_scheme(self, order: int = 2, dealias: bool = False):
        """sem_ns_set_scheme; the dealiasing buffer is kept by this object."""
        import torch
        self._dealias = None
        ptr, n = None, 0
        if dealias:
            n = lib().sem_ns_dealias_bytes(self.mesh.handle)
            self._dealias = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
            ptr = _VP((self._dealias.data_ptr() + 255) // 256 * 256)
        check(lib().sem_ns_set_scheme(self.handle, int(order), int(bool(dealias)), ptr, n, _stream()),
              "sem_ns_set_scheme")

    def advect(self, u):
        """The state's advection term of u ([3, nloc] device tensor)."""
        import torch
        out = torch.empty_like(u)
        check(lib().sem_ns_advect(self.handle, _ptr(u), _ptr(out), _stream()), "sem_ns_advect")
        return out

    def get(self, which: int):
        import torch
        out = torch.empty(self.mesh.nloc, dtype=torch.float64, device="cuda")
        check(lib().sem_ns_get(self.handle, int(which), _ptr(out), _stream()), "sem_ns_get")
        return out

    def step(self, dt, popts: PcgOpts, vopts: PcgOpts, p_guess=None):
        import torch
        need = lib().sem_ns_scratch_bytes(self.handle, ctypes.byref(popts), ctypes.byref(vopts))
        if self._scratch is None or self._scratch.numel() < need + 256:
            self._scratch = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        base = (self._scratch.data_ptr() + 255) // 256 * 256
        nbytes = self._scratch.numel() - (base - self._scratch.data_ptr())
        ps = PcgStats()
        vs = (PcgStats * 3)()
        guess = _ptr(p_guess) if p_guess is not None else None
        check(lib().sem_ns_step(self.handle, float(dt), ctypes.byref(popts), ctypes.byref(vopts), guess,
                                ctypes.byref(ps), vs, _VP(base), nbytes, _stream()), "sem_ns_step")
        return ps.as_dict(), [v.as_dict() for v in vs]

    def step_begin(self, dt):
        check(lib().sem_ns_step_begin(self.handle, float(dt), _stream()), "sem_ns_step_begin")

    def step_finish(self, popts: PcgOpts, vopts: PcgOpts, p_guess=None):
        import torch
        need = lib().sem_ns_scratch_bytes(self.handle, ctypes.byref(popts), ctypes.byref(vopts))
        if self._scratch is None or self._scratch.numel() < need + 256:
            self._scratch = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        base = (self._scratch.data_ptr() + 255) // 256 * 256
        nbytes = self._scratch.numel() - (base - self._scratch.data_ptr())
        ps = PcgStats()
        vs = (PcgStats * 3)()
        guess = _ptr(p_guess) if p_guess is not None else None
        check(lib().sem_ns_step_finish(self.handle, ctypes.byref(popts), ctypes.byref(vopts), guess,
                                       ctypes.byref(ps), vs, _VP(base), nbytes, _stream()), "sem_ns_step_finish")
        return ps.as_dict(), [v.as_dict() for v in vs]

    SLOTS = 19

    def checkpoint(self):
        """Device copies of every state field plus the step count."""
        return [self.get(w) for w in range(self.SLOTS)], lib().sem_ns_get_steps(self.handle)

    def restore(self, ck):
        fields, steps = ck
        for w, f in enumerate(fields):
            check(lib().sem_ns_set(self.handle, w, _ptr(f), _stream()), "sem_ns_set")
        check(lib().sem_ns_set_steps(self.handle, int(steps)), "sem_ns_set_steps")

    def kinetic_energy(self) -> float:
        e = ctypes.c_double()
        base = (self._red.data_ptr() + 255) // 256 * 256
        check(lib().sem_ns_kinetic_energy(self.handle, ctypes.byref(e), _VP(base), 32768, _stream()),
              "sem_ns_kinetic_energy")
        return e.value


def gemm_bf16(A, B, bias=None, act=0, out32=True, out16=False, err=None, work=None):
    """sem_gemm_bf16: act(A @ B^T + bias) with A [M, K], B [N, K] bfloat16
    CUDA tensors; work (a uint8 CUDA tensor): split-K work space
    (sem_gemm_bf16_splitk); returns (C32 or None, C16 or None)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    c32 = torch.empty((M, N), dtype=torch.float32, device="cuda") if out32 else None
    c16 = torch.empty((M, N), dtype=torch.bfloat16, device="cuda") if out16 else None
    if err is None:
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
    args = (_ptr(A), _ptr(B), M, N, K, _ptr(bias) if bias is not None else None, int(act),
            _ptr(c32) if c32 is not None else None, _ptr(c16) if c16 is not None else None, N)
    if work is not None:
        base = (work.data_ptr() + 255) // 256 * 256
        nb = work.numel() - (base - work.data_ptr())
        check(lib().sem_gemm_bf16_splitk(*args, _VP(base), nb, _ptr(err), _stream()), "sem_gemm_bf16_splitk")
    else:
        check(lib().sem_gemm_bf16(*args, _ptr(err), _stream()), "sem_gemm_bf16")
    return c32, c16


def gemm_splitk_work(M, N, K):
    """A work space for sem_gemm_bf16_splitk (16 slices)."""
    import torch
    return torch.empty(lib().sem_gemm_bf16_splitk_work_bytes(M, N, K) + 256, dtype=torch.uint8, device="cuda")


class MLP:
    """sem_mlp_*: the element-local guess network (dimensions multiples of 128)."""
    ORDER = ("W1", "b1", "W2", "b2", "W3", "b3")

    def __init__(self, n_in, n_hidden, n_out, max_rows):
        import torch
        self.I, self.H, self.O, self.R = int(n_in), int(n_hidden), int(n_out), int(max_rows)
        n = lib().sem_mlp_workspace_bytes(self.I, self.H, self.O, self.R)
        if n == 0:
            raise SemError(SEM_ERR_INVALID_ARG, "sem_mlp_workspace_bytes")
        self.workspace = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = _VP()
        check(lib().sem_mlp_create(self.I, self.H, self.O, self.R, _VP(base), n, ctypes.byref(h)), "sem_mlp_create")
        self.handle = h
        self.P = lib().sem_mlp_num_params(h)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.sem_mlp_destroy(h)
            self.handle = None

    def _flat(self, params):
        import numpy as np
        return np.ascontiguousarray(np.concatenate([np.asarray(params[k], np.float32).reshape(-1)
                                                    for k in self.ORDER]))

    def _unflat(self, flat):
        shapes = {"W1": (self.H, self.I), "b1": (self.H,), "W2": (self.H, self.H), "b2": (self.H,),
                  "W3": (self.O, self.H), "b3": (self.O,)}
        out, o = {}, 0
        for k in self.ORDER:
            n = 1
            for s in shapes[k]:
                n *= s
            out[k] = flat[o:o + n].reshape(shapes[k]).copy()
            o += n
        return out

    def set_params(self, params):
        flat = self._flat(params)
        assert flat.size == self.P
        check(lib().sem_mlp_set_params(self.handle, flat.ctypes.data_as(_VP), _stream()), "sem_mlp_set_params")

    def get_params(self):
        import numpy as np
        flat = np.zeros(self.P, np.float32)
        check(lib().sem_mlp_get_params(self.handle, flat.ctypes.data_as(_VP), _stream()), "sem_mlp_get_params")
        return self._unflat(flat)

    def get_grads(self):
        import numpy as np
        flat = np.zeros(self.P, np.float32)
        check(lib().sem_mlp_get_grads(self.handle, flat.ctypes.data_as(_VP), _stream()), "sem_mlp_get_grads")
        return self._unflat(flat)

    def forward(self, X, Y=None):
        import torch
        rows = X.shape[0]
        if Y is None:
            Y = torch.empty((rows, self.O), dtype=torch.float32, device="cuda")
        check(lib().sem_mlp_forward(self.handle, _ptr(X), rows, _ptr(Y), _stream()), "sem_mlp_forward")
        return Y

    def grad(self, X, T, rows_real=None, outs_real=None):
        rows = X.shape[0]
        loss = ctypes.c_double()
        check(lib().sem_mlp_grad(self.handle, _ptr(X), _ptr(T), rows, int(rows_real or rows),
                                 int(outs_real or self.O), ctypes.byref(loss), _stream()), "sem_mlp_grad")
        return loss.value

    def grad_energy(self, X, T, mesh, lam, assembled=False, work=None):
        """sem_mlp_grad_energy: the energy-norm loss on `mesh` (assembled:
        of the averaged correction; work: >= 2 nloc FP32 device floats,
        allocated when not given)."""
        import torch
        if work is None:
            work = torch.empty(2 * mesh.nloc, dtype=torch.float32, device="cuda")
        loss = ctypes.c_double()
        check(lib().sem_mlp_grad_energy(self.handle, mesh.handle, _ptr(X), _ptr(T), X.shape[0], float(lam),
                                        int(bool(assembled)), _ptr(work), work.numel(), ctypes.byref(loss),
                                        _stream()),
              "sem_mlp_grad_energy")
        return loss.value

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8):
        check(lib().sem_mlp_adam(self.handle, float(lr), float(beta1), float(beta2), float(eps), _stream()),
              "sem_mlp_adam")


def guess_residual(mesh, b, p1, p2, p3, r, work, pair=False):
    """r = b - A p_ext (pair: the operator in FP32-pair arithmetic)."""
    fn = "sem_guess_residual_pair" if pair else "sem_guess_residual"
    check(getattr(lib(), fn)(mesh.handle, _ptr(b), _ptr(p1), _ptr(p2), _ptr(p3), _ptr(r), _ptr(work), _stream()), fn)


def guess_features(mesh, p1, p2, p3, p4, r, sd, sr, s3, X):
    check(lib().sem_guess_features(mesh.handle, _ptr(p1), _ptr(p2), _ptr(p3),
                                   _ptr(p4) if p4 is not None else None, _ptr(r), float(sd), float(sr), float(s3),
                                   _ptr(X), X.shape[1], _stream()), "sem_guess_features")


def guess_target(mesh, p, p1, p2, p3, pscale, T):
    check(lib().sem_guess_target(mesh.handle, _ptr(p), _ptr(p1), _ptr(p2), _ptr(p3), float(pscale), _ptr(T),
                                 T.shape[1], _stream()), "sem_guess_target")


def guess_apply(mesh, Y, p1, p2, p3, pscale, out):
    check(lib().sem_guess_apply(mesh.handle, _ptr(Y), Y.shape[1], _ptr(p1), _ptr(p2), _ptr(p3), float(pscale),
                                _ptr(out), _stream()), "sem_guess_apply")


def pcg_solve_batched(meshes, bs, xs=None, scratch=None, raise_on_error=True, schwarz=None, **kw):
    """sem_pcg_solve_batched over lists of Mesh and device FP64 right-hand
    sides (schwarz: a list of Schwarz objects, one per mesh ->
    sem_pcg_solve_batched_schwarz); returns (xs, list of stats dicts)."""
    import torch
    n = len(meshes)
    opts = meshes[0].pcg_opts(precision=SEM_PCG_MIXED, **kw)
    mh = (_VP * n)(*[m.handle.value for m in meshes])
    if xs is None:
        xs = [torch.empty_like(bi) for bi in bs]
    bh = (_VP * n)(*[bi.data_ptr() for bi in bs])
    xh = (_VP * n)(*[xi.data_ptr() for xi in xs])
    need = lib().sem_pcg_batched_scratch_bytes(mh, n, ctypes.byref(opts))
    if scratch is None or scratch.numel() < need + 256:
        scratch = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
    base = (scratch.data_ptr() + 255) // 256 * 256
    stats = (PcgStats * n)()
    nb = scratch.numel() - (base - scratch.data_ptr())
    if schwarz is not None:
        sh = (_VP * n)(*[w.handle.value for w in schwarz])
        st = lib().sem_pcg_solve_batched_schwarz(mh, sh, n, bh, xh, ctypes.byref(opts), stats, _VP(base), nb,
                                                 _stream())
    else:
        st = lib().sem_pcg_solve_batched(mh, n, bh, xh, ctypes.byref(opts), stats, _VP(base), nb, _stream())
    if raise_on_error and st != SEM_OK:
        raise SemError(st, "sem_pcg_solve_batched")
    return xs, [s.as_dict() for s in stats]


def perf_model(P_opt, C, C_max=None):
    """sem_perf_model: (T_min, split) of cost C over devices with best
    performances P_opt and capacities C_max (None / <= 0: unlimited).  Host."""
    import numpy as np
    P = np.ascontiguousarray(P_opt, dtype=np.float64)
    cap = None if C_max is None else np.ascontiguousarray(C_max, dtype=np.float64)
    out = np.zeros(len(P))
    t = ctypes.c_double()
    check(lib().sem_perf_model(len(P), _VP(P.ctypes.data), None if cap is None else _VP(cap.ctypes.data),
                               float(C), ctypes.byref(t), _VP(out.ctypes.data)), "sem_perf_model")
    return t.value, out


def schwarz_fdm_1d(N, h, hL, hR, flags):
    """sem_schwarz_fdm_1d: (S[(N+3), (N+3)], lambda[N+3]) of one direction of
    an extended element (host computation)."""
    import numpy as np
    ne = N + 3
    S = np.zeros(ne * ne)
    lam = np.zeros(ne)
    check(lib().sem_schwarz_fdm_1d(int(N), float(h), float(hL), float(hR), int(flags),
                                   S.ctypes.data_as(_VP), lam.ctypes.data_as(_VP)), "sem_schwarz_fdm_1d")
    return S.reshape(ne, ne), lam


def schwarz_coarse_operator(nel, periodic, faces, G):
    """sem_schwarz_coarse_operator: (sten[27][nv], cdinv[nv]) from the N = 1
    geometric factors G[E][6][8] (host computation)."""
    import numpy as np
    nel_a = np.ascontiguousarray(nel, dtype=np.int32)
    per = np.ascontiguousarray([1 if p else 0 for p in periodic], dtype=np.int32)
    nv = int(np.prod([n + (0 if p else 1) for n, p in zip(nel, periodic)]))
    Gc = np.ascontiguousarray(G, dtype=np.float64)
    sten = np.zeros((27, nv), dtype=np.float32)
    cdinv = np.zeros(nv, dtype=np.float32)
    check(lib().sem_schwarz_coarse_operator(nel_a.ctypes.data_as(_VP), per.ctypes.data_as(_VP), int(faces),
                                            Gc.ctypes.data_as(_VP), sten.ctypes.data_as(_VP),
                                            cdinv.ctypes.data_as(_VP)), "sem_schwarz_coarse_operator")
    return sten, cdinv


def schwarz_line_table(N):
    """sem_schwarz_line_table: (table[3][slots], PJ, PK)."""
    import numpy as np
    out = np.zeros(3 * 32 * 5, dtype=np.int16)
    slots, pj, pk = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    check(lib().sem_schwarz_line_table(int(N), out.ctypes.data_as(_VP), out.size, ctypes.byref(slots),
                                       ctypes.byref(pj), ctypes.byref(pk)), "sem_schwarz_line_table")
    return out[:3 * slots.value].reshape(3, slots.value), pj.value, pk.value


class Schwarz:
    """sem_schwarz_*: the hybrid Schwarz preconditioner of `mesh` with the
    N = 1 `coarse` mesh of the same vertices (both built with geom_f32)."""

    def __init__(self, mesh: Mesh, coarse: Mesh):
        import torch
        self.mesh, self.coarse = mesh, coarse
        n = lib().sem_schwarz_workspace_bytes(mesh.handle, coarse.handle)
        self.workspace = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        base = (self.workspace.data_ptr() + 255) // 256 * 256
        h = _VP()
        check(lib().sem_schwarz_create(mesh.handle, coarse.handle, _VP(base), n, _stream(), ctypes.byref(h)),
              "sem_schwarz_create")
        self.handle = h
        self.problems = lib().sem_schwarz_problems(h)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value and _lib is not None:
            _lib.sem_schwarz_destroy(h)
            self.handle = None

    def apply(self, r, coarse_iters=3, coarse_tol=1e-2, z=None):
        """z = M r (sem_schwarz_apply), FP32 E-layout tensors; coarse_iters = 0:
        the one-level (local solves only) preconditioner."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        check(lib().sem_schwarz_apply(self.handle, _ptr(r), _ptr(z), int(coarse_iters), float(coarse_tol), _stream()),
              "sem_schwarz_apply")
        return z

    def apply3(self, mid, r, mid_weight=0.15, coarse_iters=3, coarse_tol=1e-2, z=None):
        """z = M r with the intermediate level `mid` (sem_schwarz_apply3)."""
        import torch
        if z is None:
            z = torch.empty_like(r)
        n = lib().sem_schwarz_mid_work_bytes(mid.handle)
        work = torch.empty(n + 256, dtype=torch.uint8, device="cuda")
        base = (work.data_ptr() + 255) // 256 * 256
        check(lib().sem_schwarz_apply3(self.handle, mid.handle, float(mid_weight), _ptr(r), _ptr(z), int(coarse_iters),
                                       float(coarse_tol), _VP(base), n, _stream()), "sem_schwarz_apply3")
        return z
