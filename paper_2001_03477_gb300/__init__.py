"""GB300 (sm_103a) library for the hot path of Malan et al.,
"A Geometric VOF Method for Interface Resolved Phase Change and Conservative
Thermal Energy Advection" (arXiv:2001.03477): PLIC reconstruction, the
direction-split geometric VOF sweeps with the thermal energy fluxed in tandem
(Sec. 3.3.1, 3.4.1; Weymouth-Yue or Li's Lagrangian-explicit scheme) and the
phase-change interface shift (Sec. 3.3.2); around it the mass transfer rate
from PLIC distances (Sec. 3.2), the velocity extension (Sec. 3.3.1), the
interface-Dirichlet heat diffusion (Sec. 3.4.2), many independent
subdomains stepped together on concurrent streams (vof_batched_step,
BoxBatch), and checkpoint / resume.

This module is a thin ctypes binding over the C ABI in include/vofgb.h
(libvofgb.so, built in-tree by `build.py`).  It only marshals arguments:
every step of the path runs in the library's CUDA kernels.  Tensors must be
contiguous CUDA tensors (float64 fields, uint8 state); calls are queued on
torch's current CUDA stream.  There is no CPU fallback: if the library is
not built, or no GPU is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass, field

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libvofgb.so")

VOF_OK, VOF_EINVAL, VOF_ECUDA, VOF_ECFL, VOF_ESOLVE, VOF_EWAIT = 0, 1, 2, 3, 4, 5
VOF_NSUMS = 6


class VofError(RuntimeError):
    def __init__(self, name, status, lib=None):
        msg = f"{name}: status {status}"
        if lib is not None:
            msg += f" ({lib.vof_status_string(status).decode()})"
            if status == VOF_ECUDA:
                msg += f", cudaError {lib.vof_last_cuda_error()}"
        super().__init__(msg)
        self.status = status


class _CGrid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("bc", ctypes.c_int * 3),
                ("h", ctypes.c_double), ("Cp_l", ctypes.c_double), ("Cp_g", ctypes.c_double),
                ("T_sat", ctypes.c_double), ("eps_mixed", ctypes.c_double), ("precision", ctypes.c_int),
                ("scheme", ctypes.c_int), ("normal", ctypes.c_int), ("mlp", ctypes.c_void_p)]


class _CBox(ctypes.Structure):
    _fields_ = [("grid", _CGrid), ("c", ctypes.c_void_p), ("e", ctypes.c_void_p), ("u", ctypes.c_void_p),
                ("v", ctypes.c_void_p), ("w", ctypes.c_void_p), ("dt", ctypes.c_double), ("dd", ctypes.c_void_p),
                ("dd_uniform", ctypes.c_double)]


@dataclass
class Grid:
    """Uniform grid and phase properties (vof_grid in include/vofgb.h)."""
    nx: int
    ny: int
    nz: int
    bc: tuple = (0, 0, 0)
    h: float = 1.0
    Cp_l: float = 1.0
    Cp_g: float = 1.0
    T_sat: float = 0.0
    eps_mixed: float = 1e-12
    precision: int = 0  # VOF_F64; VOF_F32_FLUX = 1: the precision form
    scheme: int = 0     # VOF_SCHEME_WY; VOF_SCHEME_LE = 1: Lagrangian-explicit sweeps
    normal: int = 0     # VOF_NORMAL_MYC; VOF_NORMAL_MLP = 1: learned normals (needs mlp); 2: Youngs
    mlp: object = field(default=None, repr=False, compare=False)  # packed network parameters (uint8 CUDA tensor)
    _c: _CGrid = field(default=None, repr=False, compare=False)

    def c_struct(self):
        g = _CGrid()
        g.nx, g.ny, g.nz = int(self.nx), int(self.ny), int(self.nz)
        for d in range(3):
            g.bc[d] = int(self.bc[d])
        g.h, g.Cp_l, g.Cp_g = float(self.h), float(self.Cp_l), float(self.Cp_g)
        g.T_sat, g.eps_mixed = float(self.T_sat), float(self.eps_mixed)
        g.precision = int(self.precision)
        g.scheme = int(self.scheme)
        g.normal = int(self.normal)
        if self.mlp is not None:
            if getattr(self.mlp, "numel", None) and self.mlp.numel() * self.mlp.element_size() < vof_mlp_packed_bytes():
                raise ValueError("mlp: shorter than vof_mlp_packed_bytes()")
            g.mlp = _ptr(self.mlp, None, "mlp").value
        else:
            g.mlp = None
        return g

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def cells(self):
        return self.nx * self.ny * self.nz

    def face_shape(self, axis):
        nz, ny, nx = self.shape
        return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][axis]


_lib = None


def lib():
    """Load libvofgb.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libvofgb.so is not built ({LIB_PATH}); run paper_2001_03477_gb300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        P, D, I, L_, S = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_long, ctypes.c_size_t
        G = ctypes.POINTER(_CGrid)
        sig = {
            "vof_reconstruct": [G, P, P, P, P, P],
            "vof_advect_sweep_x": [G, P, P, P, P, P, D, P, P, P, P, P, S, P],
            "vof_advect_sweep_y": [G, P, P, P, P, P, D, P, P, P, P, P, S, P],
            "vof_advect_sweep_z": [G, P, P, P, P, P, D, P, P, P, P, P, S, P],
            "energy_advect_consistent": [G, I, P, P, P, P, P, P, D, P, P, P],
            "vof_phase_change_shift": [G, P, P, P, P, P, D, P, P, P, S, P],
            "vof_step": [G, P, P, P, P, P, D, L_, P, D, P, P, S, P],
            "vof_mass_transfer": [G, P, P, D, D, D, P, P, P, D, P, P, S, P],
            "vof_velocity_extension": [G, P, P, D, D, D, D, I, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double), P, S, P],
            "vof_heat_diffusion": [G, P, P, D, D, D, D, I, I, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int),
                                   ctypes.POINTER(ctypes.c_double), P, S, P],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        B = ctypes.POINTER(_CBox)
        L.vof_batched_plan.argtypes = [B, I, I, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_size_t)]
        L.vof_batched_plan.restype = ctypes.c_int
        L.vof_batched_workspace_bytes.argtypes = [B, I, I]
        L.vof_batched_workspace_bytes.restype = ctypes.c_size_t
        L.vof_batched_step.argtypes = [B, I, L_, P, I, ctypes.POINTER(ctypes.c_void_p), P, S, P]
        L.vof_batched_step.restype = ctypes.c_int
        L.vof_group_workspace_bytes.argtypes = [B, I, I]
        L.vof_group_workspace_bytes.restype = ctypes.c_size_t
        L.vof_group_create.argtypes = [B, I, P, I, P, S, P, ctypes.POINTER(ctypes.c_void_p)]
        L.vof_group_create.restype = ctypes.c_int
        L.vof_group_step.argtypes = [P, L_, P]
        L.vof_group_step.restype = ctypes.c_int
        L.vof_group_destroy.argtypes = [P]
        L.vof_group_destroy.restype = None
        L.vof_step_noalloc.argtypes = [G, P, P, P, P, P, D, L_, P, D, P, P]
        L.vof_step_noalloc.restype = ctypes.c_int
        L.vof_noalloc_scratch_bytes.argtypes = []
        L.vof_noalloc_scratch_bytes.restype = ctypes.c_size_t
        L.vof_sweep_workspace_bytes.argtypes = [G]
        L.vof_sweep_workspace_bytes.restype = ctypes.c_size_t
        L.vof_shift_workspace_bytes.argtypes = [G]
        L.vof_shift_workspace_bytes.restype = ctypes.c_size_t
        L.vof_step_workspace_bytes.argtypes = [G]
        L.vof_step_workspace_bytes.restype = ctypes.c_size_t
        L.vof_step_work_counts.argtypes = [G, P, ctypes.POINTER(ctypes.c_int), P]
        L.vof_step_work_counts.restype = ctypes.c_int
        L.vof_checkpoint_save.argtypes = [ctypes.c_char_p, G, P, P, L_, D]
        L.vof_checkpoint_save.restype = ctypes.c_int
        L.vof_checkpoint_info.argtypes = [ctypes.c_char_p, G, ctypes.POINTER(ctypes.c_long),
                                          ctypes.POINTER(ctypes.c_double)]
        L.vof_checkpoint_info.restype = ctypes.c_int
        L.vof_checkpoint_load.argtypes = [ctypes.c_char_p, S, P, P]
        L.vof_checkpoint_load.restype = ctypes.c_int
        L.vof_heat_diffusion_workspace_bytes.argtypes = [G]
        L.vof_heat_diffusion_workspace_bytes.restype = ctypes.c_size_t
        L.vof_velocity_extension_workspace_bytes.argtypes = [G]
        L.vof_velocity_extension_workspace_bytes.restype = ctypes.c_size_t
        L.vof_mass_transfer_workspace_bytes.argtypes = [G]
        L.vof_mass_transfer_workspace_bytes.restype = ctypes.c_size_t
        L.vof_mass_transfer_work_counts.argtypes = [G, P, ctypes.POINTER(ctypes.c_int), P]
        L.vof_mass_transfer_work_counts.restype = ctypes.c_int
        L.vof_profile_begin.argtypes = [P]
        L.vof_profile_begin.restype = ctypes.c_int
        L.vof_profile_end.argtypes = [ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_char_p), ctypes.c_int]
        L.vof_profile_end.restype = ctypes.c_int
        L.vof_get_device_status.argtypes = []
        L.vof_get_device_status.restype = ctypes.c_int
        L.vof_status_string.argtypes = [ctypes.c_int]
        L.vof_status_string.restype = ctypes.c_char_p
        L.vof_last_cuda_error.argtypes = []
        L.vof_last_cuda_error.restype = ctypes.c_int
        L.vof_fp64_probe.argtypes = [ctypes.c_int, ctypes.c_long, ctypes.c_int, P, P]
        L.vof_fp64_probe.restype = ctypes.c_int
        L.vof_mlp_packed_bytes.argtypes = []
        L.vof_mlp_packed_bytes.restype = ctypes.c_size_t
        L.vof_mlp_pack.argtypes = [P, P, P]
        L.vof_mlp_pack.restype = ctypes.c_int
        L.vof_mlp_forward.argtypes = [P, P, ctypes.c_long, P, P]
        L.vof_mlp_forward.restype = ctypes.c_int
        L.vof_mlp_normals.argtypes = [P, P, ctypes.c_long, P, P, P]
        L.vof_mlp_normals.restype = ctypes.c_int
        L.vof_mlp_train_workspace_bytes.argtypes = [ctypes.c_int]
        L.vof_mlp_train_workspace_bytes.restype = ctypes.c_size_t
        L.vof_mlp_train_step.argtypes = [P, P, ctypes.c_long, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_long,
                                         ctypes.c_float, P, P, P, P, P, P, P, P, S, P]
        L.vof_mlp_train_step.restype = ctypes.c_int
        _lib = L
    return _lib


def _ptr(t, dtype=None, name="tensor"):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name}: expected a torch.Tensor")
    if not t.is_cuda:
        raise ValueError(f"{name}: must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _faces(g, axis):
    a, b, c = g.face_shape(axis)
    return a * b * c


def _sizes(*needs):
    """Refuse, before anything reaches the library, a tensor with fewer
    elements than the call reads or writes through it: needs are (tensor or
    None, elements, argument name).  The C ABI takes bare device pointers and
    cannot see array sizes, so a short array would be accessed out of range
    on the GPU."""
    for t, n, name in needs:
        if t is not None and hasattr(t, "numel") and t.numel() < n:
            raise ValueError(f"{name}: {t.numel()} elements, the call needs {n}")


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(name, status):
    if status != VOF_OK:
        raise VofError(name, status, lib())


def _f64():
    import torch
    return torch.float64


def _u8():
    import torch
    return torch.uint8


def vof_reconstruct(g: Grid, c, m, alpha, mixed, stream=None):
    N = g.cells
    _sizes((c, N, "c"), (m, 3 * N, "m"), (alpha, N, "alpha"), (mixed, N, "mixed"))
    cg = g.c_struct()
    _check("vof_reconstruct", lib().vof_reconstruct(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(m, _f64(), "m"),
                                                    _ptr(alpha, _f64(), "alpha"), _ptr(mixed, _u8(), "mixed"),
                                                    _stream(stream)))


def vof_sweep_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_sweep_workspace_bytes(ctypes.byref(cg)))


def vof_shift_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_shift_workspace_bytes(ctypes.byref(cg)))


_ws_cache = {}


def _cached_workspace(nb, device):
    import torch
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    key = (dev, nb)
    if key not in _ws_cache:
        _ws_cache[key] = torch.empty(nb, dtype=torch.uint8, device=dev)
    return _ws_cache[key]


def sweep_workspace(g: Grid, device=None):
    """A cached scratch buffer (torch allocation) for the stand-alone sweeps.
    It is the one buffer of its size on the device, shared by every sweep or
    shift call that omits `workspace`: calls that may overlap on the GPU
    (different streams) must pass workspaces of their own."""
    return _cached_workspace(vof_sweep_workspace_bytes(g), device)


def shift_workspace(g: Grid, device=None):
    """A cached scratch buffer (torch allocation) for the stand-alone shift,
    shared like sweep_workspace()."""
    return _cached_workspace(vof_shift_workspace_bytes(g), device)


def _sweep(name, g, c_in, e_in, c_out, e_out, uf, dt, state, theta, flux_out, diag, workspace, stream):
    N, Fa = g.cells, _faces(g, "xyz".index(name[-1]))
    _sizes((c_in, N, "c_in"), (e_in, N, "e_in"), (c_out, N, "c_out"), (e_out, N, "e_out"), (uf, Fa, "face"),
           (state, N, "state"), (theta, N, "theta"), (flux_out, Fa, "flux_out"), (diag, 1, "diag"))
    cg = g.c_struct()
    fn = getattr(lib(), name)
    if workspace is None:
        workspace = sweep_workspace(g, c_in.device)
    nbytes = workspace.numel() * workspace.element_size()
    _check(name, fn(ctypes.byref(cg), _ptr(c_in, _f64(), "c_in"), _ptr(e_in, _f64(), "e_in"),
                    _ptr(c_out, _f64(), "c_out"), _ptr(e_out, _f64(), "e_out"), _ptr(uf, _f64(), "face"),
                    float(dt), _ptr(state, _u8(), "state"), _ptr(theta, _f64(), "theta"),
                    _ptr(flux_out, _f64(), "flux_out"), _ptr(diag, _f64(), "diag"),
                    _ptr(workspace, None, "workspace"), ctypes.c_size_t(nbytes), _stream(stream)))


def vof_advect_sweep_x(g, c_in, e_in, c_out, e_out, u_face, dt, state=None, theta=None, flux_out=None, diag=None,
                       workspace=None, stream=None):
    _sweep("vof_advect_sweep_x", g, c_in, e_in, c_out, e_out, u_face, dt, state, theta, flux_out, diag, workspace,
           stream)


def vof_advect_sweep_y(g, c_in, e_in, c_out, e_out, v_face, dt, state=None, theta=None, flux_out=None, diag=None,
                       workspace=None, stream=None):
    _sweep("vof_advect_sweep_y", g, c_in, e_in, c_out, e_out, v_face, dt, state, theta, flux_out, diag, workspace,
           stream)


def vof_advect_sweep_z(g, c_in, e_in, c_out, e_out, w_face, dt, state=None, theta=None, flux_out=None, diag=None,
                       workspace=None, stream=None):
    _sweep("vof_advect_sweep_z", g, c_in, e_in, c_out, e_out, w_face, dt, state, theta, flux_out, diag, workspace,
           stream)


SWEEPS = (vof_advect_sweep_x, vof_advect_sweep_y, vof_advect_sweep_z)


def energy_advect_consistent(g, axis, c_before, c_after, e_in, e_out, flux_F, u_face, dt, state=None, theta=None,
                             stream=None):
    N = g.cells
    if int(axis) in (0, 1, 2):
        Fa = _faces(g, int(axis))
        _sizes((c_before, N, "c_before"), (c_after, N, "c_after"), (e_in, N, "e_in"), (e_out, N, "e_out"),
               (flux_F, Fa, "flux_F"), (u_face, Fa, "u_face"), (state, N, "state"), (theta, N, "theta"))
    cg = g.c_struct()
    _check("energy_advect_consistent",
           lib().energy_advect_consistent(ctypes.byref(cg), int(axis), _ptr(c_before, _f64(), "c_before"),
                                          _ptr(c_after, _f64(), "c_after"), _ptr(e_in, _f64(), "e_in"),
                                          _ptr(e_out, _f64(), "e_out"), _ptr(flux_F, _f64(), "flux_F"),
                                          _ptr(u_face, _f64(), "u_face"), float(dt), _ptr(state, _u8(), "state"),
                                          _ptr(theta, _f64(), "theta"), _stream(stream)))


def vof_phase_change_shift(g, c_in, e_in, c_out, e_out, dd=None, dd_uniform=0.0, state=None, diag=None,
                           workspace=None, stream=None):
    N = g.cells
    _sizes((c_in, N, "c_in"), (e_in, N, "e_in"), (c_out, N, "c_out"), (e_out, N, "e_out"), (dd, N, "dd"),
           (state, N, "state"), (diag, 5, "diag"))
    cg = g.c_struct()
    if workspace is None:
        workspace = shift_workspace(g, c_in.device)
    nbytes = workspace.numel() * workspace.element_size()
    _check("vof_phase_change_shift",
           lib().vof_phase_change_shift(ctypes.byref(cg), _ptr(c_in, _f64(), "c_in"), _ptr(e_in, _f64(), "e_in"),
                                        _ptr(c_out, _f64(), "c_out"), _ptr(e_out, _f64(), "e_out"),
                                        _ptr(dd, _f64(), "dd"), float(dd_uniform), _ptr(state, _u8(), "state"),
                                        _ptr(diag, _f64(), "diag"), _ptr(workspace, None, "workspace"),
                                        ctypes.c_size_t(nbytes), _stream(stream)))


def vof_step_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_step_workspace_bytes(ctypes.byref(cg)))


def _step_sizes(g, c, e, u, v, w, dd, sums):
    N = g.cells
    _sizes((c, N, "c"), (e, N, "e"), (u, _faces(g, 0), "u"), (v, _faces(g, 1), "v"), (w, _faces(g, 2), "w"),
           (dd, N, "dd"), (sums, VOF_NSUMS, "sums"))


def vof_step(g, c, e, u, v, w, dt, step_index, dd=None, dd_uniform=0.0, sums=None, workspace=None, stream=None):
    _step_sizes(g, c, e, u, v, w, dd, sums)
    cg = g.c_struct()
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    _check("vof_step",
           lib().vof_step(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(e, _f64(), "e"), _ptr(u, _f64(), "u"),
                          _ptr(v, _f64(), "v"), _ptr(w, _f64(), "w"), float(dt), int(step_index),
                          _ptr(dd, _f64(), "dd"), float(dd_uniform), _ptr(sums, _f64(), "sums"),
                          _ptr(workspace, None, "workspace"), ctypes.c_size_t(nbytes), _stream(stream)))


def vof_step_noalloc(g, c, e, u, v, w, dt, step_index, dd=None, dd_uniform=0.0, sums=None, stream=None):
    """vof_step without a workspace, for callers that cannot allocate device
    memory while they step: the scratch lives in the library's fixed array
    (grids up to VOF_NOALLOC_MAX_CELLS = 64^3 cells).  Calls that overlap on
    the GPU share that array and race; the first call on a device must come
    before any stream capture on it."""
    _step_sizes(g, c, e, u, v, w, dd, sums)
    cg = g.c_struct()
    _check("vof_step_noalloc",
           lib().vof_step_noalloc(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(e, _f64(), "e"),
                                  _ptr(u, _f64(), "u"), _ptr(v, _f64(), "v"), _ptr(w, _f64(), "w"), float(dt),
                                  int(step_index), _ptr(dd, _f64(), "dd"), float(dd_uniform),
                                  _ptr(sums, _f64(), "sums"), _stream(stream)))


VOF_NOALLOC_MAX_CELLS = 262144


def vof_mass_transfer_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_mass_transfer_workspace_bytes(ctypes.byref(cg)))


def vof_mass_transfer(g, c, e, k_l, k_g, h_fg, mdot, d_gamma=None, grad_n=None, dd_per_mdot=0.0, dd=None,
                      workspace=None, stream=None):
    """Mass transfer rate from PLIC interface distances (Sec. 3.2) into
    `mdot` (and the optional per-cell distances, gradients and shift)."""
    N = g.cells
    _sizes((c, N, "c"), (e, N, "e"), (mdot, N, "mdot"), (d_gamma, N, "d_gamma"), (grad_n, N, "grad_n"),
           (dd, N, "dd"))
    cg = g.c_struct()
    if workspace is None:
        workspace = _cached_workspace(vof_mass_transfer_workspace_bytes(g), c.device)
    nbytes = workspace.numel() * workspace.element_size()
    _check("vof_mass_transfer",
           lib().vof_mass_transfer(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(e, _f64(), "e"), float(k_l),
                                   float(k_g), float(h_fg), _ptr(mdot, _f64(), "mdot"),
                                   _ptr(d_gamma, _f64(), "d_gamma"), _ptr(grad_n, _f64(), "grad_n"),
                                   float(dd_per_mdot), _ptr(dd, _f64(), "dd"), _ptr(workspace, None, "workspace"),
                                   ctypes.c_size_t(nbytes), _stream(stream)))


def vof_velocity_extension_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_velocity_extension_workspace_bytes(ctypes.byref(cg)))


def vof_velocity_extension(g, c, mdot, rho_l, rho_g, dt, tol=1e-13, max_iter=2000, u=None, v=None, w=None,
                           ut=None, vt=None, wt=None, workspace=None, stream=None):
    """Velocity extension across the interface (Sec. 3.3.1): adds u~ to
    (u, v, w) and/or writes it to (ut, vt, wt).  Returns (CG iterations,
    final residual norm)."""
    F = [_faces(g, a) for a in range(3)]
    _sizes((c, g.cells, "c"), (mdot, g.cells, "mdot"), (u, F[0], "u"), (v, F[1], "v"), (w, F[2], "w"),
           (ut, F[0], "ut"), (vt, F[1], "vt"), (wt, F[2], "wt"))
    cg = g.c_struct()
    if workspace is None:
        workspace = _cached_workspace(vof_velocity_extension_workspace_bytes(g), c.device)
    nbytes = workspace.numel() * workspace.element_size()
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check("vof_velocity_extension",
           lib().vof_velocity_extension(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(mdot, _f64(), "mdot"),
                                        float(rho_l), float(rho_g), float(dt), float(tol), int(max_iter),
                                        _ptr(u, _f64(), "u"), _ptr(v, _f64(), "v"), _ptr(w, _f64(), "w"),
                                        _ptr(ut, _f64(), "ut"), _ptr(vt, _f64(), "vt"), _ptr(wt, _f64(), "wt"),
                                        ctypes.byref(it), ctypes.byref(res), _ptr(workspace, None, "workspace"),
                                        ctypes.c_size_t(nbytes), _stream(stream)))
    return it.value, res.value


def vof_heat_diffusion_workspace_bytes(g: Grid) -> int:
    cg = g.c_struct()
    return int(lib().vof_heat_diffusion_workspace_bytes(ctypes.byref(cg)))


VOF_CP_PHASE, VOF_CP_MIXTURE = 0, 1  # heat capacity of vof_heat_diffusion


def vof_heat_diffusion(g, c, e, k_l, k_g, dt, tol=1e-10, max_iter=10000, heat_capacity=VOF_CP_PHASE, wall_T=None,
                       workspace=None, stream=None):
    """Implicit interface-Dirichlet heat diffusion (Sec. 3.4.2) of e in
    place, each node with its phase's heat capacity (VOF_CP_PHASE) or the
    cell's mixture (VOF_CP_MIXTURE); wall_T: {(axis, side): T_w} fixed wall
    temperatures (side -1 low, +1 high).  Returns (Jacobi sweeps, last
    sweep's largest change of T)."""
    _sizes((c, g.cells, "c"), (e, g.cells, "e"))
    cg = g.c_struct()
    if workspace is None:
        workspace = _cached_workspace(vof_heat_diffusion_workspace_bytes(g), c.device)
    nbytes = workspace.numel() * workspace.element_size()
    it = ctypes.c_int(0)
    ch = ctypes.c_double(0.0)
    walls = None
    if wall_T:
        walls = (ctypes.c_double * 6)(*([float("nan")] * 6))
        for (axis, side), Tw in wall_T.items():
            walls[2 * int(axis) + (0 if side < 0 else 1)] = float(Tw)
    _check("vof_heat_diffusion",
           lib().vof_heat_diffusion(ctypes.byref(cg), _ptr(c, _f64(), "c"), _ptr(e, _f64(), "e"), float(k_l),
                                    float(k_g), float(dt), float(tol), int(max_iter), int(heat_capacity), walls,
                                    ctypes.byref(it),
                                    ctypes.byref(ch), _ptr(workspace, None, "workspace"), ctypes.c_size_t(nbytes),
                                    _stream(stream)))
    return it.value, ch.value


def _host_f64(a, name):
    """A C-contiguous float64 numpy array of a numpy array or a torch tensor
    (device tensors are copied to the host)."""
    import numpy as np
    if hasattr(a, "detach"):
        a = a.detach().cpu().numpy()
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def vof_checkpoint_save(path, g: Grid, c, e, step=0, t=0.0):
    """Write (g, step, t, c, e) to `path` (c, e: numpy arrays or torch
    tensors, device tensors copied to the host)."""
    cg = g.c_struct()
    ch, eh = _host_f64(c, "c"), _host_f64(e, "e")
    if ch.size != g.cells or eh.size != g.cells:
        raise ValueError("vof_checkpoint_save: c and e must hold one value per cell")
    _check("vof_checkpoint_save",
           lib().vof_checkpoint_save(str(path).encode(), ctypes.byref(cg), ch.ctypes.data, eh.ctypes.data,
                                     int(step), float(t)))


def vof_checkpoint_load(path):
    """(Grid, step, t, c, e) from a checkpoint; c, e as numpy arrays of the
    grid's (nz, ny, nx) shape."""
    import numpy as np
    cg = _CGrid()
    step = ctypes.c_long(0)
    t = ctypes.c_double(0.0)
    _check("vof_checkpoint_info", lib().vof_checkpoint_info(str(path).encode(), ctypes.byref(cg),
                                                            ctypes.byref(step), ctypes.byref(t)))
    g = Grid(cg.nx, cg.ny, cg.nz, tuple(cg.bc), cg.h, cg.Cp_l, cg.Cp_g, cg.T_sat, cg.eps_mixed,
             precision=cg.precision, scheme=cg.scheme)
    c = np.empty(g.shape)
    e = np.empty(g.shape)
    _check("vof_checkpoint_load", lib().vof_checkpoint_load(str(path).encode(), ctypes.c_size_t(g.cells),
                                                            c.ctypes.data, e.ctypes.data))
    return g, step.value, t.value, c, e


def vof_mass_transfer_work_counts(g, workspace, stream=None):
    """{mixed, band} cell counts of the last vof_mass_transfer run with
    `workspace`."""
    cg = g.c_struct()
    out = (ctypes.c_int * 2)()
    _check("vof_mass_transfer_work_counts",
           lib().vof_mass_transfer_work_counts(ctypes.byref(cg), _ptr(workspace, None, "workspace"), out,
                                               _stream(stream)))
    return {"mixed": out[0], "band": out[1]}


def vof_get_device_status() -> int:
    return int(lib().vof_get_device_status())


VOF_NCOUNTS = 12
VOF_F64, VOF_F32_FLUX = 0, 1  # vof_grid.precision
VOF_SCHEME_WY, VOF_SCHEME_LE = 0, 1  # vof_grid.scheme
VOF_NORMAL_MYC, VOF_NORMAL_MLP, VOF_NORMAL_YOUNGS = 0, 1, 2  # vof_grid.normal


def vof_step_work_counts(g, workspace, stream=None):
    """Work counts of the last vof_step run with `workspace`: dict with the
    mixed cells and faces of each sweep and the shift's cell counts."""
    cg = g.c_struct()
    out = (ctypes.c_int * VOF_NCOUNTS)()
    _check("vof_step_work_counts", lib().vof_step_work_counts(ctypes.byref(cg), _ptr(workspace, None, "workspace"),
                                                              out, _stream(stream)))
    v = list(out)
    return {"mixed": v[0:6:2], "faces": v[1:6:2], "shift_analytic": v[6], "shift_bisection": v[7],
            "receivers": v[8], "mlp_fallback": v[9:12]}


def vof_fp64_probe(op, iters, blocks, out, stream=None):
    """Launch the FP64 rate probe (op 0: fused multiply-adds, 1: adds);
    out: float64 CUDA tensor of blocks * 256 elements."""
    _sizes((out, blocks * 256, "out"))
    _check("vof_fp64_probe", lib().vof_fp64_probe(int(op), int(iters), int(blocks), _ptr(out, _f64(), "out"),
                                                  _stream(stream)))


def vof_profile_begin(stream=None):
    _check("vof_profile_begin", lib().vof_profile_begin(_stream(stream)))


def vof_profile_end(max_entries=4096):
    """[(launch name, ms)] of the library launches since vof_profile_begin."""
    ms = (ctypes.c_float * max_entries)()
    names = (ctypes.c_char_p * max_entries)()
    n = int(lib().vof_profile_end(ms, names, max_entries))
    if n < 0:
        raise VofError("vof_profile_end", VOF_ECUDA, lib())
    return [(names[i].decode(), float(ms[i])) for i in range(min(n, max_entries))]


# ---------------------------------------------------------------------------
# learned interface normal (vof_mlp_*)
# ---------------------------------------------------------------------------
VOF_MLP_PARAMS = 6147
MLP_SIZES = (27, 64, 64, 3)


def vof_mlp_packed_bytes() -> int:
    return int(lib().vof_mlp_packed_bytes())


def vof_mlp_pack(master, packed, stream=None):
    """BF16 weight images of the FP32 master parameters (VOF_MLP_PARAMS
    floats: W1[64][27], b1, W2[64][64], b2, W3[3][64], b3)."""
    import torch
    _sizes((master, VOF_MLP_PARAMS, "master"), (packed, vof_mlp_packed_bytes(), "packed"))
    _check("vof_mlp_pack", lib().vof_mlp_pack(_ptr(master, torch.float32, "master"), _ptr(packed, None, "packed"),
                                              _stream(stream)))


def vof_mlp_forward(packed, X, y, stream=None):
    """Network output y[n][3] (float32) of the stencils X[n][27] (float64)."""
    import torch
    n = X.numel() // 27
    _sizes((packed, vof_mlp_packed_bytes(), "packed"), (y, 3 * n, "y"))
    _check("vof_mlp_forward", lib().vof_mlp_forward(_ptr(packed, None, "packed"), _ptr(X, _f64(), "X"), n,
                                                    _ptr(y, torch.float32, "y"), _stream(stream)))


def vof_mlp_normals(packed, X, m, fallback=None, stream=None):
    """Learned normals with the MYC fallback: m[n][3] (float64) and
    fallback[n] (uint8, optional) of the stencils X[n][27]."""
    n = X.numel() // 27
    _sizes((packed, vof_mlp_packed_bytes(), "packed"), (m, 3 * n, "m"), (fallback, n, "fallback"))
    _check("vof_mlp_normals", lib().vof_mlp_normals(_ptr(packed, None, "packed"), _ptr(X, _f64(), "X"), n,
                                                    _ptr(m, _f64(), "m"), _ptr(fallback, _u8(), "fallback"),
                                                    _stream(stream)))


class MLP:
    """The learned normal's parameters on the GPU: FP32 master vector, Adam
    moments, the packed BF16 images and the training workspace (device
    memory through torch; every computation runs in the library)."""

    def __init__(self, master, device=None):
        import torch
        dev = device or torch.device("cuda")
        self.master = torch.as_tensor(master, dtype=torch.float32).to(dev).contiguous()
        assert self.master.numel() == VOF_MLP_PARAMS
        self.m = torch.zeros_like(self.master)
        self.v = torch.zeros_like(self.master)
        nb = (vof_mlp_packed_bytes() + 255) // 256 * 256
        self.packed = torch.zeros(nb, dtype=torch.uint8, device=dev)
        self.step_count = 0
        self._ws = {}
        vof_mlp_pack(self.master, self.packed)

    @staticmethod
    def init_master(seed=0):
        """He-normal weights, zero biases (numpy float32 vector)."""
        import numpy as np
        rng = np.random.default_rng(seed)
        parts = []
        for a, b in zip(MLP_SIZES[:-1], MLP_SIZES[1:]):
            parts.append(rng.normal(0.0, (2.0 / a) ** 0.5, size=(b, a)).reshape(-1))
            parts.append(np.zeros(b))
        return np.concatenate(parts).astype(np.float32)

    def workspace(self, batch):
        import torch
        if batch not in self._ws:
            nb = int(lib().vof_mlp_train_workspace_bytes(int(batch)))
            if nb == 0:
                raise ValueError(f"batch {batch}: a multiple of 128 in 128..65536")
            self._ws[batch] = torch.empty(nb + 256, dtype=torch.uint8, device=self.master.device)
        w = self._ws[batch]
        off = (-w.data_ptr()) % 256
        return w[off:], w.numel() - off

    def train_step(self, X, N, batch, lr, seed=0, grad=None, loss=None, idx=None, stream=None):
        """One Adam step (lr > 0) or only the gradient and loss (lr == 0)."""
        import torch
        ntrain = X.numel() // 27
        _sizes((N, 3 * ntrain, "N"), (grad, VOF_MLP_PARAMS, "grad"), (loss, 1, "loss"), (idx, batch, "idx"))
        ws, nb = self.workspace(batch)
        if lr > 0:
            self.step_count += 1
        _check("vof_mlp_train_step",
               lib().vof_mlp_train_step(_ptr(X, _f64(), "X"), _ptr(N, _f64(), "N"), ntrain, int(batch),
                                        int(seed) & 0xFFFFFFFFFFFFFFFF, max(self.step_count, 1), float(lr),
                                        _ptr(self.master, torch.float32, "master"),
                                        _ptr(self.m, torch.float32, "adam_m"), _ptr(self.v, torch.float32, "adam_v"),
                                        _ptr(self.packed, None, "packed"), _ptr(grad, torch.float32, "grad"),
                                        _ptr(loss, torch.float32, "loss"), _ptr(idx, torch.int64, "idx"),
                                        _ptr(ws, None, "workspace"), nb, _stream(stream)))


class Stepper:
    """Owns the workspace of vof_step for one grid (allocated through torch)."""

    def __init__(self, g: Grid, device="cuda"):
        import torch
        self.g = g
        nb = vof_step_workspace_bytes(g)
        # torch's caching allocator returns 512-byte aligned blocks
        self.workspace = torch.empty(nb, dtype=torch.uint8, device=device)
        self.sums = torch.zeros(VOF_NSUMS, dtype=torch.float64, device=device)

    def step(self, c, e, u, v, w, dt, step_index, dd=None, dd_uniform=0.0, stream=None, log=None, t=None):
        """One vof_step; with `log` (a writable text file) also appends the
        step's JSON-lines record (reads the sums and work counts back, which
        waits for the step)."""
        vof_step(self.g, c, e, u, v, w, dt, step_index, dd, dd_uniform, self.sums, self.workspace, stream)
        if log is not None:
            counts = vof_step_work_counts(self.g, self.workspace, stream)
            sums = [float(x) for x in self.sums.cpu()]
            log.write(step_record(step_index, t, sums, counts) + "\n")
        return self.sums


@dataclass
class Box:
    """One subdomain of a batch (vof_box): its grid, fields c, e (float64,
    updated in place), face velocities u, v, w, time step and shift."""
    grid: Grid
    c: object
    e: object
    u: object
    v: object
    w: object
    dt: float
    dd: object = None
    dd_uniform: float = 0.0


def _box_array(boxes, with_arrays=True):
    arr = (_CBox * max(len(boxes), 1))()
    for i, b in enumerate(boxes):
        g = b.grid if isinstance(b, Box) else b
        arr[i].grid = g.c_struct()
        if with_arrays:
            _step_sizes(g, b.c, b.e, b.u, b.v, b.w, b.dd, None)
            arr[i].c = _ptr(b.c, _f64(), "c")
            arr[i].e = _ptr(b.e, _f64(), "e")
            arr[i].u = _ptr(b.u, _f64(), "u")
            arr[i].v = _ptr(b.v, _f64(), "v")
            arr[i].w = _ptr(b.w, _f64(), "w")
            arr[i].dt = float(b.dt)
            arr[i].dd = _ptr(b.dd, _f64(), "dd")
            arr[i].dd_uniform = float(b.dd_uniform)
    return arr


def vof_batched_plan(grids, lanes):
    """Host-only plan of a batch (nothing launched): (lane of each box,
    workspace offset of each lane, total workspace bytes).  `grids`: Grid or
    Box objects."""
    arr = _box_array(grids, with_arrays=False)
    lane = (ctypes.c_int * max(len(grids), 1))()
    off = (ctypes.c_size_t * max(int(lanes), 1))()
    total = ctypes.c_size_t(0)
    _check("vof_batched_plan", lib().vof_batched_plan(arr, len(grids), int(lanes), lane, off, ctypes.byref(total)))
    return list(lane)[:len(grids)], list(off)[:int(lanes)], int(total.value)


def vof_batched_workspace_bytes(grids, lanes) -> int:
    arr = _box_array(grids, with_arrays=False)
    return int(lib().vof_batched_workspace_bytes(arr, len(grids), int(lanes)))


def vof_batched_step(boxes, step_index, sums=None, lanes=1, lane_streams=None, workspace=None, stream=None,
                     _arr=None):
    """One vof_step of every box, the boxes spread over `lanes` streams
    (`lane_streams`: torch.cuda.Stream objects; None with lanes == 1 runs them
    on `stream`).  sums: float64 [len(boxes), VOF_NSUMS] or None."""
    arr = _arr if _arr is not None else _box_array(boxes)
    _sizes((sums, len(boxes) * VOF_NSUMS, "sums"))
    nbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    ls = None
    if lane_streams is not None:
        if len(lane_streams) != int(lanes):
            raise ValueError(f"vof_batched_step: {len(lane_streams)} lane streams for {lanes} lanes")
        ls = (ctypes.c_void_p * len(lane_streams))(*[s.cuda_stream for s in lane_streams])
    _check("vof_batched_step",
           lib().vof_batched_step(arr, len(boxes), int(step_index), _ptr(sums, _f64(), "sums"), int(lanes), ls,
                                  _ptr(workspace, None, "workspace"), ctypes.c_size_t(nbytes), _stream(stream)))


class Group:
    """A batch of boxes stepped with one launch per kernel of the time step
    (vof_group_*): the boxes' workspaces and the launch tables live in one
    device buffer (allocated through torch); `step()` runs vof_group_step.
    `work_per_cta`: cells per CTA of the grid-stride kernels."""

    def __init__(self, boxes, work_per_cta=4096, device="cuda", stream=None):
        import torch
        self.boxes = list(boxes)
        self._arr = _box_array(self.boxes)
        n = len(self.boxes)
        self.sums = torch.zeros((max(n, 1), VOF_NSUMS), dtype=torch.float64, device=device)
        nb = int(lib().vof_group_workspace_bytes(self._arr, n, int(work_per_cta)))
        if nb == 0:
            raise VofError("vof_group_workspace_bytes", VOF_EINVAL, lib())
        self.workspace = torch.empty(nb + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws = self.workspace[off:]
        h = ctypes.c_void_p(0)
        _check("vof_group_create",
               lib().vof_group_create(self._arr, n, _ptr(self.sums, _f64(), "sums"), int(work_per_cta),
                                      ctypes.c_void_p(self._ws.data_ptr()), ctypes.c_size_t(nb), _stream(stream),
                                      ctypes.byref(h)))
        self._h = h
        self.work_per_cta = int(work_per_cta)

    def step(self, step_index, stream=None):
        _check("vof_group_step", lib().vof_group_step(self._h, int(step_index), _stream(stream)))
        return self.sums

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            lib().vof_group_destroy(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 -- interpreter shutdown
            pass

    @staticmethod
    def autotune(boxes, candidates=(1024, 4096, 16384, 65536), steps=2, device="cuda"):
        """The work_per_cta with the fastest grouped step on a copy of the
        boxes (fields cloned, velocities shared), by CUDA events."""
        import torch
        copy = [Box(b.grid, b.c.clone(), b.e.clone(), b.u, b.v, b.w, b.dt, b.dd, b.dd_uniform) for b in boxes]
        timings = {}

        def measure(w):
            g = Group(copy, w, device)
            g.step(0)
            s = torch.cuda.current_stream()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0.record(s)
            for k in range(steps):
                g.step(1 + k)
            t1.record(s)
            torch.cuda.synchronize()
            g.close()
            timings[w] = t0.elapsed_time(t1) / 1e3 / steps
            return timings[w]

        best = pick_fastest(measure, candidates)
        return best, timings


def pick_fastest(measure, candidates):
    """The autotuner's choice: the candidate with the smallest measure(c)
    (seconds per step); ties go to the earlier candidate."""
    best, best_t = None, None
    for cand in candidates:
        t = float(measure(cand))
        if best_t is None or t < best_t:
            best, best_t = cand, t
    return best


class BoxBatch:
    """A batch of boxes with its lane streams and workspace (allocated
    through torch).  `autotune()` picks the number of lanes by timing steps
    of a copy of (a sample of) the boxes; `step()` runs vof_batched_step."""

    def __init__(self, boxes, lanes=8, device="cuda"):
        import torch
        self.boxes = list(boxes)
        self.device = device
        self._arr = _box_array(self.boxes)
        self.sums = torch.zeros((max(len(self.boxes), 1), VOF_NSUMS), dtype=torch.float64, device=device)
        self.set_lanes(lanes)

    def set_lanes(self, lanes):
        import torch
        self.lanes = int(lanes)
        self.lane_streams = [torch.cuda.Stream(device=self.device) for _ in range(self.lanes)]
        nb = vof_batched_workspace_bytes(self.boxes, self.lanes)
        if nb == 0 and self.boxes:
            raise VofError("vof_batched_workspace_bytes", VOF_EINVAL, lib())
        self.workspace = torch.empty(max(nb, 256), dtype=torch.uint8, device=self.device)

    def step(self, step_index, stream=None):
        vof_batched_step(self.boxes, step_index, self.sums if self.boxes else None, self.lanes, self.lane_streams,
                         self.workspace, stream, _arr=self._arr)
        return self.sums

    def autotune(self, candidates=(1, 2, 4, 8, 16, 32), sample=None, steps=3, warmup=1):
        """Time `steps` batched steps of a copy of the first `sample` boxes
        (all by default; fields cloned, velocities shared) for each lane
        count with CUDA events; keep the fastest."""
        import torch
        src = self.boxes if sample is None else self.boxes[:int(sample)]
        copy = [Box(b.grid, b.c.clone(), b.e.clone(), b.u, b.v, b.w, b.dt, b.dd, b.dd_uniform) for b in src]

        def measure(lanes):
            trial = BoxBatch(copy, lanes, self.device)
            for k in range(warmup):
                trial.step(k)
            s = torch.cuda.current_stream()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            t0.record(s)
            for k in range(steps):
                trial.step(warmup + k)
            t1.record(s)
            torch.cuda.synchronize()
            return t0.elapsed_time(t1) / 1e3 / steps

        self.timings = {}

        def timed(lanes):
            self.timings[lanes] = measure(lanes)
            return self.timings[lanes]

        self.set_lanes(pick_fastest(timed, candidates))
        return self.lanes


def step_record(step_index, t, sums, counts):
    """One JSON line per step: the six sums of vof_step and its work counts
    (the run's volume and energy history; the paper reports volume against
    time)."""
    import json
    names = ("sum_c", "sum_e", "clipped", "shift_dc", "shift_unplaced", "shift_de")
    rec = {"step": int(step_index)}
    if t is not None:
        rec["t"] = float(t)
    rec.update({k: float(v) for k, v in zip(names, sums)})
    rec.update(counts)
    return json.dumps(rec, sort_keys=False)
