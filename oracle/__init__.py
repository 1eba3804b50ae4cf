"""FP64 CPU oracle for the PLIC / split-VOF / consistent-energy hot path.

TEST INFRASTRUCTURE ONLY.  The oracle is the slow, plain reference that the
CUDA library is checked against (Sec. 3.2-3.4 of Malan et al.,
arXiv:2001.03477).  Only the test suite, the package smoke check and the
benchmark's CPU-baseline leg may import this module.  It shares no code with
the CUDA path: the C source `vof_oracle.c` is compiled here with gcc
(-O2 -ffp-contract=off) and loaded through ctypes.

Parity status per function (pins live in tests/test_oracle_*.py):
  orc_volume, orc_alpha, orc_slab_volume, orc_plane_area  -- pinned
  orc_youngs, orc_cc_candidate, orc_myc                     -- pinned (planes)
  orc_weno5                                                 -- pinned
  orc_sweep_le, orc_step_scheme                             -- pinned (equal
      to the Weymouth-Yue sweep for uniform velocity; a plane moved exactly
      by a linear velocity; uniform T stays uniform; the volume identity)
  mlp (numpy): learned-normal data, network, gradients,
      BF16 rounding, MYC fallback                           -- pinned (finite
      differences, GELU identities, a library BF16 conversion, ellipsoid
      nearest points, label orientation, plane residual, training)
  diffusion.diffuse, diffusion_operator (numpy + scipy)     -- pinned (linear
      profiles about a plane are steady, T_Gamma is a fixed point, the
      slab decay converges, heights and plane distances agree for planes)
  extension.velocity_extension (numpy + scipy)              -- pinned (plane
      interface closed form, divergence cancels the source, mirror
      symmetry, zero flux, rejection without a free-flow face)
  orc_mass_transfer                                         -- pinned (plane
      distances exact, Sec. 4.1; linear and curved temperature fields with
      closed-form gradients and weights; droplet distance convergence)
  orc_sweep, orc_energy_consistent, orc_phase_shift, orc_step -- pinned by
      invariants (conservation, uniform-T preservation, translation return,
      plane translation, exact motion of a shifted plane, kinematic Stefan
      front, evaporating-droplet volume)
The pins themselves are checked by tests/test_oracle_mutants.py: a plausible
slip planted in a copy of any of these sources must fail at least one pin.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "vof_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_vof.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp",
           "-std=c99", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_volume.restype = ctypes.c_double
            L.orc_volume.argtypes = [_D, ctypes.c_double]
            L.orc_alpha.restype = ctypes.c_double
            L.orc_alpha.argtypes = [_D, ctypes.c_double]
            L.orc_slab_volume.restype = ctypes.c_double
            L.orc_slab_volume.argtypes = [_D, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double]
            L.orc_plane_area.restype = ctypes.c_double
            L.orc_plane_area.argtypes = [_D, ctypes.c_double]
            L.orc_weno5.restype = ctypes.c_double
            L.orc_weno5.argtypes = [_D, ctypes.c_double]
            for name in ("orc_youngs", "orc_myc"):
                getattr(L, name).restype = None
                getattr(L, name).argtypes = [_D, _D]
            L.orc_cc_candidate.restype = None
            L.orc_cc_candidate.argtypes = [_D, ctypes.c_int, _D]
            L.orc_myc_rule.restype = None
            L.orc_myc_rule.argtypes = [_D, _D, ctypes.c_int]
            L.orc_reconstruct.restype = None
            L.orc_reconstruct.argtypes = [_I, _I, _D, _D, _D, _D, _U8]
            L.orc_frozen.restype = None
            L.orc_frozen.argtypes = [_I, _D, _D, _D, _U8, _D]
            L.orc_sweep.restype = None
            L.orc_sweep.argtypes = [_I, _I, _D, ctypes.c_int, _D, _D, _D, ctypes.c_double, _U8, _D, _D, _D, _D]
            L.orc_energy_consistent.restype = None
            L.orc_energy_consistent.argtypes = [_I, _I, _D, ctypes.c_int, _D, _D, _D, _D, ctypes.c_double, _D]
            L.orc_phase_shift.restype = None
            L.orc_phase_shift.argtypes = [_I, _I, _D, _D, _D, _D, ctypes.c_double, _D]
            L.orc_sweep_le.restype = None
            L.orc_sweep_le.argtypes = [_I, _I, _D, ctypes.c_int, _D, _D, _D, ctypes.c_double, _D, _D, _D]
            L.orc_step_scheme.restype = None
            L.orc_step_scheme.argtypes = [_I, _I, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long, _D,
                                          ctypes.c_double, _D, ctypes.c_int]
            L.orc_mass_transfer.restype = None
            L.orc_mass_transfer.argtypes = [_I, _I, _D, _D, _D, _D, _D, _D, _D]
            L.orc_set_threads.restype = None
            L.orc_set_threads.argtypes = [ctypes.c_int]
            L.orc_get_threads.restype = ctypes.c_int
            L.orc_get_threads.argtypes = []
            L.orc_sum.restype = ctypes.c_double
            L.orc_sum.argtypes = [_D, ctypes.c_long]
            L.orc_step.restype = None
            L.orc_step.argtypes = [_I, _I, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long, _D,
                                   ctypes.c_double, _D]
            L.orc_run.restype = None
            L.orc_run.argtypes = [_I, _I, _D, _D, _D, _D, _D, _D, ctypes.c_double, ctypes.c_long, ctypes.c_long,
                                  _D, ctypes.c_double, _D]
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# numpy-facing helpers
# ---------------------------------------------------------------------------

def set_threads(n: int) -> None:
    """Host threads of the oracle's per-cell loops (results do not depend
    on the count: every sum is taken in cell order from per-cell values)."""
    lib().orc_set_threads(int(n))


def threads() -> int:
    return int(lib().orc_get_threads())


def _dp(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Grid:
    """Grid description for the oracle: dims (nx,ny,nz), per-axis bc
    (0 periodic, 1 zero-gradient), h, Cp_l, Cp_g, T_sat, eps."""

    def __init__(self, nx, ny, nz, bc=(0, 0, 0), h=1.0, Cp_l=1.0, Cp_g=1.0, T_sat=0.0, eps=1e-12):
        self.dims = np.array([nx, ny, nz], dtype=np.int32)
        self.bc = np.array(bc, dtype=np.int32)
        self.par = np.array([h, Cp_l, Cp_g, T_sat, eps], dtype=np.float64)

    @property
    def shape(self):
        return (int(self.dims[2]), int(self.dims[1]), int(self.dims[0]))

    def face_shape(self, axis):
        nz, ny, nx = self.shape
        return [(nz, ny, nx + 1), (nz, ny + 1, nx), (nz + 1, ny, nx)][axis]

    def _args(self):
        return (self.dims.ctypes.data_as(_I), self.bc.ctypes.data_as(_I), self.par.ctypes.data_as(_D))


def volume(m, alpha):
    m = _c64(m)
    return lib().orc_volume(_dp(m), float(alpha))


def alpha(m, c):
    m = _c64(m)
    return lib().orc_alpha(_dp(m), float(c))


def slab_volume(m, alpha_, axis, x0, delta):
    m = _c64(m)
    return lib().orc_slab_volume(_dp(m), float(alpha_), int(axis), float(x0), float(delta))


def plane_area(m, alpha_):
    m = _c64(m)
    return lib().orc_plane_area(_dp(m), float(alpha_))


def weno5(v, epsw=1e-6):
    v = _c64(v)
    return lib().orc_weno5(_dp(v), float(epsw))


def youngs(stencil):
    s = _c64(stencil).reshape(27)
    m = np.zeros(3)
    lib().orc_youngs(_dp(s), _dp(m))
    return m


def cc_candidate(stencil, d):
    s = _c64(stencil).reshape(27)
    m = np.zeros(3)
    lib().orc_cc_candidate(_dp(s), int(d), _dp(m))
    return m


def myc(stencil, rule=0):
    s = _c64(stencil).reshape(27)
    m = np.zeros(3)
    lib().orc_myc_rule(_dp(s), _dp(m), int(rule))
    return m


def reconstruct(g: Grid, c):
    c = _c64(c)
    N = c.size
    m = np.zeros((3,) + c.shape)
    al = np.zeros(c.shape)
    mixed = np.zeros(c.shape, dtype=np.uint8)
    lib().orc_reconstruct(*g._args(), _dp(c), _dp(m), _dp(al), mixed.ctypes.data_as(_U8))
    return m, al, mixed


def frozen(g: Grid, c, e):
    c = _c64(c); e = _c64(e)
    cc = np.zeros(c.shape, dtype=np.uint8)
    th = np.zeros(c.shape)
    lib().orc_frozen(g.dims.ctypes.data_as(_I), g.par.ctypes.data_as(_D), _dp(c), _dp(e),
                     cc.ctypes.data_as(_U8), _dp(th))
    return cc, th


def sweep(g: Grid, axis, c, e, uf, dt, cc, theta, want_flux=False):
    """Returns (c_new, e_new, clipped[, F, G])."""
    c = _c64(c).copy(); e = _c64(e).copy(); uf = _c64(uf)
    cc = np.ascontiguousarray(cc, dtype=np.uint8); theta = _c64(theta)
    F = np.zeros(g.face_shape(axis)) if want_flux else None
    G = np.zeros(g.face_shape(axis)) if want_flux else None
    diag = np.zeros(1)
    lib().orc_sweep(*g._args(), int(axis), _dp(c), _dp(e), _dp(uf), float(dt), cc.ctypes.data_as(_U8),
                    _dp(theta), _dp(F), _dp(G), _dp(diag))
    if want_flux:
        return c, e, float(diag[0]), F, G
    return c, e, float(diag[0])


def sweep_le(g: Grid, axis, c, e, uf, dt, want_flux=False):
    """Li's Lagrangian-explicit sweep (the paper's alternative Step 1).
    Returns (c_new, e_new, clipped[, F, G])."""
    c = _c64(c).copy(); e = _c64(e).copy(); uf = _c64(uf)
    F = np.zeros(g.face_shape(axis)) if want_flux else None
    G = np.zeros(g.face_shape(axis)) if want_flux else None
    diag = np.zeros(1)
    lib().orc_sweep_le(*g._args(), int(axis), _dp(c), _dp(e), _dp(uf), float(dt), _dp(F), _dp(G), _dp(diag))
    if want_flux:
        return c, e, float(diag[0]), F, G
    return c, e, float(diag[0])


def energy_consistent(g: Grid, axis, c_before, e, F, uf, dt, theta):
    c_before = _c64(c_before); e = _c64(e).copy(); F = _c64(F); uf = _c64(uf); theta = _c64(theta)
    lib().orc_energy_consistent(*g._args(), int(axis), _dp(c_before), _dp(e), _dp(F), _dp(uf), float(dt),
                                _dp(theta))
    return e


def phase_shift(g: Grid, c, e, dd=None, dd_uniform=0.0):
    """Returns (c_new, e_new, [sum dc, unplaced, sum de])."""
    c = _c64(c).copy(); e = _c64(e).copy()
    ddp = _c64(dd) if dd is not None else None
    diag = np.zeros(3)
    lib().orc_phase_shift(*g._args(), _dp(c), _dp(e), _dp(ddp), float(dd_uniform), _dp(diag))
    return c, e, diag


def mass_transfer(g: Grid, c, e, k_l, k_g, h_fg):
    """Mass transfer rate from PLIC interface distances (Sec. 3.2).
    Returns (mdot, d_gamma, grad_n): mdot at mixed cells (0 elsewhere);
    |d_Gamma| h of every pure cell with a mixed neighbour (-1 elsewhere);
    that cell's normal temperature gradient (0 elsewhere)."""
    c = _c64(c); e = _c64(e)
    mdot = np.zeros(c.shape); dg = np.zeros(c.shape); gn = np.zeros(c.shape)
    mpar = np.array([k_l, k_g, h_fg], dtype=np.float64)
    lib().orc_mass_transfer(*g._args(), _dp(c), _dp(e), _dp(mpar), _dp(mdot), _dp(dg), _dp(gn))
    return mdot, dg, gn


def total(x):
    x = _c64(x)
    return lib().orc_sum(_dp(x), x.size)


def step(g: Grid, c, e, u, v, w, dt, step_index, dd=None, dd_uniform=0.0, scheme=0):
    """One time step in place on copies; returns (c, e, sums[6]).
    scheme 0: Weymouth-Yue sweeps; 1: Lagrangian-explicit sweeps."""
    c = _c64(c).copy(); e = _c64(e).copy()
    u = _c64(u); v = _c64(v); w = _c64(w)
    ddp = _c64(dd) if dd is not None else None
    sums = np.zeros(6)
    lib().orc_step_scheme(*g._args(), _dp(c), _dp(e), _dp(u), _dp(v), _dp(w), float(dt), int(step_index),
                          _dp(ddp), float(dd_uniform), _dp(sums), int(scheme))
    return c, e, sums


def run(g: Grid, c, e, u, v, w, dt, step0, nsteps, dd=None, dd_uniform=0.0):
    c = _c64(c).copy(); e = _c64(e).copy()
    u = _c64(u); v = _c64(v); w = _c64(w)
    ddp = _c64(dd) if dd is not None else None
    sums = np.zeros(6)
    lib().orc_run(*g._args(), _dp(c), _dp(e), _dp(u), _dp(v), _dp(w), float(dt), int(step0), int(nsteps),
                  _dp(ddp), float(dd_uniform), _dp(sums))
    return c, e, sums
