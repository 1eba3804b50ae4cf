"""The binding refuses tensors smaller than the grid needs before anything
reaches the library (the C ABI takes bare device pointers and cannot see
sizes; a short array would be read or written out of range on the GPU).
CPU tensors stand in: the size is checked before the device."""
import pytest

import paper_2001_03477_gb300 as P


@pytest.fixture(scope="module")
def lib():
    from paper_2001_03477_gb300 import build
    build.build()
    return P.lib()


def t(n, dtype=None):
    import torch
    return torch.zeros(n, dtype=dtype or torch.float64)


def refuses(fn, *args, what, **kw):
    with pytest.raises(ValueError, match=f"^{what}: .* elements"):
        fn(*args, **kw)


def test_short_arrays_are_refused(lib):
    import torch
    g = P.Grid(6, 5, 4)
    N = g.cells
    F = [g.face_shape(a)[0] * g.face_shape(a)[1] * g.face_shape(a)[2] for a in range(3)]
    ok = lambda n: t(n)
    refuses(P.vof_step, g, t(N - 1), ok(N), ok(F[0]), ok(F[1]), ok(F[2]), 0.1, 0, what="c")
    refuses(P.vof_step, g, ok(N), ok(N), ok(F[0]), ok(F[1] - 1), ok(F[2]), 0.1, 0, what="v")
    refuses(P.vof_step, g, ok(N), ok(N), ok(F[0]), ok(F[1]), ok(F[2]), 0.1, 0, dd=t(N - 1), what="dd")
    refuses(P.vof_step, g, ok(N), ok(N), ok(F[0]), ok(F[1]), ok(F[2]), 0.1, 0, sums=t(5), what="sums")
    refuses(P.vof_reconstruct, g, ok(N), t(3 * N - 1), ok(N), t(N, torch.uint8), what="m")
    refuses(P.vof_advect_sweep_z, g, ok(N), ok(N), ok(N), ok(N), ok(F[1]), 0.1, what="face")
    refuses(P.vof_advect_sweep_x, g, ok(N), ok(N), ok(N), ok(N), ok(F[0]), 0.1, state=t(N - 1, torch.uint8),
            what="state")
    refuses(P.vof_phase_change_shift, g, ok(N), ok(N), ok(N), ok(N), None, 0.01, None, t(3), what="diag")
    refuses(P.vof_mass_transfer, g, ok(N), ok(N), 0.68, 0.025, 2.257e6, t(N - 1), what="mdot")
    refuses(P.vof_velocity_extension, g, ok(N), ok(N), 958.0, 0.6, 1e-3, ut=ok(F[0]), vt=ok(F[1]), wt=t(F[2] - 1),
            what="wt")
    refuses(P.vof_heat_diffusion, g, ok(N), t(N - 1), 0.68, 0.025, 1e-3, what="e")
    refuses(P.vof_batched_step, [P.Box(g, ok(N), ok(N), ok(F[0]), t(F[1] - 1), ok(F[2]), 0.1)], 0, what="v")


def test_right_sizes_pass_the_size_check(lib):
    g = P.Grid(6, 5, 4)
    N = g.cells
    F = [g.face_shape(a)[0] * g.face_shape(a)[1] * g.face_shape(a)[2] for a in range(3)]
    # larger arrays are fine too; what stops these calls is the device check
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        P.vof_step(g, t(N), t(N + 7), t(F[0]), t(F[1]), t(F[2]), 0.1, 0, sums=t(P.VOF_NSUMS))
