"""The learned-normal form of the time step (vof_grid.normal =
VOF_NORMAL_MLP): the mixed cells of every sweep take the learned normal
(tensor-core network, vof_mlp.cu) with MYC as the fallback, then their plane
constants; everything else is the step of the chosen precision.

  * a network whose output is zero has no usable normal anywhere: every
    mixed cell falls back to MYC, and the step equals the MYC step of the
    same precision bit for bit (the learned path changes nothing but the
    normal's source), with the fallbacks counted in the work counts;
  * with a trained network the fluxes still telescope: volume changes only
    by the clipped volume and the shift, energy only by the shift's
    Delta e, a uniform temperature stays uniform (Sec. 3.4.1), and the
    sphere moves like the MYC step's to within a small shape difference.
"""
import numpy as np
import pytest

from paper_2001_03477_gb300 import workloads as W
from test_parity_gpu import CASES, case, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


@pytest.fixture(scope="module")
def trained(P):
    import torch
    X, Y = W.training_stencils(30_000, seed=6)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    mlp = P.MLP(P.MLP.init_master(5))
    for s in range(3000):
        mlp.train_step(Xd, Yd, 512, 3e-3 if s < 2000 else 1e-3, seed=78)
    torch.cuda.synchronize()
    return mlp


def with_normal(P, g, mlp, precision):
    import dataclasses
    return dataclasses.replace(g, precision=precision, normal=P.VOF_NORMAL_MLP, mlp=mlp.packed)


def run_steps(P, g, c, e, vel, dt, dd, nsteps):
    import torch
    st = P.Stepper(g, device=torch.device("cuda"))
    cd, ed = dev(c), dev(e)
    u, v, w = (dev(a) for a in vel)
    sums = []
    for s in range(nsteps):
        sums.append(st.step(cd, ed, u, v, w, dt, s, dd_uniform=dd).cpu().numpy())
    torch.cuda.synchronize()
    return host(cd), host(ed), np.array(sums), P.vof_step_work_counts(g, st.workspace)


@pytest.mark.parametrize("name", CASES)
@pytest.mark.parametrize("precision", [0, 1])
def test_zero_network_equals_myc_step(P, name, precision):
    import dataclasses
    g, c, e, vel, dt, dd = case(name)
    zero = P.MLP(np.zeros(P.VOF_MLP_PARAMS, dtype=np.float32))
    gm = dataclasses.replace(g, precision=precision)
    gl = with_normal(P, g, zero, precision)
    c1, e1, s1, _ = run_steps(P, gm, c, e, vel, dt, dd, 2)
    c2, e2, s2, counts = run_steps(P, gl, c, e, vel, dt, dd, 2)
    assert np.array_equal(c1, c2) and np.array_equal(e1, e2)
    assert np.array_equal(s1, s2)
    # the last step's fallbacks: every mixed cell of every sweep
    assert counts["mlp_fallback"] == counts["mixed"]


@pytest.mark.parametrize("name", ["sphere32", "deform_ragged", "tiles_periodic", "inflow_walls"])
def test_trained_network_conserves(P, trained, name):
    g, c, e, vel, dt, dd = case(name)
    gl = with_normal(P, g, trained, 1)
    nsteps = 4
    c1, e1, sums, counts = run_steps(P, gl, c, e, vel, dt, dd, nsteps)
    assert np.isfinite(c1).all() and np.isfinite(e1).all()
    assert c1.min() >= 0.0 and c1.max() <= 1.0
    assert sum(counts["mlp_fallback"]) < sum(counts["mixed"])  # the network is used
    # Sigma c, Sigma e after each step against the step's own diagnostics:
    # c changes by -clipped + shift dc (plus boundary inflow for open cases)
    if name in ("sphere32", "tiles_periodic"):
        prev_c, prev_e = c.sum(), e.sum()
        for s in range(nsteps):
            assert abs(sums[s][0] - (prev_c - sums[s][2] + sums[s][3])) <= 1e-13 * abs(prev_c)
            assert abs(sums[s][1] - (prev_e + sums[s][5])) <= 1e-13 * abs(prev_e)
            prev_c, prev_e = sums[s][0], sums[s][1]


def test_trained_network_uniform_temperature(P, trained):
    # T = T_sat everywhere: every Delta e of the shift is Delta c (C_pl -
    # C_pg) T_sat, so T stays exactly uniform whatever the normals
    g, c, e, vel, dt, dd = case("deform_ragged")
    T0 = g.T_sat if g.T_sat != 0 else 1.0
    import dataclasses
    g = dataclasses.replace(g, T_sat=T0)
    e = (g.Cp_l * c + g.Cp_g * (1 - c)) * T0
    gl = with_normal(P, g, trained, 1)
    c1, e1, _, _ = run_steps(P, gl, c, e, vel, dt, dd, 3)
    T = e1 / (g.Cp_l * c1 + g.Cp_g * (1 - c1))
    assert np.abs(T - T0).max() <= 1e-13 * T0
