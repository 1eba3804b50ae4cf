"""The grouped batch (vof_group_*: one launch per kernel of the time step
over every box) on the GPU against one vof_step per box on a single stream,
through the C ABI.  Every box computes what vof_step computes on it (the
same kernels, sum rows and reductions), so c, e and the sums must agree bit
for bit: over several steps (both sweep orders), for any CTA granularity,
in the precision form and with Youngs' normal, and as a CUDA-graph replay.
"""
import numpy as np
import pytest

from paper_2001_03477_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NBOX = 30


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
def droplets():
    return [W.droplet_subdomain(i, n_lo=10, n_hi=40, nsub=4) for i in range(NBOX)]


def make_boxes(P, wls, precision=0, normal=0):
    import torch
    boxes = []
    for i, wl in enumerate(wls):
        g = P.Grid(wl.shape[2], wl.shape[1], wl.shape[0], wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat,
                   precision=precision, normal=normal)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        # a smooth T so that every box has work in its energy fluxes
        n = wl.shape[0]
        x = (np.arange(n) + 0.5) / n
        T = 1.0 + 0.1 * np.sin(2 * np.pi * x)[None, None, :] * np.cos(2 * np.pi * x)[None, :, None]
        e = (wl.Cp_l * wl.c + wl.Cp_g * (1 - wl.c)) * T
        dd = None
        if i % 3 == 0:
            dd = torch.full(wl.shape, wl.dd_uniform, dtype=torch.float64, device="cuda")
        boxes.append(P.Box(g, t(wl.c), t(e), t(wl.u), t(wl.v), t(wl.w), wl.dt, dd, wl.dd_uniform))
    return boxes


def per_box(P, wls, nsteps, **kw):
    import torch
    boxes = make_boxes(P, wls, **kw)
    sums = []
    for b in boxes:
        st = P.Stepper(b.grid)
        for s in range(nsteps):
            out = st.step(b.c, b.e, b.u, b.v, b.w, b.dt, s, dd=b.dd, dd_uniform=b.dd_uniform).clone()
        sums.append(out)
    torch.cuda.synchronize()
    return [(b.c.cpu().numpy(), b.e.cpu().numpy()) for b in boxes], torch.stack(sums).cpu().numpy()


def check(boxes, sums, ref):
    fields, rsums = ref
    for b, (c, e) in zip(boxes, fields):
        assert np.array_equal(b.c.cpu().numpy(), c)
        assert np.array_equal(b.e.cpu().numpy(), e)
    assert np.array_equal(sums.cpu().numpy(), rsums)


@pytest.fixture(scope="module")
def ref3(P, droplets):
    return per_box(P, droplets, 3)


@pytest.mark.parametrize("work", [64, 4096])
def test_group_equals_per_box_steps(P, droplets, ref3, work):
    import torch
    boxes = make_boxes(P, droplets)
    grp = P.Group(boxes, work)
    for s in range(3):
        sums = grp.step(s)
    torch.cuda.synchronize()
    assert P.vof_get_device_status() == P.VOF_OK
    check(boxes, sums, ref3)
    grp.close()


def test_group_graph_replay(P, droplets, ref3):
    import torch
    boxes = make_boxes(P, droplets)
    c0 = [b.c.clone() for b in boxes]
    e0 = [b.e.clone() for b in boxes]
    cap = torch.cuda.Stream()
    grp = P.Group(boxes, 1024, stream=cap)
    grp.step(0, stream=cap)  # warm-up outside the capture
    cap.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        for s in range(3):
            grp.step(s, stream=cap)
    for b, c, e in zip(boxes, c0, e0):
        b.c.copy_(c)
        b.e.copy_(e)
    graph.replay()
    torch.cuda.synchronize()
    check(boxes, grp.sums, ref3)


@pytest.mark.parametrize("precision,normal", [(1, 0), (0, 2)])
def test_group_other_forms(P, droplets, precision, normal):
    import torch
    ref = per_box(P, droplets[:12], 2, precision=precision, normal=normal)
    boxes = make_boxes(P, droplets[:12], precision=precision, normal=normal)
    grp = P.Group(boxes, 2048)
    for s in range(2):
        sums = grp.step(s)
    torch.cuda.synchronize()
    check(boxes, sums, ref)


def test_group_refuses_mixed_forms_and_learned_normal(P, droplets):
    boxes = make_boxes(P, droplets[:4])
    boxes[1].grid.precision = 1
    with pytest.raises(P.VofError):
        P.Group(boxes)
    boxes = make_boxes(P, droplets[:2], normal=1)
    for b in boxes:
        b.grid.mlp = P.MLP(np.zeros(P.VOF_MLP_PARAMS, dtype=np.float32)).packed
    with pytest.raises(P.VofError):
        P.Group(boxes)


def test_group_autotune(P, droplets):
    boxes = make_boxes(P, droplets[:10])
    best, timings = P.Group.autotune(boxes, candidates=(256, 4096), steps=2)
    assert best in (256, 4096) and set(timings) == {256, 4096}
