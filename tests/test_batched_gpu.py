"""The batched form on the GPU (vof_batched_step through the C ABI): a
batch of uneven droplet subdomains spread over 1, 3 and 8 lane streams, and
the same batch captured in a CUDA graph and replayed, against one vof_step
per box on a single stream.  The batched step runs the same kernels with the
same sums on every box, so every box's c, e and sums must be identical bit
for bit, whatever the lanes' interleaving.
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
    # uneven boxes of 10..40 cells per edge (the droplet generator with a
    # smaller range), some with a per-cell shift array
    return [W.droplet_subdomain(i, n_lo=10, n_hi=40, nsub=4) for i in range(NBOX)]


def make_boxes(P, wls, with_dd):
    import torch
    boxes = []
    for i, wl in enumerate(wls):
        g = P.Grid(wl.shape[2], wl.shape[1], wl.shape[0], wl.bc, wl.h, wl.Cp_l, wl.Cp_g, wl.T_sat)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
        dd = None
        if with_dd and i % 3 == 0:
            dd = torch.full((wl.cells,), wl.dd_uniform, dtype=torch.float64, device="cuda").reshape(wl.shape)
        boxes.append(P.Box(g, t(wl.c), t(wl.e), t(wl.u), t(wl.v), t(wl.w), wl.dt, dd, wl.dd_uniform))
    return boxes


def reference(P, wls, nsteps):
    """One vof_step per box on the current stream, box after box."""
    import torch
    boxes = make_boxes(P, wls, True)
    sums = []
    for b in boxes:
        st = P.Stepper(b.grid)
        for s in range(nsteps):
            out = st.step(b.c, b.e, b.u, b.v, b.w, b.dt, s, dd=b.dd, dd_uniform=b.dd_uniform).clone()
        sums.append(out)
    torch.cuda.synchronize()
    return [(b.c.cpu().numpy(), b.e.cpu().numpy()) for b in boxes], torch.stack(sums).cpu().numpy()


@pytest.fixture(scope="module")
def ref(P, droplets):
    return reference(P, droplets, 2)


@pytest.mark.parametrize("lanes", [1, 3, 8])
def test_batched_equals_per_box_steps(P, droplets, ref, lanes):
    import torch
    boxes = make_boxes(P, droplets, True)
    batch = P.BoxBatch(boxes, lanes)
    for s in range(2):
        sums = batch.step(s)
    torch.cuda.synchronize()
    fields, rsums = ref
    for b, (c, e) in zip(boxes, fields):
        assert np.array_equal(b.c.cpu().numpy(), c)
        assert np.array_equal(b.e.cpu().numpy(), e)
    assert np.array_equal(sums.cpu().numpy(), rsums)


def test_batched_graph_replay_equals_per_box_steps(P, droplets, ref):
    import torch
    boxes = make_boxes(P, droplets, True)
    batch = P.BoxBatch(boxes, 4)
    # capture the two steps on a side stream (the lanes fork from it and
    # join back into it), then replay once from the initial state
    c0 = [b.c.clone() for b in boxes]
    e0 = [b.e.clone() for b in boxes]
    cap = torch.cuda.Stream()
    batch.step(0, stream=cap)  # warm-up outside the capture (lazy set-up)
    cap.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=cap):
        batch.step(0, stream=cap)
        batch.step(1, stream=cap)
    for b, c, e in zip(boxes, c0, e0):
        b.c.copy_(c)
        b.e.copy_(e)
    graph.replay()
    torch.cuda.synchronize()
    fields, rsums = ref
    for b, (c, e) in zip(boxes, fields):
        assert np.array_equal(b.c.cpu().numpy(), c)
        assert np.array_equal(b.e.cpu().numpy(), e)
    assert np.array_equal(batch.sums.cpu().numpy(), rsums)


def test_autotuner_picks_a_lane_count(P, droplets):
    boxes = make_boxes(P, droplets[:12], False)
    batch = P.BoxBatch(boxes, 1)
    lanes = batch.autotune(candidates=(1, 2, 4), steps=2)
    assert lanes in (1, 2, 4)
    assert set(batch.timings) == {1, 2, 4}
