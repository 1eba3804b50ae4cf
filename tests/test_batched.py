"""Host side of the batched step (vof_batched_plan, vof_batched_workspace_bytes,
vof_batched_step's argument checks) and the lane autotuner's choice, on the
CPU: nothing here launches a kernel.

* The plan puts every box on a lane; the lanes' cell loads differ by at most
  the largest box (greedy least-loaded assignment in decreasing size).
* Each lane's workspace is 256-byte aligned, disjoint from the others and at
  least the largest vof_step workspace of its boxes.
* An empty batch is a no-op; every bad argument is refused before anything is
  queued (fake device addresses are never dereferenced).
"""
import ctypes

import pytest

import paper_2001_03477_gb300 as P

FAKE = 1 << 40  # never dereferenced: the checks run on the host before any launch


@pytest.fixture(scope="module")
def lib():
    from paper_2001_03477_gb300 import build
    build.build()
    return P.lib()


def droplet_grids(n, seed=4):
    import numpy as np
    rng = np.random.default_rng(seed)
    return [P.Grid(int(k), int(k), int(k), (0, 0, 0), 1.0 / int(k), 1000.0, 1.0, 0.0)
            for k in rng.integers(24, 97, size=n)]


def test_plan_balances_and_covers(lib):
    grids = droplet_grids(200)
    for lanes in (1, 3, 8, 16):
        lane, off, total = P.vof_batched_plan(grids, lanes)
        assert len(lane) == len(grids) and all(0 <= x < lanes for x in lane)
        load = [0] * lanes
        need = [0] * lanes
        for g, l in zip(grids, lane):
            load[l] += g.cells
            need[l] = max(need[l], P.vof_step_workspace_bytes(g))
        assert max(load) - min(load) <= max(g.cells for g in grids)
        ends = []
        for l in range(lanes):
            assert off[l] % 256 == 0
            end = off[l] + need[l]
            ends.append(end)
            if l + 1 < lanes:
                assert end <= off[l + 1]
        assert max(ends) <= total and total % 256 == 0
        assert P.vof_batched_workspace_bytes(grids, lanes) == total
        assert P.vof_batched_plan(grids, lanes) == (lane, off, total)  # deterministic


def test_plan_order_and_idle_lanes(lib):
    sizes = [10, 30, 20, 30]
    grids = [P.Grid(k, k, k) for k in sizes]
    lane, off, total = P.vof_batched_plan(grids, 6)
    # decreasing size, ties by index: boxes 1, 3, 2, 0 on lanes 0, 1, 2, 3
    assert lane == [3, 0, 2, 1]
    assert off[4] == off[5] == total  # idle lanes take no workspace
    lane1, off1, total1 = P.vof_batched_plan(grids, 1)
    assert lane1 == [0, 0, 0, 0] and off1 == [0]
    assert total1 >= max(P.vof_step_workspace_bytes(g) for g in grids)


def test_plan_rejects_bad_arguments(lib):
    grids = [P.Grid(8, 8, 8), P.Grid(0, 8, 8)]
    with pytest.raises(P.VofError):
        P.vof_batched_plan(grids, 2)
    with pytest.raises(P.VofError):
        P.vof_batched_plan(grids[:1], 0)
    assert P.vof_batched_workspace_bytes(grids, 2) == 0


def _boxes(grids, base=FAKE):
    """vof_box array at fake, disjoint device addresses."""
    arr = (P._CBox * len(grids))()
    addr = base
    for i, g in enumerate(grids):
        arr[i].grid = g.c_struct()
        nb = g.cells * 8
        arr[i].c, addr = addr, addr + nb + 256
        arr[i].e, addr = addr, addr + nb + 256
        arr[i].u = arr[i].v = arr[i].w = 1 << 44
        arr[i].dt = 0.01
        arr[i].dd = None
        arr[i].dd_uniform = 0.0
    return arr, addr


def test_step_checks_before_launch(lib):
    grids = [P.Grid(8, 8, 8), P.Grid(12, 10, 9), P.Grid(16, 16, 16)]
    arr, end = _boxes(grids)
    ws_bytes = P.vof_batched_workspace_bytes(grids, 2)
    ws = ctypes.c_void_p(1 << 45)
    nul = ctypes.c_void_p(0)
    streams = (ctypes.c_void_p * 2)(0, 0)
    S = ctypes.c_size_t

    def call(a=arr, n=3, step=0, sums=nul, lanes=2, ls=streams, w=ws, nb=ws_bytes):
        return lib.vof_batched_step(a, n, step, sums, lanes, ls, w, S(nb), nul)

    assert call(n=0, w=nul, nb=0) == P.VOF_OK  # empty batch: nothing to do
    assert call(step=-1) == P.VOF_EINVAL
    assert call(ls=None) == P.VOF_EINVAL  # two lanes need their streams
    assert call(lanes=0) == P.VOF_EINVAL
    assert call(w=nul) == P.VOF_EINVAL
    assert call(w=ctypes.c_void_p((1 << 45) + 8)) == P.VOF_EINVAL  # misaligned workspace
    assert call(nb=ws_bytes - 1) == P.VOF_EINVAL  # short workspace
    # workspace over a box's c
    assert call(w=ctypes.c_void_p(arr[1].c & ~255)) == P.VOF_EINVAL
    # sums over a box's e
    assert call(sums=ctypes.c_void_p(arr[2].e)) == P.VOF_EINVAL
    # overlapping fields of two boxes
    bad, _ = _boxes(grids)
    bad[2].c = bad[0].e + 64
    assert call(a=bad) == P.VOF_EINVAL
    # one box's c covering several other arrays
    bad, _ = _boxes(grids)
    bad[2].c = bad[0].c  # 16^3 doubles from box 0's c cover box 0's e and box 1's c
    assert call(a=bad) == P.VOF_EINVAL
    big = P.Grid(40, 40, 40)
    arr3, _ = _boxes([grids[0], grids[1], big])
    arr3[2].c = arr3[0].c - 4096 * 8  # starts before every other array and ends past box 1's e
    arr3[2].e = arr3[1].e + (1 << 30)
    assert lib.vof_batched_step(arr3, 3, 0, nul, 2, streams, ws, S(P.vof_batched_workspace_bytes(
        [grids[0], grids[1], big], 2)), nul) == P.VOF_EINVAL
    bad, _ = _boxes(grids)
    bad[1].u = None
    assert call(a=bad) == P.VOF_EINVAL
    bad, _ = _boxes(grids)
    bad[0].dt = -1.0
    assert call(a=bad) == P.VOF_EINVAL
    bad, _ = _boxes(grids)
    bad[1].grid.bc[0] = 2
    assert call(a=bad) == P.VOF_EINVAL


def test_binding_checks_lane_streams(lib):
    class FakeStream:
        cuda_stream = 0

    with pytest.raises(ValueError):
        P.vof_batched_step([], 0, lanes=2, lane_streams=[FakeStream()])


def test_autotuner_keeps_the_fastest():
    times = {1: 3.0, 2: 1.6, 4: 1.1, 8: 0.9, 16: 0.9, 32: 1.0}
    seen = []

    def measure(lanes):
        seen.append(lanes)
        return times[lanes]

    assert P.pick_fastest(measure, (1, 2, 4, 8, 16, 32)) == 8  # tie with 16: the earlier one
    assert seen == [1, 2, 4, 8, 16, 32]
    assert P.pick_fastest(lambda x: 1.0, (4,)) == 4


def test_group_plan_sizes_without_gpu():
    import ctypes
    import paper_2001_03477_gb300 as P
    boxes = []
    for n in (9, 17, 24):
        g = P.Grid(n, n, n, (0, 0, 0), 1.0 / n, 1000.0, 1.0, 1.0)
        boxes.append(g)
    arr = P._box_array(boxes, with_arrays=False)
    for i in range(len(boxes)):
        addr = (i + 1) << 36
        arr[i].c, arr[i].e = ctypes.c_void_p(addr), ctypes.c_void_p(addr + (1 << 34))
        arr[i].u = arr[i].v = arr[i].w = ctypes.c_void_p(addr + (2 << 34))
        arr[i].dt = 0.01
    L = P.lib()
    nb = L.vof_group_workspace_bytes(arr, 3, 4096)
    assert nb >= sum(P.vof_step_workspace_bytes(g) for g in boxes)
    assert L.vof_group_workspace_bytes(arr, 3, 16) == 0      # granularity below 32 cells
    assert L.vof_group_workspace_bytes(arr, 0, 4096) == 0    # empty batch
    arr[1].grid.precision = 1
    assert L.vof_group_workspace_bytes(arr, 3, 4096) == 0    # mixed precision
