"""The time step decomposes into z-slabs with halo exchanges (CPU, gloo).

A multi-GPU form of the step would split the grid into z-slabs, one per rank.
This test checks that split on the oracle. Each rank holds its slab plus
G = 3 ghost layers on each side and exchanges them with its periodic
neighbours before each sweep and before the shift. Between exchanges it
runs the oracle's frozen state, sweeps and shift on the extended slab, with
a zero-gradient z boundary that only the ghosts see.

G = 3 is the widest reach of one operation:
* a z-face flux reads the WENO5 window of three cells upwind;
* the donor's MYC stencil reads one cell beyond the donor;
* the shift of a cell reads its neighbours' planes, whose stencils reach two
  cells.

Expected: the gathered interior slabs equal the single-domain oracle bit
for bit after several steps in both sweep orders. The cases are two ranks
and a ragged split over three ranks.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
G = 3
SHAPE = (26, 20, 18)  # (nz, ny, nx)
NSTEPS = 4


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _case():
    sys.path.insert(0, ROOT)
    from paper_2001_03477_gb300 import workloads as W
    nz, ny, nx = SHAPE
    h = 1.0 / nx
    c = W.sphere_fractions(SHAPE, h, (0.45, 0.5, 0.62), 0.3, nsub=6)
    Cp_l, Cp_g = 1000.0, 1.0
    T = W.fourier_field(SHAPE, h, seed=5)
    e = (Cp_l * c + Cp_g * (1.0 - c)) * T
    vel = (0.3, -0.2, 0.45)
    u, v, w = W.uniform_faces(SHAPE, vel)
    dt = 0.5 * h
    dd = np.random.default_rng(11).uniform(-0.02, 0.02, SHAPE)
    return dict(h=h, Cp_l=Cp_l, Cp_g=Cp_g, T_sat=1.0, c=c, e=e, u=u, v=v, w=w, dt=dt, dd=dd)


def _bounds(rank, world):
    nz = SHAPE[0]
    base, extra = divmod(nz, world)
    z0 = rank * base + min(rank, extra)
    return z0, z0 + base + (1 if rank < extra else 0)


def _rank_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle as O
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        k = _case()
        nz, ny, nx = SHAPE
        z0, z1 = _bounds(rank, world)
        nl = z1 - z0
        zc = [(z0 - G + i) % nz for i in range(nl + 2 * G)]  # global z of each extended layer
        zf = [(z0 - G + i) % nz for i in range(nl + 2 * G + 1)]  # global z-face of each extended face
        c = np.ascontiguousarray(k["c"][zc])
        e = np.ascontiguousarray(k["e"][zc])
        uf = [np.ascontiguousarray(k["u"][zc]), np.ascontiguousarray(k["v"][zc]), np.ascontiguousarray(k["w"][zf])]
        dd = np.ascontiguousarray(k["dd"][zc])
        g = O.Grid(nx, ny, nl + 2 * G, (0, 0, 1), k["h"], k["Cp_l"], k["Cp_g"], k["T_sat"])
        nxt, prv = (rank + 1) % world, (rank - 1) % world

        def exchange(c, e):
            # my top interior layers -> next rank's low ghosts (tag 0);
            # my low interior layers -> previous rank's top ghosts (tag 1)
            top = torch.from_numpy(np.stack([c[nl:nl + G], e[nl:nl + G]]).copy())
            low = torch.from_numpy(np.stack([c[G:2 * G], e[G:2 * G]]).copy())
            r_low = torch.empty_like(top)
            r_top = torch.empty_like(low)
            reqs = [dist.isend(top, nxt, tag=0), dist.isend(low, prv, tag=1),
                    dist.irecv(r_low, prv, tag=0), dist.irecv(r_top, nxt, tag=1)]
            for r in reqs:
                r.wait()
            c[:G], e[:G] = r_low[0].numpy(), r_low[1].numpy()
            c[nl + G:], e[nl + G:] = r_top[0].numpy(), r_top[1].numpy()

        for step in range(NSTEPS):
            exchange(c, e)
            cc, th = O.frozen(g, c, e)
            for s in range(3):
                axis = s if step % 2 == 0 else 2 - s
                if s > 0:
                    exchange(c, e)
                c, e, _ = O.sweep(g, axis, c, e, uf[axis], k["dt"], cc, th)
            exchange(c, e)
            c, e, _ = O.phase_shift(g, c, e, dd)
        mine = torch.from_numpy(np.stack([c[G:G + nl], e[G:G + nl]]).copy())
        if rank == 0:
            out_c = np.empty(SHAPE)
            out_e = np.empty(SHAPE)
            out_c[z0:z1], out_e[z0:z1] = mine[0].numpy(), mine[1].numpy()
            for r in range(1, world):
                a, b = _bounds(r, world)
                buf = torch.empty((2, b - a, ny, nx), dtype=torch.float64)
                dist.recv(buf, r)
                out_c[a:b], out_e[a:b] = buf[0].numpy(), buf[1].numpy()
            og = O.Grid(nx, ny, nz, (0, 0, 0), k["h"], k["Cp_l"], k["Cp_g"], k["T_sat"])
            rc, re_ = k["c"], k["e"]
            for step in range(NSTEPS):
                rc, re_, _ = O.step(og, rc, re_, k["u"], k["v"], k["w"], k["dt"], step, dd=k["dd"])
            q.put((int(np.count_nonzero(out_c != rc)), int(np.count_nonzero(out_e != re_)),
                   int(np.count_nonzero((rc > 1e-12) & (rc < 1 - 1e-12))),
                   float(np.abs(rc - k["c"]).max())))
        else:
            dist.send(mine, 0)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_with_halo_exchange_equal_the_single_domain_step(world):
    import multiprocessing as mp
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
    assert all(p.exitcode == 0 for p in procs)
    bad_c, bad_e, mixed, moved = q.get(timeout=5)
    assert mixed > 200 and moved > 0.1  # the interface crosses the slab boundaries and moves
    assert bad_c == 0 and bad_e == 0
