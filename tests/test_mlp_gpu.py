"""The learned interface normal on the GPU (vof_mlp_*, tensor cores) against
the FP64 oracle of the same network (oracle/mlp.py), through the C ABI.

  * forward: identical operands (the FP32 master parameters, weights rounded
    to BF16 on both sides, FP64 stencils); the GPU's output within 1e-5 of
    |y| per stencil, or of the output layer's term magnitude where y
    cancels (FP32 accumulation; the activations enter the BF16 products as
    three-term splits);
  * normals with the MYC fallback: where the oracle's FP64 decision is
    clear of the FP32 residual round-off the GPU decides the same; every
    GPU normal is the network's (to 1e-5) or MYC's (to FP32 round-off);
  * gradient of the batch loss with respect to the BF16 weights: within
    1e-3 of the oracle's exact gradient, per parameter tensor (norm);
  * GPU training lowers the loss and its trained network, with the MYC
    fallback, lowers the mean angular error on held-out sphere stencils
    below 0.85 of MYC's (the oracle's own training does the same on the
    CPU, tests/test_oracle_mlp_gain.py).
"""
import math

import numpy as np
import pytest

import oracle as O
import oracle.mlp as M
from paper_2001_03477_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FWD_TOL = 1e-5
GRAD_TOL = 1e-3


@pytest.fixture(scope="module")
def P():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def master_to_params(master):
    """The FP32 master vector as the oracle's parameter dict (FP64 values of
    the same floats)."""
    v = np.asarray(master, dtype=np.float64)
    p, o = {}, 0
    for k, (a, b) in enumerate(zip(M.SIZES[:-1], M.SIZES[1:]), start=1):
        p[f"W{k}"] = v[o:o + a * b].reshape(b, a)
        o += a * b
        p[f"b{k}"] = v[o:o + b].copy()
        o += b
    assert o == v.size
    return p


def random_master(seed, bias=0.1):
    rng = np.random.default_rng(seed)
    parts = []
    for a, b in zip(M.SIZES[:-1], M.SIZES[1:]):
        parts.append(rng.normal(0.0, math.sqrt(2.0 / a), size=(b, a)).reshape(-1))
        parts.append(rng.normal(0.0, bias, size=b))
    return np.concatenate(parts).astype(np.float32)


def gpu_forward(P, mlp, X):
    import torch
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).cuda()
    y = torch.zeros((X.shape[0], 3), dtype=torch.float32, device="cuda")
    P.vof_mlp_forward(mlp.packed, Xd, y)
    torch.cuda.synchronize()
    assert P.vof_get_device_status() == P.VOF_OK
    return y.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n", [1, 127, 129, 1000, 100_000])
def test_forward_matches_oracle(P, n):
    master = random_master(11)
    mlp = P.MLP(master)
    rng = np.random.default_rng(n)
    # stencils: uniform fractions and exact 0 / 1 cells mixed in
    X = rng.random((n, 27))
    X[rng.random((n, 27)) < 0.2] = 0.0
    X[rng.random((n, 27)) < 0.2] = 1.0
    y = gpu_forward(P, mlp, X)
    p = master_to_params(master)
    yo, cache = M.forward(p, X, weights=M.bf16)
    # relative to |y|, or where the output cancels, to the magnitude of the
    # output layer's terms (the scale of the FP32 accumulation's error)
    terms = np.abs(cache[4]) @ np.abs(M.bf16(p["W3"])).T + np.abs(p["b3"])
    scale = np.maximum(np.linalg.norm(yo, axis=1), np.linalg.norm(terms, axis=1))
    err = np.linalg.norm(y - yo, axis=1) / scale
    assert err.max() <= FWD_TOL, (err.max(), int(np.argmax(err)))
    # and on most stencils relative to |y| itself
    assert np.median(np.linalg.norm(y - yo, axis=1) / np.linalg.norm(yo, axis=1)) <= 2e-6


def test_forward_empty_and_errors(P):
    import torch
    mlp = P.MLP(random_master(3))
    X = torch.zeros((0, 27), dtype=torch.float64, device="cuda")
    y = torch.zeros((0, 3), dtype=torch.float32, device="cuda")
    P.vof_mlp_forward(mlp.packed, X, y)  # n = 0: nothing launched
    import ctypes
    st = P.lib().vof_mlp_forward(ctypes.c_void_p(mlp.packed.data_ptr() + 4), None, 1, None, None)
    assert st == P.VOF_EINVAL  # misaligned parameters, null arrays


@pytest.fixture(scope="module")
def trained(P):
    """A network trained on the GPU (Adam) on generated stencils; returns
    (mlp, losses)."""
    import torch
    X, Y = W.training_stencils(60_000, seed=6)
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    mlp = P.MLP(P.MLP.init_master(5))
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    losses = []
    for s in range(6000):
        lr = 3e-3 if s < 3000 else 1e-3
        mlp.train_step(Xd, Yd, 512, lr, seed=77, loss=loss)
        if s < 10 or s >= 5900:
            losses.append(float(loss.item()))
    torch.cuda.synchronize()
    assert P.vof_get_device_status() == P.VOF_OK
    return mlp, losses


def test_gradient_matches_oracle(P):
    import torch
    master = random_master(21, bias=0.05)
    mlp = P.MLP(master)
    X, Y = W.training_stencils(384, seed=8)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    idx = torch.arange(256, dtype=torch.int64, device="cuda") + 64  # samples 64..319
    grad = torch.zeros(P.VOF_MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    before = mlp.master.clone()
    mlp.train_step(Xd, Yd, 256, 0.0, grad=grad, loss=loss, idx=idx)
    torch.cuda.synchronize()
    assert torch.equal(before, mlp.master)  # lr = 0: gradient only
    p = master_to_params(master)
    pb = {k: (M.bf16(v) if k.startswith("W") else v) for k, v in p.items()}
    lo, go = M.loss_and_grad(pb, X[64:320], Y[64:320])
    assert abs(float(loss.item()) - lo) <= 1e-5 * abs(lo)
    gg = master_to_params(grad.cpu().numpy())
    for k in go:
        rel = np.linalg.norm(gg[k] - go[k]) / np.linalg.norm(go[k])
        assert rel <= GRAD_TOL, (k, rel)


def test_gradient_deterministic(P):
    import torch
    mlp = P.MLP(random_master(4))
    X, Y = W.training_stencils(1024, seed=9)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    g1 = torch.zeros(P.VOF_MLP_PARAMS, dtype=torch.float32, device="cuda")
    g2 = torch.zeros_like(g1)
    mlp.train_step(Xd, Yd, 1024, 0.0, seed=3, grad=g1)
    mlp.train_step(Xd, Yd, 1024, 0.0, seed=3, grad=g2)
    torch.cuda.synchronize()
    assert torch.equal(g1, g2)


def test_adam_step_matches_oracle_update(P):
    # one Adam step from zero moments moves every parameter by lr * g /
    # (|g| + eps) (bias-corrected first step) in the direction of -g
    import torch
    master = random_master(31)
    mlp = P.MLP(master)
    X, Y = W.training_stencils(256, seed=10)
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    idx = torch.arange(256, dtype=torch.int64, device="cuda")
    grad = torch.zeros(P.VOF_MLP_PARAMS, dtype=torch.float32, device="cuda")
    mlp.train_step(Xd, Yd, 256, 1e-3, grad=grad, idx=idx)
    torch.cuda.synchronize()
    g = grad.cpu().numpy().astype(np.float64)
    expect = master.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.abs(mlp.master.cpu().numpy() - expect).max() <= 2e-6
    # the packed images hold the new values (forward of the new master)
    Xs = np.random.default_rng(1).random((300, 27))
    y = gpu_forward(P, mlp, Xs)
    yo, _ = M.forward(master_to_params(mlp.master.cpu().numpy()), Xs, weights=M.bf16)
    assert (np.linalg.norm(y - yo, axis=1) / np.linalg.norm(yo, axis=1)).max() <= FWD_TOL


def angle(a, b):
    return math.degrees(math.acos(float(np.clip(a @ b / np.linalg.norm(a) / np.linalg.norm(b), -1.0, 1.0))))


def test_training_lowers_loss_and_beats_myc(P, trained):
    import torch
    mlp, losses = trained
    assert np.mean(losses[-50:]) < 0.01 * np.mean(losses[:10])
    Xt, Yt = W.training_stencils(600, seed=99, kinds=("sphere",))
    m = torch.zeros((600, 3), dtype=torch.float64, device="cuda")
    fb = torch.zeros(600, dtype=torch.uint8, device="cuda")
    P.vof_mlp_normals(mlp.packed, torch.from_numpy(Xt).cuda(), m, fb)
    torch.cuda.synchronize()
    mg = m.cpu().numpy()
    learned = np.array([angle(mg[i], Yt[i]) for i in range(600)])
    myc = np.array([angle(O.myc(Xt[i].reshape(3, 3, 3)), Yt[i]) for i in range(600)])
    assert learned.mean() < 0.85 * myc.mean(), (learned.mean(), myc.mean())


def test_normals_and_fallback_match_oracle(P, trained):
    import torch
    mlp, _ = trained
    n = 3000
    X, Y = W.training_stencils(n, seed=123)
    # a few stencils of no surface at all (arbitrary fractions)
    rng = np.random.default_rng(4)
    X[:150] = np.clip(rng.random((150, 27)), 1e-3, 1 - 1e-3)
    m = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    fb = torch.zeros(n, dtype=torch.uint8, device="cuda")
    P.vof_mlp_normals(mlp.packed, torch.from_numpy(X).cuda(), m, fb)
    torch.cuda.synchronize()
    mg, fg = m.cpu().numpy(), fb.cpu().numpy()
    p = master_to_params(mlp.master.cpu().numpy())
    yo, _ = M.forward(p, X, weights=M.bf16)
    clear = 0
    for i in range(n):
        s = X[i]
        mo = yo[i] / np.abs(yo[i]).sum()
        myc = O.myc(s.reshape(3, 3, 3))
        res = M.plane_residual(s, mo)
        bound = M.accept_bound(s)
        use_mlp_orc = res <= bound
        if abs(res - bound) > 1e-4 * max(bound, 1e-3):  # clear of FP32 residual round-off
            clear += 1
            assert bool(fg[i] == 0) == use_mlp_orc, (i, res, bound)
        if fg[i] == 0:
            assert np.abs(mg[i] - mo).max() <= 1e-5, i
        else:
            assert np.abs(mg[i] - myc).max() <= 1e-6, i
    assert clear >= 0.95 * n
    assert 0 < int(fg.sum()) < n  # both decisions occur
