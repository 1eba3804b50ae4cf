"""The coupled Stefan problem on the oracle's pieces against the paper's
Table stefan_errors (Sec. 4.3; tests/golden/stefan_water.json).

A vapour layer sits between a wall at T_sat + 10 K and water at T_sat, with
water/steam properties from Table atm_water and a 10 mm domain. The layer
starts at 322.5 um (t0 = 0.282435 s) with a linear temperature profile in
the vapour. The time steps are 0.004 s (N = 32) and 0.002 s (N = 64), run
to t = 10 s. Each step:
* m-dot from the PLIC interface distances (oracle mass_transfer) at the
  mixed cell;
* the liquid velocity from the 1D mass balance, u_l = m-dot (1/rho_g -
  1/rho_l), on the liquid faces and on the two gas faces before the mixed
  cell. This is the sub-domain of the velocity extension, with the vapour
  at rest beyond it;
* the time step: three sweeps with the energy in tandem, then the shift
  dd = -m-dot dt / (rho_l h);
* implicit diffusion with the interface as a Dirichlet boundary and the
  heated wall, each node with the constant properties of its phase
  (diffusion heat_capacity="phase").

Result: delta(10 s) over-predicts the analytic 1.919 mm by 1.1 % at N = 32
and 0.72 % at N = 64 (0.41 % at N = 128). The paper's full solver gives
0.62 % at N = 64 and 0.39 % at N = 128, and the abstract states an error
below 1 %. With the mixture heat capacity in the diffusion instead, the same
loop is 4.8 % / 3.6 % off: the half-liquid interface cell's gas node then
holds ~1600 times the vapour's heat capacity and stays near T_sat.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle.diffusion import diffuse

HERE = os.path.dirname(os.path.abspath(__file__))
G = json.load(open(os.path.join(HERE, "golden", "stefan_water.json")))


def delta_at_end(N, dt, heat_capacity="phase"):
    rl, rg, hfg = G["rho_l"], G["rho_g"], G["h_fg"]
    Cpl, Cpg = rl * G["cp_l"], rg * G["cp_g"]
    kl, kg = G["k_l"], G["k_g"]
    Tsat, Tw = 373.15, 373.15 + G["T_sup"]
    h = G["domain_m"] / N
    g = O.Grid(N, 1, 1, (1, 0, 0), h, Cpl, Cpg, Tsat)
    x = (np.arange(N) + 0.5) * h
    d0 = G["delta0_m"]
    c = (np.clip((np.arange(N) + 1) * h - d0, 0.0, h) / h).reshape(1, 1, N)
    T = np.where(x < d0, Tsat + G["T_sup"] * (1.0 - x / d0), Tsat).reshape(1, 1, N)
    e = (Cpl * c + Cpg * (1.0 - c)) * T
    v, w = np.zeros((1, 2, N)), np.zeros((2, 1, N))
    nsteps = int(round((G["t_end_s"] - G["t0_s"]) / dt))
    for s in range(nsteps):
        mdot, _, _ = O.mass_transfer(g, c, e, kl, kg, hfg)
        mixed = ((c > 1e-12) & (c < 1 - 1e-12)).ravel()
        md = float(mdot.ravel()[mixed].mean())
        k_m = int(np.nonzero(mixed)[0][0])
        u = np.zeros((1, 1, N + 1))
        u[0, 0, max(1, k_m - 2):] = md * (1.0 / rg - 1.0 / rl)
        c, e, _ = O.step(g, c, e, u, v, w, dt, s, dd_uniform=-md * dt / (rl * h))
        e = diffuse(g, c, e, kl, kg, dt, wall_T={(0, -1): Tw}, heat_capacity=heat_capacity)
    return float((1.0 - c).sum() * h)


def test_delta0_and_analytic_end_agree_with_the_paper():
    # Eq. stefan_lamda, Eq. stefan_delta: t0 reproduces delta0 and delta(10 s) = 1.919 mm
    rg, cpg, kg = G["rho_g"], G["cp_g"], G["k_g"]
    f = lambda l: l * math.exp(l * l) * math.erf(l) - cpg * G["T_sup"] / (G["h_fg"] * math.sqrt(math.pi))
    lo, hi = 1e-6, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        lo, hi = (mid, hi) if f(mid) < 0 else (lo, mid)
    lam = 0.5 * (lo + hi)
    alpha = kg / (rg * cpg)
    assert abs(2 * lam * math.sqrt(alpha * G["t0_s"]) - G["delta0_m"]) / G["delta0_m"] < 1e-3
    assert abs(2 * lam * math.sqrt(alpha * G["t_end_s"]) - G["delta_end_m"]) / G["delta_end_m"] < 1e-3


def test_coupled_stefan_loop_reproduces_the_table():
    err = {N: (delta_at_end(N, dt) - G["delta_end_m"]) / G["delta_end_m"] for N, dt in ((32, 0.004), (64, 0.002))}
    # over-prediction like the paper's solver, converging, below 1 % at N = 64
    assert 0.0 < err[64] < err[32] < 0.02
    assert err[64] < 0.01
    # within 0.2 percentage points of the paper's 0.62 % at N = 64
    paris64 = (G["paris_delta_end_m"]["64"] - G["delta_end_m"]) / G["delta_end_m"]
    assert abs(err[64] - paris64) < 0.002
