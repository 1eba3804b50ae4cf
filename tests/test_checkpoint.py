"""Checkpoint and resume of a run's state (host code, no GPU): round trip,
and every damaged or foreign file refused."""
import os

import numpy as np
import pytest


@pytest.fixture(scope="module")
def P():
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P


def state(P):
    g = P.Grid(7, 5, 3, (0, 1, 0), 0.125, 4.0e6, 1.2e3, 373.15, 1e-12, precision=P.VOF_F32_FLUX,
               scheme=P.VOF_SCHEME_LE)
    rng = np.random.default_rng(0)
    return g, rng.random(g.shape), 1e5 * rng.random(g.shape)


def test_round_trip(P, tmp_path):
    g, c, e = state(P)
    path = tmp_path / "run.ckpt"
    P.vof_checkpoint_save(path, g, c, e, step=1234, t=5.5)
    assert not os.path.exists(str(path) + ".tmp")
    g2, step, t, c2, e2 = P.vof_checkpoint_load(path)
    assert (g2.nx, g2.ny, g2.nz, tuple(g2.bc)) == (7, 5, 3, (0, 1, 0))
    assert (g2.h, g2.Cp_l, g2.Cp_g, g2.T_sat, g2.eps_mixed) == (g.h, g.Cp_l, g.Cp_g, g.T_sat, g.eps_mixed)
    assert (g2.precision, g2.scheme, step, t) == (g.precision, g.scheme, 1234, 5.5)
    assert np.array_equal(c2, c) and np.array_equal(e2, e)
    # saving again replaces the file in place
    P.vof_checkpoint_save(path, g, c * 0.5, e, step=1235, t=6.0)
    assert P.vof_checkpoint_load(path)[1] == 1235


def test_damaged_or_foreign_files_are_refused(P, tmp_path):
    g, c, e = state(P)
    path = tmp_path / "run.ckpt"
    P.vof_checkpoint_save(path, g, c, e)
    raw = bytearray(open(path, "rb").read())
    cases = {
        "flipped payload byte": raw[:200] + bytes([raw[200] ^ 1]) + raw[201:],
        "flipped header byte": raw[:20] + bytes([raw[20] ^ 1]) + raw[21:],
        "truncated": raw[:-9],
        "trailing byte": raw + b"\0",
        "foreign magic": b"NOTACKPT" + raw[8:],
        "empty": b"",
    }
    for name, data in cases.items():
        bad = tmp_path / name.replace(" ", "_")
        open(bad, "wb").write(bytes(data))
        with pytest.raises(P.VofError):
            P.vof_checkpoint_load(bad)
    with pytest.raises(P.VofError):
        P.vof_checkpoint_load(tmp_path / "missing.ckpt")
    # a buffer of the wrong size is refused by the library itself
    import ctypes
    buf = np.empty(10)
    assert P.lib().vof_checkpoint_load(str(path).encode(), 10, buf.ctypes.data, buf.ctypes.data) == P.VOF_EINVAL


def test_wrong_field_size_is_refused(P, tmp_path):
    g, c, e = state(P)
    with pytest.raises(ValueError):
        P.vof_checkpoint_save(tmp_path / "x.ckpt", g, c[:2], e)


def test_step_record_is_one_json_line(P):
    import json
    line = P.step_record(12, 0.5, [1.0, 2.0, -1e-17, -0.25, 0.0, -300.0],
                         {"mixed": [1, 2, 3], "faces": [4, 5, 6], "shift_analytic": 7, "shift_bisection": 8,
                          "receivers": 9})
    assert "\n" not in line
    rec = json.loads(line)
    assert rec["step"] == 12 and rec["t"] == 0.5 and rec["sum_e"] == 2.0 and rec["shift_de"] == -300.0
    assert rec["mixed"] == [1, 2, 3] and rec["receivers"] == 9
