"""The C-ABI library builds for sm_103a, loads, exports every entry point
declared in include/vofgb.h, and rejects bad arguments on the host before
launching anything (no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2001_03477_gb300 import build
    build.build()
    import paper_2001_03477_gb300 as P
    return P.lib()


def declared_functions():
    src = open(os.path.join(ROOT, "include", "vofgb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:VOF_API\s+)?(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_lists_the_hot_path():
    names = declared_functions()
    for n in ("vof_reconstruct", "vof_advect_sweep_x", "vof_advect_sweep_y", "vof_advect_sweep_z",
              "vof_phase_change_shift", "energy_advect_consistent", "vof_step", "vof_step_workspace_bytes"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    for n in declared_functions():
        assert hasattr(lib, n), n


def test_host_validation_without_gpu(lib):
    import paper_2001_03477_gb300 as P
    g = P.Grid(8, 8, 8, (0, 0, 0), 1.0, 2.0, 1.0, 0.0)
    cg = g.c_struct()
    nul = ctypes.c_void_p(0)
    # null arrays
    assert lib.vof_reconstruct(ctypes.byref(cg), nul, nul, nul, nul, nul) == P.VOF_EINVAL
    assert lib.vof_advect_sweep_x(ctypes.byref(cg), nul, nul, nul, nul, nul, 0.1, nul, nul, nul, nul, nul, 0,
                                  nul) == P.VOF_EINVAL
    # partly overlapping input and output (exactly in place is allowed)
    fake = ctypes.c_void_p(1 << 40)
    ws = ctypes.c_void_p(5 << 40)
    big = lib.vof_sweep_workspace_bytes(ctypes.byref(cg))
    assert lib.vof_advect_sweep_y(ctypes.byref(cg), fake, nul, ctypes.c_void_p((1 << 40) + 64), nul,
                                  ctypes.c_void_p(1 << 41), 0.1, nul, nul, nul, nul, ws, big, nul) == P.VOF_EINVAL
    # c in place but e out of place
    e1, e2 = ctypes.c_void_p(2 << 40), ctypes.c_void_p(3 << 40)
    assert lib.vof_advect_sweep_x(ctypes.byref(cg), fake, e1, fake, e2, ctypes.c_void_p(1 << 41), 0.1, nul, nul,
                                  nul, nul, ws, big, nul) == P.VOF_EINVAL
    # sweep workspace missing, too small or misaligned
    ok_out = ctypes.c_void_p(4 << 40)
    for w_, nb in ((nul, big), (ws, big - 8), (ctypes.c_void_p((5 << 40) + 16), big)):
        assert lib.vof_advect_sweep_z(ctypes.byref(cg), fake, nul, ok_out, nul, ctypes.c_void_p(1 << 41), 0.1, nul,
                                      nul, nul, nul, w_, nb, nul) == P.VOF_EINVAL
    # bad grid
    big_step = lib.vof_step_workspace_bytes(ctypes.byref(cg))
    bad = P.Grid(0, 8, 8).c_struct()
    assert lib.vof_step_workspace_bytes(ctypes.byref(bad)) == 0
    bad2 = P.Grid(8, 8, 8, (0, 2, 0)).c_struct()
    assert lib.vof_reconstruct(ctypes.byref(bad2), fake, fake, fake, fake, nul) == P.VOF_EINVAL
    bad3 = P.Grid(8, 8, 8, precision=2).c_struct()  # neither VOF_F64 nor VOF_F32_FLUX
    assert lib.vof_step_workspace_bytes(ctypes.byref(bad3)) == 0
    assert lib.vof_reconstruct(ctypes.byref(bad3), fake, fake, fake, fake, nul) == P.VOF_EINVAL
    assert lib.vof_step_workspace_bytes(ctypes.byref(P.Grid(8, 8, 8, precision=P.VOF_F32_FLUX).c_struct())) == big_step
    # negative dt, misaligned workspace
    assert lib.vof_step(ctypes.byref(cg), fake, ctypes.c_void_p(2 << 40), fake, fake, fake, -1.0, 0, nul, 0.0, nul,
                        ctypes.c_void_p(3 << 40), 1 << 30, nul) == P.VOF_EINVAL
    assert lib.vof_step(ctypes.byref(cg), fake, ctypes.c_void_p(2 << 40), fake, fake, fake, 0.1, 0, nul, 0.0, nul,
                        ctypes.c_void_p((3 << 40) + 8), 1 << 30, nul) == P.VOF_EINVAL
    # workspace too small
    assert lib.vof_step(ctypes.byref(cg), fake, ctypes.c_void_p(2 << 40), fake, fake, fake, 0.1, 0, nul, 0.0, nul,
                        ctypes.c_void_p(3 << 40), 16, nul) == P.VOF_EINVAL
    # shift workspace missing, too small, misaligned or overlapping an output
    shb = lib.vof_shift_workspace_bytes(ctypes.byref(cg))
    ce, eo = ctypes.c_void_p(2 << 40), ctypes.c_void_p(6 << 40)
    for w_, nb in ((nul, shb), (ws, shb - 8), (ctypes.c_void_p((5 << 40) + 16), shb), (ok_out, shb)):
        assert lib.vof_phase_change_shift(ctypes.byref(cg), fake, ce, ok_out, eo, nul, 0.01, nul, nul, w_, nb,
                                          nul) == P.VOF_EINVAL
    assert lib.vof_status_string(P.VOF_ECFL).decode() == "face CFL number above 1"


def test_mass_transfer_validation_without_gpu(lib):
    import paper_2001_03477_gb300 as P
    g = P.Grid(8, 8, 8, (0, 0, 0), 1.0, 2.0, 1.0, 0.0)
    cg = g.c_struct()
    nul = ctypes.c_void_p(0)
    c, e, md = ctypes.c_void_p(1 << 40), ctypes.c_void_p(2 << 40), ctypes.c_void_p(3 << 40)
    ws = ctypes.c_void_p(5 << 40)
    nb = lib.vof_mass_transfer_workspace_bytes(ctypes.byref(cg))
    assert nb > 512 * 40

    def call(c_=c, e_=e, md_=md, dgam=nul, gn=nul, dd=nul, ws_=ws, nb_=nb, hfg=1.0, kl=1.0):
        return lib.vof_mass_transfer(ctypes.byref(cg), c_, e_, ctypes.c_double(kl), ctypes.c_double(0.1),
                                     ctypes.c_double(hfg), md_, dgam, gn, ctypes.c_double(-0.5), dd, ws_,
                                     ctypes.c_size_t(nb_), nul)
    assert call(c_=nul) == P.VOF_EINVAL
    assert call(md_=nul) == P.VOF_EINVAL
    assert call(ws_=nul) == P.VOF_EINVAL
    assert call(hfg=0.0) == P.VOF_EINVAL
    assert call(kl=-1.0) == P.VOF_EINVAL
    assert call(nb_=nb - 8) == P.VOF_EINVAL
    assert call(ws_=ctypes.c_void_p((5 << 40) + 64)) == P.VOF_EINVAL
    assert call(md_=ctypes.c_void_p((1 << 40) + 8)) == P.VOF_EINVAL          # mdot over c
    assert call(dd=ctypes.c_void_p((3 << 40) + 16)) == P.VOF_EINVAL          # dd over mdot
    assert call(gn=ctypes.c_void_p((5 << 40) + 256)) == P.VOF_EINVAL         # grad_n in the workspace
    bad = P.Grid(0, 8, 8).c_struct()
    assert lib.vof_mass_transfer_workspace_bytes(ctypes.byref(bad)) == 0
    big = P.Grid(16, 16, 16).c_struct()
    assert lib.vof_mass_transfer_workspace_bytes(ctypes.byref(big)) > 7 * nb


def test_velocity_extension_validation_without_gpu(lib):
    import paper_2001_03477_gb300 as P
    g = P.Grid(8, 8, 8, (1, 1, 1), 0.1, 2.0, 1.0, 0.0)
    cg = g.c_struct()
    nul = ctypes.c_void_p(0)
    c, md = ctypes.c_void_p(1 << 40), ctypes.c_void_p(2 << 40)
    u, v, w = (ctypes.c_void_p(k << 40) for k in (3, 4, 5))
    ws = ctypes.c_void_p(7 << 40)
    nb = lib.vof_velocity_extension_workspace_bytes(ctypes.byref(cg))
    assert nb > 512 * 100
    it, res = ctypes.c_int(0), ctypes.c_double(0.0)

    def call(c_=c, md_=md, uu=(u, v, w), tt=(nul, nul, nul), rl=958.0, rg=0.6, tol=1e-12, mi=100, ws_=ws, nb_=nb):
        return lib.vof_velocity_extension(ctypes.byref(cg), c_, md_, rl, rg, 1e-3, tol, mi, *uu, *tt,
                                          ctypes.byref(it), ctypes.byref(res), ws_, ctypes.c_size_t(nb_), nul)
    assert call(c_=nul) == P.VOF_EINVAL
    assert call(md_=nul) == P.VOF_EINVAL
    assert call(uu=(nul, nul, nul)) == P.VOF_EINVAL            # nothing to write
    assert call(uu=(u, nul, w)) == P.VOF_EINVAL                # partial set
    assert call(rg=0.0) == P.VOF_EINVAL
    assert call(tol=0.0) == P.VOF_EINVAL
    assert call(mi=0) == P.VOF_EINVAL
    assert call(nb_=nb - 8) == P.VOF_EINVAL
    assert call(ws_=ctypes.c_void_p((7 << 40) + 128)) == P.VOF_EINVAL
    assert call(uu=(ctypes.c_void_p((1 << 40) + 8), v, w)) == P.VOF_EINVAL   # u over c
    assert call(uu=(u, ctypes.c_void_p((3 << 40) + 64), w)) == P.VOF_EINVAL  # v over u
    assert lib.vof_status_string(P.VOF_ESOLVE).startswith(b"iterative solve")


def test_heat_diffusion_validation_without_gpu(lib):
    import paper_2001_03477_gb300 as P
    g = P.Grid(8, 8, 8, (1, 1, 1), 0.1, 2.0, 1.0, 0.0)
    cg = g.c_struct()
    nul = ctypes.c_void_p(0)
    c, e, ws = ctypes.c_void_p(1 << 40), ctypes.c_void_p(2 << 40), ctypes.c_void_p(7 << 40)
    nb = lib.vof_heat_diffusion_workspace_bytes(ctypes.byref(cg))
    assert nb > 512 * 80
    it, ch = ctypes.c_int(0), ctypes.c_double(0.0)

    def call(c_=c, e_=e, kl=0.5, dt=1e-3, tol=1e-12, mi=10, ws_=ws, nb_=nb, hc=0, walls=None, grid=cg):
        return lib.vof_heat_diffusion(ctypes.byref(grid), c_, e_, kl, 0.1, dt, tol, mi, hc, walls, ctypes.byref(it),
                                      ctypes.byref(ch), ws_, ctypes.c_size_t(nb_), nul)
    assert call(hc=2) == P.VOF_EINVAL
    nan = float("nan")
    assert call(walls=(ctypes.c_double * 6)(nan, nan, nan, nan, float("inf"), nan)) == P.VOF_EINVAL
    gp = P.Grid(8, 8, 8, (0, 1, 1), 0.1, 2.0, 1.0, 0.0).c_struct()  # x periodic: no wall temperature there
    assert call(walls=(ctypes.c_double * 6)(300.0, nan, nan, nan, nan, nan), grid=gp) == P.VOF_EINVAL
    assert call(c_=nul) == P.VOF_EINVAL
    assert call(e_=nul) == P.VOF_EINVAL
    assert call(kl=-1.0) == P.VOF_EINVAL
    assert call(dt=0.0) == P.VOF_EINVAL
    assert call(tol=0.0) == P.VOF_EINVAL
    assert call(mi=0) == P.VOF_EINVAL
    assert call(nb_=nb - 8) == P.VOF_EINVAL
    assert call(e_=ctypes.c_void_p((1 << 40) + 8)) == P.VOF_EINVAL   # e over c
    assert call(ws_=ctypes.c_void_p((2 << 40) - 256)) == P.VOF_EINVAL  # workspace over e


def test_workspace_size_scales(lib):
    import paper_2001_03477_gb300 as P
    a = P.vof_step_workspace_bytes(P.Grid(32, 32, 32))
    b = P.vof_step_workspace_bytes(P.Grid(64, 64, 64))
    assert a >= 32 ** 3 * 25 and b >= 64 ** 3 * 25 and b > 5 * a
    s = P.vof_sweep_workspace_bytes(P.Grid(64, 64, 64))
    assert 64 ** 3 * 12 <= s < b
    # planes (32 B) and shifts (8 B) of every cell, plus the lists
    sh = P.vof_shift_workspace_bytes(P.Grid(64, 64, 64))
    assert 64 ** 3 * 44 <= sh < b


def test_binding_refuses_cpu_tensors(lib):
    import torch
    import paper_2001_03477_gb300 as P
    g = P.Grid(4, 4, 4)
    c = torch.zeros(4, 4, 4, dtype=torch.float64)
    with pytest.raises(ValueError):
        P.vof_reconstruct(g, c, c, c, c)


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """No CPU fallback: without the built library every call raises."""
    import torch
    import paper_2001_03477_gb300 as P
    monkeypatch.setattr(P, "LIB_PATH", str(tmp_path / "absent.so"))
    monkeypatch.setattr(P, "_lib", None)
    with pytest.raises(RuntimeError):
        P.lib()
    g = P.Grid(4, 4, 4)
    c = torch.zeros(4, 4, 4, dtype=torch.float64)
    with pytest.raises(RuntimeError):
        P.vof_mass_transfer(g, c, c, 1.0, 1.0, 1.0, c)
    with pytest.raises(RuntimeError):
        P.vof_step_workspace_bytes(g)


@pytest.mark.parametrize("lang,std", [("c", "-std=c99"), ("c++", "-std=c++17")])
def test_header_compiles_alone(tmp_path, lang, std):
    """include/vofgb.h is self-contained plain C (usable from C and C++)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc" if lang == "c" else "g++")
    if cc is None:
        pytest.skip("no host compiler")
    src = tmp_path / ("t.c" if lang == "c" else "t.cpp")
    src.write_text('#include "vofgb.h"\nint main(void) { vof_grid g; (void)g; return (int)VOF_OK; }\n')
    r = subprocess.run([cc, std, "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_every_declaration_cites_its_passage():
    # Each entry point of the C header sits under a comment that cites the
    # paper's passage defining the operation (a section, equation or table)
    # or says that the paper has no counterpart.
    with open(os.path.join(ROOT, "include", "vofgb.h")) as f:
        h = f.read()
    names = []
    for m in re.finditer(r"VOF_API [^;]*?\b(vof_\w+|energy_\w+)\(", h):
        # the nearest comment that starts a line (not a struct field's)
        start = h.rfind("\n/*", 0, m.start())
        comment = h[start:h.index("*/", start)]
        text = " ".join(comment.replace("*", " ").split())
        if not any(t in text for t in ("Sec.", "Eq.", "Table", "no counterpart")):
            names.append(m.group(1))
    assert not names, f"declarations without a citation: {names}"
