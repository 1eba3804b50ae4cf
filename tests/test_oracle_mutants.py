"""The oracle's pins reject plausible slips in the oracle itself.

Every parity claim of the CUDA path rests on the oracle, and the oracle is
trusted because its pins (tests/test_oracle_geometry.py, _invariants.py,
_boundary.py, _le.py, _mass_transfer.py) tie it to what the paper and the
mathematics fix: exact volumes, exact plane motion, conservation, uniform
temperature preserved, closed-form mass-transfer rates, and so on.  This file
checks that those pins have teeth.  Each mutant below is one plausible
mistake planted in a copy of oracle/vof_oracle.c (a wrong constant, a dropped
term, a flipped sign, a transposed index or operand).  The copy is compiled
on the CPU with the oracle's own compiler flags into a temporary directory,
the pins run against it in a child process, and at least one pin must fail.
The unchanged source, compiled the same way, must pass the same pins, so a
broken harness cannot pass for a caught mutant.  Nothing here touches the
committed oracle or its library.

The numpy oracles of the learned normal (oracle/mlp.py), the interface-
Dirichlet diffusion (oracle/diffusion.py) and the velocity extension
(oracle/extension.py) get the same treatment: the mutated module is loaded
under its own name in the child before its pins run.

The pin set leaves out the 32^3 sphere return of one period (a minute of
CPU time; every mutant below is caught without it).  Two kinds of change are
deliberately not mutants: the Strang order (x, y, z on even steps; reading
of the configuration, not of a physical law that a pin could fix) and the
tie rules of the readings (c_c at exactly 1/2, the MYC tie), which only
parity with a second implementation can pin.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "vof_oracle.c")

PINS = [
    "tests/test_oracle_geometry.py",
    "tests/test_oracle_invariants.py",
    "tests/test_oracle_boundary.py",
    "tests/test_oracle_le.py",
    "tests/test_oracle_mass_transfer.py",
]
SKIP = ["tests/test_oracle_invariants.py::TestTranslation::test_sphere_translation_returns"]

# (name, text in vof_oracle.c, replacement).  Each text occurs exactly once.
MUTANTS = [
    # volume V(m, alpha), Sec. 3.2 (Scardovelli-Zaleski inclusion-exclusion)
    ("volume: first branch constant 6 -> 2",
     "return a * a * a / (6.0 * m1 * m2 * m3);", "return a * a * a / (2.0 * m1 * m2 * m3);"),
    ("volume: second branch drops its m1^2 term",
     "double v2 = a * (a - m1) / (2.0 * m2 * m3) + m1 * m1 / (6.0 * m2 * m3);",
     "double v2 = a * (a - m1) / (2.0 * m2 * m3);"),
    ("volume: symmetry V(alpha) = 1 - V(1 - alpha) taken at alpha",
     "return 1.0 - vol_sorted_low(s[0], s[1], s[2], 1.0 - alpha);",
     "return 1.0 - vol_sorted_low(s[0], s[1], s[2], alpha);"),
    ("volume: mirror shift with the wrong sign",
     "if (m[d] < 0.0) { mpos[d] = -m[d]; sh -= m[d]; }", "if (m[d] < 0.0) { mpos[d] = -m[d]; sh += m[d]; }"),
    ("slab volume: offset of the slab with the wrong sign",
     "double a2 = alpha - m[axis] * x0;", "double a2 = alpha + m[axis] * x0;"),
    ("plane area: polygon area without the factor 1/2",
     "area += 0.5 * (cx * n[0] + cy * n[1] + cz * n[2]);", "area += (cx * n[0] + cy * n[1] + cz * n[2]);"),
    ("plane constant: bisection returns the worse end of its bracket",
     "double am = (vh < vl) ? hi : lo;", "double am = (vh < vl) ? lo : hi;"),
    # MYC normal, Sec. 3.2 [Aulisa07]
    ("Youngs: m = +grad c",
     "        m[d] = -g;\n", "        m[d] = g;\n"),
    ("centred columns: transverse slope from the other axis' column pair",
     "double a1 = -(h[2][1] - h[0][1]) * 0.5;", "double a1 = -(h[1][2] - h[1][0]) * 0.5;"),
    ("centred columns: orientation reversed",
     "double sg = (lower >= upper) ? 1.0 : -1.0;", "double sg = (lower >= upper) ? -1.0 : 1.0;"),
    ("MYC: the candidate test reversed",
     "int use_cc = (rule == 0) ? (cmax <= ymax) : (cmax >= ymax);",
     "int use_cc = (rule == 0) ? (cmax >= ymax) : (cmax <= ymax);"),
    ("Youngs: unweighted transverse sums",
     "static const double w[3] = {1.0, 2.0, 1.0};", "static const double w[3] = {1.0, 1.0, 1.0};"),
    # WENO5 face temperature, Sec. 3.4.1 [Shu09]
    ("WENO5: candidate q0 coefficient -7 -> -6",
     "double q0 = (2.0 * vm2 - 7.0 * vm1 + 11.0 * v0) / 6.0;", "double q0 = (2.0 * vm2 - 6.0 * vm1 + 11.0 * v0) / 6.0;"),
    ("WENO5: linear weight 0.6 -> 0.5",
     "double a1 = 0.6 / ((epsw + b1) * (epsw + b1));", "double a1 = 0.5 / ((epsw + b1) * (epsw + b1));"),
    ("WENO5: smoothness indicator of stencil 1 takes stencil 0's slope",
     "double b1 = (13.0 / 12.0) * d1 * d1 + 0.25 * e1 * e1;", "double b1 = (13.0 / 12.0) * d1 * d1 + 0.25 * e0 * e0;"),
    # Weymouth-Yue sweep with tandem energy, Sec. 3.3.1, Eq. disc_et_adv
    ("sweep: donor slab on the wrong side of the donor",
     "double x0 = a > 0.0 ? 1.0 - da : 0.0;\n        double vol = orc_slab_volume(m, al, axis, x0, da);",
     "double x0 = a > 0.0 ? 0.0 : 1.0 - da;\n        double vol = orc_slab_volume(m, al, axis, x0, da);"),
    ("sweep: pure donor fluxes c of the downwind cell",
     "    } else {\n        Fv = cd * a;\n    }\n    /* WENO5 stencil centred on the donor",
     "    } else {\n        Fv = c[cell_id(dims, bc, pos[0], pos[1], pos[2])] * a;\n    }\n"
     "    /* WENO5 stencil centred on the donor"),
    ("sweep: WENO5 stencil ordered downwind to upwind",
     "    /* WENO5 stencil centred on the donor, ordered upwind to downwind */\n    double v[5];\n"
     "    for (int r = -2; r <= 2; ++r) {\n        int q[3] = {don[0], don[1], don[2]};\n"
     "        q[axis] += (a > 0.0) ? r : -r;",
     "    /* WENO5 stencil centred on the donor, ordered upwind to downwind */\n    double v[5];\n"
     "    for (int r = -2; r <= 2; ++r) {\n        int q[3] = {don[0], don[1], don[2]};\n"
     "        q[axis] += (a > 0.0) ? -r : r;"),
    ("sweep: T of the cells as e without the heat capacity",
     "const double *theta, double *Fout,\n                       double *Gout, double *diag) {\n"
     "    long N = (long)dims[0] * dims[1] * dims[2];\n    double lam = dt / par[0];\n"
     "    double *T = (double *)malloc(sizeof(double) * N);\n    double *cn = (double *)malloc(sizeof(double) * N);\n"
     "    double *en = (double *)malloc(sizeof(double) * N);\n    double *clipv = (double *)malloc(sizeof(double) * N);\n"
     "#pragma omp parallel for schedule(static)\n"
     "    for (long id = 0; id < N; ++id) T[id] = e[id] / heat_cap(par, c[id]);",
     "const double *theta, double *Fout,\n                       double *Gout, double *diag) {\n"
     "    long N = (long)dims[0] * dims[1] * dims[2];\n    double lam = dt / par[0];\n"
     "    double *T = (double *)malloc(sizeof(double) * N);\n    double *cn = (double *)malloc(sizeof(double) * N);\n"
     "    double *en = (double *)malloc(sizeof(double) * N);\n    double *clipv = (double *)malloc(sizeof(double) * N);\n"
     "#pragma omp parallel for schedule(static)\n"
     "    for (long id = 0; id < N; ++id) T[id] = e[id];"),
    ("heat capacity: the gas term weighted by c",
     "return par[1] * c + par[2] * (1.0 - c); }", "return par[1] * c + par[2] * c; }"),
    ("frozen state: T^n from the liquid heat capacity",
     "double Tn = e[id] / heat_cap(par, c[id]);", "double Tn = e[id] / par[1];"),
    ("periodic axis: the last face read from its own slot, not from face 0",
     "    if (bc[axis] == 0 && p[axis] == dims[axis]) p[axis] = 0;\n", ""),
    ("sweep: dilatation term c_c (a_r - a_l) dropped",
     "double lf = Fl - ccv * al, rf = Fr - ccv * ar;", "double lf = Fl, rf = Fr;"),
    ("sweep: phase heat capacities swapped in the energy flux G",
     "    *G = (Tf * par[1]) * Fv + (Tf * par[2]) * (a - Fv);\n}\n\n/* Sweep along",
     "    *G = (Tf * par[2]) * Fv + (Tf * par[1]) * (a - Fv);\n}\n\n/* Sweep along"),
    ("frozen state: Theta from C_p(c) instead of C_p(c_c)",
     "theta[id] = heat_cap(par, (double)b) * Tn;", "theta[id] = heat_cap(par, c[id]) * Tn;"),
    ("sweep: clipped volume with the wrong sign",
     "double enew = (e[id] + le) - re;\n                double cc2 = cnew;\n                if (cc2 < 0.0) cc2 = 0.0;\n"
     "                if (cc2 > 1.0) cc2 = 1.0;\n                clipv[id] = cnew - cc2;",
     "double enew = (e[id] + le) - re;\n                double cc2 = cnew;\n                if (cc2 < 0.0) cc2 = 0.0;\n"
     "                if (cc2 > 1.0) cc2 = 1.0;\n                clipv[id] = cc2 - cnew;"),
    # phase-change shift, Sec. 3.3.2 and the energy jump of Sec. 3.4.1
    ("shift: |m|_1 instead of |m|_2 in alpha + |m| dd",
     "double mn2 = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);\n                double sft = mn2 * ddv;",
     "double mn2 = fabs(m[0]) + fabs(m[1]) + fabs(m[2]);\n                double sft = mn2 * ddv;"),
    ("shift: the plane moved against the sign of dd",
     "double sft = mn2 * ddv;", "double sft = -mn2 * ddv;"),
    ("shift: energy jump with the wrong sign",
     "double de = dc * dCp * par[3];", "double de = -dc * dCp * par[3];"),
    ("shift: receivers of the advancing phase instead of the receding one",
     "if ((sft < 0.0) != full) continue;", "if ((sft < 0.0) == full) continue;"),
    ("shift: neighbour's plane extended with the offset's sign flipped",
     "double shiftv = -(mq[0] * (-ox) + mq[1] * (-oy) + mq[2] * (-oz));",
     "double shiftv = (mq[0] * (-ox) + mq[1] * (-oy) + mq[2] * (-oz));"),
    ("unfused energy update: phase heat capacities swapped in G",
     "Gs[side] = (Tf * par[1]) * F + (Tf * par[2]) * (a - F);", "Gs[side] = (Tf * par[2]) * F + (Tf * par[1]) * (a - F);"),
    ("frozen state: c_c = 1 below one half",
     "unsigned char b = c[id] > 0.5 ? 1 : 0;", "unsigned char b = c[id] > 0.5 ? 0 : 1;"),
    ("zero-gradient boundary: the ghost copies the far end of the line",
     "    if (i < 0) return 0;\n    if (i >= n) return n - 1;", "    if (i < 0) return n - 1;\n    if (i >= n) return 0;"),
    # mass transfer rate from PLIC distances, Sec. 3.2
    ("mass transfer: normal gradient with the wrong sign",
     "double g = c[id] > 0.5 ? (Tg - T) / dist : (T - Tg) / dist;",
     "double g = c[id] > 0.5 ? (T - Tg) / dist : (Tg - T) / dist;"),
    ("mass transfer: Delta x from the node to the mixed cell",
     "double X[3] = {0.5 - dx, 0.5 - dy, 0.5 - dz};", "double X[3] = {0.5 + dx, 0.5 + dy, 0.5 + dz};"),
    ("mass transfer: node distance with the plane's offset added",
     "bs = dpl[q] - ndx;", "bs = dpl[q] + ndx;"),
    ("mass transfer: neighbours' phases swapped in the averages",
     "int ph = c[q] > 0.5 ? 1 : 0;", "int ph = c[q] > 0.5 ? 0 : 1;"),
    ("mass transfer: conductivities of the two phases transposed",
     "mdot[id] = (k_g * gg - k_l * gl) / h_fg;", "mdot[id] = (k_l * gg - k_g * gl) / h_fg;"),
    ("mass transfer: weights gamma without the 1 / |Delta x|^2",
     "double gam = xi / (double)(dx * dx + dy * dy + dz * dz);", "double gam = xi;"),
    # Li's Lagrangian-explicit sweep (Sec. 3.3.1, reading A19)
    ("Lagrangian explicit: stretch 1 + (a_l - a_r)",
     "return 1.0 + (ar - al);  /* exactly 1 where the velocity is uniform */",
     "return 1.0 + (al - ar);  /* exactly 1 where the velocity is uniform */"),
    ("Lagrangian explicit: dilatation term of the cell's own c dropped",
     "double cnew = (cv + (Fl - cv * al)) - (Fr - cv * ar);", "double cnew = (cv + Fl) - Fr;"),
    ("Lagrangian explicit: Theta from the liquid heat capacity only",
     "double th = (T[id] * par[1]) * cv + (T[id] * par[2]) * (1.0 - cv);", "double th = T[id] * par[1];"),
    ("Lagrangian explicit: preimage width |a| J instead of |a| / J",
     "double w = (J > da) ? da / J : 1.0;", "double w = (J > da) ? da * J : 1.0;"),
]

# the oracle's own compile line (oracle/__init__.py, build())
CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-fopenmp", "-std=c99"]

CHILD = r"""
import os, sys
root, lib = sys.argv[1], sys.argv[2]
sys.path.insert(0, root)
os.chdir(root)
import oracle
oracle._LIB_PATH = lib
oracle.build = lambda force=False: lib
import pytest
args = sys.argv[3:]
sys.exit(pytest.main(args))
"""


def _compile(src_text: str, work: str, tag: str) -> str:
    src = os.path.join(work, f"{tag}.c")
    lib = os.path.join(work, f"lib{tag}.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", *CFLAGS, "-o", lib, src, "-lm"], check=True, capture_output=True)
    return lib


def _run_pins(lib: str) -> tuple[int, str]:
    args = [*PINS, "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    for s in SKIP:
        args += ["--deselect", s]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, lib, *args], capture_output=True, text=True,
                       env=env, timeout=600)
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-3:])
    return r.returncode, tail


def _source() -> str:
    with open(SRC) as f:
        return f.read()


def test_mutant_texts_occur_once():
    src = _source()
    names = [m[0] for m in MUTANTS]
    assert len(set(names)) == len(names)
    for name, old, new in MUTANTS:
        assert src.count(old) == 1, name
        assert old != new, name


def test_pins_reject_every_mutant(tmp_path):
    src = _source()
    workers = max(1, min(8, os.cpu_count() or 1))
    work = str(tmp_path)
    jobs = [("unchanged", src)] + [(name, src.replace(old, new)) for name, old, new in MUTANTS]

    def compile_and_run(i):
        return _run_pins(_compile(jobs[i][1], work, f"m{i}"))

    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        res = dict(zip([name for name, _ in jobs], ex.map(compile_and_run, range(len(jobs)))))
    rc, tail = res.pop("unchanged")
    assert rc == 0, f"the unchanged oracle fails its own pins under this harness:\n{tail}"
    # pytest exit code 1: tests ran and at least one failed; anything else
    # (an import error, a crash) is a harness failure, not a caught mutant
    survivors = [n for n, (rc, _) in res.items() if rc == 0]
    broken = {n: t for n, (rc, t) in res.items() if rc not in (0, 1)}
    assert not broken, f"harness failures: {broken}"
    assert not survivors, f"mutants no pin rejects: {survivors}"


# (module, name, text in oracle/<module>.py, replacement)
PY_PINS = {
    "mlp": ["tests/test_oracle_mlp.py"],
    "diffusion": ["tests/test_oracle_diffusion.py"],
    "extension": ["tests/test_oracle_extension.py"],
}
PY_MUTANTS = [
    # learned normal (the network, its gradient, Adam, BF16, the fallback)
    ("mlp", "GELU with erf(x / 2)",
     "return 0.5 * x * (1.0 + erf(x / math.sqrt(2.0)))", "return 0.5 * x * (1.0 + erf(x / 2.0))"),
    ("mlp", "GELU derivative: density term without its 1/sqrt(2)",
     "x * np.exp(-0.5 * x * x) / math.sqrt(2.0 * math.pi)", "x * np.exp(-0.5 * x * x) / math.sqrt(math.pi)"),
    ("mlp", "gradient of W3 from the first hidden layer",
     'g["W3"] = g_y.T @ a2', 'g["W3"] = g_y.T @ a1'),
    ("mlp", "gradient through the unit normalisation without its projection",
     "g_y = (g_yh - yh * np.sum(g_yh * yh, axis=1, keepdims=True)) / ny", "g_y = g_yh / ny"),
    ("mlp", "Adam without the first moment's bias correction",
     "mh = mom[k] / (1 - beta1 ** t)", "mh = mom[k]"),
    ("mlp", "BF16 ties rounded down instead of to even",
     "lsb = (bits >> 16) & 1", "lsb = 0 * bits"),
    ("mlp", "second layer takes the first layer's bias",
     'z2 = a1 @ weights(p["W2"]).T + p["b2"]', 'z2 = a1 @ weights(p["W2"]).T + p["b1"]'),
    ("mlp", "plane residual: neighbour offsets with the wrong sign",
     "r.append(volume(mm, al - mm @ o) - s[k])", "r.append(volume(mm, al + mm @ o) - s[k])"),
    ("mlp", "ellipsoid nearest point with a2 - t",
     "    return a2 * y / (a2 + t)", "    return a2 * y / (a2 - t)"),
    ("mlp", "plane stencil: cell corner at o + 1/2",
     "a = (d - n @ (o - 0.5)) / l1", "a = (d - n @ (o + 0.5)) / l1"),
    # interface-Dirichlet diffusion (Sec. 3.4.2)
    ("diffusion", "height function: interface at H - 3",
     "theta = (H - 3.5) if liquid_p else (3.5 - H)", "theta = (H - 3.0) if liquid_p else (3.0 - H)"),
    ("diffusion", "plane distance with the node's offset added",
     "t = (al[M] - mm @ x0) / ma", "t = (al[M] + mm @ x0) / ma"),
    ("diffusion", "second difference over one side's distance",
     "denom = 0.5 * (dists[-1] + dists[1])", "denom = dists[1]"),
    ("diffusion", "heated wall a whole cell away",
     "terms[s] = (2.0 / h, None, 0.0, Tw * 2.0 / h)", "terms[s] = (1.0 / h, None, 0.0, Tw * 1.0 / h)"),
    ("diffusion", "phase-wise energy replaced by the mixture's",
     "        return e + Cd * (T1 - T0)", "        return Cd * T1"),
    ("diffusion", "conductivities of the phases swapped",
     "kp = k_l if liquid_p else k_g", "kp = k_g if liquid_p else k_l"),
    # velocity extension (Sec. 3.3.1)
    ("extension", "face density from one cell only",
     "cf = 0.5 * (c[P] + c[Q])", "cf = c[P]"),
    ("extension", "source with the density jump reversed",
     "(1.0 / rho_g - 1.0 / rho_l)", "(1.0 / rho_l - 1.0 / rho_g)"),
    ("extension", "face correction along +grad p",
     "val = -(dt / rho_f(L, R)) * (p[R] - p[L]) / h", "val = -(dt / rho_f(L, R)) * (p[L] - p[R]) / h"),
    ("extension", "one gas layer instead of two",
     "    for L in (1, 2):\n        new = []", "    for L in (1,):\n        new = []"),
    ("extension", "liquid neighbours coupled instead of no-slip",
     "if Q is None or liquid[Q]:", "if Q is None:"),
    ("extension", "couplings over h instead of h^2",
     "beta = dt / rho_f(P, Q) / (h * h)", "beta = dt / rho_f(P, Q) / h"),
]

PY_CHILD = r"""
import importlib.util, os, sys
root, name, path = sys.argv[1], sys.argv[2], sys.argv[3]
sys.path.insert(0, root)
os.chdir(root)
import oracle
spec = importlib.util.spec_from_file_location("oracle." + name, path)
mod = importlib.util.module_from_spec(spec)
sys.modules["oracle." + name] = mod
spec.loader.exec_module(mod)
setattr(oracle, name, mod)
import pytest
sys.exit(pytest.main(sys.argv[4:]))
"""


def _py_source(name: str) -> str:
    with open(os.path.join(ROOT, "oracle", name + ".py")) as f:
        return f.read()


def _run_py_pins(job) -> tuple[int, str]:
    name, path = job
    args = [*PY_PINS[name], "-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", PY_CHILD, ROOT, name, path, *args], capture_output=True, text=True,
                       env=env, timeout=600)
    tail = "\n".join((r.stdout + r.stderr).strip().splitlines()[-3:])
    return r.returncode, tail


def test_py_mutant_texts_occur_once():
    names = [(m[0], m[1]) for m in PY_MUTANTS]
    assert len(set(names)) == len(names)
    for name, label, old, new in PY_MUTANTS:
        assert _py_source(name).count(old) == 1, label
        assert old != new, label


def test_pins_reject_every_numpy_oracle_mutant(tmp_path):
    workers = max(1, min(8, os.cpu_count() or 1))
    work = str(tmp_path)
    jobs = {}
    for name in PY_PINS:  # the unchanged modules, loaded the same way
        path = os.path.join(work, f"unchanged_{name}.py")
        with open(path, "w") as f:
            f.write(_py_source(name))
        jobs[("unchanged", name)] = (name, path)
    for i, (name, label, old, new) in enumerate(PY_MUTANTS):
        path = os.path.join(work, f"m{i}_{name}.py")
        with open(path, "w") as f:
            f.write(_py_source(name).replace(old, new))
        jobs[(label, name)] = (name, path)
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        res = dict(zip(jobs, ex.map(_run_py_pins, jobs.values())))
    for name in PY_PINS:
        rc, tail = res.pop(("unchanged", name))
        assert rc == 0, f"the unchanged oracle/{name}.py fails its own pins under this harness:\n{tail}"
    survivors = [k for k, (rc, _) in res.items() if rc == 0]
    broken = {k: t for k, (rc, t) in res.items() if rc not in (0, 1)}
    assert not broken, f"harness failures: {broken}"
    assert not survivors, f"mutants no pin rejects: {survivors}"
