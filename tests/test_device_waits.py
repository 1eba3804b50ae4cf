"""Every wait in the CUDA sources is bounded, and nothing traps.

A kernel that spins on a condition another agent must make true (an
mbarrier phase the tensor core completes, a grid-barrier generation the last
CTA advances) must give up after a time limit, record a status bit the host
reads, and return, so that a fault elsewhere cannot hang the GPU.  A kernel
must also never end the context on purpose (trap, a failing device assert).
This CPU test reads the library's sources and checks:
  * every mbarrier try_wait / test_wait sits in mbar_wait, whose loop
    returns false once the global timer has run one second past its start;
  * every spin on the cooperative solver's barrier generation checks
    ext_now_ns() against a limit inside the loop;
  * no trap instruction, __trap() or device assert() appears.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2001_03477_gb300", "csrc")


def sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = re.sub(r"//[^\n]*", "", fh.read())
    return out


def body_of(text, start):
    """Balanced-brace body starting at the first '{' at or after start."""
    j = text.index("{", start)
    k, depth = j + 1, 1
    while depth:
        depth += {"{": 1, "}": -1}.get(text[k], 0)
        k += 1
    return text[j + 1:k - 1]


def test_mbarrier_waits_are_bounded():
    srcs = sources()
    uses = [(f, m.start()) for f, t in srcs.items() for m in re.finditer(r"mbarrier\.(try_wait|test_wait)", t)]
    assert uses, "expected the tensor-core kernels' mbarrier waits"
    for f, pos in uses:
        t = srcs[f]
        fn = t.rfind("bool mbar_wait(", 0, pos)
        assert fn >= 0, f"{f}: an mbarrier wait outside mbar_wait"
        body = body_of(t, fn)
        assert t.index("{", fn) < pos < t.index("{", fn) + len(body) + 2, f"{f}: wait not inside mbar_wait's body"
        assert re.search(r"gtimer\(\)\s*-\s*t0\s*>\s*1000000000ull\)\s*return false", body), f
    # and every caller looks at the result
    for f, t in srcs.items():
        for m in re.finditer(r"\bmbar_wait\(", t):
            line_start = t.rfind("\n", 0, m.start()) + 1
            line = t[line_start:t.index("\n", m.start())]
            if "bool mbar_wait(" in line:
                continue
            assert re.search(r"(if\s*\(!?|=|&&|\|\||return)\s*[^;]*mbar_wait\(", line), f"{f}: result ignored: {line}"


def test_grid_barrier_spins_are_bounded():
    srcs = sources()
    spins = [(f, m) for f, t in srcs.items() for m in re.finditer(r"while\s*\(\s*\*\s*vgen\s*==", t)]
    assert spins, "expected the cooperative solver's grid barrier"
    for f, m in spins:
        body = body_of(srcs[f], m.end())
        assert re.search(r"ext_now_ns\(\)\s*-\s*t0\s*>", body) and "break" in body, f


def test_nothing_traps():
    for f, t in sources().items():
        assert "__trap" not in t, f
        assert not re.search(r"\btrap\s*;", t), f
        assert not re.search(r"(?<![_\w])assert\s*\(", t), f
