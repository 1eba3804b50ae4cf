"""Every kernel launched with programmatic dependent launch waits first.

launch_pdl (csrc/vof_launch.h) lets a kernel be scheduled before the kernel
ahead of it on the stream has completed; what keeps the order is the
griddepcontrol.wait that the kernel itself executes (pdl_wait()).  A kernel
launched this way without that wait as its first statement would read its
inputs while the previous kernel may still write them -- a race the parity
tests need not catch.  This CPU test reads the CUDA sources and checks, for
every kernel passed to launch_pdl, that the body of its __global__ wrapper
starts with pdl_wait() (after __shared__ declarations only), and that
pdl_wait() appears nowhere but at such a start.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2001_03477_gb300", "csrc")


def sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh", ".h")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = re.sub(r"//[^\n]*", "", fh.read())  # comments out
    return out


def launched_with_pdl(srcs):
    names = set()
    for text in srcs.values():
        for m in re.finditer(r"\blaunch_pdl\(\s*([A-Za-z_]\w*)", text):
            names.add(m.group(1))
    names.discard("void")  # the helper's own declaration
    return names


def kernel_bodies(srcs, name):
    """Bodies of the __global__ definitions of `name` (text between its braces)."""
    bodies = []
    for text in srcs.values():
        for m in re.finditer(r"__global__\s+void\s+(?:__launch_bounds__\([^)]*\)\s*)?" + name + r"\s*\(", text):
            # skip the parameter list, then take the balanced braces
            i, depth = m.end(), 1
            while depth:
                depth += {"(": 1, ")": -1}.get(text[i], 0)
                i += 1
            j = text.index("{", i)
            assert text[i:j].strip() == "", f"{name}: unexpected text before the body"
            k, depth = j + 1, 1
            while depth:
                depth += {"{": 1, "}": -1}.get(text[k], 0)
                k += 1
            bodies.append(text[j + 1:k - 1])
    return bodies


def first_statement(body):
    for st in body.split(";"):
        st = st.strip()
        if st and not st.startswith("__shared__"):
            return st
    return ""


def test_every_pdl_kernel_waits_first():
    srcs = sources()
    names = launched_with_pdl(srcs)
    # the step's kernels: tile pass, quiet pass, four per sweep, five of the
    # shift, the fused reduction
    for k in ("k_tiles", "k_quiet", "k_stream_row", "k_stream_col", "k_prep", "k_faces", "k_update",
              "k_shift_stream", "k_shift_planes", "k_shift_own", "k_shift_receivers", "k_shift_sums",
              "k_reduce_fused"):
        assert k in names, k
    for name in sorted(names):
        bodies = kernel_bodies(srcs, name)
        assert bodies, f"no __global__ definition of {name}"
        for b in bodies:
            assert first_statement(b) == "pdl_wait()", f"{name} does not start with pdl_wait()"


def test_pdl_wait_only_at_kernel_starts():
    srcs = sources()
    names = launched_with_pdl(srcs)
    calls = sum(len(re.findall(r"\bpdl_wait\(\)\s*;", t)) for t in srcs.values())
    starts = sum(len(kernel_bodies(srcs, n)) for n in names)
    assert calls == starts
