"""Source check of the programmatic-dependent launch chain (no GPU).

A kernel launched with programmatic stream serialisation may start while the
kernel ahead of it in the stream is still running; it is correct only if it
waits for its dependencies (griddepcontrol.wait, in pdl_begin()) before it
touches memory.  This test finds every kernel launched through launch_pdl (or
with the attribute set by hand) and checks that its body begins with
pdl_begin().
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                    "paper_2509_21754_gb300", "csrc")


def sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = fh.read()
    return out


def kernel_body_start(src: str, name: str):
    """First statement of the __global__ definition of `name`, or None."""
    for m in re.finditer(r"__global__[^;{]*?\b" + re.escape(name) + r"\s*\(", src):
        i, depth = m.end() - 1, 0
        while True:
            c = src[i]
            if c == "(":
                depth += 1
            elif c == ")":
                depth -= 1
                if depth == 0:
                    break
            i += 1
        j = i + 1
        while src[j] in " \n":
            j += 1
        if src[j] == "{":
            return src[j + 1:].lstrip().split("\n", 1)[0].strip()
    return None


def pdl_kernels(srcs):
    names = set()
    for text in srcs.values():
        for m in re.finditer(r"launch_pdl\(\s*([A-Za-z_]\w*)", text):
            names.add(m.group(1))
        # hand-built configurations that allow programmatic serialisation
        for m in re.finditer(r"cudaLaunchAttributeProgrammaticStreamSerialization", text):
            tail = text[m.end():m.end() + 2000]
            k = re.search(r"cudaLaunchKernelEx\(&cfg,\s*([A-Za-z_]\w*)", tail)
            if k:
                names.add(k.group(1))
    names -= {"k", "void"}   # the helper's own definition
    return names


def test_every_programmatic_dependent_kernel_waits_first():
    srcs = sources()
    names = pdl_kernels(srcs)
    assert {"k_split_pass", "k_blk_cc", "k_emit_rows", "k_medmad_cluster"} <= names
    for n in sorted(names):
        firsts = [kernel_body_start(t, n) for t in srcs.values()]
        firsts = [f for f in firsts if f is not None]
        assert firsts, f"kernel {n} not found"
        for f in firsts:
            assert f == "pdl_begin();", f"{n} starts with {f!r}, not pdl_begin()"


def test_pdl_begin_only_waits():
    """No kernel lets its dependents start early: their parked CTAs would hold
    SM resources that the other stream of a detect needs."""
    for f, text in sources().items():
        assert "griddepcontrol.launch_dependents" not in text, f
