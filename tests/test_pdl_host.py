"""Source checks of the programmatic dependent launches (no GPU).

A kernel enqueued with launch_dependent() may start while the kernel before
it in the stream is still running; it is correct only if it waits
(grid_dep_wait) before it touches global memory, and the ordering of later
kernels relies on every such kernel doing so.  These tests read the CUDA
sources: every kernel launched that way must call grid_dep_wait() before any
statement other than shared-memory declarations and thread-index
arithmetic, and no launch_dependent() may directly follow a memset or copy
in its enqueue function.
"""
import os
import re

import pytest

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1802_02619_gb300", "csrc")


def _sources():
    out = {}
    for f in sorted(os.listdir(CSRC)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(CSRC, f)) as fh:
                out[f] = fh.read()
    return out


def _dependent_kernels(srcs):
    names = set()
    for text in srcs.values():
        # call sites only (the kernels are named k_*; the helper's own
        # definition takes a function-pointer parameter)
        for m in re.finditer(r"launch_dependent\(\s*(k_\w*)", text):
            names.add(m.group(1))
    return sorted(names)


def _kernel_body(srcs, name):
    """Body of the __global__ function `name` (the first definition)."""
    pat = re.compile(r"__global__\s+void[^;{]*?\b" + re.escape(name) + r"\s*\(")
    for text in srcs.values():
        m = pat.search(text)
        if not m:
            continue
        i = text.index("{", text.index(")", m.end()))
        depth = 0
        for k in range(i, len(text)):
            if text[k] == "{":
                depth += 1
            elif text[k] == "}":
                depth -= 1
                if depth == 0:
                    return text[i + 1:k]
    raise AssertionError("kernel %s not found" % name)


# statements allowed before the wait: shared-memory declarations, aliases
# into dynamic shared memory, thread/lane/warp indices, type aliases
_ALLOWED = [
    r"(extern\s+)?__shared__\b.*",
    r"\w+\s*&\s*\w+\s*=\s*(\*\s*)?reinterpret_cast<\w+\s*\*>\(smem_raw\)(\[\w+\])?",
    r"const\s+int\s+(lane|warp|tid)\s*=\s*threadIdx\.x[^;]*(,\s*\w+\s*=\s*threadIdx\.x[^;]*)?",
    r"using\s+\w+\s*=.*",
]


def test_some_kernels_are_dependent_launches():
    names = _dependent_kernels(_sources())
    assert {"k_rows", "k_radix_scatter", "k_radix_local", "k_work_scan"} <= set(names), names


@pytest.mark.parametrize("name", _dependent_kernels(_sources()))
def test_dependent_kernel_waits_first(name):
    body = _kernel_body(_sources(), name)
    assert "grid_dep_wait();" in body, name
    head = body[:body.index("grid_dep_wait();")]
    head = re.sub(r"//[^\n]*", "", head)
    for stmt in (x.strip() for x in head.split(";")):
        if not stmt:
            continue
        assert any(re.fullmatch(p, stmt, re.S) for p in _ALLOWED), \
            "%s: statement before grid_dep_wait(): %r" % (name, stmt)


def test_no_dependent_launch_right_after_a_memory_operation():
    for f, text in _sources().items():
        for m in re.finditer(r"launch_dependent\(\s*k_", text):
            # from the previous launch statement (or the end of the previous
            # function) to the one holding this call: no memset or copy
            here = text.rfind("LCO_LAUNCH(", 0, m.start())
            start = max(text.rfind("LCO_LAUNCH(", 0, here), text.rfind("\n}\n", 0, here))
            between = text[start:here]
            assert not re.search(r"cudaMemsetAsync|cudaMemcpyAsync|cudaMemcpy2DAsync", between), \
                "%s: a dependent launch follows a memory operation:\n%s" % (f, between[-400:])
