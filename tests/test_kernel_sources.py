"""Source-level invariants of the CUDA kernels (no GPU).

The recorded solver graph links consecutive kernel nodes programmatically,
so a kernel may start before its predecessor has finished; every kernel
must therefore wait for its predecessors (pdl_entry) before it reads or
writes anything.  A kernel added without that wait would race its
predecessor whenever the graph holds it, so every kernel definition in the
library is checked here.
"""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_1610_10053_gb300", "csrc")


def kernel_bodies():
    out = []
    for name in sorted(os.listdir(CSRC)):
        if not name.endswith((".cu", ".cuh")):
            continue
        src = open(os.path.join(CSRC, name)).read()
        for m in re.finditer(r"__global__", src):
            k = re.compile(r"\bk_[A-Za-z0-9_]+\s*\(").search(src, m.end())
            depth, i = 0, k.end() - 1
            while True:
                if src[i] == "(":
                    depth += 1
                elif src[i] == ")":
                    depth -= 1
                    if depth == 0:
                        break
                i += 1
            brace, semi = src.find("{", i), src.find(";", i)
            if semi != -1 and semi < brace:
                continue  # a declaration
            body = src[brace + 1:brace + 400]
            out.append((name, k.group(0).rstrip("( "), body))
    return out


def test_every_kernel_waits_for_its_predecessors_first():
    kernels = kernel_bodies()
    assert len(kernels) >= 60
    for name, kern, body in kernels:
        first = body.strip().split(";")[0].strip()
        assert first == "pdl_entry()", (name, kern, first)


def test_no_early_launch_trigger():
    """Letting dependents launch from a kernel's start parked their blocks on
    the SMs and measured slower; no kernel triggers them early."""
    for name in os.listdir(CSRC):
        if name.endswith((".cu", ".cuh", ".h")):
            src = open(os.path.join(CSRC, name)).read()
            assert "launch_dependents" not in src, name
            assert "cudaTriggerProgrammaticLaunchCompletion" not in src, name
