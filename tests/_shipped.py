"""Access to the shipped kernel headers from CPU tests: compiles the host
harness (tests/host_harness.cu) against the package's csrc headers with the
host compiler pass of nvcc, and reads integer constants out of the headers,
so the model tests check the code the kernels are built from."""
from __future__ import annotations

import os
import re
import shutil
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1905_00473_gb300", "csrc")
_harness = None


def header_constant(header: str, name: str) -> int:
    """Value of `constexpr int <name> = <integer>;` in csrc/<header>."""
    text = open(os.path.join(CSRC, header)).read()
    m = re.search(r"constexpr\s+int\s+" + re.escape(name) + r"\s*=\s*(\d+)\s*;", text)
    if m is None:
        raise LookupError(f"{name} not found in {header}")
    return int(m.group(1))


def harness() -> str:
    """Path of the compiled host harness (built once per process)."""
    global _harness
    if _harness is None:
        nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
        out = os.path.join(tempfile.mkdtemp(prefix="pr_harness_"), "host_harness")
        subprocess.run([nvcc, "-std=c++17", "-O1", "-diag-suppress", "550", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), "-o", out,
                        os.path.join(ROOT, "tests", "host_harness.cu")],
                       check=True, capture_output=True)
        _harness = out
    return _harness


def balanced_rows(queries):
    """tb::balanced_row(rows_total, n, K, b, G) of tb_common.cuh for each
    query tuple, evaluated by the compiled harness."""
    text = "".join(f"{r} {n} {k} {b} {g}\n" for r, n, k, b, g in queries)
    res = subprocess.run([harness()], input=text, capture_output=True, text=True, check=True)
    vals = [int(x) for x in res.stdout.split()]
    assert len(vals) == len(queries)
    return vals


def queue_plan(instances):
    """qplan::build of queue_plan.h for instances [(n, slices, m)], evaluated
    by the compiled harness: (counters, passes, items, units), passes as tuples
    (inst, k, cls, g0, levels, strips) and items as (pass, vslice, dep, need)
    in queue order, and units (first, count) as the CTAs claim them;
    counters is -1 if the plan was refused."""
    text = "".join(f"{n} {s} {m}\n" for n, s, m in instances)
    res = subprocess.run([harness(), "plan"], input=text, capture_output=True, text=True, check=True)
    ndep, passes, items, units = None, [], [], []
    for line in res.stdout.splitlines():
        tag, *vals = line.split()
        vals = [int(v) for v in vals]
        if tag == "D":
            ndep = vals[0]
        elif tag == "P":
            passes.append(tuple(vals))
        elif tag == "I":
            items.append(tuple(vals))
        elif tag == "U":
            units.append(tuple(vals))
    return ndep, passes, items, units
