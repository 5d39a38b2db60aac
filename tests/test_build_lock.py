"""build() from several processes at once (the ranks of a multi-process launch each call it): one
compiles, the others wait for it and find the stamp up to date, and the library they return loads.
Runs one full build of the library on the CPU (nvcc cross-compiles)."""
import ctypes
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import paper_2309_00651_gb300.build as b
calls = [0]
run = b.subprocess.run
def counting_run(*a, **k):
    calls[0] += 1
    return run(*a, **k)
b.subprocess.run = counting_run
lib = b.build()
print(calls[0], lib)
"""


def test_concurrent_builds_compile_once():
    from paper_2309_00651_gb300 import build as B
    B.build()
    stamp = os.path.join(B.BUILD, "stamp")
    os.remove(stamp)  # the next build() has to compile
    code = CHILD.format(root=ROOT)
    procs = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True)
             for _ in range(3)]
    outs = [p.communicate(timeout=1200) for p in procs]
    for p, (out, err) in zip(procs, outs):
        assert p.returncode == 0, err[-2000:]
    results = [out.split() for out, _ in outs]
    calls = sorted(int(r[0]) for r in results)
    assert calls[0] == 0 and calls[1] == 0          # two waited and found the stamp up to date
    assert calls[2] == len(B.SOURCES) + 1           # one compiled every unit and linked once
    assert all(r[1] == B.LIB for r in results)
    assert os.path.exists(stamp)
    lib = ctypes.CDLL(B.LIB)
    assert hasattr(lib, "hfx_create") and hasattr(lib, "hfx_test_live_allocations")
