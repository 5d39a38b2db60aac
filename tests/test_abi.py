"""The C-ABI library builds, loads, exports every symbol include/*.h declare, and rejects
bad arguments on the host before touching a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2309_00651_gb300 import build, hfx
    build.build()
    return hfx.load_library()


def declared_symbols():
    text = ""
    inc = os.path.join(ROOT, "include")
    for name in sorted(os.listdir(inc)):
        if name.endswith(".h"):
            with open(os.path.join(inc, name)) as f:
                text += f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hfx_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for n in ("hfx_create", "hfx_apply", "hfx_apply_batched", "hfx_set_workspace", "hfx_workspace_bytes",
              "hfx_sync_status", "hfx_last_error", "hfx_destroy", "hfx_ace_workspace_bytes", "hfx_ace_build",
              "hfx_ace_apply", "hfx_screen_pairs"):
        assert n in names


def test_every_declaration_cites_its_passage_or_says_it_has_none():
    """The comment in front of every entry point names the passage of the paper it computes
    (Sec., Eq., the appendix) or states that the paper has no counterpart (plumbing, measurement,
    testing hooks)."""
    inc = os.path.join(ROOT, "include")
    found = 0
    for name in sorted(os.listdir(inc)):
        if not name.endswith(".h"):
            continue
        with open(os.path.join(inc, name)) as f:
            text = f.read()
        for m in re.finditer(r"(/\*(?:(?!\*/).)*\*/)\s*((?:[a-z_0-9]+\s+\**)+?(hfx_[a-z_0-9]+)\s*\()", text, flags=re.S):
            found += 1
            comment = re.sub(r"\s*\n\s*\*\s*", " ", m.group(1))  # one line, without the leading stars
            assert re.search(r"Sec\.|Eq\.|appendix|no counterpart", comment), f"{name}: {m.group(3)}"
    assert found >= len(declared_symbols()) - 4  # (a few share one comment: profile_enable/read, ...)


def test_library_exports_every_declared_symbol(lib):
    from paper_2309_00651_gb300 import hfx
    for name in declared_symbols():
        assert hasattr(lib, name), f"{name} not exported"
    assert set(declared_symbols()) <= set(hfx.EXPORTED)


def test_host_side_argument_errors(lib):
    from paper_2309_00651_gb300 import hfx
    box = hfx.HfxBox()
    for a in range(3):
        box.lattice[a][a] = 10.0
    out = ctypes.c_void_p()
    g = (ctypes.c_int32 * 3)(32, 32, 32)
    # NULL out
    assert lib.hfx_create(ctypes.byref(box), g, 20.0, 0, 0.25, 1, None) == -1
    # a grid edge with a prime factor 7
    bad = (ctypes.c_int32 * 3)(28, 32, 32)
    assert lib.hfx_create(ctypes.byref(box), bad, 20.0, 0, 0.25, 1, ctypes.byref(out)) == -2
    assert "grid edge" in lib.hfx_last_error().decode()
    assert not out.value
    # odd edge
    odd = (ctypes.c_int32 * 3)(15, 32, 32)
    assert lib.hfx_create(ctypes.byref(box), odd, 20.0, 0, 0.25, 1, ctypes.byref(out)) == -2
    # unknown precision / kernel
    assert lib.hfx_create(ctypes.byref(box), g, 20.0, 0, 0.25, 7, ctypes.byref(out)) == -1
    assert lib.hfx_create(ctypes.byref(box), g, 20.0, 9, 0.25, 1, ctypes.byref(out)) == -1
    # sphere kernel without a cutoff
    assert lib.hfx_create(ctypes.byref(box), g, 0.0, 1, 0.25, 1, ctypes.byref(out)) == -1
    # degenerate cell
    flat = hfx.HfxBox()
    assert lib.hfx_create(ctypes.byref(flat), g, 20.0, 0, 0.25, 1, ctypes.byref(out)) == -1
    # NULL contexts
    assert lib.hfx_workspace_bytes(None, 16, 136) == 0
    assert lib.hfx_apply(None, None, 16, None, 0, 0, None, None, None) == -1
    assert lib.hfx_sync_status(None, None) == -1
    assert lib.hfx_set_workspace(None, None, 0) == -1
    assert lib.hfx_ace_workspace_bytes(None, 16, 0) == 0
    assert lib.hfx_ace_build(None, None, None, 16, None, None, None, None, 0, None) == -1
    assert lib.hfx_ace_apply(None, None, 16, None, 4, 0, None, None, 0, None) == -1
    assert lib.hfx_screen_pairs(None, None, 16, 1e-6, None, None, None, None, 0, None) == -1
    assert lib.hfx_scdm_workspace_bytes(None, 16) == 0
    assert lib.hfx_scdm_localise(None, None, 16, None, None, None, None, 0, None) == -1
    sp = hfx.HfxSinrParams(0.001, 1.0, 1.0, 0.01, 4)
    assert lib.hfx_sinr_update_n(None, 10, 1.0, 1, 1, None, None, None, None, None) == -1
    assert lib.hfx_sinr_update_n(ctypes.byref(sp), 10, 1.0, 1, 2, None, None, None, None, None) == -1  # n_sy
    assert lib.hfx_sinr_update_n(ctypes.byref(sp), 10, 1.0, 1, 1, None, None, None, None, None) == -1  # NULL arrays
    bad = hfx.HfxSinrParams(0.001, 1.0, 1.0, 0.01, 17)
    assert lib.hfx_sinr_update_v(ctypes.byref(bad), 10, 1.0, None, None, None, None, None, None) == -1  # L
    nog = hfx.HfxSinrParams(0.001, 1.0, 1.0, 0.0, 4)
    assert lib.hfx_sinr_update_x(ctypes.byref(nog), 10, 1.0, None, None, None, None, None) == -1  # gamma
    assert lib.hfx_sinr_update_x(ctypes.byref(sp), 0, 1.0, None, None, None, None, None) == 0  # nothing to do
    lib.hfx_destroy(None)


def test_failure_injection_hook_on_the_host(lib):
    """hfx_test_fail_allocation / hfx_test_live_allocations work without a GPU: argument errors are
    found before any allocation, so a pending failure stays pending and nothing is held."""
    from paper_2309_00651_gb300 import hfx
    live0 = hfx.hfx_test_live_allocations()
    assert live0 >= 0
    box = hfx.HfxBox()
    for a in range(3):
        box.lattice[a][a] = 10.0
    out = ctypes.c_void_p()
    odd = (ctypes.c_int32 * 3)(15, 32, 32)
    hfx.hfx_test_fail_allocation(0)
    try:
        assert lib.hfx_create(ctypes.byref(box), odd, 20.0, 0, 0.25, 1, ctypes.byref(out)) == -2
        assert not out.value
        assert hfx.hfx_test_live_allocations() == live0
    finally:
        hfx.hfx_test_fail_allocation(-1)


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2309_00651_gb300 import hfx
    saved = hfx._lib
    try:
        hfx._lib = None
        with pytest.raises(RuntimeError, match="libhfx.so not found"):
            hfx.load_library(str(tmp_path / "missing.so"))
    finally:
        hfx._lib = saved
