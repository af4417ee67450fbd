"""CPU-only checks of the C ABI: the library builds and loads, exports every function that
include/art.h declares, the ctypes structures match the C layout, and argument checks that
need no GPU return ART_EINVAL."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1711_06277_gb300 import _lib as C

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "art.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(art_[a-z_]+)\s*\(", text)))


def test_exports_every_declared_symbol():
    lib = C.lib()
    names = _declared()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(C.EXPORTED) == names


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "art.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu\n", sizeof(art_params), offsetof(art_params, rot),
         offsetof(art_params, queue_capacity), sizeof(art_stats),
         offsetof(art_stats, L_in), offsetof(art_stats, status));
  return 0;
}''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = list(map(int, subprocess.check_output([str(exe)]).split()))
    want = [ctypes.sizeof(C.ArtParams), C.ArtParams.rot.offset, C.ArtParams.queue_capacity.offset,
            ctypes.sizeof(C.ArtStats), C.ArtStats.L_in.offset, C.ArtStats.status.offset]
    assert got == want


def test_params_default():
    p = C.ArtParams()
    C.lib().art_params_default(ctypes.byref(p))
    assert (p.level0, p.level_max, p.m_ray, p.tau_max) == (4, -1, 4.0, 7.0)
    assert list(p.rot) == [1, 0, 0, 0, 1, 0, 0, 0, 1]
    assert p.schedule == C.ART_SCHED_PERSISTENT


def test_strerror_names_every_status():
    seen = set()
    for s in range(0, -8, -1):
        msg = C.strerror(s)
        assert msg and msg != "unknown status"
        seen.add(msg)
    assert len(seen) == 8
    assert C.strerror(-99) == "unknown status"


def test_invalid_arguments_without_gpu():
    L = C.lib()
    h = ctypes.c_void_p()
    lo = (ctypes.c_double * 3)(0, 0, 0)
    fake = ctypes.c_void_p(0x1000)
    assert L.art_create_grid(ctypes.byref(h), 0, 4, 4, lo, 0.25, fake, None, None) == C.ART_EINVAL
    assert L.art_create_grid(ctypes.byref(h), 4, 4, 4, lo, -1.0, fake, None, None) == C.ART_EINVAL
    assert L.art_create_grid(ctypes.byref(h), 4, 4, 4, lo, 0.25, None, None, None) == C.ART_EINVAL
    assert L.art_create_grid(ctypes.byref(h), 2048, 2048, 1024, lo, 0.25, fake, None, None) == C.ART_EINVAL
    assert L.art_create_grid(None, 4, 4, 4, lo, 0.25, fake, None, None) == C.ART_EINVAL
    p = C.ArtParams()
    L.art_params_default(ctypes.byref(p))
    assert L.art_trace(None, ctypes.byref(p), fake, None, None, None) == C.ART_EINVAL
    assert L.art_add_sources(None, 1, None, None) == C.ART_EINVAL
    assert L.art_get_stats(None, None) == C.ART_EINVAL
    assert L.art_xn_update(None, 10, fake, fake, fake, None, 0.0, 1.0, 0) == C.ART_EINVAL
    assert L.art_xn_update(None, 10, fake, fake, fake, None, 1.0, -1.0, 0) == C.ART_EINVAL
    assert L.art_xn_update(None, 10, fake, fake, fake, None, 1.0, 1.0, 7) == C.ART_EINVAL
    assert L.art_dt_substep(None, 10, fake, fake, fake, 1.0, 0.1, None, fake) == C.ART_EINVAL
    assert L.art_dt_scratch_bytes(1000) > 0
    L.art_destroy_grid(None)


def test_binding_fails_loudly_without_library(monkeypatch):
    # The binding never substitutes another implementation: a missing library is an error.
    import importlib
    from paper_1711_06277_gb300 import build
    monkeypatch.setattr(build, "LIB", "/nonexistent/libart.so")
    monkeypatch.setattr(build, "up_to_date", lambda: True)
    mod = importlib.reload(C)
    try:
        with pytest.raises(OSError):
            mod.lib()
    finally:
        monkeypatch.undo()
        importlib.reload(C)
