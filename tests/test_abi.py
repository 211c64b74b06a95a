"""CPU-side checks of the C ABI: libskel.so builds, loads, exports exactly
the functions include/skel.h declares, and its host-only logic (coherence
protocol step, dispatch table) behaves as specified.  No GPU needed: none of
these calls reaches the CUDA runtime's device functions."""
import ctypes as C
import os
import re
import subprocess

import pytest

from oracle import coherence as coh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sk():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1405_2915_gb300 as m
    return m


def header_functions():
    text = open(os.path.join(ROOT, "include", "skel.h")).read()
    return set(re.findall(r"^(?:int|int64_t|const char \*)\s*\*?(skel_\w+)\(", text, re.M))


def test_header_binding_and_exports_agree(sk):
    from paper_1405_2915_gb300 import _lib
    declared = header_functions()
    assert len(declared) >= 30
    assert declared == set(_lib.SIGNATURES)
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (skel_\w+)", out))
    assert declared == exported


def test_coherence_step_matches_protocol_model(sk):
    for valid in range(4):
        for unit in (coh.HOST, coh.DEVICE):
            for mode in (coh.READ, coh.WRITE, coh.READWRITE):
                assert sk.skel_coherence_step(valid, unit, mode) == coh.step(valid, unit, mode)
    with pytest.raises(sk.SkelError):
        sk.skel_coherence_step(4, 1, 1)


def test_dispatch_table_parse_and_errors(sk, tmp_path):
    sk.skel_load_dispatch_table(None)
    assert sk.skel_dispatch_size() == 0
    good = tmp_path / "t.tbl"
    good.write_text("# skeleton fn dtype bucket radius residency variant block ept tile\n"
                    "0 3 0 12 0 0 2 256 4 0\n"
                    "1 0 0 5 0 0 1 256 4 0   # comment\n\n")
    sk.skel_load_dispatch_table(str(good))
    assert sk.skel_dispatch_size() == 2
    bad = tmp_path / "bad.tbl"
    bad.write_text("0 3 0 12 0 0 2 256\n")
    with pytest.raises(sk.SkelError) as e:
        sk.skel_load_dispatch_table(str(bad))
    assert e.value.code == -8
    assert sk.skel_dispatch_size() == 2          # a failed load changes nothing
    with pytest.raises(sk.SkelError):
        sk.skel_load_dispatch_table(str(tmp_path / "missing.tbl"))
    sk.skel_load_dispatch_table(None)
    assert sk.skel_dispatch_size() == 0


def test_variant_registry_and_force(sk):
    for name in ("map", "reduce", "scan", "mapoverlap1d", "mapoverlap2d", "maparray", "batched"):
        n = sk.skel_variant_count(name)
        assert n >= 1
        assert all(sk.skel_variant_name(name, v) != "?" for v in range(n))
    sk.skel_force_variant("map", 2, 256, 4)
    sk.skel_force_variant("map", -1)
    with pytest.raises(sk.SkelError):
        sk.skel_force_variant(99, 0)


def test_container_host_logic(sk):
    import numpy as np
    c = sk.Container.empty((3, 5), np.float32)
    assert c.info() == (np.float32, (3, 5), 0)
    v = c.view(5, (5,))
    with pytest.raises(sk.SkelError):
        c.close()                                 # live view
    with pytest.raises(sk.SkelError):
        c.view(12, (5,))                          # out of range
    v.close()
    c.close()
    a = np.arange(6, dtype=np.int32)
    h = sk.Container.from_host(a)
    assert h.info() == (np.int32, (6,), sk.UNIT_HOST)
    assert h.stats() == {"h2d": 0, "d2h": 0, "h2d_bytes": 0, "d2h_bytes": 0}
    h.close()


def test_debug_hooks_validate(sk):
    sk.skel_set_debug(2, 2_000_000)
    with pytest.raises(sk.SkelError):
        sk.skel_set_debug(2, 0)
    with pytest.raises(sk.SkelError):
        sk.skel_set_debug(77, 0)
