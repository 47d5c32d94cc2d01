"""The C-ABI library builds, loads and exports every symbol include/mrhash.h declares; the ctypes mirrors match the C
struct layouts; host-only helpers (Eq. 4 hash) agree with hand-computed values. No GPU calls."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2511_21459_b300 as mrh
from paper_2511_21459_b300 import build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mrhash.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return mrh.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mrh_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", mrh.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (mrh_\w+)", out))
    assert set(names) <= exported
    assert set(mrh.EXPORTS) == set(names)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "mrhash.h"
int main(void) {
  printf("%zu %zu %zu\n", sizeof(mrh_map_params), sizeof(mrh_pinhole), sizeof(mrh_stats));
  printf("%zu %zu %zu %zu\n", offsetof(mrh_map_params, var_threshold), offsetof(mrh_map_params, max_blocks),
         offsetof(mrh_map_params, storage), offsetof(mrh_map_params, max_range));
  printf("%zu %zu\n", offsetof(mrh_stats, live_blocks), offsetof(mrh_stats, status));
  return 0;
}
''')
    exe = tmp_path / "sz"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    lines = subprocess.check_output([str(exe)], text=True).split("\n")
    a = [int(x) for x in lines[0].split()]
    assert a == [ctypes.sizeof(mrh.Params), ctypes.sizeof(mrh.Pinhole), ctypes.sizeof(mrh.Stats)]
    b = [int(x) for x in lines[1].split()]
    assert b == [mrh.Params.var_threshold.offset, mrh.Params.max_blocks.offset, mrh.Params.storage.offset,
                 mrh.Params.max_range.offset]
    c = [int(x) for x in lines[2].split()]
    assert c == [mrh.Stats.live_blocks.offset, mrh.Stats.status.offset]


def test_hash_eq4_hand_values(lib):
    # H(x, y, z) = (x p1 xor y p2 xor z p3) mod n with p1 = 73856093, p2 = 19349669, p3 = 83492791
    assert mrh.hash_slot(1, 0, 0, 32) == 73856093
    assert mrh.hash_slot(0, 1, 0, 32) == 19349669
    assert mrh.hash_slot(0, 0, 1, 32) == 83492791
    assert mrh.hash_slot(1, 0, 0, 16) == 73856093 % 65536
    assert mrh.hash_slot(1, 1, 0, 20) == (73856093 ^ 19349669) % (1 << 20)
    assert mrh.hash_slot(1, 1, 1, 22) == (73856093 ^ 19349669 ^ 83492791) % (1 << 22)
    # negative coordinates wrap as 32-bit two's complement
    assert mrh.hash_slot(-1, 0, 0, 32) == (-73856093) % (1 << 32)
    assert mrh.hash_slot(-3, 7, -11, 20) == (((-3 * 73856093) % 2 ** 32) ^ ((7 * 19349669) % 2 ** 32) ^
                                             ((-11 * 83492791) % 2 ** 32)) % (1 << 20)
    assert mrh.hash_slot(0, 0, 0, 16) == 0


def test_status_strings_and_version(lib):
    assert lib.mrh_status_string(0) == b"ok"
    assert lib.mrh_status_string(3).startswith(b"hash")
    for code in range(10):
        assert lib.mrh_status_string(code) != b"unknown status", code
    assert b"sm_103a" in lib.mrh_version()


def test_invalid_params_rejected_before_any_device_call(lib):
    import synth
    p = mrh.params_from(synth.tiny())
    h = ctypes.c_void_p()
    bad = [("n_levels", 0), ("n_levels", 4), ("base_voxel_size", 0.0), ("truncation", -1.0), ("truncation", 1.0),
           ("hash_slots_log2", 4), ("storage", 5), ("has_color", 2), ("min_obs", -1)]
    for field, value in bad:
        q = mrh.Params.from_buffer_copy(p)
        setattr(q, field, value)
        assert lib.mrh_map_create(ctypes.byref(q), 0, ctypes.byref(h)) == 1, field
    assert lib.mrh_map_create(None, 0, ctypes.byref(h)) == 1


def test_map_files_rejected_before_any_device_call(lib, tmp_path):
    """mrh_load_map validates the header (magic, version, parameter size) before it creates a map."""
    h = ctypes.c_void_p(1)
    assert lib.mrh_load_map(os.fsencode(str(tmp_path / "missing.mrhmap")), 0, ctypes.byref(h)) == 1
    assert h.value is None
    size = ctypes.sizeof(mrh.Params)
    good = b"MRHMAP\0\1" + (1).to_bytes(4, "little") + size.to_bytes(4, "little")
    for bad in (b"", b"MRHMAP", b"MRHMAQ\0\1" + good[8:], good[:8] + (2).to_bytes(4, "little") + good[12:],
                good[:12] + (size + 4).to_bytes(4, "little"), good):  # the last one stops inside the parameters
        f = tmp_path / "bad.mrhmap"
        f.write_bytes(bad)
        assert lib.mrh_load_map(os.fsencode(str(f)), 0, ctypes.byref(h)) == 1, bad
    assert lib.mrh_load_map(None, 0, ctypes.byref(h)) == 1
    assert lib.mrh_save_map(None, os.fsencode(str(tmp_path / "x")), None) == 1


def test_mesh_case_table_matches_the_oracles(lib):
    """The library builds its Marching Cubes case table on the host (no GPU call); it is an independent second
    construction from the same definition as the oracle's, so the two must agree entry for entry."""
    import numpy as np
    import oracle
    nt_g, tri_g, ec_g = mrh.mesh_case_table()
    nt_o, tri_o, ec_o = oracle.mc_table()
    assert np.array_equal(ec_g, ec_o)
    assert np.array_equal(nt_g, nt_o)
    for c in range(256):
        assert np.array_equal(tri_g[c, :nt_g[c]], tri_o[c, :nt_o[c]]), c
