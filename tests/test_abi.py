"""The C-ABI library loads and exports every symbol include/aerosketch.h declares
(no compute calls: these run without a GPU)."""
import ctypes as ct
import os
import re
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "aerosketch.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_]+\*?\s+\*?([a-z_]+)\s*\(", src, flags=re.M)))


def _lib():
    from paper_2601_02019_gb300 import binding
    if not os.path.exists(binding.LIB_PATH):
        pytest.skip("library not built")
    return binding


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["sketch_create", "sketch_update", "sketch_query", "sketch_merge", "sketch_stats",
              "sketch_destroy", "as_status_str"]:
        assert n in names


def test_library_exports_every_declared_symbol():
    b = _lib()
    L = ct.CDLL(b.LIB_PATH)
    missing = [n for n in _declared() if not hasattr(L, n)]
    assert not missing
    assert set(_declared()) <= set(b.EXPORTED)


def test_status_strings():
    b = _lib()
    L = b.load_library()
    assert L.as_status_str(0) == b"AS_OK"
    assert L.as_status_str(7) == b"AS_ENOTSUP"


def test_struct_layouts_match_c():
    """sizeof/offsetof of the ABI structs as gcc sees them equal the ctypes mirror."""
    b = _lib()
    prog = r'''
#include <stddef.h>
#include <stdio.h>
#include "aerosketch.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(as_config), sizeof(as_stats), sizeof(as_event),
         offsetof(as_config, seed), offsetof(as_stats, device_status), offsetof(as_event, ritz_1),
         offsetof(as_config, delta), offsetof(as_event, amp_choice), sizeof(as_server_config),
         sizeof(as_server_counters), offsetof(as_server_counters, span_s));
  return 0;
}
'''
    with tempfile.TemporaryDirectory() as td:
        c = os.path.join(td, "p.c")
        exe = os.path.join(td, "p")
        open(c, "w").write(prog)
        r = subprocess.run(["gcc", "-I", os.path.dirname(HEADER), c, "-o", exe], capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("gcc unavailable: " + r.stderr[:200])
        vals = [int(v) for v in subprocess.run([exe], capture_output=True, text=True).stdout.split()]
    assert vals == [ct.sizeof(b.AsConfig), ct.sizeof(b.AsStats), ct.sizeof(b.AsEvent),
                    b.AsConfig.seed.offset, b.AsStats.device_status.offset, b.AsEvent.ritz_1.offset,
                    b.AsConfig.delta.offset, b.AsEvent.amp_choice.offset, ct.sizeof(b.AsServerConfig),
                    ct.sizeof(b.AsServerCounters), b.AsServerCounters.span_s.offset]


def test_footprint_is_host_arithmetic():
    """sketch_footprint needs no device (FP32 form): the snapshot store adds
    exactly 2 d floats per unit of snapshot rank, the state grows with d and l,
    and a bad configuration is refused."""
    b = _lib()
    f0 = b.footprint(512, 64)
    assert b.footprint(512, 64, snapshot_rank=100) - f0 == 8 * 512 * 100
    assert b.footprint(1024, 64) > f0 and b.footprint(512, 128) > f0
    # at least C and its rebuild target (2l x d FP32 each) and G (2l x 2l FP64)
    assert f0 >= 2 * (128 * 512 * 4) + 128 * 128 * 8
    with pytest.raises(b.AeroSketchError):
        b.footprint(64, 40)
    with pytest.raises(b.AeroSketchError):
        b.footprint(64, 8, snapshot_rank=-1)
