"""CPU checks of the C ABI library: it loads, exports every symbol that
include/sip.h declares, its structs match the header's layout, the host-side
plane layout matches brute-force enumeration, and without a GPU it refuses
to run (no CPU fallback)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_1303_4538_gb300 import sip

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sip.h")


def _declared():
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(sip_[a-z_0-9]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    L = sip.lib()
    names = _declared()
    assert "sip_factor" in names and "sip_solve" in names and "sip_iterate" in names
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(names) == set(sip.EXPORTED)


def test_struct_layout_matches_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(r'''
#include <stdio.h>
#include <stddef.h>
#include "sip.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu\n", sizeof(sip_block_desc), offsetof(sip_block_desc, ap),
         offsetof(sip_block_desc, b), offsetof(sip_block_desc, x), offsetof(sip_block_desc, symmetric));
  printf("%zu %zu %zu %zu %zu %zu %zu\n", sizeof(sip_options), offsetof(sip_options, max_spin),
         offsetof(sip_options, tile_j), offsetof(sip_options, debug_stall), offsetof(sip_options, graphs),
         offsetof(sip_options, rows_per_thread), offsetof(sip_options, autotune));
  printf("%zu\n", sizeof(sip_interface));
  printf("%zu %zu %zu %zu\n", sizeof(sip_server_stats), offsetof(sip_server_stats, queued),
         offsetof(sip_server_stats, budget_bytes), offsetof(sip_server_stats, oldest_running_ms));
  printf("%zu %zu %zu %zu\n", sizeof(sip_pcorr_desc), offsetof(sip_pcorr_desc, dx), offsetof(sip_pcorr_desc, g),
         offsetof(sip_pcorr_desc, uz));
  return 0;
}
''')
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    out = subprocess.check_output([str(exe)]).decode().split()
    got = [int(v) for v in out]
    D, O, I = sip.sip_block_desc, sip.sip_options, sip.sip_interface
    want = [ctypes.sizeof(D), D.ap.offset, D.b.offset, D.x.offset, D.symmetric.offset,
            ctypes.sizeof(O), O.max_spin.offset, O.tile_j.offset, O.debug_stall.offset, O.graphs.offset,
            O.rows_per_thread.offset, O.autotune.offset, ctypes.sizeof(I)]
    S = sip.sip_server_stats
    want += [ctypes.sizeof(S), S.queued.offset, S.budget_bytes.offset, S.oldest_running_ms.offset]
    C = sip.sip_pcorr_desc
    want += [ctypes.sizeof(C), C.dx.offset, C.g.offset, C.uz.offset]
    assert got == want


@pytest.mark.parametrize("shape", [(3, 2, 2), (1, 1, 7), (5, 1, 1), (1, 6, 1), (4, 5, 3), (7, 3, 6), (2, 9, 4)])
def test_plane_layout_against_enumeration(shape):
    nx, ny, nz = shape
    t = sip.plane_layout(nx, ny, nz)
    # brute force: list cells in (s, k, j) order; position = rank in that order
    cells = sorted(((i + j + k, k, j, i) for k in range(nz) for j in range(ny) for i in range(nx)))
    pos = {(i, j, k): n for n, (s, k, j, i) in enumerate(cells)}
    got = {(i, j, k): int(t[k, i + j + k]) + j for k in range(nz) for j in range(ny) for i in range(nx)}
    assert got == pos
    # a permutation of 0..N-1, planes contiguous
    assert sorted(got.values()) == list(range(nx * ny * nz))


def test_no_cpu_fallback_without_gpu():
    try:
        import torch
        if torch.cuda.is_available():
            pytest.skip("a GPU is present")
    except ImportError:
        pass
    h = ctypes.c_void_p()
    rc = sip.lib().sip_create(ctypes.byref(h), 0, None)
    assert rc == sip.SIP_ERR_NO_DEVICE
    with pytest.raises(sip.SipError):
        sip.Context(0)


def test_default_options():
    o = sip.default_options()
    assert o.alpha == pytest.approx(0.92) and o.mode == sip.SIP_MODE_F64 and o.inner_iters == 4


def test_null_handles_are_invalid_arguments():
    L = sip.lib()
    assert L.sip_trim(None) == sip.SIP_ERR_INVALID_ARG
    assert L.sip_destroy(None) == sip.SIP_OK
