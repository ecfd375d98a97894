"""Shared-memory placement of the copied tiles (host logic of tf_ct_kernels.cuh, no GPU):
a host program built with nvcc prints the offsets and this test checks them.

* The forward column kernel's layer tiles arrive by tensor copies, whose shared-memory
  destination must start on a 128-byte boundary: every model column's tile must, for every
  layer row count ny (an odd ny once put the second tile on a 64-byte boundary), and the
  tiles must not overlap.
* The rows_c2r bulk-copy kernel copies each input row to its own position: every row must
  start on a 16-byte boundary (the bulk copy's rule), after the end of the previous row."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_copied_tiles_are_aligned(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    exe = tmp_path / "smem_placement"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(HERE, "..", "include"), "-o", str(exe),
                    os.path.join(HERE, "c_abi", "smem_placement.cu")], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    tiles, rows = {}, {}
    for line in out.splitlines():
        f = line.split()
        if f[0] == "tile":
            ny, c, off, size = map(int, f[1:])
            assert off % 128 == 0, (ny, c, off)
            tiles.setdefault(ny, []).append((off, size))
        else:
            n1, hs, r, off = map(int, f[1:])
            assert off % 16 == 0, (n1, r, off)
            rows.setdefault((n1, hs), []).append(off)
    assert len(tiles) == 256
    for ny, t in tiles.items():
        for (o0, s0), (o1, _) in zip(t, t[1:]):
            assert o1 >= o0 + s0, ny          # consecutive tiles do not overlap
    for (n1, hs), offs in rows.items():
        for a, b in zip(offs, offs[1:]):
            assert b >= a + hs * 8, n1        # each row's hs complex values fit before the next
