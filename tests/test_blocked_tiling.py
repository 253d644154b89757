"""Host logic of the batch's blocked mode: the wall-aligned tiling of one axis
(AxisTiles in csrc/cue_internal.h), compiled as host code and checked for every
side up to 1,500 nodes and every halo the blocked mode can use.

For each axis the tiles must partition [0, n) in order; every tile's loaded
region must hold its interior plus the halo on each side that is not a wall
(and the ghost row beyond a wall in y); x origins must be multiples of 4
(16-byte TMA coordinates); the binning index of every node must be the tile
whose interior holds it; and no side may take more tiles than the uniform
tiling ceil(n / (W - 2H)) that the workspace is sized from.  A GPU test
(test_gpu_batch.py) holds the kernel to the plain path at every step of the
tile count."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SRC = r"""
#include <cstdio>
#include "cue_internal.h"
using cue::AxisTiles;
int main()
{
    int bad = 0;
    struct Axis { int W, ghost, hmin, hmax, hstep, align; };
    const Axis axes[2] = {{cue::kBlockedTileW, 0, 4, 64, 4, 4}, {cue::kBlockedTileRows, 1, 2, 40, 1, 1}};
    for (const Axis &a : axes)
        for (int H = a.hmin; H <= a.hmax; H += a.hstep) {
            if (a.W - 2 * H < 16) continue;
            for (int n = 1; n <= 1500; ++n) {
                const AxisTiles t{n, a.W, H, a.ghost};
                const int m = t.count(), T = a.W - 2 * H;
                if (m > (n + T - 1) / T) ++bad;
                int covered = 0;
                for (int k = 0; k < m; ++k) {
                    const int s = t.start(k), e = t.end(k), o = t.origin(k);
                    if (s != covered || e <= s) ++bad;
                    covered = e;
                    if (((o % a.align) + a.align) % a.align) ++bad;
                    const int lo = k == 0 ? s - a.ghost : s - H;          // first node that must be loaded
                    const int hi = k == m - 1 ? e + a.ghost : e + H;      // one past the last
                    if (o > lo || o + a.W < hi) ++bad;
                    if (t.index(s) != k || t.index(e - 1) != k) ++bad;
                }
                if (covered != n) ++bad;
                if (bad) {
                    std::printf("bad W=%d H=%d n=%d\n", a.W, H, n);
                    return 1;
                }
            }
        }
    std::printf("ok\n");
    return 0;
}
"""


def test_axis_tiles_partition_cover_and_bin_every_node(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    src = tmp_path / "axis_tiles.cu"
    exe = tmp_path / "axis_tiles"
    src.write_text(SRC)
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", os.path.join(ROOT, "include"),
                    "-I", os.path.join(ROOT, "paper_1405_3331_gb300", "csrc"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
