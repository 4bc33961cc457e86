"""The tile table of the fused Pi kernel (tc_pi_fused_tile_order, host code in libgw.so): for a range of N_aux it
lists every lower 128 x 256 tile (bm, bn2 <= bm / 2) exactly once, so that every output element (r, c <= r) lies
in exactly one computed tile; the work-item count and the K-panel width agree with it.  A small C++ program linked
against the library does the check on the CPU (no GPU call)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2107_10423_gb300")

SRC = r"""
#include "pi_tc.cuh"
#include <cstdio>
#include <set>
#include <utility>
#include <vector>
int main() {
  const int ns[] = {1, 84, 127, 128, 129, 255, 256, 257, 378, 1008, 1025, 2016, 4095, 8064, 8191};
  for (int n : ns) {
    std::vector<uint32_t> t;
    gw::tc_pi_fused_tile_order(n, t);
    const int nbt = (n + 127) / 128;
    std::set<std::pair<int, int>> seen;
    for (uint32_t v : t) {
      const int bm = (int)(v & 0xffffu), bn2 = (int)(v >> 16);
      if (bm >= nbt || bn2 > bm / 2) { std::printf("n %d: tile (%d, %d) outside the lower triangle\n", n, bm, bn2); return 1; }
      if (!seen.insert({bm, bn2}).second) { std::printf("n %d: tile (%d, %d) twice\n", n, bm, bn2); return 1; }
    }
    long want = 0;
    for (int bm = 0; bm < nbt; ++bm) want += bm / 2 + 1;
    if ((long)t.size() != want) { std::printf("n %d: %zu tiles, want %ld\n", n, t.size(), want); return 1; }
    if (gw::tc_pi_fused_items(n, 3) != 3 * want) { std::printf("n %d: item count\n", n); return 1; }
    // every output element of the lower triangle falls in a listed tile
    for (int r = 0; r < n; r += (n > 600 ? 7 : 1))
      for (int c = 0; c <= r; c += (n > 600 ? 5 : 1))
        if (!seen.count({r / 128, c / 256})) { std::printf("n %d: element (%d, %d) not covered\n", n, r, c); return 1; }
  }
  const int ks[] = {1, 95, 255, 256, 257, 48640, 778240};
  for (int k : ks)
    if (gw::tc_pi_panel_cols(k) % 256 != 0 || gw::tc_pi_panel_cols(k) < k || gw::tc_pi_panel_cols(k) >= k + 256) {
      std::printf("K %d: panel columns %ld\n", k, gw::tc_pi_panel_cols(k));
      return 1;
    }
  std::printf("ok\n");
  return 0;
}
"""


def test_tile_table_covers_the_lower_triangle_once(gwlib, tmp_path):
    nvcc = os.environ.get("NVCC") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc")
                                      else shutil.which("nvcc"))
    if not nvcc:
        pytest.skip("nvcc not found")
    src = tmp_path / "tiles.cu"
    src.write_text(SRC)
    exe = tmp_path / "tiles"
    cmd = [nvcc, "-std=c++17", "-I" + os.path.join(ROOT, "include"), "-I" + os.path.join(PKG, "csrc"), str(src),
           "-o", str(exe), "-L" + PKG, "-lgw", "-Xlinker", "-rpath=" + PKG]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
