"""The model system's gather assigns the threads of a CTA to the x-rows (q, r) of its
owner cells in row-type order.  This host test compiles a small program against the
kernel header and checks, for d = 2, 3 and k = 1..8, that the thread slots map one to one
onto the (owner, row) pairs of a CTA, that the spare slots are idle, and that the row types
come in the order (0, 0), (0, > 0), (> 0, 0), (> 0, > 0).  No GPU is needed."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2503_00246_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <set>
#include <tuple>
#include "gp_cell.cuh"

template <int D, int K>
int check() {
  using namespace gp;
  constexpr int OPC = gather_owners_per_cta(D, K);
  constexpr int KR = CellShape<D, K>::KR;
  std::set<std::tuple<int, int, int>> seen;
  int bad = 0, last_type = -1;
  for (int u = 0; u < GATHER_THREADS; ++u) {
    int o = -1, q = -1, r = -1;
    const bool live = gather_slot<D, K>(u, o, q, r);
    if (u >= OPC * KR) { bad += live; continue; }
    if (!live || o < 0 || o >= OPC || q < 0 || q >= K || r < 0 || r >= (D == 3 ? K : 1)) { ++bad; continue; }
    if (!seen.insert(std::make_tuple(o, q, r)).second) ++bad;
    // type rank: (0,0) -> 0, (0,>0) -> 1, (>0,0) -> 2, (>0,>0) -> 3 (2D: q == 0 -> 0, else 3)
    const int type = D == 2 ? (q == 0 ? 0 : 3) : (q == 0 ? (r == 0 ? 0 : 1) : (r == 0 ? 2 : 3));
    if (type < last_type) ++bad;
    last_type = type;
  }
  if ((int)seen.size() != OPC * KR) ++bad;
  if (bad) std::printf("FAIL d=%d k=%d (%d)\n", D, K, bad);
  return bad;
}

template <int D, int... Ks>
int all(std::integer_sequence<int, Ks...>) { return (check<D, Ks + 1>() + ...); }

int main() {
  const int bad = all<2>(std::make_integer_sequence<int, 8>{}) + all<3>(std::make_integer_sequence<int, 8>{});
  std::printf(bad ? "FAILED\n" : "OK\n");
  return bad ? 1 : 0;
}
"""


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_gather_slots_cover_every_owner_row_once(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    src = tmp_path / "slots.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "slots"
    subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", CSRC, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0 and out.stdout.strip().endswith("OK"), out.stdout + out.stderr
