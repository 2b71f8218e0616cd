"""Host-side check (no GPU) of how the library classifies a caller's pointer: device memory of the
current device is used in place, host memory is staged, and device memory of ANOTHER GPU is
rejected (the kernels must not read a peer's memory without peer access).  The classification is a
plain function of the pointer attributes (csrc/pointer_kind.h); this test compiles it into a small
harness with mocked attribute values."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HDR = os.path.join(ROOT, "paper_1301_2102_gb300", "csrc", "pointer_kind.h")

HARNESS = r"""
#include <cstdio>
#include "pointer_kind.h"
int main() {
  using bmr::MemKind; using bmr::mem_kind;
  struct C { bool ok; int type, pdev, cur; MemKind want; } cases[] = {
    {false, 2, 0, 0, MemKind::host},          // attributes unavailable: treated as host memory
    {true, 0, -2, 0, MemKind::host},          // unregistered (pageable) host memory
    {true, 1, 0, 0, MemKind::host},           // pinned host memory
    {true, 2, 0, 0, MemKind::device},         // device memory of the current device
    {true, 2, 3, 3, MemKind::device},
    {true, 2, 1, 0, MemKind::other_device},   // device memory of another GPU
    {true, 2, 0, 5, MemKind::other_device},
    {true, 2, 0, -1, MemKind::other_device},  // current device unknown
    {true, 3, 7, 0, MemKind::device},         // managed memory
  };
  int bad = 0;
  for (const C& c : cases)
    if (mem_kind(c.ok, c.type, c.pdev, c.cur) != c.want) { std::printf("case %d %d %d %d\n", c.ok, c.type, c.pdev, c.cur); ++bad; }
  std::printf("%d\n", bad);
  return bad;
}
"""


def test_pointer_classification(tmp_path):
    src = tmp_path / "h.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "h"
    subprocess.run(["g++", "-std=c++17", "-I", os.path.dirname(HDR), str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout
