"""The request server's first-fit free list (tiles, region slots and arena
byte offsets) against a brute-force bitmap model, compiled on the host with
g++ (the header has no CUDA dependency)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_free_list_matches_bitmap_model(tmp_path):
    if shutil.which("g++") is None:
        pytest.skip("needs g++")
    exe = str(tmp_path / "freelist_test")
    subprocess.run(["g++", "-O1", "-std=c++17", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "paper_2211_15963_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "freelist_test.cc"), "-o", exe],
                   check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
