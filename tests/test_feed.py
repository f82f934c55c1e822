"""The resident server's host feeder (csrc/cos_feed.h: staging, round-robin, ring
reuse) driven on the CPU by a host-only probe against a simulated device; every
staged entry is checked against an independent record of the request chains (see
tests/native/feed_probe.cc), and every run must finish all its requests."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "feed_probe.cc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    inc = None
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "include", "cuda_runtime.h")):
            inc = os.path.join(cand, "include")
    if not cxx or not inc:
        pytest.skip("needs a C++ compiler and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("feed") / "feed_probe")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, SRC, "-o", exe], check=True, capture_output=True)
    return exe


@pytest.mark.parametrize("seed,cap,backlog,active,requests", [
    (1, 16, 8, 4, 30), (2, 16, 8, 4, 30), (3, 16, 8, 4, 30), (4, 16, 16, 6, 30),
    (5, 32, 4, 8, 40), (6, 64, 32, 8, 60), (7, 1024, 512, 16, 80), (8, 64, 64, 2, 40),
])
def test_feeder_against_simulated_device(probe, seed, cap, backlog, active, requests):
    r = subprocess.run([probe, str(seed), str(cap), str(backlog), str(active), str(requests)],
                       capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout + r.stderr
    assert int(r.stdout.split()[2]) == requests
