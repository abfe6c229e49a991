"""The pyramid and detection device code run on the host (no GPU) under
AddressSanitizer, against the oracle: the check that stands in for a bounds
checking build and for compute-sanitizer, which is closed on the GPU pool.

tests/emu/blockemu.h emulates thread blocks with one host thread per CUDA
thread and real barriers for __syncthreads, named barriers and the warp
collectives; the harnesses give every CTA's shared memory a heap buffer of
exactly its computed size (and the pyramid's launch size must cover every
tile's plan), so any out-of-bounds shared or global access, any wrong
keypoint or pyramid value, and any collective called from divergent lanes
(a deadlock the emulator reports) fails the test. The device headers are
compiled unchanged except for two host spellings: the named barrier's inline
PTX becomes an emulated barrier, and a function-scope __shared__ variable a
block-shared static (blocks run one at a time)."""
import os
import re
import shutil
import subprocess

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2609_30459_gb300", "csrc")
EMU = os.path.join(ROOT, "tests", "emu")


def _host_copy(dst):
    for name in ("common.cuh", "pyramid_dev.cuh", "detect_dev.cuh"):
        s = open(os.path.join(CSRC, name)).read()
        s = re.sub(r'asm volatile\("bar\.sync (\d), %0;" ::"r"\(n\) : "memory"\);',
                   r"emu_bar(\1, n);", s)
        s = s.replace("__shared__ PassPlan plan;", "static PassPlan plan;")
        open(os.path.join(dst, name), "w").write(s)


def _build(tmp_path, main):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no g++")
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(os.path.join(cuda_inc, "cuda_runtime.h")):
        pytest.skip("no CUDA headers")
    _host_copy(str(tmp_path))
    exe = str(tmp_path / (main + ".bin"))
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address", "-pthread",
           "-I", str(tmp_path), "-I", EMU, "-I", cuda_inc, "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(ROOT, "oracle", "src"), "-o", exe, os.path.join(EMU, main + ".cpp"),
           os.path.join(ROOT, "oracle", "src", "pyramid_detect.cpp")]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr:
        pytest.skip("AddressSanitizer not available")
    assert r.returncode == 0, r.stderr[-3000:]
    return exe


def _run(exe, *args, timeout=600):
    r = subprocess.run([exe, *map(str, args)], capture_output=True, text=True, timeout=timeout,
                       env={**os.environ, "ASAN_OPTIONS": "detect_leaks=0"})
    out = r.stdout + r.stderr
    assert r.returncode == 0, out[-4000:]
    assert "FAILS 0" in out, out[-4000:]
    return out


def test_pyramid_pass_on_host(tmp_path):
    oracle.build()
    out = _run(_build(tmp_path, "pyr_check"))
    assert re.search(r"cases (\d+)", out) and int(re.search(r"cases (\d+)", out).group(1)) > 30


def test_detection_on_host(tmp_path):
    oracle.build()
    _run(_build(tmp_path, "det_check"))
