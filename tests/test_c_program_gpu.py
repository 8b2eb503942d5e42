"""The C ABI from a plain C program (tests/c_program.c, built with gcc and
linked against libszx.so and the CUDA runtime): its stream is byte-identical
to the oracle's and its decodes bit-identical."""
import os
import subprocess

import numpy as np
import pytest

import oracle

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
LIBDIR = os.path.join(ROOT, "paper_2201_13020_b300", "lib")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _build(tmp):
    exe = os.path.join(tmp, "c_program")
    cmd = ["gcc", "-O2", "-std=c11", os.path.join(HERE, "c_program.c"), "-I", os.path.join(ROOT, "include"),
           "-I", os.path.join(CUDA, "include"), "-L", LIBDIR, "-lszx", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{LIBDIR}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-lm", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_c_program_compiles(tmp_path):
    _build(str(tmp_path))


@pytest.mark.gpu
def test_c_program_matches_the_oracle(tmp_path):
    exe = _build(str(tmp_path))
    r = subprocess.run([exe, str(tmp_path)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    x = np.fromfile(tmp_path / "x.bin", dtype=np.float32)
    stream = np.fromfile(tmp_path / "stream.bin", dtype=np.uint8)
    y = np.fromfile(tmp_path / "y.bin", dtype=np.float32)
    part = np.fromfile(tmp_path / "part.bin", dtype=np.float32)
    ref = oracle.compress(x, 1e-3, 128)
    assert np.array_equal(stream, ref)
    yr = oracle.decompress(ref)
    assert np.array_equal(y.view(np.uint32), yr.view(np.uint32))
    assert np.array_equal(part.view(np.uint32), yr[100 * 128:300 * 128].view(np.uint32))
