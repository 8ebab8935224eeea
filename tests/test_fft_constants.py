"""Compile-time constants of the device FFT helpers, checked on the host (no
GPU): the exact cos(2 pi m / 32) table and its rounding to bfloat16 that the
BF16 frame-pair transforms use as twiddles.  A small host program built with
nvcc from the same header prints them; the references are the mathematics
(numpy's cosine in FP64, rounded to FP32) and round-to-nearest-even on the
FP32 bit pattern."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1603_02126_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "epic_fft.cuh"
int main() {
  using namespace epic::fft;
  for (int m = -40; m <= 40; ++m) {
    const float c = cos32(m);
    std::printf("%d %.9e %u\n", m, static_cast<double>(c), static_cast<unsigned>(bf16_bits(c)));
  }
  const float extra[] = {1.0f, -1.0f, 0.5f, 3.0f, 1.00390625f, 1.005859375f, 1.0f + 1.0f / 256.0f,
                         1.0f + 3.0f / 256.0f, 1e-20f, -7.25e10f, 0.70710678f, 1.9999999f};
  for (float x : extra) std::printf("x %.9e %u\n", static_cast<double>(x), static_cast<unsigned>(bf16_bits(x)));
  return 0;
}
"""


def _nvcc():
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return os.path.join(cand, "bin", "nvcc")
    return shutil.which("nvcc")


def _bf16_rne(x: np.float32) -> int:
    """Round-to-nearest-even of an FP32 value to bfloat16, on the bits."""
    b = int(np.array([x], dtype=np.float32).view(np.uint32)[0])
    return ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF


@pytest.fixture(scope="module")
def printed(tmp_path_factory):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("nvcc not found")
    d = tmp_path_factory.mktemp("fftconst")
    src, exe = d / "consts.cu", d / "consts"
    src.write_text(PROGRAM)
    subprocess.run([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-I" + CSRC, str(src),
                    "-o", str(exe)], check=True, capture_output=True, text=True)
    return subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")


def test_cos32_is_the_exact_cosine_rounded_to_fp32(printed):
    for line in printed:
        if not line or line.startswith("x"):
            continue
        m, c, _ = line.split()
        exact = np.cos(2.0 * np.pi * int(m) / 32.0)     # FP64; the quarter turns come out near 1e-16
        if int(m) % 8 == 0 and int(m) % 16 != 0:
            assert float(c) == 0.0, (m, c)              # cos of an odd multiple of pi/2
        else:
            assert np.float32(float(c)) == np.float32(exact), (m, c, exact)


def test_bf16_bits_round_to_nearest_even(printed):
    for line in printed:
        if not line:
            continue
        parts = line.split()
        x, bits = np.float32(float(parts[1])), int(parts[2])
        assert bits == _bf16_rne(x), (line, hex(bits), hex(_bf16_rne(x)))
