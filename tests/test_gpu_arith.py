"""The library's own arithmetic building blocks (fr_arith.cuh) against CUDA's correctly rounded
operations on 2^20 inputs each (tests/cuda/arith_check.cu, compiled for sm_103a here):
* rcp_t(double): the hardware reciprocal approximation refined by two Newton steps (each step
  squares the relative error: 2^-23 -> 2^-46 -> below 2^-53); within 1 ulp of 1.0/x, over
  exponents -60..60 and the density/pressure range [1/16, 16);
* f32_from_double_bits: double -> float from the bit pattern, within 1 float ulp of
  __double2float_rn (it rounds half away from zero, CUDA half to even);
* f_to_double_bits: float -> double from the bit pattern, exact;
* ff_from_double: the double-word split hi + lo, within 2^-47 relative."""
import os
import subprocess
import tempfile

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2306_06744_gb300", "csrc")


def test_arith_building_blocks():
    from paper_2306_06744_gb300 import build as B
    exe = os.path.join(tempfile.mkdtemp(), "arith_check")
    cmd = [B._nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-I" + CSRC,
           os.path.join(HERE, "cuda", "arith_check.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    vals = dict(line.split() for line in out.strip().splitlines())
    assert int(vals["rcp"]) <= 1, vals
    assert int(vals["f32"]) <= 1, vals
    assert int(vals["f64"]) == 0, vals
    assert float(vals["ffrel"]) <= 2.0 ** -47, vals
