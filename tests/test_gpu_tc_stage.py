"""The tensor-core DFT-matrix stage (tcgen05.mma, split BF16, FP32 accumulation) against the same
radix-16 stage on the CUDA cores: same outputs to the split-BF16 products' accuracy (the hi + lo
halves of each operand carry 16 bits, the dropped lo x lo product about 2^-16 of each term),
measured times positive, and no bounded wait given up."""
import pytest

from paper_2107_03958_gb300.api import measure_tc_stage

pytestmark = pytest.mark.gpu


def test_tensor_core_stage_matches_cuda_core_stage():
    r = measure_tc_stage(reps=200)
    assert r["max_rel_err"] < 1e-4, r
    assert r["us_cuda_core"] > 0 and r["us_tensor"] > 0, r
