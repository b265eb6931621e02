"""The FP32 kernels' division of (u - q)/(u + q) is the IEEE-754 correctly
rounded quotient, checked exhaustively on the device: the refined reciprocal
for every significand and exponent, the ratio for every FP32 u with
0 < u + q < 2^126 (scalar and paired form), and random normal operand pairs."""
from __future__ import annotations

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

N_POSITIVE_BELOW_2_126 = 0x7E800000     # bit patterns 0x00000000 .. 0x7E7FFFFF


@pytest.mark.parametrize("q", [0.002, 0.0005, 0.0137, 0.3])
def test_division_is_correctly_rounded(gpu, q):
    rep = gpu.rdc_check_division(q, n_random=1 << 27, seed=12345)
    assert rep["checked"][0] == 251 << 23
    # -0 and the negative u with |u| < q (each gives u + q > 0), plus every
    # positive u below 2^126
    qf_bits = int(np.float32(q).view(np.uint32))
    assert rep["checked"][1] == N_POSITIVE_BELOW_2_126 + qf_bits
    assert rep["checked"][2] == 1 << 27
    assert rep["mismatches"] == [0, 0, 0], rep
    assert rep["first_bad"] == [0xFFFFFFFF] * 3


def test_division_check_rejects_bad_q(gpu):
    for q in (0.0, -1.0, float("nan"), float("inf")):
        with pytest.raises(gpu.RdcError) as e:
            gpu.rdc_check_division(q)
        assert e.value.status == gpu.RDC_EINVAL
