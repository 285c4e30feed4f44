"""GPU parity of the Halton engine (Sec. 2.2): radical inverses in the first
64 prime bases, plain, Faure-permuted and linearly scrambled, bit-exact."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    from paper_2307_15584_gb300 import binding

    return binding


@pytest.mark.parametrize("mode", [0, 1, 2])
# lane layouts: w dimensions x floor(32 / w) rows per warp step -- 8 x 4, two chunks of 32, 16 x 2,
# 7 x 4 (four lanes idle), 32 + a one-dimension chunk of 32 rows, base 2 alone (no tables);
# counts that end mid-unit and mid-step
@pytest.mark.parametrize("s,begin,count", [(8, 0, 4099), (64, 12345, 777), (16, (1 << 32) - 1500, 1500),
                                           (7, 3, 3001), (33, 99, 2049), (1, 5, 10007)])
def test_halton_bit_exact(B, oracle, mode, s, begin, count):
    primes = [oracle.lib().qo_prime(j) for j in range(s)]
    mult = np.array([1 + (7 * j + 3) % (p - 1) if p > 2 else 1 for j, p in enumerate(primes)], np.uint32)
    u = torch.empty((count, s), dtype=torch.int32, device="cuda")
    f = torch.empty((count, s), dtype=torch.float32, device="cuda")
    B.qmc_halton_points(s, mode, mult if mode == 2 else None, begin, count, u, f)
    ref = oracle.halton_points(s, begin, count, mode, mult)
    np.testing.assert_array_equal(B.as_u32(u), ref)
    np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32), oracle.map_u32_to_unifloat(ref).view(np.uint32))


def test_halton_argument_errors(B):
    u = torch.empty(64, dtype=torch.int32, device="cuda")
    for args in ((0, 0, None), (65, 0, None), (4, 3, None), (4, 2, None), (4, 2, np.array([1, 3, 1, 1]))):
        with pytest.raises(B.QMCError):
            B.qmc_halton_points(args[0], args[1], args[2], 0, 8, u, None)


@pytest.mark.parametrize("which", ["u32", "f32"])
def test_halton_single_output(B, oracle, which):
    """Either output alone: the same values, nothing written to the other."""
    s, begin, count = 12, 777, 3333
    u = torch.empty((count, s), dtype=torch.int32, device="cuda") if which == "u32" else None
    f = torch.empty((count, s), dtype=torch.float32, device="cuda") if which == "f32" else None
    B.qmc_halton_points(s, B.HALTON_FAURE, None, begin, count, u, f)
    ref = oracle.halton_points(s, begin, count, oracle.HALTON_FAURE)
    if u is not None:
        np.testing.assert_array_equal(B.as_u32(u), ref)
    else:
        np.testing.assert_array_equal(f.cpu().numpy().view(np.uint32), oracle.map_u32_to_unifloat(ref).view(np.uint32))
