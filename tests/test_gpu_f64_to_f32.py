"""The learned-curvature gather converts its FP64 volume fractions to float
from the bit patterns (integer instructions, off GB300's narrow FP64 pipe).
That conversion must round exactly as the hardware's IEEE conversion:
checked on random bit patterns of every class and on the boundaries where
round-to-nearest-even decides (ties in the normal and subnormal ranges, the
largest float, the smallest subnormal, overflow)."""
import numpy as np
import pytest
import torch

from paper_2509_26361_gb300 import ebit

pytestmark = pytest.mark.gpu


def _cases():
    rng = np.random.default_rng(5)
    bits = [rng.integers(0, 2 ** 63, 200_000, dtype=np.int64).astype(np.uint64)]
    bits.append(bits[0] | np.uint64(1 << 63))  # negative twins
    # exponents near the float range: 2^-160 .. 2^130, random fractions
    e = rng.integers(1023 - 160, 1023 + 130, 200_000).astype(np.uint64)
    fr = rng.integers(0, 2 ** 52, 200_000, dtype=np.int64).astype(np.uint64)
    bits.append((e << np.uint64(52)) | fr)
    # fractions whose dropped bits are exactly half, half +- 1 (ties and near-ties)
    keep = rng.integers(0, 2 ** 23, 50_000, dtype=np.int64).astype(np.uint64) << np.uint64(29)
    for d in (-1, 0, 1):
        tie = keep | np.uint64((1 << 28) + d)
        bits.append((e[:50_000] << np.uint64(52)) | tie)
    out = np.concatenate(bits).view(np.float64)
    f32 = np.finfo(np.float32)
    special = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, 0.5, 1.0 - 2 ** -53, float(f32.max),
               float(f32.max) * (1 + 2 ** -25), float(f32.max) * (1 + 2 ** -24), float(f32.tiny),
               float(f32.tiny) * (1 - 2 ** -24), 2.0 ** -149, 2.0 ** -150, 2.0 ** -150 * (1 + 2 ** -30),
               3 * 2.0 ** -150, 2.0 ** -151, 5e-324, 2.0 ** -1022]
    return np.concatenate([out, np.array(special), -np.array(special)])


def test_bit_pattern_conversion_rounds_like_the_hardware():
    x = torch.from_numpy(_cases()).cuda()
    got = ebit.ebit_selftest_f64_to_f32(x)
    ref = x.to(torch.float32)  # the device's IEEE conversion
    torch.cuda.synchronize()
    nan = torch.isnan(ref)
    assert torch.equal(torch.isnan(got), nan)
    g, r = got[~nan].view(torch.int32), ref[~nan].view(torch.int32)
    bad = (g != r).nonzero().flatten()
    assert bad.numel() == 0, [(float(x[~nan][i]), int(g[i]), int(r[i])) for i in bad[:5].tolist()]
