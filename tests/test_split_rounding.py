"""The two-term representation of x that the low-precision near-panel
products use (hi = round(x), lo = round(x - hi), both BF16 or both TF32,
round to nearest): the pair carries x to about the square of the unit
roundoff, while one rounding alone is off by up to the unit roundoff in
every entry.  Checked here with PyTorch's CPU BF16 conversion (round to
nearest even) and an explicit TF32 rounding of FP32 bit patterns, on
N(0,1) values and on values spread over many binades."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _bf16(x):
    return x.to(torch.bfloat16).to(torch.float32)


def _tf32(x):
    # round the 23-bit FP32 significand to 10 bits, to nearest, ties away from zero
    # (what cvt.rna.tf32.f32 does); inputs here are finite and normal
    b = x.view(torch.int32)
    r = (b + 0x1000) & ~0x1FFF
    return r.view(torch.float32)


@pytest.mark.parametrize("rnd,eps", [(_bf16, 2.0 ** -7), (_tf32, 2.0 ** -10)])
def test_hi_lo_split(rnd, eps):
    u = eps / 2   # unit roundoff of round to nearest (7 / 10 stored significand bits)
    g = torch.Generator().manual_seed(7)
    x = torch.randn(200000, generator=g, dtype=torch.float32)
    x = torch.cat([x, x * torch.exp2(torch.randint(-30, 30, (200000,), generator=g).float())])
    hi = rnd(x)
    lo = rnd(x - hi)
    one = (x - hi).abs() / x.abs()
    two = (x - (hi + lo)).abs() / x.abs()
    # one rounding: within the unit roundoff u relative, and it reaches a good part of it
    assert one.max().item() <= u * 1.0001 and one.max().item() > u / 2
    # the pair: within u^2 relative (lo is itself rounded to the same precision)
    assert two.max().item() <= u * u * 1.0001, two.max().item()
    # x - hi is exact in FP32 (Sterbenz: hi is within a factor 2 of x), so lo is
    # the rounding of the exact remainder
    assert torch.equal((x - hi) + hi, x)
