"""The comparison helpers' own arithmetic (no GPU): the node values a 16-bit
grid record holds, against PyTorch's CPU conversions, at random values and
at exact halfway cases where round-to-nearest-even decides."""
import numpy as np
import torch

import parity


def _torch_round(v32: np.ndarray, dtype) -> np.ndarray:
    return torch.from_numpy(v32).to(dtype).to(torch.float64).numpy()


def test_record_values_round_to_nearest_even():
    rng = np.random.default_rng(3)
    v = np.concatenate([rng.normal(-1.0, 0.5, 4000), rng.uniform(-6, 6, 4000), [0.0, -0.0, 5.0, -5.0]])
    v32 = v.astype(np.float32)
    # bfloat16 halfway cases: lower 16 bits exactly 0x8000, upper half even and odd
    bits = (np.arange(200, dtype=np.uint32) + np.uint32(0x3F80)) << np.uint32(16) | np.uint32(0x8000)
    half_bf = bits.view(np.float32)
    # binary16 halfway cases: 1 + (2k + 1) * 2^-11 in [1, 2) lies halfway between two FP16 values
    half_f16 = (1.0 + (2 * np.arange(200) + 1) * 2.0 ** -11).astype(np.float32)
    for fmt, dtype, extra in (("bf16", torch.bfloat16, half_bf), ("f16", torch.float16, half_f16)):
        x = np.concatenate([v32, extra, -extra])
        np.testing.assert_array_equal(parity.record_values(x, fmt), _torch_round(x, dtype))
    assert parity.record_values(np.float32([1.00390625]), "bf16")[0] == 1.0           # tie to even (down)
    assert parity.record_values(np.float32([1.01171875]), "bf16")[0] == 1.015625      # tie to even (up)
    np.testing.assert_array_equal(parity.record_values(v32, "f32"), v32.astype(np.float64))
