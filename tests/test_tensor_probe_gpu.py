"""The fifth-generation tensor-core path the surrogate's inference kernel is built
on: one tcgen05 product through the library's operand layout and descriptors,
checked against an FP64 matrix product of the same BF16 values; and the hardware
tanh the activations use, checked against its documented accuracy class."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16_bits(x):
    """Round-to-nearest-even BF16 bit patterns of float32 values (as int16)."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16).astype(np.uint16)
    return r.view(np.int16)


def _bf16_value(bits):
    return (bits.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


@pytest.mark.parametrize("k", [16, 64, 128])
def test_umma_product_matches_fp64(k):
    import torch
    from paper_1001_3301_gb300 import probe_umma
    rng = np.random.default_rng(100 + k)
    a = _bf16_bits(rng.standard_normal((128, k)).astype(np.float32))
    b = _bf16_bits(rng.standard_normal((128, k)).astype(np.float32))
    # distinct structure so that a transposed or shifted operand cannot pass
    a[5, :] = _bf16_bits(np.arange(k, dtype=np.float32) / k)
    d = probe_umma(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()).cpu().numpy()
    ref = _bf16_value(a) @ _bf16_value(b).T
    err = np.abs(d - ref).max()
    assert err <= 1e-4 * np.sqrt(k) * max(1.0, np.abs(ref).max()), err


def test_tanh_approx_accuracy():
    import torch
    from paper_1001_3301_gb300 import probe_tanh
    x = torch.linspace(-12, 12, 200001, device="cuda")
    y = probe_tanh(x).double().cpu().numpy()
    ref = np.tanh(x.double().cpu().numpy())
    # tanh.approx.f32: relative error below 2^-10.9 (PTX ISA)
    assert np.max(np.abs(y - ref) / np.maximum(np.abs(ref), 1e-30)) < 2 ** -10.5
    yb = probe_tanh(x, packed_bf16=True).double().cpu().numpy()
    xb = x.to(torch.bfloat16).double().cpu().numpy()
    refb = np.tanh(xb)
    assert np.max(np.abs(yb - refb)) < 2 ** -6


def test_tensor_rates_positive():
    from paper_1001_3301_gb300 import probe_tensor_rates
    r = probe_tensor_rates()
    print(r)
    assert all(v > 0 for v in r.values())
