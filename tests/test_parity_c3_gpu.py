"""GPU parity at the largest single-GPU workload, the one bench.py times: the
512 x 256 x 512 disk with envelope (67.1 M cells, 79 bins, seed 2) at midplane
tau550 = 1 and 100. Every cell of the grid is compared with the FP64 oracle run on
every ray (OpenMP over rays), in each precision mode of the scan and with the
opacity table rounded to bfloat16, and in every warp-per-ray launch shape that holds
its 512-cell rays as well as the shape the autotuner picks (tolerances in
tests/_parity.py)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import synth
from tests import _parity

pytestmark = pytest.mark.gpu

NR, NTH, NPH, NNU, SEED = 512, 256, 512, 79, 2


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1001_3301_gb300  # noqa: F401  (raises if the library is missing)


@pytest.fixture(scope="module", params=[1.0, 100.0], ids=["tau1", "tau100"])
def c3(request):
    w = synth.disk3d(NR, NTH, NPH, n_nu=NNU, tau550=request.param, seed=SEED)
    orc = oracle.irradiate_workload(w, nthreads=oracle.max_threads())
    yield w, orc
    del orc


def _trace(w, precision="fp32_kahan", shape=None, autotune=False, kappa_bf16=False):
    import torch
    from paper_1001_3301_gb300 import Tracer
    with Tracer.from_grid(w.grid, precision) as tr:
        tr.set_opacity_table(w.nu, w.kappa, w.t_sub, kappa_bf16)
        tr.set_star(w.t_star, w.r_star)
        r = torch.from_numpy(w.rho32()).cuda()
        t = torch.from_numpy(w.tdust32()).cuda()
        q = torch.empty_like(r)
        a = torch.empty_like(r)
        if autotune:
            shape = tr.autotune(r, t, q, a, reps=2)
        if shape is not None:
            tr.set_tuning(*shape)
        q, a, e = tr.irradiate(r, t, q, a, energy=True)
        torch.cuda.synchronize()
        used = tr.tuning()
        shapes = tr.tunings()
        out = q.double().cpu().numpy(), a.double().cpu().numpy(), e
        del r, t, q, a
    return out, used, shapes


def test_c3_kahan_every_ray_shape_and_autotuned(c3):
    """Compensated FP32 (the bench's mode): the autotuned shape and every compiled
    warp-per-ray shape, one-chunk and chunked, each over all 67 M cells, energies of
    the whole grid."""
    w, orc = c3
    (q, a, e), used, shapes = _trace(w, autotune=True)
    st = _parity.assert_parity(w, q, a, e, orc, label=f"autotuned {used}")
    assert st["n_mask"] > 10_000_000
    for s in shapes:
        if s[0] not in (1, 2) or tuple(s) == tuple(used):
            continue
        (q, a, e), _, _ = _trace(w, shape=s)
        _parity.assert_parity(w, q, a, e, orc, label=f"{s}")


@pytest.mark.parametrize("precision,rtol", [("fp32_plain", 1e-5), ("fp64", 3e-7)])
def test_c3_other_precisions(c3, precision, rtol):
    """The plain FP32 scan within the same 1e-5 (rays of 512 cells); the FP64 mode
    exact to the float32 rounding of its outputs."""
    w, orc = c3
    (q, a, e), used, _ = _trace(w, precision)
    _parity.assert_parity(w, q, a, e, orc, rtol_q=rtol, rtol_a=rtol,
                          rtol_energy=1e-6 if precision != "fp64" else 1e-9, label=f"{precision} {used}")


def test_c3_bf16_table(c3):
    """kappa rounded to bfloat16 on the device: within 1e-5 of the oracle given the
    same rounded table (the rounding itself moves q_abs by up to ~1e-3)."""
    w, _ = c3
    k32 = w.kappa.astype(np.float32)
    bits = k32.view(np.uint32).astype(np.uint64)
    kb = ((((bits + 0x7FFF + ((bits >> 16) & 1)) >> 16) << 16).astype(np.uint32)
          .view(np.float32).astype(np.float64))
    orc_b = oracle.irradiate_workload(w, kappa=kb, nthreads=oracle.max_threads())
    (q, a, e), used, _ = _trace(w, kappa_bf16=True)
    _parity.assert_parity(w, q, a, e, orc_b, label=f"bf16 {used}")
