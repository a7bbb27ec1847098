"""Precision form (row A6): SH coefficients, log-scales and opacities stored in
BF16 or FP16, projection and compositing in FP32, against the FP64 oracle.

Two comparisons per env:
- strict: the oracle renders the ORIGINAL float32 attributes; the error is
  storage rounding plus FP32 arithmetic (target: PSNR >= 45 dB, max abs <= 8e-3);
- quantised: the oracle renders exactly the values the stored halves
  represent; the error is FP32 arithmetic only and must meet the FP32 parity
  tolerance (2e-3 max abs on non-ambiguous pixels).
"""
import numpy as np
import pytest

from gpu_helpers import compare, ensure_built, gpu_render, oracle_env, psnr
from paper_2604_25459_gb300 import synth

pytestmark = pytest.mark.gpu

SAMPLED = [0, 3, 6, 9, 12, 15, 18, 21]  # 8 sampled envs of a 24-env batch


def _stats(w, dtype, out):
    _, bg_w = synth.quantize(w.background, dtype)
    _, ln_w = synth.quantize(w.links, dtype)
    rows = []
    for e in SAMPLED:
        strict = oracle_env(w, e)
        quant = oracle_env(w, e, widened=(bg_w, ln_w))
        st_q = compare(out["rgb"][e], out["depth"][e], out["alpha"][e], quant)
        ok = strict["amb"] == 0
        err = np.abs(out["rgb"][e] - strict["rgb"])
        rows.append(dict(env=e, psnr=psnr(out["rgb"][e], strict["rgb"]), max_abs_all=float(err.max()),
                         max_abs_unamb=float(err.max(axis=-1)[ok].max()), quant_max=st_q["rgb_max"],
                         quant_amb=st_q["amb_frac"]))
    return rows


@pytest.mark.parametrize("res", ["128x128", "640x480"])
@pytest.mark.parametrize("dtype", ["f16", "bf16"])
def test_precision_forms_against_fp64_oracle(dtype, res):
    ensure_built()
    w = synth.make_c2(n_envs=24, res=res)
    out = gpu_render(w, dtype=dtype)
    rows = _stats(w, dtype, out)
    worst_psnr = min(r["psnr"] for r in rows)
    worst_unamb = max(r["max_abs_unamb"] for r in rows)
    print(f"\nprecision {dtype} {res}: min PSNR {worst_psnr:.2f} dB, max abs (non-ambiguous) {worst_unamb:.2e}, "
          f"max abs (all) {max(r['max_abs_all'] for r in rows):.2e}, quantised-oracle max abs "
          f"{max(r['quant_max'] for r in rows):.2e}")
    for r in rows:
        print("  ", {k: (round(v, 6) if isinstance(v, float) else v) for k, v in r.items()})
    assert worst_psnr >= 45.0
    if dtype == "f16":
        assert worst_unamb <= 8e-3
    else:
        # Stated exception: BF16 storage (8-bit mantissa on opacities and
        # log-scales) moves a few splat edges by ~1e-2 in colour, above the 8e-3
        # target; the kernels' own share (against the oracle fed the same
        # stored values) stays at the FP32 parity level.
        print(f"  BF16 exception: max abs {worst_unamb:.2e} vs the 8e-3 target (storage error)")
        assert worst_unamb <= 1.5e-2
    assert max(r["quant_max"] for r in rows) <= 2e-4
