"""Host logic of the forward-stability study (Sec. 7.1) on the CPU: the
sampling of displacement gradients, the per-sample normwise error, and the
skipping of samples that are not deformations (det(I + G) <= 0), with a
stand-in pointwise evaluation in place of the device kernel."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import stability as S


@pytest.mark.parametrize("eps", [1e-8, 1e-3, 1.0, 1e2])
def test_sample_gradients_magnitudes_and_signs(eps):
    rng = np.random.Generator(np.random.PCG64(3))
    G = S.sample_gradients(20000, eps, rng)
    assert G.shape == (20000, 3, 3)
    a = np.abs(G)
    assert a.min() >= eps / 10.0 and a.max() <= eps
    # uniform magnitudes: the mean is the interval's midpoint; signs are balanced
    assert abs(a.mean() / (0.55 * eps) - 1.0) < 0.01
    assert abs((G < 0).mean() - 0.5) < 0.01


def test_rel_error_is_worst_normwise_error_over_valid_samples():
    ref = torch.tensor([[[1.0, -4.0]], [[2.0, 0.5]], [[1.0, 1.0]]], dtype=torch.float64)
    lo = ref.clone()
    lo[0, 0, 1] += 0.04    # 0.04 / 4 = 1e-2
    lo[1, 0, 0] += 0.002   # 0.002 / 2 = 1e-3
    lo[2, 0, 0] += 1.0     # 1.0, but not valid
    valid = torch.tensor([True, True, False])
    assert S.rel_error(lo, ref, valid) == pytest.approx(1e-2)
    assert math.isnan(S.rel_error(lo, ref, torch.zeros(3, dtype=torch.bool)))


def _fake_eval(ctx, handle, G, H, prec, form=0, elem=0):
    """S = sym(G) + tr(G) I, P = (I + G) S, dP = H S: exact polynomials of the
    inputs, computed in FP64 or FP32 like the device evaluation."""
    dt = torch.float64 if prec == hx.HX_FP64 else torch.float32
    g, h = G.to(dt), H.to(dt)
    eye = torch.eye(3, dtype=dt)
    s = 0.5 * (g + g.transpose(1, 2)) + g.diagonal(dim1=1, dim2=2).sum(-1)[:, None, None] * eye
    return s, (eye + g) @ s, h @ s


class _Mesh:
    device = torch.device("cpu")
    ctx = handle = None


def test_study_records_every_scale_and_skips_non_deformations(monkeypatch):
    monkeypatch.setattr(hx, "hx_material_eval", _fake_eval)
    scales = [1e-6, 1e-2, 1.0, 1e2]
    out = S.study(_Mesh(), scales=scales, samples=400, forms=(0, 2))
    assert set(out) == {"stable", "standard"}
    for rec in out.values():
        assert rec["eps"] == scales
        # small gradients: every sample is a deformation; at eps = 100 many are not
        assert rec["valid"][0] == rec["valid"][1] == 400
        assert 0 < rec["valid"][3] < 400
        for name in ("S", "P", "dP"):
            e = np.array(rec[name])
            assert np.isfinite(e).all()
            # FP32 evaluation of a few products: errors of a few units of FP32 rounding
            assert (e < 1e-5).all() and (e > 0).any()
