"""Failure detection on the GPU without a GPU fault: the staged apply's waits
for its bulk-copied stage are bounded. With the hx_set_wait_test hook no bulk
copy is issued, so the stage never fills and every CTA's wait gives up after
a short limit; the CTA sets the device timeout flag and returns, hx_sync
reports HX_ERR_TIMEOUT, and the context stays usable: the next apply, with
the hook off, matches the oracle. Nothing here faults, traps or hangs."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases
from tests._util import rel_inf

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("variant", [2, 3, 4, 5])
@pytest.mark.parametrize("p", [2, 4])
def test_staged_wait_runs_out_and_reports_timeout(p, variant):
    m = cases.small_cube(3, p, "cNH", seed=171 + p)  # 27 elements: several tiles and a ragged tail
    M, X, u = cases.state_for(m, "cNH", seed=172 + p)
    mat = cases.oracle_material("cNH")
    du = I.random_direction(m.n_dofs, 173 + p)
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        G.precompute(torch.tensor(u, dtype=torch.float64, device="cuda"), hx.HX_FP32, hx.HX_SPATIAL_TENSORS)
        hx.hx_set_apply_variant(G.ctx, G.handle, hx.HX_FP32, hx.HX_SPATIAL_TENSORS, variant)
        du_t = torch.tensor(du, dtype=torch.float32, device="cuda")
        hx.hx_set_wait_test(G.ctx, G.handle, 1, 1 << 20)  # about half a millisecond per wait
        t0 = time.perf_counter()
        try:
            G.apply(du_t)
        except hx.HxError as e:  # this staged tile cannot launch on this mesh: nothing to test
            assert e.status == hx.HX_ERR_CUDA
            pytest.skip(f"variant {variant} does not launch at p = {p}")
        with pytest.raises(hx.HxError) as e:
            G.sync(60000)
        assert e.value.status == hx.HX_ERR_TIMEOUT, str(e.value)
        assert time.perf_counter() - t0 < 30.0
        G.sync(60000)  # the flag was cleared when it was reported
        hx.hx_set_wait_test(G.ctx, G.handle, 0, 0)
        out = G.apply(du_t)
        G.sync(60000)
        ref = O.apply(M, mat, u, du_t.double().cpu().numpy())
        assert rel_inf(out.double().cpu().numpy(), ref) < 1e-5
    finally:
        G.close()


def test_wait_test_rejects_a_negative_limit():
    m = cases.small_cube(1, 2, "cNH")
    G = hx.Mesh(m, cases.MATS["cNH"])
    try:
        with pytest.raises(hx.HxError) as e:
            hx.hx_set_wait_test(G.ctx, G.handle, 1, -1)
        assert e.value.status == hx.HX_ERR_ARG
    finally:
        G.close()
