"""Host logic of the benchmark's side reports (residual sweep, per-Newton-step
costs), run on the CPU against a stand-in binding and stand-in CUDA events:
the call sequence, the byte accounting of the residual and the handling of a
failing case. No kernel runs here; the GPU numbers come from bench.py itself."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import bench
from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I


class _Event:
    clock = [0.0]

    def __init__(self, enable_timing=True):
        self.t = None

    def record(self, stream=None):
        self.t = _Event.clock[0]

    def elapsed_time(self, other):
        return other.t - self.t


class _FakeMesh:
    calls = []
    fail_p = None

    def __init__(self, m, mat, device=0, structured=True, ctx=None):
        if m.p == _FakeMesh.fail_p:
            raise hx.HxError(hx.HX_ERR_CUDA, "stand-in failure")
        self.input = m
        self.n_nodes = m.n_dofs // 3
        self.n_dofs = m.n_dofs
        self.n_qp = m.n_elem * (m.p + 1) ** 3
        self.device = torch.device("cpu")
        self.ctx, self.handle = object(), object()
        self.closed = False

    def node_coords(self):
        return torch.zeros(self.n_nodes, 3, dtype=torch.float64)

    def zeros(self, prec=hx.HX_FP64):
        return torch.zeros(self.n_dofs, dtype=torch.float64 if prec == hx.HX_FP64 else torch.float32)

    def precompute(self, u, store_prec=hx.HX_FP64, storage=hx.HX_CACHE_TENSORS):
        assert u.dtype == torch.float64
        _FakeMesh.calls.append(("precompute", store_prec, storage))
        _Event.clock[0] += 3.0

    def sync(self, timeout_ms=-1):
        pass

    def close(self):
        self.closed = True


def _tick(ms):
    def f(*a, **k):
        _Event.clock[0] += ms
    return f


@pytest.fixture
def fake_gpu(monkeypatch):
    _FakeMesh.calls = []
    _FakeMesh.fail_p = None
    _Event.clock[0] = 0.0
    small = I.workload_jittered_cube
    monkeypatch.setattr(I, "workload_jittered_cube", lambda p, n=32, seed=I.SEED_BASE + 2: small(p, n=2, seed=seed))
    monkeypatch.setattr(hx, "Mesh", _FakeMesh)
    monkeypatch.setattr(hx, "hx_residual", _tick(1e-4))
    monkeypatch.setattr(hx, "hx_tangent_apply", _tick(2.0))
    monkeypatch.setattr(hx, "hx_diagonal", _tick(4.0))
    monkeypatch.setattr(hx, "hx_autotune", lambda *a, **k: (0, [1.0] * 6))
    monkeypatch.setattr(torch.cuda, "Event", _Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "current_stream", lambda *a: None)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda *a: None)
    return _FakeMesh


def test_residual_bytes_counts_vectors_and_geometry():
    # 3 DoF vectors' worth of reads/writes plus 10 geometry values per point
    assert bench.residual_bytes(300, 50, 4) == 2 * 300 * 4 + 10 * 50 * 4
    assert bench.residual_bytes(300, 50, 8) == 2 * bench.residual_bytes(300, 50, 4)


def test_residual_sweep_reports_every_case(fake_gpu):
    res = bench.run_residual_sweep(0, hbm_peak=1000.0, degrees=(2, 3))
    assert [(r["p"], r["prec"]) for r in res] == [(2, "f32"), (2, "f64"), (3, "f32"), (3, "f64")]
    for r in res:
        assert "error" not in r
        assert r["ms"] == pytest.approx(1e-4)
        m, _, _ = I.workload_jittered_cube(r["p"])
        s = 4 if r["prec"] == "f32" else 8
        n_qp = m.n_elem * (r["p"] + 1) ** 3
        assert r["n_dofs"] == m.n_dofs
        assert r["gdofs"] == pytest.approx(m.n_dofs / 1e-7 / 1e9, rel=1e-3)
        assert r["hbm_frac"] == pytest.approx(bench.residual_bytes(m.n_dofs, n_qp, s) / 1e-7 / 1e9 / 1000.0,
                                              abs=1e-4)


def test_residual_sweep_records_a_failing_case_and_goes_on(fake_gpu):
    fake_gpu.fail_p = 2
    res = bench.run_residual_sweep(0, hbm_peak=1000.0, degrees=(2, 3))
    assert [("error" in r) for r in res] == [True, True, False, False]
    assert "stand-in failure" in res[0]["error"]


def test_newton_step_costs_in_applies(fake_gpu):
    res = bench.run_newton_step_costs(0, p=2)
    assert [(r["prec"], r["storage"]) for r in res] == [
        ("f32", "cache_tensors"), ("f32", "spatial_tensors"), ("f64", "cache_tensors"), ("f64", "spatial_tensors")]
    for r in res:
        assert "error" not in r, r
        assert r["apply_ms"] == pytest.approx(2.0)
        assert r["precompute_ms"] == pytest.approx(3.0)
        assert r["diagonal_ms"] == pytest.approx(4.0)
        assert r["precompute_in_applies"] == pytest.approx(1.5)
        assert r["diagonal_in_applies"] == pytest.approx(2.0)
    # every case refreshed its cache at the precision and strategy it reports
    pre = [c for c in fake_gpu.calls if c[0] == "precompute"]
    assert (hx.HX_FP32, hx.HX_SPATIAL_TENSORS) in [(c[1], c[2]) for c in pre]
    assert (hx.HX_FP64, hx.HX_CACHE_TENSORS) in [(c[1], c[2]) for c in pre]
    assert np.isfinite([r["precompute_ms"] for r in res]).all()


@pytest.mark.parametrize("p", [1, 2, 4, 6])
def test_sweep_flops_counts_every_sweep(p):
    """Count the sweeps one by one: per component, forward interpolation in
    x, y, z (each n^3 outputs of n multiply-adds), the three collocation
    derivatives (same size), and the transposes of all six backward."""
    n = p + 1
    per_sweep = n ** 3 * n * 2           # n^3 outputs, n FMAs (2 flops) each
    forward = 3 * (3 + 3) * per_sweep    # 3 components x (3 interpolation + 3 derivative sweeps)
    assert bench.sweep_flops(1, p) == 2 * forward
    assert bench.sweep_flops(10, p) == 10 * bench.sweep_flops(1, p)


def test_fma_peaks_and_pipe_fraction(monkeypatch):
    calls = []
    monkeypatch.setattr(hx, "hx_create", lambda device=0, stream=None: "ctx")
    monkeypatch.setattr(hx, "hx_destroy", lambda ctx: calls.append(("destroy", ctx)))
    monkeypatch.setattr(hx, "hx_measure_fma_peak",
                        lambda ctx, prec: 1.25e12 if prec == hx.HX_FP64 else 75e12)
    pk = bench.fma_peaks(0)
    assert pk == {"fp64_tflops": 1.25, "fp32_tflops": 75.0} and calls == [("destroy", "ctx")]
    # 10 elements of p = 2 in 1 ms: 72 * 81 * 10 flops / 1e-3 s
    tf, frac = bench.pipe_fraction(10, 2, 1.0, "f64", pk)
    assert tf == pytest.approx(round(72 * 81 * 10 / 1e-3 / 1e12, 3))
    assert frac == pytest.approx(round(72 * 81 * 10 / 1e-3 / 1.25e12, 4))
    assert bench.pipe_fraction(10, 2, 1.0, "f32", {"error": "x"})[1] is None

    def boom(ctx, prec):
        raise hx.HxError(hx.HX_ERR_CUDA, "probe failed")
    monkeypatch.setattr(hx, "hx_measure_fma_peak", boom)
    pk = bench.fma_peaks(0)
    assert "probe failed" in pk["error"] and calls[-1] == ("destroy", "ctx")


class _FakeOpMesh(_FakeMesh):
    """Operators as exact functions of their inputs, evaluated in the input's
    precision: the FP32 and FP64 calls agree up to FP32 rounding."""

    def residual(self, u, out=None):
        if self.input.frames is not None and _FakeOpMesh.fail_fiber:
            raise hx.HxError(hx.HX_ERR_NAN, "stand-in failure")
        return u * 2.0 + 1e-3

    def apply(self, du, out=None):
        return du / 3.0

    def diagonal(self, prec=hx.HX_FP64):
        return self.zeros(prec) + (1.0 / 3.0)


def test_fp32_errors_report_every_result_per_law(fake_gpu, monkeypatch):
    monkeypatch.setattr(hx, "Mesh", _FakeOpMesh)
    _FakeOpMesh.fail_fiber = False
    res = bench.run_fp32_errors(0, n=2, p=2)
    keys = {"residual", "diagonal", "tangent_recompute", "tangent_cache_F", "tangent_cache_tensors",
            "tangent_spatial_tensors"}
    for law in ("cNH", "iNH", "fiber"):
        assert set(res[law]) == keys, res[law]
        assert all(0.0 <= v < 1e-7 for v in res[law].values()), res[law]
    # x/3 and 1/3 are not FP32 numbers: the FP32 results differ from the FP64 ones by rounding
    assert res["cNH"]["tangent_cache_F"] > 0.0 and res["cNH"]["diagonal"] > 0.0
    _FakeOpMesh.fail_fiber = True
    res = bench.run_fp32_errors(0, n=2, p=2)
    assert "stand-in failure" in res["fiber"]["error"] and "error" not in res["iNH"]


def test_fp32_error_fibre_state_keeps_both_families_active():
    """Every point of the fibre case has M1.C.M1 - 1 well above 0 for both
    families, so FP32 and FP64 take the same fibre switch decisions."""
    import math
    from oracle import oracle as O
    m, mat, field, seed = bench.fp32_error_case("fiber", n=4, p=2)
    M = O.OracleMesh(m)
    u = field(O.node_coords(M)).ravel()
    _, _, F = O.qp_fields(M, u, np.arange(M.n_elem))
    C = np.einsum("qki,qkj->qij", F.reshape(-1, 3, 3), F.reshape(-1, 3, 3))
    for ph in (mat["phi"], -mat["phi"]):
        M1 = np.array([math.cos(ph), math.sin(ph), 0.0])
        assert np.einsum("i,qij,j->q", M1, C, M1).min() - 1.0 > 0.05


def test_reference_arm_line_uses_all_host_cores(capsys, monkeypatch):
    """The reference arm (the oracle on the host cores) prints the contract's
    JSON line and uses every host core even where the launcher pinned
    OpenMP to one thread per rank."""
    import argparse
    import json
    from oracle import oracle as O
    monkeypatch.delenv("RANK", raising=False)
    O.set_threads(1)
    import time
    args = argparse.Namespace(p=2, steps=2, warmup=3, gpus=1)
    t0 = time.perf_counter()
    bench.run_reference(args)
    wall = time.perf_counter() - t0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    # the timed steps did the work the line claims: whole mesh, within the run
    assert line["config"]["step"] == "the whole mesh per step"
    assert line["ms_per_step"] * 1e-3 * line["steps"] < wall
    assert abs(line["value"] - line["config"]["n_dofs"] / (line["ms_per_step"] * 1e-3) / 1e9) < 1e-9 * line["value"]
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == "GDoF/s"
    assert line["value"] > 0 and line["higher_is_better"] is True and line["steps"] == 2
    assert line["cpu_baseline"]["cores"] == bench.host_cores() == O.num_threads()
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": "GDoF/s", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_reference_arm_other_ranks_do_nothing(capsys, monkeypatch):
    import argparse
    monkeypatch.setenv("RANK", "1")
    bench.run_reference(argparse.Namespace(p=2, steps=1, warmup=3, gpus=2))
    assert capsys.readouterr().out == ""


class _FakeLawMesh(_FakeMesh):
    bad_storage = None

    def precompute(self, u, store_prec=hx.HX_FP64, storage=hx.HX_CACHE_TENSORS):
        if storage == _FakeLawMesh.bad_storage:
            raise hx.HxError(hx.HX_ERR_UNSUPPORTED, "stand-in failure")
        super().precompute(u, store_prec, storage)

    def apply_bytes(self, storage, prec):
        return 2.0e6 if prec == hx.HX_FP32 else 4.0e6


def test_law_workloads_report(fake_gpu, monkeypatch):
    monkeypatch.setattr(hx, "Mesh", _FakeLawMesh)
    _FakeLawMesh.bad_storage = hx.HX_RECOMPUTE
    flushes = []
    orig_zero = torch.Tensor.zero_

    def zero_(t):  # the flush happens outside the events' bracket
        flushes.append(_Event.clock[0])
        _Event.clock[0] += 100.0
        return orig_zero(t)
    monkeypatch.setattr(torch.Tensor, "zero_", zero_)
    wl = [("small cube", I.box_mesh(2, 2), dict(I.MAT_CNH), I.sine_field(1, strain=0.05))]
    res = bench.run_law_workloads(0, hbm_peak=1000.0, steps=4, flush_bytes=1024, workloads=wl)
    assert len(res) == 1 and res[0]["workload"] == "small cube" and "error" not in res[0]
    cases = res[0]["cases"]
    assert [(c["prec"], c["storage"]) for c in cases] == [
        (pr, st) for pr in ("f32", "f64") for st in ("recompute", "cache_F", "cache_tensors", "spatial_tensors")]
    for c in cases:
        if c["storage"] == "recompute":
            assert "stand-in failure" in c["error"]
            continue
        assert c["ms"] == pytest.approx(2.0)  # the stand-in apply's time only, not the flush's
        b = 2.0e6 if c["prec"] == "f32" else 4.0e6
        assert c["hbm_frac"] == pytest.approx(round(b / 2e-3 / 1e9 / 1000.0, 4))
    assert len(flushes) == 6 * 4  # one flush before every timed apply


def test_newton_traction_report(fake_gpu, monkeypatch):
    """The load is stepped up to the full Neumann vector of hx_traction_load
    (the real host routine); every step is reported."""
    seen = []

    def newton(ctx, mesh, u, f_ext=None, **kw):
        seen.append(f_ext.clone())
        u -= 0.001
        return {"newton_iters": 3, "cg_iters": 40, "res0": 1.0, "res": 1e-10, "converged": True}, hx.HX_OK
    monkeypatch.setattr(hx, "hx_newton_solve", newton)
    res = bench.run_newton_traction(0, n=2, p=2, steps=4)
    assert "error" not in res, res
    assert res["newton_iters_per_step"] == [3, 3, 3, 3] and res["cg_iters"] == 160 and res["status"] == "HX_OK"
    m = I.box_mesh(2, 2, jitter=0.1, seed=I.SEED_BASE + 6, clamp=True)
    full = hx.hx_traction_load(m, I.box_boundary_faces(2, 2, 2, 1), traction=(0.0, 0.0, -0.02))
    for k, f in enumerate(seen, start=1):
        assert np.allclose(f.numpy(), full * k / 4, rtol=0, atol=1e-15)
    assert res["mean_face_deflection"] == [-0.004] * 3


def test_strip_comments_keeps_code_and_literals():
    from paper_2408_12479_gb300 import build as B
    src = 'int a = 1; // note\n/* block\n comment */ const char *s = "// not a comment /* */";\nchar c = \'"\';  x =\n y;'
    assert B.strip_comments(src) == 'int a = 1; const char *s = "// not a comment /* */"; char c = \'"\'; x = y;'
    # comment-only and formatting-only edits leave the result unchanged; a code edit does not
    assert B.strip_comments("a  =  b; /* x */\n") == B.strip_comments("a = b; // y\n")
    assert B.strip_comments("a = b;") != B.strip_comments("a = c;")


def test_kernel_sources_follow_the_includes():
    import os
    from paper_2408_12479_gb300 import build as B
    names = {os.path.basename(f) for f in B.kernel_sources()}
    assert {"hx_ops.cu", "hx_core.cuh", "hx_internal.h", "hx.h", "hx_api.cu", "hx_batch_degree.cuh"} <= names
    assert "hx_loads.cpp" not in names and "hx_loads.h" not in names  # host-only, outside the kernels


def test_measured_traffic_needs_the_current_digest(tmp_path, monkeypatch):
    from paper_2408_12479_gb300 import build as B
    (tmp_path / "profiles").mkdir()
    prof = tmp_path / "profiles" / "k_apply_cNH_p4_f32_spatial_tensors.md"
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    prof.write_text(f"traffic_bytes_per_launch: 123456\nsource_digest: {B.kernel_digest()}\n")
    assert bench.measured_traffic(4, "f32", "spatial_tensors") == 123456.0
    prof.write_text("traffic_bytes_per_launch: 123456\nsource_digest: 0123abcd\n")
    assert bench.measured_traffic(4, "f32", "spatial_tensors") is None
    assert bench.measured_traffic(5, "f32", "spatial_tensors") is None  # no summary for that case


def test_headline_line_is_short_strict_json():
    """The last stdout line carries the contract's keys only, stays within a
    few KB with a full sweep summary, and non-finite numbers become null."""
    import json
    sweep = [{"p": p, "prec": pr, "storage": st, "gdofs": 10.0 * p + (st == "spatial_tensors"),
              "hbm_frac": 0.4, "ms": 0.1}
             for p in (2, 3, 4, 5, 6) for pr in ("f32", "f64")
             for st in ("recompute", "cache_F", "cache_tensors", "spatial_tensors")]
    fields = {k: None for k in bench.HEADLINE_KEYS}
    fields.update({"metric": bench.METRIC, "value": 55.0, "unit": "GDoF/s", "steps": 20, "warmup": 5,
                   "ms_per_step": float("nan"),
                   "config": {"workload": "w", "per_storage_ms": {"a": 1.0}, "x": float("inf")},
                   "roofline": {"frac": np.float32(0.41), "traffic": None}, "clocks": {"sm_mhz": 2070.0},
                   "sweep_best": bench.sweep_summary(sweep), "residual": [1.0] * 10000,
                   "solve_48": bench.solve_summary({"hp_mg_fp32": {"seconds": 1.5, "iterations": 40,
                                                                   "true_rel_residual": 9.9e-9},
                                                    "hp_mg_fp64": {"seconds": 9.0, "iterations": 40,
                                                                   "true_rel_residual": 9.8e-9},
                                                    "speedup_fp32_precond": 6.0, "levels": ["x"] * 50})})
    line = bench.headline_line(fields)
    assert len(line) < 2048
    d = json.loads(line)
    assert list(d) == list(bench.HEADLINE_KEYS)
    assert "residual" not in d
    assert d["ms_per_step"] is None and d["config"]["x"] is None
    assert abs(d["roofline"]["frac"] - 0.41) < 1e-6
    assert d["sweep_best"]["f32"]["4"] == [41.0, 0.4, None, "S"]
    assert set(d["sweep_best"]["f64"]) == {"2", "3", "4", "5", "6"}
    assert d["solve_48"] == {"hp_mg_fp32": [1.5, 40, 9.9e-9], "hp_mg_fp64": [9.0, 40, 9.8e-9], "speedup": 6.0}
    assert bench.solve_summary({"error": "x"}) == {"error": "x"}


def test_emit_prints_strict_json(capsys):
    import json
    bench.emit({"report": "x", "v": [float("nan"), 1.0, float("-inf")], "n": np.int64(3)})
    out = capsys.readouterr().out
    assert "NaN" not in out and "Infinity" not in out
    assert json.loads(out) == {"report": "x", "v": [None, 1.0, None], "n": 3}


def test_guarded_records_the_error():
    def bad():
        raise RuntimeError("boom")
    r = bench.guarded(bad)
    assert r == {"error": "RuntimeError: boom"}
    assert bench.guarded(lambda a, b=1: a + b, 1, b=2) == 3


@pytest.mark.parametrize("apply_ms,steps", [(0.1175, 20), (0.1175, 5000), (3.0, 20), (50.0, 1)])
def test_reps_per_step_lasts_the_minimum(apply_ms, steps):
    R = bench.reps_per_step(apply_ms, steps, 1.2)
    assert R >= 1
    assert R * steps * apply_ms >= 1200.0 or R == 1
    if R > 1:  # and not much longer than needed
        assert (R - 1) * steps * apply_ms < 1200.0
