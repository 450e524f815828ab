"""Benchmark of the matrix-free hyperelastic tangent apply on GB300.

Default workload: compressible neo-Hookean on the 32^3 cube with interior
vertices jittered by +-10% of h, p = 4 (6,440,067 DoFs), FP32, with the
fastest of the quadrature-point storage strategies. One apply is K(u_k) du over
the whole mesh (gather, sum-factorized gradient, quadrature-point material
tangent, integration, scatter: one fused kernel plus the zeroing of the
output). As in the paper's protocol (Sec. 7.2: repeat until at least a second
has passed), one timed step is a block of R back-to-back applies, R chosen so
that the K timed steps last at least a second; the qp cache is refreshed once
before timing. Metric: GDoF/s over all 3*n_nodes DoFs.

Output: one JSON line per side report ({"report": name, ...}: storage sweep,
residual, Newton-step costs, FP32 errors, other laws, batch, solve, Newton,
stability), then, LAST, the compact headline line of the contract.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
For N > 1 (torchrun) every rank runs an independent replica (weak scaling, no
collective in the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "tangent-operator apply GDoF/s (p=2-6, FP64 vs FP32) and fraction of HBM roofline"
L2_BYTES = 129 * 1024 * 1024
# The paper's own node-level figures (Sec. 7.2), quoted for context: another
# machine and FP64, so no ratio is formed with them.
PAPER_CONTEXT = {"hardware": "2x Intel Xeon Platinum 8360Y (72 cores, AVX-512), DDR4-3200", "precision": "f64",
                 "workload": "uniformly refined cubes, 2.5-5 MDoF, p = 1..8",
                 "tangent_apply_peak_gdofs": {"cNH": 1.75, "iNH": 1.75, "fiber": 1.25},
                 "dram_gbs_p4_tensors": [260, 280], "residual_spatial_gdofs": [0.05, 0.08], "source": "Sec. 7.2"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.lines = []
        self.skip = 0

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 5.0:  # first sample before timing starts
                time.sleep(0.02)
            self.skip = len(self.lines)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.skip:]:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_traffic(p, prec, storage):
    """DRAM bytes (read + write) per launch of the apply kernel from the
    committed ncu summary of this (p, prec, storage) workload, if the summary
    was taken on the current kernel sources; else None."""
    from paper_2408_12479_gb300.build import kernel_digest
    path = os.path.join(ROOT, "profiles", f"k_apply_cNH_p{p}_{prec}_{storage}.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for ln in open(path):
        if ":" in ln and ln.strip().startswith(("traffic_bytes_per_launch", "source_digest")):
            k, v = ln.strip().strip("`").split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_digest") != kernel_digest() or "traffic_bytes_per_launch" not in vals:
        return None
    return float(vals["traffic_bytes_per_launch"])


def max_over_ranks(ms, world):
    """Slowest rank's time (ms): the job's time for the weak-scaling value."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(n_dofs, t_max_ms, world):
    """Whole-job GDoF/s: every rank applies its own replica of n_dofs."""
    return world * n_dofs / (t_max_ms * 1e-3) / 1e9


def build_case(p, prec, storage, device, law="cNH", n=32):
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    m, field, seed = I.workload_jittered_cube(p, n=n)
    mat = dict(I.MAT_CNH)
    G = hx.Mesh(m, mat, device=device)
    X = G.node_coords().cpu().numpy()
    u = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
    du64 = torch.tensor(I.random_direction(m.n_dofs, seed + 3), dtype=torch.float64, device=G.device)
    du = du64 if prec == hx.HX_FP64 else du64.float()
    G.precompute(u, prec, storage)
    out = torch.empty_like(du)
    G.tune = hx.hx_autotune(G.ctx, G.handle, du, out, reps=5)
    return G, m, u, du, out


def time_steps(G, du, out, steps, warmup):
    import torch
    from paper_2408_12479_gb300 import hx
    for _ in range(warmup):
        hx.hx_tangent_apply(G.ctx, G.handle, du, out)
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        hx.hx_tangent_apply(G.ctx, G.handle, du, out)
    e1.record(s)
    torch.cuda.synchronize()
    G.sync(60000)
    return e0.elapsed_time(e1) / steps


def _event_ms(fn, steps, warmup):
    """Mean ms of fn() over `steps` calls after `warmup`, by CUDA events on the
    current stream (the library's calls run on it)."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(s)
    for _ in range(steps):
        fn()
    e1.record(s)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def sweep_flops(n_elem, p):
    """Algorithmic flops of the sum-factorized sweeps of one tangent apply:
    per element and component, three interpolation sweeps and three
    collocation-derivative sweeps forward and their transposes backward, each
    (p+1)^3 outputs of (p+1) multiply-adds: 72 (p+1)^4 flops per element. The
    plain count (no even-odd saving) and without the quadrature-point work, so
    the pipe fraction built on it is a lower bound."""
    return 72 * (p + 1) ** 4 * n_elem


def fma_peaks(device):
    """Measured FP64 and FP32 FMA peaks of the device (hx_measure_fma_peak),
    in TFLOP/s; an error is recorded instead if the probe fails."""
    from paper_2408_12479_gb300 import hx
    ctx = None
    try:
        ctx = hx.hx_create(device)
        return {"fp64_tflops": round(hx.hx_measure_fma_peak(ctx, hx.HX_FP64) / 1e12, 3),
                "fp32_tflops": round(hx.hx_measure_fma_peak(ctx, hx.HX_FP32) / 1e12, 3)}
    except Exception as exc:  # recorded in the report; the headline line still prints
        return {"error": str(exc)[:200]}
    finally:
        if ctx is not None:
            hx.hx_destroy(ctx)


def pipe_fraction(n_elem, p, ms, prec_name, peaks_fp):
    """(sweep TFLOP/s, fraction of the measured FMA peak of that precision)."""
    tf = sweep_flops(n_elem, p) / (ms * 1e-3) / 1e12
    peak = (peaks_fp or {}).get("fp64_tflops" if prec_name == "f64" else "fp32_tflops")
    return round(tf, 3), (round(tf / peak, 4) if peak else None)


def _rel_inf(a, b):
    """max |a - b| / max |b| (the parity tests' error measure)."""
    return float((a - b).abs().max() / b.abs().max())


def fp32_error_case(law, n=16, p=4):
    """Mesh, material and state of the FP32-error report for one law: the
    n^3 jittered cube at degree p with its 5 % sine state; for the fibre law
    per-element frames along the axes (families in the x-y plane at +-40
    degrees) and x, y stretched by 8 % so that every I* is well above 1."""
    from paper_2408_12479_gb300 import inputs as I
    m, field, seed = I.workload_jittered_cube(p, n=n)
    mat = {"cNH": I.MAT_CNH, "iNH": I.MAT_INH, "fiber": I.MAT_FIBER}[law]
    if law == "fiber":
        m.frames = I.constant_frames(m.n_elem)
        field.affine = np.diag([0.08, 0.08, 0.0])
        field.x0 = np.zeros(3)
    return m, dict(mat), field, seed


def run_fp32_errors(device, n=16, p=4):
    """Error of every FP32 result against the FP64 result of the same call on
    the same inputs (the FP64 path matches the oracle to 1e-12 in the parity
    tests): residual, tangent apply per storage strategy, diagonal; per law.
    FP32 calls get the FP32-rounded vectors and the FP64 calls the same
    values, so only arithmetic differences are measured."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = {}
    for law in ("cNH", "iNH", "fiber"):
        rec = {}
        G = None
        try:
            m, mat, field, seed = fp32_error_case(law, n, p)
            G = hx.Mesh(m, mat, device=device)
            X = G.node_coords().cpu().numpy()
            u64 = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
            u32 = u64.float()
            du32 = torch.tensor(I.random_direction(m.n_dofs, seed + 3), dtype=torch.float32, device=G.device)
            rec["residual"] = _rel_inf(G.residual(u32).double(), G.residual(u32.double()))
            for st in (hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS):
                G.precompute(u64, hx.HX_FP64, st)
                G.precompute(u64, hx.HX_FP32, st)
                rec["tangent_" + hx.STORAGE_NAMES[st]] = _rel_inf(G.apply(du32).double(), G.apply(du32.double()))
            rec["diagonal"] = _rel_inf(G.diagonal(hx.HX_FP32).double(), G.diagonal(hx.HX_FP64))
            G.sync(60000)
            rec = {k: float("%.3g" % v) for k, v in rec.items()}
        except Exception as exc:  # recorded in the report; the headline line still prints
            rec["error"] = str(exc)[:200]
        finally:
            if G is not None:
                G.close()
            torch.cuda.empty_cache()
        res[law] = rec
    res["workload"] = f"{n}^3 jittered cube, p={p}, 5 % sine state (fibre: +8 % x, y stretch)"
    return res


def _event_ms_flushed(fn, steps, warmup, flush):
    """Mean ms of fn() with an L2 flush (a write of `flush`, larger than L2)
    before every call; CUDA events enclose fn() alone."""
    import torch
    for _ in range(warmup):
        fn()
    s = torch.cuda.current_stream()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for e0, e1 in ev:
        flush.zero_()
        e0.record(s)
        fn()
        e1.record(s)
    torch.cuda.synchronize()
    return sum(e0.elapsed_time(e1) for e0, e1 in ev) / steps


def law_workloads():
    """The iNH and fibre workloads at full size: (name, mesh, material,
    state field)."""
    from paper_2408_12479_gb300 import inputs as I
    m, field, _ = I.workload_compressed_cube(n=48, p=4, J_target=0.9)
    yield "iNH kappa=1e3 mu, 48^3 jittered cube, p=4, J~0.9", m, dict(I.MAT_INH), field
    yield ("fiber, tube 16x8x64 with Q2 geometry, p=3, 2 % inflation + 1 % sines", I.tube_mesh(3),
           dict(I.MAT_FIBER), I.inflation_field(I.SEED_BASE + 4))


def run_law_workloads(device, hbm_peak, steps=10, flush_bytes=256 << 20, workloads=None):
    """Tangent-apply throughput of the iNH and fibre workloads per precision
    and storage strategy (autotuned variant), with an L2 flush before every
    timed apply. A case that fails records its error."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = []
    flush = None
    try:
        workloads = list(workloads if workloads is not None else law_workloads())
    except Exception as exc:  # recorded in the report; the headline line still prints
        return [{"error": str(exc)[:200]}]
    for name, m, mat, field in workloads:
        rec = {"workload": name, "n_dofs": m.n_dofs, "cases": []}
        G = None
        try:
            G = hx.Mesh(m, mat, device=device)
            if flush is None:
                flush = torch.empty(flush_bytes, dtype=torch.uint8, device=G.device)
            X = G.node_coords().cpu().numpy()
            u = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
            du64 = torch.tensor(I.random_direction(m.n_dofs, 7), dtype=torch.float64, device=G.device)
            for pr in (hx.HX_FP32, hx.HX_FP64):
                du = du64.float() if pr == hx.HX_FP32 else du64
                out = torch.empty_like(du)
                for st in (hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS):
                    case = {"prec": "f32" if pr == hx.HX_FP32 else "f64", "storage": hx.STORAGE_NAMES[st]}
                    try:
                        G.precompute(u, pr, st)
                        variant, _ = hx.hx_autotune(G.ctx, G.handle, du, out, reps=3)
                        t = _event_ms_flushed(lambda: hx.hx_tangent_apply(G.ctx, G.handle, du, out), steps, 2, flush)
                        G.sync(60000)
                        b = G.apply_bytes(st, pr)
                        case.update({"ms": round(t, 4), "gdofs": round(m.n_dofs / (t * 1e-3) / 1e9, 3),
                                     "hbm_frac": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4), "tile_variant": variant})
                    except Exception as exc:  # recorded; the other cases go on
                        case["error"] = str(exc)[:200]
                    rec["cases"].append(case)
        except Exception as exc:  # recorded in the report; the headline line still prints
            rec["error"] = str(exc)[:200]
        finally:
            if G is not None:
                G.close()
            torch.cuda.empty_cache()
        res.append(rec)
    return res


def residual_bytes(n_dofs, n_qp, s):
    """Algorithmic bytes of one cNH residual: read u, write r, and the stored
    J0^-1 (9) and JxW (1) per quadrature point; the state is recomputed from u
    at every point, so nothing else is read."""
    return 2 * n_dofs * s + 10 * n_qp * s


def run_residual_sweep(device, hbm_peak, degrees=(2, 3, 4, 5, 6)):
    """R(u) on the 32^3 jittered cube (cNH), p = 2..6, FP32 and FP64: one call
    is the zeroing of r plus one fused kernel. A case that fails records its
    error and the sweep goes on."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = []
    for pp in degrees:
        for pr in (hx.HX_FP32, hx.HX_FP64):
            G = None
            try:
                m, field, seed = I.workload_jittered_cube(pp)
                G = hx.Mesh(m, dict(I.MAT_CNH), device=device)
                X = G.node_coords().cpu().numpy()
                u = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
                if pr == hx.HX_FP32:
                    u = u.float()
                r = torch.empty_like(u)
                t = _event_ms(lambda: hx.hx_residual(G.ctx, G.handle, u, r), 20 if pr == hx.HX_FP32 else 4, 2)
                G.sync(60000)
                b = residual_bytes(G.n_dofs, G.n_qp, u.element_size())
                res.append({"p": pp, "prec": "f32" if pr == hx.HX_FP32 else "f64", "n_dofs": G.n_dofs,
                            "ms": round(t, 4), "gdofs": round(G.n_dofs / (t * 1e-3) / 1e9, 3),
                            "hbm_frac": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4)})
                del u, r
            except Exception as exc:  # recorded in the report; the headline line still prints
                res.append({"p": pp, "prec": "f32" if pr == hx.HX_FP32 else "f64", "error": str(exc)[:200]})
            finally:
                if G is not None:
                    G.close()
                torch.cuda.empty_cache()
    return res


def run_scatter_modes(device, p=4, steps=50):
    """The headline apply (32^3 jittered cube, FP32, spatial tensors, the
    autotuned variant) with the default atomic scatter and with the ordered,
    bitwise repeatable assembly (element buffer plus ordered node gather)."""
    import torch
    from paper_2408_12479_gb300 import hx
    G, m, u, du, out = build_case(p, hx.HX_FP32, hx.HX_SPATIAL_TENSORS, device)
    try:
        res = {"workload": f"cNH tangent apply, 32^3 jittered cube, p={p}, FP32, spatial tensors",
               "n_dofs": m.n_dofs, "tile_variant": G.tune[0]}
        for name, mode in (("atomic", hx.HX_SCATTER_ATOMIC), ("ordered", hx.HX_SCATTER_ORDERED)):
            hx.hx_set_scatter_mode(G.ctx, G.handle, mode)
            t = _event_ms(lambda: hx.hx_tangent_apply(G.ctx, G.handle, du, out), steps, 3)
            G.sync(60000)
            res[name] = {"ms": round(t, 4), "gdofs": round(m.n_dofs / (t * 1e-3) / 1e9, 3)}
        a = out.clone()
        hx.hx_tangent_apply(G.ctx, G.handle, du, out)
        res["ordered_repeats_bitwise"] = bool(torch.equal(a, out))
        return res
    finally:
        G.close()
        del u, du, out
        torch.cuda.empty_cache()


def run_newton_step_costs(device, p):
    """What each Newton step pays once (Alg. 1): hx_precompute_qp and
    hx_diagonal on the 32^3 jittered cube at degree p, per storage strategy and
    precision, in ms and in tangent applies of the same case."""
    import torch
    from paper_2408_12479_gb300 import hx
    res = []
    for pr in (hx.HX_FP32, hx.HX_FP64):
        for st in (hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS):
            G = None
            try:
                G, m, u, du, out = build_case(p, pr, st, device)
                t_apply = _event_ms(lambda: hx.hx_tangent_apply(G.ctx, G.handle, du, out), 10, 2)
                t_pre = _event_ms(lambda: G.precompute(u, pr, st), 5, 1)
                d = G.zeros(pr)
                t_diag = _event_ms(lambda: hx.hx_diagonal(G.ctx, G.handle, d), 5, 1)
                G.sync(60000)
                res.append({"p": p, "prec": "f32" if pr == hx.HX_FP32 else "f64",
                            "storage": hx.STORAGE_NAMES[st], "precompute_ms": round(t_pre, 4),
                            "diagonal_ms": round(t_diag, 4), "apply_ms": round(t_apply, 4),
                            "precompute_in_applies": round(t_pre / t_apply, 2),
                            "diagonal_in_applies": round(t_diag / t_apply, 2)})
                del u, du, out, d
            except Exception as exc:  # recorded in the report; the headline line still prints
                res.append({"p": p, "prec": "f32" if pr == hx.HX_FP32 else "f64",
                            "storage": hx.STORAGE_NAMES[st], "error": str(exc)[:200]})
            finally:
                if G is not None:
                    G.close()
                torch.cuda.empty_cache()
    return res


def run_batch(device, steps=20, storage=None):
    """64 cNH cubes of mixed size and degree (each with its own state) applied
    in one persistent launch per step, FP32, the given caching strategy."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    ctx = hx.hx_create(device)
    meshes, dus, outs = [], [], []
    for m, field, seed in I.workload_batch():
        G = hx.Mesh(m, dict(I.MAT_CNH), device=device, ctx=ctx)
        X = G.node_coords().cpu().numpy()
        G.precompute(torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device), hx.HX_FP32,
                     hx.HX_CACHE_F if storage is None else storage)
        meshes.append(G)
        dus.append(torch.tensor(I.random_direction(m.n_dofs, seed), dtype=torch.float32, device=G.device))
        outs.append(torch.empty_like(dus[-1]))
    batch = hx.hx_batch_create(ctx, meshes)
    for _ in range(3):
        hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        hx.hx_batch_tangent_apply(ctx, batch, dus, outs)
    e1.record()
    torch.cuda.synchronize()
    hx.hx_sync(ctx, 60000)
    ms = e0.elapsed_time(e1) / steps
    n_dofs = sum(G.n_dofs for G in meshes)
    name = hx.STORAGE_NAMES[hx.HX_CACHE_F if storage is None else storage]
    res = {"workload": f"64 cNH cubes, n ~ U{{8..24}}, p ~ U{{2..5}}, FP32, {name}, one persistent launch",
           "n_meshes": len(meshes), "n_dofs": n_dofs, "ms": round(ms, 4),
           "gdofs": round(n_dofs / (ms * 1e-3) / 1e9, 3),
           "degrees": sorted(set(G.input.p for G in meshes))}
    hx.hx_batch_destroy(batch)
    for G in meshes:
        G.close()
    hx.hx_destroy(ctx)
    return res


def run_batch_cg(device, n_meshes=64, tol=1e-8, max_iter=5000, degree=3, smoothing_range=15.0, storage=None,
                 strain=0.002):
    """The first n_meshes cubes of the 64-cube workload (cNH, n ~ U{8..24}, p ~ U{2..5}, each with its own
    sine state, here scaled to 0.2 % strain: clamped on x = 0, the finest cubes'
    tangents meet negative curvature at 1 % (and most cubes' at the workload's
    5 %), where CG cannot run; the single-mesh CG reports the same meshes),
    every cube clamped on x = 0: one FP64 CG per cube on
    K_i x_i = rhs_i with an FP32 Chebyshev(degree)-Jacobi preconditioner,
    all cubes in lockstep with one CUDA graph per iteration
    (hx_batch_cg_solve); then the same 64 solves one mesh at a time
    (hx_cg_solve) for comparison."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    st_ = hx.HX_SPATIAL_TENSORS if storage is None else storage
    ctx = hx.hx_create(device)
    meshes, rhss, batch = [], [], None
    res = {"workload": "%d of the 64 cNH cubes, n ~ U{8..24}, p ~ U{2..5}, %g %% sine states, clamped at x=0, "
                       "FP64 CG, FP32 Chebyshev(%d)-Jacobi, tol %g" % (n_meshes, 100 * strain, degree, tol)}
    try:
        for m, field, seed in I.workload_batch(n_meshes):
            n = m.box[0]
            m.dirichlet = I.box_dirichlet_x0(n, n, n, m.p)
            field.amp *= strain / 0.05
            G = hx.Mesh(m, dict(I.MAT_CNH), device=device, ctx=ctx)
            X = G.node_coords().cpu().numpy()
            u = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
            u[torch.tensor(m.dirichlet, device=G.device).bool()] = 0.0
            G.precompute(u, hx.HX_FP64, st_)
            G.precompute(u, hx.HX_FP32, st_)
            r = torch.tensor(I.random_direction(m.n_dofs, seed + 9), dtype=torch.float64, device=G.device)
            r[torch.tensor(m.dirichlet, device=G.device).bool()] = 0.0
            meshes.append(G)
            rhss.append(r)
        batch = hx.hx_batch_create(ctx, meshes)
        xs = [torch.zeros_like(r) for r in rhss]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, rels, st = hx.hx_batch_cg_solve(ctx, batch, rhss, xs, tol, max_iter, degree, smoothing_range, hx.HX_FP32)
        torch.cuda.synchronize()
        t_batch = time.perf_counter() - t0
        res["n_dofs"] = sum(G.n_dofs for G in meshes)
        broke = [i for i, r in enumerate(rels) if r != r]
        ok = [i for i, r in enumerate(rels) if r == r]
        res["batched"] = {"seconds": round(t_batch, 3), "status": hx.STATUS_NAMES.get(st, st),
                          "iters_min_max": [min(its), max(its)],
                          "max_true_rel_residual": max(rels[i] for i in ok) if ok else None,
                          "graph_iterations": max(its), "breakdowns": [[i, meshes[i].input.name] for i in broke]}
        # one mesh at a time, same preconditioner (the eigenvalue estimate as in the batch)
        t0 = time.perf_counter()
        its1, st1s = [], []
        for G, r in zip(meshes, rhss):
            dinv = 1.0 / G.diagonal(hx.HX_FP64)
            lam = hx.hx_estimate_lambda_max(G.ctx, G.handle, dinv, iters=20, seed=7)
            x = torch.zeros_like(r)
            try:
                it, rel, st1 = hx.hx_cg_solve(G.ctx, G.handle, r, x, tol, max_iter, degree, 1.2 * lam,
                                              smoothing_range, hx.HX_FP32)
            except hx.HxError as e:
                it, st1 = -1, e.status
            its1.append(it)
            st1s.append(st1)
        torch.cuda.synchronize()
        t_seq = time.perf_counter() - t0
        res["one_at_a_time"] = {"seconds": round(t_seq, 3), "iters_min_max": [min(its1), max(its1)],
                                "iterations_total": sum(i for i in its1 if i > 0),
                                "breakdowns": [i for i, s_ in enumerate(st1s) if s_ == hx.HX_ERR_NAN]}
        res["speedup_batched"] = round(t_seq / t_batch, 3)
    finally:
        if batch is not None:
            hx.hx_batch_destroy(batch)
        for G in meshes:
            G.close()
        hx.hx_destroy(ctx)
        torch.cuda.empty_cache()
    return res


def run_solve(device, n=48, p=4, tol=1e-8, max_iter=20000, degree=5, smoothing_range=15.0, J_target=0.9999,
              sine_amp=1e-5):
    """Newton-step solve on the compressed iNH cube (kappa = 1e3 mu): FP64 CG on
    K(u) du = -R(u) with a Chebyshev(degree)-Jacobi preconditioner applied in
    FP32 and, for comparison, in FP64; both stop at the same FP64 true-residual
    ratio. The state keeps the pressure below mu (J ~ 0.9999) so that K is
    positive definite; at J ~ 0.9 the pressure (~95 mu) makes rotation-dominated
    modes unstable and CG reports the non-positive curvature (recorded too)."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    m, field, seed = I.workload_compressed_cube(n=n, p=p, J_target=J_target, sine_amp=sine_amp)
    mat = dict(I.MAT_INH)
    G = hx.Mesh(m, mat, device=device)
    X = G.node_coords().cpu().numpy()
    u = torch.tensor(field(X).ravel(), dtype=torch.float64, device=G.device)
    G.precompute(u, hx.HX_FP64, hx.HX_CACHE_TENSORS)
    G.precompute(u, hx.HX_FP32, hx.HX_CACHE_TENSORS)
    r = G.residual(u)
    rhs = -r
    dinv = 1.0 / G.diagonal(hx.HX_FP64)
    lam = hx.hx_estimate_lambda_max(G.ctx, G.handle, dinv, iters=40, seed=7)
    G.sync(120000)
    res = {"workload": f"iNH kappa=1e3 mu, {n}^3 jittered cube, p={p}, J~{J_target}, symmetry clamps",
           "n_dofs": G.n_dofs, "lambda_max_est": lam, "lambda_max_used": 1.2 * lam, "degree": degree,
           "smoothing_range": smoothing_range, "tol": tol}
    for name, pp in (("fp32_precond", hx.HX_FP32), ("fp64_precond", hx.HX_FP64)):
        x = torch.zeros_like(u)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        it, rel, st = hx.hx_cg_solve(G.ctx, G.handle, rhs, x, tol, max_iter, degree, 1.2 * lam, smoothing_range, pp)
        torch.cuda.synchronize()
        res[name] = {"iterations": it, "true_rel_residual": rel, "seconds": round(time.perf_counter() - t0, 3),
                     "status": hx.STATUS_NAMES.get(st, st)}
    res["speedup_fp32_precond"] = round(res["fp64_precond"]["seconds"] / res["fp32_precond"]["seconds"], 3)
    # the same system with the hp-multigrid V-cycle (p-levels, then h-levels
    # and the coarse FP64 CG) as preconditioner
    mg = hx.Multigrid(G, smoother_degree=3, precond_prec=hx.HX_FP32, storage=hx.HX_CACHE_TENSORS, lambda_iters=20,
                      h_levels=10, coarse_cg_iters=200, coarse_cg_tol=1e-6)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg.setup(u)
        t_setup = time.perf_counter() - t0
        x = torch.zeros_like(u)
        t0 = time.perf_counter()
        it, rel, st = mg.cg_solve(rhs, x, tol, max_iter)
        torch.cuda.synchronize()
        res["hp_mg_fp32_precond"] = {"levels": mg.levels(), "iterations": it, "true_rel_residual": rel,
                                     "seconds": round(time.perf_counter() - t0, 3),
                                     "setup_seconds": round(t_setup, 3), "status": hx.STATUS_NAMES.get(st, st)}
    except hx.HxError as e:
        res["hp_mg_fp32_precond"] = {"status": str(e)[:160]}
    finally:
        mg.close()
    # and with the p-levels only (the degree-1 level smoothed by Chebyshev)
    mg = hx.Multigrid(G, smoother_degree=3, coarse_degree=20, coarse_range=200.0, precond_prec=hx.HX_FP32,
                      storage=hx.HX_CACHE_TENSORS, lambda_iters=20)
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mg.setup(u)
        t_setup = time.perf_counter() - t0
        x = torch.zeros_like(u)
        t0 = time.perf_counter()
        it, rel, st = mg.cg_solve(rhs, x, tol, max_iter)
        torch.cuda.synchronize()
        res["mg_fp32_precond"] = {"levels": mg.levels(), "iterations": it, "true_rel_residual": rel,
                                  "seconds": round(time.perf_counter() - t0, 3), "setup_seconds": round(t_setup, 3),
                                  "status": hx.STATUS_NAMES.get(st, st)}
    except hx.HxError as e:
        res["mg_fp32_precond"] = {"status": str(e)[:160]}
    finally:
        mg.close()
    G.close()
    # the literal J ~ 0.9 state: CG must stop with a non-positive-curvature status
    m9, f9, _ = I.workload_compressed_cube(n=n, p=p, J_target=0.9, sine_amp=0.005)
    G9 = hx.Mesh(m9, mat, device=device)
    u9 = torch.tensor(f9(G9.node_coords().cpu().numpy()).ravel(), dtype=torch.float64, device=G9.device)
    G9.precompute(u9, hx.HX_FP64, hx.HX_CACHE_TENSORS)
    G9.precompute(u9, hx.HX_FP32, hx.HX_CACHE_TENSORS)
    d9 = 1.0 / G9.diagonal(hx.HX_FP64)
    lam9 = hx.hx_estimate_lambda_max(G9.ctx, G9.handle, d9, iters=40, seed=7)
    try:
        it9, rel9, st9 = hx.hx_cg_solve(G9.ctx, G9.handle, -G9.residual(u9), torch.zeros_like(u9), tol, 200, degree,
                                        1.2 * lam9, smoothing_range, hx.HX_FP32)
        res["J0.9_state"] = {"status": hx.STATUS_NAMES.get(st9, st9), "iterations": it9}
    except hx.HxError as e:
        res["J0.9_state"] = {"status": str(e)[:120]}
    G9.close()
    return res


def run_solve_full(device, n=48, p=4, tol=1e-8, max_iter=500, J_target=0.9999, sine_amp=1e-5):
    """The compressed-cube solve at its full size (iNH, kappa = 1e3 mu, n^3
    jittered elements, p = 4, symmetry clamps): FP64 CG on K(u) du = -R(u)
    preconditioned by the hp-multigrid V-cycle (p 4 -> 2 -> 1, then h-levels
    down to the coarse FP64 CG) run in FP32 and, for comparison, in FP64;
    both stop at the same FP64 true-residual ratio. J ~ 0.9999 keeps K
    positive definite (at J ~ 0.9 the pressure makes CG meet negative
    curvature, see the 16^3 solve report). All levels and the outer operator
    use the spatial-tensor cache."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    m, field, seed = I.workload_compressed_cube(n=n, p=p, J_target=J_target, sine_amp=sine_amp)
    G = hx.Mesh(m, dict(I.MAT_INH), device=device)
    res = {"workload": f"iNH kappa=1e3 mu, {n}^3 jittered cube, p={p}, J~{J_target}, symmetry clamps",
           "n_dofs": m.n_dofs, "tol": tol}
    try:
        u = torch.tensor(field(G.node_coords().cpu().numpy()).ravel(), dtype=torch.float64, device=G.device)
        G.precompute(u, hx.HX_FP64, hx.HX_SPATIAL_TENSORS)
        rhs = -G.residual(u)
        for name, pp in (("hp_mg_fp32", hx.HX_FP32), ("hp_mg_fp64", hx.HX_FP64)):
            mg = hx.Multigrid(G, smoother_degree=3, precond_prec=pp, storage=hx.HX_SPATIAL_TENSORS, lambda_iters=20,
                              h_levels=10, coarse_cg_iters=200, coarse_cg_tol=1e-6)
            try:
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                mg.setup(u)
                t_setup = time.perf_counter() - t0
                x = torch.zeros_like(u)
                t0 = time.perf_counter()
                it, rel, st = mg.cg_solve(rhs, x, tol, max_iter)
                torch.cuda.synchronize()
                res[name] = {"iterations": it, "true_rel_residual": rel, "seconds": round(time.perf_counter() - t0, 3),
                             "setup_seconds": round(t_setup, 3), "status": hx.STATUS_NAMES.get(st, st),
                             "levels": ["p%d:%dx%dx%d" % mg.level(l) for l in range(len(mg.levels()))]}
            finally:
                mg.close()
        a, b = res.get("hp_mg_fp32", {}), res.get("hp_mg_fp64", {})
        if a.get("seconds") and b.get("seconds"):
            res["speedup_fp32_precond"] = round(b["seconds"] / a["seconds"], 3)
    finally:
        G.close()
        torch.cuda.empty_cache()
    return res


def run_newton_full(device, n=48, p_cube=4, J_target=0.9999, p_tube=3, steps_tube=4):
    """Newton's method (Alg. 1) end to end on the two full-size workloads.
    (1) The compressed cube as a boundary-value problem: iNH, kappa = 1e3 mu,
    n^3 jittered elements, p = 4, symmetry clamps and the far faces' normal
    displacements prescribed to J = 0.9999, from u = 0 inside; FP64 CG with
    the FP32 hp-multigrid; its exact solution is the homogeneous compression,
    against which the result is checked. (2) The fibre tube (16 x 8 x 64
    elements, p = 3, Q2 geometry) inflated by a dead inner pressure of 0.02 in
    load steps, mirror-plane constraints; FP64 CG with FP32 Chebyshev(5)-
    Jacobi."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = {}
    m, delta = I.workload_triaxial_compression(n=n, p=p_cube, J_target=J_target)
    G = hx.Mesh(m, dict(I.MAT_INH), device=device)
    mg = None
    try:
        rec = {"workload": f"iNH kappa=1e3 mu, {n}^3 jittered cube, p={p_cube}, triaxial compression to J={J_target}",
               "n_dofs": m.n_dofs}
        mg = hx.Multigrid(G, smoother_degree=3, precond_prec=hx.HX_FP32, storage=hx.HX_SPATIAL_TENSORS,
                          lambda_iters=20, h_levels=10, coarse_cg_iters=200, coarse_cg_tol=1e-6)
        X = G.node_coords().reshape(-1)
        exact = delta * X
        u = torch.where(torch.tensor(m.dirichlet, device=G.device).bool(), exact, torch.zeros_like(exact))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=1e-16, eps_rel=1e-10, max_newton=10,
                                     storage=hx.HX_SPATIAL_TENSORS, cg_tol=1e-8, cg_max_iter=500, mg=mg)
        torch.cuda.synchronize()
        rec.update({"seconds": round(time.perf_counter() - t0, 3), "status": hx.STATUS_NAMES.get(st, st),
                    "newton_iters": rep["newton_iters"], "cg_iters": rep["cg_iters"],
                    "final_res_rel": rep["res"] / max(rep["res0"], 1e-300),
                    "max_err_vs_closed_form_rel": float((u - exact).abs().max() / abs(delta)),
                    "levels": ["p%d:%dx%dx%d" % mg.level(l) for l in range(len(mg.levels()))]})
        res["cube"] = rec
    finally:
        if mg is not None:
            mg.close()
        G.close()
        torch.cuda.empty_cache()
    m, faces, pressure = I.workload_tube_inflation(p=p_tube)
    G = hx.Mesh(m, dict(I.MAT_FIBER), device=device)
    try:
        f = torch.tensor(hx.hx_traction_load(m, faces, pressure=pressure), dtype=torch.float64, device=G.device)
        X = G.node_coords().reshape(-1, 3)
        u = (1e-3 * X * torch.tensor([1.0, 1.0, 0.0], dtype=torch.float64, device=G.device)).reshape(-1)
        u[torch.tensor(m.dirichlet, device=G.device).bool()] = 0.0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, cg, st, rep = [], 0, hx.HX_OK, None
        for k in range(1, steps_tube + 1):
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, f * (k / steps_tube), eps_abs=1e-12, eps_rel=1e-10,
                                         max_newton=15, storage=hx.HX_SPATIAL_TENSORS, precond_prec=hx.HX_FP32,
                                         cg_tol=1e-8, cg_max_iter=20000)
            its.append(rep["newton_iters"])
            cg += rep["cg_iters"]
            if st != hx.HX_OK:
                break
        torch.cuda.synchronize()
        R = torch.hypot(X[:, 0], X[:, 1])
        U = u.reshape(-1, 3)
        u_r = (U[:, 0] * X[:, 0] + U[:, 1] * X[:, 1]) / R
        inner = R < 1.0 + 1e-9
        res["tube"] = {"workload": f"fibre tube 16x8x64, p={p_tube}, inner pressure {pressure} in {steps_tube} "
                                   f"load steps, mirror-plane constraints", "n_dofs": m.n_dofs,
                       "seconds": round(time.perf_counter() - t0, 3), "status": hx.STATUS_NAMES.get(st, st),
                       "newton_iters_per_step": its, "cg_iters": cg,
                       "final_res_rel": rep["res"] / max(rep["res0"], 1e-300),
                       "inner_radial_displacement_min_max": [float(u_r[inner].min()), float(u_r[inner].max())]}
    finally:
        G.close()
        torch.cuda.empty_cache()
    return res


def solve_summary(r):
    """The full-size solve's key figures for the headline line."""
    if not isinstance(r, dict) or "error" in r:
        return r
    out = {}
    for k in ("hp_mg_fp32", "hp_mg_fp64"):
        v = r.get(k, {})
        out[k] = [v.get("seconds"), v.get("iterations"), v.get("true_rel_residual")]
    out["speedup"] = r.get("speedup_fp32_precond")
    return out


def run_stability(device):
    """Forward-stability study (Sec. 7.1): 200 strain scales 1e-8..1e2, 1000
    samples each, FP32 vs FP64 with the stable and the standard forms, per
    law; reports every 20th scale of the relative-error curves of P and dP."""
    import math
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    from paper_2408_12479_gb300 import stability
    mats = {"cNH": dict(I.MAT_CNH), "iNH": dict(I.MAT_INH), "fiber": dict(I.MAT_FIBER)}
    t0 = time.perf_counter()
    out = {}
    for law, mat in mats.items():
        m = I.box_mesh(1, 1, name="point")
        if law == "fiber":
            m.frames = I.constant_frames(1)
        G = hx.Mesh(m, mat, device=device)
        res = stability.study(G, samples=1000)
        G.close()
        out[law] = {f: {"eps": [rec["eps"][i] for i in range(0, 200, 20)],
                        "P": [rec["P"][i] for i in range(0, 200, 20)],
                        "dP": [rec["dP"][i] for i in range(0, 200, 20)],
                        "max_P_eps_le_1e-2": max(x for e, x in zip(rec["eps"], rec["P"]) if e <= 1e-2),
                        "max_dP_eps_le_1e-2": max(x for e, x in zip(rec["eps"], rec["dP"]) if e <= 1e-2)}
                    for f, rec in res.items()}
        for f in out[law]:
            for k in ("P", "dP"):
                out[law][f][k] = [None if math.isnan(x) else float("%.3g" % x) for x in out[law][f][k]]
    out["seconds"] = round(time.perf_counter() - t0, 2)
    out["samples_per_scale"] = 1000
    out["scales"] = 200
    return out


def run_newton(device, n=8, p=4, stretch=1.1, steps=5):
    """Newton's method (Alg. 1) on uniaxial tension of an n^3 cube, p, cNH,
    reached in load steps; FP32- and FP64-preconditioned CG updates."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = {"workload": f"cNH uniaxial stretch {stretch} in {steps} load steps, {n}^3 cube, p={p}"}
    for name, pp in (("fp32_precond", hx.HX_FP32), ("fp64_precond", hx.HX_FP64), ("mg_fp32_precond", hx.HX_FP32)):
        m, _ = I.workload_uniaxial(n, p, 1.0)
        G = hx.Mesh(m, dict(I.MAT_CNH), device=device)
        mg = hx.Multigrid(G, precond_prec=hx.HX_FP32, storage=hx.HX_SPATIAL_TENSORS) if name.startswith("mg") else None
        X = G.node_coords()
        inc = torch.zeros_like(X)
        inc[:, 0] = (stretch - 1.0) / steps * X[:, 0]
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device=G.device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, cg = [], 0
        for _ in range(steps):
            u += inc.reshape(-1)
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, None, eps_abs=1e-12, eps_rel=1e-9, max_newton=15,
                                         storage=hx.HX_SPATIAL_TENSORS, precond_prec=pp, cg_tol=1e-6,
                                         cg_max_iter=20000, mg=mg)
            its.append(rep["newton_iters"])
            cg += rep["cg_iters"]
        torch.cuda.synchronize()
        res["n_dofs"] = m.n_dofs
        res[name] = {"newton_iters_per_step": its, "cg_iters": cg, "seconds": round(time.perf_counter() - t0, 3),
                     "final_res_rel": rep["res"] / max(rep["res0"], 1e-300), "status": hx.STATUS_NAMES.get(st, st)}
        if mg is not None:
            res[name]["levels"] = mg.levels()
            mg.close()
        G.close()
    return res


def run_newton_traction(device, n=8, p=4, traction=(0.0, 0.0, -0.02), steps=4):
    """Newton's method (Alg. 1) under a Neumann load: an n^3 jittered cNH
    cube clamped on x = 0 with a dead traction on x = 1 (a cantilever), the
    load applied in `steps` equal steps; f_ext from hx_traction_load, updates
    by FP32-preconditioned CG. Reports the iterations, the relative residual
    of the last step and the mean deflection of the loaded face."""
    import torch
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I
    res = {"workload": f"cNH cantilever, {n}^3 jittered cube clamped at x=0, traction {list(traction)} on x=1, "
                       f"p={p}, {steps} load steps"}
    G = None
    try:
        m = I.box_mesh(n, p, jitter=0.1, seed=I.SEED_BASE + 6, clamp=True)
        f = hx.hx_traction_load(m, I.box_boundary_faces(n, n, n, 1), traction=traction)
        G = hx.Mesh(m, dict(I.MAT_CNH), device=device)
        X = G.node_coords()
        f_dev = torch.tensor(f, dtype=torch.float64, device=G.device)
        u = torch.zeros(m.n_dofs, dtype=torch.float64, device=G.device)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, cg, st, rep = [], 0, hx.HX_OK, None
        for k in range(1, steps + 1):
            rep, st = hx.hx_newton_solve(G.ctx, G.handle, u, f_dev * (k / steps), eps_abs=1e-14, eps_rel=1e-9,
                                         max_newton=15, storage=hx.HX_SPATIAL_TENSORS, precond_prec=hx.HX_FP32,
                                         cg_tol=1e-6, cg_max_iter=20000)
            its.append(rep["newton_iters"])
            cg += rep["cg_iters"]
            if st != hx.HX_OK:
                break
        torch.cuda.synchronize()
        face = (X[:, 0] - X[:, 0].max()).abs() < 1e-12
        res.update({"n_dofs": m.n_dofs, "newton_iters_per_step": its, "cg_iters": cg,
                    "seconds": round(time.perf_counter() - t0, 3),
                    "final_res_rel": rep["res"] / max(rep["res0"], 1e-300), "status": hx.STATUS_NAMES.get(st, st),
                    "mean_face_deflection": [round(float(v), 8) for v in u.view(-1, 3)[face].mean(dim=0)]})
    except Exception as exc:  # recorded in the report; the headline line still prints
        res["error"] = str(exc)[:200]
    finally:
        if G is not None:
            G.close()
    return res


def host_cores() -> int:
    """Host cores this process may run on (launchers such as torchrun set
    OMP_NUM_THREADS=1 per rank; the CPU legs run on rank 0 alone and use all
    cores)."""
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def strict(o):
    """o with every non-finite float replaced by None (and numpy scalars by
    Python numbers), so that json.dumps(..., allow_nan=False) accepts it."""
    if isinstance(o, (float, np.floating)):
        return float(o) if math.isfinite(o) else None
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, dict):
        return {k: strict(v) for k, v in o.items()}
    if isinstance(o, (list, tuple)):
        return [strict(v) for v in o]
    return o


def emit(obj):
    """Print one strict-JSON line."""
    print(json.dumps(strict(obj), allow_nan=False), flush=True)


def guarded(fn, *a, **k):
    """fn(*a, **k), or {"error": ...} if it raises: a failing side report is
    recorded and the headline line still prints."""
    try:
        return fn(*a, **k)
    except Exception as exc:  # recorded in the report
        return {"error": f"{type(exc).__name__}: {str(exc)[:200]}"}


def reps_per_step(apply_ms, steps, target_s=1.2):
    """Applies per timed step so that `steps` steps last at least target_s
    (the paper's protocol repeats an operation until a second has passed)."""
    return max(1, int(math.ceil(target_s * 1e3 / (max(steps, 1) * max(apply_ms, 1e-6)))))


def sweep_summary(sweep):
    """Best storage strategy per (precision, degree) of the sweep:
    {prec: {p: [GDoF/s, HBM fraction, FMA-pipe fraction, strategy]}}."""
    out = {}
    for r in sweep or []:
        if "gdofs" not in r:
            continue
        cur = out.setdefault(r["prec"], {}).get(str(r["p"]))
        if cur is None or r["gdofs"] > cur[0]:
            out[r["prec"]][str(r["p"])] = [r["gdofs"], r["hbm_frac"], r.get("fma_frac"),
                                           {"recompute": "R", "cache_F": "F", "cache_tensors": "T",
                                            "spatial_tensors": "S"}.get(r["storage"], r["storage"])]
    return out


HEADLINE_KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                 "scaling", "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks",
                 "cpu_baseline", "fma_peaks", "sweep_best", "solve_48")


def headline_line(fields):
    """The final stdout line: the contract's keys only (side reports go on
    earlier lines), strict JSON."""
    line = {k: fields.get(k) for k in HEADLINE_KEYS}
    return json.dumps(strict(line), allow_nan=False)


def cpu_baseline(m, field, seed, p, mat_d, target_s=10.0):
    """The FP64 oracle's full-tensor apply over the whole mesh, on all host
    cores, repeated until target_s has passed (at least once)."""
    from oracle import oracle as O
    O.set_threads(host_cores())
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = field(X).ravel()
    from paper_2408_12479_gb300 import inputs as I
    du = I.random_direction(m.n_dofs, seed + 3)
    mat = O.Material.from_dict(mat_d)
    reps = 0
    t0 = time.perf_counter()
    while True:
        O.apply(M, mat, u, du)
        reps += 1
        dt = time.perf_counter() - t0
        if dt >= target_s:
            break
    return {"value": m.n_dofs * reps / dt / 1e9, "unit": "GDoF/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{reps} FP64 full-tensor oracle applies of the whole mesh ({m.n_elem} elements) in {dt:.1f} s"}


def run_reference(args, budget_s=150.0):
    """Reference arm: the FP64 CPU oracle, timed as it stands on the host
    cores. Each step applies the whole mesh; only if K + W whole-mesh steps
    would take longer than budget_s does a step apply the leading elements
    instead (the line then names that sample). ms_per_step is the measured
    time of the work one step does."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_2408_12479_gb300 import inputs as I
    O.set_threads(host_cores())
    p = args.p
    m, field, seed = I.workload_jittered_cube(p)
    mat_d = dict(I.MAT_CNH)
    M = O.OracleMesh(m)
    X = O.node_coords(M)
    u = field(X).ravel()
    du = I.random_direction(m.n_dofs, seed + 3)
    mat = O.Material.from_dict(mat_d)
    k_probe = min(m.n_elem, 256)
    t0 = time.perf_counter()
    O.apply(M, mat, u, du, elems=np.arange(k_probe, dtype=np.int32))
    per_elem = (time.perf_counter() - t0) / k_probe
    n_run = args.steps + args.warmup
    k = m.n_elem if n_run * per_elem * m.n_elem <= budget_s else max(8, int(budget_s / n_run / per_elem))
    elems = None if k >= m.n_elem else np.arange(k, dtype=np.int32)
    for _ in range(args.warmup):
        O.apply(M, mat, u, du, elems=elems)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.apply(M, mat, u, du, elems=elems)
    dt = (time.perf_counter() - t0) / max(args.steps, 1)
    dofs = m.n_dofs if elems is None else m.n_dofs * k / m.n_elem
    gdofs = dofs / dt / 1e9
    sample = ("the whole mesh per step" if elems is None else
              f"the first {k} of {m.n_elem} elements per step ({dofs:.0f} DoFs by element fraction)")
    line = {"impl": "reference", "metric": METRIC, "value": gdofs, "unit": "GDoF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": f"cNH tangent apply, 32^3 jittered cube, p={p}", "p": p,
                                            "n_dofs": m.n_dofs, "law": "cNH", "prec": "f64",
                                            "storage": "none (full-tensor oracle)", "step": sample},
            "cpu_baseline": {"value": gdofs, "unit": "GDoF/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": gdofs, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(line)


def run_sweep(local, hbm_peak, peaks_fp):
    """Tangent apply on the 32^3 jittered cube, p = 2..6 x FP32/FP64 x every
    storage strategy (autotuned variant), with HBM and FMA-pipe fractions."""
    import torch
    from paper_2408_12479_gb300 import hx
    sweep = []
    for pp in (2, 3, 4, 5, 6):
        for pr in (hx.HX_FP32, hx.HX_FP64):
            for st in (hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS):
                rec = {"p": pp, "prec": "f32" if pr else "f64", "storage": hx.STORAGE_NAMES[st]}
                Gs = None
                try:
                    Gs, ms_, us, dus, outs = build_case(pp, pr, st, local)
                    reps = 30 if pr == hx.HX_FP32 else 5
                    t = time_steps(Gs, dus, outs, reps, 2)
                    b = Gs.apply_bytes(st, pr)
                    tf, pf = pipe_fraction(ms_.n_elem, pp, t, rec["prec"], peaks_fp)
                    rec.update({"sweep_tflops": tf, "fma_frac": pf, "n_dofs": ms_.n_dofs, "ms": round(t, 4),
                                "gdofs": round(ms_.n_dofs / (t * 1e-3) / 1e9, 3), "tile_variant": Gs.tune[0],
                                "variant_ms": [round(x, 4) for x in Gs.tune[1]],
                                "hbm_frac": round(b / (t * 1e-3) / 1e9 / hbm_peak, 4)})
                    del us, dus, outs
                except Exception as exc:  # recorded; the sweep goes on
                    rec["error"] = str(exc)[:200]
                finally:
                    if Gs is not None:
                        Gs.close()
                    torch.cuda.empty_cache()
                sweep.append(rec)
    return sweep


def run_profile_op(args):
    """One operator on the benchmark's mesh (32^3 jittered cube, --p, --prec,
    --storage; the autotuned apply variant unless --variant is given), run
    --warmup + --steps times: the command the committed ncu summaries of the
    individual kernels were taken with. Prints one short line, no contract."""
    import torch
    from paper_2408_12479_gb300 import hx
    names = {v: k for k, v in hx.STORAGE_NAMES.items()}
    prec = hx.HX_FP32 if args.prec == "f32" else hx.HX_FP64
    storage = names["spatial_tensors" if args.storage == "best" else args.storage]
    G, m, u, du, out = build_case(args.p, prec, storage, 0)
    if args.variant >= 0:
        hx.hx_set_apply_variant(G.ctx, G.handle, prec, storage, args.variant)
    up = u if prec == hx.HX_FP64 else u.float()
    d = G.zeros(prec)
    ops = {"apply": lambda: hx.hx_tangent_apply(G.ctx, G.handle, du, out),
           "residual": lambda: hx.hx_residual(G.ctx, G.handle, up, out),
           "precompute": lambda: G.precompute(u, prec, storage),
           "diagonal": lambda: hx.hx_diagonal(G.ctx, G.handle, d)}
    torch.cuda.nvtx.range_push("timed")  # profilers restrict capture to this range
    ms = _event_ms(ops[args.profile_op], max(args.steps, 1), args.warmup)
    torch.cuda.nvtx.range_pop()
    G.sync(60000)
    print(json.dumps({"profile_op": args.profile_op, "p": args.p, "prec": args.prec,
                      "storage": hx.STORAGE_NAMES[storage], "variant": args.variant if args.variant >= 0 else G.tune[0],
                      "ms": round(ms, 4)}))
    G.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="hx")
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--no-sweep", action="store_true", help="headline only (no side reports)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--storage", default="best", choices=["best", "recompute", "cache_F", "cache_tensors", "spatial_tensors"])
    ap.add_argument("--prec", default="f32", choices=["f32", "f64"])
    ap.add_argument("--min-seconds", type=float, default=1.2, help="least length of the timed region")
    ap.add_argument("--profile-op", default=None, choices=["apply", "residual", "precompute", "diagonal"],
                    help="run one operator --warmup + --steps times for a profiler and exit (no contract line)")
    ap.add_argument("--variant", type=int, default=-1,
                    help="pin the apply variant (0-5) instead of the autotuner's (profiling commands)")
    ap.add_argument("--solve-full", type=int, default=48,
                    help="the compressed-cube solve at full size with the hp-multigrid preconditioner (n given; 0: off)")
    ap.add_argument("--no-newton-full", dest="newton_full", action="store_false",
                    help="skip Newton's method on the full-size compressed cube and fibre tube")
    ap.add_argument("--batch-cg", type=int, default=16,
                    help="batched CG over the first n cubes of the 64-cube workload, and one at a time (0: off)")
    ap.add_argument("--solve", type=int, default=16,
                    help="also run the FP32- vs FP64-preconditioned CG solve on an n^3 compressed cube (n given)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile_op:
        run_profile_op(args)
        return

    import torch
    import torch.distributed as dist
    from paper_2408_12479_gb300 import hx
    from paper_2408_12479_gb300 import inputs as I

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    hbm_peak, peak_kind = peaks()

    p = args.p
    prec = hx.HX_FP32 if args.prec == "f32" else hx.HX_FP64
    # pick the fastest storage strategy on a short run (or take the given one)
    best = None
    per_storage = {}
    names = {v: k for k, v in hx.STORAGE_NAMES.items()}
    cands = (hx.HX_RECOMPUTE, hx.HX_CACHE_F, hx.HX_CACHE_TENSORS, hx.HX_SPATIAL_TENSORS) if args.storage == "best" else (names[args.storage],)
    for storage in cands:
        if len(cands) == 1:
            best = (storage, None)
            break
        G, m, u, du, out = build_case(p, prec, storage, local)
        ms = time_steps(G, du, out, 20, 3)
        per_storage[hx.STORAGE_NAMES[storage]] = ms
        if best is None or ms < best[1]:
            best = (storage, ms)
        G.close()
        del u, du, out
        torch.cuda.empty_cache()
    storage = best[0]
    G, m, u, du, out = build_case(p, prec, storage, local)
    if args.variant >= 0:  # a pinned variant (profiling commands), instead of the autotuner's
        hx.hx_set_apply_variant(G.ctx, G.handle, prec, storage, args.variant)
        G.tune = (args.variant, G.tune[1])
    n_dofs = m.n_dofs
    bytes_alg = G.apply_bytes(storage, prec)
    # applies per timed step: the K steps last at least --min-seconds
    R = reps_per_step(time_steps(G, du, out, 50, 5), args.steps, args.min_seconds)
    if world > 1:  # every rank runs the same R (the slowest rank's choice)
        R = int(round(max_over_ranks(float(R), world)))

    def step():
        for _ in range(R):
            hx.hx_tangent_apply(G.ctx, G.handle, du, out)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    hx.hx_launch_count(G.ctx, reset=True)
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_push("timed")  # profilers can restrict capture to this range
        e0.record(s)
        for _ in range(args.steps):
            step()
        e1.record(s)
        torch.cuda.nvtx.range_pop()
        torch.cuda.synchronize()
    launches = hx.hx_launch_count(G.ctx)
    G.sync(60000)
    ms_step = e0.elapsed_time(e1) / args.steps
    t_max = max_over_ranks(ms_step, world)
    if world > 1:
        dist.barrier()
    value = weak_value(n_dofs * R, t_max, world)
    ms_apply = ms_step / R
    achieved = bytes_alg / (ms_apply * 1e-3) / 1e9

    # end to end through the host-buffer C-ABI call (pinned host vectors)
    bytes_vec = n_dofs * du.element_size()
    e2e = None
    if not args.no_e2e:
        du_h = du.cpu().pin_memory()
        out_h = torch.empty_like(du_h).pin_memory()
        k_e2e = max(5, min(args.steps, 50))

        def host_rate(slabs):
            hx.hx_set_host_apply_slabs(G.ctx, G.handle, slabs)
            for _ in range(2):
                hx.hx_tangent_apply_host(G.ctx, G.handle, du_h, out_h, prec)
            t0 = time.perf_counter()
            for _ in range(k_e2e):
                hx.hx_tangent_apply_host(G.ctx, G.handle, du_h, out_h, prec)
            return n_dofs / ((time.perf_counter() - t0) / k_e2e) / 1e9

        whole = host_rate(0)
        e2e = {"value": round(host_rate(1), 4), "unit": "GDoF/s", "h2d_bytes_per_step": bytes_vec,
               "d2h_bytes_per_step": bytes_vec, "steps": k_e2e,
               "path": "hx_tangent_apply_host, pinned host vectors, z-slabs with overlapped copies",
               "whole_vector_copies": round(whole, 4)}
    tune = G.tune
    G.close()
    del u, du, out
    torch.cuda.empty_cache()

    peaks_fp = sweep = solve_full = None
    if rank == 0 and not args.no_sweep:
        peaks_fp = fma_peaks(local)
        sweep = run_sweep(local, hbm_peak, peaks_fp)
        emit({"report": "sweep", "fma_peaks": peaks_fp, "cases": sweep})
        emit({"report": "residual", "cases": guarded(run_residual_sweep, local, hbm_peak)})
        emit({"report": "newton_step_costs", "cases": guarded(run_newton_step_costs, local, p)})
        emit({"report": "scatter_modes", **guarded(run_scatter_modes, local, p)})
        emit({"report": "fp32_error", **guarded(run_fp32_errors, local)})
        emit({"report": "law_workloads", "cases": guarded(run_law_workloads, local, hbm_peak)})
        emit({"report": "batch", "cache_F": guarded(run_batch, local, storage=hx.HX_CACHE_F),
              "spatial_tensors": guarded(run_batch, local, storage=hx.HX_SPATIAL_TENSORS)})
        if args.batch_cg:
            emit({"report": "batch_cg", **guarded(run_batch_cg, local, n_meshes=args.batch_cg)})
        if args.solve:
            emit({"report": "solve", **guarded(run_solve, local, n=args.solve)})
        if args.solve_full:
            solve_full = guarded(run_solve_full, local, n=args.solve_full)
            emit({"report": "solve_full", **solve_full})
        newton = guarded(run_newton, local)
        newton["traction"] = guarded(run_newton_traction, local)
        emit({"report": "newton", **newton})
        if args.newton_full:
            emit({"report": "newton_full", **guarded(run_newton_full, local)})
        emit({"report": "stability", **guarded(run_stability, local)})
        emit({"report": "paper_context", **PAPER_CONTEXT})

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        m2, field, seed = I.workload_jittered_cube(p)
        cpu = guarded(cpu_baseline, m2, field, seed, p, dict(I.MAT_CNH))

    if rank == 0:
        fields = {
            "metric": METRIC, "value": round(value, 4), "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(t_max, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.prec, "data": "synthetic",
            "config": {"workload": f"cNH tangent apply, 32^3 jittered cube, p={p}",
                       "p": p, "n_dofs": n_dofs, "law": "cNH", "prec": args.prec,
                       "storage": hx.STORAGE_NAMES[storage], "applies_per_step": R,
                       "ms_per_apply": round(ms_apply, 5),
                       "l2": "inputs %.0f MB > L2 129 MB" % (bytes_alg / 1e6),
                       "per_storage_ms": {k: round(v, 4) for k, v in per_storage.items() if v},
                       "tile_variant": tune[0]},
            "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                         "frac": round(achieved / hbm_peak, 4),
                         "traffic": measured_traffic(p, args.prec, hx.STORAGE_NAMES[storage]),
                         "peak_kind": peak_kind, "bytes_per_launch": bytes_alg,
                         "duration": "events over the timed steps / applies (zeroing + apply)"},
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "cpu_baseline": cpu,
            "fma_peaks": peaks_fp,
            "sweep_best": sweep_summary(sweep),
            "solve_48": solve_summary(solve_full),
        }
        print(headline_line(fields), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
