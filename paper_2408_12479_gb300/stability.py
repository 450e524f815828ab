"""Forward-stability study of Sec. 7.1 on the GPU.

Displacement gradients G are sampled with every component uniform in
[eps/10, eps] with a random sign, for scales eps from 1e-8 to 1e2; at each
scale the law's S, P and directional derivative dP (direction H sampled the
same way at unit scale) are evaluated in FP64 and in FP32 with the same
formulation -- the stable forms (with exact or Alg. 2 J^-2/3) or the standard
forms -- and the relative error of the FP32 result is the largest, over the
samples, of max_ij |T32_ij - T64_ij| / max_ij |T64_ij|. Samples with
det(I + G) <= 0 (not deformations; frequent from eps ~ 1 on) are skipped and
counted.
"""
from __future__ import annotations

import numpy as np

from . import hx

FORMS = {0: "stable", 1: "stable_fastJ", 2: "standard"}


def sample_gradients(n: int, eps: float, rng: np.random.Generator) -> np.ndarray:
    """[n, 3, 3] tensors with |G_ij| uniform in [eps/10, eps], random sign."""
    mag = rng.uniform(eps / 10.0, eps, size=(n, 3, 3))
    sign = np.where(rng.random((n, 3, 3)) < 0.5, -1.0, 1.0)
    return mag * sign


def rel_error(lo, ref, valid):
    """Largest over the valid samples of the normwise relative error per
    sample (NaN if no sample is valid)."""
    num = (lo - ref).abs().reshape(lo.shape[0], -1).amax(dim=1)
    den = ref.abs().reshape(ref.shape[0], -1).amax(dim=1)
    e = (num / den)[valid]
    return float(e.max()) if e.numel() else float("nan")


def study(mesh, scales=None, samples=1000, seed=2024, forms=(0, 1, 2)):
    """Relative FP32 errors of S, P and dP per scale and form on the mesh's
    law (fibre tensors of element 0). Returns {form: {"eps": [...], "S": [...],
    "P": [...], "dP": [...]}}."""
    import torch
    scales = np.logspace(-8, 2, 200) if scales is None else np.asarray(scales, dtype=np.float64)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {FORMS[f]: {"eps": [], "S": [], "P": [], "dP": [], "valid": []} for f in forms}
    for eps in scales:
        G = torch.tensor(sample_gradients(samples, eps, rng), device=mesh.device)
        H = torch.tensor(sample_gradients(samples, 1.0, rng), device=mesh.device)
        # FP32 runs see the inputs rounded to FP32; the FP64 reference uses the same rounded values
        G = G.float().double()
        H = H.float().double()
        # samples with det(I + G) <= 0 are not deformations; they are skipped
        jac = torch.linalg.det(torch.eye(3, dtype=torch.float64, device=G.device) + G)
        for f in forms:
            ref = hx.hx_material_eval(mesh.ctx, mesh.handle, G, H, hx.HX_FP64, form=f)
            lo = hx.hx_material_eval(mesh.ctx, mesh.handle, G, H, hx.HX_FP32, form=f)
            valid = (jac > 0) & torch.isfinite(ref[1]).reshape(samples, -1).all(dim=1) & \
                torch.isfinite(ref[2]).reshape(samples, -1).all(dim=1)
            rec = out[FORMS[f]]
            rec["eps"].append(float(eps))
            rec["valid"].append(int(valid.sum()))
            for name, a, b in zip(("S", "P", "dP"), lo, ref):
                rec[name].append(rel_error(a, b, valid))
    return out
