"""The no-allocation Chebyshev-Jacobi smoother.

hx_chebyshev_smooth_noalloc serves callers that cannot allocate device memory
while running (an application whose memory another framework's caching
allocator has reserved, or a latency-critical loop where cudaMalloc would
synchronise the device): its scratch vectors live in a static device array of
the library instead of mesh workspace. This file is collected last so that a
run stopping at the first failure has already run every other test; it also
passes on its own in a fresh process.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2408_12479_gb300 import hx
from paper_2408_12479_gb300 import inputs as I
from tests import cases

pytestmark = pytest.mark.gpu

MAX_DOFS = 1 << 20


def _smoother_case(prec):
    dt = torch.float64 if prec == hx.HX_FP64 else torch.float32
    m = cases.small_cube(3, 3, "iNH", seed=401, clamp=True)
    M, X, u = cases.state_for(m, "iNH", seed=402, strain=0.01)
    u[M.dirichlet] = 0.0
    G = hx.Mesh(m, cases.MATS["iNH"])
    G.precompute(torch.tensor(u, dtype=torch.float64, device="cuda"), prec, hx.HX_CACHE_TENSORS)
    dinv = 1.0 / G.diagonal(prec)
    rhs = torch.tensor(I.random_direction(m.n_dofs, 403), dtype=dt, device="cuda")
    rhs[torch.tensor(M.dirichlet, device="cuda")] = 0.0
    x0 = 0.1 * torch.tensor(I.random_direction(m.n_dofs, 404), dtype=dt, device="cuda")
    return G, rhs, dinv, x0


@pytest.mark.parametrize("prec,tol", [(hx.HX_FP64, 1e-12), (hx.HX_FP32, 1e-5)])
@pytest.mark.parametrize("zero_initial", [False, True])
def test_noalloc_matches_allocating_smoother(prec, tol, zero_initial):
    G, rhs, dinv, x0 = _smoother_case(prec)
    try:
        ref = x0.clone()
        hx.hx_chebyshev_smooth(G.ctx, G.handle, rhs, ref, dinv, 5, 2.0, 15.0, zero_initial)
        scale = ref.abs().max().item()
        for _ in range(2):  # two calls in a row share the static scratch array
            x = x0.clone()
            hx.hx_chebyshev_smooth_noalloc(G.ctx, G.handle, rhs, x, dinv, 5, 2.0, 15.0, zero_initial)
            G.sync(60000)
            assert (x - ref).abs().max().item() <= tol * scale
    finally:
        G.close()


def test_noalloc_rejects_meshes_beyond_the_limit():
    m = I.box_mesh(24, 2)  # 3 * 49^3 = 352,947 DoFs: within the limit
    n_ok = 3 * m.n_nodes
    assert n_ok <= MAX_DOFS
    big = I.box_mesh(24, 3)  # 3 * 73^3 = 1,166,913 DoFs: over the limit
    assert 3 * big.n_nodes > MAX_DOFS
    G = hx.Mesh(big, cases.MATS["cNH"])
    try:
        v = G.zeros()
        with pytest.raises(hx.HxError) as e:
            hx.hx_chebyshev_smooth_noalloc(G.ctx, G.handle, v, torch.zeros_like(v), torch.ones_like(v), 2, 2.0, 15.0)
        assert e.value.status == hx.HX_ERR_ARG
        assert "1048576" in str(e.value)
    finally:
        G.close()


def _large_case(prec):
    """A 24^3 Q2 cube (352,947 DoFs): the allocating smoother's workspace
    (two vectors, 5.6 MB in FP64) is larger than the device's allocation
    granularity, so cudaMemGetInfo sees it."""
    dt = torch.float64 if prec == hx.HX_FP64 else torch.float32
    m, field, seed = I.workload_jittered_cube(2, n=24)
    G = hx.Mesh(m, cases.MATS["cNH"])
    X = G.node_coords().cpu().numpy()
    G.precompute(torch.tensor(field(X).ravel(), dtype=torch.float64, device="cuda"), prec, hx.HX_CACHE_TENSORS)
    dinv = 1.0 / G.diagonal(prec)
    rhs = torch.tensor(I.random_direction(m.n_dofs, seed + 5), dtype=dt, device="cuda")
    x = torch.zeros_like(rhs)
    return G, rhs, dinv, x


def test_noalloc_call_allocates_nothing():
    """On a mesh whose smoother workspace does not exist yet, the no-allocation
    call leaves the device's free memory as it was; the allocating smoother on
    the same mesh then takes its workspace, so the measurement does see an
    allocation of that size."""
    prec = hx.HX_FP64
    # first call in this process: the array's address lookup and the loading
    # of the kernels that the call launches happen here, not in the measured call
    G0, rhs0, dinv0, x00 = _large_case(prec)
    try:
        hx.hx_chebyshev_smooth_noalloc(G0.ctx, G0.handle, rhs0, x00, dinv0, 3, 2.0, 15.0, 0)
        G0.sync(60000)
    finally:
        G0.close()
    G, rhs, dinv, x = _large_case(prec)
    try:
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        dev0 = torch.cuda.current_device()
        hx.hx_chebyshev_smooth_noalloc(G.ctx, G.handle, rhs, x, dinv, 3, 2.0, 15.0, 0)
        G.sync(60000)
        torch.cuda.synchronize()
        free1 = torch.cuda.mem_get_info()[0]
        assert free1 == free0
        assert torch.cuda.current_device() == dev0
        ref = torch.zeros_like(x)
        hx.hx_chebyshev_smooth(G.ctx, G.handle, rhs, ref, dinv, 3, 2.0, 15.0, 0)
        G.sync(60000)
        torch.cuda.synchronize()
        free2 = torch.cuda.mem_get_info()[0]
        work = 2 * G.n_dofs * 8
        assert free0 - free2 >= work - (2 << 20)
        assert (x - ref).abs().max().item() <= 1e-12 * ref.abs().max().item()
    finally:
        G.close()
