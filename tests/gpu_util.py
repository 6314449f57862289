"""Shared helpers of the GPU parity tests: the CUDA path through the C ABI on
one side, the FP64 oracle on the other, fed the same seeded inputs."""
import numpy as np
import pytest

import oracle


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2302_08341_gb300 import capi
    return capi


def oracle_params(capi_params, ny, nx):
    p = capi_params
    return oracle.Params(ny=ny, nx=nx, dx=p.dx, g=p.g, alpha=p.alpha, dt_cap=p.dt_cap,
                         dt_fixed=p.dt_fixed, h_eps=p.h_eps, h_floor=p.h_floor,
                         rain_block=p.rain_block, edge_slope=p.edge_slope, limiter=p.limiter,
                         east_outflow=p.east_outflow, south_outflow=p.south_outflow)


def gpu_links_to_oracle(qx, qy):
    """GPU layout (link east / south of each cell) -> oracle's full link
    arrays with the west / north wall links."""
    ny, nx = qx.shape
    ox = np.zeros((ny, nx + 1)); ox[:, 1:] = qx
    oy = np.zeros((ny + 1, nx)); oy[1:, :] = qy
    return ox, oy


def oracle_member_from_gpu(h, qx, qy, t=0.0):
    ox, oy = gpu_links_to_oracle(qx, qy)
    return oracle.Member(h=np.array(h, np.float64), qx=ox, qy=oy, t=t)


def compare(gpu, ref, tol):
    err = float(np.max(np.abs(np.asarray(gpu, np.float64) - ref))) if np.size(ref) else 0.0
    assert err <= tol, f"max |diff| {err:.3e} > {tol:.1e}"
    return err
