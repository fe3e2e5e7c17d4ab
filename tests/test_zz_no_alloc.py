"""lbm_step_noalloc: the allocation-free single step.

Callers that cannot allocate device memory (code running under CUDA graph
capture, plugins whose host application owns every allocation, real-time loops
that must not stall in an allocator) step a lattice from their own state
buffers with this entry point. Here it is checked, through the C-ABI, against
the handle-based lbm_step on the same state, for two calls in a row (the
second call reads what the first one wrote, and both reuse the same built-in
scratch array). This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2403_16122_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-6  # the tolerance the layout-equivalence tests use


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2403_16122_gb300 import build, lbm

    build.build()
    lbm.load()
    return torch, lbm


def _to_device(torch, pops, aux, L, pitch):
    """Host state (27 population planes with h_0 unshifted, 5 carried planes;
    doubles) -> device buffers in the library's grouped FP32 layout: the
    population buffer as 8 planes of (g_i, h_i) pairs then 8 planes of f_i,
    the own-site buffer as (g_0, h_0 - L f_l, f_0, f_l) then
    ((phi u)_x, (phi u)_y, p, S) per site; rows of `pitch` sites."""
    ny, nx = pops.shape[1:]
    P = np.zeros((24, ny, pitch), np.float32)
    A = np.zeros((8, ny, pitch), np.float32)
    P4 = P[:16].reshape(8, ny, pitch, 2)  # pair planes viewed as (i, y, x, g/h)
    for i in range(1, 9):
        P4[i - 1, :, :nx, 0] = pops[i]
        P4[i - 1, :, :nx, 1] = pops[9 + i]
        P[15 + i, :, :nx] = pops[18 + i]
    O = A.reshape(2, ny, pitch, 4)
    O[0, :, :nx, 0] = pops[0]
    O[0, :, :nx, 1] = pops[9] - L * aux[0]
    O[0, :, :nx, 2] = pops[18]
    O[0, :, :nx, 3] = aux[0]
    for k in range(4):
        O[1, :, :nx, k] = aux[1 + k]
    return torch.from_numpy(P).cuda(), torch.from_numpy(A).cuda()


def _to_host(P, A, L, nx):
    P = P.cpu().numpy().astype(np.float64)
    A = A.cpu().numpy().astype(np.float64)
    _, ny, pitch = P.shape
    P4 = P[:16].reshape(8, ny, pitch, 2)
    O = A.reshape(2, ny, pitch, 4)
    pops = np.zeros((27, ny, nx))
    aux = np.zeros((5, ny, nx))
    for i in range(1, 9):
        pops[i] = P4[i - 1, :, :nx, 0]
        pops[9 + i] = P4[i - 1, :, :nx, 1]
        pops[18 + i] = P[15 + i, :, :nx]
    aux[0] = O[0, :, :nx, 3]
    pops[0] = O[0, :, :nx, 0]
    pops[9] = O[0, :, :nx, 1] + L * aux[0]
    pops[18] = O[0, :, :nx, 2]
    for k in range(4):
        aux[1 + k] = O[1, :, :nx, k]
    return pops, aux


def test_noalloc_step_matches_handle_step_twice(env):
    torch, lbm = env
    p, phi0, T0 = inputs.sessile(nx=100, ny=70, R=24.0, theta_deg=70.0)
    L = p["Cp"] * (p["T_m"] - p["T_w"]) / p["Ste"]
    pitch = (p["nx"] + 31) // 32 * 32
    lat = lbm.Lattice([p])
    lat.set_kernel(lbm.LBM_KERNEL_TILE, 32, 8)
    lat.init(phi0, T0).step(40)
    pops, aux = lat.get_state()

    bufs = [_to_device(torch, pops, aux, L, pitch),
            (torch.zeros((24, p["ny"], pitch), dtype=torch.float32, device="cuda"),
             torch.zeros((8, p["ny"], pitch), dtype=torch.float32, device="cuda"))]
    d_obs = torch.zeros(lbm.LBM_OBS_COUNT, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        (Pi, Ai), (Po, Ao) = bufs[call % 2], bufs[(call + 1) % 2]
        d_obs.fill_(-1.0)
        lbm.lbm_step_noalloc(p, Pi.data_ptr(), Ai.data_ptr(), Po.data_ptr(), Ao.data_ptr(),
                             pitch, d_obs.data_ptr(), stream)
        torch.cuda.synchronize()
        lat.step(1)
        want_pops, want_aux = lat.get_state()
        got_pops, got_aux = _to_host(Po, Ao, L, p["nx"])
        assert np.abs(got_pops - want_pops).max() <= TOL, call
        assert np.abs(got_aux - want_aux).max() <= TOL, call
        got_obs = d_obs.cpu().numpy()
        want_obs = lat.observables()
        for j, k in enumerate(lbm.OBS_NAMES):
            assert got_obs[j] == pytest.approx(want_obs[k], rel=TOL, abs=1e-9), (call, k)


def test_noalloc_rejects_what_it_cannot_hold(env):
    torch, lbm = env
    # Every case below is refused by the host-side checks before any device
    # work is queued, so the placeholder addresses are never dereferenced.
    big = inputs.params(nx=2080, ny=1024)  # 65 x 128 = 8320 tiles > 8192
    assert ((2080 + 31) // 32) * ((1024 + 7) // 8) > lbm.LBM_NOALLOC_MAX_TILES
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_noalloc(big, 16, 16, 16, 16, 2080, 16, 0)
    assert e.value.code == lbm.LBM_ETOOLARGE
    small = inputs.params(nx=40, ny=16)
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_noalloc(small, 16, 16, 16, 16, 39, 16, 0)  # pitch < nx
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_noalloc(small, 0, 16, 16, 16, 64, 16, 0)  # null input
    assert e.value.code == lbm.LBM_EINVAL
