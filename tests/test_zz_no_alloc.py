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


# Offsets inside a block of 768 population floats: chunks by the y component
# of the direction (P: 2, 5, 6 at 0; Z: 1, 3 at 288; M: 4, 7, 8 at 480); in a
# chunk of n directions the k-th keeps (g, h) pairs at 64 k + 2 l and f at
# 64 n + 32 k + l.
CHUNK = {2: (0, 0, 3), 5: (0, 1, 3), 6: (0, 2, 3), 1: (288, 0, 2), 3: (288, 1, 2),
         4: (480, 0, 3), 7: (480, 1, 3), 8: (480, 2, 3)}
GH_OFF = {i: c + 64 * k for i, (c, k, n) in CHUNK.items()}
F_OFF = {i: c + 64 * n + 32 * k for i, (c, k, n) in CHUNK.items()}


def _blocked(pops, aux, L, pitch):
    """Host state (27 population planes with h_0 unshifted, 5 carried planes;
    doubles) -> the library's blocked FP32 layout: row blocks of 32 sites,
    each holding 768 population floats (the chunks above) and 320 own-site
    floats ((g_0, h_0 - L f_l, f_0, f_l), then ((phi u)_x, (phi u)_y, p, S),
    then 64 unused)."""
    ny, nx = pops.shape[1:]
    nb = pitch // 32

    def wide(a):  # [ny, nx] -> [ny, nb, 32], zero beyond nx
        w = np.zeros((ny, pitch))
        w[:, :nx] = a
        return w.reshape(ny, nb, 32)

    P = np.zeros((ny, nb, 768), np.float32)
    A = np.zeros((ny, nb, 320), np.float32)
    for i in range(1, 9):
        P[:, :, GH_OFF[i]:GH_OFF[i] + 64:2] = wide(pops[i])
        P[:, :, GH_OFF[i] + 1:GH_OFF[i] + 64:2] = wide(pops[9 + i])
        P[:, :, F_OFF[i]:F_OFF[i] + 32] = wide(pops[18 + i])
    own = [pops[0], pops[9] - L * aux[0], pops[18], aux[0]]
    for c in range(4):
        A[:, :, c:128:4] = wide(own[c])
        A[:, :, 128 + c:256:4] = wide(aux[1 + c])
    return P.ravel(), A.ravel()


def _unblocked(P, A, L, nx, ny, pitch):
    nb = pitch // 32
    P = P.astype(np.float64).reshape(ny, nb, 768)
    A = A.astype(np.float64).reshape(ny, nb, 320)

    def narrow(v):  # [ny, nb, 32] -> [ny, nx]
        return v.reshape(ny, pitch)[:, :nx]

    pops = np.zeros((27, ny, nx))
    aux = np.zeros((5, ny, nx))
    for i in range(1, 9):
        pops[i] = narrow(P[:, :, GH_OFF[i]:GH_OFF[i] + 64:2])
        pops[9 + i] = narrow(P[:, :, GH_OFF[i] + 1:GH_OFF[i] + 64:2])
        pops[18 + i] = narrow(P[:, :, F_OFF[i]:F_OFF[i] + 32])
    own = [narrow(A[:, :, c:128:4]) for c in range(4)]
    for c in range(4):
        aux[1 + c] = narrow(A[:, :, 128 + c:256:4])
    aux[0] = own[3]
    pops[0], pops[9], pops[18] = own[0], own[1] + L * aux[0], own[2]
    return pops, aux


CASES = {
    # sessile drop: bottom wall, periodic x, ragged blocks and tiles
    "sessile_pitch_128": (dict(nx=100, ny=70, R=24.0, theta_deg=70.0), 128, None),
    # the same with a pitch wider than it needs
    "sessile_pitch_160": (dict(nx=100, ny=70, R=24.0, theta_deg=70.0), 160, None),
    # closed box: walls on every side, no periodic axis, two Dirichlet walls
    "closed_box": (dict(nx=45, ny=37, R=12.0, theta_deg=120.0), 64,
                   dict(periodic_x=0, periodic_y=0, dirichlet_x_hi=1)),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_noalloc_step_matches_handle_step_twice(env, case):
    torch, lbm = env
    kw, pitch, over = CASES[case]
    p, phi0, T0 = inputs.sessile(**kw)
    if over:
        p = dict(p, **over)
    L = p["Cp"] * (p["T_m"] - p["T_w"]) / p["Ste"]
    lat = lbm.Lattice([p])
    lat.set_kernel(lbm.LBM_KERNEL_TILE, 32, 8)
    lat.init(phi0, T0).step(40)
    pops, aux = lat.get_state()
    P0, A0 = _blocked(pops, aux, L, pitch)
    bufs = [(torch.from_numpy(P0).cuda(), torch.from_numpy(A0).cuda()),
            (torch.zeros(P0.size, dtype=torch.float32, device="cuda"),
             torch.zeros(A0.size, dtype=torch.float32, device="cuda"))]
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
        got_pops, got_aux = _unblocked(Po.cpu().numpy(), Ao.cpu().numpy(), L, p["nx"], p["ny"],
                                       pitch)
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
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_noalloc(small, 16, 16, 16, 16, 48, 16, 0)  # pitch not a multiple of 32
    assert e.value.code == lbm.LBM_EINVAL
    # an output buffer that overlaps an input (pitch 64, 16 rows: 24576
    # population floats): out starts inside in
    base, aux = 1 << 20, 1 << 24
    with pytest.raises(lbm.LbmError) as e:
        lbm.lbm_step_noalloc(small, base, aux, base + 4096, aux + (1 << 22), 64, 16, 0)
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError) as e:  # output populations overlap the output own-site data
        lbm.lbm_step_noalloc(small, base, aux, aux + (1 << 22) - 4096, aux + (1 << 22), 64, 16, 0)
    assert e.value.code == lbm.LBM_EINVAL
