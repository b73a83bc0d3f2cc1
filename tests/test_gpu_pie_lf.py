"""PIE sweeps over large frames (Section 4's regime n >> M) against the oracle.

2048^2 frames with M = 128 (p = 64, r = 13: the paper's m~/p = 1 at eps = 1e-7)
on a 5120^2 object scanned by a 3 x 3 raster of stride 1536: neighbours overlap,
positions two apart do not, so the greedy colouring gives four colours (4, 2,
2 and 1 positions), each swept as one batch of the split-BF16 large-frame
transforms. Noise-free data and a start within +-10 % of the truth keep the
comparison well conditioned; the tolerance is the split-BF16 class's (the
transforms match the exact partial DFT to about 1e-5)."""
import numpy as np
import pytest

from oracle import coeffs, pie as opie
from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

N_FRAME, M, SIDE, STRIDE = 2048, 128, 5120, 1536


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    pft.load()
    return torch, pft


@pytest.fixture(scope="module")
def problem(env):
    torch, _ = env
    obj = synth.make_object(SIDE)
    probe = synth.make_probe(N_FRAME)
    pos = synth.raster_scan(3, 3, STRIDE, 0)
    o = torch.from_numpy(obj.astype(np.complex64)).cuda()
    w = torch.from_numpy(probe.astype(np.complex64)).cuda()
    inten = synth.simulate_intensities_torch(o, w, pos)
    start = (obj * (1 + 0.2 * (np.random.default_rng(9).random(obj.shape) - 0.5))).astype(np.complex64)
    return dict(obj=obj, probe=probe, pos=pos, inten=inten, start=start)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_large_frame_pft_sweeps_match_oracle(env, problem):
    torch, pft = env
    P = problem
    ctx = pft.LargeFramePie((SIDE, SIDE), torch.from_numpy(P["probe"].astype(np.complex64)).cuda(), P["pos"],
                            P["inten"], M=M)
    assert ctx.colours() == (4, 4)
    col = opie.greedy_colouring(P["pos"], N_FRAME, N_FRAME)
    order = opie.colour_major_order(col)
    T = opie.pft_transform(*coeffs.plan_2d(N_FRAME, N_FRAME, M, M, 64, 64))
    d = opie.amplitudes(P["inten"].cpu().numpy().astype(np.float64), M)
    z = torch.from_numpy(P["start"]).cuda()
    zo = P["start"].astype(np.complex128)
    probe = P["probe"].astype(np.complex64).astype(np.complex128)
    for _ in range(2):
        st = ctx.iteration(z, 1.0)
        zo_prev = zo
        zo, phi = opie.pie_sweep(zo, probe, P["pos"], d, T, 1.0, order)
        assert st["phi"] == pytest.approx(phi, rel=1e-3)
        assert st["rel_change"] == pytest.approx(opie.relative_change(zo, zo_prev), rel=1e-3)
    assert rel(z.cpu().numpy(), zo) < 1e-4


def test_large_frame_refusals(env, problem):
    torch, pft = env
    P = problem
    w = torch.from_numpy(P["probe"].astype(np.complex64)).cuda()
    bad = P["pos"].copy()
    bad[4, 1] += 1                                       # an odd column
    with pytest.raises(pft.PftError) as e:
        pft.LargeFramePie((SIDE, SIDE), w, bad, P["inten"], M=M)
    assert e.value.code == -1
    inten = P["inten"].clone()
    inten[2, 0, 0] = float("nan")
    with pytest.raises(pft.PftError) as e:
        pft.LargeFramePie((SIDE, SIDE), w, P["pos"], inten, M=M)
    assert e.value.code == -4
    with pytest.raises(pft.PftError) as e:                # a shape the large-frame transforms do not build
        pft.LargeFramePie((SIDE, SIDE), w, P["pos"], P["inten"], M=64)
    assert e.value.code == -2
