"""Failure paths of the PIE sweeps, made without faulting the GPU.

Bounded device waits: the test hook raises a wait's target by one arrival that
no CTA ever makes (a flag nothing sets), so the grid barrier of the persistent
launch form, or the predecessor wait of the dataflow form, runs its 2 s
timeout. The kernel then sets the sweep's error word, every CTA stops waiting
and the launch ends; the host reports PFT_ERR_TIMEOUT and the context keeps
working. Non-finite data, written on the host: a NaN or infinite intensity is
refused when the context is built, and a NaN in the object comes back as
PFT_ERR_NONFINITE from the sweeps and the error metrics, not as a silently
wrong result.
"""
import time

import numpy as np
import pytest

from oracle import coeffs, pie as opie
from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    pft.load()
    return torch, pft


def c64(a, torch):
    return torch.from_numpy(np.ascontiguousarray(a).astype(np.complex64)).cuda()


def ctx_for(P, torch, pft, inten=None):
    inten = P["intensities"] if inten is None else inten
    return pft.PieContext(P["obj"].shape, c64(P["probe"], torch), P["pos"],
                          torch.from_numpy(inten.astype(np.float32)).cuda(), M=P["M"])


def oracle_pft_sweep(P, start):
    T = opie.pft_transform(*coeffs.plan_2d(32, 32, 16, 16, 8, 8))
    order = opie.colour_major_order(opie.greedy_colouring(P["pos"], 32, 32))
    z, _ = opie.pie_sweep(start.astype(np.complex64).astype(np.complex128), P["probe"], P["pos"],
                          opie.amplitudes(P["intensities"], 16), T, 1.0, order)
    return z


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("form", ["persistent", "dataflow"])
def test_unreachable_wait_times_out_and_the_context_recovers(env, form):
    torch, pft = env
    P = synth.small_raster_problem()
    ctx = ctx_for(P, torch, pft)
    launch = pft.LAUNCH_PERSISTENT if form == "persistent" else pft.LAUNCH_DATAFLOW
    ctx.set_persistent(pft.TRANSFORM_PFT, launch)
    assert ctx.info()["persistent_pft"] == launch
    ctx.test_unreachable_wait(pft.TEST_WAIT_GRID_BARRIER if form == "persistent" else pft.TEST_WAIT_DATAFLOW)
    z = c64(P["init"], torch)
    t0 = time.time()
    with pytest.raises(pft.PftError) as e:
        ctx.iteration(z, pft.TRANSFORM_PFT, 1.0)          # with stats: the sweep reports its own timeout
    assert e.value.code == -5 and time.time() - t0 < 30.0
    # without stats the sweep stays asynchronous and the next call reports the timeout
    ctx.iteration(z, pft.TRANSFORM_PFT, 1.0, stats=False)
    torch.cuda.synchronize()
    ctx.test_unreachable_wait(pft.TEST_WAIT_NONE)
    z = c64(P["init"], torch)
    with pytest.raises(pft.PftError) as e:
        ctx.iteration(z, pft.TRANSFORM_PFT, 1.0)
    assert e.value.code == -5
    # the status was consumed: the same context now sweeps normally and matches the oracle
    z = c64(P["init"], torch)
    ctx.iteration(z, pft.TRANSFORM_PFT, 1.0)
    assert ctx.info()["persistent_pft"] == launch
    assert rel(z.cpu().numpy(), oracle_pft_sweep(P, P["init"])) < TOL


def test_hook_refuses_unknown_kinds(env):
    torch, pft = env
    P = synth.small_raster_problem()
    ctx = ctx_for(P, torch, pft)
    with pytest.raises(pft.PftError) as e:
        ctx.test_unreachable_wait(7)
    assert e.value.code == -1


@pytest.mark.parametrize("where", ["crop", "high"])
def test_nan_intensity_is_refused(env, where):
    """A NaN intensity, inside the PFT crop or only in the full data, is refused
    when the context is built (it would otherwise reach every later sweep)."""
    torch, pft = env
    P = synth.small_raster_problem()
    inten = P["intensities"].copy()
    inten[5, 0, 0] = np.nan if where == "crop" else inten[5, 0, 0]
    inten[9, 16, 16] = np.inf if where == "high" else inten[9, 16, 16]   # the Nyquist corner: outside the crop
    with pytest.raises(pft.PftError) as e:
        ctx_for(P, torch, pft, inten)
    assert e.value.code == -4


@pytest.mark.parametrize("transform", ["pft", "full"])
def test_nan_object_is_reported_as_nonfinite(env, transform):
    """A NaN written into the object on the host spreads through the sweep and
    comes back as PFT_ERR_NONFINITE from the sweep, from Algorithm 3 and from
    both error metrics; the context then sweeps a clean object normally."""
    torch, pft = env
    P = synth.small_raster_problem()
    ctx = ctx_for(P, torch, pft)
    tr = pft.TRANSFORM_PFT if transform == "pft" else pft.TRANSFORM_FULL
    bad = P["init"].copy()
    r, c = P["pos"][7]
    bad[r + 10, c + 11] = np.nan                  # inside the patch of position 7
    z = c64(bad, torch)
    with pytest.raises(pft.PftError) as e:
        ctx.iteration(z, tr, 1.0)
    assert e.value.code == -4
    z = c64(bad, torch)
    with pytest.raises(pft.PftError) as e:
        ctx.warm_start_then_refine(z, pft.Schedule(1.0, 1.0, 0.0, 0.0, 2, 2))
    assert e.value.code == -4
    truth = c64(P["obj"], torch)
    with pytest.raises(pft.PftError) as e:
        ctx.nrmse(z, truth)
    assert e.value.code == -4
    with pytest.raises(pft.PftError) as e:
        pft.nrmse_noalloc(z, truth)
    assert e.value.code == -4
    z = c64(P["init"], torch)
    ctx.iteration(z, pft.TRANSFORM_PFT, 1.0)
    assert rel(z.cpu().numpy(), oracle_pft_sweep(P, P["init"])) < TOL
