"""The allocation-free error reduction, pie_nrmse_noalloc, called through the C ABI.

The call exists for callers that cannot call cudaMalloc when they need the
error: a plug-in under a host framework that owns every device allocation
through its own pool, or a latency-critical loop where an allocation can
synchronise the whole device. Every call reuses one fixed device array, so the
checks below make several calls in a row and require each to give the same
value as the context's own reduction (pie_nrmse) and as a float64 computation
of min_phi ||e^{i phi} z - t|| / ||t|| on the same complex64 inputs.

This file is named to be collected last, so a run that stops at its first
failure has run every other test before this one; it also passes on its own in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

from oracle import pie as opie
from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5  # relative, both sides reduce the same complex64 inputs in FP64


@pytest.fixture(scope="module")
def lib():
    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    return pft.load()


def _call(lib, z, t, mask, count=None):
    out = ctypes.c_double()
    rc = lib.pie_nrmse_noalloc(z.data_ptr(), t.data_ptr(), None if mask is None else mask.data_ptr(),
                               z.numel() if count is None else count, ctypes.byref(out), None)
    assert rc == 0, lib.pft_last_error()
    return out.value


def test_noalloc_matches_pie_nrmse_on_consecutive_calls(lib):
    import torch

    from paper_2408_03532_gb300 import pft
    # the 128 x 128 raster problem: its illuminated mask leaves the border out,
    # so the masked reduction covers a strict subset over four blocks
    P = synth.small_raster_problem()
    ctx = pft.PieContext(P["obj"].shape, torch.from_numpy(P["probe"].astype(np.complex64)).cuda(), P["pos"],
                         torch.from_numpy(P["intensities"].astype(np.float32)).cuda(), M=16)
    mask_np = opie.illuminated_mask(P["probe"], P["pos"], P["obj"].shape)
    assert 0 < mask_np.sum() < mask_np.size
    mask = torch.from_numpy(mask_np.astype(np.uint8).ravel()).cuda()
    truth_np = P["obj"].astype(np.complex64)
    truth = torch.from_numpy(truth_np).cuda()
    zs = [(P["init"] * np.exp(0.4j)).astype(np.complex64),
          (P["obj"] * 0.9 * np.exp(-1.2j) + 0.05).astype(np.complex64)]
    zt = [torch.from_numpy(z).cuda() for z in zs]
    for rep in range(2):  # two calls in a row, twice: nothing carries over between calls
        for z_np, z in zip(zs, zt):
            got = _call(lib, z, truth, mask)
            assert got == pytest.approx(ctx.nrmse(z, truth), rel=TOL)
            ref = opie.nrmse(z_np.astype(np.complex128), truth_np.astype(np.complex128), mask_np)
            assert got == pytest.approx(ref, rel=TOL)
    # NULL mask: every element
    ref = opie.nrmse(zs[0].astype(np.complex128), truth_np.astype(np.complex128))
    assert _call(lib, zt[0], truth, None) == pytest.approx(ref, rel=TOL)
    assert pft.nrmse_noalloc(zt[0], truth) == pytest.approx(ref, rel=TOL)


def test_noalloc_many_blocks_ragged_count_random_mask(lib):
    import torch
    rng = np.random.default_rng(11)
    # 1000 x 1000 = 1,000,000 elements: 245 blocks of 4096, the last one holding 576
    side = 1000
    t_np = (rng.standard_normal((side, side)) + 1j * rng.standard_normal((side, side))).astype(np.complex64)
    m_np = rng.random((side, side)) < 0.37
    t = torch.from_numpy(t_np).cuda()
    mask = torch.from_numpy(m_np.astype(np.uint8).ravel()).cuda()
    cases = [
        # a rotated, scaled copy with noise: error of order 0.1
        (0.8 * np.exp(2.3j) * t_np + 0.05 * rng.standard_normal((side, side))).astype(np.complex64),
        # a rotated copy with a relative perturbation of 1e-6, where |z|^2 + |t|^2 - 2|<z,t>|
        # would lose every digit in FP64 round-off
        (np.exp(-0.7j) * t_np * (1 + 1e-6 * rng.standard_normal((side, side)))).astype(np.complex64),
    ]
    for z_np in cases + cases:  # two calls in a row, then both again
        z = torch.from_numpy(z_np).cuda()
        ref = opie.nrmse(z_np.astype(np.complex128), t_np.astype(np.complex128), m_np)
        assert _call(lib, z, t, mask) == pytest.approx(ref, rel=TOL)
        # a ragged prefix of the flattened arrays (not a multiple of the block size)
        cnt = 777_777
        ref = opie.nrmse(z_np.ravel()[:cnt].astype(np.complex128), t_np.ravel()[:cnt].astype(np.complex128),
                         m_np.ravel()[:cnt])
        assert _call(lib, z, t, mask, cnt) == pytest.approx(ref, rel=TOL)


def test_noalloc_refuses_sizes_beyond_its_array(lib):
    import torch
    z = torch.zeros(4, dtype=torch.complex64, device="cuda")
    out = ctypes.c_double()
    # checked on the host before any GPU work: the pointers are never read
    rc = lib.pie_nrmse_noalloc(z.data_ptr(), z.data_ptr(), None, 4096 * 4096 + 1, ctypes.byref(out), None)
    assert rc == -1 and b"maximum" in lib.pft_last_error()
    rc = lib.pie_nrmse_noalloc(z.data_ptr(), z.data_ptr(), None, 0, ctypes.byref(out), None)
    assert rc == -1
