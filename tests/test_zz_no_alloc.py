"""The allocation-free error reduction against the context's error reduction.

pie_nrmse_noalloc exists for callers that cannot allocate device memory when
they need the error (inside CUDA-graph capture, in latency-critical loops where
an allocation may synchronise the device, or under a framework that owns all
device memory). It must give the same value as pie_nrmse, call after call,
although every call reuses one fixed device array.
"""
import ctypes

import numpy as np
import pytest

from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_noalloc_matches_pie_nrmse_on_consecutive_calls():
    import torch

    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    lib = pft.load()
    # a flat probe on a raster that covers every pixel, so the context's
    # illuminated mask is the whole object and both calls see the same pixels
    obj = synth.make_object(64)
    probe = np.ones((32, 32), np.complex64)
    pos = synth.raster_scan(3, 3, 16, 0)
    inten = synth.simulate_intensities(obj, probe, pos)
    ctx = pft.PieContext(obj.shape, torch.from_numpy(probe).cuda(), pos,
                         torch.from_numpy(inten.astype(np.float32)).cuda(), M=16)
    truth = torch.from_numpy(obj.astype(np.complex64)).cuda()
    z1 = torch.from_numpy((synth.random_init(64, seed=7) * np.exp(0.4j)).astype(np.complex64)).cuda()
    z2 = torch.from_numpy((obj * 0.9 * np.exp(-1.2j) + 0.05).astype(np.complex64)).cuda()
    mask = torch.ones(64 * 64, dtype=torch.uint8, device="cuda")
    ref1, ref2 = ctx.nrmse(z1, truth), ctx.nrmse(z2, truth)
    got1 = pft.nrmse_noalloc(z1, truth, mask)
    got2 = pft.nrmse_noalloc(z2, truth, mask)
    assert got1 == pytest.approx(ref1, rel=TOL)
    assert got2 == pytest.approx(ref2, rel=TOL)
    assert pft.nrmse_noalloc(z1, truth) == pytest.approx(ref1, rel=TOL)  # NULL mask: all elements
    # a count beyond the fixed array's capacity is refused before any GPU work
    out = ctypes.c_double()
    rc = lib.pie_nrmse_noalloc(z1.data_ptr(), truth.data_ptr(), None, 4096 * 4096 + 1, ctypes.byref(out), None)
    assert rc == -1 and b"maximum" in lib.pft_last_error()
