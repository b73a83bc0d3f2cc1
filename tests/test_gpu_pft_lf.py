"""GPU parity of the large-frame PFT and its adjoint (n = 2048 ... 16384;
M = 128, p = 64, r = 13; the paper's regime n >> M) against the FP64 oracle.

Stage A runs as split-BF16 tensor-core products (three partial products per
term, relative error about 3 * 2^-18 per product), stage B in FP32; the bound
5e-5 per frame (relative L2) is the same as for the n = 256 split-BF16 path.
"""
import numpy as np
import pytest

from oracle import coeffs, dft, pft as opft
from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 5e-5
M = 128


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    pft.load()
    return torch, pft


def rel_frames(a, b):
    return np.linalg.norm((a - b).reshape(len(a), -1), axis=1) / np.linalg.norm(b.reshape(len(b), -1), axis=1)


@pytest.mark.parametrize("n,batch", [(2048, 3), (4096, 1), (8192, 1)])
def test_forward_matches_oracle(env, n, batch):
    torch, pft = env
    x = synth.random_frames(batch, n, seed=n // 1024 + batch)
    plan = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16)
    assert plan.info["p1"] == 64 and plan.info["q1"] == n // 64 and plan.info["r1"] == 13
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = opft.pft2(x.astype(np.complex128), *coeffs.plan_2d(n, n, M, M, 64, 64), chunk=1)
    err = rel_frames(y, ref)
    assert err.max() < TOL, err


def test_structured_frames_and_exact_transform(env):
    """A frame whose energy sits in the kept band (plane waves) and a smooth
    frame: the PFT reproduces the exact partial DFT within the approximation
    and split accuracy."""
    torch, pft = env
    n = 2048
    yy, xx = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    x = np.empty((2, n, n), np.complex64)
    x[0] = np.exp(2j * np.pi * (7 * yy - 40 * xx) / n) + 0.5 * np.exp(2j * np.pi * (-60 * yy + 3 * xx) / n)
    x[1] = np.exp(-((yy - n / 2) ** 2 + (xx - n / 3) ** 2) / (2 * 150.0 ** 2))
    y = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16).forward(torch.from_numpy(x).cuda()).cpu().numpy()
    exact = np.stack([dft.partial_dft2(x[i].astype(np.complex128), M, M) for i in range(2)])
    assert rel_frames(y, exact).max() < TOL


def test_chunked_batch_matches_single_frames(env):
    """More frames than one workspace pass holds: every frame's forward and
    adjoint equal the same frame transformed alone."""
    torch, pft = env
    n = 2048
    plan = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16)
    B = 33  # a pass holds 15 frames of 2048^2
    x = torch.randn(B, n, n, dtype=torch.complex64, device="cuda", generator=torch.Generator("cuda").manual_seed(5))
    y = plan.forward(x)
    xa = plan.adjoint(y)
    for f in (0, 14, 15, 31, 32):
        assert torch.equal(plan.forward(x[f:f + 1]), y[f:f + 1])
        assert torch.equal(plan.adjoint(y[f:f + 1]), xa[f:f + 1])


@pytest.mark.parametrize("n,batch", [(2048, 3), (4096, 1), (8192, 1)])
def test_adjoint_matches_oracle(env, n, batch):
    torch, pft = env
    yv = synth.random_frames(batch, M, seed=70 + n // 1024)
    plan = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16)
    x = plan.adjoint(torch.from_numpy(yv).cuda()).cpu().numpy()
    ref = opft.pft2_adjoint(yv.astype(np.complex128), *coeffs.plan_2d(n, n, M, M, 64, 64), chunk=1)
    err = rel_frames(x, ref)
    assert err.max() < TOL, err


@pytest.mark.parametrize("n", [2048, 16384])
def test_adjoint_identity(env, n):
    """<A x, y> = <x, A^H y> for the large-frame pair, to the split's accuracy."""
    torch, pft = env
    plan = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16)
    g = torch.Generator("cuda").manual_seed(n)
    x = torch.randn(1, n, n, dtype=torch.complex64, device="cuda", generator=g)
    y = torch.randn(1, M, M, dtype=torch.complex64, device="cuda", generator=g)
    c128 = torch.complex128
    Ax = plan.forward(x).to(c128)
    Ahy = plan.adjoint(y).to(c128)
    lhs = torch.vdot(y.to(c128).flatten(), Ax.flatten())
    rhs = torch.vdot(Ahy.flatten(), x.to(c128).flatten())
    scale = float(torch.linalg.vector_norm(Ax) * torch.linalg.vector_norm(y))
    assert abs(complex(lhs - rhs)) <= 2 * TOL * scale


def test_plane_waves_at_16384(env):
    """n = 16384 (q = 256): a sum of in-band plane waves has the closed-form
    partial DFT n^2 * amplitude at its two frequencies and 0 elsewhere."""
    torch, pft = env
    n = 16384
    u = torch.arange(n, device="cuda", dtype=torch.float64)
    def wave(a, b):
        return torch.exp(2j * torch.pi * (a * u[:, None] + b * u[None, :]) / n)
    x = (wave(5, -33) + (0.25 - 0.5j) * wave(-64, 63)).to(torch.complex64)[None]
    y = pft.Plan(n, M, precision=pft.PREC_SPLIT_BF16).forward(x)[0].cpu().numpy().astype(np.complex128)
    exact = np.zeros((M, M), np.complex128)
    exact[5 + M // 2, -33 + M // 2] = n * n
    exact[-64 + M // 2, 63 + M // 2] = (0.25 - 0.5j) * n * n
    assert np.linalg.norm(y - exact) / np.linalg.norm(exact) < TOL


def test_unsupported_and_empty(env):
    torch, pft = env
    with pytest.raises(pft.PftError) as e:
        pft.Plan(2048, M)                       # FP32 is not built for large frames
    assert e.value.code == -2
    plan = pft.Plan(2048, M, precision=pft.PREC_SPLIT_BF16)
    assert plan.forward(torch.empty(0, 2048, 2048, dtype=torch.complex64, device="cuda")).shape == (0, M, M)
    assert plan.adjoint(torch.empty(0, M, M, dtype=torch.complex64, device="cuda")).shape == (0, 2048, 2048)
