"""GPU parity of the batched PFT, its adjoint and the FFT kernels against the
FP64 oracle (tolerance: 1e-5 relative L2 for FP32 arithmetic)."""
import numpy as np
import pytest

from oracle import coeffs, dft, pft as opft
from paper_2408_03532_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-5
SHAPES = [(32, 16), (64, 16), (64, 32), (64, 64), (128, 16), (128, 32), (128, 64), (256, 16), (256, 32),
          (256, 64)]


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft
    libbuild.build()
    pft.load()
    return torch, pft


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_frames(a, b):
    return np.linalg.norm((a - b).reshape(len(a), -1), axis=1) / np.linalg.norm(b.reshape(len(b), -1), axis=1)


def oracle_plans(n, M):
    return coeffs.plan_2d(n, n, M, M, M // 2, M // 2)


@pytest.mark.parametrize("n,M", SHAPES)
def test_forward_matches_oracle(env, n, M):
    torch, pft = env
    B = 7  # ragged: fewer frames than CTAs
    x = synth.random_frames(B, n, seed=n + M)
    plan = pft.Plan(n, M)
    assert plan.info["r1"] == 13 and plan.info["p1"] == M // 2
    y = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = opft.pft2(x.astype(np.complex128), *oracle_plans(n, M))
    assert rel_frames(y, ref).max() < TOL


@pytest.mark.parametrize("n,M", SHAPES)
def test_adjoint_matches_oracle(env, n, M):
    torch, pft = env
    y = synth.random_frames(5, M, seed=3 * n + M)
    plan = pft.Plan(n, M)
    x = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    ref = opft.pft2_adjoint(y.astype(np.complex128), *oracle_plans(n, M))
    assert rel_frames(x, ref).max() < TOL


@pytest.mark.parametrize("n,M", [(64, 32), (256, 32)])
def test_adjoint_identity_on_gpu(env, n, M):
    """<A x, y> = <x, A^H y> for the GPU operator pair."""
    torch, pft = env
    plan = pft.Plan(n, M)
    x = synth.random_frames(4, n, seed=11)
    y = synth.random_frames(4, M, seed=12)
    Ax = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    Ahy = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy().astype(np.complex128)
    lhs = np.vdot(y.astype(np.complex128), Ax)
    rhs = np.vdot(Ahy, x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_pft_approximates_exact_partial_dft(env):
    """The GPU PFT is within the paper's approximation of the exact transform."""
    torch, pft = env
    x = synth.random_frames(3, 128, seed=5)
    y = pft.Plan(128, 32).forward(torch.from_numpy(x).cuda()).cpu().numpy()
    exact = dft.partial_dft2(x.astype(np.complex128), 32, 32)
    assert rel(y, exact) < TOL


def test_tables_reproduce_twiddles(env):
    """sum_j B[l, j] W'[t, j] e^{+i pi t/p}... i.e. the FP32 tables rebuild each
    twiddle e^{-2 pi i t (l - q/2)/n} e^{-i pi t/p} to eps + FP32 rounding, and W'
    equals i^j times the oracle's W (Algorithm 1)."""
    torch, pft = env
    n, M = 128, 32
    plan = pft.Plan(n, M)
    B, W = plan.tables(0)
    p, q = plan.info["p1"], plan.info["q1"]
    t = np.arange(-M // 2, M // 2)[:, None]
    l = np.arange(q)[None, :]
    approx = W.astype(np.complex128) @ B.astype(np.float64).T
    exact = np.exp(-2j * np.pi * t * (l - q / 2) / n) * np.exp(-1j * np.pi * t / p)
    assert np.abs(approx - exact).max() < 1e-7 + 2e-6
    P1, _ = oracle_plans(n, M)
    assert np.allclose(W, P1["W"] * (1j ** np.arange(13))[None, :], rtol=2e-7, atol=1e-6)


@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_fft2_matches_oracle(env, n):
    torch, pft = env
    x = synth.random_frames(3, n, seed=n)
    X = pft.fft2(torch.from_numpy(x).cuda()).cpu().numpy()
    assert rel_frames(X, dft.full_dft2(x.astype(np.complex128))).max() < TOL
    Y = pft.fft2(torch.from_numpy(x).cuda(), inverse=True).cpu().numpy()
    assert rel_frames(Y, dft.full_idft2(x.astype(np.complex128)) * n * n).max() < TOL


@pytest.mark.parametrize("n,M", [(256, 32), (256, 64), (128, 32), (32, 16)])
def test_fft_crop_matches_oracle(env, n, M):
    torch, pft = env
    x = synth.random_frames(5, n, seed=7)
    y = pft.fft_crop(torch.from_numpy(x).cuda(), M).cpu().numpy()
    assert rel_frames(y, dft.fft_then_crop(x.astype(np.complex128), M, M)).max() < TOL


@pytest.mark.parametrize("M", [32, 64])
def test_full_size_batch_sampled(env, M):
    """4096 frames of 256 x 256 in the launch configuration the benchmark times;
    sampled frames are checked one by one against the oracle."""
    torch, pft = env
    B, n = 4096, 256
    x = torch.randn(B, n, n, dtype=torch.complex64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    plan = pft.Plan(n, M)
    y = plan.forward(x)
    xa = plan.adjoint(y)
    torch.cuda.synchronize()
    P1, P2 = oracle_plans(n, M)
    for f in (0, 1, 2047, 4095):
        xf = x[f].cpu().numpy().astype(np.complex128)
        assert rel(y[f].cpu().numpy(), opft.pft2(xf, P1, P2)) < TOL
        ref_adj = opft.pft2_adjoint(y[f].cpu().numpy().astype(np.complex128), P1, P2)
        assert rel(xa[f].cpu().numpy(), ref_adj) < TOL


def test_edge_cases_and_errors(env):
    torch, pft = env
    plan = pft.Plan(64, 32)
    empty = torch.empty(0, 64, 64, dtype=torch.complex64, device="cuda")
    assert plan.forward(empty).shape == (0, 32, 32)
    one = torch.from_numpy(synth.random_frames(1, 64, seed=1)).cuda()
    assert plan.forward(one[0]).shape == (32, 32)
    with pytest.raises(pft.PftError) as e:
        pft.Plan(64, 31)
    assert e.value.code == -1
    with pytest.raises(pft.PftError) as e:
        pft.Plan(96, 32)  # q = 6 is not a power of two
    assert e.value.code == -2
    with pytest.raises(pft.PftError):
        pft.Plan(64, 32, eps=1e-12)  # needs more than 13 terms


# rectangular frames: (n1, n2, M1, M2); p = M / 2 per axis
RECT = [(128, 256, 32, 32), (256, 128, 32, 32), (64, 128, 32, 32), (128, 128, 32, 64), (256, 256, 64, 32),
        (128, 128, 16, 32)]


@pytest.mark.parametrize("n1,n2,M1,M2", RECT)
def test_rectangular_plans_match_oracle(env, n1, n2, M1, M2):
    """Rectangular frames and outputs (Algorithm 4 per axis, each axis with its
    own p, q, r and tables): forward and adjoint against the oracle's
    Algorithm 5 on 6 frames, and the adjoint identity."""
    torch, pft = env
    plan = pft.Plan(n1, M1, n2=n2, M2=M2)
    i = plan.info
    assert (i["n1"], i["n2"], i["M1"], i["M2"]) == (n1, n2, M1, M2)
    assert (i["p1"], i["p2"]) == (M1 // 2, M2 // 2) and (i["q1"], i["q2"]) == (2 * n1 // M1, 2 * n2 // M2)
    P1, P2 = coeffs.plan_2d(n1, n2, M1, M2, M1 // 2, M2 // 2)
    rng = np.random.default_rng(n1 + 3 * n2 + 5 * M1 + 7 * M2)
    x = (rng.standard_normal((6, n1, n2)) + 1j * rng.standard_normal((6, n1, n2))).astype(np.complex64)
    y = (rng.standard_normal((6, M1, M2)) + 1j * rng.standard_normal((6, M1, M2))).astype(np.complex64)
    Ax = plan.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    assert Ax.shape == (6, M1, M2)
    assert rel_frames(Ax, opft.pft2(x.astype(np.complex128), P1, P2)).max() < TOL
    Ahy = plan.adjoint(torch.from_numpy(y).cuda()).cpu().numpy()
    assert Ahy.shape == (6, n1, n2)
    assert rel_frames(Ahy, opft.pft2_adjoint(y.astype(np.complex128), P1, P2)).max() < TOL
    lhs = np.vdot(y.astype(np.complex128), Ax.astype(np.complex128))
    rhs = np.vdot(Ahy.astype(np.complex128), x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    # each axis has its own tables: axis 2's are those of a square plan of that axis's shape
    B2, W2 = plan.tables(1)
    B2s, W2s = pft.Plan(n2, M2).tables(0)
    assert W2.shape == (M2, 13) and np.array_equal(W2, W2s) and np.array_equal(B2, B2s)


def test_rectangular_plan_limits(env):
    torch, pft = env
    with pytest.raises(pft.PftError) as e:   # rectangular plans are FP32
        pft.Plan(128, 32, n2=256, precision=pft.PREC_SPLIT_BF16)
    assert e.value.code == -2
    with pytest.raises(pft.PftError) as e:   # a shape pair with no kernel built
        pft.Plan(32, 16, n2=256, M2=64)
    assert e.value.code == -2
