"""Independent reconstructions of different sizes swept together (one CUDA
graph per sweep; one launch per shape class, or per class and colour)."""
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


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def small_instances():
    """Six instances over four shape classes, noise-free data."""
    specs = [dict(side=96, n=32, M=16, npos=40, seed=11), dict(side=160, n=64, M=32, npos=30, seed=12),
             dict(side=128, n=64, M=16, npos=25, seed=13), dict(side=256, n=128, M=32, npos=20, seed=14),
             dict(side=100, n=32, M=16, npos=50, seed=15), dict(side=192, n=64, M=32, npos=45, seed=16)]
    out = []
    for sp in specs:
        inst = synth.make_instance(sp)
        inst["intensities"] = synth.simulate_intensities(inst["obj"], inst["probe"], inst["pos"])
        out.append(inst)
    return out


def to_gpu(insts, torch):
    return [dict(obj_shape=i["obj"].shape, probe=torch.from_numpy(i["probe"].astype(np.complex64)).cuda(),
                 positions=i["pos"], intensities=torch.from_numpy(i["intensities"].astype(np.float32)).cuda(),
                 M=i["M"]) for i in insts]


def oracle_sweep(inst, transform, mode, beta):
    n, M = inst["probe"].shape[0], inst["M"]
    start = inst["init"].astype(np.complex64).astype(np.complex128)
    if transform == "pft":
        P1, P2 = coeffs.plan_2d(n, n, M, M, M // 2, M // 2)
        T, d = opie.pft_transform(P1, P2), opie.amplitudes(inst["intensities"], M)
    else:
        T, d = opie.full_transform(n, n), opie.amplitudes(inst["intensities"])
    if mode == "coloured":
        order = opie.colour_major_order(opie.greedy_colouring(inst["pos"], n, n))
        return opie.pie_sweep(start, inst["probe"], inst["pos"], d, T, beta, order)
    return opie.batched_sweep(start, inst["probe"], inst["pos"], d, T, beta, delta_rel=1e-3)


@pytest.mark.parametrize("mode", ["coloured", "batched"])
@pytest.mark.parametrize("transform", ["pft", "full"])
def test_small_batch_matches_oracle_per_instance(env, mode, transform):
    torch, pft = env
    insts = small_instances()
    B = pft.PieBatch(to_gpu(insts, torch), mode=pft.MODE_COLOURED if mode == "coloured" else pft.MODE_BATCHED)
    assert B.classes()[0] == 4
    objs = [torch.from_numpy(i["init"].astype(np.complex64)).cuda() for i in insts]
    tr = pft.TRANSFORM_PFT if transform == "pft" else pft.TRANSFORM_FULL
    phi = B.iteration(objs, tr, 0.9)
    for i, inst in enumerate(insts):
        zo, po = oracle_sweep(inst, transform, mode, 0.9)
        assert rel(objs[i].cpu().numpy(), zo) < TOL, i
        assert phi[i] == pytest.approx(po, rel=TOL)


def test_dataflow_batch_equals_per_colour_launches(env):
    """The coloured batch in its two launch forms (one dataflow launch per
    class, or one launch per class and colour) gives the same objects bit for
    bit over two sweeps; the dataflow form makes one launch per class."""
    torch, pft = env
    insts = small_instances()
    A = pft.PieBatch(to_gpu(insts, torch))
    B = pft.PieBatch(to_gpu(insts, torch))
    A.set_launch(pft.LAUNCH_PER_COLOUR)
    B.set_launch(pft.LAUNCH_DATAFLOW)
    assert B.classes() == (4, 4)
    assert A.classes()[1] > 4
    za = [torch.from_numpy(i["init"].astype(np.complex64)).cuda() for i in insts]
    zb = [z.clone() for z in za]
    for _ in range(2):
        pa = A.iteration(za, pft.TRANSFORM_PFT, 0.9)
        pb = B.iteration(zb, pft.TRANSFORM_PFT, 0.9)
    for i in range(len(insts)):
        assert torch.equal(za[i], zb[i]), i
        assert pb[i] == pytest.approx(pa[i], rel=1e-6)
    with pytest.raises(pft.PftError):
        B.set_launch(pft.LAUNCH_PERSISTENT)


def test_batch_equals_separate_contexts_at_full_recipe(env):
    """The 64-instance recipe (objects 256^2-2048^2, probes 64^2-256^2, 50-2000
    Fermat positions, M in {16, 32, 64}): one batched PFT sweep gives, instance
    by instance, exactly the object of a sweep with a context of its own (the
    same kernel on the same data; only the launch grouping differs), in both
    coloured launch forms."""
    torch, pft = env
    specs = synth.uneven_batch_recipe(64)
    insts = []
    for sp in specs:
        inst = synth.make_instance(sp)
        obj = torch.from_numpy(inst["obj"].astype(np.complex64)).cuda()
        pr = torch.from_numpy(inst["probe"].astype(np.complex64)).cuda()
        inten = synth.simulate_intensities_torch(obj, pr, inst["pos"])
        insts.append(dict(obj_shape=inst["obj"].shape, probe=pr, positions=inst["pos"],
                          intensities=inten, M=sp["M"], init=inst["init"]))
    B = pft.PieBatch(insts)
    nclass, nlaunch = B.classes()
    assert nclass >= 5 and nlaunch > nclass  # one launch per class and colour
    objs = [torch.from_numpy(i["init"].astype(np.complex64)).cuda() for i in insts]
    B.iteration(objs, pft.TRANSFORM_PFT, 1.0, stats=False)
    B.set_launch(pft.LAUNCH_DATAFLOW)  # and one dataflow launch per class
    assert B.classes() == (nclass, nclass)
    objs_flow = [torch.from_numpy(i["init"].astype(np.complex64)).cuda() for i in insts]
    B.iteration(objs_flow, pft.TRANSFORM_PFT, 1.0, stats=False)
    torch.cuda.synchronize()
    for i in range(len(insts)):
        assert torch.equal(objs_flow[i], objs[i]), i
    for i in (0, 17, 41, 63):
        ctx = pft.PieContext(insts[i]["obj_shape"], insts[i]["probe"], insts[i]["positions"],
                             insts[i]["intensities"], M=insts[i]["M"], autotune=False)
        z = torch.from_numpy(insts[i]["init"].astype(np.complex64)).cuda()
        ctx.iteration(z, pft.TRANSFORM_PFT, 1.0, stats=False)
        torch.cuda.synchronize()
        assert torch.equal(z, objs[i]), i


@pytest.mark.parametrize("transform", ["pft", "full"])
def test_recipe_classes_match_oracle(env, transform):
    """One instance of every shape class (n, M) of the 64-instance recipe, the
    one with the fewest positions, swept together in one batch; each object is
    compared with the oracle's sweep of that instance (noise-free data, a start
    within +-10 % of the truth, so the comparison is well conditioned). The
    full transform includes the 256^2 probes' 8-CTA kernel."""
    torch, pft = env
    specs = synth.uneven_batch_recipe(64)
    pick = {}
    for sp in specs:
        key = (sp["n"], sp["M"])
        if key not in pick or sp["npos"] < pick[key]["npos"]:
            pick[key] = sp
    assert len(pick) >= 8
    insts = []
    for key in sorted(pick):
        inst = synth.make_instance(pick[key])
        inst["intensities"] = synth.simulate_intensities(inst["obj"], inst["probe"], inst["pos"])
        rng = np.random.default_rng(pick[key]["seed"])
        inst["init"] = inst["obj"] * (1 + 0.2 * (rng.random(inst["obj"].shape) - 0.5))
        insts.append(inst)
    B = pft.PieBatch(to_gpu(insts, torch))
    assert B.classes()[0] == len(insts)
    objs = [torch.from_numpy(i["init"].astype(np.complex64)).cuda() for i in insts]
    tr = pft.TRANSFORM_PFT if transform == "pft" else pft.TRANSFORM_FULL
    phi = B.iteration(objs, tr, 1.0)
    for i, inst in enumerate(insts):
        zo, po = oracle_sweep(inst, transform, "coloured", 1.0)
        assert rel(objs[i].cpu().numpy(), zo) < TOL, (i, inst["probe"].shape, inst["M"])
        assert phi[i] == pytest.approx(po, rel=1e-4)
