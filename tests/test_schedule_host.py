"""The scan schedule the library builds on the host (no GPU): greedy colours
and the colour-major order against the oracle, and the dataflow predecessor
lists against the property that makes a dataflow sweep equal to the
sequential one (Section 2.1 visits positions one after another): every earlier
overlapping position must be done before a position reads its patch, and the
lists must only name earlier overlapping positions."""
import numpy as np
import pytest

from oracle import pie as opie
from paper_2408_03532_gb300 import synth


@pytest.fixture(scope="module")
def pft():
    from paper_2408_03532_gb300 import build as libbuild
    from paper_2408_03532_gb300 import pft as _pft
    libbuild.build()
    _pft.load()
    return _pft


def earlier_overlapping(pos, sched, n):
    P = np.asarray(pos)[sched]
    return [set(np.nonzero(np.abs(P[:s] - P[s]).max(axis=1) < n)[0].tolist()) for s in range(len(sched))]


def check_predecessors(pos, n, S):
    sched, off, dep = S["sched"], S["dep_off"], S["dep"]
    E = earlier_overlapping(pos, sched, n)
    done_before = []
    for s in range(len(sched)):
        D = dep[off[s]:off[s + 1]].tolist()
        assert set(D) <= E[s], s                # only earlier overlapping items
        assert len(set(D)) == len(D), s
        for b in D:                             # none is implied by another member of E(s)
            assert not any(b in E[a] for a in E[s]), (s, b)
        covered = set(D)
        for d in D:
            covered |= done_before[d]
        assert E[s] <= covered, s               # every earlier overlapping item is done first
        done_before.append(covered)


def test_small_raster_schedule_matches_oracle(pft):
    P = synth.small_raster_problem()
    S = pft.pie_scan_schedule(P["pos"], 32, P["obj"].shape)
    col = opie.greedy_colouring(P["pos"], 32, 32)
    assert np.array_equal(S["colour"], col)
    assert S["ncolours"] == col.max() + 1
    assert np.array_equal(S["sched"], opie.colour_major_order(col))
    check_predecessors(P["pos"], 32, S)


@pytest.mark.parametrize("seed", [None, 3])
def test_spiral_schedule_in_any_order(pft, seed):
    """300 Fermat positions of 64^2 patches on a 384^2 object, in index order
    and in a random visiting order."""
    P = synth.spiral_problem(side=384, n=64, count=300, peak_photons=None, M=16)
    order = None if seed is None else np.random.default_rng(seed).permutation(300)
    S = pft.pie_scan_schedule(P["pos"], 64, P["obj"].shape, order)
    col = opie.greedy_colouring(P["pos"], 64, 64, order)
    assert np.array_equal(S["colour"], col)
    assert np.array_equal(S["sched"], opie.colour_major_order(col, order))
    check_predecessors(P["pos"], 64, S)
    # the longest chain of waits is the colour count
    depth = np.zeros(300, int)
    for s in range(300):
        D = S["dep"][S["dep_off"][s]:S["dep_off"][s + 1]]
        depth[s] = 1 + (depth[D].max() if len(D) else 0)
    assert depth.max() <= S["ncolours"]


@pytest.mark.parametrize("seed", [None, 5])
def test_sequential_schedule_is_the_visiting_order(pft, seed):
    """One colour per position: the schedule is the visiting order itself
    (Section 2.1's sequential j, or Section 4.2's random order), and the
    dataflow predecessors are still sound, now for that order."""
    P = synth.spiral_problem(side=384, n=64, count=300, peak_photons=None, M=16)
    order = np.arange(300) if seed is None else np.random.default_rng(seed).permutation(300)
    S = pft.pie_scan_schedule(P["pos"], 64, P["obj"].shape, None if seed is None else order, sequential=True)
    assert S["ncolours"] == 300
    assert np.array_equal(S["colour"], opie.sequential_colouring(order))
    assert np.array_equal(S["sched"], order)
    check_predecessors(P["pos"], 64, S)
    # disjoint patches still get no predecessor: four touching patches
    S = pft.pie_scan_schedule(np.array([[0, 0], [0, 16], [16, 0], [16, 16]], np.int32), 16, (32, 32),
                              sequential=True)
    assert S["ncolours"] == 4 and len(S["dep"]) == 0


def test_disjoint_and_single_positions(pft):
    # patches that touch but do not overlap: one colour, no predecessors
    pos = np.array([[0, 0], [0, 16], [16, 0], [16, 16]], np.int32)
    S = pft.pie_scan_schedule(pos, 16, (32, 32))
    assert S["ncolours"] == 1 and len(S["dep"]) == 0
    # the same patch four times: a chain, each item waits for the one before
    S = pft.pie_scan_schedule(np.zeros((4, 2), np.int32), 16, (32, 32))
    assert S["ncolours"] == 4
    assert S["dep"].tolist() == [0, 1, 2] and S["dep_off"].tolist() == [0, 0, 1, 2, 3]


def test_invalid_arguments(pft):
    with pytest.raises(pft.PftError):
        pft.pie_scan_schedule(np.array([[20, 0]], np.int32), 16, (32, 32))   # patch outside
    with pytest.raises(pft.PftError):
        pft.pie_scan_schedule(np.zeros((3, 2), np.int32), 16, (32, 32), order=[0, 0, 1])
