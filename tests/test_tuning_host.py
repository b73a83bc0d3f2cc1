"""Host logic of the Algorithm 3 timing and step-size search (tuning.py), on a
stand-in context whose warm_start_then_refine returns a scripted NRMSE trace:
the number of full sweeps found, the timed call's budget, and the ranking."""
import pytest

torch = pytest.importorskip("torch")

from paper_2408_03532_gb300 import pft, tuning  # noqa: E402


class FakeCtx:
    """NRMSE after PFT sweep k: 0.6 - 0.1 k with TV, 0.6 + 0.01 k without (the
    climb of an unregularised PFT phase); each full sweep then halves the gap
    to 0.1. Records every schedule it is called with."""

    def __init__(self):
        self.calls = []

    def warm_start_then_refine(self, z, s, truth=None):
        self.calls.append((s, truth is not None))
        out, e = [], 0.6
        for _ in range(s.max_pft):
            e = e - 0.1 if s.tv_pft > 0 else e + 0.01
            e = max(e, 0.15)
            out.append({"phase": "pft", "nrmse": e if truth is not None else float("nan")})
        for _ in range(s.max_full):
            e = 0.1 + 0.5 * (e - 0.1)
            out.append({"phase": "full", "nrmse": e if truth is not None else float("nan")})
        return out


@pytest.fixture(autouse=True)
def no_cuda_sync(monkeypatch):
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)


def test_sweeps_to_target_counts_refine_sweeps():
    ctx, z = FakeCtx(), torch.zeros(4, dtype=torch.complex64)
    # plain: 0.6 -> 0.35 -> 0.225 -> 0.1625 -> 0.13125 -> ...: 4 full sweeps reach 0.14
    k, nf, tr = tuning.sweeps_to_target(ctx, z.clone(), z, z, pft.Schedule(1, 1, 0, 0, 0, 10), 0.14)
    assert (k, nf) == (0, 4) and len(tr) == 10
    # 3 PFT sweeps with TV (0.3), then 0.2, 0.15, 0.125: 3 full sweeps
    k, nf, _ = tuning.sweeps_to_target(ctx, z.clone(), z, z, pft.Schedule(1, 1, 0, 0, 3, 10, tv_pft=0.01), 0.14)
    assert (k, nf) == (3, 3)
    # a target below the floor is never reached
    assert tuning.sweeps_to_target(ctx, z.clone(), z, z, pft.Schedule(1, 1, 0, 0, 0, 5), 0.05)[1] is None


def test_time_to_target_times_the_exact_budget_without_truth():
    ctx, z = FakeCtx(), torch.zeros(4, dtype=torch.complex64)
    r = tuning.time_to_target(ctx, z.clone(), z, z, pft.Schedule(1, 1, 0, 0, 3, 40, tv_pft=0.01), 0.14, reps=2)
    assert r["reached"] and (r["pft_sweeps"], r["full_sweeps"]) == (3, 3) and r["s"] is not None
    timed = [s for s, traced in ctx.calls if not traced]
    assert timed and all(s.max_pft == 3 and s.max_full == 3 and s.tol_pft == 0 and s.tol_full == 0 for s in timed)


def test_search_ranks_by_modelled_time():
    ctx, z = FakeCtx(), torch.zeros(4, dtype=torch.complex64)
    costs = {"full": 1.0, "pft_coloured": 1.0, "pft_batched": 0.5, "pft_coloured_tv": 1.1, "pft_batched_tv": 0.6}
    rows = tuning.search(ctx, z.clone(), z, z, 0.14, 10, betas=(1.0,), tvs=(0.0, 0.01), counts=(1, 3),
                         costs=costs)
    assert len(rows) == 8
    # modelled times: batched 1 sweep no TV 0.5 + 4 = 4.5; batched 1 with TV 0.6 + 4 = 4.6; batched 3
    # with TV 1.8 + 3 = 4.8; coloured 1 no TV 1 + 4 = 5; ...; coloured 3 no TV 3 + 4 = 7
    best, second = rows[0], rows[1]
    assert best["pft_batched"] and best["tv_pft"] == 0.0 and best["pft_sweeps"] == 1
    assert best["model_s"] == pytest.approx(4.5) and second["model_s"] == pytest.approx(4.6)
    assert rows[-1]["model_s"] == pytest.approx(7.0)
    modelled = [r["model_s"] for r in rows if r["model_s"] is not None]
    assert modelled == sorted(modelled)
