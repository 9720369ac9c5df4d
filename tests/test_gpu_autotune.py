"""The autotuner of the batched schedule on the GPU (lsefit_plan_autotune through
paper_1512_08017_gb300.autotune): the tuning it returns fits the batch as the
oracle does, and it is no slower than the library's default schedule."""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    import paper_1512_08017_gb300 as lib
    return lib


def _time(L, x, y, b, plan, reps=10):
    out = L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, plan=plan)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        L.fit_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, plan=plan, out=out)
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps, out


def test_autotune_picks_a_correct_schedule_no_slower_than_default(L, tmp_path, monkeypatch):
    from paper_1512_08017_gb300 import autotune
    from test_gpu_batched import check_batch

    monkeypatch.setenv("LSEFIT_CACHE_DIR", str(tmp_path))
    b = synth.ragged_batch(num_series=6000, lmin=16, lmax=200000, seed=77)
    x = torch.from_numpy(b["x"]).cuda()
    y = torch.from_numpy(b["y"]).cuda()
    best, results = autotune.tune_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5, reps=3)
    assert len(results) == len(autotune.builtin_candidates())
    ms = dict((tuple(sorted(c.items())), t) for c, t in results)
    assert all(t > 0 for t in ms.values())
    # the returned tuning is the fastest measured (resolved values of that candidate)
    fastest = min(results, key=lambda r: r[1])[0]
    for k, v in fastest.items():
        if v:
            assert best[k] == v, (k, best, fastest)
    plan = L.BatchPlan(b["offsets"], 5, tuning=best, degree=b["degree"])
    t_best, out = _time(L, x, y, b, plan)
    assert check_batch(L, b, {**out, "Xt": out["Xt"], "sums": out["sums"], "map": out["map"]}, "comp",
                       series=range(0, 6000, 7), sums_every=8) > 800
    t_default, _ = _time(L, x, y, b, L.BatchPlan(b["offsets"], 5, degree=b["degree"]))
    assert t_best <= 1.10 * t_default + 0.02, (t_best, t_default, best)
    # a second call is answered from the cache, without measuring
    best2, results2 = autotune.tune_batched(x, y, b["offsets"], b["degree"], b["interval"], m_max=5)
    assert best2 == best and results2 == []
    assert len(autotune.load_cache()) == 1
