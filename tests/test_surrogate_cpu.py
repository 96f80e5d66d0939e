"""Host logic of the warm-start comparison (no GPU): how long the cold run is
continued for the reference permeability, and which permeabilities the
errors compare.  The solver runs and the prediction are replaced by fakes;
the geometry is built on the host as in a real run."""
import numpy as np
import pytest

from paper_1507_06565_gb300 import surrogate as S


def test_relaxation_steps_is_the_slowest_viscous_decay_time():
    # nz^2 / (pi^2 nu) with nu = (tau - 1/2) / 3: tau = 0.8 -> nu = 0.1
    case = S.channel_case(600000, (32, 32, 64))
    assert case.tau == pytest.approx(0.8)
    assert S.relaxation_steps(case) == pytest.approx(64 ** 2 / (np.pi ** 2 * 0.1))


def test_warm_vs_cold_judges_both_runs_against_the_continued_cold_run(monkeypatch):
    calls = []

    def fake_time_to_steady(case, u0=None, tol=1e-8, interval=500, max_steps=2_000_000, geom=None,
                            flags=S.WALL_FLAGS, ref_steps=0):
        calls.append({"warm": u0 is not None, "ref_steps": ref_steps, "tol": tol, "interval": interval})
        if u0 is None:   # cold: converged K 2.0, reference (continued) K 2.002
            return {"status": 0, "steps": 1000, "residual": tol, "seconds": 4.0, "permeability": 2.0,
                    "ref_steps": ref_steps, "permeability_ref": 2.002}
        return {"status": 0, "steps": 600, "residual": tol, "seconds": 2.0, "permeability": 2.001}

    class FakeField:
        def contiguous(self):
            return self

    monkeypatch.setattr(S, "time_to_steady", fake_time_to_steady)
    monkeypatch.setattr(S, "predict", lambda params, case, geom=None: FakeField())
    import torch

    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a, **k: None)
    shape = (32, 32, 64)
    rows = S.warm_vs_cold(None, [600000, 600001], shape, tol=1e-8, interval=500, ref_relaxations=4.0)
    assert len(rows) == 2 and len(calls) == 4
    expect_ref = int(np.ceil(4.0 * S.relaxation_steps(S.channel_case(600000, shape)) / 500)) * 500
    for r, (cold, warm) in zip(rows, (calls[0:2], calls[2:4])):
        # the cold run carries the untimed continuation, the warm run none
        assert not cold["warm"] and cold["ref_steps"] == expect_ref and expect_ref % 500 == 0
        assert warm["warm"] and warm["ref_steps"] == 0
        assert cold["tol"] == warm["tol"] == 1e-8
        assert r["k_err_cold"] == pytest.approx(abs(2.0 / 2.002 - 1.0))
        assert r["k_err_warm"] == pytest.approx(abs(2.001 / 2.002 - 1.0))
        assert r["k_rel_diff"] == pytest.approx(abs(2.001 / 2.0 - 1.0))
        # the prediction's time is counted in the warm run's wall time
        assert r["warm"]["seconds"] >= 2.0 and r["warm"]["inference_s"] >= 0.0
