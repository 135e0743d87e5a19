"""Host logic of the default bench run's oracle legs (CPU): every workload of the
run gets a cpu_baseline object beside its GPU figures; a workload without a
bounded oracle sample says why; a failing sample is reported, never raised;
--no-cpu-baseline skips them.  The GPU measurements are stubbed here."""
import types

import pytest


@pytest.fixture()
def bench(monkeypatch):
    import bench as b
    for name in ("run_small_lp", "run_batch", "run_knapsack", "run_qp", "run_shared"):
        monkeypatch.setattr(b, name, lambda args, _n=name: {"value": 1.0, "unit": "x", "fn": _n})
    return b


def _args(no_cpu=False):
    return types.SimpleNamespace(steps=5, warmup=3, fp64_steps=3, no_cpu_baseline=no_cpu)


def test_every_workload_gets_an_oracle_leg(bench, monkeypatch):
    calls = []

    def leg(name):
        calls.append(name)
        if name == "qp_200k":
            raise RuntimeError("boom")
        if name in bench.ORACLE_SKIPPED:
            return None
        return {"value": 2.0, "unit": "x", "cores": 1, "kind": "oracle", "sample": "s"}

    monkeypatch.setattr(bench, "oracle_leg", leg)
    out = bench.run_subworkloads(_args())
    assert set(out) == {"small_lp_200x400", "ragged_lp_4096", "knapsack_1000x100000",
                        "qp_200k", "shared_dense_512"}
    assert calls == list(out)
    assert out["small_lp_200x400"]["cpu_baseline"]["value"] == 2.0
    assert out["qp_200k"]["cpu_baseline"]["error"] == "RuntimeError: boom"
    assert out["qp_200k"]["value"] == 1.0  # the GPU figure is kept
    for name in bench.ORACLE_SKIPPED:
        cb = out[name]["cpu_baseline"]
        assert cb["value"] is None and cb["note"].startswith("not sampled")
    assert all("cpu_baseline_s" in v for v in out.values())


def test_no_cpu_baseline_skips_the_legs(bench, monkeypatch):
    monkeypatch.setattr(bench, "oracle_leg", lambda name: pytest.fail("leg ran"))
    out = bench.run_subworkloads(_args(no_cpu=True))
    assert all("cpu_baseline" not in v for v in out.values())


def test_small_lp_leg_runs_the_oracle(bench):
    cb = bench.oracle_leg("small_lp_200x400")
    assert cb["kind"] == "oracle" and cb["unit"] == "s" and cb["cores"] == 1
    assert cb["value"] > 0 and "optimal" in cb["sample"]
