"""The 1/sqrt precision ladder (Sec. IV): every method against the oracle,
with the error each one's arithmetic allows, and their ordering."""
import numpy as np
import pytest
import torch

from paper_2106_11143_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# conditioned-error bounds: the seed's ~2^-22 error, tripled by the cube
# (rsq); one Newton step squares it (about 1.5 e^2, x3); two steps and
# SQRT+DIV reach FP64 rounding.
BOUND = {"sqrtdiv": 2e-14, "rsq": 3e-6, "rsq_nr1": 1e-11, "rsq_nr2": 2e-14}


@pytest.fixture(scope="module")
def nb():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2106_11143_gb300 as nbm
    nbm.lib()
    return nbm


def test_ladder_accuracy_and_order(nb, orc):
    n = 2049
    pos, _ = W.random_cloud(n, seed=13)
    phys = W.phys()
    ax, ay, az, _, absf = orc.coulomb(orc.make_params(**phys), *pos, want_absf=True)
    ref = np.stack([ax, ay, az])
    errs = {}
    for m, bound in BOUND.items():
        s = nb.System(pos)
        nb.forces(nb.Params.from_phys(phys, precision=m), s)
        nb.sync_status()
        g = s.acc().cpu().numpy()
        errs[m] = float(np.max(np.sqrt(np.sum((g - ref) ** 2, axis=0)) / absf))
        assert errs[m] <= bound, (m, errs[m])
    print(errs)
    assert errs["rsq"] > 1e3 * errs["rsq_nr1"]
    assert errs["rsq_nr1"] > errs["rsq_nr2"]


def test_ladder_chain_experiment_runs(nb):
    from paper_2106_11143_gb300 import ladder
    r = ladder.chain(methods=["sqrtdiv", "rsq", "rsq_nr1", "fp64"], steps=400)
    print(r)
    assert r["sqrtdiv"] == 0.0
    assert 0.0 < r["rsq"] < 1e-3
    assert r["rsq_nr1"] < r["rsq"]
    assert 0.12 < r["q_mathieu"] < 0.25


def test_ladder_pancake_experiment(nb):
    """The N = 128 radial-plane crystal, cooled from a disc start: SQRT+DIV is
    the reference, the bare seed differs most, one Newton step brings the
    difference to FP64 rounding, and the crystal lies in one radial plane."""
    from paper_2106_11143_gb300 import ladder
    r = ladder.pancake(methods=["sqrtdiv", "rsq", "rsq_nr1"], steps=3000)
    print(r)
    assert r["sqrtdiv"] == 0.0
    assert 0.0 < r["rsq"] < 1e-6
    assert r["rsq_nr1"] < 1e-12  # a regular crystal: no chaotic growth
    assert r["flatness"] < 1e-6


def test_ladder_speed_runs_every_method_one_sided(nb):
    from paper_2106_11143_gb300 import ladder
    out = ladder.speed(sizes=(1000, 16384), reps=1)
    assert set(out["1000"]) == set(ladder.METHODS)
    assert set(out["16384"]) == set(ladder.METHODS) | {"fp64_sym", "df64_sym"}
    row = out["16384"]
    assert row["sqrtdiv"]["speedup_vs_sqrtdiv_pct"] == 0.0
    # the half-pair kernel does about half the pair arithmetic
    assert row["fp64_sym"]["ms"] < 0.8 * row["fp64"]["ms"]


def test_step_rate_sweep_runs(nb):
    """The step-rate sweep (one call with and without step windows, one call
    per step, caller graph replays) on two small sizes."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    rows = bench.step_sweep(sizes=(10, 1000), precisions=["fp64", "mixed_split"])
    assert len(rows) == 4
    for r in rows:
        for k in ("ms_per_step", "plain_ms_per_step", "per_call_ms_per_step", "graph_ms_per_step"):
            assert r[k] > 0, k


def test_workload_runs_module(nb):
    """The end-to-end workload runner on its small pieces."""
    from paper_2106_11143_gb300 import runs
    from paper_2106_11143_gb300 import workloads as W
    r = runs.cloud_run(W.cloud_harmonic_1024(), "fp64", 10)
    assert r["steps"] == 10 and r["device_ms"] > 0 and np.isfinite(r["final_energy_J"][3])
    k = runs.kz(nsteps=4, chunk=2)
    assert k["steps"] == 4 and k["instances"] == 512


def test_autotuner_quick_round_trip(nb, tmp_path):
    """The autotuner in quick mode (one-sided shapes at n = 3000, symmetric
    blocks at n = 1e5, fp64 and mixed_split): every entry is a valid override;
    applied from its JSON cache, the forces agree with the default shapes to
    rounding (a shape only reorders the sums)."""
    import json
    import torch
    from paper_2106_11143_gb300 import tune
    from paper_2106_11143_gb300 import workloads as W
    entries = []
    for prec in ("fp64", "mixed_split"):
        entries += tune.tune_pair(prec, quick=True, log=lambda *a: None)
        entries += tune.tune_symmetric(prec, quick=True, log=lambda *a: None)
    assert entries and all(e["ms"] > 0 for e in entries)
    path = tmp_path / "cache.json"
    json.dump({"device": torch.cuda.get_device_name(), "entries": entries}, open(path, "w"))
    pos, _ = W.random_cloud(3000, seed=8)
    par = nb.Params.from_phys(W.phys())
    s = nb.System(pos)
    nb.forces(par, s)
    ref = s.acc().clone()
    try:
        assert tune.load(str(path))
        nb.forces(par, s)
        torch.cuda.synchronize()
        nb.sync_status()
        tuned = s.acc()
        assert torch.max(torch.abs(tuned - ref)).item() <= 1e-12 * torch.max(torch.abs(ref)).item()
    finally:
        nb.set_tuning("force", "fp64", 0, 0, 0)
