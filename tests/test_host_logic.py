"""Host-side logic of the C ABI that runs without a GPU: the ensemble
schedule (longest-processing-time packing) and the tuning-override
validation."""
import numpy as np
import pytest

from paper_2106_11143_gb300 import workloads as W


@pytest.fixture(scope="module")
def api():
    from paper_2106_11143_gb300 import api as a
    from paper_2106_11143_gb300 import build
    build.build()
    a.lib()
    return a


def test_plan_every_instance_once_and_lpt_bound(api):
    w = W.kz_ensemble()
    off = w["offsets"]
    cost = np.diff(off).astype(float) ** 2
    for n_bins in (1, 7, 152, 512):
        order, start, mx, mean = api.plan_batched(off, n_bins)
        assert sorted(order.tolist()) == list(range(len(off) - 1))
        assert start[0] == 0 and start[-1] == len(off) - 1 and np.all(np.diff(start.astype(int)) >= 0)
        loads = [cost[order[start[b]:start[b + 1]]].sum() for b in range(n_bins)]
        assert max(loads) == mx
        assert abs(np.mean(loads) - mean) <= 1e-9 * mean
        # Graham's bound for LPT: makespan <= (4/3 - 1/(3m)) OPT, OPT >= max(mean, max item)
        opt_lb = max(cost.sum() / n_bins, cost.max())
        assert mx <= (4 / 3 - 1 / (3 * n_bins)) * opt_lb * (1 + 1e-12) or mx <= (4 / 3) * opt_lb


def test_plan_is_deterministic_and_lpt_greedy(api):
    off = np.array([0, 3, 13, 14, 24, 30])
    o1 = api.plan_batched(off, 2)
    o2 = api.plan_batched(off, 2)
    assert np.array_equal(o1[0], o2[0]) and np.array_equal(o1[1], o2[1])
    # costs 9, 100, 1, 100, 36 taken in the order 1, 3, 4, 0, 2 (ties by index),
    # each to the lightest bin (ties to the lower bin): {1, 4} = 136, {3, 0, 2} = 110
    order, start, mx, mean = o1
    bins = [sorted(order[start[b]:start[b + 1]].tolist()) for b in range(2)]
    assert bins == [[1, 4], [0, 2, 3]]
    assert mx == 136.0 and mean == 123.0


def test_plan_rejects_bad_input(api):
    with pytest.raises(api.NBError):
        api.plan_batched(np.array([0, 5, 3]), 2)
    with pytest.raises(api.NBError):
        api.plan_batched(np.array([0, 5]), 0)


def test_tuning_validation(api):
    with pytest.raises(api.NBError):
        api.set_tuning("force", "fp64", 0, 100, 48)
    with pytest.raises(api.NBError):
        api.set_tuning("potential", "fp64", 0, 100, 64, R=2)
    with pytest.raises(api.NBError):
        api.set_tuning("ensemble", "fp64", 0, 100, 1024)
    with pytest.raises(api.NBError):
        api.set_tuning("symmetric_vjp", "fp64", 0, 100, 512)
    with pytest.raises(api.NBError):
        api.set_tuning("symmetric_vjp", "fp64", 0, 100, 128, R=2)
    api.set_tuning("symmetric_vjp", "fp64", 0, 100, 256, R=0)
    api.set_tuning("force", "fp64", 0, 100, 64, R=2, blocks_per_sm=8)
    # step windows, single-block steps, epilogue lanes: R is 0 or 1, block >= 1
    for kind in ("step_windows", "small_steps", "epilogue_lanes"):
        api.set_tuning(kind, "fp64", 0, 100, 1, R=0)
        api.set_tuning(kind, "fp64", 0, 100, 64, R=1)
        with pytest.raises(api.NBError):
            api.set_tuning(kind, "fp64", 0, 100, 1, R=2)
        with pytest.raises(api.NBError):
            api.set_tuning(kind, "fp64", 0, 100, -1, R=1)
    with pytest.raises(api.NBError):
        api.set_tuning(9, "fp64", 0, 100, 1, R=1)  # no such kind
    for block in (32, 64):  # the small symmetric blocks
        api.set_tuning("symmetric", "fp64", 0, 100, block, R=1)
    with pytest.raises(api.NBError):
        api.set_tuning("symmetric", "fp64", 0, 100, 96, R=1)
    api.set_tuning("force", "fp64", 0, 0, 0)  # clear


def test_system_state_round_trip(api, tmp_path):
    """state_dict / from_state keep every array bit for bit, through a file."""
    import numpy as np
    import torch
    rng = np.random.default_rng(3)
    s = api.System(rng.standard_normal((3, 17)), rng.standard_normal((3, 17)),
                   q=rng.standard_normal(17), device="cpu", step=41, m=rng.uniform(1, 2, 17))
    s.ax.copy_(torch.from_numpy(rng.standard_normal(17)))
    path = tmp_path / "state.pt"
    torch.save(s.state_dict(), path)
    r = api.System.from_state(torch.load(path), device="cpu")
    assert r.n == 17 and r.step == 41
    for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "q", "m"):
        assert torch.equal(getattr(r, k), getattr(s, k)), k


def test_system_packed_state(api):
    """The nine state arrays are rows of System.state (rows padded to 32
    doubles, 256 B): writes through either name are seen through the other,
    rows start 256-byte aligned, and a view's state is the column slice."""
    import numpy as np
    import torch
    rng = np.random.default_rng(5)
    for n in (1, 31, 32, 33, 100):
        pos, vel = rng.standard_normal((3, n)), rng.standard_normal((3, n))
        s = api.System(pos, vel, device="cpu")
        assert s.state.shape == (9, max(32, -(-n // 32) * 32)) and s.state.is_contiguous()
        for k, name in enumerate(api.STATE_NAMES):
            row = getattr(s, name)
            assert row.shape == (n,) and row.data_ptr() == s.state[k].data_ptr()
            assert row.data_ptr() % 256 == (s.state.data_ptr() % 256)
        assert np.array_equal(s.pos().numpy(), pos) and np.array_equal(s.vel().numpy(), vel)
        assert torch.count_nonzero(s.acc()) == 0
        s.state[7, :n] = 3.0
        assert torch.all(s.ay == 3.0)
        s.vz.fill_(-1.0)
        assert torch.all(s.state[5, :n] == -1.0)
        if n > 3:
            v = s.view(1, 3)
            assert v.state.shape == (9, 2) and torch.equal(v.state[0], s.x[1:3])
            assert v.vz.data_ptr() == s.vz[1:].data_ptr()


def test_checkpoint_file_round_trip(api, tmp_path):
    """save_checkpoint / load_checkpoint: the framework-free file keeps every
    array, the step counter and the parameters bit for bit, with and without
    q, m and params; malformed files raise ValueError."""
    import numpy as np
    import torch
    rng = np.random.default_rng(4)
    n = 23
    s = api.System(rng.standard_normal((3, n)) * 1e-5, rng.standard_normal((3, n)),
                   q=rng.standard_normal(n), device="cpu", step=(1 << 40) + 3, m=rng.uniform(1, 2, n))
    s.az.copy_(torch.from_numpy(rng.standard_normal(n)))
    par = api.Params(k_coulomb=8.9875517923e9, mass=6.6e-26, charge=1.602176634e-19, soft2=1e-18,
                     trap="rf", precision="df64", omega=(0.1, 2.0 / 3.0, 1e6), omega_rate=(0.0, -1e-3, 7.0),
                     q_mathieu=0.3, omega_rf=6.283e7, rf_phase=1.0 / 7.0, gamma=1e-20, dt=2e-9,
                     t0=1e-7, noise_T=5e-4, seed=(1 << 63) + 5, instance=9)
    path = tmp_path / "state.nbck"
    api.save_checkpoint(path, s, par)
    r, p = api.load_checkpoint(path, device="cpu")
    assert r.n == n and r.step == s.step and p == par
    for k in ("x", "y", "z", "vx", "vy", "vz", "ax", "ay", "az", "q", "m"):
        assert torch.equal(getattr(r, k), getattr(s, k)), k
    # no charges, masses or params
    s2 = api.System(rng.standard_normal((3, 5)), device="cpu", step=7)
    api.save_checkpoint(tmp_path / "b.nbck", s2)
    r2, p2 = api.load_checkpoint(tmp_path / "b.nbck", device="cpu")
    assert p2 is None and r2.q is None and r2.m is None and r2.step == 7
    assert torch.equal(r2.x, s2.x)
    # malformed files
    raw = path.read_bytes()
    for bad in (b"XXXXXXX\n" + raw[8:], raw[:-8], raw + b"\0"):
        (tmp_path / "bad.nbck").write_bytes(bad)
        with pytest.raises(ValueError):
            api.load_checkpoint(tmp_path / "bad.nbck", device="cpu")


PLAN_NS = [1, 2, 3, 7, 8, 15, 16, 17, 31, 32, 33, 47, 48, 49, 63, 64, 65, 100, 127, 128, 129, 255, 256,
           257, 499, 500, 501, 999, 1000, 1001, 1499, 1500, 1501, 1999, 2000, 2047, 2048, 2499, 2500,
           2999, 3000, 3001, 4095, 4096, 4097, 7999, 8000, 8191, 8192, 9999, 10000, 24000, 32767,
           32768, 59999, 60000, 100000, 262151]


def test_plan_invariants(api):
    """Every launch plan (host only, no GPU) covers all n ions and all
    partners: the one-sided kernel's i-tiles and j-chunks tile [0, n) and its
    grid stays within the launch limits; the symmetric kernel's blocks of a
    supported size cover [0, n), with one partial slot per block for small
    schedules and the in-place round-ordered output for large ones; the
    single-block path is
    offered only within its 512-ion limit and never with the symmetric
    kernel."""
    import math
    for kind, precs in (("force", list(api.PRECISIONS)), ("potential", ["fp64"]), ("vjp", ["fp64"])):
        for prec in precs:
            for n in PLAN_NS:
                p = api.plan_info(kind, prec, n)
                if p["symmetric"]:
                    assert p["G"] in ((1, 2, 4, 8, 16, 32) if kind == "force" else (4, 8)), (kind, prec, n, p)
                    nbk = math.ceil(n / (32 * p["G"]))
                    assert p["n_it"] == nbk and nbk <= 60000, (kind, prec, n, p)  # blocks
                    # round-ordered in-place adds for large schedules or partials, else one slot per block
                    inplace = nbk >= 96 or nbk * 3 * n * 8 > 1e9
                    assert p["n_jc"] == (1 if inplace else nbk), (kind, prec, n, p)
                else:
                    assert p["block"] in (32, 64, 128, 256) and p["R"] in (1, 2, 4), (kind, prec, n, p)
                    assert p["n_it"] == math.ceil(n / (p["block"] * p["R"])), (kind, prec, n, p)
                    assert p["jchunk"] >= 1
                    assert (p["n_jc"] - 1) * p["jchunk"] < n <= p["n_jc"] * p["jchunk"], (kind, prec, n, p)
                    assert p["n_jc"] <= 65535  # grid.y
                if p["single_block"]:
                    assert kind == "force" and n <= 512 and not p["symmetric"], (prec, n, p)


def test_plan_thresholds(api):
    """The documented defaults: the symmetric force kernel from n = 500
    (mixed_split), 1000 (mixed), 1500 (fp64) and 2000 (df64), never in the
    ladder modes; the symmetric VJP from n = 2500; the single-block steps up
    to 32 ions (48 for df64, 16 for sqrtdiv); and the tuning overrides."""
    for prec, start in (("mixed_split", 500), ("mixed", 1000), ("fp64", 1500), ("df64", 2000)):
        assert not api.plan_info("force", prec, start - 1)["symmetric"]
        assert api.plan_info("force", prec, start)["symmetric"]
    for prec in ("sqrtdiv", "rsq", "rsq_nr1", "rsq_nr2"):
        assert not api.plan_info("force", prec, 100000)["symmetric"]
    # no memory cap: the half-pair kernel needs only its output, so it serves
    # every size up to its 60000-block schedule limit
    for prec in ("fp64", "df64", "mixed", "mixed_split"):
        for n in (2_000_000, 20_000_000):
            p = api.plan_info("force", prec, n)
            assert p["symmetric"] and p["n_jc"] == 1, (prec, n, p)
    assert api.plan_info("vjp", "fp64", 5_000_000)["symmetric"]
    assert not api.plan_info("vjp", "fp64", 2499)["symmetric"]
    assert api.plan_info("vjp", "fp64", 2500)["symmetric"]
    for prec, top in (("fp64", 32), ("mixed", 32), ("mixed_split", 32), ("df64", 48), ("sqrtdiv", 16),
                      ("rsq", 32), ("rsq_nr1", 32), ("rsq_nr2", 32)):
        assert api.plan_info("force", prec, top)["single_block"] == 1, prec
        assert api.plan_info("force", prec, top + 1)["single_block"] == 0, prec
    try:
        api.set_tuning("symmetric", "fp64", 0, 1 << 40, 128, R=0)
        assert not api.plan_info("force", "fp64", 100000)["symmetric"]
        api.set_tuning("symmetric", "fp64", 0, 1 << 40, 64, R=1)
        p = api.plan_info("force", "fp64", 600)
        assert p["symmetric"] and p["G"] == 2
        api.set_tuning("small_steps", "fp64", 0, 1 << 40, 1, R=1)
        assert api.plan_info("force", "fp64", 400)["single_block"] == 0  # symmetric plan: not eligible
        api.set_tuning("force", "fp64", 0, 0, 0)
        api.set_tuning("small_steps", "fp64", 0, 1 << 40, 1, R=1)
        assert api.plan_info("force", "fp64", 200)["single_block"] == 1
        assert api.plan_info("force", "fp64", 513)["single_block"] == 0  # above the block's limit
    finally:
        api.set_tuning("force", "fp64", 0, 0, 0)
    with pytest.raises(api.NBError):
        api.plan_info("force", "fp64", 0)


def test_vjp_and_potential_plans_shared_by_precisions(api):
    """The potential and VJP plans do not depend on the precision argument
    (the NB_DF64 VJP runs on the fp64 VJP plan), and a symmetric-VJP override
    given for NB_FP64 reshapes them all."""
    for n in (100, 2499, 2500, 16383, 16384, 100000):
        for kind in ("potential", "vjp"):
            base = api.plan_info(kind, "fp64", n)
            for prec in ("df64", "mixed", "mixed_split"):
                assert api.plan_info(kind, prec, n) == base, (kind, prec, n)
    try:
        api.set_tuning("symmetric_vjp", "fp64", 0, 1 << 40, 256, R=1)
        for prec in ("fp64", "df64"):
            p = api.plan_info("vjp", prec, 3000)
            assert p["symmetric"] and p["G"] == 8, (prec, p)
        api.set_tuning("symmetric_vjp", "fp64", 0, 1 << 40, 128, R=0)
        assert not api.plan_info("vjp", "df64", 100000)["symmetric"]
    finally:
        api.set_tuning("force", "fp64", 0, 0, 0)


def test_symmetric_schedule(api):
    """The half-pair kernels' work schedule: every unordered block pair and
    every block's own item exactly once; each round touches each block
    exactly once, so the adds into a block happen one round after another;
    items are numbered in round order (an item waits only on lower-numbered
    ones, which keeps the grid progressing); rounds number nbk."""
    for nbk in list(range(1, 41)) + [195, 196, 391, 1001]:
        P, Q, R = api.sym_schedule(nbk)
        assert len(P) == nbk * (nbk + 1) // 2
        assert np.all(P <= Q) and np.all(P >= 0) and np.all(Q < nbk)
        pairs = P.astype(np.int64) * nbk + Q
        assert len(np.unique(pairs)) == len(pairs)  # each block pair once; with P <= Q: all of them
        assert np.all(np.diff(R) >= 0) and R[0] == 0 and R[-1] == nbk - 1
        for r in range(nbk):
            sel = R == r
            touched = np.concatenate([P[sel], Q[sel][Q[sel] != P[sel]]])
            assert np.array_equal(np.sort(touched), np.arange(nbk)), (nbk, r)
    with pytest.raises(api.NBError):
        api.sym_schedule(0)


def test_noalloc_capacity_holds_to_a_million(api):
    """nb_energy_noalloc's fixed array (2^20 doubles) holds the potential
    plan's partials (n_jc * n) plus 3 * 128 + 4 reduction doubles for every
    n up to 1e6 with the default plan on 152 SMs (the host-only planner's
    GPU), and no longer at 1.1e6, which its GPU test rejects."""
    cap = 1 << 20
    ns = sorted(set(np.unique(np.geomspace(1, 1_000_000, 400).astype(np.int64)).tolist()
                    + list(range(999_000, 1_000_001, 97)) + [1_000_000]))
    for n in ns:
        p = api.plan_info("potential", "fp64", n)
        assert p["n_jc"] * n + 3 * 128 + 4 <= cap, (n, p)
    p = api.plan_info("potential", "fp64", 1_100_000)
    assert p["n_jc"] * 1_100_000 + 388 > cap


def test_bench_roofline_and_kernel_label(api):
    """bench.py's roofline entry: convention-A flops (20 per evaluation) on
    the evaluations the planned kernel performs -- (N^2 + sum_b n_b^2)/2 for
    the half-pair kernel's blocks, N^2 for the one-sided kernel -- over the
    kernel time, against 2 flops x the measured lanes/clk/SM x 152 SMs x the
    sampled clock; the kernel label follows the library's own plan."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    peaks = {"dfma": {"lanes_per_clk_per_sm": 2.0, "sm_mhz": 2070.0},
             "ffma": {"lanes_per_clk_per_sm": 128.0, "sm_mhz": 2070.0}}
    n = 100000
    r = bench.roofline(api, "mixed_split", n, 4.853, peaks, 2070.0)
    p = api.plan_info("force", "mixed_split", n)
    assert p["symmetric"] == 1
    bi = 32 * p["G"]
    full, rem = divmod(n, bi)
    evals = (n * n + full * bi * bi + rem * rem) // 2
    assert r["evaluations_per_launch"] == evals
    assert abs(r["achieved"] - 20 * evals / 4.853e-3 / 1e12) < 1e-3
    assert abs(r["peak"] - 2 * 128 * 152 * 2070e6 / 1e12) < 1e-3
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-4
    f = bench.roofline(api, "fp64", n, 91.0, peaks, 2070.0)
    assert abs(f["peak"] - 2 * 2 * 152 * 2070e6 / 1e12) < 1e-3
    assert f["conv_B"]["frac"] < f["frac"] < 1.2  # 16 executed FP64 flops per evaluation
    for prec in ("fp64", "df64", "mixed", "mixed_split"):
        for n in (400, 1499, 1500, 2000, 16384, 100000):
            sym = api.plan_info("force", prec, n)["symmetric"] == 1
            r = bench.roofline(api, prec, n, 1.0, peaks, None)
            assert r["kernel"].startswith("k_pair_sym" if sym else "k_pair_force"), (prec, n)
            assert r["evaluations_per_launch"] == (n * n if not sym else r["evaluations_per_launch"])
    # a traffic figure recorded for other kernel sources is not reported; the one in
    # profiles/ for the headline case is, while the kernel sources match its hash
    assert bench.recorded_traffic("mixed_split", 12345)[0] is None
    t, src = bench.recorded_traffic("mixed_split", 100000)
    assert t is not None and 1e6 < t < 1e8 and src.endswith(".md"), (t, src)
    # the issue roofline: recorded warp instructions per launch over the kernel
    # time, against 4 per clock per SM x 152 SMs x the clock
    c, _ = bench.recorded_counters("mixed_split", 100000)
    r = bench.roofline(api, "mixed_split", 100000, 4.12, peaks, 2070.0)
    iss = r["issue"]
    assert abs(iss["peak"] - 4 * 152 * 2070e6 / 1e9) < 1e-2
    assert abs(iss["achieved"] - c["inst"] / 4.12e-3 / 1e9) < 1e-2
    assert abs(iss["frac"] - iss["achieved"] / iss["peak"]) < 1e-4 and 0.5 < iss["frac"] <= 1.0
    assert 15 < iss["warp_instructions_per_32_evaluations"] < 40
    # the FMA pipe by its work: FP32 lane-cycles per evaluation (a packed
    # .f32x2 instruction two) x evaluations over the kernel time, against the
    # FFMA lanes per clock x 152 SMs x the clock
    mix = bench.recorded_opmix("mixed_split")
    cyc = mix["fadd"] + mix["ffma"] + mix["fmul"] + 2 * (mix["fadd2"] + mix["ffma2"] + mix["fmul2"])
    fm = r["fma_pipe"]
    assert abs(fm["lane_cycles_per_evaluation"] - cyc) < 1e-3 and 20 < cyc < 30
    assert abs(fm["achieved"] - cyc * r["evaluations_per_launch"] / 4.12e-3 / 1e12) < 1e-3
    assert abs(fm["peak"] - 128 * 152 * 2070e6 / 1e12) < 1e-3
    assert abs(fm["frac"] - fm["achieved"] / fm["peak"]) < 1e-4 and fm["frac"] > iss["frac"]
    # convention B on the FP32 pipe: executed flops (FMA 2, add or multiply 1,
    # packed twice that) over 2 flops x the FFMA rate
    flops = 2 * mix["ffma"] + mix["fadd"] + mix["fmul"] + 2 * (2 * mix["ffma2"] + mix["fadd2"] + mix["fmul2"])
    cb = r["conv_B"]
    assert abs(cb["flops_per_evaluation"] - flops) < 1e-3 and 30 < flops < 40
    assert abs(cb["achieved"] - flops * r["evaluations_per_launch"] / 4.12e-3 / 1e12) < 1e-3
    assert abs(cb["frac"] - cb["achieved"] / r["peak"]) < 1e-4 and r["frac"] < cb["frac"] < fm["frac"]
    assert "fma_pipe" not in bench.roofline(api, "fp64", 100000, 91.09, peaks, 2070.0)
    # every path at N = 1e5 has recorded counters, and the unit named as binding
    # is the one with the largest fraction (FP64 pipe for the paths with FP64
    # adds in the pair loop, the FMA pipe for the split forms)
    times = {"fp64": 91.09, "df64": 33.98, "mixed": 31.92, "mixed_split": 4.120, "mixed_split_rsq": 3.675}
    want = {"fp64": "FP64 pipe", "df64": "FP64 pipe", "mixed": "FP64 pipe", "mixed_split": "FMA pipe",
            "mixed_split_rsq": "FMA pipe"}
    for prec, ms in times.items():
        r = bench.roofline(api, prec, 100000, ms, peaks, 2070.0)
        assert r["binding"] == want[prec], (prec, r.get("binding"))
        fr = {"issue": r["issue"]["frac"], "FP64 pipe": r["fp64_pipe"]["frac"],
              "FMA pipe": r.get("fma_pipe", {}).get("frac")}[r["binding"]]
        assert 0.5 < fr <= 1.0, (prec, fr)
    assert abs(bench.roofline(api, "fp64", 100000, 90.98, peaks, 2070.0)["fp64_pipe"]
               ["fp64_instructions_per_evaluation"] - 10.26) < 0.05
    # with a measured add rate, each FP64-bound path's fraction of the ceiling
    # its own mix of adds and FMAs allows
    peaks3 = dict(peaks, dadd={"lanes_per_clk_per_sm": 1.684, "sm_mhz": 2070.0})
    for prec in ("fp64", "df64", "mixed"):
        fp = bench.roofline(api, prec, 100000, times[prec], peaks3, 2070.0)["fp64_pipe"]
        mix = bench.recorded_opmix(prec)
        mix = {k: v for k, v in mix.items() if k in ("dadd", "dfma", "dmul")}
        lanes = sum(mix.values()) / sum(v / {"dadd": 1.684, "dfma": 2.0}[k] for k, v in mix.items() if v)
        assert abs(fp["mix_ceiling"] - lanes * 152 * 2070e6 / 1e12) < 1e-3, prec
        assert 0.85 < fp["frac_of_mix_ceiling"] <= 1.05, (prec, fp["frac_of_mix_ceiling"])
    assert "mix_ceiling" not in bench.roofline(api, "fp64", 100000, 90.98, peaks, 2070.0)["fp64_pipe"]


def test_batched_each_validation(api):
    """nb_step_batched_each checks every entry of its host table before it
    touches the device; an empty ensemble only advances the step."""
    import ctypes as C
    L = api.lib()
    base = W.phys(omega=(1e6, 1e6, 2e5), dt=1e-9)

    def table(*edits):
        ps = [api.Params.from_phys(base, **e) for e in edits]
        return (api.NbParams * len(ps))(*[p.to_c() for p in ps]), len(ps)

    sysm = api.NbSystem()
    sysm.n, sysm.step = 0, 5
    call = lambda tab, n, off: L.nb_step_batched_each(tab, n, off, C.byref(sysm), 3, None)
    offs = lambda k: np.zeros(k + 1, dtype=np.int64)
    tab, n = table({}, {})
    off = offs(2)
    offp = off.ctypes.data_as(C.POINTER(C.c_int64))
    assert call(tab, -1, offp) == 1
    assert call(None, 2, offp) == 1
    assert call(tab, 1025, offp) == 1
    tab, n = table({}, {"mass": 0.0})
    assert call(tab, n, offp) == 1
    assert L.nb_last_error().decode().startswith("per_inst[1]: mass")
    tab, n = table({}, {"precision": "df64"})
    assert call(tab, n, offp) == 1 and "precision" in L.nb_last_error().decode()
    tab, n = table({"precision": "mixed"}, {"precision": "mixed"})
    assert call(tab, n, offp) == 6  # NB_ENOTSUP
    tab, n = table({"dt": 0.0}, {})
    assert call(tab, n, offp) == 1
    bad = np.array([0, 0, 1], dtype=np.int64)
    tab, n = table({}, {})
    assert call(tab, n, bad.ctypes.data_as(C.POINTER(C.c_int64))) == 1  # offsets must end at n
    assert sysm.step == 5
    assert call(tab, n, offp) == 0 and sysm.step == 8
    assert L.nb_step_batched_each(None, 0, None, C.byref(sysm), 2, None) == 0 and sysm.step == 10


def test_workloads_have_no_coincident_ions():
    """Reading C1: the oracle skips the self pair by index, the kernels give a
    pair at r = 0 (without softening) no force; the two agree as long as no
    two distinct ions coincide, so every configured workload (each ensemble
    instance on its own) is checked for that."""
    import time
    t0 = time.time()
    singles = [W.cloud_harmonic_1024(), W.cloud_rf_16384(), W.cloud_large(), W.adjoint_cloud()]
    for w in singles:
        assert W.min_pair_distance(w["pos"]) > 0.0, w["name"]
    for w in (W.kz_ensemble(), W.kz_quench_sweep()):
        off = w["offsets"]
        for k in range(len(off) - 1):
            assert W.min_pair_distance(w["pos"][:, off[k]:off[k + 1]]) > 0.0, (w["name"], k)
    assert time.time() - t0 < 120
