"""Host-side logic of bench.py's multi-process path (replicas, no data-path
collective): the max-over-ranks reduction and the whole-job value on two
gloo ranks, rank-0-only output, and the reference arm's non-zero ranks."""
import importlib.util
import os
import subprocess
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        ws, r, _ = b.dist_env()
        # each rank timed its own replica: rank r took 10·(r+1) ms for 5 steps
        el_ms, e2e_s = b.max_over_ranks(dist, [10.0 * (rank + 1), 0.001 * (2 - rank)], "cpu")
        ms = el_ms / 5
        printed = b.emit({"rank": r}, r)
        out.put((rank, ws, r, el_ms, e2e_s, b.job_value(ws, 1000, ms), printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_and_value():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ws, r, el_ms, e2e_s, value, printed in res:
        assert (ws, r) == (2, rank)
        assert el_ms == 20.0 and e2e_s == pytest.approx(0.002)  # the slowest rank's times
        assert value == pytest.approx(2 * 1000 / (4.0e-3))       # both replicas over the max time
        assert printed == (rank == 0)


def test_max_over_ranks_without_group():
    b = _bench()
    assert b.max_over_ranks(None, [1, 2.5], "cpu") == [1.0, 2.5]
    assert b.job_value(1, 512 ** 3, 1.0) == pytest.approx(512 ** 3 / 1e-3)


def test_reference_arm_other_ranks_exit_without_work():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env,
                       timeout=120)
    assert r.returncode == 0
    assert r.stdout.strip() == ""


def test_l2_note_flags_grids_whose_spectrum_fits_in_l2():
    b = _bench()
    # 512^3: half spectrum 512·512·257·8 B = 539 MB > 129 MB
    assert b.l2_note((512, 512, 512)).startswith("every pass's arrays larger")
    # 256^3: 67 MB spectrum stays in L2 between passes
    assert b.l2_note((256, 256, 256)).startswith("L2-influenced")


def test_traffic_record_matches_current_sources_or_is_dropped(monkeypatch):
    b = _bench()
    # the committed record is keyed to the sources of the recorded kernels
    rec = b.recorded_traffic("xdiv", 512 ** 3)
    assert rec is None or 1.0e9 < rec < 1.2e9  # 8 B per unknown = 1.07 GB per pass
    # a record keyed to other sources is not used
    monkeypatch.setattr(b, "kernel_digest", lambda: "0000000000000000")
    assert b.recorded_traffic("xdiv", 512 ** 3) is None


def test_solve_dram_frac_sums_every_pass_or_is_none():
    b = _bench()
    passes = {"zfwd": 0.17, "yfwd": 0.17, "xdiv": 0.27, "yinv": 0.17, "zinv": 0.17}
    frac = b.solve_dram_frac(passes, 512 ** 3, 0.94, 6793.8)
    if b.recorded_traffic("xdiv", 512 ** 3) is not None:
        # five passes of about 1.03 GB each in 0.94 ms: about 0.8 of 6.79 TB/s
        assert 0.7 < frac < 0.9
    assert b.solve_dram_frac(dict(passes, other=0.1), 512 ** 3, 0.94, 6793.8) is None
    assert b.solve_dram_frac({}, 512 ** 3, 0.94, 6793.8) is None


def test_digest_ignores_comments_but_not_code():
    b = _bench()
    src = 'int a = 1; // note\n/* block\n */ const char *s = "// kept"; int d = 2 /* x */ + 3;\n'
    assert b.code_only(src) == b.code_only(src.replace("note", "other").replace("block", "text"))
    assert "// kept" in b.code_only(src)
    assert b.code_only(src) != b.code_only(src.replace("2 /* x */ + 3", "2 + 4"))


def test_batch_errors_against_the_oracle():
    import numpy as np
    import oracle
    oracle.build()
    b = _bench()
    rng = np.random.default_rng(5)
    fs = [rng.standard_normal(s).astype(np.float32) for s in ((8, 12, 6), (6, 4, 8))]
    exact = [oracle.solve(f.astype(np.float64)) for f in fs]
    assert max(b.batch_errors(oracle, fs, exact)) < 1e-14
    wrong = [exact[0], exact[1] * 1.01]
    errs = b.batch_errors(oracle, fs, wrong)
    assert errs[0] < 1e-14 and abs(errs[1] - 0.01) < 1e-9


def test_batch_sample_size_is_bounded_and_at_least_one():
    import numpy as np
    import oracle
    oracle.build()
    b = _bench()
    fs = [np.zeros((16, 16, 16)) for _ in range(5)]
    assert b.batch_sample_size(oracle, fs, 0.0) == 1
    assert b.batch_sample_size(oracle, fs, 1e6) == 5


def test_traffic_record_only_for_the_captured_kernels():
    b = _bench()
    if b.recorded_traffic("xdiv", 512 ** 3) is None:
        pytest.skip("no record for the current sources")
    assert b.recorded_traffic("xdiv", 256 ** 3, (256, 256, 256)) is None
    assert b.recorded_traffic("xdiv", 512 ** 3, (512, 512, 512), "helmholtz") is None


def test_clock_rows_parsed_with_throttle_reasons():
    b = _bench()
    rows = "\n".join([
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, 1980, 2070, 1390.5, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 10.0, 0x0, Not Active, Not Active, Not Active, Not Active",  # skipped
        "garbage",
    ])
    c = b.parse_clocks(rows)
    assert c == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    hot = rows.replace("Not Active, Not Active, Not Active, Active", "Active, Not Active, Active, Not Active")
    assert b.parse_clocks(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert b.parse_clocks("")["sm_mhz"] is None


def test_cpu_baseline_leg_times_the_oracle():
    b = _bench()
    rate, t, reps, cores = b.oracle_rate(16, max_seconds=0.2, min_reps=2)
    assert reps >= 2 and t > 0 and cores >= 1
    assert rate == pytest.approx(16 ** 3 / t)
