"""bench.py's multi-rank harness on CPU: two gloo ranks (replicas only, no data-path collective) agree on the
barrier and on the maximum of their timings, the reference arm prints from rank 0 alone, and the GPU arm's JSON
line carries every key of its contract (with stand-ins for the library)."""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist, r, ws, local = bench._dist()
    bench._barrier(dist)
    out[rank] = (r, ws, bench._max_over_ranks(dist, 1.5 + rank))
    dist.destroy_process_group()


def test_two_gloo_ranks_share_barrier_and_max_timing():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    mp.start_processes(_rank, args=(_free_port(), out), nprocs=2, start_method="spawn", join=True)
    assert sorted(out.keys()) == [0, 1]
    for rank in (0, 1):
        r, ws, m = out[rank]
        assert (r, ws) == (rank, 2) and m == 2.5


def test_reference_arm_prints_from_rank_zero_only(tmp_path):
    port = _free_port()
    procs = []
    for rank in (0, 1):
        env = dict(os.environ, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE="2", RANK=str(rank),
                   LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                                       "--gpus", "2", "--steps", "1", "--warmup", "0"],
                                      cwd=ROOT, env=env, stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = [p.communicate(timeout=600) for p in procs]
    assert all(p.returncode == 0 for p in procs), [o[1][-2000:] for o in outs]
    lines0 = [l for l in outs[0][0].splitlines() if l.startswith("{")]
    lines1 = [l for l in outs[1][0].splitlines() if l.startswith("{")]
    assert len(lines0) == 1 and not lines1
    rec = json.loads(lines0[0])
    assert rec["impl"] == "reference" and rec["value"] > 0 and rec["e2e"]["h2d_bytes_per_step"] == 0


def test_gpu_arm_json_contract_with_a_stand_in_library(monkeypatch, capsys):
    """bench.run_ours end to end on the host with the library and the CUDA calls replaced by stand-ins that return
    fixed numbers: every key of the JSON line is present and consistent (this checks the harness, not the GPU)."""
    import types
    import torch
    sys.path.insert(0, ROOT)
    import bench
    import paper_2403_08063_gb300 as pkg
    import synthetic as syn

    class Event:
        clock = 0.0

        def __init__(self, enable_timing=True):
            self.t = 0.0

        def record(self, stream=None):
            Event.clock += 0.05
            self.t = Event.clock

        def elapsed_time(self, other):
            return (other.t - self.t) * 1e3

    class StandIn:
        set_rhs_calls = 0

        def __init__(self, R, n, keys, coeff=False, precision=0, inner_cycles=1, **kw):
            self.n, self.nl = n, len(keys)

        def set_rhs(self, f, k=None):
            StandIn.set_rhs_calls += 1

        def levels(self):
            return [(self.nl, self.n), (self.nl, self.n // 2)]

        def solve(self, u, rtol=1e-10, max_cycles=100):
            return 12, 5e-11

        def solve_host(self, f, k=None, u=None, rtol=1e-10, max_cycles=100):
            return u, 12, 5e-11

        def profile(self, on=True):
            pass

        def profile_read(self):
            return {"smooth_f32_finest": (117.9, 480), "smooth_f32": (37.7, 2400), "residual_f64": (34.5, 20)}

        def smoother_shape(self, level):
            return (2, 16, 32, 4, 4)

        def tail_level(self):
            return -1

        def close(self):
            pass

    class Sampler:
        def __init__(self, index):
            pass

        def start(self):
            pass

        def stop(self):
            return {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": [], "samples": 3}

    def inputs(workload, device, seed=0):
        R, n, keys = syn.workload_forest("uniform_2x8")
        f = torch.zeros(len(keys), n ** 3, dtype=torch.float64)
        return R, n, keys, torch.ones_like(f), f

    monkeypatch.setattr(pkg, "Forest", StandIn)
    monkeypatch.setattr(pkg, "alu_peaks", lambda: (1.2, 70.0))
    monkeypatch.setattr(torch.cuda, "Event", Event)
    for name in ("synchronize", "set_device", "current_stream"):
        monkeypatch.setattr(torch.cuda, name, lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda.nvtx, "range_push", lambda *a, **k: None)
    monkeypatch.setattr(torch.cuda.nvtx, "range_pop", lambda *a, **k: None)
    monkeypatch.setattr(torch.Tensor, "pin_memory", lambda self: self)
    monkeypatch.setattr(bench, "ClockSampler", Sampler)
    monkeypatch.setattr(bench, "_inputs", inputs)
    args = types.SimpleNamespace(workload="uniform_8x64_k", inner_cycles=4, tail="auto", smoother_shape="",
                                 warmup=3, steps=5, rtol=1e-10, no_cpu_baseline=True, gpus=1, no_other_configs=True,
                                 coarse_coef="faces")
    bench.run_ours(args)
    lines = [l for l in capsys.readouterr().out.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
                "vs_baseline", "dtype", "data", "config", "roofline", "e2e", "gpu_launches", "clocks", "setup_ms",
                "smoother_finest", "time_to_rtol_s"):
        assert key in d, key
    assert d["steps"] == 5 and d["warmup"] == 3 and d["n_gpus"] == 1 and d["cycles_per_solve"] == [12] * 5
    assert d["gpu_launches"] == 2900 and d["config"]["workload"] == "uniform_8x64_k"
    roof = d["roofline"]
    assert roof["kernel"] == "smooth_f32_finest" and roof["bound"] == "hbm" and roof["launches"] == 480
    assert abs(roof["frac"] - roof["achieved"] / roof["peak"]) < 1e-12
    assert d["smoother_finest"]["sweeps"] == 240
    cells = 8 * 8 ** 3  # the stand-in forest: 8 leaves of 8^3
    # achieved = 8 algorithmic bytes per cell and one-colour launch over the family's mean launch time
    assert abs(roof["achieved"] - 8.0 * cells * 480 / 0.1179 / 1e9) < 1e-9 * roof["achieved"]
    assert roof["algorithmic_bytes_per_cell"] == 8.0 and roof["schedule_bytes_per_cell"] == 10.0
    assert abs(roof["frac_schedule_bytes"] - 1.25 * roof["frac"]) < 1e-12
    cyc = d["cycle_roofline"]
    assert abs(cyc["achieved_gbs"] - d["value"] * 78.0) < 1e-9 and abs(cyc["frac"] * cyc["peak_gbs"] -
                                                                     cyc["achieved_gbs"]) < 1e-9
    assert d["e2e"]["h2d_bytes_per_step"] == 2 * cells * 8 and d["e2e"]["d2h_bytes_per_step"] == cells * 8
    assert d["alu_peaks_tflops"]["fp64_fma"] == 1.2 and d["alu_peaks_tflops"]["fp32_fma"] == 70.0
    assert d["config"]["coarse_coefficients"].startswith("face-averaged")
    alt = d["other_coarse_operator"]
    assert alt["coarse_coefficients"].startswith("rediscretised") and alt["fp64"]["cycles"] == 12
    assert abs(cyc["frac_with_face_coarse_bytes"] * cyc["peak_gbs"] - d["value"] * (78.0 + 40.0 / 7.0)) < 1e-9
    # the timed forest's set-up, two set-up repeats, the FP64 forest's, the two forests of the other coarse operator
    assert StandIn.set_rhs_calls == 6


def test_host_cpu_description():
    sys.path.insert(0, ROOT)
    import bench
    d = bench._host_cpu()
    assert d["nproc"] == os.cpu_count() and isinstance(d["cpu_model"], str) and d["cpu_model"]
