"""Benchmark of the LOPC hot path on B300.

One step = compress + decompress of a 3D float32 512^3 field (seeded sum of 256
Gaussian bumps plus 3-octave value noise; NOA bound 1e-3 x range) through the C ABI,
with inputs resident in HBM.  Prints ONE JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the plain C reference of the same method) on
a bounded sample of the same workload, on the host cores.  Under torchrun (N > 1)
every rank compresses its own field (replicas; the path does not shard) and rank 0
prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "compress/decompress GB/s (1 B300, bit-exact) & % HBM peak; batched vs per-field; p50/p99"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [c.strip() for c in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = max(smax, float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def make_input(n: int, seed: int):
    from paper_2603_26968_b300 import synth as S
    return S.make_field(S.spec_3d_f32(seed=seed, n=n))


def cpu_oracle_sample(x: np.ndarray, eb: float, sub: int):
    """Oracle compress + decompress of the central sub^3 block (bounded CPU work)."""
    import oracle
    c = [(s - sub) // 2 for s in x.shape]
    blk = np.ascontiguousarray(x[c[0]:c[0] + sub, c[1]:c[1] + sub, c[2]:c[2] + sub])
    t0 = time.perf_counter()
    st = oracle.compress(blk, 1, eb)
    oracle.decompress(st)
    dt = time.perf_counter() - t0
    return blk.nbytes, dt, len(st)


def run_reference(args, rank):
    if rank != 0:
        return
    x = make_input(args.size, seed=1)
    sub = args.cpu_sample
    for _ in range(args.warmup):
        cpu_oracle_sample(x, args.eb, sub)
    tot_b, tot_t = 0, 0.0
    for _ in range(args.steps):
        nb, dt, _ = cpu_oracle_sample(x, args.eb, sub)
        tot_b += nb
        tot_t += dt
    gbs = tot_b / tot_t / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": gbs, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_t / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3d_f32_{args.size}^3 bumps+value-noise, NOA eb {args.eb}; reference arm = CPU oracle "
                               f"on the central {sub}^3 block per step", "field_bytes": int(x.nbytes)},
        "cpu_baseline": {"value": gbs, "unit": "GB/s", "cores": 1, "kind": "oracle",
                         "sample": f"central {sub}^3 block of the field, compress+decompress, single thread"},
        "e2e": {"value": gbs, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=512)
    ap.add_argument("--eb", type=float, default=1e-3)
    ap.add_argument("--extra-ebs", default="1e-2,1e-4")
    ap.add_argument("--cpu-sample", type=int, default=128)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    from paper_2603_26968_b300 import lopc
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    x_np = make_input(args.size, seed=1 + rank)
    nbytes = x_np.nbytes
    dev = torch.device("cuda", local)
    x = torch.from_numpy(x_np).to(dev)
    d = lopc.make_desc(tuple(x.shape), x.dtype, lopc.NOA, args.eb)
    out = torch.empty(lopc.compress_bound(d), dtype=torch.uint8, device=dev)
    ws = torch.empty(lopc.compress_workspace_size(d), dtype=torch.uint8, device=dev)
    xhat = torch.empty_like(x)
    dws = torch.empty(lopc.decompress_workspace_size(d), dtype=torch.uint8, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (126 MB)
    stream = torch.cuda.current_stream()

    def step(eb):
        st = lopc.compress(x, eb, lopc.NOA, out=out, workspace=ws)
        lopc.decompress(st, out=xhat, desc=d, workspace=dws)
        return st

    def timed(eb, k, w, profile=False):
        for _ in range(w):
            step(eb)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        times, tc, td = [], [], []
        if profile:
            lopc.profile_reset()
            lopc.profile_enable(True)
        size = 0
        for _ in range(k):
            flush.zero_()                       # L2 flush between timed steps
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            st = lopc.compress(x, eb, lopc.NOA, out=out, workspace=ws)
            e1.record(stream)
            lopc.decompress(st, out=xhat, desc=d, workspace=dws)
            e2.record(stream)
            torch.cuda.synchronize()
            size = st.numel()
            tc.append(e0.elapsed_time(e1))
            td.append(e1.elapsed_time(e2))
            times.append(e0.elapsed_time(e2))
        prof = lopc.profile_read() if profile else {}
        if profile:
            lopc.profile_enable(False)
        if dist:
            dist.barrier()
        return np.array(times), np.array(tc), np.array(td), size, prof

    # headline: the configured bound, with clocks and per-kernel events
    with ClockSampler(local) as clk:
        times, tc, td, ssize, prof = timed(args.eb, args.steps, args.warmup, profile=True)
    ms_step = float(times.mean())
    if dist:
        t = torch.tensor([ms_step], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_step = float(t.item())
    rounds, runs = lopc.last_stats()
    sweeps, sweeps_max = lopc.last_fixpoint_stats()
    phases = dict(zip(["pass_load", "pass_flags", "pass_fixpoint", "pass_writeback", "pass_bin_record",
                       "rerun_load", "rerun_fixpoint", "unused"], lopc.last_phase_cycles()))
    hbm, peak_kind = peaks()
    cr = nbytes / ssize
    w = 4
    algo_comp = nbytes * 2 + ssize                 # NOA: range pass + tile pass read x; write stream
    algo_dec = ssize + nbytes
    comp_gbs = nbytes / (tc.mean() * 1e-3) / 1e9
    dec_gbs = nbytes / (td.mean() * 1e-3) / 1e9

    # per-kernel table and the dominant kernel's roofline
    npts = nbytes // w
    # algorithmic bytes per step of each kernel: what the method must move (range and
    # tile pass read x; the subbin encoder writes its records; decode reads the stream
    # and writes x_hat); a rerun must read the subbins and masks of the tiles it reruns
    algo_bytes = {"range": nbytes, "tile_pass": nbytes, "encode_subbins": ssize, "decode": ssize + nbytes,
                  "pack": 2 * ssize}
    kern = {}
    for name, (launches, total_ms) in prof.items():
        kern[name] = {"launches": launches, "total_ms": total_ms, "ms_per_launch": total_ms / max(1, launches)}
    dom = max(kern.items(), key=lambda kv: kv[1]["total_ms"])[0] if kern else None
    roof = None
    if dom:
        per_step_launches = kern[dom]["launches"] / args.steps
        if dom in algo_bytes:
            bytes_per_launch = algo_bytes[dom] / per_step_launches
        elif dom == "tile_rerun":
            # a rerun reads the subbins (4 B) and lower masks (2 B) of its tiles' points
            bytes_per_launch = (runs - npts / 4096) * 4096 * 6 / max(1, rounds)
        else:
            bytes_per_launch = 0
        achieved = bytes_per_launch / (kern[dom]["ms_per_launch"] * 1e-3) / 1e9
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None, "peak_kind": f"{peak_kind} (copy)"}
    gpu_launches = int(sum(v["launches"] for v in kern.values()))

    # other bounds of the same config
    extra = {}
    for eb in [float(v) for v in args.extra_ebs.split(",") if v]:
        t2, c2, d2, s2, _ = timed(eb, max(1, args.steps // 2), 1)
        r2, n2 = lopc.last_stats()
        f2 = lopc.last_fixpoint_stats()
        extra[f"{eb:g}"] = {"fixpoint_sweeps": f2[0], "fixpoint_sweeps_max": f2[1], "ms_per_step": float(t2.mean()), "compress_gbs": nbytes / (c2.mean() * 1e-3) / 1e9,
                            "decompress_gbs": nbytes / (d2.mean() * 1e-3) / 1e9, "cr": nbytes / s2,
                            "repair_rounds": r2, "tile_runs": n2}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    hx = torch.from_numpy(x_np).pin_memory()
    hs = torch.empty(out.numel(), dtype=torch.uint8).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    e2e_t = []
    h2d = d2h = 0
    for i in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x.copy_(hx, non_blocking=True)
        st = lopc.compress(x, args.eb, lopc.NOA, out=out, workspace=ws)
        n = st.numel()
        hs[:n].copy_(st, non_blocking=True)
        out[:n].copy_(hs[:n], non_blocking=True)
        lopc.decompress(out[:n], out=xhat, desc=d, workspace=dws)
        hy.copy_(xhat, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
        h2d, d2h = nbytes + n, n + nbytes
    e2e_gbs = nbytes / float(np.mean(e2e_t)) / 1e9

    # aggregate over ranks (replicas): total bytes / max time
    value = world * nbytes / (ms_step * 1e-3) / 1e9
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        nb, dt, _ = cpu_oracle_sample(x_np, args.eb, args.cpu_sample)
        cpu = {"value": nb / dt / 1e9, "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"central {args.cpu_sample}^3 block of the field, compress+decompress, single thread"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"3d_f32_{args.size}^3 (256 Gaussian bumps + 3-octave value noise), NOA eb "
                                   f"{args.eb:g}; step = compress + decompress", "field_bytes": nbytes,
                       "parallelism": "replicas" if world > 1 else "single", "l2": "flushed between steps (256 MB write); input 512 MB > L2"},
            "compress": {"gbs": comp_gbs, "ms": float(tc.mean()), "hbm_frac_algorithmic": algo_comp / (tc.mean() * 1e-3) / 1e9 / hbm,
                         "input_frac": comp_gbs / hbm, "cr": cr, "repair_rounds": rounds, "tile_runs": runs,
                         "fixpoint_sweeps": sweeps, "fixpoint_sweeps_max": sweeps_max, "phase_cycles": phases},
            "decompress": {"gbs": dec_gbs, "ms": float(td.mean()), "hbm_frac_algorithmic": algo_dec / (td.mean() * 1e-3) / 1e9 / hbm},
            "other_bounds": extra,
            "kernels": kern,
            "roofline": roof,
            "gpu_launches": gpu_launches,
            "e2e": {"value": e2e_gbs, "unit": "GB/s", "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "cpu_baseline": cpu,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
