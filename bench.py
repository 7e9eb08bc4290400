"""Throughput benchmark: noisy shots/s of the 42-qubit windowed Clifford+T
workload on GB300, FP32 coefficients (headline) and FP64 beside it.

A step = one launch sequence of the whole hot path (compiled program, all
event kinds, noise, measurement, early discard, tallies) over one batch of
shots. Inputs (the compiled program) are resident in HBM before timing;
L2 (129 MB) is flushed between steps with a 512 MB memset outside the timed
events. Multi-GPU: every rank runs its own shot range (weak scaling, no data
path collective; each step's job is split into contiguous shot ranges, and the
tally is summed over ranks); the time is the max over ranks.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--shots S] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = ("w42: 42 qubits (38 data + 4 ancilla), seeded random stabilizer state, 18 blocks of "
            "T on a random 4-qubit window + 60-gate Clifford + 4 ancilla parity checks + inverse + T^dag "
            "(72 T positions), coefficient cap 2^8, uniform depolarizing p=1e-3, circuit seed 1, Philox seed 0")
WORKLOADS = {
    "w42": WORKLOAD,
    "w97": ("w97: 97 qubits (89 data + 8 ancilla), 24 blocks of T on a random 6-qubit window + 160-gate Clifford "
            "+ 8 ancilla parity checks + inverse + T^dag (144 T positions), coefficient cap 2^12, uniform "
            "depolarizing p=5e-4, circuit seed 4, Philox seed 0"),
    "batch64": ("batch64: one launch over 64 windowed circuits, qubits uniform 17..49, window 2..6 (caps 2^4..2^12), "
                "6..24 blocks, p log-uniform in [1e-4, 3e-3], shots per circuit geometric with mean 1e6 "
                "(77.1 M shots per step), generator seed 2"),
}
# Algorithmic work per counted unit (lane ops, FP + integer): a T/Rz output entry (two complex
# multiply-adds and the key XOR/parity), a diagonal T/Rz entry, a measurement entry visit
# (norm and filter or pairing), a noise entry touch (key XOR and phase)
OPS_T_OUT, OPS_T_DIAG, OPS_MEAS, OPS_NOISE = 18, 9, 8, 3
# FP64 flops of the same units in the FP64 path (coefficients FP64): a T/Rz output entry
# a v + b xi v' (two complex products and a complex sum), a diagonal entry (a + b xi) v (one
# complex product), a measurement entry visit (|v|^2 and its accumulation); noise entries
# permute and negate (no flops)
FLOPS_T_OUT, FLOPS_T_DIAG, FLOPS_MEAS = 14, 6, 4
# What the equivalent fraction is: the whole method's work per shot, the shared noiseless prefix
# included, over the measured time, against the same peak. The prefix runs once per compile and
# no shot executes it, so this is the rate a design that re-ran the prefix per shot would need
# to match; it is not a utilisation and can exceed 1.
EQUIV_NOTE = ("whole-method work per shot (shared noiseless prefix included, which runs once per compile and "
              "is executed by no shot) / time / peak: the rate a per-shot re-run of the prefix would need, "
              "not a utilisation; can exceed 1")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=6)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--shots", type=int, default=1 << 24,
                    help="shots per step per GPU (default: 6 steps of 2^24 = 1.0e8 shots, the w42 job size)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--first-cap", type=int, default=0)
    ap.add_argument("--flush-mb", type=int, default=512, help="L2 flush buffer between steps (0 = none)")
    ap.add_argument("--workload", default="w42", choices=["w42", "w97", "batch64"])
    ap.add_argument("--graph", action="store_true", help="replay chunks from a captured CUDA graph")
    ap.add_argument("--warp-per-shot", action="store_true",
                    help="a warp per shot even where the library would run a lane per shot")
    ap.add_argument("--chunk", type=int, default=0, help="shots per chunk (0 = library default)")
    ap.add_argument("--autotune", action="store_true", help="time launch-shape candidates first")
    ap.add_argument("--grad-patterns", type=int, default=100000,
                    help="error patterns per step of the gradient leg (0 = skip it)")
    ap.add_argument("--no-fidelity", action="store_true", help="skip the exact-fidelity leg")
    ap.add_argument("--no-legs", action="store_true",
                    help="skip the batch64, w97 and FP32-vs-FP64 precision legs of the default w42 line")
    ap.add_argument("--w97-chunks", type=int, default=2,
                    help="graph-replayed 1e8-shot chunks per step of the w97 leg")
    ap.add_argument("--sweep", action="store_true",
                    help="w42 sweeps instead of the bench line: noise p in {5e-4, 1e-3, 2e-3} and shots resident "
                         "per SM (one JSON line per point)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks
class Clocks:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.p = None
        self.path = os.path.join(ROOT, f".clocks_{os.getpid()}.csv")  # removed after reading
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if not self.p:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            lines = fh.readlines()
        try:
            os.remove(self.path)
        except OSError:
            pass
        for line in lines:
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def lane_mode_of(pass_ms):
    """A run whose bucketing pre-pass took time ran lane per shot."""
    return pass_ms[0] > 0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def profile_traffic(kernel_src_hash, name, shots_per_launch):
    """DRAM bytes per launch from the committed ncu summary `name`, if it was
    taken on the current kernel source: a per-launch figure as it stands, or a
    per-shot figure (traffic that grows with the shots) times the bench's
    shots per launch."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        txt = open(path).read()
    except OSError:
        return None
    m = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_src_hash:
        return None
    t = re.search(r"dram_bytes_per_shot:\s*([0-9.e+]+)", txt)
    if t:
        return float(t.group(1)) * shots_per_launch
    t = re.search(r"dram_bytes_per_launch_full:\s*([0-9.e+]+)", txt)
    return float(t.group(1)) if t else None


def kernel_hash():
    """sha256 prefix of the shot kernels' sources, code only: every line with its
    `//` comment and surrounding whitespace removed, blank lines dropped (the
    files hold no block comments and no string with `//`)."""
    h = hashlib.sha256()
    for f in ("kernels.cu", "kernels.cuh", "program.h", "device_common.cuh", "lanes.cu", "shot_common.cuh"):
        for line in open(os.path.join(ROOT, "paper_2512_23037_gb300", "csrc", f), encoding="utf-8"):
            code = line.split("//", 1)[0].strip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


# ----------------------------------------------------------------- oracle timing
def oracle_rate(circ, noise, seed, budget_s, threads):
    import oracle
    t0 = time.perf_counter()
    oracle.run(circ, circ.n, noise, circ.cap, seed, 0, 400, threads=threads, records=False)
    est = 400 / max(time.perf_counter() - t0, 1e-6)
    n = int(max(400, min(est * budget_s, 5_000_000)))
    t0 = time.perf_counter()
    r = oracle.run(circ, circ.n, noise, circ.cap, seed, 1_000_000_000, n, threads=threads, records=False)
    dt = time.perf_counter() - t0
    return n / dt, n, dt, r


def _ops(k, post):
    """Lane ops from the oracle's exact counters: the whole shot, or (post) only
    the part after the noiseless-run prefix that the kernel actually executes."""
    if post:
        return (OPS_T_OUT * k["post_t_out"] + OPS_T_DIAG * k["post_t_diag"] + OPS_MEAS * k["post_meas"]
                + OPS_NOISE * k["post_noise"])
    return (OPS_T_OUT * k["t_out_entries"] + OPS_T_DIAG * k["t_diag_entries"] + OPS_MEAS * k["meas_entries"]
            + OPS_NOISE * k["noise_entries"])


def _flops(k, post):
    """FP64 flops of the FP64 path from the oracle's exact counters (see _ops)."""
    if post:
        return FLOPS_T_OUT * k["post_t_out"] + FLOPS_T_DIAG * k["post_t_diag"] + FLOPS_MEAS * k["post_meas"]
    return FLOPS_T_OUT * k["t_out_entries"] + FLOPS_T_DIAG * k["t_diag_entries"] + FLOPS_MEAS * k["meas_entries"]


def ops_per_shot_items(items, sample=2000):
    """Shot-weighted algorithmic work per shot over a workload's circuits, from
    the oracle's counters on a sample of the same workload (seed 0): lane ops
    (executed: after the shared noiseless prefix; whole method) and FP64 flops
    of the FP64 path (executed; whole method)."""
    import oracle
    per = sample if len(items) == 1 else max(50, sample // 10)
    tot = [0.0, 0.0, 0.0, 0.0]
    tot_w = 0
    for c, nz, shots in items:
        r = oracle.run(c, c.n, nz, c.cap, 0, 0, per, threads=os.cpu_count() or 1, records=False)
        k = r["counts"]
        for j, v in enumerate((_ops(k, True), _ops(k, False), _flops(k, True), _flops(k, False))):
            tot[j] += v / k["shots"] * shots
        tot_w += shots
    return [v / tot_w for v in tot]


def grad_bench(S, C, torch, stream, n_pat, steps, warmup):
    """Patterns/s of the fidelity gradient (forward projection + two adjoint
    sweeps per pattern) on the 42-qubit workload with every T/T^dag pair as
    Rz(+-theta_i), 72 angles theta_i = pi/4 + N(0, 0.01), p = 1e-3."""
    circ, noise = C.workload("w42rz")
    theta = C.rz_thetas(1, 72)
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    out = {"workload": "w42rz: the w42 circuit with T/T^dag -> Rz(+theta_i)/Rz(-theta_i), 72 angles "
                       "theta_i = pi/4 + N(0, 0.01) (seed 1), error patterns of p=1e-3, Philox seed 0",
           "patterns_per_step": n_pat, "params": 72}
    for prec in ("fp64", "fp32"):
        for w in range(warmup):
            S.soft_fidelity_grad(h, theta, n_pat, (1 << 40) + w * n_pat, 0, prec, stream=stream)
        torch.cuda.synchronize()
        ms = 0.0
        counts = [0, 0, 0, 0]
        sums = None
        for k in range(steps):
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            fid, pacc, grad, st, sm = S.soft_fidelity_grad(h, theta, n_pat, k * n_pat, 0, prec, stream=stream,
                                                           sums=True)
            ev1.record(stream)
            torch.cuda.synchronize()
            ms += ev0.elapsed_time(ev1)
            binc = torch.bincount(st.long(), minlength=4).cpu().tolist()
            counts = [a + b for a, b in zip(counts, binc[:4])]
            sm = sm.cpu().tolist()
            sums = sm if sums is None else [a + b for a, b in zip(sums, sm)]
        out[prec] = {"value": n_pat * steps / (ms / 1000), "unit": "patterns/s", "ms_per_step": ms / steps,
                     "status_counts": {"ok": counts[0], "zero_acceptance": counts[1], "unsupported": counts[2],
                                       "error": counts[3]},
                     "ratio_estimator": (sums[1] / sums[0]) if sums and sums[0] > 0 else None}
    h.free()
    return out


def sweep(args):
    """Throughput of the 42-qubit workload against the noise rate (discard
    rate grows with p), FP32 and FP64, and against the shots resident per SM:
    lane-per-shot blocks per SM (128 shots each), and a few warp-per-shot shapes
    (blocks per SM x groups per block); CUDA events over K steps of --shots."""
    import torch
    import paper_2512_23037_gb300 as S
    from paper_2512_23037_gb300 import circuits as C
    S.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(max(args.flush_mb, 1) * 1024 * 1024, dtype=torch.uint8, device="cuda")

    def rate(h, precision, **kw):
        for w in range(args.warmup):
            S.soft_tally(S.soft_run_shots(h, args.shots, (1 << 36) + w * args.shots, 0, precision=precision,
                                          stream=stream, **kw))
        ms, tal = 0.0, None
        for k in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = S.soft_run_shots(h, args.shots, k * args.shots, 0, precision=precision, stream=stream, **kw)
            e1.record(stream)
            tal = S.soft_tally(r)
            ms += e0.elapsed_time(e1)
        return args.shots * args.steps / (ms / 1000), tal

    for p in (5e-4, 1e-3, 2e-3):
        circ, noise = C.windowed(1, p=p)
        h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
        v32, tal = rate(h, "fp32")
        v64, _ = rate(h, "fp64")
        print(json.dumps({"sweep": "noise", "workload": "w42", "p": p, "fp32_shots_per_s": v32,
                          "fp64_shots_per_s": v64, "discard_rate": tal["discarded"] / tal["shots"],
                          "ler_kept": tal["logical_errors"] / max(tal["kept"], 1)}))
    circ, noise = C.workload("w42")
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    for bps in (1, 2, 3, 4, 5, 6):
        v32, _ = rate(h, "fp32", blocks_per_sm=bps)
        print(json.dumps({"sweep": "shots_per_sm", "workload": "w42", "scheduling": "lane per shot",
                          "blocks_per_sm": bps, "shots_resident_per_sm": bps * 128, "fp32_shots_per_s": v32}))
    for bps, gpb in ((1, 1), (2, 4), (6, 4)):
        v32, _ = rate(h, "fp32", blocks_per_sm=bps, groups_per_block=gpb, lanes=False)
        print(json.dumps({"sweep": "shots_per_sm", "workload": "w42", "scheduling": "warp per shot",
                          "blocks_per_sm": bps, "groups_per_block": gpb, "shots_resident_per_sm": bps * gpb,
                          "fp32_shots_per_s": v32}))
    return 0


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2512_23037_gb300 import circuits as C
    circ, noise = C.workload("w42")
    threads = os.cpu_count() or 1
    budget = 4.0
    for _ in range(args.warmup):
        oracle_rate(circ, noise, 0, 0.5, threads)
    rates, tot_n, tot_t = [], 0, 0.0
    for _ in range(args.steps):
        rate, n, dt, _ = oracle_rate(circ, noise, 0, budget, threads)
        rates.append(rate)
        tot_n += n
        tot_t += dt
    value = tot_n / tot_t
    line = {"metric": "shots/s", "value": value, "unit": "shots/s", "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD},
            "cpu_baseline": {"value": value, "unit": "shots/s", "cores": threads, "kind": "oracle",
                             "sample": f"{tot_n} shots of the same workload over {args.steps} steps "
                                       f"(~{budget:.0f} s each, shots 1e9..)"},
            "e2e": {"value": value, "unit": "shots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- extra legs of the w42 line
def _events_ms(stream, torch, fn):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1), out


def _tally_list(t):
    return [t["shots"], t["discarded"], t["overflow"], t["kept"], t["logical_errors"]]


def leg_batch64(S, C, torch, peak_ops, flush):
    """The batching configuration: one launch sequence over 64 windowed circuits
    (77.1 M shots per step), autotuned launch shape, chunks replayed from a CUDA
    graph; FP32 and FP64, one warm-up and two timed steps each."""
    items = C.batch_of_windowed(2, 64)
    hs = [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz, _ in items]
    shots = [s for _, _, s in items]
    n = sum(shots)
    stream = torch.cuda.Stream()
    from paper_2512_23037_gb300.autotune import autotune
    res = autotune(hs, precision="fp32", stream=stream, sample_shots=1 << 22)
    tune = res["best"]
    ops_shot, ops_full, _, _ = ops_per_shot_items(items)
    out = {"workload": WORKLOADS["batch64"], "shots_per_step": n, "graph_replay": True, "launch_shape": tune,
           "autotune_table_ms": [[round(ms, 3), kw] for ms, kw in res["table"]]}
    for prec in ("fp32", "fp64"):
        def run(k, first0):
            return S.soft_run_batch(hs, shots, [first0 + k * n] * len(hs), 0, precision=prec, stream=stream,
                                    graph=True, **tune)
        S.soft_tally(run(0, 1 << 36))
        ms_tot, tal = 0.0, None
        for k in range(2):
            flush.zero_()
            torch.cuda.synchronize()
            ms, r = _events_ms(stream, torch, lambda: run(k, 0))
            tal = S.soft_tally(r)
            ms_tot += ms
            r.free()
        achieved = ops_shot * n * 2 / (ms_tot / 1000)
        out[prec] = {"value": 2 * n / (ms_tot / 1000), "unit": "shots/s", "ms_per_step": ms_tot / 2,
                     "dtype": "f32" if prec == "fp32" else "f64", "tally_last_step": tal,
                     "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                                  "unit": "Tops/s", "frac": achieved / peak_ops,
                                  "equivalent_frac_whole_method": ops_full * n * 2 / (ms_tot / 1000) / peak_ops,
                                  "traffic": None, "kernel": "lane_kernel + shot_kernel (whole launch sequence)",
                                  "ops_per_shot": ops_shot, "ops_per_shot_whole_method": ops_full}}
    for h in hs:
        h.free()
    return out


def leg_w97(S, C, torch, peak_ops, n_chunks):
    """The large throughput configuration: 97 qubits, 1e8-shot chunks replayed
    from one captured CUDA graph, n_chunks chunks per step; FP32 and FP64, a
    warm-up run of two 1e6-shot chunks (same kernels and graph path) and one
    timed step each."""
    circ, noise = C.workload("w97")
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    chunk = 100_000_000
    n = n_chunks * chunk
    stream = torch.cuda.Stream()
    ops_shot, ops_full, _, _ = ops_per_shot_items([(circ, noise, 1)])
    out = {"workload": WORKLOADS["w97"], "shots_per_step": n, "chunk_shots": chunk, "graph_replay": True,
           "steps": 1}
    for prec in ("fp32", "fp64"):
        S.soft_tally(S.soft_run_shots(h, 2_000_000, 1 << 40, 0, precision=prec, stream=stream, graph=True,
                                      chunk_shots=1_000_000))
        torch.cuda.synchronize()
        ms, r = _events_ms(stream, torch, lambda: S.soft_run_shots(h, n, 0, 0, precision=prec, stream=stream,
                                                                    graph=True, chunk_shots=chunk))
        tal = S.soft_tally(r)
        r.free()
        achieved = ops_shot * n / (ms / 1000)
        out[prec] = {"value": n / (ms / 1000), "unit": "shots/s", "ms_per_step": ms,
                     "dtype": "f32" if prec == "fp32" else "f64", "tally": tal,
                     "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                                  "unit": "Tops/s", "frac": achieved / peak_ops,
                                  "equivalent_frac_whole_method": ops_full * n / (ms / 1000) / peak_ops,
                                  # the 64-entry lanes' DRAM bytes per 1e8-shot launch (its ncu summary)
                                  "traffic": profile_traffic(kernel_hash(), "lane_kernel_w97.md", chunk) if prec == "fp32" else None,
                                  "kernel": ("lane_kernel (64-entry lanes: the noiseless maps reach 64 entries) + "
                                             "shot_kernel (shots that outgrow them)") if prec == "fp32" else
                                            "shot_kernel (warp per shot: 64-entry lanes are FP32 only)",
                                  "ops_per_shot": ops_shot, "ops_per_shot_whole_method": ops_full}}
    h.free()
    return out


def leg_precision(S, C, torch, n, grad_patterns):
    """FP32 coefficients against FP64 on the same shots of w42 (seed 0, shots
    [2^37, 2^37 + n)): shots whose status or records differ, the kept, discard and
    logical-error rates, the exact-fidelity sums; and on the same error patterns
    of w42rz, F and the gradient. The FP64 path is the reference here: both are
    checked against the oracle shot for shot in the tests."""
    circ, noise = C.workload("w42")
    h = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
    rw = h.info["record_words"]
    first = 1 << 37
    runs = {}
    for prec in ("fp32", "fp64"):
        st = torch.empty(n, dtype=torch.uint8, device="cuda")
        rec = torch.empty((n, rw), dtype=torch.int64, device="cuda")
        r = S.soft_run_shots(h, n, first, 0, precision=prec, record_mode=S.REC_ALL, d_records=rec.data_ptr(),
                             d_status=st.data_ptr())
        t = S.soft_tally(r)
        r.free()
        rf = S.soft_run_shots(h, n, first, 0, precision=prec, fidelity=True)
        tf = S.soft_tally(rf)
        rf.free()
        runs[prec] = (st, rec, t, tf)
    s32, r32, t32, f32 = runs["fp32"]
    s64, r64, t64, f64 = runs["fp64"]
    diff = (s32 != s64) | (r32 != r64).any(dim=1)
    out = {"workload": WORKLOADS["w42"], "shots": n,
           "shots_differing": int(diff.sum().item()),
           "status_differing": int((s32 != s64).sum().item()),
           "tally_fp32": _tally_list(t32), "tally_fp64": _tally_list(t64),
           "kept_rate_diff": (t32["kept"] - t64["kept"]) / n,
           "discard_rate_diff": (t32["discarded"] - t64["discarded"]) / n,
           "ler_fp32": t32["logical_errors"] / max(t32["kept"], 1),
           "ler_fp64": t64["logical_errors"] / max(t64["kept"], 1),
           "fidelity_sum_fp32": f32["sum_fidelity"], "fidelity_sum_fp64": f64["sum_fidelity"],
           "fidelity_sum_rel_diff": abs(f32["sum_fidelity"] - f64["sum_fidelity"]) / max(abs(f64["sum_fidelity"]),
                                                                                        1e-300),
           "kept_fidelity_mode": [f32["kept"], f64["kept"]]}
    h.free()
    if grad_patterns > 0:
        circ, noise = C.workload("w42rz")
        theta = C.rz_thetas(1, 72)
        hg = S.soft_compile_circuit(circ.array(), circ.n, noise, circ.cap)
        g = {p: S.soft_fidelity_grad(hg, theta, grad_patterns, 0, 0, p) for p in ("fp32", "fp64")}
        ok = (g["fp32"][3] == 0) & (g["fp64"][3] == 0)
        out["gradient"] = {"patterns": grad_patterns, "ok_both": int(ok.sum().item()),
                           "status_differing": int((g["fp32"][3] != g["fp64"][3]).sum().item()),
                           "max_abs_F_diff": float((g["fp32"][0] - g["fp64"][0])[ok].abs().max().item()),
                           "max_abs_grad_diff": float((g["fp32"][2] - g["fp64"][2])[ok].abs().max().item()),
                           "max_abs_grad_fp64": float(g["fp64"][2][ok].abs().max().item())}
        hg.free()
    return out


# ----------------------------------------------------------------- GPU arm
def main():
    args = parse()
    if args.impl == "reference":
        return reference_arm(args)
    if args.sweep:
        return sweep(args)
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2512_23037_gb300 as S
    from paper_2512_23037_gb300 import circuits as C
    S.load()
    if args.workload == "batch64":
        items = C.batch_of_windowed(2, 64)
    else:
        circ0, noise0 = C.workload(args.workload)
        items = [(circ0, noise0, args.shots)]
    stream = torch.cuda.current_stream() if not args.graph else torch.cuda.Stream()
    n = sum(s for _, _, s in items)  # shots per step per GPU
    from paper_2512_23037_gb300.sharding import all_reduce_tally, shot_range

    def firsts(k, off=0):
        # step k's job holds world x (shots per GPU) shots of each circuit; this rank runs its
        # contiguous part of it, so that the job's result does not depend on the rank count
        return [shot_range(rank, world, s * world, off + k * s * world)[0] for _, _, s in items]
    dev_props = torch.cuda.get_device_properties(local)
    flush = torch.empty(max(args.flush_mb, 1) * 1024 * 1024, dtype=torch.uint8, device="cuda")
    tune = {"group_size": args.group, "first_cap": args.first_cap, "chunk_shots": args.chunk}

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def compile_all():
        return [S.soft_compile_circuit(c.array(), c.n, nz, c.cap) for c, nz, _ in items]

    def launch(handles, first, precision, fidelity=False, time_passes=False):
        if len(handles) == 1:
            return S.soft_run_shots(handles[0], items[0][2], first[0], 0, precision=precision, stream=stream,
                                    graph=args.graph, fidelity=fidelity, lanes=not args.warp_per_shot,
                                    time_passes=time_passes, **tune)
        return S.soft_run_batch(handles, [s for _, _, s in items], first, 0, precision=precision,
                                stream=stream, graph=args.graph, fidelity=fidelity, time_passes=time_passes, **tune)

    def job_tally(t):
        return all_reduce_tally(t, torch.distributed, device="cuda") if world > 1 else t

    def time_path(precision, steps, warmup, fidelity=False):
        hs = compile_all()
        for w in range(warmup):
            r = launch(hs, firsts(w, 1 << 36), precision, fidelity)
            S.soft_tally(r)
            r.free()
        barrier()
        total_ms, launches, kernel_ms, tallies = 0.0, 0, [], []
        for k in range(steps):
            if args.flush_mb:
                flush.zero_()
            torch.cuda.synchronize()
            ev0 = torch.cuda.Event(enable_timing=True)
            ev1 = torch.cuda.Event(enable_timing=True)
            ev0.record(stream)
            r = launch(hs, firsts(k), precision, fidelity, time_passes=not args.graph)
            ev1.record(stream)
            tallies.append(S.soft_tally(r))
            ms, nl = S.soft_run_timing(r)
            # per pass (bucketing pre-pass, first pass, rerun pass) when events were recorded between them
            if args.graph:
                kernel_ms.append([0.0, ms, 0.0, 0])
            else:
                pms, _, n_rr = S.soft_run_pass_timing(r)
                kernel_ms.append(pms + [n_rr])
            launches += nl
            total_ms += ev0.elapsed_time(ev1)
            r.free()
        barrier()
        t = torch.tensor([total_ms], device="cuda", dtype=torch.float64)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item()), launches, kernel_ms, [job_tally(x) for x in tallies], hs

    tuned = None
    if args.autotune:
        from paper_2512_23037_gb300.autotune import autotune
        # a sample of 2^22 shots: lane-per-shot runs pay a pre-pass per launch, so small samples
        # would favour the warp per shot over what the full step measures
        res = autotune(compile_all(), precision="fp32", stream=stream, sample_shots=1 << 22)
        tune.update(res["best"])
        tuned = {"best": res["best"], "table_ms": [[round(ms, 3), kw] for ms, kw in res["table"]]}

    clocks = Clocks(local) if rank == 0 else None
    ms32, launches32, kms32, tal32, c32 = time_path("fp32", args.steps, args.warmup)
    clock_info = clocks.stop() if clocks else None
    ms64 = None
    if not args.no_fp64:
        ms64, launches64, kms64, tal64, _ = time_path("fp64", args.steps, args.warmup)

    # exact-fidelity mode: the same shots with the final chain projected (variance-reduced LER)
    fid_leg = None
    if not args.no_fidelity:
        msf, _, _, talf, _ = time_path("fp32", max(1, args.steps // 2), 1, fidelity=True)
        sf = sum(t["sum_fidelity"] for t in talf)
        sw = sum(t["sum_weight"] for t in talf)
        kept = sum(t["kept"] for t in tal32[:len(talf)])
        le = sum(t["logical_errors"] for t in tal32[:len(talf)])
        fid_leg = {"value": n * world * len(talf) / (msf / 1000), "unit": "shots/s", "dtype": "f32",
                   "ler_fidelity_estimate": (1 - sf / sw) if sw else None,
                   "ler_sampled_same_shots": (le / kept) if kept else None, "kept": int(sw)}

    # Rz adjoint gradient: fixed error patterns of the 42-qubit workload with 72 Rz angles
    grad_leg = None
    if args.grad_patterns > 0 and world == 1:
        grad_leg = grad_bench(S, C, torch, stream, args.grad_patterns, max(2, args.steps // 2), 1)

    # end to end through the C ABI, every step: host op lists -> compile + upload -> run -> tally
    # to host. Pipelined as a user would run it: the host compiles step k + 1 while step k runs
    # on the device (runs are asynchronous on their stream; compiling waits for no other work).
    # The same steps one after another are reported beside it.
    ops_host = [c.array() for c, _, _ in items]

    def compile_step():
        return [S.soft_compile_circuit(a, c.n, nz, c.cap) for a, (c, nz, _) in zip(ops_host, items)]

    def e2e_loop(pipelined):
        barrier()
        t0 = time.perf_counter()
        hs = compile_step()
        h2d = sum(h.info["program_bytes"] for h in hs)
        for k in range(args.steps):
            r = launch(hs, firsts(k, 1 << 38), "fp32")
            nxt = compile_step() if pipelined and k + 1 < args.steps else None
            S.soft_tally(r)
            r.free()
            for h in hs:
                h.free()
            if k + 1 < args.steps:
                hs = nxt if nxt is not None else compile_step()
        ms = 1000 * (time.perf_counter() - t0)
        barrier()
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        if world > 1:
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item()), h2d

    e2e_serial_ms, _ = e2e_loop(False)
    e2e_ms, h2d = e2e_loop(True)

    if rank != 0:
        return 0
    shots_all = n * world * args.steps
    value = shots_all / (ms32 / 1000)
    ops_shot, ops_full, flops64_shot, flops64_full = ops_per_shot_items(items)
    peaks = measured_peaks()
    sm_clock = peaks.get("sm_max_mhz", 2070.0)
    sms = dev_props.multi_processor_count
    peak_ops = sms * 128 * sm_clock * 1e6  # FP32/INT32 lanes x clock
    # measured issue-rate peaks of the pipes (the FP64 path's roof), clocks sampled while they run
    pclk = Clocks(local)
    pipe = {name: S.soft_peak_pipe_rate(kind, stream) for name, kind in
            (("fp64_fma", S.PEAK_FP64_FMA), ("fp32_fma", S.PEAK_FP32_FMA), ("int32_logic", S.PEAK_INT32_LOGIC))}
    pipe_clocks = pclk.stop()
    peak_fp64 = pipe["fp64_fma"][0]
    legs = {}
    if args.workload == "w42" and world == 1 and not args.no_legs:
        legs["batch64"] = leg_batch64(S, C, torch, peak_ops, flush)
        legs["w97"] = leg_w97(S, C, torch, peak_ops, args.w97_chunks)
        legs["precision_error"] = leg_precision(S, C, torch, n, min(args.grad_patterns, 100000))
    # dominant kernel: the first-pass shot kernel (lane per shot where it applies), timed with the
    # passes that finish its work (bucketing pre-pass, rerun of outgrown maps) by CUDA events between
    # them on the launching stream; the work is every shot's executed lane ops
    pass_ms = [sum(k[j] for k in kms32) / len(kms32) for j in range(3)]
    avg_launch_ms = sum(pass_ms)
    achieved = ops_shot * n / (avg_launch_ms / 1000)
    fp64_roof = None
    if ms64 is not None:
        # the FP64 path against the measured FP64 pipe: its algorithmic FP64 flops over the same passes
        pass64 = [sum(k[j] for k in kms64) / len(kms64) for j in range(3)]
        a64 = flops64_shot * n / (sum(pass64) / 1000)
        fp64_roof = {"bound": "fp64", "achieved": a64 / 1e12, "peak": peak_fp64 / 1e12, "unit": "TFLOP/s",
                     "frac": a64 / peak_fp64, "equivalent_frac_whole_method": flops64_full * n / (sum(pass64) / 1000) / peak_fp64,
                     "traffic": None, "kernel": "lane_kernel<double>" if lane_mode_of(pass64) else "shot_kernel<double>",
                     "pass_ms_per_step": {"prepass": pass64[0], "first_pass": pass64[1], "rerun": pass64[2]},
                     "flops_per_shot": flops64_shot, "flops_per_shot_whole_method": flops64_full,
                     "work": "FP64 flops of T/Rz output entries (14), diagonal entries (6) and measurement entry "
                             "visits (4) a shot executes after the shared noiseless prefix (oracle counters)",
                     "peak_basis": "measured: soft_peak_pipe_rate(FP64 FMA) in this run, 2 flops per FMA",
                     "alu_frac": ops_shot * n / (sum(pass64) / 1000) / peak_ops, "equivalent_note": EQUIV_NOTE}
    lane_mode = lane_mode_of(pass_ms)
    chunks = -(-n // args.chunk) if args.chunk else -(-n // (1 << 24))
    # the ncu summary of this workload's first-pass kernel (w42, w97), if one matches the source
    traffic = profile_traffic(kernel_hash(), ("lane_kernel_%s.md" if lane_mode else "shot_kernel_%s.md") % args.workload,
                              -(-n // chunks))
    line = {
        "metric": "shots/s", "value": value, "unit": "shots/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms32 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "shots_per_step_per_gpu": n, "coefficients": "complex64",
                   "probabilities_and_tallies": "fp64", "l2": "flushed between steps (512 MB memset)",
                   "parallelism": f"shot ranges x{world}", "graph_replay": bool(args.graph),
                   "launch_shape": {k: v for k, v in tune.items() if v} or "library default"},
        "fp64_plain": None if ms64 is None else {
            "value": shots_all / (ms64 / 1000), "unit": "shots/s", "ms_per_step": ms64 / args.steps,
            "dtype": "f64", "roofline": fp64_roof},
        "tally_last_step": tal32[-1],
        "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                     "frac": achieved / peak_ops, "equivalent_frac_whole_method": ops_full * n / (avg_launch_ms / 1000) / peak_ops,
                     "traffic": traffic,
                     "kernel": "lane_kernel" if lane_mode else "shot_kernel",
                     "pass_ms_per_step": {"prepass": pass_ms[0], "first_pass": pass_ms[1], "rerun": pass_ms[2]},
                     "rerun_shots_per_step": sum(k[3] for k in kms32) / len(kms32),
                     "ops_per_shot": ops_shot, "ops_per_shot_whole_method": ops_full,
                     "work": "lane ops a shot executes after the noiseless-run prefix it shares with every "
                             "shot (oracle counters); the whole method per shot is ops_per_shot_whole_method",
                     "peak_basis": f"{sms} SMs x 128 lanes x {sm_clock:.0f} MHz (sm_max_mhz of measured)",
                     "equivalent_note": EQUIV_NOTE},
        "gpu_launches": launches32,
        "error_shots_last_step": tal32[-1]["shots"] - tal32[-1]["discarded"] - tal32[-1]["overflow"] - tal32[-1]["kept"],
        "e2e": {"value": shots_all / (e2e_ms / 1000), "unit": "shots/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 56, "pipelined": "the host compiles step k+1 while step k runs",
                "serial_value": shots_all / (e2e_serial_ms / 1000)},
        "clocks": clock_info,
        "pipe_peaks": {"fp64_fma_tflops": pipe["fp64_fma"][0] / 1e12, "fp32_fma_tflops": pipe["fp32_fma"][0] / 1e12,
                       "int32_logic_tops": pipe["int32_logic"][0] / 1e12, "clocks": pipe_clocks,
                       "how": "soft_peak_pipe_rate: independent FMA / logic chains on every SM, best of 5 launches"},
    }
    line.update(legs)
    if fid_leg:
        line["fidelity_mode"] = fid_leg
    if grad_leg:
        line["gradient"] = grad_leg
    if tuned:
        line["autotune"] = tuned
    if not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        rate, ncpu, dt, _ = oracle_rate(items[0][0], items[0][1], 0, 12.0, threads)
        line["cpu_baseline"] = {"value": rate, "unit": "shots/s", "cores": threads, "kind": "oracle",
                                "sample": f"{ncpu} shots of {'the same workload' if len(items) == 1 else 'circuit 0 of the batch'} ({dt:.1f} s, shots 1e9..)"}
    print(json.dumps(line))
    return 0


if __name__ == "__main__":
    sys.exit(main())
