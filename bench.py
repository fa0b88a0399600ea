"""Benchmark: Wang-Landau flip attempts per second of the replica-exchange
Wang-Landau path on the batched 2D Ising workload (L = 32 and L = 64, 16
windows x 4 walkers per window at 75 % overlap, 32 seeds per size, exchange
every 10^4 sweeps) -- one step = 10^4 sweeps of every walker plus one exchange
phase.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is device-timed (CUDA events on the library's
stream around rewl_run + rewl_exchange, L2 flushed between steps); `e2e` is
wall-clock through the public API (the CUDA-graph cycle rewl_run_cycles) with
host descriptors in and ln g pieces out every step; `roofline` relates the
sweep launches' algorithmic instruction rate, timed by events around rewl_run
inside the same timed steps, to the GPU's thread-instruction peak;
`cpu_baseline` is the CPU oracle on the host cores on a bounded sample of the
same workload.
Under torchrun each rank runs its own batch (distinct seeds, weak scaling).
"""
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

SWEEPS_PER_STEP = 10_000
# Algorithmic thread-instructions of one single-spin trial, counted from the
# minimal operation sequence: Philox4x32-10 share 30 (Ising, two trials per
# block) / 60 (Potts), site and neighbour indices 11, the -ln u threshold 35,
# neighbour reads and the energy change 20, the ln g lookup and comparison 8,
# the accepted move and the ln g / H updates 6.
INSTR_PER_TRIAL = {0: 110, 1: 146}
MAX_SM_MHZ = 2070.0
# exchange interval of the time-to-converge runs (Config 0 names 10^3 sweeps;
# Config 2 names none, the same interval is used)
CONVERGE_EXCHANGE = 1000


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.p = None

    def __enter__(self):
        import tempfile
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        idx = vis.split(",")[self.gpu] if vis and vis.split(",")[0].isdigit() else str(self.gpu)
        # samples go to a file: a pipe nobody reads would fill and stall the
        # sampler during long regions
        self.f = tempfile.TemporaryFile(mode="w+")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", idx, f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
        self.f.seek(0)
        self.out = self.f.read()
        self.f.close()

    def summary(self):
        rows = []
        for line in (self.out or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), hw=f[5], hwt=f[6], swt=f[7], pcap=f[8]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        reasons = set()
        for r in rows:
            for k, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"), ("swt", "sw_thermal_slowdown"),
                            ("pcap", "sw_power_cap")):
                if r[k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(rows)}


def _profile_fields(kernel_src_sha):
    """Figures of the committed ncu summary of the sweep kernel, if it was
    taken on the current kernel source: DRAM bytes per sweep phase, issue-lane
    slots per trial (inst_executed * 32 / trials) and issue slots active."""
    path = os.path.join(ROOT, "profiles", "sweep_kernel_ising_config1.md")
    try:
        txt = open(path).read()
    except OSError:
        return {}
    m = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    if not m or m.group(1) != kernel_src_sha:
        return {}
    out = {}
    for key, name in (("traffic_bytes_per_launch_full", "traffic"),
                      ("measured_issue_lane_slots_per_trial", "instr_per_trial_measured"),
                      ("issue_slots_active_pct", "issue_slots_active_pct")):
        t = re.search(key + r":\s*([0-9.eE+]+)", txt)
        if t:
            out[name] = float(t.group(1))
    return out


def _kernel_sha():
    h = hashlib.sha256()
    for f in ("rewl_kernels.cu", "rewl_device.cuh", "rewl_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1407_5140_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def cpu_oracle_rate(ds, budget_s, threads):
    """Oracle attempts/s on whole instances of the workload, sweeps in chunks until
    the time budget is spent."""
    import oracle as O
    done = 0
    t0 = time.perf_counter()
    used = []
    for d in ds:
        o = O.Oracle(d["model"], d["L"], d["q"], d["e_min"], d["e_max"], d["n_windows"], d["overlap"],
                     d["walkers_per_window"], d["flatness"], d["ln_f_final"], seed=d["seed"],
                     instance=d["instance_id"], threads=threads)
        o.init()
        t_init = time.perf_counter()
        chunk = 5
        sweeps = 0
        while time.perf_counter() - t0 < budget_s * (len(used) + 1) / len(ds):
            o.run(chunk)
            sweeps += chunk
        t_run = time.perf_counter() - t_init
        used.append((d, sweeps, t_run))
        done += sweeps * d["n_windows"] * d["walkers_per_window"] * d["L"] ** 2
    total_t = sum(u[2] for u in used)
    desc = "; ".join(f"{d['walkers_per_window'] * d['n_windows']} walkers L={d['L']} x {s} sweeps"
                     for d, s, _ in used)
    return done / total_t, desc, total_t


def rank_instances(ds, rank):
    """Weak scaling: every rank runs the whole batch with its own seeds."""
    out = [dict(d) for d in ds]
    for d in out:
        d["seed"] += 1000 * rank
    return out


def max_over_ranks(value, world, device="cpu"):
    """The slowest rank's step time (torch.distributed, any backend)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def run_ours(args, rank, world):
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W

    dev = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(dev)
    ds = rank_instances(W.config1(), rank)
    attempts_per_step = W.attempts_per_sweep(ds) * SWEEPS_PER_STEP
    # a stream of our own: torch's default stream has handle 0, which the
    # library would replace by a stream it creates
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for _ in range(args.warmup):
        ctx.run(SWEEPS_PER_STEP)
        ctx.exchange()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    launches0 = ctx.launch_count()
    times, ks = [], []
    with ClockSampler(dev) as clk:
        for _ in range(args.steps):
            flush.fill_(1)
            a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            ctx.run(SWEEPS_PER_STEP)       # sweep launches of every size class, joined on `stream`
            m.record(stream)
            ctx.exchange()
            b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b) / 1000.0)
            ks.append(a.elapsed_time(m) / 1000.0)
        torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    t_step = max_over_ranks(sum(times) / len(times), world, device="cuda")
    value = attempts_per_step * world / t_step
    clocks = clk.summary()
    k_time = sum(ks) / len(ks)
    ctx.close()

    # end to end through the public API: descriptors in (host), ln g out (host)
    t0 = time.perf_counter()
    e2e_ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    for _ in range(args.steps):
        e2e_ctx.run_cycles(1, SWEEPS_PER_STEP)
        for k in range(len(ds)):
            e2e_ctx.get_dos(k, per_window=True)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    h2d, d2h = e2e_ctx.transfer_bytes()          # every copy the library made, counted by it
    e2e_ctx.close()
    e2e = {"value": attempts_per_step * args.steps / e2e_t * world, "unit": "attempts/s",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "includes": "create (descriptors H2D, init kernel) + K steps + per-step ln g read-back; bytes are the "
                       "library's own count of its host<->device copies (rewl_transfer_bytes)"}

    instr = INSTR_PER_TRIAL[0]
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_instr = n_sm * 4 * 32 * MAX_SM_MHZ * 1e6
    achieved = instr * attempts_per_step / k_time
    prof = _profile_fields(_kernel_sha())
    roofline = {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_instr / 1e12, "unit": "Tinstr/s",
                "frac": achieved / peak_instr, "traffic": prof.get("traffic"),
                "peak_source": f"{n_sm} SMs x 4 schedulers x 32 lanes x {MAX_SM_MHZ:.0f} MHz (max SM clock)",
                "instr_per_trial": instr, "kernel_time_s": k_time,
                "instr_per_trial_measured": prof.get("instr_per_trial_measured"),
                "issue_slots_active_pct": prof.get("issue_slots_active_pct"),
                "measured_fields_from": "ncu capture in profiles/sweep_kernel_ising_config1.md (L=64 launch, "
                                        "20 sweeps; null when the kernel source changed since)"}
    if prof.get("instr_per_trial_measured"):
        roofline["frac_at_measured_instr"] = prof["instr_per_trial_measured"] * attempts_per_step / k_time / peak_instr
    return dict(value=value, t_step=t_step, e2e=e2e, roofline=roofline, clocks=clocks, launches=launches,
                attempts_per_step=attempts_per_step, ds=ds)


def time_to_converge(threads):
    """Config 0 (2D Ising L=8, 4 windows x 1 walker) and Config 2 (q=10 Potts
    L=32, 32 windows x 8 walkers) run to ln f = 2^-20 on the GPU through the
    public API (rewl_run_to_convergence: exchanges every 10^3 sweeps), with the
    clocks sampled meanwhile; the ln g error against the exact DOS (Config 0)
    and the invariant ln sum g = N ln q (Config 2).  The CPU oracle runs Config
    0 to convergence in full on the host cores; for Config 2 its time is the
    attempts the run needed (identical trajectories) over the oracle's measured
    attempts/s on the same instance, labelled extrapolated."""
    import math
    import numpy as np
    import torch
    import oracle as O
    from oracle import concat as cc
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W

    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    out = {"exchange_every": CONVERGE_EXCHANGE, "ln_f_final": 2.0 ** -20}
    runs = {"config0": W.config0()[0], "config2": W.config2()[0]}
    with ClockSampler(int(os.environ.get("LOCAL_RANK", 0))) as clk:
        for name, d in runs.items():
            ctx = R.Rewl([R.instance(**d)], stream=stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ok = ctx.run_to_convergence(CONVERGE_EXCHANGE, 50_000_000, poll_cycles=20)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
            c = ctx.counters(0)
            lg, _ = ctx.get_dos(0)
            sweeps = int(c["conv_sweep"].max())
            N = d["L"] ** 2
            walkers = d["n_windows"] * d["walkers_per_window"]
            ent = {"converged": bool(ok), "seconds": secs, "sweeps_slowest_window": sweeps,
                   "sweeps_run": int(ctx.status(0)["sweeps"]), "walkers": walkers,
                   "attempts_to_converge": sweeps * walkers * N}
            if d["model"] == W.ISING:
                ent["eps_vs_exact"] = _mean_rel_err(lg, _golden_ising(d["L"]))
            else:
                ent["log_sum_minus_N_ln_q"] = _log_sum(lg) - N * math.log(d["q"])
            out[name] = ent
            ctx.close()
    out["clocks"] = clk.summary()
    # the oracle on the host cores
    d = runs["config0"]
    o = O.Oracle(d["model"], d["L"], d["q"], d["e_min"], d["e_max"], d["n_windows"], d["overlap"],
                 d["walkers_per_window"], d["flatness"], d["ln_f_final"], seed=d["seed"], threads=threads)
    o.init()
    t0 = time.perf_counter()
    ok = o.run_to_convergence(CONVERGE_EXCHANGE, 50_000_000)
    secs = time.perf_counter() - t0
    lg, _ = cc.concatenate(o.pieces(), o.lo, o.w, o.reach, 4.0, math.log(2))
    cpu = {"config0": {"kind": "full run", "converged": bool(ok), "seconds": secs,
                       "sweeps_slowest_window": int(np.max(o.counters()["conv_sweep"])),
                       "eps_vs_exact": _mean_rel_err(lg, _golden_ising(d["L"]))}}
    d = runs["config2"]
    rate, desc, t = cpu_oracle_rate([d], 5.0, threads)
    cpu["config2"] = {"kind": "extrapolated: attempts to converge of the GPU run (same trajectory) / oracle attempts/s",
                      "seconds": out["config2"]["attempts_to_converge"] / rate, "oracle_attempts_per_s": rate,
                      "sample": desc}
    cpu["cores"] = threads
    out["cpu_oracle"] = cpu
    return out


def profile_case():
    """The benchmark's batch and launch shape with short launches: two cycles
    of 20 sweeps + exchange, for ncu (kernel durations of a few ms)."""
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W
    torch.cuda.set_device(0)
    ds = W.config1()
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    for _ in range(2):
        ctx.run(20)
        ctx.exchange()
    torch.cuda.synchronize()
    st = ctx.status(0)
    ctx.close()
    print(json.dumps({"profile_case": "config1 batch, 2 x (20 sweeps + exchange)", "sweeps": st["sweeps"]}))


def profile_case_large():
    """A lattice kept in global memory: one q = 10 Potts L = 400 instance
    (windows of about 490 bins, one walker each: 2610 walkers, 418 MB of
    lattices, more than L2), two cycles of 2 sweeps + exchange, for ncu."""
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W
    torch.cuda.set_device(0)
    ds = W.potts_fss(sizes=(400,), seeds=1, walkers=1, seed0=80000)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    for _ in range(2):
        ctx.run(2)
        ctx.exchange()
    torch.cuda.synchronize()
    st = ctx.status(0)
    ctx.close()
    print(json.dumps({"profile_case": "q=10 Potts L=400, 2610 windows x 1 walker, 2 x (2 sweeps + exchange)",
                      "sweeps": st["sweeps"]}))


def _golden_ising(L):
    """Exact ln g of the L x L Ising model on its bin grid, from the fixture
    written by tests/golden/make_golden.py (nan where no configuration)."""
    import numpy as np
    path = os.path.join(ROOT, "tests", "golden", f"ising_L{L}_exact_lng.txt")
    rows = np.loadtxt(path, usecols=(0, 1))
    N = L * L
    out = np.full(N + 1, np.nan)
    out[((rows[:, 0] + 2 * N) // 4).astype(int)] = rows[:, 1]
    return out


def _mean_rel_err(lg, ref):
    import numpy as np
    ok = np.isfinite(lg) & np.isfinite(ref) & (ref != 0)
    return float(np.mean(np.abs(lg[ok] - ref[ok]) / np.abs(ref[ok])))


def _log_sum(lg):
    import numpy as np
    v = lg[np.isfinite(lg)]
    m = v.max()
    return float(m + np.log(np.exp(v - m).sum()))


def _converge(ctx, exchange_interval, poll_cycles, cap_s, tag):
    """run_to_convergence in chunks of 50 cycles with a wall-time cap; progress
    (converged windows, ln f range) on stderr."""
    import numpy as np
    t0 = time.perf_counter()
    while True:
        done = ctx.run_to_convergence(exchange_interval, 50 * exchange_interval, poll_cycles=poll_cycles)
        st = ctx.status(0)
        lnf = st["ln_f"]
        print(f"[{tag}] {time.perf_counter() - t0:7.1f} s, sweeps {st['sweeps']}, windows converged "
              f"{int(np.sum(lnf == 0))}/{lnf.size} (instance 0)", file=sys.stderr, flush=True)
        if done or time.perf_counter() - t0 > cap_s:
            return done


def _stage_table(stage_sweeps):
    """Per WL stage k (ln f = 2^-k): sweeps the stage took, mean over the
    windows of all instances, and the sweep at which its last window ended it
    (mean over instances); from rewl_get_stage_sweeps."""
    import numpy as np
    rows = []
    for k in range(33):
        durs, ends = [], []
        for ss in stage_sweeps:
            end = ss[:, k]
            if np.all(end < 0):
                continue
            prev = ss[:, k - 1] if k > 0 else np.zeros_like(end)
            prev = np.where(prev < 0, 0, prev)           # a warm start begins later
            ok = end >= 0
            durs.extend((end - prev)[ok].tolist())
            ends.append(int(end[ok].max()))
        if durs:
            rows.append({"stage": k, "mean_window_sweeps": float(np.mean(durs)),
                         "max_window_sweeps": int(np.max(durs)), "last_window_end": float(np.mean(ends))})
    return rows


def warm_start_workload(seeds=4, exchange_interval=1000, poll_cycles=5, cap_s=900.0, models=(0, 1)):
    """Time to ln f = 2^-20, learned warm start vs plain REWL, on one GPU: the
    network is trained on plain-REWL DOS at L = 8..48 (Ising and q=10 Potts),
    then Ising L = 128 and q=10 Potts L = 64 (64 windows x 4 walkers, `seeds`
    instances each in one batch) run to convergence from ln g = 0, ln f = 1
    (plain) and from the network's ln g at ln f = 2^-4 (learned).  Reports wall
    time, sweeps of each instance's slowest window (the MC time of Eq. (7)),
    and the ln g error: Ising against the exact DOS, Potts against the plain
    run's DOS and through ln sum g = N ln q."""
    import math
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import warmstart as WS
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    clk = ClockSampler(0)
    clk.__enter__()
    t0 = time.perf_counter()
    train = W.config4_training()
    gen = R.Rewl([R.instance(**d) for d in train], stream=stream)
    ok = _converge(gen, exchange_interval, poll_cycles, cap_s, "training runs")
    t_gen = time.perf_counter() - t0
    X, T = WS.training_set(gen, train)
    gen.close()
    t1 = time.perf_counter()
    net = R.Mlp(max_batch=4096, seed=11, stream=stream)
    hist = WS.train(net, X, T, steps=3000, batch=4096, lr=2e-3, seed=2, log_every=1000, lr_end=1e-4)
    rms = float(np.sqrt(np.mean((WS.predict(net, X) - T) ** 2)))
    t_train = time.perf_counter() - t1
    out = {"metric": "time to ln f=2^-20, learned vs plain", "unit": "s", "n_gpus": 1, "data": "synthetic",
           "training": {"instances": len(train), "converged": bool(ok), "samples": int(X.shape[0]),
                        "generate_s": t_gen, "train_s": t_train, "train_steps": 3000,
                        "rms_error_s_per_site": rms, "loss_history": hist},
           "results": []}
    for tgt in W.config4_targets():
        L, model = tgt["L"], tgt["model"]
        if model not in models:
            continue
        ds = [dict(tgt, seed=tgt["seed"] + k) for k in range(seeds)]
        runs = {}
        for mode in ("plain", "learned"):
            ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
            ctx.run(1)                       # plan and first launch outside the timed region
            torch.cuda.synchronize()
            if mode == "learned":
                for k in range(seeds):
                    ctx.warm_start(k, net, 2.0 ** -4)
            ts = time.perf_counter()
            conv = _converge(ctx, exchange_interval, poll_cycles, cap_s, f"L={L} {mode}")
            torch.cuda.synchronize()
            secs = time.perf_counter() - ts
            sweeps = [int(ctx.counters(k)["conv_sweep"].max()) for k in range(seeds)]
            dos = [ctx.get_dos(k)[0] for k in range(seeds)]
            runs[mode] = dict(seconds=secs, converged=bool(conv), sweeps_slowest_window=sweeps, dos=dos,
                              stages=_stage_table([ctx.stage_sweeps(k) for k in range(seeds)]))
            ctx.close()
        res = {"instance": ("Ising" if model == R.ISING else "Potts q=10") + f" L={L}, 64 windows x 4 walkers",
               "seeds": seeds}
        for mode, r in runs.items():
            ent = {"seconds": r["seconds"], "converged": r["converged"],
                   "sweeps_slowest_window": r["sweeps_slowest_window"],
                   "mean_sweeps": float(np.mean(r["sweeps_slowest_window"])), "per_stage": r["stages"]}
            if model == R.ISING:
                ex = _golden_ising(L)
                ent["eps_vs_exact"] = [_mean_rel_err(lg, ex) for lg in r["dos"]]
            else:
                ent["log_sum_minus_N_ln_q"] = [_log_sum(lg) - L * L * math.log(10) for lg in r["dos"]]
            res[mode] = ent
        if model != R.ISING:
            res["learned"]["eps_vs_plain"] = [_mean_rel_err(a, b) for a, b in
                                             zip(runs["learned"]["dos"], runs["plain"]["dos"])]
            res["plain"]["eps_seed_to_seed"] = [_mean_rel_err(runs["plain"]["dos"][k], runs["plain"]["dos"][0])
                                               for k in range(1, seeds)]
        res["sweep_ratio_learned_over_plain"] = res["learned"]["mean_sweeps"] / res["plain"]["mean_sweeps"]
        res["time_ratio_learned_over_plain"] = res["learned"]["seconds"] / res["plain"]["seconds"]
        out["results"].append(res)
    net.close()
    clk.__exit__(None, None, None)
    out["clocks"] = clk.summary()
    print(json.dumps(out))


def potts_tc_workload(exchange_interval=1000, poll_cycles=5, cap_s=1500.0):
    """q = 10 Potts transition temperature from the specific-heat maxima of
    L = 16..64 lattices (Sec. IV A), all sizes and seeds in one batch run to
    ln f = 2^-20; per size the peak temperature of every seed, its bootstrap
    error over the seeds, and the extrapolation Tc(L) = Tc + a / L^2 against
    the exact 1 / ln(1 + sqrt q)."""
    import math
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import thermo as TH
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ds = W.potts_fss()
    ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
    ctx.run(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv = _converge(ctx, exchange_interval, poll_cycles, cap_s, "potts fss")
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    q = ds[0]["q"]
    tc_exact = 1.0 / math.log(1.0 + math.sqrt(q))
    sizes = sorted({d["L"] for d in ds})
    per = []
    for L in sizes:
        ks = [k for k, d in enumerate(ds) if d["L"] == L]
        peaks, heights, sweeps, lsum = [], [], [], []
        for k in ks:
            lg, e = ctx.get_dos(k)
            t, c = TH.cv_peak(lg, e, 0.6, 0.85)
            peaks.append(t)
            heights.append(c / (L * L))
            sweeps.append(int(ctx.counters(k)["conv_sweep"].max()))
            lsum.append(_log_sum(lg) - L * L * math.log(q))
        m, se = TH.bootstrap(np.array(peaks), n_resamples=200, seed=L)
        per.append({"L": L, "windows": ds[ks[0]]["n_windows"], "T_peak": peaks, "T_peak_mean": m,
                    "T_peak_bootstrap_err": se, "C_max_per_site": heights, "sweeps_slowest_window": sweeps,
                    "log_sum_minus_N_ln_q": lsum})
    Ls = [p["L"] for p in per]
    tcs = [p["T_peak_mean"] for p in per]
    errs = [max(p["T_peak_bootstrap_err"], 1e-6) for p in per]
    tc_inf, tc_err, a = TH.extrapolate_tc(Ls, tcs, errs)
    tc_inf3, tc_err3, a3 = TH.extrapolate_tc(Ls[2:], tcs[2:], errs[2:])
    out = {"metric": "q=10 Potts transition temperature from C_v maxima", "n_gpus": 1, "data": "synthetic",
           "converged": bool(conv), "seconds": secs, "seeds_per_size": len(ds) // len(sizes),
           "sizes": per, "Tc_inf_fit_all": tc_inf, "Tc_inf_fit_all_err": tc_err, "fit_all_a": a,
           "Tc_inf_fit_L_ge_32": tc_inf3, "Tc_inf_fit_L_ge_32_err": tc_err3, "Tc_exact": tc_exact}
    ctx.close()
    print(json.dumps(out))


def potts_tc_large_workload(sizes=(32, 48, 64, 80, 100, 128), seeds=4, width=490, stage_final=20,
                            exchange_interval=None, poll_cycles=5, cap_s=2400.0, seed0=60000, save=None,
                            e_range=None, lattice_placement=0):
    """q = 10 Potts transition temperature from C_v maxima (Sec. IV A): one
    batch per lattice size (its seeds together), the batches driven
    concurrently from host threads on their own streams, so each size runs
    at its own pace (a sweep of L = 400 is 16 times one of L = 100); windows
    of about `width` bins at 75 % overlap, one walker each, run to
    ln f = 2^-stage_final; lattices above L = 128 stay in global memory.
    Exchanges every max(50, 10^7 / N) sweeps unless `exchange_interval` is
    given.  Per size the C_v peak of the mean DOS with the paper's bootstrap
    error (Sec. II B: per-window pieces of the seeds resampled with
    replacement, 200 times, each resample joined) when there are several
    seeds, and the fit Tc(L) = Tc + a / L^2 against the exact
    1 / ln(1 + sqrt q).  `save`: write every instance's pieces and geometry to
    this .npz file (for pooling runs).  e_range = (a, b): energies restricted
    to [a N, b N], which must hold the canonical weight of the temperatures
    searched (the ground-state edge of large lattices is by far the slowest
    part of a full-range run and carries no weight near Tc)."""
    import math
    import threading
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import thermo as TH
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    q = 10
    tc_exact = 1.0 / math.log(1.0 + math.sqrt(q))
    n_seeds = dict(zip(sizes, seeds)) if isinstance(seeds, (tuple, list)) else {L: seeds for L in sizes}
    runs = {}
    for L in sizes:
        ds = W.potts_fss(sizes=(L,), seeds=n_seeds[L], walkers=1, seed0=seed0, width=width, e_range=e_range)
        for d in ds:
            d["ln_f_final"] = 2.0 ** -stage_final
        x = exchange_interval or max(50, int(round(1e7 / (L * L))))
        runs[L] = {"ds": ds, "x": x, "stream": torch.cuda.Stream()}

    def drive(L):
        r = runs[L]
        try:
            t0 = time.perf_counter()
            ctx = R.Rewl([R.instance(**d) for d in r["ds"]], stream=r["stream"])
            if lattice_placement:
                ctx.set_option(R.OPT_LATTICE_PLACEMENT, lattice_placement)
            ctx.run(1)
            r["stream"].synchronize()
            r["create_s"] = time.perf_counter() - t0
            done = False
            while not done and time.perf_counter() - t0 < cap_s:
                done = ctx.run_to_convergence(r["x"], 20 * r["x"], poll_cycles=poll_cycles)
            r["stream"].synchronize()
            r["seconds"] = time.perf_counter() - t0
            r["converged"] = bool(done)
            r["ctx"] = ctx
            print(f"[potts fss] L={L}: {'converged' if done else 'stopped'} after {r['seconds']:.0f} s",
                  file=sys.stderr, flush=True)
        except Exception as e:          # reported in the output line
            r["error"] = repr(e)

    with ClockSampler(0) as clk:
        t0 = time.perf_counter()
        th = [threading.Thread(target=drive, args=(L,)) for L in sizes]
        for t in th:
            t.start()
        for t in th:
            t.join()
        secs = time.perf_counter() - t0
    per, saved = [], {}
    for L in sizes:
        r = runs[L]
        seeds = n_seeds[L]
        ent = {"L": L, "windows": r["ds"][0]["n_windows"], "seeds": seeds, "exchange_every": r["x"],
               "seconds": r.get("seconds"), "converged": r.get("converged", False)}
        if "error" in r:
            ent["error"] = r["error"]
            per.append(ent)
            continue
        ctx = r["ctx"]
        g = ctx.geometry(0)
        pieces = np.stack([ctx.get_dos(k, per_window=True)[0] for k in range(seeds)])
        _, e = ctx.get_dos(0)
        saved.update({f"L{L}_pieces": pieces, f"L{L}_lo": g["lo"], f"L{L}_ww": g["ww"], f"L{L}_reach": g["reach"],
                      f"L{L}_e": e, f"L{L}_conv_sweep": np.array([ctx.counters(k)["conv_sweep"] for k in range(seeds)])})
        ent["sweeps_slowest_window"] = [int(ctx.counters(k)["conv_sweep"].max()) for k in range(seeds)]
        if ent["converged"]:
            lo_t, hi_t = 0.66, 0.76

            def tpk(lg, e=e):
                return TH.cv_peak(lg, e, lo_t, hi_t)[0]

            def cmax(lg, e=e, L=L):
                return TH.cv_peak(lg, e, lo_t, hi_t)[1] / (L * L)

            if seeds > 1:
                _, _, obs = TH.bootstrap_dos(pieces, g["lo"], g["ww"], g["reach"], 1.0, math.log(q), n_resamples=200,
                                             seed=L, observables={"T_peak": tpk, "C_max_per_site": cmax})
                ent.update({"T_peak": obs["T_peak"][0], "T_peak_bootstrap_err": obs["T_peak"][1],
                            "C_max_per_site": obs["C_max_per_site"][0],
                            "C_max_bootstrap_err": obs["C_max_per_site"][1]})
            else:
                lg = ctx.get_dos(0)[0]
                ent.update({"T_peak": tpk(lg), "C_max_per_site": cmax(lg)})
            ent["log_sum_minus_N_ln_q"] = [_log_sum(ctx.get_dos(k)[0]) - L * L * math.log(q) for k in range(seeds)]
        per.append(ent)
        ctx.close()
    if save:
        np.savez_compressed(save, **saved)
    fits = {}
    ok = [p for p in per if "T_peak_bootstrap_err" in p]
    if len(ok) >= 3:
        Ls = [p["L"] for p in ok]
        for lmin in sorted({Ls[0]} | {L for L in Ls if L in (64, 100)}):
            idx = [k for k, L in enumerate(Ls) if L >= lmin]
            if len(idx) >= 3:
                t, e_, a = TH.extrapolate_tc([Ls[k] for k in idx], [ok[k]["T_peak"] for k in idx],
                                             [max(ok[k]["T_peak_bootstrap_err"], 1e-7) for k in idx])
                fits[f"L_ge_{lmin}"] = {"Tc_inf": t, "err": e_, "a": a}
    out = {"metric": "q=10 Potts transition temperature from C_v maxima", "n_gpus": 1, "data": "synthetic",
           "workload": f"q=10 Potts L={list(sizes)}, windows of ~{width} bins at 75 %, 1 walker each, "
                       f"{[n_seeds[L] for L in sizes]} seeds per size, one batch per size run concurrently, "
                       f"ln f_final = 2^-{stage_final}, energies "
                       f"{'[-2N, 0]' if e_range is None else f'[{e_range[0]} N, {e_range[1]} N]'}",
           "seconds": secs, "walkers": int(sum(r["ds"][0]["n_windows"] * n_seeds[L] for L, r in runs.items())),
           "sizes": per, "fits": fits, "Tc_exact": tc_exact, "clocks": clk.summary()}
    print(json.dumps(out))


def config_throughput_workload(steps=3, warmup=3, sweeps=10000):
    """Attempts/s of the other batch shapes on one GPU: the single 2D Ising
    L = 8 instance (4 windows x 1 walker), the q = 10 Potts L = 32 instance
    (32 windows x 8 walkers) and the uneven batch (64 Ising instances, L from
    {16..64}, and 32 q = 10 Potts instances, L from {16, 24, 32}).  One step =
    `sweeps` sweeps + one exchange, CUDA events on the library's stream, L2
    flushed between steps; the issue-rate fraction counts 110 (Ising) and 146
    (Potts) algorithmic thread instructions per trial against the sweep
    launches' time."""
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sm * 4 * 32 * MAX_SM_MHZ * 1e6
    rows = {}
    with ClockSampler(0) as clk:
        for name, ds in (("ising_L8_4x1", W.config0()), ("potts_q10_L32_32x8", W.config2()),
                         ("uneven_64_ising_32_potts", W.config3())):
            ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
            for _ in range(warmup):
                ctx.run(sweeps)
                ctx.exchange()
            torch.cuda.synchronize()
            tot, ks = [], []
            for _ in range(steps):
                flush.fill_(1)
                a, m, b = (torch.cuda.Event(enable_timing=True) for _ in range(3))
                a.record(stream)
                ctx.run(sweeps)
                m.record(stream)
                ctx.exchange()
                b.record(stream)
                b.synchronize()
                tot.append(a.elapsed_time(b) / 1e3)
                ks.append(a.elapsed_time(m) / 1e3)
            ctx.close()
            att = W.attempts_per_sweep(ds) * sweeps
            instr = sum(INSTR_PER_TRIAL[d["model"]] * d["n_windows"] * d["walkers_per_window"] * d["L"] ** 2
                        for d in ds) * sweeps
            t, k = sum(tot) / steps, sum(ks) / steps
            rows[name] = {"instances": len(ds), "walkers": sum(d["n_windows"] * d["walkers_per_window"] for d in ds),
                          "attempts_per_s": att / t, "ms_per_step": t * 1e3,
                          "issue_rate_frac": instr / k / peak, "sweeps_per_step": sweeps}
    print(json.dumps({"metric": "WL flip attempts/s per batch shape", "unit": "attempts/s", "n_gpus": 1,
                      "data": "synthetic", "steps": steps, "warmup": warmup, "l2": "flushed between steps",
                      "results": rows, "clocks": clk.summary()}))


def exchange_study_workload(intervals=(100, 1000, 10000, 0), cap_s=600.0):
    """Algorithmic effect of the replica-exchange frequency (Sec. IV B): MC
    sweeps of the slowest window to finish the first WL iteration and the first
    eight, q = 10 Potts 48 x 48 with 15 windows and one walker each, for
    exchanges every X sweeps (X = 0: no exchange).  Per-window sweep counts at
    convergence are exact (no polling error)."""
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import thermo as TH
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ds = W.exchange_study()
    res = []
    for X in intervals:
        ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream)
        t0 = time.perf_counter()
        step = X if X else 1000
        done = False
        while not done and time.perf_counter() - t0 < cap_s:
            for _ in range(20):
                if X:
                    ctx.run_cycles(1, X)
                else:
                    ctx.run(step)
            done = ctx.status(0)["all_converged"]
        secs = time.perf_counter() - t0
        first = [int(ctx.counters(k)["conv_sweep"].max()) for k, d in enumerate(ds) if d["ln_f_final"] == 1.0]
        eight = [int(ctx.counters(k)["conv_sweep"].max()) for k, d in enumerate(ds) if d["ln_f_final"] < 1.0]
        ex = ctx.counters(0)
        alpha = float(ex["ex_acc"].sum()) / max(1.0, float(ex["ex_prop"].sum()))
        m1, e1 = TH.bootstrap(np.array(first, float), seed=1)
        m8, e8 = TH.bootstrap(np.array(eight, float), seed=8)
        res.append({"exchange_every": X or None, "converged": bool(done), "seconds": secs,
                    "sweeps_first_iteration": first, "mean_first": m1, "err_first": e1,
                    "sweeps_eight_iterations": eight, "mean_eight": m8, "err_eight": e8,
                    "exchange_acceptance": alpha})
        ctx.close()
    base = [r for r in res if r["exchange_every"] is None][0]
    for r in res:
        r["speedup_first"] = base["mean_first"] / r["mean_first"]
        r["speedup_eight"] = base["mean_eight"] / r["mean_eight"]
    print(json.dumps({"metric": "algorithmic speedup from replica exchange", "n_gpus": 1, "data": "synthetic",
                      "workload": "q=10 Potts 48x48, 15 windows at 75%, m=1, 8 seeds", "results": res}))


def balanced_windows_workload(seeds=8, L=48, q=10, h=15, overlap=0.75, exchange_interval=1000, cap_s=600.0):
    """Run-time-balanced windows (Sec. V): a pilot run with equal windows
    measures the sweeps each window's slowest walker needs for the first WL
    iteration; windows resized by (t_mean / t)^(1/2) are then compared with
    equal ones on fresh seeds -- sweeps of the slowest window for the first
    iteration and for the first eight (q = 10 Potts 48 x 48, 15 windows, one
    walker each, exchanges every 10^3 sweeps)."""
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import thermo as TH
    from paper_1407_5140_gb300 import windows as WN
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    B = 2 * L * L + 1
    elo, ehi = WN.equal_windows(B, h, overlap)

    def run(seed0, win, finals):
        ds = [W._inst(W.POTTS, L, q, h, 1, seed0 + 10 * s + j, ln_f_final=f)
              for s in range(seeds) for j, f in enumerate(finals)]
        ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream, windows=[win] * len(ds))
        t0 = time.perf_counter()
        done = ctx.run_to_convergence(exchange_interval, 0)
        while not done and time.perf_counter() - t0 < cap_s:
            done = ctx.run_to_convergence(exchange_interval, 20 * exchange_interval, poll_cycles=20)
        secs = time.perf_counter() - t0
        per = {f: [ctx.counters(k)["conv_sweep"] for k, d in enumerate(ds) if d["ln_f_final"] == f] for f in finals}
        ctx.close()
        return per, secs, bool(done)

    pilot, t_pilot, ok_pilot = run(20000, (elo, ehi), [1.0])
    t_win = np.mean(np.array(pilot[1.0], float), axis=0)          # per window, mean over seeds
    blo, bhi = WN.balanced_windows(elo, ehi, t_win, B, overlap, 9)
    out = {"metric": "sweeps to finish WL iterations, equal vs run-time-balanced windows", "n_gpus": 1,
           "data": "synthetic", "workload": f"q={q} Potts {L}x{L}, {h} windows at {int(overlap * 100)}%, m=1, "
                                             f"{seeds} seeds", "pilot_seconds": t_pilot, "pilot_converged": ok_pilot,
           "pilot_window_sweeps": t_win.tolist(), "equal": {"lo": elo.tolist(), "hi": ehi.tolist()},
           "balanced": {"lo": blo.tolist(), "hi": bhi.tolist()}}
    for name, win in (("equal", (elo, ehi)), ("balanced", (blo, bhi))):
        per, secs, ok = run(30000, win, [1.0, 2.0 ** -7])
        first = np.array([c.max() for c in per[1.0]], float)
        eight = np.array([c.max() for c in per[2.0 ** -7]], float)
        m1, e1 = TH.bootstrap(first, seed=1)
        m8, e8 = TH.bootstrap(eight, seed=8)
        out[name].update({"seconds": secs, "converged": ok, "first_iteration_mean": m1, "first_iteration_err": e1,
                          "eight_iterations_mean": m8, "eight_iterations_err": e8,
                          "first_iteration_per_window": np.mean([c for c in per[1.0]], axis=0).tolist()})
    out["speedup_first"] = out["equal"]["first_iteration_mean"] / out["balanced"]["first_iteration_mean"]
    out["speedup_eight"] = out["equal"]["eight_iterations_mean"] / out["balanced"]["eight_iterations_mean"]
    print(json.dumps(out))


def balanced_converge_workload(seeds=4, L=64, q=10, h=64, m=4, overlap=0.75, exchange_interval=1000,
                               cap_s=900.0, model=1, compare_equal=True):
    """Time to ln f = 2^-20 on equal and on run-time-balanced windows (Sec. V):
    q = 10 Potts L = 64, 64 windows x 4 walkers; a first-iteration pilot on
    equal windows sizes the balanced set, then fresh seeds run to convergence
    on each.  Reports sweeps of the slowest window, wall time, and how far the
    two DOS agree (and ln sum g - N ln q)."""
    import math
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import windows as WN
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    B = 2 * L * L + 1 if model == W.POTTS else L * L + 1
    min_w = 9 if model == W.POTTS else 5
    elo, ehi = WN.equal_windows(B, h, overlap)

    def run(seed0, win, final):
        ds = [W._inst(model, L, q, h, m, seed0 + s, ln_f_final=final) for s in range(seeds)]
        ctx = R.Rewl([R.instance(**d) for d in ds], stream=stream, windows=[win] * seeds)
        ctx.run(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ok = _converge(ctx, exchange_interval, 5, cap_s, f"L={L} {'pilot' if final == 1.0 else 'run'}")
        secs = time.perf_counter() - t0
        conv = [ctx.counters(k)["conv_sweep"] for k in range(seeds)]
        dos = [ctx.get_dos(k)[0] for k in range(seeds)]
        ctx.close()
        return conv, dos, secs, ok

    clk = ClockSampler(0)
    clk.__enter__()
    pconv, _, psecs, pok = run(40000, (elo, ehi), 1.0)
    t_win = np.mean(np.array(pconv, float), axis=0)
    blo, bhi = WN.balanced_windows(elo, ehi, t_win, B, overlap, min_w)
    name_m = f"q={q} Potts" if model == W.POTTS else "Ising"
    out = {"metric": "time to ln f=2^-20, equal vs run-time-balanced windows", "unit": "s", "n_gpus": 1,
           "data": "synthetic", "workload": f"{name_m} L={L}, {h} windows x {m} walkers, {seeds} seeds",
           "pilot_seconds": psecs, "pilot_converged": pok,
           "balanced_widths": (bhi - blo + 1).tolist()}
    res = {}
    sets = (("equal", (elo, ehi)), ("balanced", (blo, bhi))) if compare_equal else (("balanced", (blo, bhi)),)
    for name, win in sets:
        conv, dos, secs, ok = run(41000 if name == "equal" else 42000, win, 2.0 ** -20)
        sw = [int(c.max()) for c in conv]
        res[name] = dos
        out[name] = {"seconds": secs, "converged": ok, "sweeps_slowest_window": sw, "mean_sweeps": float(np.mean(sw)),
                     "log_sum_minus_N_ln_q": [_log_sum(lg) - L * L * math.log(q if model == W.POTTS else 2)
                                              for lg in dos]}
        if model == W.ISING:
            out[name]["eps_vs_exact"] = [_mean_rel_err(lg, _golden_ising(L)) for lg in dos]
    clk.__exit__(None, None, None)
    out["clocks"] = clk.summary()
    if compare_equal:
        out["eps_balanced_vs_equal"] = [_mean_rel_err(a, b) for a, b in zip(res["balanced"], res["equal"])]
        out["eps_equal_seed_to_seed"] = [_mean_rel_err(res["equal"][k], res["equal"][0]) for k in range(1, seeds)]
        out["sweep_ratio_balanced_over_equal"] = out["balanced"]["mean_sweeps"] / out["equal"]["mean_sweeps"]
        out["time_ratio_balanced_over_equal"] = out["balanced"]["seconds"] / out["equal"]["seconds"]
    print(json.dumps(out))


def self_tuning_workload(L=128, h=64, m=4, seeds=4, overlap=0.75, exchange_interval=1000, model=0, q=2,
                         tune_at=(0, 1, 2, 3, 4, 5), tune_avg=1, skip_equal=False):
    """Time to ln f = 2^-20 on equal and on self-tuning windows (Sec. V), the
    same seeds on both: the self-tuning batch starts on equal windows; after
    each stage in `tune_at` it resizes the windows from the sweeps per window
    of the last `tune_avg` stages (when the slowest took more than 1.2 times
    the mean) and continues from each instance's joined ln g at the next
    ln f.  Ising L = 128, 64 windows x 4 walkers, `seeds` instances per
    batch; error against the exact DOS; per-window sweeps of every stage."""
    import numpy as np
    import torch
    from paper_1407_5140_gb300 import rewl as R
    from paper_1407_5140_gb300 import windows as WN
    from paper_1407_5140_gb300 import workloads as W

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    B = L * L + 1 if model == W.ISING else 2 * L * L + 1
    min_w = 5 if model == W.ISING else 9
    elo, ehi = WN.equal_windows(B, h, overlap)
    exact = _golden_ising(L) if model == W.ISING else None
    name_m = "Ising" if model == W.ISING else f"q={q} Potts"
    out = {"metric": "time to ln f=2^-20, equal vs self-tuning windows", "unit": "s", "n_gpus": 1,
           "data": "synthetic", "workload": f"{name_m} L={L}, {h} windows x {m} walkers, {seeds} seeds in one "
                                             f"batch, exchange every {exchange_interval} sweeps",
           "tune_at": list(tune_at), "tune_avg": tune_avg}

    def make(lo, hi):
        ds = [W._inst(model, L, q, h, m, 50000 + s) for s in range(seeds)]
        return R.Rewl([R.instance(**d) for d in ds], stream=stream, windows=[(lo, hi)] * seeds)

    def errs(ctx):
        if exact is None:
            return None
        return [_mean_rel_err(ctx.get_dos(i)[0], exact) for i in range(seeds)]

    def per_window(ctx):
        # mean over the instances of each window's sweeps in each stage run here
        ss = [ctx.stage_sweeps(i) for i in range(seeds)]
        rows = {}
        for k in range(33):
            d = [WN.stage_durations(s, k) for s in ss]
            if all(x is not None for x in d) and np.all(np.array([s[:, k] for s in ss]) >= 0):
                rows[k] = np.mean(d, axis=0).round(1).tolist()
        return rows

    with ClockSampler(0) as clk:
        if not skip_equal:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ctx = make(elo, ehi)
            while not ctx.run_to_convergence(exchange_interval, 50 * exchange_interval, poll_cycles=5):
                pass
            torch.cuda.synchronize()
            out["equal"] = {"seconds": time.perf_counter() - t0,
                            "sweeps_slowest_window": [int(ctx.counters(i)["conv_sweep"].max()) for i in range(seeds)],
                            "eps_vs_exact": errs(ctx),
                            "stage_table": _stage_table([ctx.stage_sweeps(i) for i in range(seeds)]),
                            "per_window_stage_sweeps": per_window(ctx)}
            ctx.close()
            print(f"[self-tuning] equal windows: {out['equal']['seconds']:.1f} s", file=sys.stderr, flush=True)
        t0 = time.perf_counter()
        ctx, (flo, fhi), resizes, sweeps = WN.self_tuning_run(
            make, (elo, ehi), B, overlap, min_w, exchange_interval, n_inst=seeds, tune_at=tune_at, tune_avg=tune_avg,
            max_width=3 * int(ehi[0] - elo[0] + 1),
            log=lambda msg: print(f"[self-tuning] {msg}", file=sys.stderr, flush=True))
        torch.cuda.synchronize()
        out["self_tuning"] = {"seconds": time.perf_counter() - t0, "sweeps_run": sweeps, "resizes": resizes,
                              "eps_vs_exact": errs(ctx),
                              "final_widths": (np.asarray(fhi) - np.asarray(flo) + 1).tolist(),
                              "stage_table_last_batch": _stage_table([ctx.stage_sweeps(i) for i in range(seeds)]),
                              "per_window_stage_sweeps_last_batch": per_window(ctx)}
        ctx.close()
    out["clocks"] = clk.summary()
    if not skip_equal:
        out["time_ratio_self_tuning_over_equal"] = out["self_tuning"]["seconds"] / out["equal"]["seconds"]
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-converge", action="store_true",
                    help="skip the time-to-converge runs (Config 0 and Config 2 to ln f = 2^-20)")
    ap.add_argument("--profile-case-large", action="store_true",
                    help="a Potts L=400 batch (lattices in global memory) with 2-sweep launches (for ncu captures)")
    ap.add_argument("--profile-case", action="store_true",
                    help="only the workload's launch shape with 20 sweeps per launch (for ncu captures)")
    ap.add_argument("--sizes", default=None, help="potts-tc-large: comma-separated lattice sides")
    ap.add_argument("--seeds", default=None, help="potts-tc-large: independent runs per size (one number, or one per size)")
    ap.add_argument("--width", type=int, default=None, help="potts-tc-large: bins per window")
    ap.add_argument("--stage-final", type=int, default=None, help="potts-tc-large: last WL stage (ln f = 2^-k)")
    ap.add_argument("--cap-s", type=float, default=None, help="potts-tc-large: wall-time cap of the run")
    ap.add_argument("--seed0", type=int, default=None, help="potts-tc-large: first seed")
    ap.add_argument("--e-range", default=None, help="potts-tc-large: energies [a N, b N] as 'a,b'")
    ap.add_argument("--lattice-placement", type=int, default=0,
                    help="potts-tc-large: 1 = lattices in global memory, 2 = shared (default: by size)")
    ap.add_argument("--save", default=None, help="potts-tc-large: .npz file for the per-window pieces")
    ap.add_argument("--ising-only", action="store_true", help="warm-start: the Ising L=128 target only")
    ap.add_argument("--tune-at", default=None,
                    help="self-tuning: comma-separated stages after which windows may be resized")
    ap.add_argument("--tune-avg", type=int, default=1,
                    help="self-tuning: stages averaged for each resize decision")
    ap.add_argument("--skip-equal", action="store_true", help="self-tuning: run the self-tuning batch only")
    ap.add_argument("--workload", default="throughput", choices=["throughput", "warm-start", "potts-tc", "exchange", "balanced-windows",
                             "balanced-converge", "balanced-converge-ising", "self-tuning", "potts-tc-large", "configs"],
                    help="warm-start: time to converge, learned vs plain (Ising L=128, Potts q=10 L=64); "
                         "potts-tc: q=10 Potts transition from C_v maxima, L=16..64; "
                         "exchange: sweeps to finish WL iterations vs exchange frequency; "
                         "balanced-windows: equal vs run-time-balanced windows; "
                         "balanced-converge: time to converge on equal vs balanced windows (Potts q=10 L=64)")
    args = ap.parse_args()
    if args.profile_case_large:
        profile_case_large()
        return
    if args.profile_case:
        profile_case()
        return
    if args.workload == "warm-start":
        warm_start_workload(models=(0,) if args.ising_only else (0, 1))
        return
    if args.workload == "potts-tc":
        potts_tc_workload()
        return
    if args.workload == "exchange":
        exchange_study_workload()
        return
    if args.workload == "balanced-windows":
        balanced_windows_workload()
        return
    if args.workload == "balanced-converge":
        balanced_converge_workload()
        return
    if args.workload == "balanced-converge-ising":      # Ising L=128, balanced windows only
        balanced_converge_workload(L=128, q=2, model=0, compare_equal=False)
        return
    if args.workload == "self-tuning":
        self_tuning_workload(tune_at=tuple(int(x) for x in args.tune_at.split(",")) if args.tune_at else (0, 1, 2, 3, 4, 5),
                             tune_avg=args.tune_avg, skip_equal=args.skip_equal)
        return
    if args.workload == "potts-tc-large":
        kw = {}
        if args.sizes:
            kw["sizes"] = tuple(int(x) for x in args.sizes.split(","))
        if args.seeds:
            sd = [int(x) for x in args.seeds.split(",")]
            kw["seeds"] = sd[0] if len(sd) == 1 else tuple(sd)
        if args.width:
            kw["width"] = args.width
        if args.stage_final:
            kw["stage_final"] = args.stage_final
        if args.cap_s:
            kw["cap_s"] = args.cap_s
        if args.seed0 is not None:
            kw["seed0"] = args.seed0
        if args.e_range:
            kw["e_range"] = tuple(float(x) for x in args.e_range.split(","))
        if args.lattice_placement:
            kw["lattice_placement"] = args.lattice_placement
        potts_tc_large_workload(save=args.save, **kw)
        return
    if args.workload == "configs":
        config_throughput_workload()
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    threads = os.cpu_count() or 1
    from paper_1407_5140_gb300 import workloads as W
    workload = ("2D Ising REWL batch: L=32 and L=64, 16 windows x 4 walkers at 75% overlap, "
                "32 seeds per size (4096 walkers), 10^4 sweeps + 1 exchange per step")
    config = {"workload": workload, "instances": 64, "walkers": 4096, "sweeps_per_step": SWEEPS_PER_STEP,
              "l2": "flushed between steps (256 MiB write)"}

    if args.impl == "reference":
        if rank != 0:
            return
        import oracle  # noqa: F401  (C oracle, built by build())
        ds = W.config1()
        sample = [ds[0], ds[32]]
        rates = []
        for _ in range(args.warmup + args.steps):
            r, desc, t = cpu_oracle_rate(sample, args.cpu_budget / max(1, args.steps), threads)
            rates.append(r)
        v = statistics.mean(rates[args.warmup:])
        print(json.dumps({"impl": "reference", "metric": "WL flip attempts/s", "value": v, "unit": "attempts/s",
                          "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
                          "ms_per_step": W.attempts_per_sweep(ds) * SWEEPS_PER_STEP / v * 1e3,
                          "ms_per_step_kind": "extrapolated: the step's attempts (64 instances x 10^4 sweeps) over the "
                                              "rate measured on a sample of 2 of the 64 instances",
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                          "data": "synthetic", "config": config,
                          "cpu_baseline": {"value": v, "unit": "attempts/s", "cores": threads, "kind": "oracle",
                                           "sample": "per step: " + desc + " (2 of the 64 instances; the rate is "
                                                     "extrapolated to the whole batch)"},
                          "e2e": {"value": v, "unit": "attempts/s", "h2d_bytes_per_step": 0,
                                  "d2h_bytes_per_step": 0}}))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = run_ours(args, rank, world)
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank != 0:
        return
    cpu = None
    ttc = None
    if world == 1:
        ds = r["ds"]
        v, desc, t = cpu_oracle_rate([ds[0], ds[32]], args.cpu_budget, threads)
        cpu = {"value": v, "unit": "attempts/s", "cores": threads, "kind": "oracle",
               "sample": desc + f" ({t:.1f} s of oracle time)"}
        if not args.no_converge:
            ttc = time_to_converge(threads)
    out = {"metric": "WL flip attempts/s", "value": r["value"], "unit": "attempts/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["t_step"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic", "config": config,
           "roofline": r["roofline"], "cpu_baseline": cpu, "e2e": r["e2e"], "clocks": r["clocks"],
           "gpu_launches": r["launches"], "time_to_converge": ttc}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
