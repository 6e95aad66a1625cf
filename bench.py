"""Benchmark: encrypted vital-sign windows per second on one or more B300s.

Workload (the configuration the headline metric is quoted on): the full
vital-sign chain (K1 -> K2 | K4 -> K5 -> K7 -> K3 -> |X|^2 -> sharpen ->
weighted average; depth 11) at N = 2^15 with 12 + 4 primes, one 10 s window
= 200 frames x 256 range bins = 16 input ciphertexts.  A step evaluates a
batch of B windows of one user (every launch covers the whole batch);
B = 64 by default (profiles/vital_chain_batch_sweep.md).

Inputs are synthetic: uniform residues for the ciphertexts and switching keys
(under RLWE a ciphertext or key is indistinguishable from such words, and the
circuit is data-oblivious, so this is exactly the cloud's view), the plan's
public constants designed and encoded by the library itself.  Each step
reads B x 96 MiB of ciphertexts, more than the 126 MB L2.

Timed region (device-resident): K steps on one stream, bracketed by a barrier
and torch.cuda.synchronize, CUDA events per step.  e2e: the same windows from
pinned host buffers through the serving API (mmfhe_server, two stream slots:
a batch's host <-> device copies run under the previous batch's kernels);
the synchronous mmfhe_eval with host buffers is reported beside it.
Per-kernel roofline: one extra profiled step with CUDA events around every
launch (algorithmic bytes from the library).  cpu_baseline: the CPU oracle,
one whole window's chain per host process.

Multi-GPU: replicas (windows of different users are independent); each rank
evaluates its own batch, no data-path collective; timing = max over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted windows/s and p99 latency, batched+learned vs plain, same decrypted MAE"
WORKLOAD = ("vital-sign chain (K1,K2 | K4,K5,K7,K3,|X|^2,sharpen,avg; depth 11), CKKS N=2^15, "
            "Q=60+11x40 bits, P=4x60 bits, dnum=3, 200 frames x 256 bins per 10 s window, 16 input cts")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=None,
                    help="windows per step (per GPU); default 64 (vital), 16 (gesture)")
    ap.add_argument("--impl", default="mine", choices=["mine", "reference"])
    ap.add_argument("--cpu-sample-s", type=float, default=None,
                    help="time-box of the CPU oracle baseline per process; default: one whole vital window "
                         "(gesture: 20 s, a whole gesture window takes the oracle minutes)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--workload", default="vital",
                    choices=["vital", "batching", "serving", "serving-mix", "fc", "per-frame", "gesture",
                             "ntt-ablation"],
                    help="vital: the headline chain at B windows per step; batching: uneven windows through the "
                         "batcher against one call per window; serving: Poisson arrivals from many users through "
                         "the serving loop")
    ap.add_argument("--users", type=int, default=64, help="serving workload: simulated edge devices")
    ap.add_argument("--loads", default="20,60,120,200", help="serving workload: offered windows/s, one phase each")
    ap.add_argument("--phase-s", type=float, default=5.0, help="serving workload: arrival time per phase")
    ap.add_argument("--key-budget-gib", type=float, default=48.0, help="serving workload: resident key budget")
    ap.add_argument("--windows", type=int, default=64, help="batching workload: windows per step")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch-list", action="store_true",
                    help="vital workload: set-up, warm-up and the timed steps only (no e2e, no profiled step, no CPU "
                         "baseline), for an ncu launch list whose last launches are the timed steps")
    ap.add_argument("--learned", type=float, default=None, metavar="B_OVER_A",
                    help="gesture workload: the learned feature map p + B_OVER_A p^2 (depth 9, two Q primes "
                         "less) in place of the paper's p (p^2)^2")
    ap.add_argument("--complex-slots", action="store_true",
                    help="vital and gesture workloads: Re + i Im in one complex slot (half the input ciphertexts)")
    ap.add_argument("--tiles", default=None,
                    help="cols_width,rows_threads,keyip_windows,conv_rows[,keyip_pipe[,combine_pipe]]: set the "
                         "tile shapes instead of autotuning")
    ap.add_argument("--keyip-fusion", action="store_true",
                    help="form the key inner product inside the ModDown passes instead of storing it with its "
                         "own kernel (ablation; same words, slower on B300)")
    args = ap.parse_args()
    if args.batch is None:
        args.batch = 16 if args.workload == "gesture" else 64
    return args


# ---------------------------------------------------------------------------
# distributed plumbing (replicas: a barrier and a max, on CPU via gloo)
# ---------------------------------------------------------------------------
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allsum(world, x):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def job_throughput(world, windows, seconds):
    """Whole-job windows/s of replicas: every rank's windows over the slowest
    rank's time (each rank evaluates its own users' windows; no exchange)."""
    return allsum(world, windows) / allmax(world, seconds)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        # the raw samples (the JSON line carries their summary); MMFHE_CLOCKS_DIR keeps them
        self.path = os.path.join(os.environ.get("MMFHE_CLOCKS_DIR", tempfile.gettempdir()),
                                 "mmfhe_clocks_rank%d.csv" % device)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle sample (the baseline / reference arm)
# ---------------------------------------------------------------------------
class OracleSample:
    """Oracle set-up for the same workload (untimed), then time-boxed runs of
    one window's chain; progress is measured in key-switch limb units, the
    oracle's dominant cost, against a counting run of the whole chain."""

    def __init__(self, seed=4242):
        import synth
        from oracle import ckks as ck
        from oracle import circuits as cc
        from oracle import params as pm
        from oracle import plain
        self.ck, self.cc = ck, cc
        P = pm.vital_params()
        circ = cc.VitalCircuit(P, cc.VitalConfig(bins=256))
        rots = circ.rotations()
        kd = synth.KeyDraws(seed, P.n, P.q, P.p, P.dnum, rots)
        sk = ck.SecretKey(P, kd.secret)
        pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
        self.rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
        self.gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
        del kd
        self.consts = circ.constants()
        win = synth.vital_window(seed, frames=200, bins=256, randomize_rates=True)
        s1, s2 = plain.preprocess(win.z)
        lay = circ.lay

        def stream(x, sd):
            re, im = lay.pack(x.real), lay.pack(x.imag)
            return [(ck.encrypt(P, pk, ck.encode(P, re[c], P.scale, P.L), *synth.encryption_draws(sd + 2 * c, P.n)),
                     ck.encrypt(P, pk, ck.encode(P, im[c], P.scale, P.L), *synth.encryption_draws(sd + 2 * c + 1, P.n)))
                    for c in range(lay.groups)]

        self.s1, self.s2 = stream(s1, seed + 100), stream(s2, seed + 200)
        self.P, self.circ = P, circ
        counter = cc.CountingEvaluator(P)
        shapes = [(cc._Shape(P.L), cc._Shape(P.L)) for _ in range(lay.groups)]
        circ.run(counter, {k: cc._Shape(0) for k in circ.constant_keys()}, shapes, shapes)
        self.total_weight = counter.ks_weight

    def run(self, budget_s):
        """Returns (windows per second, elapsed seconds, completed fraction);
        budget_s None: the whole chain."""
        ev = self.cc.BudgetEvaluator(self.P, self.rlk, self.gks, float("inf") if budget_s is None else budget_s)
        t0 = time.perf_counter()
        try:
            self.circ.run(ev, self.consts, self.s1, self.s2)
        except self.cc.SampleBudgetExceeded:
            pass
        dt = time.perf_counter() - t0
        frac = ev.ks_weight / self.total_weight
        return frac / dt, dt, frac


class GestureOracleSample(OracleSample):
    """The same time-boxed oracle sample for the gesture chain: one 3 s
    window (30 ciphertext pairs; the two encrypted pairs repeat, the cost of
    a pair does not depend on its values)."""

    def __init__(self, seed=4343):
        import synth
        from oracle import ckks as ck
        from oracle import circuits as cc
        from oracle import params as pm
        from oracle import plain
        self.ck, self.cc = ck, cc
        P = pm.gesture_params()
        circ = cc.GestureCircuit(P, cc.GestureConfig())
        rots = circ.rotations()
        kd = synth.KeyDraws(seed, P.n, P.q, P.p, P.dnum, rots)
        sk = ck.SecretKey(P, kd.secret)
        pk = ck.gen_public_key(P, sk, kd.pk_a, kd.pk_e)
        self.rlk = ck.gen_relin_key(P, sk, kd.rlk_a, kd.rlk_e)
        self.gks = {k: ck.gen_galois_key(P, sk, k, *kd.gk[k]) for k in rots}
        del kd
        self.consts = circ.constants(gesture_random_mats(circ.cfg, seed))
        packed = circ.lay.pack(plain.gesture_preprocess(synth.gesture_window(seed).z))
        two = [tuple(ck.encrypt(P, pk, ck.encode(P, v, P.scale, P.L), *synth.encryption_draws(seed + 2 * i + h, P.n))
                     for h, v in enumerate(packed[i])) for i in range(2)]
        self.pairs = [two[i % 2] for i in range(circ.lay.pairs)]
        self.P, self.circ = P, circ
        counter = cc.CountingEvaluator(P)

        class Shapes(dict):
            def __missing__(self, k):
                return None
        circ.run(counter, Shapes(), [(cc._Shape(P.L), cc._Shape(P.L))] * circ.lay.pairs)
        self.total_weight = counter.ks_weight

    def run(self, budget_s):
        ev = self.cc.BudgetEvaluator(self.P, self.rlk, self.gks, float("inf") if budget_s is None else budget_s)
        t0 = time.perf_counter()
        try:
            self.circ.run(ev, self.consts, self.pairs)
        except self.cc.SampleBudgetExceeded:
            pass
        dt = time.perf_counter() - t0
        frac = ev.ks_weight / self.total_weight
        return frac / dt, dt, frac


def gesture_random_mats(cfg, seed):
    """Random-init weights of the gesture network (the chain's cost does not
    depend on them): FC1 width x (A R D + 1), FC2 and FC3 width x width with
    the constant row."""
    g = np.random.default_rng(seed)
    W, (d1, d2, c) = cfg.width, cfg.fc_dims
    W0 = np.zeros((W, cfg.ard + 1))
    W0[:d1] = g.normal(0, 1.0 / np.sqrt(cfg.ard), (d1, cfg.ard + 1))
    mats = [W0]
    for a, b in ((d1, d2), (d2, c)):
        M = np.zeros((W, W))
        M[:b, :a] = g.normal(0, 1.0 / np.sqrt(a), (b, a))
        M[:b, W - 1] = g.normal(0, 0.1, b)
        M[W - 1, W - 1] = 1.0
        mats.append(M)
    return mats


def _oracle_sample_worker(job):
    """One process of the parallel CPU baseline: its own oracle set-up, then
    the time-boxed sample (spawned processes; the oracle is single-threaded)."""
    kind, budget_s, seed = job
    sample = GestureOracleSample(seed) if kind == "gesture" else OracleSample(seed)
    return sample.run(budget_s)


def cpu_baseline(kind, budget_s, max_procs=8):
    """The oracle as it stands on the host cores: one single-threaded process
    per core (up to max_procs).  budget_s None: each process evaluates one
    whole window's chain and times it; otherwise each times the first budget_s
    of its window's chain.  The job's throughput is the sum of the processes'
    rates."""
    import multiprocessing as mp
    procs = max(1, min(max_procs, cpu_cores()))
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_oracle_sample_worker, [(kind, budget_s, 4242 + 17 * i) for i in range(procs)])
    rate = float(sum(r[0] for r in res))
    dt = float(np.mean([r[1] for r in res]))
    frac = float(np.mean([r[2] for r in res]))
    what = "gesture window's" if kind == "gesture" else "window's"
    if budget_s is None:
        sample = ("%d processes, each one whole %s chain (%.1f s on average, set-up untimed); throughput summed "
                  "over the processes" % (procs, what, dt))
    else:
        sample = ("%d processes, each the first %.1f s of one %s chain (%.2f%% of its key-switch limb units on "
                  "average); throughput summed over the processes" % (procs, dt, what, 100 * frac))
    return {"value": rate, "unit": "windows/s", "cores": procs, "kind": "oracle",
            "host_cores_available": cpu_cores(), "sample": sample}


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def _reference_step(seed):
    """One step of the reference arm: the oracle's set-up (untimed), then one
    whole window's chain, timed."""
    return OracleSample(seed).run(None)


def run_reference(args, rank, world):
    """The oracle as it stands, on the host cores: K steps, each one whole
    window's chain on one core, run concurrently (one spawned process per
    step, up to the host's cores at a time)."""
    if rank != 0:
        return
    import multiprocessing as mp
    procs = max(1, min(args.steps, cpu_cores()))
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(procs) as pool:
        res = pool.map(_reference_step, [4242 + 17 * i for i in range(args.steps)])
    wall = time.perf_counter() - t0
    times = [r[1] for r in res]
    value = float(np.mean([1.0 / t for t in times]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "batch_windows": 1, "parallelism": "single-threaded CPU oracle per step"},
        "cpu_baseline": {"value": value, "unit": "windows/s", "cores": 1, "kind": "oracle",
                         "sample": "each step one whole window's chain on one core (set-up untimed); %d steps run "
                                   "concurrently on %d cores, %.0f s wall; warm-up steps are not run (the oracle "
                                   "has nothing to warm)" % (args.steps, procs, wall)},
        "e2e": {"value": value, "unit": "windows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ("internal.h", "kernels.h", "kernels.cu", "modarith.cuh", "ntt_impl.cuh")


def csrc_hash():
    """Hash of the device-kernel sources (the files ncu counters depend on)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2603_22437_b300", "csrc")
    for f in KERNEL_SOURCES + tuple(sorted(x for x in os.listdir(d) if x.startswith("ntt_l"))):
        h.update(f.encode())
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        j = json.load(open(p))
        return float(j["hbm_gbs"]), "measured"
    return 6400.0, "fallback"


def ncu_traffic(kernel, batch, workload=None):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if it
    was captured on the current kernel sources; scaled from the captured batch
    to `batch` windows (every launch covers all windows of the batch).
    workload=None: the vital chain; "gesture": the gesture chain's capture."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    if j.get("csrc_hash") != csrc_hash():
        return None
    sec = j if workload is None else j.get(workload, {})
    k = sec.get("kernels", {}).get(kernel)
    if k is None:
        return None
    return k.get("dram_bytes_per_launch_full_size") * batch / sec.get("batch", batch)


ISSUE_PROFILE = os.path.join("profiles", "ncu_issue_rates.json")
SM_COUNT = 148
ISSUE_PER_SM_CLK = 4     # one warp instruction per clock from each of an SM's four schedulers


def ncu_issue(kernel, sm_mhz):
    """The dominant kernel's instruction issue against the hardware: warp
    instructions per active SM cycle from the committed ncu capture (one
    kernel, two launches, --clock-control none) of the current kernel
    sources, against the issue limit of 4 per SM per clock x 148 SMs x the SM
    clock sampled during the timed region; and each integer pipe's share of
    its own peak (ncu's pct_of_peak_sustained_active)."""
    p = os.path.join(ROOT, ISSUE_PROFILE)
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    if j.get("csrc_hash") != csrc_hash():
        return None
    k = j.get("kernels", {}).get(kernel)
    if k is None:
        return None
    ipc = k["inst_per_active_sm_cycle"]
    clk = sm_mhz or k["sm_mhz"]
    return {"inst_per_sm_cycle": ipc, "issue_limit_per_sm_cycle": ISSUE_PER_SM_CLK,
            "achieved_warp_inst_per_s": ipc * SM_COUNT * clk * 1e6,
            "peak_warp_inst_per_s": ISSUE_PER_SM_CLK * SM_COUNT * clk * 1e6,
            "frac": ipc / ISSUE_PER_SM_CLK, "sm_mhz": clk,
            "pipes_pct_of_peak": k["pipes_pct_of_peak"], "warps_active_pct": k.get("warps_active_pct"),
            "stalls_per_issue": k.get("stalls_per_issue"),
            "source": ISSUE_PROFILE + " (" + k.get("capture", "") + ")"}


def pick_tiles(ctx, args, batch):
    """Tile shapes: given (--tiles), defaults (--no-autotune) or autotuned."""
    fused = 1 if args.keyip_fusion else 0
    if args.tiles:
        v = [int(x) for x in args.tiles.split(",")]
        ctx.set_tuning(*v[:4], keyip_fused=fused, keyip_pipe=v[4] if len(v) > 4 else 0,
                       combine_pipe=v[5] if len(v) > 5 else 0)
        return ctx.tuning()
    t = ctx.tuning() if args.no_autotune else ctx.autotune(batch)
    ctx.set_tuning(t["ntt_cols_width"], t["ntt_rows_threads"], t["keyip_windows"], t["conv_rows"], fused,
                   t["keyip_pipe"], t["combine_pipe"])
    return ctx.tuning()


def roofline_of(prof, bf64_peak, bf32_peak, batch, mac_peak=None):
    """Roofline of the dominant kernel (most event time in the profiled step).

    Two ceilings apply to every NTT pass: HBM (algorithmic bytes / time against
    the measured copy bandwidth) and the integer pipes.  The integer work of a
    pass is its butterflies plus, for the fused ModUp / ModDown strided passes,
    the base conversion's multiply-accumulates; each is timed against its own
    register-resident loop measured on the same GPU, and the fraction is the
    time those ceilings allow over the measured time (reported in butterfly
    equivalents: products weighted by the ratio of the two ceilings).  The
    bound reported is the nearer one (the larger fraction); the other is kept
    under "other"."""
    hbm_peak, peak_kind = measured_peaks()
    name, (nl, ms, byts, bfs, macs) = max(prof.items(), key=lambda kv: kv[1][1])
    tot_ms = sum(v[1] for v in prof.values())
    sec = ms / 1000.0
    hbm = {"bound": "hbm", "achieved": byts / sec / 1e9, "peak": hbm_peak, "unit": "GB/s",
           "frac": byts / sec / 1e9 / hbm_peak, "peak_source": peak_kind,
           "algorithmic_bytes_per_launch": byts / nl}
    alu = None
    if bfs > 0:
        equiv = bfs + (macs * bf64_peak / mac_peak if mac_peak and macs else 0.0)
        alu = {"bound": "alu", "achieved": equiv / sec / 1e9, "peak": bf64_peak / 1e9,
               "unit": "Gbutterfly-equivalent/s", "frac": equiv / sec / bf64_peak,
               "peak_source": "measured: register-resident loops of the same 64-bit butterfly and of the base "
                              "conversion's Montgomery multiply-accumulate on all SMs",
               "butterflies_per_launch": bfs / nl, "conversion_macs_per_launch": macs / nl,
               "butterflies_only_frac": bfs / sec / bf64_peak}
    main, other = (alu, hbm) if alu and alu["frac"] > hbm["frac"] else (hbm, alu)
    r = {"kernel": name}
    r.update(main)
    r.update({"traffic": ncu_traffic(name, batch), "other": other, "launches_per_step": nl,
              "avg_launch_us": 1000.0 * ms / nl, "share_of_step": ms / tot_ms,
              "butterfly_peak_per_s": {"u64": bf64_peak, "u32": bf32_peak}, "mac_peak_per_s": mac_peak,
              "kernels": {k: {"launches": v[0], "ms": round(v[1], 3),
                              "GBps": round(v[2] / max(v[1], 1e-9) / 1e6, 1),
                              "Gbfly_s": round(v[3] / max(v[1], 1e-9) / 1e6, 1),
                              "Gmac_s": round(v[4] / max(v[1], 1e-9) / 1e6, 1)}
                          for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}})
    return r


def run_mine(args, rank, world, local):
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.vital_params()
    ctx = M.Context(params, device=local)
    plan = ctx.plan(M.vital_config(complex_slots=args.complex_slots))
    plan.encode_consts()
    rots = plan.rotations()
    P_q, P_p = params.primes_q, params.primes_p
    n = 1 << params.log_n
    g = synth.rng(7000 + rank)
    keys = ctx.keys(rank)
    qp = P_q + P_p

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))

    relin_w = key_words()
    gal_w = {k: key_words() for k in rots}
    keys_words = (relin_w, gal_w)
    keys.set_relin(relin_w)
    for k in rots:
        keys.set_galois(k, gal_w[k])
    n_in, n_out, out_levels = plan.io()
    B = args.batch
    tiles = pick_tiles(ctx, args, B)
    in_words = n_in * 2 * len(P_q) * n
    out_words = sum(2 * (l + 1) * n for l in out_levels)
    # device-resident inputs: B windows of uniform ciphertexts
    host_in = []
    for w in range(B):
        cts = synth.uniform_ciphertexts(100 * rank + w, P_q, n, n_in)
        host_in.append(cts.reshape(-1))
    d_in = [torch.from_numpy(x.view(np.int64)).to(dev) for x in host_in]
    d_out = [torch.empty(out_words, dtype=torch.int64, device=dev) for _ in range(B)]
    stream = torch.cuda.Stream(device=dev)

    def step(ins, outs):
        ctx.eval(plan, keys, ins, outs, stream=stream, vital=True)

    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step(d_in, d_out)
    torch.cuda.synchronize()

    # ---- timed region: device-resident ----
    ctx.mem_peak_reset()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(d_in, d_out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    mem = ctx.mem_stats()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value = job_throughput(world, B * args.steps, sum(step_ms) / 1000.0)
    if args.launch_list:
        return {"metric": METRIC, "value": value, "unit": "windows/s", "launch_list_run": True, "batch_windows": B,
                "steps": args.steps, "launches_per_step": launches // max(1, args.steps),
                "launches_total": ctx.launch_count(), "ms_per_step": float(np.mean(step_ms))}

    # ---- e2e: pinned host buffers, host <-> device copies inside the timed region ----
    pin_in = [torch.from_numpy(x.view(np.int64)).pin_memory() for x in host_in]
    pin_out = [torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(B)]
    # (a) one synchronous mmfhe_eval per step: copies in, evaluate, copies out, in sequence
    step(pin_in, pin_out)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step(pin_in, pin_out)
    torch.cuda.synchronize()
    e2e_sync = job_throughput(world, B * args.e2e_steps, time.perf_counter() - t0)
    # (b) the serving API (two stream slots): the next batch's copies run under this batch's kernels
    srv = ctx.server(M.vital_config(complex_slots=args.complex_slots), max_batch=B, streams=2, batch_wait_us=20000)
    srv.add_user(rank, *keys_words)
    e2e_steps = max(8, args.e2e_steps)   # enough batches that the pipeline's fill and drain are amortised
    outs_ring = [[torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(B)] for _ in range(2)]
    for w in range(B):   # warm-up: the server's plan, key upload and pools
        srv.submit(rank, 200, pin_in[w], outs_ring[0][w])
    srv.drain()
    barrier(world)
    t0 = time.perf_counter()
    for s_ in range(e2e_steps):
        for w in range(B):
            srv.submit(rank, 200, pin_in[w], outs_ring[s_ % 2][w])
    srv.drain()
    e2e_pipe_s = time.perf_counter() - t0
    srv_stats = srv.stats()
    srv.close()
    if srv_stats["failed"] or srv_stats["completed"] != srv_stats["submitted"]:
        raise RuntimeError("serving e2e: %d of %d windows failed" % (srv_stats["failed"], srv_stats["submitted"]))
    e2e = {"value": job_throughput(world, B * e2e_steps, e2e_pipe_s), "unit": "windows/s",
           "h2d_bytes_per_step": B * in_words * 8, "d2h_bytes_per_step": B * out_words * 8,
           "api": "mmfhe_server (2 stream slots, batches of %d filled within 20 ms, copies overlap the previous "
                  "batch's kernels)" % B,
           "mean_batch": srv_stats["mean_batch"],
           "synchronous_mmfhe_eval": {"value": e2e_sync, "unit": "windows/s"}}

    # ---- per-kernel profile of one more step ----
    ctx.profile(True)
    step(d_in, d_out)
    torch.cuda.synchronize()
    prof = ctx.profile()
    ctx.profile(False)
    bf64_peak, bf32_peak = ctx.butterfly_peak()
    roofline = roofline_of(prof, bf64_peak, bf32_peak, B, ctx.mac_peak())
    roofline["issue"] = ncu_issue(roofline["kernel"], clk.get("sm_mhz") if clk else None)
    variants = None
    if not args.complex_slots:
        del d_in, d_out
        variants = {"complex_slots": time_complex_variant(ctx, M, synth, params, B, args, rank, world, stream, dev)}
    line = {
        "metric": METRIC, "value": value, "unit": "windows/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD + (", complex-slot packing (Re + i Im in one slot, 8 input cts)"
                                           if args.complex_slots else ""),
                   "batch_windows": B, "windows_per_step_all_gpus": world * B,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (%d MiB of ciphertexts per step)" % (B * in_words * 8 >> 20),
                   "tiles": tiles},
        "latency_ms": {"p50": srv_stats["p50_ms"], "p99": srv_stats["p99_ms"],
                       "note": "per window, submit to output written, through mmfhe_server in the e2e run "
                               "(%d windows)" % (B * e2e_steps),
                       "step_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))}},
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk,
        "memory": memory_line(mem, B, "5.3 GB peak cloud GPU memory per batched vital window (paper Table 5, "
                                      "RTX 3090 Ti)"),
        "accuracy": accuracy_line(),
        "learned_vs_plain": learned_line(),
        "variants": variants,
        "wall_s_timed": wall,
    }
    return line


def time_complex_variant(ctx, M, synth, params, B, args, rank, world, stream, dev):
    """The same chain with complex-slot packing (Re + i Im in one slot: 8
    input ciphertexts per window instead of 16, one conjugation key more):
    device-resident inputs, the same tiles, W warm-up and K timed steps."""
    import torch
    plan = ctx.plan(M.vital_config(complex_slots=True))
    plan.encode_consts()
    n = 1 << params.log_n
    qp = params.primes_q + params.primes_p
    g = synth.rng(7100 + rank)
    keys = ctx.keys(1000 + rank)

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))
    keys.set_relin(key_words())
    for k in plan.rotations():
        keys.set_galois(k, key_words())
    n_in, _, out_levels = plan.io()
    out_words = sum(2 * (l + 1) * n for l in out_levels)
    d_in = [torch.from_numpy(synth.uniform_ciphertexts(300 + 100 * rank + w, params.primes_q, n, n_in)
                             .reshape(-1).view(np.int64)).to(dev) for w in range(B)]
    d_out = [torch.empty(out_words, dtype=torch.int64, device=dev) for _ in range(B)]
    for _ in range(args.warmup):
        ctx.eval(plan, keys, d_in, d_out, stream=stream, vital=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    for a, b in ev:
        a.record(stream)
        ctx.eval(plan, keys, d_in, d_out, stream=stream, vital=True)
        b.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = [a.elapsed_time(b) for a, b in ev]
    keys.unload()
    return {"value": job_throughput(world, B * args.steps, sum(ms) / 1000.0), "unit": "windows/s",
            "ms_per_step": float(np.mean(ms)), "input_cts_per_window": n_in,
            "note": "the same chain and outputs with Re + i Im packed into one complex slot by the client "
                    "(8 input ciphertexts instead of the paper's 16); same timing rules as value"}


def memory_line(mem, batch, paper):
    """Device memory the library held over the timed region (its own
    accounting: contexts, keys, plan constants, scratch pools)."""
    return {"peak_gib": mem["peak_bytes"] / 2.0 ** 30, "held_after_gib": mem["device_bytes"] / 2.0 ** 30,
            "per_window_gib": mem["peak_bytes"] / 2.0 ** 30 / batch, "batch_windows": batch,
            "source": "mmfhe_mem_stats_get high-water mark, reset before the timed steps", "paper": paper}


ACCURACY_PROFILE = os.path.join("profiles", "accuracy_vital_64_windows.json")


LEARNED_PROFILE = os.path.join("profiles", "gesture_learned_vs_plain.json")


def learned_line():
    """Batched learned chain against the plain one, from the committed record:
    the gesture chain with the learned feature map a p + b p^2 (depth 9) and
    with the paper's p (p^2)^2 (depth 11), windows/s at B = 16 and the
    held-out accuracy of each chain's network trained by the library on the
    same windows (tests/test_gpu_gesture_learned.py)."""
    p = os.path.join(ROOT, LEARNED_PROFILE)
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    j["source"] = LEARNED_PROFILE
    return j


def accuracy_line():
    """Decrypted rates against the FP64 pipeline over 64 seeded windows, from
    the committed record of tests/test_gpu_accuracy.py (the bench's own
    windows are uniform words, which decrypt to nothing)."""
    p = os.path.join(ROOT, ACCURACY_PROFILE)
    if not os.path.exists(p):
        return None
    j = json.load(open(p))
    keys = ("windows", "copies", "split_windows", "inside_precision_window", "within_1e-3_bpm_both_bands",
            "below_floor", "above_ceiling", "mae_bpm", "max_bpm", "max_err_target_bin")
    out = {k: j[k] for k in keys if k in j}
    if j.get("copies"):
        # a window whose two bands need separate normalization factors is
        # encrypted twice: ciphertext windows evaluated per client window
        out["copies_per_window"] = j["copies"] / j["windows"]
    out["source"] = ACCURACY_PROFILE + " (tests/test_gpu_accuracy.py, B = 64, seeds 4000..4063)"
    return out


# Uneven windows: whole-second lengths between 5 and 20 s at 20 frames/s; six
# lengths spanning the three padded sizes (F_pad = 128, 256, 512).
BATCH_FRAMES = (100, 140, 200, 260, 340, 400)


def run_batching(args, rank, world, local):
    """Uneven windows of one user through the batcher (groups by frame count,
    batches of up to --batch windows, one captured CUDA graph per batch shape)
    against the same windows evaluated one mmfhe_eval call per window, and the
    batcher without graphs.  All three return identical words (checked), so
    their decrypted accuracy is identical."""
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.vital_params()
    ctx = M.Context(params, device=local)
    n = 1 << params.log_n
    g = synth.rng(9000 + rank)
    draw = np.random.default_rng(31 + rank)
    frames = [int(f) for f in draw.choice(BATCH_FRAMES, size=args.windows)]
    base = M.vital_config()
    t0 = time.perf_counter()
    bat = ctx.batcher(base, max_batch=args.batch, use_graphs=True)
    bat_ng = ctx.batcher(base, max_batch=args.batch, use_graphs=False)
    plans = {F: bat.plan(F) for F in sorted(set(frames))}
    rots = sorted(set().union(*[set(p.rotations()) for p in plans.values()]))
    io = {F: p.io() for F, p in plans.items()}
    plan_s = time.perf_counter() - t0
    qp = params.primes_q + params.primes_p
    keys = ctx.keys(rank)

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))

    keys.set_relin(key_words())
    for k in rots:
        keys.set_galois(k, key_words())
    tiles = pick_tiles(ctx, args, args.batch)
    out_words = {F: sum(2 * (l + 1) * n for l in io[F][2]) for F in io}
    d_in = [torch.from_numpy(synth.uniform_ciphertexts(7000 + w, params.primes_q, n, io[F][0]).reshape(-1)
                             .view(np.int64)).to(dev) for w, F in enumerate(frames)]
    outs = {m: [torch.empty(out_words[F], dtype=torch.int64, device=dev) for F in frames]
            for m in ("graph", "nograph", "plain")}
    plain_plans = plans   # the batcher's own plans (no budget: never evicted)
    stream = torch.cuda.Stream(device=dev)

    def run(mode):
        if mode == "plain":
            for w, F in enumerate(frames):
                ctx.eval(plain_plans[F], keys, [d_in[w]], [outs[mode][w]], stream=stream)
            return
        b = bat if mode == "graph" else bat_ng
        for w, F in enumerate(frames):
            b.submit(keys, F, d_in[w], outs[mode][w])
        b.flush(stream)

    res = {}
    for mode in ("graph", "nograph", "plain"):
        for _ in range(max(1, args.warmup)):
            run(mode)   # first graph flush captures the graphs
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        barrier(world)
        for i in range(args.steps):
            ev[i][0].record(stream)
            run(mode)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        res[mode] = {"value": job_throughput(world, len(frames) * args.steps, sum(ms) / 1000.0),
                     "ms_per_step": float(np.mean(ms))}
    differ = []
    for w in range(len(frames)):
        for m in ("graph", "nograph"):
            if not torch.equal(outs[m][w], outs["plain"][w]):
                bad = (outs[m][w] != outs["plain"][w]).nonzero().flatten()
                differ.append({"window": w, "frames": frames[w], "mode": m, "words": int(bad.numel()),
                               "first_word": int(bad[0]), "out_words": out_words[frames[w]]})
    same = not differ
    st = bat.stats()
    line = {
        "metric": METRIC, "value": res["graph"]["value"], "unit": "windows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["graph"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "uneven vital-sign windows through the batcher: %d windows per step, lengths drawn "
                               "from %s frames (5-20 s at 20 Hz), 256 bins, N=2^15 chain; batches of <= %d windows "
                               "per (frame count, key set), one CUDA graph per batch shape"
                               % (len(frames), list(BATCH_FRAMES), args.batch),
                   "frames_histogram": {str(F): frames.count(F) for F in sorted(set(frames))},
                   "tiles": tiles, "plan_setup_s": plan_s},
        "batched_graphs": res["graph"], "batched_no_graphs": res["nograph"], "plain_one_call_per_window": res["plain"],
        "speedup_vs_plain": res["graph"]["value"] / res["plain"]["value"],
        "identical_words_all_modes": bool(same),
        "differing_windows": differ[:12],
        "batcher_stats": st,
    }
    return line


def run_serving(args, rank, world, local):
    """Poisson arrivals of 10 s vital-sign windows from --users devices, each
    with its own key set, through the serving loop (continuous batching over
    users, keys resident under a budget and reloaded on demand), one phase
    per offered load.  Latency = submit -> output in host memory."""
    import threading

    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    params = M.vital_params()
    ctx = M.Context(params, device=local)
    n = 1 << params.log_n
    g = synth.rng(5000 + rank)
    plan = ctx.plan(M.vital_config())
    rots = plan.rotations()
    n_in, _, lv = plan.io()
    out_words = sum(2 * (l + 1) * n for l in lv)
    qp = params.primes_q + params.primes_p

    def key_words():
        return torch.from_numpy(np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n)
                                                                          for _ in range(2)])
                                                                for _ in range(params.dnum)])).view(np.int64)).pin_memory()

    # one pinned copy of key words serves every simulated device (reloads read it)
    relin = key_words()
    gal = {r: key_words() for r in rots}
    key_set = (1 + len(rots)) * relin.numel() * 8
    budget = int(args.key_budget_gib * 2**30)
    srv = ctx.server(M.vital_config(), max_batch=args.batch, streams=2, key_budget_bytes=budget)
    for u in range(args.users):
        srv.add_user(u, relin, gal)
    nbuf = 8
    ins = [torch.from_numpy(synth.uniform_ciphertexts(8000 + i, params.primes_q, n, n_in).reshape(-1)
                            .view(np.int64)).pin_memory() for i in range(nbuf)]
    outs = [torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(1024)]
    draw = np.random.default_rng(77 + rank)
    # warm-up: plan encoding, first key loads, pools
    warm = [srv.submit(int(draw.integers(args.users)), 200, ins[i % nbuf], outs[i]) for i in range(2 * args.batch)]
    for t in warm:
        srv.wait(t)
    phases = []
    ring = 0
    for load in [float(x) for x in args.loads.split(",")]:
        st0 = srv.stats()
        arrivals = np.cumsum(draw.exponential(1.0 / load, size=int(load * args.phase_s * 1.5) + 8))
        arrivals = arrivals[arrivals < args.phase_s]
        tickets = []
        t0 = time.perf_counter()
        for i, at in enumerate(arrivals):
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            u = int(draw.integers(args.users))
            tickets.append(srv.submit(u, 200, ins[i % nbuf], outs[ring % len(outs)]))
            ring += 1
        lat = [srv.wait(t) for t in tickets]
        t_end = time.perf_counter()
        st1 = srv.stats()
        phases.append({
            "offered_windows_per_s": load, "windows": len(tickets),
            "achieved_windows_per_s": len(tickets) / (t_end - t0),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "batches": st1["batches"] - st0["batches"],
            "mean_batch": (st1["completed"] - st0["completed"]) / max(1, st1["batches"] - st0["batches"]),
            "key_loads": st1["key_loads"] - st0["key_loads"],
            "key_evictions": st1["key_evictions"] - st0["key_evictions"],
        })
    st = srv.stats()
    srv.close()
    top = max(phases, key=lambda p: p["achieved_windows_per_s"])
    line = {
        "metric": METRIC, "value": top["achieved_windows_per_s"], "unit": "windows/s", "n_gpus": world,
        "steps": len(phases), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving: Poisson arrivals of 10 s vital-sign windows (N=2^15 chain, 200 frames x 256 "
                               "bins) from %d devices with their own key sets; batches of <= %d windows mixing "
                               "users, 2 stream slots; %.0f GiB key budget (%.2f GiB per key set, so %d of %d "
                               "devices resident); pinned host inputs and outputs"
                               % (args.users, args.batch, args.key_budget_gib, key_set / 2**30,
                                  int(budget // key_set), args.users)},
        "latency_ms": {"p50": top["p50_ms"], "p99": top["p99_ms"], "note": "at the highest achieved load"},
        "phases": phases, "server_stats": st,
    }
    return line


def run_serving_mix(args, rank, world, local):
    """Poisson arrivals from --users devices mixing 10 s vital-sign windows and
    3 s gesture windows (every fourth device is a gesture device): two
    parameter sets on one GPU (vital N=2^15 Delta=2^40, gesture N=2^15
    Delta=2^50), one serving loop each, both running concurrently on their
    own streams; keys resident under a budget per server.  Latency = submit ->
    output in host memory, per window kind."""
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    g = synth.rng(5100 + rank)
    kinds = {}
    for name, params, cfg, budget_gib, max_batch in (
            ("vital", M.vital_params(), M.vital_config(), args.key_budget_gib, args.batch),
            ("gesture", M.gesture_params(), M.gesture_config(), 16.0, 4)):
        ctx = M.Context(params, device=local)
        n = 1 << params.log_n
        plan = ctx.plan(cfg)
        rots = plan.rotations()
        n_in, _, lv = plan.io()
        qp = params.primes_q + params.primes_p

        def key_words():
            return torch.from_numpy(np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n)
                                                                              for _ in range(2)])
                                                                    for _ in range(params.dnum)])).view(np.int64)).pin_memory()

        relin = key_words()
        gal = {r: key_words() for r in rots}
        srv = ctx.server(cfg, max_batch=max_batch, streams=2, key_budget_bytes=int(budget_gib * 2**30),
                         batch_wait_us=20000)
        if name == "gesture":
            for l, W in enumerate(gesture_random_mats(GestureShape, 13)):
                srv.set_fc_layer(l, W)
        nbuf = 4
        ins = [torch.from_numpy(synth.uniform_ciphertexts(8100 + 10 * len(kinds) + i, params.primes_q, n, n_in)
                                .reshape(-1).view(np.int64)).pin_memory() for i in range(nbuf)]
        out_words = sum(2 * (l + 1) * n for l in lv)
        outs = [torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(256)]
        kinds[name] = dict(ctx=ctx, srv=srv, ins=ins, outs=outs, relin=relin, gal=gal,
                           frames=200 if name == "vital" else 60,
                           key_set=(1 + len(rots)) * relin.numel() * 8, budget_gib=budget_gib, ring=0)
    devices = [("gesture" if u % 4 == 0 else "vital") for u in range(args.users)]
    for u, kname in enumerate(devices):
        k = kinds[kname]
        k["srv"].add_user(u, k["relin"], k["gal"])

    def submit(u):
        k = kinds[devices[u]]
        t = k["srv"].submit(u, k["frames"], k["ins"][k["ring"] % len(k["ins"])], k["outs"][k["ring"] % len(k["outs"])])
        k["ring"] += 1
        return devices[u], t

    draw = np.random.default_rng(78 + rank)
    warm = [submit(u) for u in list(range(min(8, args.users))) * 2]   # plans, first key loads, pools
    for kname, t in warm:
        kinds[kname]["srv"].wait(t)
    phases = []
    for load in [float(x) for x in args.loads.split(",")]:
        st0 = {kn: k["srv"].stats() for kn, k in kinds.items()}
        arrivals = np.cumsum(draw.exponential(1.0 / load, size=int(load * args.phase_s * 1.5) + 8))
        arrivals = arrivals[arrivals < args.phase_s]
        tickets = []
        t0 = time.perf_counter()
        for at in arrivals:
            dt = at - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            tickets.append(submit(int(draw.integers(args.users))))
        lat = {"vital": [], "gesture": []}
        for kname, t in tickets:
            lat[kname].append(kinds[kname]["srv"].wait(t))
        t_end = time.perf_counter()
        st1 = {kn: k["srv"].stats() for kn, k in kinds.items()}
        ph = {"offered_windows_per_s": load, "windows": len(tickets),
              "achieved_windows_per_s": len(tickets) / (t_end - t0)}
        for kname in kinds:
            L = lat[kname]
            b = st1[kname]["batches"] - st0[kname]["batches"]
            ph[kname] = {"windows": len(L), "p50_ms": float(np.percentile(L, 50)) if L else None,
                         "p99_ms": float(np.percentile(L, 99)) if L else None, "batches": b,
                         "mean_batch": (st1[kname]["completed"] - st0[kname]["completed"]) / max(1, b),
                         "key_loads": st1[kname]["key_loads"] - st0[kname]["key_loads"]}
        phases.append(ph)
    stats = {kn: k["srv"].stats() for kn, k in kinds.items()}
    for k in kinds.values():
        k["srv"].close()
    top = max(phases, key=lambda p: p["achieved_windows_per_s"])
    all_lat_p99 = max(top[kn]["p99_ms"] or 0.0 for kn in kinds)
    return {
        "metric": METRIC, "value": top["achieved_windows_per_s"], "unit": "windows/s", "n_gpus": world,
        "steps": len(phases), "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "serving mix: Poisson arrivals from %d devices (3 of 4 send 10 s vital-sign windows, "
                               "N=2^15 Delta=2^40 chain; 1 of 4 sends 3 s gesture windows, N=2^15 Delta=2^50 "
                               "chain), own key sets; one serving loop per parameter set on one GPU, 2 stream "
                               "slots each; key budgets %.0f / %.0f GiB (%.2f / %.2f GiB per key set)"
                               % (args.users, kinds["vital"]["budget_gib"], kinds["gesture"]["budget_gib"],
                                  kinds["vital"]["key_set"] / 2**30, kinds["gesture"]["key_set"] / 2**30)},
        "latency_ms": {"p99_worst_kind": all_lat_p99, "vital_p50": top["vital"]["p50_ms"],
                       "vital_p99": top["vital"]["p99_ms"], "gesture_p50": top["gesture"]["p50_ms"],
                       "gesture_p99": top["gesture"]["p99_ms"], "note": "at the highest achieved load"},
        "phases": phases, "server_stats": stats,
    }


def run_ntt_ablation(args, rank, world, local):
    """Word-size ablation: the batched negacyclic NTT (forward + inverse) of B
    RNS polynomials at N = 2^15, 64-bit words (the chains' primes) against
    32-bit words (30-bit primes) for the same modulus size: the vital chain's
    Q (500 bits: 12 x 64-bit limbs, 17 x 32-bit) and its key-switching QP
    (740 bits: 16 limbs, 25 limbs).  Device-resident rows, CUDA events."""
    import torch

    import paper_2603_22437_b300 as M

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.vital_params()
    ctx = M.Context(params, device=local)
    log_n, n = params.log_n, 1 << params.log_n
    B = args.batch
    g = np.random.default_rng(3)
    stream = torch.cuda.Stream(device=dev)
    peak64, peak32 = ctx.butterfly_peak()
    reps = max(3, args.steps)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {}
    for name, limbs64, limbs32 in (("Q of the vital chain (500 bits)", 12, 17), ("QP of its key switch (740 bits)", 16, 25)):
        bits64 = sum(np.log2(float(q)) for q in (params.primes_q + params.primes_p)[:limbs64])
        primes32 = M.ntt32_primes(log_n, 30, limbs32)
        bits32 = sum(np.log2(float(q)) for q in primes32)
        # 64-bit: the evaluator's batched transform over Q primes (the QP case uses all Q rows plus
        # the first P rows' worth of extra Q-prime rows: the work per row is the same)
        nl = min(limbs64, len(params.primes_q))
        blocks = B * limbs64 // nl
        x64 = torch.from_numpy(np.stack([g.integers(0, params.primes_q[i % nl], n, dtype=np.uint64)
                                         for i in range(blocks * nl)]).view(np.int64)).to(dev)
        ms64 = timed(lambda: (ctx.ntt_batch(x64, blocks, nl, False, stream), ctx.ntt_batch(x64, blocks, nl, True, stream)))
        nt = M.Ntt32(log_n, primes32, device=local)
        x32 = torch.from_numpy(np.stack([g.integers(0, primes32[i % limbs32], n, dtype=np.uint32)
                                         for i in range(B * limbs32)]).view(np.int32)).to(dev)
        ms32 = timed(lambda: (nt.run(x32, False, stream), nt.run(x32, True, stream)))
        nt.close()
        bf64 = 2 * blocks * nl * (n // 2) * log_n
        bf32 = 2 * B * limbs32 * (n // 2) * log_n
        out[name] = {
            "polys": B, "u64": {"limbs": limbs64, "modulus_bits": round(bits64, 1), "ms_fwd_inv": ms64,
                                "Gbutterfly_s": bf64 / ms64 / 1e6, "frac_of_u64_ceiling": bf64 / ms64 / 1e6 / (peak64 / 1e9),
                                "GB_s_hbm": 2 * 2 * blocks * nl * n * 8 / ms64 / 1e6},
            "u32": {"limbs": limbs32, "modulus_bits": round(bits32, 1), "ms_fwd_inv": ms32,
                    "Gbutterfly_s": bf32 / ms32 / 1e6, "frac_of_u32_ceiling": bf32 / ms32 / 1e6 / (peak32 / 1e9),
                    "GB_s_hbm": 2 * 2 * B * limbs32 * n * 4 / ms32 / 1e6},
            # modulus bits transformed per ms: rows x mean bits per row / time
            "u32_speedup_per_modulus_bit": (B * bits32 / ms32) / (blocks * nl * (bits64 / limbs64) / ms64),
        }
        del x64, x32
        torch.cuda.empty_cache()
    q500 = out["Q of the vital chain (500 bits)"]
    return {
        "metric": "RNS polynomial NTTs/s (forward + inverse), 64-bit vs 32-bit words at equal modulus",
        "value": B / (q500["u32"]["ms_fwd_inv"] / 1000.0), "unit": "polys/s", "n_gpus": world,
        "steps": reps, "warmup": args.warmup, "ms_per_step": q500["u32"]["ms_fwd_inv"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32 vs u64", "data": "synthetic",
        "config": {"workload": "word-size ablation: batched negacyclic NTT + inverse of %d RNS polynomials at "
                               "N=2^15, 64-bit limbs (the chain's primes) vs 32-bit limbs (30-bit primes) of equal "
                               "modulus size" % B},
        "butterfly_peak_per_s": {"u64": peak64, "u32": peak32}, "ablation": out,
    }


def run_fc(args, rank, world, local):
    """Encrypted inference of the learned polynomial network (three dense
    layers 120 -> 32 -> 16 -> 6 with squares, N = 2^14, depth 5) on synthetic
    gesture features: the network is trained on the GPU in plaintext, folded
    to pure squares, and --batch encrypted feature vectors are classified per
    launch.  Reports inferences/s and the plaintext training accuracy."""
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.fc_params()
    ctx = M.Context(params, device=local)
    n = 1 << params.log_n
    dims = (120, 32, 16, 6)
    X, y = synth.gesture_dataset(0, 6000)
    alpha = float(np.float32(0.1))
    t0 = time.perf_counter()
    w, train_acc = ctx.train_poly_net(X[:5000], y[:5000], dims, alpha=alpha, epochs=20, batch=128, lr=0.05, seed=3)
    train_s = time.perf_counter() - t0
    mats = M.fold_poly_net(dims, alpha, w, 128)
    plan = ctx.plan(M.fc_config(dims))
    for l, W in enumerate(mats):
        plan.set_fc_layer(l, W)
    g = synth.rng(6000 + rank)
    qp = params.primes_q + params.primes_p
    keys = ctx.keys(rank)

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))

    keys.set_relin(key_words())
    for k in plan.rotations():
        keys.set_galois(k, key_words())
    tiles = pick_tiles(ctx, args, args.batch)
    _, _, lv = plan.io()
    B = args.batch
    d_in = [torch.from_numpy(synth.uniform_ciphertexts(500 + i, params.primes_q, n, 1).reshape(-1).view(np.int64))
            .to(dev) for i in range(B)]
    d_out = [torch.empty(2 * (lv[0] + 1) * n, dtype=torch.int64, device=dev) for _ in range(B)]
    stream = torch.cuda.Stream(device=dev)
    for _ in range(args.warmup):
        ctx.eval(plan, keys, d_in, d_out, stream=stream)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    for i in range(args.steps):
        ev[i][0].record(stream)
        ctx.eval(plan, keys, d_in, d_out, stream=stream)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    ms = [a.elapsed_time(b) for a, b in ev]
    test_acc = float(np.mean([np.argmax(cc_fc_forward(mats, x)) == t for x, t in zip(X[5000:], y[5000:])]))
    return {
        "metric": "encrypted polynomial-network inferences/s", "value": job_throughput(world, B * args.steps,
                                                                                      sum(ms) / 1000.0),
        "unit": "inferences/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.mean(ms)), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": {"workload": "learned polynomial network 120 -> 32 -> 16 -> 6 (dense layers, square "
                               "activations) on synthetic 6-class gesture features, CKKS N=2^14, depth 5, "
                               "%d encrypted feature vectors per launch" % B, "tiles": tiles},
        "plaintext_training": {"train_accuracy": train_acc, "test_accuracy": test_acc, "seconds": train_s,
                               "samples": 5000, "epochs": 20},
    }


def run_per_frame(args, rank, world, local):
    """The vital chain with per-frame packing (the paper's slow baseline: one
    ciphertext per frame and part, 4F = 800 input ciphertexts per window)
    against batched packing (16 per window) on the same windows count B,
    same formulas and outputs."""
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    params = M.vital_params()
    ctx = M.Context(params, device=local)
    n = 1 << params.log_n
    g = synth.rng(7100 + rank)
    qp = params.primes_q + params.primes_p
    plans = {"per_frame": ctx.plan(M.vital_config(per_frame=True)), "batched": ctx.plan(M.vital_config())}
    for p in plans.values():
        p.encode_consts()
    rots = sorted(set(plans["per_frame"].rotations()) | set(plans["batched"].rotations()))
    keys = ctx.keys(rank)

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))

    keys.set_relin(key_words())
    for k in rots:
        keys.set_galois(k, key_words())
    B = args.batch
    tiles = pick_tiles(ctx, args, B)
    stream = torch.cuda.Stream(device=dev)
    res = {}
    for name, plan in plans.items():
        n_in, _, lv = plan.io()
        host = synth.uniform_ciphertexts(7200, params.primes_q, n, n_in).reshape(-1).view(np.int64)
        one = torch.from_numpy(host).to(dev)
        d_in = [one.clone() for _ in range(B)]
        del one
        d_out = [torch.empty(sum(2 * (l + 1) * n for l in lv), dtype=torch.int64, device=dev) for _ in range(B)]
        for _ in range(max(1, args.warmup)):
            ctx.eval(plan, keys, d_in, d_out, stream=stream, vital=True)
        torch.cuda.synchronize()
        l0 = ctx.launch_count()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for i in range(args.steps):
            ev[i][0].record(stream)
            ctx.eval(plan, keys, d_in, d_out, stream=stream, vital=True)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        res[name] = {"value": job_throughput(world, B * args.steps, sum(ms) / 1000.0), "ms_per_step": float(np.mean(ms)),
                     "input_ciphertexts_per_window": n_in, "launches_per_step": (ctx.launch_count() - l0) // args.steps}
        del d_in, d_out
        torch.cuda.empty_cache()
    return {
        "metric": METRIC, "value": res["per_frame"]["value"], "unit": "windows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": res["per_frame"]["ms_per_step"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": "vital-sign chain with per-frame packing (one ciphertext per frame and part, "
                               "200 frames x 256 bins, 800 input cts per window) against batched packing, "
                               "N=2^15, B=%d windows per launch" % B, "tiles": tiles},
        "per_frame": res["per_frame"], "batched": res["batched"],
        "batched_over_per_frame": res["batched"]["value"] / res["per_frame"]["value"],
    }


GESTURE_WORKLOAD = ("gesture chain (K3 Doppler DFT, K1, K6 notch, soft power gamma=4, weighting, frame sum, "
                    "FC1^2, FC2^2, FC3; depth 11), CKKS N=2^15, Q=60+11x50 bits, P=4x60 bits, dnum=3, "
                    "60 frames x 4 antennas x 64 bins x 32 chirps per 3 s window, 60 input cts")


class GestureShape:
    """The gesture network's shape (the sizes of the library's default
    gesture_config)."""
    antennas, bins, chirps, fc_dims, width = 4, 64, 32, (31, 16, 6), 32
    ard = 4 * 64 * 32


def run_gesture(args, rank, world, local):
    """The gesture chain on B windows per step (every ciphertext pair of every
    window in each launch): windows/s, e2e through mmfhe_eval with pinned host
    buffers, per-kernel roofline, clocks."""
    import torch

    import paper_2603_22437_b300 as M
    import synth

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    learned = args.learned is not None
    coef = (1.0, args.learned) if learned else None
    params = M.gesture_params(learned=learned)
    ctx = M.Context(params, device=local)
    plan = ctx.plan(M.gesture_config(complex_slots=args.complex_slots, feature_coef=coef))
    plan.encode_consts()
    for l, W in enumerate(gesture_random_mats(GestureShape, 11)):
        plan.set_fc_layer(l, W)
    P_q, P_p = params.primes_q, params.primes_p
    n = 1 << params.log_n
    g = synth.rng(7300 + rank)
    qp = P_q + P_p
    keys = ctx.keys(rank)

    def key_words():
        return np.ascontiguousarray(np.stack([np.stack([synth.uniform_residues(g, qp, n) for _ in range(2)])
                                              for _ in range(params.dnum)]))

    relin_w = key_words()
    gal_w = {k: key_words() for k in plan.rotations()}
    keys.set_relin(relin_w)
    for k in plan.rotations():
        keys.set_galois(k, gal_w[k])
    n_in, _, out_levels = plan.io()
    B = args.batch
    tiles = pick_tiles(ctx, args, B)
    in_words = n_in * 2 * len(P_q) * n
    out_words = sum(2 * (l + 1) * n for l in out_levels)
    # one window of uniform ciphertexts, copied to every slot of the batch
    host = synth.uniform_ciphertexts(7400 + rank, P_q, n, n_in).reshape(-1)
    one = torch.from_numpy(host.view(np.int64)).to(dev)
    d_in = [one.clone() for _ in range(B)]
    del one
    d_out = [torch.empty(out_words, dtype=torch.int64, device=dev) for _ in range(B)]
    stream = torch.cuda.Stream(device=dev)

    def step(ins, outs):
        ctx.eval(plan, keys, ins, outs, stream=stream)

    for _ in range(args.warmup):
        step(d_in, d_out)
    torch.cuda.synchronize()
    ctx.mem_peak_reset()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ctx.launch_count()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in range(args.steps):
        ev[i][0].record(stream)
        step(d_in, d_out)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    barrier(world)
    launches = ctx.launch_count() - launches0
    clk = clocks.stop()
    mem = ctx.mem_stats()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    value = job_throughput(world, B * args.steps, sum(step_ms) / 1000.0)
    # e2e: (a) one synchronous mmfhe_eval per step on pinned host buffers (copies in, evaluation,
    # copies out in sequence); (b) the serving API with two stream slots, the next batch's copies
    # under this batch's kernels (the feature stage runs in chunks of whole windows, so two
    # batches' scratch fit beside each other)
    pin_one = torch.from_numpy(host.view(np.int64)).pin_memory()
    pin_in = [pin_one] * B            # the windows of a step share one pinned input (read only)
    pin_out = [torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(B)]
    step(pin_in, pin_out)
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        step(pin_in, pin_out)
    torch.cuda.synchronize()
    e2e_sync = job_throughput(world, B * args.e2e_steps, time.perf_counter() - t0)
    gcfg = M.gesture_config(complex_slots=args.complex_slots, feature_coef=coef)
    srv = ctx.server(gcfg, max_batch=B, streams=2, batch_wait_us=20000)
    for l, W in enumerate(gesture_random_mats(GestureShape, 11)):
        srv.set_fc_layer(l, W)
    srv.add_user(rank, relin_w, gal_w)
    e2e_steps = max(4, args.e2e_steps)
    outs_ring = [[torch.empty(out_words, dtype=torch.int64).pin_memory() for _ in range(B)] for _ in range(2)]
    for w in range(B):   # warm-up: the server's plan, key upload and pools
        srv.submit(rank, gcfg.frames, pin_in[w], outs_ring[0][w])
    srv.drain()
    barrier(world)
    t0 = time.perf_counter()
    for s_ in range(e2e_steps):
        for w in range(B):
            srv.submit(rank, gcfg.frames, pin_in[w], outs_ring[s_ % 2][w])
    srv.drain()
    e2e_pipe_s = time.perf_counter() - t0
    srv_stats = srv.stats()
    srv.close()
    if srv_stats["failed"] or srv_stats["completed"] != srv_stats["submitted"]:
        raise RuntimeError("gesture serving e2e: %d of %d windows failed" % (srv_stats["failed"], srv_stats["submitted"]))
    e2e = {"value": job_throughput(world, B * e2e_steps, e2e_pipe_s), "unit": "windows/s",
           "h2d_bytes_per_step": B * in_words * 8, "d2h_bytes_per_step": B * out_words * 8,
           "api": "mmfhe_server (2 stream slots, batches of %d filled within 20 ms, copies overlap the previous "
                  "batch's kernels)" % B,
           "mean_batch": srv_stats["mean_batch"],
           "synchronous_mmfhe_eval": {"value": e2e_sync, "unit": "windows/s"}}
    mem_srv = ctx.mem_stats()
    ctx.profile(True)
    step(d_in, d_out)
    torch.cuda.synchronize()
    prof = ctx.profile()
    ctx.profile(False)
    bf64_peak, bf32_peak = ctx.butterfly_peak()
    roofline = roofline_of(prof, bf64_peak, bf32_peak, B, ctx.mac_peak())
    roofline["traffic"] = ncu_traffic(roofline["kernel"], B, "gesture")
    if roofline["traffic"] is not None:
        roofline["traffic_source"] = "profiles/ncu_traffic.json (gesture capture, scaled by the batch)"
    return {
        "metric": "encrypted gesture windows/s", "value": value, "unit": "windows/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": GESTURE_WORKLOAD + (", complex-slot packing (Re + i Im in one slot, 30 input cts)"
                                                   if args.complex_slots else "")
                   + (", learned feature map p + %g p^2 (depth 9, Q = 60 + 9 x 50 bits) in place of p (p^2)^2"
                      % args.learned if learned else ""),
                   "batch_windows": B, "windows_per_step_all_gpus": world * B,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (%d MiB of ciphertexts per step)" % (B * in_words * 8 >> 20),
                   "weights": "random-init FC weights of the network's shape", "tiles": tiles},
        "latency_ms": {"p50": srv_stats["p50_ms"], "p99": srv_stats["p99_ms"],
                       "note": "per window, submit to output written, through mmfhe_server in the e2e run "
                               "(%d windows)" % (B * e2e_steps),
                       "step_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))}},
        "paper_context": "5.76 s per 3 s gesture window on one RTX 3090 Ti (FIDESlib), batched packing",
        "e2e": e2e, "gpu_launches": launches, "roofline": roofline, "clocks": clk, "wall_s_timed": wall,
        "memory": dict(memory_line(mem, B, "7.5 GB peak cloud GPU memory per batched gesture window (paper Table "
                                           "5, RTX 3090 Ti)"),
                       peak_with_two_serving_slots_gib=mem_srv["peak_bytes"] / 2.0 ** 30),
    }


def cc_fc_forward(mats, x):
    """FP64 forward of the folded network (the labels encrypted inference must reproduce)."""
    v = np.zeros(128)
    v[: len(x)] = x
    v[127] = 1.0
    for l, W in enumerate(mats):
        v = W @ v
        if l < len(mats) - 1:
            v = v * v
    return v[:6]


def main():
    args = parse()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload in ("batching", "serving", "serving-mix", "fc", "per-frame", "ntt-ablation"):
        line = {"batching": run_batching, "serving": run_serving, "serving-mix": run_serving_mix, "fc": run_fc,
                "per-frame": run_per_frame, "ntt-ablation": run_ntt_ablation}[args.workload](args, rank, world, local)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    if args.workload == "gesture":
        line = run_gesture(args, rank, world, local)
        if rank == 0 and world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline("gesture", args.cpu_sample_s or 20.0)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    line = run_mine(args, rank, world, local)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and not args.launch_list:
        line["cpu_baseline"] = cpu_baseline("vital", args.cpu_sample_s)
    if rank == 0:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
