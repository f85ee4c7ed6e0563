"""Benchmark: MLUPS of the reduced polyatomic ES-BGK lattice-Boltzmann step on
GB300, with the HBM roofline of the dominant kernel and the FP64 oracle timed
on the host cores as a baseline (on every core, one independent box per
process, and on one thread).

Workload: 3-D periodic decaying wave field on a 256^3 grid of each BCC
sublattice (2 x 256^3 = 33,554,432 points), FP32, uniform rho = 1,
theta = theta0 plus 8 seeded random Fourier modes (amplitude 1e-3 in rho, u,
theta), diatomic gas (gamma = 7/5), nu = 0.02, eta_B/eta = 0.6, Pr = 0.71, b = 0.
A step is one pass of the whole hot path: pull-stream + collide + rotational
exchange, MacCormack advection and FTCS diffusion of E_R. The population
arrays (2 x 11 GB) are far larger than L2, so no L2 flush is needed.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl rpk|reference]
Under torchrun (N > 1) every rank runs its own lattice (independent replicas,
weak scaling, no collective in the data path); rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import rpk_inputs as I  # noqa: E402

METRIC = "MLUPS & HBM GB/s vs peak; surrogate speedup vs plain LBM at <=1% L1 err"
THETA0 = 0.2948964908710633
GAS = dict(gamma=1.4, nu=0.02, lam=0.6, Pr=0.71, b=0.0)
STORE_BYTES = {"f64": 8, "f32": 4, "f16dev": 2, "bf16dev": 2}
FALLBACK_HBM_GBS = 6800.0
FALLBACK_BF16_TFLOPS = 1900.0  # burst; about 1700 sustained


def algorithmic_bytes_per_point(prec, rot_mode="conservative"):
    """Bytes one point must move per step (rows a1-a8 of the hot path):
    41 populations read + 41 written, plus the moment/rotational fields
    (read rho, u, theta, E_R: 24 B; write 24 B) in the field precision."""
    sb = STORE_BYTES[prec]
    fb = 8 if prec == "f64" else 4
    return {"step": 41 * 2 * sb + 12 * fb,
            # collide kernel alone: populations, e in, and e*, rho, u (3), kappa out
            # (the paper's theta_R solver also writes theta_T for its last half step)
            "collide": 41 * 2 * sb + (8 if rot_mode == "paper" else 7) * fb}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for k in ("hbm_gbs", "hbm_copy_gbs", "hbm_GBs"):
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def load_bf16_peak(sustained=False):
    """Dense BF16 tensor peak in TFLOP/s: the measured cuBLAS figure if the
    peaks file holds one, else the fallback."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    keys = ("bf16_tflops_sustained",) if sustained else ("bf16_tflops",)
    try:
        with open(path) as f:
            d = json.load(f)
        for k in keys:
            if k in d:
                return float(d[k]), "measured"
    except (OSError, ValueError):
        pass
    return (1700.0 if sustained else FALLBACK_BF16_TFLOPS), "fallback"


def ncu_traffic(prec):
    """DRAM bytes per point of the collide kernel from the committed ncu
    summary and the summary's one-line description of the capture, if the
    kernel source has not changed since it was captured; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_collide_%s.txt" % prec)
    csrc = os.path.join(ROOT, "paper_2201_05280_gb300", "csrc")
    srcs = [os.path.join(csrc, f) for f in ("rpk_lattice.cuh", "rpk_vec2.cuh", "rpk_device.cuh",
                                            "rpk_pair.cuh", "rpk_collide.cuh")]
    try:
        kv = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                kv[k.strip()] = v.strip()
        h = hashlib.sha256()
        for src in srcs:
            with open(src, "rb") as f:
                h.update(f.read())
        sha = h.hexdigest()
        if kv.get("kernel_source_sha256") != sha:
            return None
        return float(kv["dram_bytes_per_point"]), kv.get("capture", "")
    except (OSError, KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for name, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def make_fields(n, seed=I.SEED, workload="waves"):
    if workload == "tgv":
        return I.taylor_green(n, THETA0, TGV_MA * np.sqrt(GAS["gamma"] * THETA0))
    f, _ = I.fourier_modes(n, n, n, THETA0, nmodes=8, amp=1e-3, seed=seed)
    return f


TGV_MA, TGV_RE = 0.3, 1600.0


def gas_for(workload, n):
    """(gamma, nu, lam, Pr, b): the decaying-wave gas, or the Taylor-Green
    vortex at Ma 0.3, Re 1600 on an n^3 box (L = n/(2 pi), eta_B/eta = 0.6)."""
    if workload == "tgv":
        u0 = TGV_MA * np.sqrt(GAS["gamma"] * THETA0)
        return dict(GAS, nu=u0 * (n / (2 * np.pi)) / TGV_RE)
    return dict(GAS)


def relax_params(rpk, gas=GAS):
    eta, etaB, kap = rpk.gas_from_nondim(gas["gamma"], gas["nu"], gas["lam"], gas["Pr"])
    return rpk.map_gas(gas["gamma"], eta, etaB, kap, gas["b"])


def _oracle_state(n):
    """The FP64 oracle, as it stands, initialised on an n^3 box of the workload."""
    import oracle as O
    from oracle import params as PM
    eta, etaB, kap = PM.gas_from_nondim(GAS["gamma"], GAS["nu"], GAS["lam"], GAS["Pr"])
    d, tau, tau1, b, kr = PM.relax_from_gas(GAS["gamma"], eta, etaB, kap, GAS["b"])
    f = make_fields(n)
    thmax = float(np.max((3 * f["T"] + d * f["R"]) / (3 + d)))
    P = O.make_params(d, tau, tau1, b, kr, 1.0, PM.nsub_for(d, tau, tau1, kr, thmax, 3), 0)
    return O.State(P, n, n, n).init_fields(f["rho"], f["u"], f["T"], f["R"])


def oracle_mlups(n, steps, warmup=1):
    """The oracle on one host thread: MLUPS and seconds on an n^3 box."""
    S = _oracle_state(n)
    if warmup:
        S.step(warmup)
    t = time.perf_counter()
    S.step(steps)
    dt = time.perf_counter() - t
    return S.npts * steps / dt / 1e6, dt


def _oracle_proc(n, steps, warmup, barrier, q):
    S = _oracle_state(n)
    if warmup:
        S.step(warmup)
    barrier.wait(timeout=600)
    t = time.perf_counter()
    S.step(steps)
    q.put((S.npts * steps, time.perf_counter() - t))


def oracle_mlups_allcore(n, steps, warmup=1, procs=None):
    """The same oracle on every host core: one independent n^3 box per process
    (spawned, so no process inherits a CUDA context), timed from a common
    barrier; MLUPS = all points x steps / the slowest process's time.
    Returns (MLUPS, seconds, processes)."""
    import multiprocessing as mp
    import oracle as O
    O.build()  # once, before the processes load it
    procs = procs or len(os.sched_getaffinity(0))
    ctx = mp.get_context("spawn")
    barrier, q = ctx.Barrier(procs), ctx.Queue()
    ps = [ctx.Process(target=_oracle_proc, args=(n, steps, warmup, barrier, q)) for _ in range(procs)]
    for p in ps:
        p.start()
    try:
        res = [q.get(timeout=1200) for _ in ps]
    finally:
        for p in ps:
            p.join(timeout=60)
            if p.is_alive():
                p.terminate()
    work = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    return work / dt / 1e6, dt, procs


def run_reference(args, rank):
    if rank != 0:
        return 0
    n = args.ref_n
    value, dt, procs = oracle_mlups_allcore(n, args.steps, args.warmup)
    sample = ("%d independent %d^3 boxes (%d points each), one per host core, x %d steps"
              % (procs, n, 2 * n ** 3, args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "3-D periodic decaying wave field (8 seeded Fourier modes), "
                                   "oracle on %d^3 samples of the 256^3 workload" % n,
                       "grid": [n, n, n], "points": 2 * n ** 3 * procs, "gas": GAS},
            "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def batch_line(rpk, ntubes, diffusion):
    """One graph-captured persistent launch of ntubes tubes of the sweep
    (autotuned): MLUPS, milliseconds and the roofline of the populations'
    traffic (41 x 4 B read and written per point update)."""
    import torch
    specs, f = I.tube_sweep(ntubes, THETA0)
    cs = rpk.sound_speed(GAS["gamma"])
    tubes = []
    for sp in specs:
        nu = sp["kn"] * cs * sp["nx"]
        eta, etaB, kap = rpk.gas_from_nondim(GAS["gamma"], nu, sp["lam"], sp["pr"])
        rr = rpk.map_gas(GAS["gamma"], eta, etaB, kap, 0.0)
        tubes.append({"nx": sp["nx"], "nsteps": sp["nsteps"], "relax": rr, "res": sp["res"]})
    stream = torch.cuda.Stream()
    bt = rpk.Batch(tubes, precision="f32", save_every=32, stream=stream)
    bt.set_diffusion(diffusion)
    bt.init_fields(f["rho"], f["u"], f["T"], f["R"])
    tune = bt.autotune()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    bt.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    bt.close()
    updates = sum(2 * t["nx"] * t["nsteps"] for t in tubes)
    gbs = updates * 41 * 2 * 4 / (ms * 1e-3) / 1e9
    return {"workload": "%d quasi-1-D shock tubes of the sweep, %s rotational diffusion" % (ntubes, diffusion),
            "value": updates / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms": ms, "autotune": tune,
            "population_gbs": gbs, "frac": gbs / load_peaks()[0], "gpu_launches": 1}


def run_batch(args):
    """Batched shock-tube sweep: --tubes quasi-1-D tubes, lengths U[500, 4000],
    pressure ratio U[2, 20] (right state on the left isentrope), Kn log-U[1e-3,
    1e-1], eta_B/eta U[0.3, 2], Pr 0.71, each run for 0.35 L/c_s steps, moments
    saved every 32 steps; one persistent, graph-captured launch, configuration
    chosen by the autotuner. Prints one JSON line (not the lattice line)."""
    import torch
    import paper_2201_05280_gb300 as rpk
    from paper_2201_05280_gb300 import build as B
    B.build()
    torch.cuda.set_device(0)
    specs, f = I.tube_sweep(args.tubes, THETA0)
    cs = np.sqrt(GAS["gamma"] * THETA0)
    tubes = []
    for sp in specs:
        nu = sp["kn"] * cs * sp["nx"]
        eta, etaB, kap = rpk.gas_from_nondim(GAS["gamma"], nu, sp["lam"], sp["pr"])
        r = rpk.map_gas(GAS["gamma"], eta, etaB, kap, 0.0)
        tubes.append({"nx": sp["nx"], "nsteps": sp["nsteps"], "relax": r, "res": sp["res"]})
    stream = torch.cuda.Stream()
    bt = rpk.Batch(tubes, precision="f32", save_every=32, stream=stream)
    bt.set_diffusion(args.diffusion)
    bt.init_fields(f["rho"], f["u"], f["T"], f["R"])
    tune = bt.autotune()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        bt.run()
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m = bt.read_moments(check=False)
    updates = sum(2 * t["nx"] * t["nsteps"] for t in tubes)
    finite = bool(np.all(np.isfinite(m["rho"])))
    line = {"metric": METRIC, "mode": "batch", "value": updates / (ms * 1e-3) / 1e6,
            "unit": "MLUPS", "n_gpus": 1, "ms": ms, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "batched sweep: %d quasi-1-D shock tubes" % args.tubes,
                       "points": int(sum(2 * t["nx"] for t in tubes)),
                       "point_updates": int(updates), "save_every": 32,
                       "lengths": [500, 4000], "pressure_ratio": [2, 20], "kn": [1e-3, 1e-1],
                       "eta_B_over_eta": [0.3, 2.0], "rotational_diffusion": args.diffusion},
            "autotune": tune, "gpu_launches": 1, "all_finite": finite,
            "clocks": clk.summary()}
    # populations read once and written once per point update; the tube's
    # other fields stay in shared memory for the whole run
    peak, src = load_peaks()
    gbs = updates * 41 * 2 * 4 / (ms * 1e-3) / 1e9
    line["roofline"] = {"bound": "hbm", "kernel": "k_batch (one persistent launch)",
                        "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "peak_source": src, "algorithmic_bytes_per_point_update": 328,
                        "traffic": None}
    print(json.dumps(line))
    bt.close()
    return 0


def run_surrogate(args):
    """Learned surrogate against the plain batched LBM. Trains the network on
    the LBM's snapshots of --train-tubes tubes of the sweep (the library's own
    forward, backward and Adam kernels), then advances --tubes held-out tubes
    (another seed of the same sweep) twice: by the plain batched LBM (one
    graph-captured persistent launch) and by the surrogate rollout with its
    LBM spot checks and hand-over. Reports the wall-clock ratio and the
    relative L1 density error of every tube against the plain LBM. Prints one
    JSON line (not the lattice line)."""
    import torch
    import paper_2201_05280_gb300 as rpk
    from paper_2201_05280_gb300 import build as B
    from paper_2201_05280_gb300 import surrogate as SG
    B.build()
    torch.cuda.set_device(0)
    t0 = time.time()
    specs, f = I.tube_sweep(args.train_tubes, THETA0, seed=args.train_seed)
    tubes, cond = SG.make_tubes(specs, f, THETA0)
    data = SG.TrainingSet(tubes, cond, f, diffusion=args.diffusion)
    torch.cuda.synchronize()
    t_data = time.time() - t0
    n_pairs = len(data)
    cfg = SG.default_config(THETA0)
    net = rpk.Net(SG.CIN, SG.COUT, args.width, args.blocks, seed=args.train_seed)
    t0 = time.time()
    hist = SG.train(net, cfg, data, args.train_steps, batch=args.batch, crop_len=args.crop,
                    noise=[float(v) for v in args.noise.split(",")], seed=args.train_seed)
    torch.cuda.synchronize()
    t_train = time.time() - t0
    del data
    torch.cuda.empty_cache()

    specs, f = I.tube_sweep(args.tubes, THETA0, seed=args.eval_seed)
    etubes, econd = SG.make_tubes(specs, f, THETA0)
    blk0 = SG.initial_blocks(etubes, f)
    bt = rpk.Batch(etubes, precision="f32", save_every=1 << 30)
    bt.set_diffusion(args.diffusion)
    bt.init_fields(f["rho"], f["u"], f["T"], f["R"])
    tune = bt.autotune()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    bt.init_device(blk0).run()  # captures the graph
    torch.cuda.synchronize()
    bt.init_device(blk0)
    with ClockSampler(0) as clk_lbm:
        e0.record()
        bt.run()
        e1.record()
        torch.cuda.synchronize()
    lbm_ms = e0.elapsed_time(e1)
    ref = bt.moments_device()
    torch.cuda.synchronize()
    ref = ref.cpu().numpy()
    offs = bt.block_offsets
    bt.close()
    # the network alone: one ragged forward pass over every held-out tube
    # (padded with its reservoirs), timed with CUDA events on the network's stream
    seqs, out = [], 0
    for o, t, c in zip(offs, etubes, econd):
        L = (2 * t["nx"] + 2 * cfg.pad + 3) // 4 * 4
        seqs.append(dict(src=int(o), out=out, nx=t["nx"], len=L, res=SG.reservoirs(t), cond=c))
        out += L
    xin, _, _ = rpk.sur_pack(cfg, blk0, seqs)
    lens = [d["len"] for d in seqs]
    for _ in range(3):
        net.forward_ragged(xin, lens)
    torch.cuda.synchronize()
    fw = []
    for _ in range(5):
        e0.record()
        net.forward_ragged(xin, lens)
        e1.record()
        torch.cuda.synchronize()
        fw.append(e0.elapsed_time(e1))
    fwd_ms = statistics.median(fw)
    coarse = sum(lens) // 4
    w = args.width
    flop_pos = 2 * (4 * SG.CIN * w + args.blocks * 2 * 5 * w * w + w * 4 * SG.COUT)
    fwd_tflops = coarse * flop_pos / (fwd_ms * 1e-3) / 1e12
    peak = load_bf16_peak()
    ccfg = SG.default_config(THETA0, spot_every=args.spot_every, l1_tol=args.l1_tol,
                             anchor=int(args.anchor), lbm_threads=tune["threads"],
                             lbm_ctas_per_sm=tune["ctas_per_sm"],
                             lbm_diffusion=1 if args.diffusion == "implicit" else 0)
    R = rpk.Rollout(net, ccfg, etubes, econd)
    st = blk0.clone()
    R.run(st)  # warm-up (graph capture of its LBM, workspaces)
    st = blk0.clone()
    torch.cuda.synchronize()
    with ClockSampler(0) as clk_sur:
        t1 = time.perf_counter()
        e0.record()
        res = R.run(st)
        e1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t1
    sur_ms = e0.elapsed_time(e1)
    got = st.cpu().numpy()
    l1 = np.array([np.abs(got[o:o + 2 * t["nx"]] - ref[o:o + 2 * t["nx"]]).sum() /
                   np.abs(ref[o:o + 2 * t["nx"]]).sum() for o, t in zip(offs, etubes)])
    handed = res["fail_step"] >= 0
    windows_total = int(sum(t["nsteps"] // cfg.jump for t in etubes))
    line = {"metric": METRIC, "mode": "surrogate", "value": lbm_ms / sur_ms, "unit": "x (plain LBM ms / surrogate ms)",
            "n_gpus": 1, "higher_is_better": True, "dtype": "bf16 network, f32 LBM", "data": "synthetic",
            "config": {"workload": "%d held-out quasi-1-D shock tubes of the sweep (seed %d)" % (args.tubes, args.eval_seed),
                       "train_tubes": args.train_tubes, "train_pairs": n_pairs, "train_crops_seen": int(args.train_steps * args.batch),
                       "jump": cfg.jump, "spot_every": args.spot_every, "l1_tol": args.l1_tol,
                       "anchor": int(args.anchor), "rotational_diffusion": args.diffusion,
                       "network": {"width": args.width, "blocks": args.blocks,
                                                               "params": net.num_params}},
            "lbm_ms": lbm_ms, "surrogate_ms": sur_ms, "surrogate_wall_s": wall,
            "surrogate_parts_ms": dict(zip(("network", "spot_checks", "final_lbm", "reruns"), res["ms"].tolist())),
            "l1": {"mean": float(l1.mean()), "p90": float(np.percentile(l1, 90)), "max": float(l1.max()),
                   "frac_le_1pct": float((l1 <= 0.01).mean())},
            "roofline": {"bound": "tensor", "kernel": "network forward (k_conv_tc + k_conv)",
                         "achieved": fwd_tflops, "peak": peak[0], "unit": "TFLOP/s",
                         "frac": fwd_tflops / peak[0], "peak_source": peak[1],
                         "flop_per_coarse_position": flop_pos, "positions": coarse,
                         "forward_ms": fwd_ms, "traffic": None},
            "tubes_handed_to_lbm": int(handed.sum()), "network_windows": int(res["windows"].sum()),
            "windows_total": windows_total, "spot_checks": int(res["checks"].sum()),
            "training": {"data_s": t_data, "train_s": t_train, "steps": args.train_steps,
                         "loss_first": float(np.mean(hist[:50])) if hist else None,
                         "loss_last": float(np.mean(hist[-200:])) if hist else None},
            "autotune": tune, "clocks": {"lbm": clk_lbm.summary(), "surrogate": clk_sur.summary()}}
    print(json.dumps(line))
    R.close()
    return 0


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over all ranks (x itself without a process group):
    the job's time is its slowest rank's."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mlups(world, npts, steps, ms):
    """Whole-job throughput of `world` replicas of npts points each over `steps`
    steps in `ms` milliseconds (the slowest rank's)."""
    return world * npts * steps / (ms * 1e-3) / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="rpk", choices=["rpk", "reference"])
    ap.add_argument("--n", type=int, default=256, help="cells per axis of each sublattice")
    ap.add_argument("--precision", default="f32", choices=list(STORE_BYTES))
    ap.add_argument("--ref-n", type=int, default=16, help="oracle sample box for --impl reference")
    ap.add_argument("--cpu-n", type=int, default=24, help="oracle sample box for cpu_baseline")
    ap.add_argument("--cpu-steps", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the 16-bit storage runs and the batched sweep added to the line")
    ap.add_argument("--extra-tubes", type=int, default=1024,
                    help="tubes of the batched sweep added to the lattice line")
    ap.add_argument("--mode", default="lattice", choices=["lattice", "batch", "surrogate"],
                    help="lattice: the 3-D step (default); batch: the shock-tube sweep; "
                         "surrogate: learned surrogate vs plain batched LBM")
    ap.add_argument("--tubes", type=int, default=None,
                    help="tubes in --mode batch (4096) / held-out tubes in --mode surrogate (512)")
    ap.add_argument("--diffusion", default="ftcs", choices=["ftcs", "implicit"],
                    help="rotational diffusion of the batched tubes: the paper's FTCS "
                         "sub-steps or the backward-Euler variant")
    ap.add_argument("--train-tubes", type=int, default=512)
    ap.add_argument("--train-steps", type=int, default=16000)
    ap.add_argument("--train-seed", type=int, default=1001)
    ap.add_argument("--eval-seed", type=int, default=2002)
    ap.add_argument("--width", type=int, default=128)
    ap.add_argument("--blocks", type=int, default=6)
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--crop", type=int, default=1024)
    ap.add_argument("--noise", default="3e-4,3e-4,1e-4,1e-4")
    ap.add_argument("--spot-every", type=int, default=16)
    ap.add_argument("--l1-tol", type=float, default=1e-2)
    ap.add_argument("--anchor", type=int, default=0)
    ap.add_argument("--workload", default="waves", choices=["waves", "tgv"],
                    help="decaying wave field (default) or Taylor-Green vortex Ma 0.3 Re 1600")
    ap.add_argument("--rot-mode", default="conservative", choices=["conservative", "paper"],
                    help="rotational-energy solver: the conservative form (default) or the "
                         "paper's theta_R solver")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank)
    if args.mode == "batch":
        args.tubes = args.tubes or 4096
        return run_batch(args)
    if args.mode == "surrogate":
        args.tubes = args.tubes or 512
        return run_surrogate(args)

    import torch
    import paper_2201_05280_gb300 as rpk
    from paper_2201_05280_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        B.build()
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    n = args.n
    f = make_fields(n, workload=args.workload)
    gas = gas_for(args.workload, n)
    r = relax_params(rpk, gas)
    stream = torch.cuda.Stream()
    lat = rpk.Lattice(n, n, n, precision=args.precision, stream=stream)
    lat.set_relax(r["delta"], r["tau"], r["tau1"], r["b"], r["k_r"])
    lat.set_rot_mode(args.rot_mode)
    lat.init_fields(f["rho"], f["u"], f["T"], f["R"])
    nsub = lat.info()["nsub"]
    npts = lat.npts

    lat.step(args.warmup)
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev) as clk:
        lat.timing(True)
        e0.record(stream)
        lat.step(args.steps)
        e1.record(stream)
        barrier()
    ktimes = lat.timing_read()
    lat.timing(False)
    ms = max_over_ranks(e0.elapsed_time(e1), dist)
    diag = lat.diagnostics()
    value = job_mlups(world, npts, args.steps, ms)

    # end to end through the public API with pinned host buffers
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in f.items()}
        outs = {k: torch.empty(sz, dtype=torch.float64).pin_memory()
                for k, sz in (("rho", npts), ("u", 3 * npts), ("T", npts), ("R", npts),
                              ("Erot", npts))}
        lat2 = rpk.Lattice(n, n, n, precision=args.precision, stream=stream)
        lat2.set_relax(r["delta"], r["tau"], r["tau1"], r["b"], r["k_r"])
        lat2.set_rot_mode(args.rot_mode)
        lat2.init_fields(pin["rho"], pin["u"], pin["T"], pin["R"])  # warm the staging path
        lat2.step(3)
        lat2.read_moments(outs)
        barrier()
        t0 = time.perf_counter()
        lat2.init_fields(pin["rho"], pin["u"], pin["T"], pin["R"])
        lat2.step(args.steps)
        lat2.read_moments(outs)
        barrier()
        wall = max_over_ranks(time.perf_counter() - t0, dist)
        lat2.close()
        h2d = 6 * npts * 8
        d2h = 7 * npts * 8
        e2e = {"value": world * npts * args.steps / wall / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "note": "per job of K steps: fields uploaded once from pinned host memory, "
                       "moments read back once; bytes per step = job bytes / K"}

    # the same workload with 16-bit deviation storage, and a batched sweep:
    # short runs in the same process, so that the line carries them too
    extras = None
    if not args.no_extras and world == 1:
        extras = {"storage": {}, "batch": None}
        for prec in ("f16dev", "bf16dev"):
            if prec == args.precision:
                continue
            lx = rpk.Lattice(n, n, n, precision=prec, stream=stream)
            lx.set_relax(r["delta"], r["tau"], r["tau1"], r["b"], r["k_r"])
            lx.set_rot_mode(args.rot_mode)
            lx.init_fields(f["rho"], f["u"], f["T"], f["R"])
            lx.step(args.warmup)
            torch.cuda.synchronize()
            e0.record(stream)
            lx.step(args.steps)
            e1.record(stream)
            torch.cuda.synchronize()
            xms = e0.elapsed_time(e1)
            st = lx.diagnostics(check=False)["status"]
            lx.close()
            sb = algorithmic_bytes_per_point(prec)["step"]
            gbs = sb * npts * args.steps / (xms * 1e-3) / 1e9
            extras["storage"][prec] = {"value": job_mlups(1, npts, args.steps, xms), "unit": "MLUPS",
                                       "ms_per_step": xms / args.steps, "step_bytes_per_point": sb,
                                       "step_gbs": gbs, "step_frac": gbs / load_peaks()[0],
                                       "device_status": st}
        torch.cuda.empty_cache()
        extras["batch"] = batch_line(rpk, args.extra_tubes, "implicit")
        torch.cuda.empty_cache()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return 0

    ab = algorithmic_bytes_per_point(args.precision, args.rot_mode)
    peak, peak_src = load_peaks()
    coll_ms, coll_n = ktimes["collide"]
    coll_avg_s = coll_ms / max(coll_n, 1) * 1e-3
    achieved = ab["collide"] * npts / coll_avg_s / 1e9
    # the committed capture is of the conservative form's collide kernel
    traffic = ncu_traffic(args.precision) if args.rot_mode == "conservative" else None
    step_gbs = ab["step"] * npts * args.steps / (ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "k_collide_pair (pull-stream + collide + exchange, two points per thread)"
                if args.n % 2 == 0 else "k_collide (pull-stream + collide + exchange)",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_source": peak_src,
                "algorithmic_bytes_per_point": ab["collide"],
                "traffic": None if traffic is None else traffic[0] * npts,
                "traffic_bytes_per_point": None if traffic is None else traffic[0],
                "traffic_source": None if traffic is None else traffic[1],
                "kernel_ms": {k: v[0] / max(v[1], 1) for k, v in ktimes.items()},
                "kernel_share": {k: v[0] / sum(x[0] for x in ktimes.values())
                                 for k, v in ktimes.items()},
                # the whole step against the same peak, at the algorithmic
                # bytes of one step (populations once each way + the fields)
                "step_algorithmic_bytes_per_point": ab["step"],
                "step_gbs": step_gbs, "step_frac": step_gbs / peak}
    cpu_mlups, cpu_dt = oracle_mlups(args.cpu_n, args.cpu_steps, warmup=1)
    all_mlups, all_dt, procs = oracle_mlups_allcore(args.cpu_n, args.cpu_steps, warmup=1)
    launches = sum(v[1] for v in ktimes.values())
    line = {"metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "f32" else args.precision, "data": "synthetic",
            "config": {"workload": ("3-D periodic %d^3 decaying wave field, %s" % (n, args.precision)
                                    if args.workload == "waves" else
                                    "3-D Taylor-Green vortex %d^3, Ma 0.3, Re 1600, %s" % (n, args.precision)),
                       "grid": [n, n, n], "points": npts, "gas": gas, "nsub": nsub,
                       "rotational_form": args.rot_mode,
                       "l2": "inputs larger than L2 (%.1f GB of populations)" %
                             (2 * 41 * npts * STORE_BYTES[args.precision] / 1e9),
                       "parallelism": "replicas x%d" % world},
            "roofline": roofline,
            "cpu_baseline": {"value": all_mlups, "unit": "MLUPS", "cores": procs, "kind": "oracle",
                             "sample": "%d independent %d^3 boxes (%d points each), one per host "
                                       "core, x %d steps, %.1f s" %
                                       (procs, args.cpu_n, 2 * args.cpu_n ** 3, args.cpu_steps, all_dt),
                             "single_thread": {"value": cpu_mlups, "cores": 1,
                                               "sample": "one %d^3 box x %d steps, %.1f s" %
                                                         (args.cpu_n, args.cpu_steps, cpu_dt)}},
            "e2e": e2e, "gpu_launches": launches, "extras": extras,
            "clocks": clk.summary(),
            "device_status": diag["status"]}
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
