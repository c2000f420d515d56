"""Benchmark: max-null permutation testing, NaivePT and RapidPT, on GB300s.

One step = the whole NaivePT hot path on one batch: pt_prepare (per-voxel
moments, unit-norm centring) + pt_maxnull_naive (split of the data into two
FP16 pieces, labels, fused tensor-core contraction + max-null + exceedance
counts, finalise) for the brain-shaped workload n=100 (50/50), 91x109x91 grid
masked to 231,719 voxels, 10,000 relabellings. Metric: T entries (relabelling
x voxel t statistics) per second. Inputs (X 361 MB, FP16 data pieces 104 MB)
are larger than L2. Steps follow one another on one stream; the only host wait
inside a step is pt_prepare's (it sizes the launches by the voxel counts).

At one GPU the line also carries:
* "precision": each arithmetic path of the fused kernel (FP32 CUDA cores,
  BF16x2 and BF16x3 tensor cores) timed on the same workload, with its errors
  against the FP64 oracle (max-null on the CPU leg's sampled rows, t entries of
  sampled rows of T, thresholds);
* "rapidpt": RapidPT (Alg. 2: training rows, subspace tracking, sampled
  recovery) against NaivePT on the RapidPT workload (n=200, 500,000 voxels,
  100,000 relabellings, r=50, 400 training rows, 0.35% sampling): each method's
  max-null wall time, and RapidPT's accuracy against the exhaustive max-null
  (KL divergence, FWER 0.05/0.01 thresholds, and the same measures between two
  halves of the exhaustive max-null, the estimators' own floor);
* "large": the same comparison on n=400, 600,000 voxels, 100,000 relabellings
  (RapidPT r=100, 800 training rows), with NaivePT checked against the oracle
  on sampled rows;
* "batched" (64 uneven studies in one call), "glm" (two covariates), "anova"
  (one-way F of three groups) and "cluster" (largest cluster of {t >= 3.2}
  per relabelling, the observed map's clusters and their p-values);
* "cpu_baseline": the FP64 oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision bf16x3|bf16x2|fp32] [--no-tune] [--no-rapid] [--no-batched]
                  [--no-glm] [--no-large] [--no-precision] [--no-cpu-baseline] [--quick]

Default K = 500 steps (about 0.7 s of timed work at one GPU, so that several
nvidia-smi clock samples fall inside the timed region).

With N > 1 it runs under torch.distributed.run, one rank per GPU: one study
whose relabellings (N x 10,000 from one PCG32 list) are sharded 10,000 per
rank (weak scaling); every step gathers the maxima and argmax and sums the
exceedance counts over NCCL; value = entries of all ranks / max-over-ranks time.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "T entries/s (perm x voxel t) & max-null wall time, RapidPT vs NaivePT, 1 GB300"
# ncu dram__bytes_read.sum + dram__bytes_write.sum of one tuned launch of the
# fused kernel on brain_n100_v232k, per precision (BF16x3: 160.21 MB read +
# 4.67 MB written; FP16x2: 108.21 MB read + 3.54 MB written); None where no
# capture of the current kernel exists.
TRAFFIC_BYTES = {2: 164.89e6, 3: 111.97e6}
WORKLOAD = "brain_n100_v232k"
# NaivePT arithmetic of the RapidPT-vs-NaivePT and large legs: FP16x2 (two FP16
# pieces of 2^15 Xn), the fastest path that meets the FP32-class tolerances.
NAIVE_PREC = 3
PREC = {"fp32": 0, "bf16x2": 1, "bf16x3": 2, "fp16x2": 3}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, \
            "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms; stop() reports the
    samples taken inside [t0, t1] (the timed region), or all samples, flagged, when
    the region held none."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                self.rows.append((time.time(), f))

    def stop(self, t0=None, t1=None):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        inside = [f for t, f in self.rows if t0 is not None and t0 <= t <= t1]
        rows = inside if inside else [f for _, f in self.rows]
        for f in rows:
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm),
                "window": "timed region" if inside else "whole sampling (no sample fell "
                          "inside the timed region)"}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(Xm_host, n1, perms, seconds_target=15.0, start_rows=1, Xt=None):
    """Time the FP64 oracle on whole relabelling rows (all voxels) of the workload,
    growing the sample until it takes about ``seconds_target``. Returns
    (entries/s, rows, seconds, cores, outputs of the last timed run)."""
    import oracle
    cores = cpu_cores()
    v = Xm_host.shape[1]
    if Xt is None:
        Xt = oracle.voxel_major(Xm_host)
    rows = max(1, start_rows)
    while True:
        sel = perms[:rows]
        t0 = time.perf_counter()
        out = _oracle_rows(Xt, n1, sel, cores)
        dt = time.perf_counter() - t0
        if dt >= seconds_target * 0.5 or rows >= perms.shape[0]:
            return rows * v / dt, rows, dt, cores, out
        grow = max(2, int(seconds_target / max(dt, 1e-3)))
        rows = min(perms.shape[0], rows * grow)


def _oracle_rows(Xt, n1, perms, cores):
    import ctypes
    import oracle
    lib = oracle._load()
    v, n = Xt.shape
    P = perms.shape[0]
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    out = [np.empty(P), np.empty(P, np.int64), np.empty(P), np.empty(v, np.uint32), np.empty(v),
           np.empty(v, np.uint32), np.empty(v)]
    p = lambda a: ctypes.c_void_p(a.ctypes.data)  # noqa: E731
    rc = lib.oracle_naive(p(Xt), n, v, int(n1), p(perms), P, 0, int(cores), 0.0,
                          *[p(a) for a in out])
    assert rc == 0
    return out


def run_reference(args):
    """Reference arm: the FP64 CPU oracle of the same workload on the host cores."""
    ws, rank, _ = dist_env()
    if ws > 1 and rank != 0:
        return
    import torch
    from paper_1703_01506_gb300 import synth
    w = synth.workload(WORKLOAD, device="cpu")
    X, mask = w["X"], w["mask"].bool()
    Xm = X[:, mask].numpy()
    v = Xm.shape[1]
    import oracle
    oracle.build()
    Xt = oracle.voxel_major(Xm)
    cores = cpu_cores()
    # size one step so that the warm-up and timed steps take about 90 s in all
    # (at most 5 s of CPU work per step)
    step_s = max(0.05, min(5.0, 90.0 / max(1, args.steps + args.warmup)))
    rate, rows, dt, _, _ = oracle_sample(Xm, w["n1"], w["perms"], seconds_target=4.0, Xt=Xt)
    step_rows = max(1, int(round(rows * step_s / max(dt, 1e-6))))
    step_rows = min(step_rows, w["perms"].shape[0])
    for i in range(args.warmup):
        _oracle_rows(Xt, w["n1"], w["perms"][:step_rows], cores)
    times = []
    for i in range(args.steps):
        sel = w["perms"][(i * step_rows) % w["P"]:][:step_rows]
        t0 = time.perf_counter()
        _oracle_rows(Xt, w["n1"], sel, cores)
        times.append(time.perf_counter() - t0)
    ms = 1000.0 * sum(times) / len(times)
    value = sel.shape[0] * v / (ms / 1000.0)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "T entries/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD + ": n=100 (50/50), %d voxels, P=10000" % v,
                   "sample": "%d relabellings x all voxels per step" % step_rows},
        "cpu_baseline": {"value": value, "unit": "T entries/s", "cores": cores, "kind": "oracle",
                         "sample": "%d relabelling rows x %d voxels per step" % (step_rows, v)},
        "e2e": {"value": value, "unit": "T entries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def hist_kl(p_samples, q_samples, bins=100):
    """KL(P || Q) of two max-null samples over a common histogram (empty
    bins of Q smoothed by one count): the accuracy summary of the paper's
    Sec. 5.5, computed on the host."""
    lo = float(min(p_samples.min(), q_samples.min()))
    hi = float(max(p_samples.max(), q_samples.max()))
    hp, edges = np.histogram(p_samples, bins=bins, range=(lo, hi))
    hq, _ = np.histogram(q_samples, bins=edges)
    pp = (hp + 1e-12) / hp.sum()
    qq = (hq + 1.0) / (hq + 1.0).sum()
    m = hp > 0
    return float(np.sum(pp[m] * np.log(pp[m] / qq[m])))


def fwer_thr(m, alpha):
    """FWER threshold of a max-null: the c-th largest value, c = floor(alpha P) + 1."""
    srt = np.sort(np.asarray(m, dtype=np.float64))[::-1]
    c = int(np.floor(alpha * srt.size)) + 1
    return float(srt[min(c, srt.size) - 1])


def rapid_vs_naive(dev, B, torch, X, mask, n1, perms, r, ell, eta, passes=1):
    """Each method's wall time from pt_prepare to the max-null vector on one
    workload, RapidPT's phase split, and its accuracy against the exhaustive
    NaivePT max-null (KL, FWER 0.05/0.01 thresholds, resampling risk)."""
    P = perms.shape[0]
    stream = torch.cuda.current_stream(dev)
    mx_naive = torch.empty(P, dtype=torch.float32, device=dev)
    am = torch.empty(P, dtype=torch.int32, device=dev)

    def naive_run():
        c = B.pt_prepare(X, n1, mask, stream=stream)
        B.pt_maxnull_naive_ex(c, perms, B.naive_opts(NAIVE_PREC), mx_naive, am, None)
        B.pt_sync(c)
        v = B.pt_num_valid_voxels(c)
        c.close()
        return v

    opts = B.rapid_opts(train_passes=passes)
    mx_rapid = torch.empty(P, dtype=torch.float32, device=dev)
    phase = {}

    def rapid_run():
        t0 = time.perf_counter()
        c = B.pt_prepare(X, n1, mask, stream=stream)
        V = B.pt_num_valid_voxels(c)
        U = torch.empty((V, r), dtype=torch.float32, device=dev)
        t1 = time.perf_counter()
        info = B.pt_rapid_train(c, perms, ell, r, eta, opts, U, mx_rapid[:ell])
        torch.cuda.synchronize(dev)
        t2 = time.perf_counter()
        B.pt_rapid_recover(c, perms, ell, U, r, eta, info.sigma, info.mu, opts, mx_rapid[ell:])
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        c.close()
        phase.update(prepare_ms=(t1 - t0) * 1e3, train_ms=(t2 - t1) * 1e3,
                     recover_ms=(t3 - t2) * 1e3, sigma=info.sigma, mu=info.mu,
                     train_steps=int(info.train_steps), m_per_perm=int(info.m_per_perm))

    def timed(fn, reps):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        ev0.record(stream)
        for _ in range(reps):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        return ev0.elapsed_time(ev1) / reps

    v = naive_run()
    c = B.pt_prepare(X, n1, mask, stream=stream)
    B.pt_autotune_naive(c, perms, B.naive_opts(NAIVE_PREC))
    c.close()
    naive_ms = timed(naive_run, 3)
    rapid_run()
    rapid_ms = timed(rapid_run, 1)
    # Resampling risk (Sec. 5.5, Eq. 6) of the two methods' voxel decisions at
    # FWER 0.05, from the corrected p-value maps the library computes.
    from paper_1703_01506_gb300 import metrics
    c = B.pt_prepare(X, n1, mask, stream=stream)
    vm = B.pt_num_voxels(c)
    p_naive = torch.empty(vm, dtype=torch.float32, device=dev)
    p_rapid = torch.empty(vm, dtype=torch.float32, device=dev)
    B.pt_fwer_pvalues(c, mx_naive, p_naive)
    B.pt_fwer_pvalues(c, mx_rapid, p_rapid)
    B.pt_sync(c)
    c.close()
    risk = metrics.resampling_risk(p_naive.cpu().numpy(), p_rapid.cpu().numpy(), 0.05)
    a = mx_naive.cpu().numpy().astype(np.float64)
    b = mx_rapid.cpu().numpy().astype(np.float64)
    thr = {}
    for alpha in (0.05, 0.01):
        ta, tb = fwer_thr(a, alpha), fwer_thr(b, alpha)
        thr["fwer%g" % alpha] = {"naive": ta, "rapid": tb, "rel_diff": (tb - ta) / ta}
    half = P // 2
    out = {
        "naive_ms": naive_ms, "rapid_ms": rapid_ms, "rapid_over_naive": rapid_ms / naive_ms,
        "naive_entries_per_s": P * v / (naive_ms * 1e-3),
        "rapid_entries_per_s": P * v / (rapid_ms * 1e-3),
        "rapid_phases_ms": {k: phase[k] for k in ("prepare_ms", "train_ms", "recover_ms")},
        "rapid_info": {k: phase[k] for k in ("sigma", "mu", "train_steps", "m_per_perm")},
        "opts": {"train_passes": opts.train_passes, "qr_every": opts.qr_every,
                 "admm_iters": opts.admm_iters, "admm_rho": opts.admm_rho,
                 "shift_mode": opts.shift_mode, "training_rows_precision": "bf16x3",
                 "naive_precision": "fp16x2"},
        "accuracy_vs_naive": {
            "kl": hist_kl(a, b), **thr, "resampling_risk_fwer0.05": risk,
            # the estimator's own floor: two exhaustive max-nulls over disjoint halves
            # of the relabellings (same distribution, independent samples)
            "kl_exact_halves": hist_kl(a[:half], a[half:]),
            "thr_rel_diff_exact_halves": {"fwer%g" % al: fwer_thr(a[half:], al) /
                                          fwer_thr(a[:half], al) - 1.0 for al in (0.05, 0.01)}},
        "timing": "device events; NaivePT 3 runs, RapidPT 1 run after 1 warm-up each",
    }
    return out, v, a, am.cpu().numpy()


def rapid_leg(dev, B, synth, torch, passes=1, rows=None):
    """RapidPT vs NaivePT max-null wall time on the RapidPT workload (n=200,
    500,000 voxels, 100,000 relabellings, r=50, 400 training rows, 0.35%
    sampling): each method's time from pt_prepare to the max-null vector, with
    the exhaustive NaivePT result as the accuracy reference."""
    name = "brain_n200_v500k"
    w = synth.workload(name, device=dev)
    X, mask, n1 = w["X"], w["mask"], w["n1"]
    perms = torch.as_tensor(w["perms"][:rows] if rows else w["perms"]).to(dev)
    P, r, ell, eta = perms.shape[0], w["rank"], w["n_train"], w["sample_rate"]
    out, v, a_naive, _ = rapid_vs_naive(dev, B, torch, X, mask, n1, perms, r, ell, eta, passes)
    out = {"workload": "%s: n=200 (100/100), %d voxels, no signal, P=%d, r=%d, n_train=%d, "
                       "sample_rate=%g" % (name, v, P, r, ell, eta), **out}
    out["recovery_updates"] = recovery_updates_study(dev, B, torch, X, mask, n1, perms, r, ell,
                                                     eta, a_naive, passes)
    return out


def recovery_updates_study(dev, B, torch, X, mask, n1, perms, r, ell, eta, a_naive, passes,
                           rows=2000):
    """U updates during recovery (pt_rapid_opts.rec_step = 1, sequential) against
    the frozen U of Alg. 2, on the first `rows` recovery relabellings after the
    same training: accuracy of each against NaivePT's maxima of those rows, and
    the time of each recovery."""
    stream = torch.cuda.current_stream(dev)
    c = B.pt_prepare(X, n1, mask, stream=stream)
    V = B.pt_num_valid_voxels(c)
    U = torch.empty((V, r), dtype=torch.float32, device=dev)
    opts = B.rapid_opts(train_passes=passes)
    sub = perms[:ell + rows]
    tmax = torch.empty(ell, dtype=torch.float32, device=dev)
    info = B.pt_rapid_train(c, sub, ell, r, eta, opts, U, tmax)
    res = {}
    ref = a_naive[ell:ell + rows]
    for name, step in (("frozen", 0.0), ("updates", 1.0)):
        o = B.rapid_opts(train_passes=passes, rec_step=step)
        mx = torch.empty(rows, dtype=torch.float32, device=dev)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        B.pt_rapid_recover(c, sub, ell, U, r, eta, info.sigma, info.mu, o, mx)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        b = mx.cpu().numpy().astype(np.float64)
        res[name] = {"recover_ms": dt * 1e3, "kl": hist_kl(ref, b),
                     "sd_ratio": float(b.std() / ref.std()),
                     "mean_diff": float(b.mean() - ref.mean()),
                     **{"fwer%g" % al: fwer_thr(b, al) / fwer_thr(ref, al) - 1.0
                        for al in (0.05, 0.01)}}
    c.close()
    res["rows"] = "recovery relabellings %d..%d of the same workload and training" % (
        ell, ell + rows - 1)
    return res


def large_leg(dev, B, synth, torch, passes=1):
    """The largest workload: n=400 (200/200), 600,000 voxels of the smoothed
    field with a +0.2 SD effect of radius 8, 100,000 relabellings; NaivePT
    (BF16x3, FP64 winner statistic) and RapidPT (r=100, 800 training rows,
    0.35% sampling) each timed from pt_prepare to the max-null, with RapidPT's
    thresholds against NaivePT's. Returns (object, host data for the CPU leg)."""
    name = "brain_n400_v600k"
    w = synth.workload(name, device=dev)
    X, mask, n1 = w["X"], w["mask"], w["n1"]
    perms = torch.as_tensor(w["perms"]).to(dev)
    P, r, ell, eta = perms.shape[0], w["rank"], w["n_train"], w["sample_rate"]
    out, v, mx_naive, am_naive = rapid_vs_naive(dev, B, torch, X, mask, n1, perms, r, ell, eta,
                                                passes)
    out = {"workload": "%s: n=400 (200/200), %d voxels, +0.2 SD effect r=8, P=%d, r=%d, "
                       "n_train=%d, sample_rate=%g" % (name, v, P, r, ell, eta), **out}
    host = {"X": X[:, mask.bool()].cpu().numpy(), "n1": n1, "perms": w["perms"],
            "maxnull": mx_naive, "argmax": am_naive}
    del X
    return out, host


def precision_leg(dev, B, torch, X, mask, n1, perms, t_rows_sel, reps=20):
    """Each arithmetic path of the fused kernel (FP32 CUDA cores, BF16x2 and
    BF16x3 tensor cores) on the benchmark workload: fused-kernel and call time,
    the full max-null (thresholds), and rows of T at the relabellings
    t_rows_sel (for the t-entry error against the oracle's rows)."""
    stream = torch.cuda.current_stream(dev)
    P = perms.shape[0]
    out = {}
    for name, prec in (("fp32", 0), ("bf16x2", 1), ("bf16x3", 2), ("fp16x2", 3)):
        ctx = B.pt_prepare(X, n1, mask, stream=stream)
        opts = B.naive_opts(prec)
        if prec:
            B.pt_autotune_naive(ctx, perms, opts)
        mx = torch.empty(P, dtype=torch.float32, device=dev)
        am = torch.empty(P, dtype=torch.int32, device=dev)
        k = reps if prec else max(3, reps // 4)
        for _ in range(2):
            B.pt_maxnull_naive_ex(ctx, perms, opts, mx, am, None)
        B.pt_sync(ctx)
        B.pt_profile_enable(ctx, True)
        B.pt_profile_read(ctx)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(k):
            B.pt_maxnull_naive_ex(ctx, perms, opts, mx, am, None)
        e1.record(stream)
        B.pt_sync(ctx)
        kern_ms, nk = B.pt_profile_read(ctx)
        B.pt_profile_enable(ctx, False)
        T = B.pt_t_rows(ctx, perms[torch.as_tensor(t_rows_sel, device=dev)], prec)
        B.pt_sync(ctx)
        ctx.close()
        out[name] = {"kernel_ms": kern_ms / max(nk, 1), "call_ms": e0.elapsed_time(e1) / k,
                     "maxnull": mx.cpu().numpy().astype(np.float64), "argmax": am.cpu().numpy(),
                     "t_rows": T.cpu().numpy().astype(np.float64)}
    return out


def precision_summary(paths, ref_rows, ref_max, ref_argmax, ref_t):
    """Errors of each path against the FP64 oracle: max-null on the oracle's
    sampled rows (relative), argmax agreement there, t entries of the sampled T
    rows (|dt| / max(|t|, 1)), and the FWER thresholds of the full max-null
    (an order statistic moves by at most the largest per-row error, so the
    threshold error against the oracle is bounded by the max-null error)."""
    res = {}
    base = paths["bf16x3"]["maxnull"]
    for name, p in paths.items():
        m = p["maxnull"][ref_rows]
        rel = np.abs(m - ref_max) / np.maximum(np.abs(ref_max), 1.0)
        ok = np.isfinite(ref_t)
        terr = np.abs(p["t_rows"][ok] - ref_t[ok]) / np.maximum(np.abs(ref_t[ok]), 1.0)
        res[name] = {
            "kernel_ms": p["kernel_ms"], "call_ms": p["call_ms"],
            "maxnull_max_rel_err": float(rel.max()),
            "argmax_agree": float(np.mean(p["argmax"][ref_rows] == ref_argmax)),
            "t_entry_max_rel_err": float(terr.max()),
            "t_entry_mean_rel_err": float(terr.mean()),
            "fwer_thr": {"%g" % a: fwer_thr(p["maxnull"], a) for a in (0.05, 0.01)},
            "thr_rel_diff_vs_bf16x3": {"%g" % a: fwer_thr(p["maxnull"], a) / fwer_thr(base, a) - 1
                                       for a in (0.05, 0.01)},
            "thr_err_bound_vs_oracle": float(np.max(np.abs(m - ref_max)))}
    res["speedup_bf16x3_over_fp32_kernel"] = paths["fp32"]["kernel_ms"] / paths["bf16x3"]["kernel_ms"]
    res["speedup_bf16x2_over_fp32_kernel"] = paths["fp32"]["kernel_ms"] / paths["bf16x2"]["kernel_ms"]
    res["speedup_fp16x2_over_fp32_kernel"] = paths["fp32"]["kernel_ms"] / paths["fp16x2"]["kernel_ms"]
    res["reference"] = ("FP64 oracle (oracle/naive_fp64.c), %d sampled relabelling rows x all "
                        "voxels for maxima, %d rows for t entries, computed in the CPU leg"
                        % (len(ref_rows), ref_t.shape[0]))
    return res


def batched_leg(dev, B, synth, torch, studies=64, P=10000):
    """Many independent studies of uneven shape in one call: 64 studies with
    n ~ U{24..400} (n1 = n/2) and v ~ U{50k..600k} voxels (PCG32 seeded 1000 + k),
    10,000 relabellings each, FP16x2. Each study is a smoothed brain-shaped field
    in [0, 1] (FWHM 8 voxels, the first v voxels of an ellipsoid mask on a
    121x145x121 grid, seeded 1000 + k). Compares pt_maxnull_naive_batched (one
    persistent launch per launch class, replayed as a CUDA graph) with one
    pt_maxnull_naive_ex call per study on the same stream, and times each
    study's fused kernel alone (the library's event pair)."""
    shapes = synth.uneven_study_shapes(studies)
    stream = torch.cuda.current_stream(dev)
    ctxs, perms, mx, am = [], [], [], []
    sa = tuple(a * 1.4 for a in (34, 44, 37))
    for k, (n, n1, v) in enumerate(shapes):
        X, mask = synth.brain_field(n, n1, grid=synth.BIG_GRID, center=synth.BIG_CENTER,
                                    semi_axes=sa, seed=1000 + k, device=dev, v_limit=v)
        ctxs.append(B.pt_prepare(X, n1, mask, stream=stream))
        del X, mask
        perms.append(torch.as_tensor(synth.perms_pcg32(n, P, seed=1000 + k)).to(dev))
        mx.append(torch.empty(P, dtype=torch.float32, device=dev))
        am.append(torch.empty(P, dtype=torch.int32, device=dev))
    entries = float(P) * sum(v for _, _, v in shapes)
    opts = B.naive_opts(NAIVE_PREC)

    def batched():
        B.pt_maxnull_naive_batched(ctxs, perms, opts, mx, am)

    def sequential():
        for c, p_, m_, a_ in zip(ctxs, perms, mx, am):
            B.pt_maxnull_naive_ex(c, p_, opts, m_, a_, None)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        return e0.elapsed_time(e1) / reps

    B.pt_autotune_naive_batched(ctxs, perms, opts)
    batched()  # plans and captures the graph
    b_ms = timed(batched, 5)
    s_ms = timed(sequential, 3)
    # each study's fused kernel alone (the library's event pair around it)
    per = []
    for c, p_, m_, a_ in zip(ctxs, perms, mx, am):
        B.pt_profile_enable(c, True)
        B.pt_profile_read(c)
        B.pt_maxnull_naive_ex(c, p_, opts, m_, a_, None)
        ms_k, nk = B.pt_profile_read(c)
        B.pt_profile_enable(c, False)
        per.append(ms_k / max(nk, 1))
    for c in ctxs:
        B.pt_sync(c)
        c.close()
    ns = [n for n, _, _ in shapes]
    pk, _ = peaks()
    flops = sum(2.0 * n * P * v for n, _, v in shapes)
    hw = sum(2.0 * 2 * ((n + 15) // 16 * 16) * P * v for n, _, v in shapes)
    order = np.argsort(per)

    def study(i):
        n, _, v = shapes[i]
        return {"n": n, "v": v, "kernel_ms": per[i],
                "entries_per_s": P * v / (per[i] * 1e-3),
                "issued_tflops": 4.0 * ((n + 15) // 16 * 16) * P * v / (per[i] * 1e-3) / 1e12}
    return {"workload": "%d studies, n ~ U{24..400} (here %d..%d), v ~ U{50k..600k} "
                        "(total %d voxels), P=%d each, smoothed [0,1] fields (FWHM 8)"
                        % (studies, min(ns), max(ns), sum(v for _, _, v in shapes), P),
            "entries": entries, "batched_ms": b_ms, "sequential_ms": s_ms,
            "batched_over_sequential": s_ms / b_ms,
            "batched_entries_per_s": entries / (b_ms * 1e-3),
            "sequential_entries_per_s": entries / (s_ms * 1e-3),
            "roofline": {"algorithmic_tflops": flops / (b_ms * 1e-3) / 1e12,
                         "frac_of_burst_peak": flops / (b_ms * 1e-3) / 1e12 / pk["bf16_tflops"],
                         "issued_tflops": hw / (b_ms * 1e-3) / 1e12,
                         "hw_frac_of_burst_peak": hw / (b_ms * 1e-3) / 1e12 / pk["bf16_tflops"],
                         "flops": "algorithmic 2 n P v per study; issued 2 FP16 pieces x "
                                  "2 n_pad P v (n_pad = n rounded up to 16)"},
            "sequential_kernel_ms_sum": float(sum(per)),
            "sequential_outside_kernels_ms": s_ms - float(sum(per)),
            "fastest_studies": [study(i) for i in order[:3]],
            "slowest_studies": [study(i) for i in order[-4:]],
            "timing": "device events over 5 graph replays / 3 loops of per-study calls; "
                      "per-study kernel times from one profiled call each"}


def glm_leg(dev, B, synth, torch, q=2, reps=20):
    """NaivePT with q nuisance covariates (pt_prepare_glm) on the benchmark
    workload (n=100, 231,719 voxels, 10,000 relabellings): the covariate-adjusted
    t of the group column; covariates are seeded N(0,1) values per subject."""
    w = synth.workload(WORKLOAD, device=dev)
    X, mask, n1 = w["X"], w["mask"], w["n1"]
    n = X.shape[0]
    Z = np.random.default_rng(5).standard_normal((n, q))
    perms = torch.as_tensor(w["perms"]).to(dev)
    P = perms.shape[0]
    stream = torch.cuda.current_stream(dev)
    ctx = B.pt_prepare_glm(X, n1, Z, mask, stream=stream)
    v = B.pt_num_voxels(ctx)
    mx = torch.empty(P, dtype=torch.float32, device=dev)
    am = torch.empty(P, dtype=torch.int32, device=dev)
    ct = torch.empty(v, dtype=torch.int32, device=dev)
    opts = B.naive_opts(2)
    B.pt_autotune_naive(ctx, perms, opts)
    for _ in range(3):
        B.pt_maxnull_naive_ex(ctx, perms, opts, mx, am, ct)
    B.pt_sync(ctx)
    B.pt_profile_enable(ctx, True)
    B.pt_profile_read(ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        B.pt_maxnull_naive_ex(ctx, perms, opts, mx, am, ct)
    e1.record(stream)
    B.pt_sync(ctx)
    kern_ms, k = B.pt_profile_read(ctx)
    ms = e0.elapsed_time(e1) / reps
    ctx.close()
    return {"workload": "%s with %d covariates (N(0,1), seeded): group t adjusted by least "
                        "squares, %d voxels, P=%d" % (WORKLOAD, q, v, P),
            "maxnull_ms": ms, "kernel_ms": kern_ms / max(k, 1),
            "entries_per_s": float(P) * v / (ms * 1e-3),
            "timing": "device events over %d calls of pt_maxnull_naive_ex (context prepared "
                      "once)" % reps}


def cpu_leg(Xm, n1, perms_np, t_rows_sel, large_host=None, large_rows=32):
    """The CPU leg: the FP64 oracle (oracle/) on the host cores. It times a
    bounded sample of whole relabelling rows of the benchmark workload (the
    cpu_baseline), and the rows it computes, plus the oracle's rows of T at
    t_rows_sel and a spread sample of rows of the n=400 workload, are the
    references of the precision and large objects."""
    import oracle
    Xt = oracle.voxel_major(Xm)
    rate, rows, dt, cores, out = oracle_sample(Xm, n1, perms_np, seconds_target=15.0, Xt=Xt)
    v = Xm.shape[1]
    base = {"value": rate, "unit": "T entries/s", "cores": cores, "kind": "oracle",
            "sample": "%d relabelling rows x %d voxels, %.1f s" % (rows, v, dt)}
    ref = {"rows": np.arange(rows), "maxnull": out[0], "argmax": out[1],
           "t_rows": oracle.t_rows(None, n1, perms_np[t_rows_sel], nthreads=cores, Xt=Xt)}
    del Xt
    large = None
    if large_host is not None:
        h = large_host
        P = h["perms"].shape[0]
        sel = np.linspace(0, P - 1, large_rows).round().astype(np.int64)
        Xt4 = oracle.voxel_major(h["X"])
        t0 = time.perf_counter()
        o4 = _oracle_rows(Xt4, h["n1"], h["perms"][sel], cores)
        dt4 = time.perf_counter() - t0
        m_gpu = h["maxnull"][sel]
        rel = np.abs(m_gpu - o4[0]) / np.maximum(np.abs(o4[0]), 1.0)
        large = {"rows": int(sel.size), "oracle_s": dt4,
                 "maxnull_max_rel_err": float(rel.max()),
                 "argmax_agree": float(np.mean(h["argmax"][sel] == o4[1])),
                 "thr_err_bound": float(np.max(np.abs(m_gpu - o4[0]))),
                 "note": "GPU NaivePT max-null vs the FP64 oracle on %d relabellings spread "
                         "over the %d; the FWER thresholds are order statistics of the "
                         "max-null, so they differ from the oracle's by at most the largest "
                         "per-row error" % (sel.size, P)}
    return base, ref, large


def anova_leg(dev, B, synth, torch, sizes=(33, 33, 34), reps=3):
    """One-way F of three groups as the voxel statistic (pt_maxnull_anova) on the
    benchmark workload (n=100, 231,719 voxels, 10,000 relabellings): the two
    group sums per relabelling from the FP16x2 contraction, B and its maxima and
    counts, the winner's F in FP64."""
    w = synth.workload(WORKLOAD, device=dev)
    X, mask = w["X"], w["mask"]
    perms = torch.as_tensor(w["perms"]).to(dev)
    P = perms.shape[0]
    stream = torch.cuda.current_stream(dev)
    ctx = B.pt_prepare(X, sizes[0], mask, stream=stream)
    v = B.pt_num_voxels(ctx)
    mx, _, _ = B.pt_maxnull_anova(ctx, perms, list(sizes), NAIVE_PREC)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        mx, _, _ = B.pt_maxnull_anova(ctx, perms, list(sizes), NAIVE_PREC)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / reps
    ctx.close()
    m = mx.cpu().numpy().astype(np.float64)
    # the same factor with two seeded N(0,1) covariates per subject (one-way
    # ANCOVA: pt_prepare_glm context, BF16x3 pieces of the unit residual)
    Z = np.random.default_rng(5).standard_normal((X.shape[0], 2))
    ctx = B.pt_prepare_glm(X, sizes[0], Z, mask, stream=stream)
    mc, _, _ = B.pt_maxnull_anova(ctx, perms, list(sizes), 2)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    for _ in range(reps):
        mc, _, _ = B.pt_maxnull_anova(ctx, perms, list(sizes), 2)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_c = e0.elapsed_time(e1) / reps
    B.pt_sync(ctx)
    ctx.close()
    mc = mc.cpu().numpy().astype(np.float64)
    return {"workload": "%s, groups %s (one-way F), %d voxels, P=%d" % (WORKLOAD, list(sizes), v, P),
            "ms_per_call": ms, "entries_per_s": P * v / (ms * 1e-3),
            "fwer_thr": {"%g" % a: fwer_thr(m, a) for a in (0.05, 0.01)},
            "with_covariates": {"covariates": "2, seeded N(0,1) per subject; F of the factor "
                                              "adjusted for them (BF16x3)",
                                "ms_per_call": ms_c, "entries_per_s": P * v / (ms_c * 1e-3),
                                "fwer_thr": {"%g" % a: fwer_thr(mc, a) for a in (0.05, 0.01)}},
            "timing": "device events over %d calls" % reps}


def cluster_leg(dev, B, synth, torch, tau=3.2, conn=18, reps=3):
    """Cluster-level inference on the benchmark workload (n=100, 231,719 voxels,
    10,000 relabellings): the largest cluster of {t >= tau} per relabelling
    (pt_cluster_maxnull: the FP16x2 contraction writes one bit per entry, u >= u(tau); union-find over the active voxels of the 91x109x91 grid)
    and the observed map's clusters with their cluster-level FWER p-values."""
    w = synth.workload(WORKLOAD, device=dev)
    X, mask, n1 = w["X"], w["mask"], w["n1"]
    perms = torch.as_tensor(w["perms"]).to(dev)
    P = perms.shape[0]
    dims = (91, 109, 91)
    stream = torch.cuda.current_stream(dev)
    ctx = B.pt_prepare(X, n1, mask, stream=stream)
    ms = B.pt_cluster_maxnull(ctx, perms, tau, dims, conn, NAIVE_PREC)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        B.pt_cluster_maxnull(ctx, perms, tau, dims, conn, NAIVE_PREC, out=ms)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_call = e0.elapsed_time(e1) / reps
    label, size = B.pt_cluster_observed(ctx, tau, dims, conn)
    B.pt_sync(ctx)
    v = B.pt_num_voxels(ctx)
    ctx.close()
    m = np.sort(ms.cpu().numpy())
    lab = label.cpu().numpy()
    sz = size.cpu().numpy()
    reps_ = np.unique(lab[lab >= 0])
    ks = np.sort(np.array([sz[r] for r in reps_], dtype=np.int64))[::-1]
    pv = [(1.0 + (P - np.searchsorted(m, k, side="left"))) / (P + 1.0) for k in ks[:5]]
    return {"workload": "%s: n=100, %d voxels, P=%d, tau=%g (t), %d-connectivity"
                        % (WORKLOAD, v, P, tau, conn),
            "ms_per_call": ms_call, "entries_per_s": P * v / (ms_call * 1e-3),
            "max_cluster_null": {"median": float(np.median(m)), "p95": float(m[int(0.95 * P)]),
                                 "max": int(m[-1])},
            "observed_clusters": int(reps_.size),
            "largest_observed": [{"k": int(k), "p_fwe_cluster": float(p)}
                                 for k, p in zip(ks[:5], pv)],
            "timing": "device events over %d calls (bit rows u >= u(tau) from the contraction, union-find over the active voxels, max)"
                      % reps}


def run_ours(args):
    if args.cluster_only:
        import torch
        from paper_1703_01506_gb300 import binding as B
        from paper_1703_01506_gb300 import synth
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        B.load()
        print(json.dumps({"cluster": cluster_leg(dev, B, synth, torch)}), flush=True)
        return
    if args.anova_only:
        import torch
        from paper_1703_01506_gb300 import binding as B
        from paper_1703_01506_gb300 import synth
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        B.load()
        print(json.dumps({"anova": anova_leg(dev, B, synth, torch)}), flush=True)
        return
    if args.rapid_only:
        import torch
        from paper_1703_01506_gb300 import binding as B
        from paper_1703_01506_gb300 import synth
        dev = torch.device("cuda", 0)
        torch.cuda.set_device(dev)
        B.load()
        print(json.dumps({"rapidpt": rapid_leg(dev, B, synth, torch, args.rapid_passes,
                                                args.rapid_rows)}), flush=True)
        return
    import torch
    import torch.distributed as dist
    from paper_1703_01506_gb300 import binding as B
    from paper_1703_01506_gb300 import synth

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.load()
    prec = PREC[args.precision]

    w = synth.workload(WORKLOAD, device=dev)
    X, mask, n1 = w["X"], w["mask"], w["n1"]
    n = X.shape[0]
    # One study, relabellings sharded across ranks (weak scaling: 10,000 per rank
    # of one PCG32 list of world x 10,000); rank 0 holds the single-GPU list.
    P_all = ws * w["P"]
    perms_np = w["perms"] if ws == 1 else synth.perms_pcg32(n, P_all, seed=1)
    if ws > 1:
        from paper_1703_01506_gb300 import shard
        a_, b_ = shard.shard_rows(P_all, ws, rank)
        perms_np = perms_np[a_:b_]
    P = perms_np.shape[0]
    perms = torch.as_tensor(perms_np).to(dev)
    stream = torch.cuda.current_stream(dev)
    maxnull = torch.empty(P, dtype=torch.float32, device=dev)
    argmax = torch.empty(P, dtype=torch.int32, device=dev)

    def merge():
        """The study's result across ranks: every rank's maxima and argmax
        gathered in relabelling order, exceedance counts summed (NCCL)."""
        if ws == 1:
            return maxnull, argmax, step.counts
        return (shard.merge_maxnull(maxnull, P_all), shard.merge_maxnull(argmax, P_all),
                shard.merge_counts(step.counts))

    def launch(ctx, profile=False):
        if profile:
            B.pt_profile_enable(ctx, True)
        counts = step.counts
        if counts is None or counts.numel() != B.pt_num_voxels(ctx):
            counts = step.counts = torch.empty(B.pt_num_voxels(ctx), dtype=torch.int32, device=dev)
        B.pt_maxnull_naive_ex(ctx, perms, B.naive_opts(prec), maxnull, argmax, counts)
        step.merged = merge()
        return ctx

    def step(profile=False):
        return launch(B.pt_prepare(X, n1, mask, stream=stream), profile)
    step.counts = None

    ctx = step()
    B.pt_sync(ctx)
    v = B.pt_num_voxels(ctx)
    tuned = None
    if prec != 0 and not args.no_tune:
        # The library's autotuner times the fused kernel's launch configurations
        # on this problem once and records the fastest for later calls.
        cfg, tune_ms = B.pt_autotune_naive(ctx, perms, B.naive_opts(prec))
        tuned = {"voxel_tile": cfg.voxel_tile, "stages": cfg.stages,
                 "ksteps_per_stage": cfg.ksteps_per_stage, "items_per_sm": cfg.items_per_sm,
                 "kernel_ms_when_tuned": tune_ms}
    ctx.close()
    for _ in range(args.warmup):
        ctx = step()
        B.pt_sync(ctx)
        ctx.close()
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    launches0 = B.pt_kernel_launch_count()
    kern_ms, kern_n = 0.0, 0
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    t_wall0 = time.time()
    ev0.record(stream)
    prev = None
    for _ in range(args.steps):
        # pt_prepare waits for the stream once (it sizes the launches by the
        # count of voxels with a defined t), which also finishes the previous
        # step; that step's kernel time is read and its context closed (its
        # workspaces go back to the library's cache) before this step launches.
        ctx = B.pt_prepare(X, n1, mask, stream=stream)
        if prev is not None:
            ms_k, n_k = B.pt_profile_read(prev)
            kern_ms += ms_k
            kern_n += n_k
            prev.close()
        prev = launch(ctx, profile=True)
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    t_wall1 = time.time()
    B.pt_sync(prev)  # error bits (every warm-up step was checked the same way)
    ms_k, n_k = B.pt_profile_read(prev)
    kern_ms += ms_k
    kern_n += n_k
    prev.close()
    launches = B.pt_kernel_launch_count() - launches0
    clk = clocks.stop(t_wall0, t_wall1)
    ms = ev0.elapsed_time(ev1) / args.steps
    if ws > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    entries = float(P) * v
    value = ws * entries / (ms / 1000.0)

    if args.quick:
        if rank == 0:
            print(json.dumps({"quick": True, "ms_per_step": ms, "value": value,
                              "kernel_ms": kern_ms / max(kern_n, 1), "precision": args.precision}),
                  flush=True)
        if ws > 1:
            dist.destroy_process_group()
        return

    # ---- end to end through host buffers (pinned), transfers inside the timed region:
    # the library reads X and the mask straight from page-locked host memory (only the
    # mask voxels' values cross the link); relabellings are copied; results copied back.
    Xh = X.cpu().pin_memory()
    mh = mask.cpu().pin_memory()
    ph = torch.as_tensor(perms_np).pin_memory()
    pd = torch.empty_like(perms)

    mx_h = torch.empty(P_all, dtype=torch.float32).pin_memory()
    am_h = torch.empty(P_all, dtype=torch.int32).pin_memory()
    ct_h = torch.empty(v, dtype=torch.int32 if ws == 1 else torch.int64).pin_memory()

    def e2e_step():
        pd.copy_(ph, non_blocking=True)
        c = B.pt_prepare(Xh, n1, mh, stream=stream)
        B.pt_maxnull_naive_ex(c, pd, B.naive_opts(prec), maxnull, argmax, step.counts)
        m_, a_, c_ = merge()
        mx_h.copy_(m_, non_blocking=True)
        am_h.copy_(a_, non_blocking=True)
        ct_h.copy_(c_, non_blocking=True)
        B.pt_sync(c)
        c.close()

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms_e2e = e0.elapsed_time(e1) / args.steps
    if ws > 1:
        t = torch.tensor([ms_e2e], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_e2e = float(t.item())
    h2d = n * v * 4 + mh.numel() + ph.numel() * 4  # mask voxels' values, mask, relabellings
    d2h = mx_h.numel() * 4 + am_h.numel() * 4 + ct_h.numel() * ct_h.element_size()

    # ---- roofline of the dominant kernel (fused contraction + reduction) ----
    pk, src = peaks()
    avg_kern_ms = kern_ms / max(kern_n, 1)
    if prec == 0:
        flops = 2.0 * n * entries  # algorithmic: 2 flops per subject per entry
        fp32_peak = None
        roof = {"bound": "alu", "achieved": flops / (avg_kern_ms * 1e-3) / 1e12,
                "unit": "TFLOP/s", "note": "plain FP32 CUDA-core path"}
    else:
        flops = 2.0 * n * entries
        # The fused kernel runs about a millisecond per step and the timed region
        # lasts well under the seconds-long loop of the sustained figure, so the
        # burst BF16 peak is its denominator.
        timed_s = ms * args.steps / 1000.0
        peak_key = "bf16_tflops" if timed_s < 2.0 else "bf16_tflops_sustained"
        peak = pk.get(peak_key, pk.get("bf16_tflops"))
        ach = flops / (avg_kern_ms * 1e-3) / 1e12
        pieces = 3 if prec == 2 else 2
        n_pad = (n + 15) // 16 * 16
        hw = 2.0 * pieces * n_pad * entries / (avg_kern_ms * 1e-3) / 1e12
        # DRAM bytes per launch of this kernel from the ncu capture summarised in
        # profiles/tc_contract_kernel_bf16x3_brain_n100_v232k.md (BF16x3, tuned launch).
        traffic = TRAFFIC_BYTES.get(prec) if tuned is not None else None
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": traffic,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum, one launch"
                if traffic else None,
                "peak_source": "%s %s (MEASURED_PEAKS.json; timed region %.2f s)"
                               % (src, "bf16 burst" if peak_key == "bf16_tflops" else
                                  "bf16 sustained", timed_s),
                "kernel": "tc_contract_kernel<256>", "kernel_ms": avg_kern_ms,
                "launch_config": tuned,
                "hw_tflops": hw, "hw_frac": hw / peak,
                "algorithmic": "2n flops per T entry (n=%d); hardware issues %d data pieces x "
                               "n_pad=%d" % (n, pieces, n_pad)}

    line = {
        "metric": METRIC, "value": value, "unit": "T entries/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "bf16x2/f32acc", 2: "bf16x3/f32acc", 3: "fp16x2/f32acc"}[prec],
        "data": "synthetic",
        "config": {"workload": "%s: n=100 (50/50), 91x109x91 grid, ellipsoid mask %d voxels, "
                               "FWHM 8 smoothing, +0.3 SD effect r=10, P=%d relabellings per "
                               "GPU (PCG32 Fisher-Yates)" % (WORKLOAD, v, P),
                   "precision": args.precision,
                   "parallelism": "one study, relabellings sharded over %d GPUs (%d each); "
                                  "maxima gathered and counts summed over NCCL inside every "
                                  "step" % (ws, P) if ws > 1 else "single GPU",
                   "l2": "inputs larger than L2 (X %.0f MB, BF16 pieces %.0f MB)"
                         % (X.numel() * 4 / 1e6, v * ((n + 15) // 16 * 16) * 6 / 1e6),
                   "step": "pt_prepare + pt_maxnull_naive (labels, fused contraction, finalise)"},
        "roofline": roof,
        "clocks": clk,
        "e2e": {"value": ws * entries / (ms_e2e / 1000.0), "unit": "T entries/s",
                "ms_per_step": ms_e2e, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "kernel_launches_per_step": launches / args.steps,
        "maxnull_wall_ms": ms,
    }
    t_sel = np.array([0, 1, P // 2, P - 1])
    paths = None
    if ws == 1 and not args.no_precision:
        paths = precision_leg(dev, B, torch, X, mask, n1, perms, t_sel)
    if ws == 1 and not args.no_rapid:
        line["rapidpt"] = rapid_leg(dev, B, synth, torch, args.rapid_passes, args.rapid_rows)
    if ws == 1 and not args.no_batched:
        line["batched"] = batched_leg(dev, B, synth, torch)
    if ws == 1 and not args.no_glm:
        line["glm"] = glm_leg(dev, B, synth, torch)
    if ws == 1 and not args.no_cluster:
        line["cluster"] = cluster_leg(dev, B, synth, torch)
        line["anova"] = anova_leg(dev, B, synth, torch)
    large_host = None
    if ws == 1 and not args.no_large:
        line["large"], large_host = large_leg(dev, B, synth, torch, args.rapid_passes)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        Xm = w["X"][:, mask.bool()].cpu().numpy()
        base, ref, large_or = cpu_leg(Xm, n1, perms_np, t_sel, large_host)
        line["cpu_baseline"] = base
        if paths is not None:
            line["precision"] = precision_summary(paths, ref["rows"], ref["maxnull"],
                                                  ref["argmax"], ref["t_rows"])
        if large_or is not None:
            line["large"]["naive_vs_oracle"] = large_or
    elif paths is not None:
        line["precision"] = {k: {"kernel_ms": p_["kernel_ms"], "call_ms": p_["call_ms"]}
                             for k, p_ in paths.items()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp16x2", choices=list(PREC))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rapid-passes", type=int, default=1,
                    help="RapidPT training passes in the RapidPT leg (default 1, Alg. 2)")
    ap.add_argument("--rapid-rows", type=int, default=0,
                    help="relabellings of the RapidPT leg (default all 100,000)")
    ap.add_argument("--cluster-only", action="store_true",
                    help="run only the cluster-level leg (one line with its object)")
    ap.add_argument("--anova-only", action="store_true",
                    help="run only the F-statistic leg (one line with its object)")
    ap.add_argument("--rapid-only", action="store_true",
                    help="run the RapidPT leg alone (profiling); prints only its object")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-study batched leg")
    ap.add_argument("--no-rapid", action="store_true",
                    help="skip the RapidPT vs NaivePT leg (n=200, 500k voxels, 1e5 relabellings)")
    ap.add_argument("--no-glm", action="store_true",
                    help="skip the covariate-adjusted NaivePT leg")
    ap.add_argument("--no-cluster", action="store_true",
                    help="skip the cluster-level leg (largest cluster per relabelling)")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the n=400, 600k-voxel NaivePT/RapidPT leg")
    ap.add_argument("--no-precision", action="store_true",
                    help="skip the per-precision timing and error leg")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip the autotuner (default launch configurations)")
    ap.add_argument("--quick", action="store_true",
                    help="device-timed steps only (no e2e, no CPU leg): for profiler runs")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
