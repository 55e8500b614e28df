#!/usr/bin/env python
"""Benchmark of the CPRAND-MIX hot path on one GB300 (or N replicas under torchrun).

Headline workload: the 1500 x 1500 x 1500 FP32 tensor (13.5 GB) of rank 50 with factor congruence
0.5 and 0.1% noise (the synthetic recipe of Sec. 4.2), R = 50, S = 2000 samples per least-squares
solve, P_hat = 2^14 fit entries, stopped by the best-fit stall rule (10 iterations without strict
improvement) or 200 iterations.

One step = one complete CPRAND-MIX decomposition (Alg. 5): ||X||, mixing of all three modes, the
mode-unfolding copies, random start, outer iterations until the stopping rule fires, unmixing.  The
input tensor is resident in HBM when the timed region starts and is far larger than L2 (13.5 GB vs
129 MB), so no flush is needed.

metric: ALS iters/s = outer iterations per second of the iteration phase (the preprocess, mixing
included, is timed separately and reported as time_to_solution and in time_to_fit).
e2e: the same call through the C ABI with the tensor in pinned host memory: every step copies X to
the device, decomposes it and copies lambda and the factors back, as a stream of decompositions (the
next step's copy, on a second stream into a second device buffer, overlaps the current
decomposition); e2e.serial is the same with nothing overlapped.

The other parts of the metric, measured after the timed regions: time to fit at F* - 1e-3, with F*
the converged fit of the library's exact CP-ALS (FP64 Gram / solve / fit, Alg. 1) on the same stored
tensor, for the library, for a plain FP64 GPU form of CPRAND-MIX in stock PyTorch, and for the exact
CP-ALS itself; the gather bandwidth; the same workload in BF16 storage; the 400^3 and 100^4
workloads.

--impl reference times the CPU oracle (oracle/, FP64 NumPy) on the same workload: one step is one
outer iteration of the oracle's CPRAND (the mixing pass is timed on a slab and reported separately).
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = {
    "workload": "cprand_mix 1500x1500x1500 fp32 (13.5 GB), rank-50 congruence-0.5 factors, 0.1% noise; "
                "R=50, S=2000, P_hat=2^14, stall rule k=10, max 200 iterations",
    "dims": [1500, 1500, 1500], "R": 50, "S": 2000, "congruence": 0.5, "eta": 0.001, "P_hat": 16384,
    "max_iters": 200, "stall_iters": 10, "fit_tol": -1.0, "data_seed": 1005, "philox_seed": 2005,
}
W400 = {"dims": [400, 400, 400], "R": 10, "S": 230, "congruence": 0.9, "eta": 0.01, "P_hat": 16384,
        "max_iters": 200, "fit_tol": 1e-4, "data_seed": 1001, "philox_seed": 2001}
W100 = {"dims": [100, 100, 100, 100], "R": 16, "S": 450, "congruence": 0.5, "eta": 0.01, "P_hat": 16384,
        "max_iters": 200, "fit_tol": 1e-4, "data_seed": 1002, "philox_seed": 2002}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=6)
    ap.add_argument("--skip-extras", action="store_true",
                    help="skip the studies that run after the timed regions (time to fit, the plain FP64 "
                         "GPU form, CP-ALS, the other workloads); used for profiler runs")
    ap.add_argument("--quality-sweep", action="store_true",
                    help="instead of the benchmark: the recovery study of Sec. 4.2 (Table 1 parameters), fit and "
                         "score of CPRAND-MIX and CPRAND over synthetic tensors, three starts per rank")
    ap.add_argument("--sweep-tensors", type=int, default=50, help="tensors per (size, C, eta) cell")
    ap.add_argument("--sweep-sizes", default="3x400,4x90", help="order x dimension of the sweep's tensors")
    ap.add_argument("--mix-shape", action="append", default=None, metavar="I1xI2x...:dtype",
                    help="instead of the benchmark: time the mixing call alone on this tensor shape "
                         "(float32 or bfloat16; repeatable), as the benchmark's extras do for other workloads")
    ap.add_argument("--mix-reps", type=int, default=4)
    ap.add_argument("--profile-grid", default=None, metavar="I1xI2x...:R:S:iters",
                    help="run CPRAND-MIX on the whole-GPU loop twice (the second call is the one to capture) "
                         "on a synthetic FP32 tensor of the headline's recipe and print its timings")
    ap.add_argument("--workload", choices=["1500", "400"], default="1500",
                    help="the decomposition a step runs (default: the 1500^3 headline workload)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "sm_max_mhz": 2070.0}, \
            "fallback"


def sm_count():
    import torch
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def opts_for(cb, w, **kw):
    """cpr_opts of a workload: its Philox seed, fit set size and stopping rules."""
    base = dict(seed=w["philox_seed"], fit_samples=w["P_hat"], max_iters=w["max_iters"],
                fit_tol=w.get("fit_tol", 1e-4), stall_iters=w.get("stall_iters", 0),
                noise_eta=w["eta"] if w.get("fit_tol", 1e-4) > 0 else -1.0)
    base.update(kw)
    return cb.cpr_default_opts(**base)


def make_workload(w, dtype_name="float32", device="cuda"):
    import torch
    from synth import make_problem
    return make_problem(tuple(w["dims"]), w["R"], C=w["congruence"], eta=w["eta"], seed=w["data_seed"],
                        dtype=getattr(torch, dtype_name), device=device)


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def exact_fit_gpu(X, dims, lam, factors, slab=64):
    """Exact fit 1 - ||X - X~|| / ||X|| (Sec. 4.2) of a CP model on the stored tensor, FP64 on the
    GPU, the model formed slab by slab along the last mode (out of every timed region)."""
    import torch
    N = len(dims)
    lam = lam.double()
    A = [a.double() for a in factors]
    Xf = X.reshape(-1)
    inner = int(np.prod(dims[:-1]))
    letters = "abcdefgh"[:N]
    spec = "r," + ",".join("%sr" % c for c in letters) + "->" + letters[::-1]
    err2 = torch.zeros((), dtype=torch.float64, device=X.device)
    nrm2 = torch.zeros((), dtype=torch.float64, device=X.device)
    for k0 in range(0, dims[-1], slab):
        k1 = min(dims[-1], k0 + slab)
        Xt = torch.einsum(spec, lam, *A[:-1], A[-1][k0:k1]).reshape(-1)
        xs = Xf[k0 * inner:k1 * inner].double()
        err2 += torch.sum((xs - Xt) ** 2)
        nrm2 += torch.sum(xs * xs)
    return 1.0 - math.sqrt(err2.item()) / math.sqrt(nrm2.item())


def dct2_fp64_(T, n, signs, slab=48):
    """In place: T <- T x_n (F_n D_n) with F_n the orthonormal DCT-II and D_n = diag(signs), in stock
    PyTorch FP64 operations: each fiber sign-flipped, reordered (even entries, then the odd ones
    reversed), transformed by torch.fft, rotated by exp(-i pi k / (2 I)) and scaled (the standard
    FFT form of the DCT-II); slab by slab along another mode to bound the temporary memory."""
    import torch
    I = T.shape[n]
    dev = T.device
    perm = torch.cat([torch.arange(0, I, 2, device=dev), torch.arange(1, I, 2, device=dev).flip(0)])
    k = torch.arange(I, device=dev, dtype=torch.float64)
    rot = torch.exp(-1j * math.pi * k / (2.0 * I))
    scale = torch.full((I,), math.sqrt(2.0 / I), dtype=torch.float64, device=dev)
    scale[0] = math.sqrt(1.0 / I)
    other = (n + 1) % T.dim()
    shape = [1] * T.dim()
    shape[n] = I
    for s0 in range(0, T.shape[other], slab):
        s1 = min(T.shape[other], s0 + slab)
        blk = T.narrow(other, s0, s1 - s0)
        v = (blk * signs.view(shape)).index_select(n, perm)
        V = torch.fft.fft(v, dim=n)
        blk.copy_((V * rot.view(shape)).real * scale.view(shape))
        del v, V


def plain_fp64_gpu(X, dims, w, seed, stop):
    """The plain FP64 GPU form the metric compares against: CPRAND-MIX (Alg. 5 with the orthonormal
    DCT-II and a random sign flip per mode, CPRAND on the mixed tensor, unmixing) in stock PyTorch
    FP64 operations on the same GPU, one decomposition, a host-side loop and stopping test (one
    device-to-host read of the sampled fit per outer iteration).  Its random draws come from torch's
    generator, so its trajectory differs from the library's; what is compared is the time to reach
    the same true fit.  Returns the wall time at the end of every outer iteration (from the call),
    the unmixing time, and the unmixed factors after every iteration."""
    import torch
    dev = X.device
    N = len(dims)
    R, S, Ph = w["R"], w["S"], w["P_hat"]
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Th = X.double().view(*dims[::-1]).permute(*range(N - 1, -1, -1))   # Th[i1, i2, ...], FP64
    ops = []
    for n, I in enumerate(dims):
        d = torch.randint(0, 2, (I,), generator=gen, device=dev).double() * 2.0 - 1.0
        dct2_fp64_(Th, n, d)
        ops.append(d)
    torch.cuda.synchronize()
    t_mix = time.perf_counter() - t0
    norm_x = torch.linalg.vector_norm(Th)
    P = float(np.prod(dims))
    A = [None] + [torch.rand(I, R, generator=gen, device=dev, dtype=torch.float64) for I in dims[1:]]
    lam = torch.ones(R, device=dev, dtype=torch.float64)
    fit_idx = [torch.randint(0, I, (Ph,), generator=gen, device=dev) for I in dims]
    fit_x = Th[tuple(fit_idx)]
    times, snaps, sfits = [], [], []
    last, best, stall = None, -float("inf"), 0
    for t in range(w["max_iters"]):
        for n in range(N):
            idx = [torch.randint(0, I, (S,), generator=gen, device=dev) for I in dims]
            Z = torch.ones(S, R, device=dev, dtype=torch.float64)
            for m in range(N):
                if m != n:
                    Z = Z * A[m][idx[m]]
            Xs = torch.movedim(Th, n, -1)[tuple(idx[m] for m in range(N) if m != n)]   # S x I_n
            G = Z.T @ Z
            At = torch.cholesky_solve(Z.T @ Xs, torch.linalg.cholesky(G))          # R x I_n
            lam = torch.linalg.vector_norm(At, dim=1)
            A[n] = (At / lam[:, None]).T
        model = torch.ones(Ph, R, device=dev, dtype=torch.float64)
        for m in range(N):
            model = model * A[m][fit_idx[m]]
        e = fit_x - model @ lam
        fit = 1.0 - (torch.sqrt(P * torch.mean(e * e)) / norm_x).item()
        times.append(time.perf_counter() - t0)
        sfits.append(fit)
        snaps.append((lam.clone(), [a.clone() for a in A]))
        if fit > best:
            best, stall = fit, 0
        else:
            stall += 1
        done = t + 1 >= w["max_iters"] or (w.get("stall_iters", 0) > 0 and stall >= w["stall_iters"])
        if w.get("fit_tol", -1) > 0 and last is not None and abs(fit - last) <= w["fit_tol"]:
            done = True
        last = fit
        if done or stop(t + 1):
            break
    del Th
    torch.cuda.empty_cache()
    a = time.perf_counter()
    out = [unmix_dct_fp64(Ah, d) for d, Ah in zip(ops, A)]
    torch.cuda.synchronize()
    t_unmix = time.perf_counter() - a
    return {"times": times, "t_unmix": t_unmix, "t_mix": t_mix, "ops": ops, "snaps": snaps, "sfits": sfits,
            "iters": len(times),
            "factors": out, "lam": lam}


def unmix_dct_fp64(Ah, signs):
    """A = D F^T Ahat (Alg. 5 unmixing) with the dense orthonormal DCT-II matrix, FP64."""
    import torch
    I = Ah.shape[0]
    k = torch.arange(I, device=Ah.device, dtype=torch.float64)
    F = torch.cos(math.pi * (2.0 * k[None, :] + 1.0) * k[:, None] / (2.0 * I)) * math.sqrt(2.0 / I)
    F[0] *= math.sqrt(0.5)
    return signs[:, None] * (F.T @ Ah)


def first_true_crossing(trace, target, true_fit_at, kmax):
    """The first outer iteration k (1-based) whose true fit reaches the target, found from the sampled
    fit trace (the paper's estimate is within about 1e-3 of the true fit) and confirmed with exact fits:
    start where the trace comes within 2e-3 of the target, walk up until the true fit reaches it, then
    down while the iteration before still does.  Returns (k, true fit at k) or (None, last true fit)."""
    k = next((i + 1 for i, f in enumerate(trace) if f >= target - 2e-3), None)
    if k is None:
        return None, None
    f = true_fit_at(k)
    while f < target and k < kmax:
        k += 1
        f = true_fit_at(k)
    if f < target:
        return None, f
    while k > 1:
        g = true_fit_at(k - 1)
        if g < target:
            break
        k, f = k - 1, g
    return k, f


def device_time(fn, reps=5):
    """Median device time (s) of fn() over reps calls after one warm-up call, CUDA events on the current
    stream."""
    import torch
    stream = torch.cuda.current_stream()
    fn()
    ts = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1) / 1e3)
    return float(np.median(ts))


def time_to_fit_study(cb, X, dims, w, run_trace, free_ws):
    """Time to reach F* - 1e-3 (F* = converged exact fit of the library's exact CP-ALS, Alg. 1, with FP64
    Gram / solve / fit, on the same stored tensor) for the library's CPRAND-MIX, the plain FP64 GPU
    form and the exact CP-ALS, all on this GPU.  run_trace: the sampled-fit trace of a rule-governed
    library run; free_ws(): releases the benchmark's workspace before the large comparison runs."""
    import torch
    R, S = w["R"], w["S"]
    out = {}
    # exact CP-ALS to convergence: F*
    trace = torch.zeros(w["max_iters"], dtype=torch.float64, device="cuda")
    als_opts = cb.cpr_default_opts(seed=w["philox_seed"], max_iters=w["max_iters"], fit_tol=1e-6,
                                   fit_trace_dev=trace.data_ptr())
    t0 = time.perf_counter()
    als = cb.cpr_cp_als(X, dims, R, opts=als_opts)
    torch.cuda.synchronize()
    als_wall = time.perf_counter() - t0
    als_trace = trace[:als["iters"]].cpu().numpy()
    f_star = exact_fit_gpu(X, dims, als["lam"], als["factors"])
    target = f_star - 1e-3
    out.update({"F_star": f_star, "F_star_source": "exact FP64-accumulate CP-ALS (library cpr_cp_als, Alg. 1) "
                "run to |dF| <= 1e-6 on the stored tensor, exact fit recomputed in FP64",
                "target_true_fit": target})
    als_ws = als["ws"]
    del als

    def als_fit_at(k):
        o = cb.cpr_cp_als(X, dims, R, opts=cb.cpr_default_opts(seed=w["philox_seed"], fixed_iters=k), ws=als_ws)
        return exact_fit_gpu(X, dims, o["lam"], o["factors"])
    k_als, f_als = first_true_crossing(als_trace, target, als_fit_at, len(als_trace))
    t_als = None
    if k_als is not None:
        t_als = device_time(lambda: cb.cpr_cp_als(X, dims, R, opts=cb.cpr_default_opts(
            seed=w["philox_seed"], fixed_iters=k_als), ws=als_ws), reps=3)
    out["cp_als_fp64"] = {"iters_to_converge": len(als_trace), "wall_s_to_converge": als_wall,
                          "s_per_iter": als_wall / max(1, len(als_trace)), "iters_to_target": k_als,
                          "true_fit_at_target_iter": f_als, "seconds_to_target": t_als,
                          "what": "cpr_cp_als: exact MTTKRP over the unfolding copies (FP32 products, FP64 "
                                  "folds), FP64 Gram-Hadamard Cholesky solve and exact fit, graph-captured loop"}
    del als_ws
    torch.cuda.empty_cache()

    # the library's CPRAND-MIX
    lib_ws = [None]

    def ours_fit_at(k):
        o = cb.cpr_cprand_mix(X, dims, R, S, opts=opts_for(cb, w, fixed_iters=k), ws=lib_ws[0])
        lib_ws[0] = o["ws"]
        return exact_fit_gpu(X, dims, o["lam"], o["factors"])
    k_ours, f_ours = first_true_crossing(run_trace, target, ours_fit_at, w["max_iters"])
    t_ours = None
    if k_ours is not None:
        run = cb.PreparedRun(X, dims, R, S, opts=opts_for(cb, w, fixed_iters=k_ours), mix=True)
        t_ours = device_time(run)
        del run
    lib_ws[0] = None
    torch.cuda.empty_cache()
    out["ours_s"], out["ours_iters"], out["ours_true_fit"] = t_ours, k_ours, f_ours
    out["ours_note"] = ("device time of the whole public call (norm, mixing, unfolding copies, iterations, "
                        "unmixing) with fixed_iters = the first iteration whose true fit reaches the target")

    # the plain FP64 GPU form (stock PyTorch)
    free_ws()
    plain = plain_fp64_gpu(X, dims, w, seed=w["philox_seed"], stop=lambda t: False)

    def plain_fit_at(k):
        lam_k, A_k = plain["snaps"][k - 1]
        return exact_fit_gpu(X, dims, lam_k, [unmix_dct_fp64(a, d) for a, d in zip(A_k, plain["ops"])])
    k_plain, f_plain = first_true_crossing(plain["sfits"], target, plain_fit_at, plain["iters"])
    t_plain = None if k_plain is None else plain["times"][k_plain - 1] + plain["t_unmix"]
    it_s = plain["times"][-1] - plain["times"][0]
    out["plain_fp64_gpu"] = {
        "iters": plain["iters"], "iters_to_target": k_plain, "true_fit_at_target_iter": f_plain,
        "seconds_to_target": t_plain, "mix_s": plain["t_mix"],
        "iters_per_s": (plain["iters"] - 1) / it_s if plain["iters"] > 1 and it_s > 0 else None,
        "what": "CPRAND-MIX in stock PyTorch FP64 ops (DCT-II mixing by torch.fft, index gathers, Cholesky "
                "solves), host-side loop and stopping test; wall time from the call"}
    del plain
    torch.cuda.empty_cache()
    out["plain_fp64_gpu_s"] = t_plain
    out["speedup_vs_plain_fp64_gpu"] = (t_plain / t_ours) if (t_plain and t_ours) else None
    out["speedup_vs_cp_als_fp64"] = (t_als / t_ours) if (t_als and t_ours) else None
    return out


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding as cb

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    w = WORKLOAD if args.workload == "1500" else dict(W400, workload="cprand_mix 400x400x400 fp32, R=10, S=230")
    dims = tuple(w["dims"])
    prob = make_workload(w, device=dev)
    X = prob.X
    del prob
    P = X.numel()
    opts = opts_for(cb, w, batch_index=rank)
    run = cb.PreparedRun(X, dims, w["R"], w["S"], opts=opts, mix=True)
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()

    # warm-up; the second warm-up step (events around the launches of the production kernels: the
    # mixing passes, the iteration loop, the rest) also finds the kernel with the most device time
    prod_mask = sum(1 << cb.KERNEL_CLASSES.index(c) for c in ("mix", "loop", "other"))
    run()
    cb.cpr_profile_begin(prod_mask)
    run()
    prof_all = cb.cpr_profile_end()
    for _ in range(max(0, args.warmup - 2)):
        run()
    torch.cuda.synchronize()
    dom = max(("mix", "loop"), key=lambda c: prof_all[c][0])

    # timed region 1: the production path, no profiler
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    iters, it_ms, launches, fits = 0, 0.0, 0, []
    for _ in range(args.steps):
        r = run()
        iters += r["iters"]
        it_ms += r["ms_iterate"]
        launches += r["kernel_launches"]
        fits.append(r["fit_est"])
        assert r["status"] == cb.OK, r
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    total_ms = ev0.elapsed_time(ev1)
    # timed region 2: the same steps with CUDA events around every launch of the dominant kernel class
    torch.cuda.synchronize()
    cb.cpr_profile_begin(1 << cb.KERNEL_CLASSES.index(dom))
    iters2 = 0
    for _ in range(args.steps):
        iters2 += run()["iters"]
    torch.cuda.synchronize()
    prof = cb.cpr_profile_end()
    clk = clocks.stop()   # sampled across both timed regions
    vals = torch.tensor([total_ms, it_ms, float(iters)], dtype=torch.float64, device=dev)
    if world > 1:
        tmax = vals[:2].clone()
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        isum = vals[2:].clone()
        dist.all_reduce(isum, op=dist.ReduceOp.SUM)
        total_ms_all, it_ms_all, iters_all = float(tmax[0]), float(tmax[1]), float(isum[0])
    else:
        total_ms_all, it_ms_all, iters_all = total_ms, it_ms, float(iters)
    value = iters_all / (it_ms_all / 1e3)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    Xh = X.cpu().pin_memory()
    R = w["R"]
    lam_h = torch.empty(R, dtype=torch.float64).pin_memory()
    fac_h = [torch.empty((d, R), dtype=torch.float64).pin_memory() for d in dims]
    h2d = P * X.element_size()
    d2h = 8 * (R + sum(d * R for d in dims))
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_iters = 0
    for _ in range(args.e2e_steps):
        X.copy_(Xh, non_blocking=True)
        r = run()
        e2e_iters += r["iters"]
        lam_h.copy_(run.lam, non_blocking=True)
        for fh, fd in zip(fac_h, run.factors):
            fh.copy_(fd, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    # the same steps as a stream of decompositions: the next step's tensor is copied from pinned host
    # memory on a second stream into a second device buffer while the current step decomposes (one
    # workspace; a buffer takes a new tensor once the call that read it has finished)
    Xb = torch.empty_like(X)
    bufs = [X, Xb]
    cs = torch.cuda.Stream(device=dev)
    main = torch.cuda.current_stream()
    arrived = [torch.cuda.Event(), torch.cuda.Event()]
    freed = [torch.cuda.Event(), torch.cuda.Event()]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pipe_iters = 0
    with torch.cuda.stream(cs):
        bufs[0].copy_(Xh, non_blocking=True)
        arrived[0].record(cs)
    for k in range(args.e2e_steps):
        cur = k & 1
        if k + 1 < args.e2e_steps:
            nxt = cur ^ 1
            if k >= 1:
                cs.wait_event(freed[nxt])      # the call of step k - 1 read this buffer
            with torch.cuda.stream(cs):
                bufs[nxt].copy_(Xh, non_blocking=True)
                arrived[nxt].record(cs)
        main.wait_event(arrived[cur])
        run.set_input(bufs[cur])
        r = run()
        freed[cur].record(main)
        pipe_iters += r["iters"]
        lam_h.copy_(run.lam, non_blocking=True)
        for fh, fd in zip(fac_h, run.factors):
            fh.copy_(fd, non_blocking=True)
    torch.cuda.synchronize()
    pipe_s = time.perf_counter() - t0
    run.set_input(X)
    del Xb
    torch.cuda.empty_cache()
    barrier()
    del Xh
    true_fit = exact_fit_gpu(X, dims, run.lam, run.factors)

    # the rule-governed run's sampled-fit trace (for the time-to-fit search)
    trace = torch.zeros(w["max_iters"], dtype=torch.float64, device=dev)
    run.opts.fit_trace_dev = trace.data_ptr()
    r = run()
    run_trace = trace[:r["iters"]].cpu().numpy()
    run.opts.fit_trace_dev = None

    pk, pk_src = peaks()
    roof = roofline(dom, prof, w, P, X.element_size(), iters2, pk, pk_src)
    mix_ms, mix_n = prof_all["mix"]
    out = {
        "metric": "ALS iters/s", "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms_all / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (Sec. 4.2 recipe, seeded)",
        "config": dict(w, parallelism="replicas" if world > 1 else "single GPU",
                       l2="input tensor %.1f GB > 129 MB L2, no flush" % (P * X.element_size() / 1e9)),
        "time_to_solution_ms": total_ms_all / args.steps,
        "iters_per_step": iters / args.steps,
        "phase_ms_per_step": {"iterate": it_ms / args.steps, "setup_mix_finish": (total_ms - it_ms) / args.steps},
        "us_per_outer_iteration": 1e3 * it_ms / max(1, iters),
        "fit_est_last": fits[-1], "true_fit_last": true_fit,
        "gpu_launches": int(launches) * (1 if world == 1 else world),
        "clocks": clk,
        "e2e": {"value": pipe_iters * (world if world > 1 else 1) / pipe_s, "unit": "iters/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "s_per_step": pipe_s / args.e2e_steps,
                "note": "a stream of %d decompositions through the public call, each tensor copied from pinned "
                        "host memory (H2D inside the timed region; the next tensor's copy on a second stream "
                        "overlaps the current decomposition), D2H of lambda and the factors after every call; "
                        "iterations / wall time" % args.e2e_steps,
                "serial": {"value": e2e_iters * (world if world > 1 else 1) / e2e_s, "s_per_step": e2e_s / args.e2e_steps,
                           "note": "the same with each step's copy, call and read-back one after another"}},
        "kernel_ms_per_step": {c: prof_all[c][0] for c in ("mix", "loop", "other")},
        "dominant_kernel": dom,
        "roofline": roof,
    }
    if mix_n > 0:
        mb = 2.0 * P * X.element_size()
        out["mixing"] = {"kernel": "k_mix_fft_ct (factored DCT-II, compiled stage plan)", "passes": mix_n,
                         "ms_per_pass": mix_ms / mix_n, "algorithmic_bytes_per_pass": mb,
                         "GBs": mb / (mix_ms / mix_n / 1e3) / 1e9,
                         "frac_of_hbm_peak": mb / (mix_ms / mix_n / 1e3) / 1e9 / pk["hbm_gbs"],
                         "peak_GBs": pk["hbm_gbs"], "peak_source": pk_src,
                         "note": "2 P b per pass (read + write); the last pass also writes the mode-N unfolding"}
    loop_ms, loop_n = prof_all["loop"]
    if loop_n > 0 and dom != "loop":
        out["loop_kernel"] = roofline("loop", {"loop": prof_all["loop"]}, w, P, X.element_size(),
                                      iters_per_launch_total=None, pk=pk, pk_src=pk_src)
    if rank == 0 and world == 1 and not args.skip_extras:
        def free_ws():
            run.ws = None
            torch.cuda.empty_cache()
        extras = {}
        try:
            extras["time_to_fit"] = time_to_fit_study(cb, X, dims, w, run_trace, free_ws)
        except Exception as exc:          # a study failing must not lose the bench line
            extras["time_to_fit"] = {"error": repr(exc)}
        del run
        torch.cuda.empty_cache()
        for name, fn in (("bf16", lambda: bf16_variant(cb, X, dims, w)),
                         ("workload_400cubed", lambda: other_workload(cb, W400)),
                         ("config_c_error", lambda: config_c_error(cb)),
                         ("gather", lambda: gather_bandwidth(cb, X, dims)),
                         ("mixing_other_shapes", lambda: mixing_shapes(cb)),
                         ("batch_64", lambda: batch_rate(cb)),
                         ("complex_form", lambda: complex_form_rate(cb))):
            try:
                extras[name] = fn()
            except Exception as exc:
                extras[name] = {"error": repr(exc)}
            torch.cuda.empty_cache()
        out.update(extras)
        if not args.no_cpu_baseline:
            try:
                out["cpu_baseline"] = cpu_baseline(X, dims, w)
            except Exception as exc:
                out["cpu_baseline"] = {"error": repr(exc)}
    if world > 1:
        dist.destroy_process_group()
    return out


def kernel_traffic(cls):
    """DRAM bytes per launch of a kernel class from the committed ncu summary, if the kernel's source is
    unchanged since the capture (file hash recorded next to the number); else None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        f = ln.split()
        if len(f) >= 3 and f[0] == cls and not ln.startswith("#"):
            src = os.path.join(ROOT, "paper_1701_06600_gb300", "csrc", f[2].split(":")[0])
            want = f[2].split(":")[1] if ":" in f[2] else ""
            if os.path.exists(src) and hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] == want:
                return float(f[1])
    return None


def roofline(cls, prof, w, P, b, iters_per_launch_total, pk, pk_src):
    """Roofline of one kernel class over a timed region: achieved = algorithmic bytes of a launch / its
    average CUDA-event duration.

    mix: one mode-n pass of the factored DCT-II reads the tensor and writes it once (the last pass also
    writes the mode-N unfolding copy): (2N + 1) P b / N bytes per launch on average.
    loop: the whole iteration loop of one decomposition (the whole-GPU kernel): per outer iteration and
    mode the sampled fibers, S I_n b bytes (the factor rows and the fit entries are L2-resident), plus
    the fit values once (P_hat 8 bytes); flops 2 S R I_n per mode for the contraction."""
    ms, n = prof[cls]
    if n <= 0:
        return None
    dims, R, S, Ph = w["dims"], w["R"], w["S"], w["P_hat"]
    N = len(dims)
    per_launch_s = ms / n / 1e3
    if cls == "mix":
        nbytes = (2.0 * N + 1.0) * P * b / N
        ach = nbytes / per_launch_s / 1e9
        return {"bound": "hbm", "kernel": "k_mix_fft_ct (factored DCT-II, stage plan compiled for I_n = %d)" % dims[0],
                "achieved": ach, "peak": pk["hbm_gbs"], "unit": "GB/s", "frac": ach / pk["hbm_gbs"],
                "peak_source": pk_src, "traffic": kernel_traffic("mix"), "per_launch_ms": ms / n,
                "algorithmic_bytes": nbytes, "launches": n}
    ipl = (iters_per_launch_total / n) if iters_per_launch_total else None
    rec = {"kernel": "k_grid_run (whole outer-iteration loop, one cooperative launch of one CTA per SM)",
           "per_launch_ms": ms / n, "launches": n, "peak": pk["hbm_gbs"], "unit": "GB/s", "bound": "hbm",
           "peak_source": pk_src, "traffic": kernel_traffic("loop")}
    if ipl:
        nbytes = ipl * sum(S * I * b for I in dims) + Ph * 8
        ach = nbytes / per_launch_s / 1e9
        rec.update({"achieved": ach, "frac": ach / pk["hbm_gbs"], "algorithmic_bytes": nbytes,
                    "algorithmic_flops": ipl * sum(2.0 * S * R * I for I in dims), "iters_per_launch": ipl,
                    "note": "latency-bound: per mode update three grid barriers and chains of dependent steps "
                            "(FP64 Gram, R x R inverse, FP64 refinement)"})
    return rec


def bf16_variant(cb, X, dims, w, steps=5):
    """The headline decomposition on the same tensor stored in BF16 (6.75 GB): FP32 accumulation, FP64
    R x R solve; iters/s of the iteration phase, the whole call, and the final exact fit on the BF16
    tensor."""
    import torch
    Xb = X.to(torch.bfloat16)
    run = cb.PreparedRun(Xb, dims, w["R"], w["S"], opts=opts_for(cb, w), mix=True)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    iters, it_ms = 0, 0.0
    for _ in range(steps):
        r = run()
        iters += r["iters"]
        it_ms += r["ms_iterate"]
    e1.record()
    torch.cuda.synchronize()
    f = exact_fit_gpu(Xb, dims, run.lam, run.factors)
    del run, Xb
    return {"what": "the headline workload stored in BF16", "iters_per_s": iters / (it_ms / 1e3),
            "ms_per_call": e0.elapsed_time(e1) / steps, "iters_per_call": iters / steps, "final_true_fit": f}


def other_workload(cb, w, steps=10):
    """Another configuration's decomposition (CPRAND-MIX with the paper's rules): iters/s and ms per call."""
    import torch
    prob = make_workload(w)
    dims = tuple(w["dims"])
    run = cb.PreparedRun(prob.X, dims, w["R"], w["S"], opts=opts_for(cb, w, noise_eta=w["eta"]), mix=True)
    run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    iters, it_ms = 0, 0.0
    for _ in range(steps):
        r = run()
        iters += r["iters"]
        it_ms += r["ms_iterate"]
    e1.record()
    torch.cuda.synchronize()
    f = exact_fit_gpu(prob.X, dims, run.lam, run.factors)
    return {"dims": list(dims), "R": w["R"], "S": w["S"], "iters_per_s": iters / (it_ms / 1e3),
            "us_per_outer_iteration": 1e3 * it_ms / iters, "ms_per_call": e0.elapsed_time(e1) / steps,
            "iters_per_call": iters / steps, "final_true_fit": f}


def config_c_error(cb, iters=5):
    """The 100^4 BF16 workload (R = 16, S = 450): per-iteration error of the library's CPRAND-MIX against
    the FP64 oracle's CPRAND (Alg. 3) run on the mixed tensor the GPU stored (both see the same BF16
    data and the same Philox draws): |F^_gpu - F^_oracle| per outer iteration and the relative
    Frobenius error of the (mixed-basis) factors after the last one."""
    import torch
    from oracle import cp, mixing
    from synth import to_oracle_array
    w = W100
    dims = tuple(w["dims"])
    prob = make_workload(w, dtype_name="bfloat16")
    trace = torch.zeros(iters, dtype=torch.float64, device="cuda")
    out = cb.cpr_cprand_mix(prob.X, dims, w["R"], w["S"], opts=cb.cpr_default_opts(
        seed=w["philox_seed"], fixed_iters=iters, fit_trace_dev=trace.data_ptr()))
    Th = to_oracle_array(cb.cpr_mix_tensor(prob.X, dims, seed=w["philox_seed"]), dims)
    ops = mixing.mixing_operators(w["philox_seed"], 0, dims)
    t0 = time.perf_counter()
    ref = cp.cprand(Th, w["R"], w["S"], seed=w["philox_seed"], rule=cp.StopRule(fixed_iters=iters))
    t_ref = time.perf_counter() - t0
    ref_f = mixing.unmix_factors(ref["factors"], ops)
    gpu_f = [a.cpu().numpy() for a in out["factors"]]
    fe = [float(np.linalg.norm(a - b) / np.linalg.norm(b)) for a, b in zip(gpu_f, ref_f)]
    return {"what": "100^4 BF16, R=16, S=450: library vs FP64 oracle on the GPU-stored mixed tensor",
            "abs_fit_error_per_iter": np.abs(trace.cpu().numpy() - ref["fits"]).tolist(),
            "factor_rel_error_after_last": fe, "oracle_s": t_ref}


def complex_form_rate(cb, iters=10):
    """The complex-transform form of CPRAND-MIX (Alg. 4) on the 400^3 workload: setup (norm, unitary-DFT
    mixing, copies) and device time per outer iteration over a fixed number of iterations, after one
    warm-up call; its host loop synchronizes once per iteration."""
    w = W400
    prob = make_workload(w)
    dims = tuple(w["dims"])
    opts = cb.cpr_default_opts(seed=w["philox_seed"], fixed_iters=1, fit_samples=w["P_hat"])
    warm = cb.cpr_cprand_mix_fft(prob.X, dims, w["R"], w["S"], opts=opts)
    opts = cb.cpr_default_opts(seed=w["philox_seed"], fixed_iters=iters, fit_samples=w["P_hat"])
    out = cb.cpr_cprand_mix_fft(prob.X, dims, w["R"], w["S"], opts=opts, ws=warm["ws"])
    del warm
    return {"what": "CPRAND-MIX with the unitary DFT (Alg. 4) on 400^3: complex mixed tensor, real factors, "
                    "stacked real least squares; host loop, one synchronization per outer iteration",
            "iters": out["iters"], "ms_setup": out["ms_setup"], "us_per_iter": 1e3 * out["ms_iterate"] / out["iters"],
            "fit_est_last": out["fit_est"]}


MIX_SHAPES = [((1500, 1500, 1500), "bfloat16"), ((400, 400, 400), "float32"),
              ((100, 100, 100, 100), "bfloat16"), ((100, 100, 100, 100), "float32"), ((1500, 1500, 200), "float32")]


def profile_grid_case(spec):
    """A small case of the whole-GPU loop for profilers: the headline workload's recipe (congruence 0.5,
    0.1% noise, data and Philox seeds) on the given dims, R and S, CPRAND-MIX with a fixed number of
    outer iterations on loop_path 5, called twice with one workspace."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding as cb
    dims_s, R, S, iters = spec.split(":")
    w = dict(WORKLOAD, dims=[int(v) for v in dims_s.split("x")], R=int(R), S=int(S))
    prob = make_workload(w)
    dims = tuple(w["dims"])
    opts = opts_for(cb, w, fixed_iters=int(iters), loop_path=cb.LOOP_GRID)
    first = cb.cpr_cprand_mix(prob.X, dims, w["R"], w["S"], opts=opts)
    out = cb.cpr_cprand_mix(prob.X, dims, w["R"], w["S"], opts=opts, ws=first["ws"])
    return {"profile_grid": spec, "status": out["status"], "iters": out["iters"], "ms_setup": out["ms_setup"],
            "us_per_iter": 1e3 * out["ms_iterate"] / max(out["iters"], 1), "fit_est": out["fit_est"]}


def mixing_shapes(cb, reps=4, shapes=None):
    """The mixing preprocess alone (cpr_mix_tensor: the operator tables, then one factored-DCT pass per
    mode) on other tensors: device time per call by CUDA events over `reps` calls after one warm-up
    call, against N passes x (P b read + P b written)."""
    import torch
    pk, pk_src = peaks()
    res = []
    for dims, dt in (shapes or MIX_SHAPES):
        P = int(np.prod(dims))
        X = torch.randn(P, device="cuda", dtype=getattr(torch, dt))
        cb.cpr_mix_tensor(X, dims, seed=7)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            Y = cb.cpr_mix_tensor(X, dims, seed=7)
            del Y
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        nbytes = len(dims) * 2 * P * X.element_size()
        res.append({"dims": list(dims), "dtype": dt, "ms_per_call": ms, "passes": len(dims),
                    "GBs": nbytes / (ms / 1e3) / 1e9, "frac_of_hbm_peak": nbytes / (ms / 1e3) / 1e9 / pk["hbm_gbs"]})
        del X
        torch.cuda.empty_cache()
    return {"what": "cpr_mix_tensor per call (operator tables + N passes), algorithmic bytes N x 2 P b",
            "peak_GBs": pk["hbm_gbs"], "peak_source": pk_src, "shapes": res}


def batch_rate(cb, B=64):
    """The batching workload: B independent 3-way FP32 tensors (every dim uniform in [64, 512], rank
    uniform in [4, 32], congruence uniform in [0, 0.9], 1% noise), CPRAND-MIX with S = round(10 R ln R)
    (at least R) and the paper's stopping rules, all in one batched call.  Device time of the call by
    CUDA events, after a warm-up call with the same workspace."""
    import torch
    from synth import batch_problem_specs, make_problem
    specs = batch_problem_specs(1004, B=B)
    Xs, dims_l, Rs, Ss, opts = [], [], [], [], []
    for b, sp in enumerate(specs):
        prob = make_problem(sp["dims"], sp["R"], C=sp["C"], eta=0.01, seed=1000 * (b + 1) + 4,
                            dtype=torch.float32, device="cuda")
        Xs.append(prob.X)
        dims_l.append(sp["dims"])
        Rs.append(sp["R"])
        Ss.append(max(sp["R"], int(math.floor(10.0 * sp["R"] * math.log(sp["R"]) + 0.5))))
        opts.append(cb.cpr_default_opts(seed=2004, batch_index=b, noise_eta=0.01))
    _, ws = cb.cpr_cprand_batched(Xs, dims_l, Rs, Ss, opts, mix=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    outs, ws = cb.cpr_cprand_batched(Xs, dims_l, Rs, Ss, opts, mix=True, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    iters = sum(o["iters"] for o in outs)
    nbytes = sum(int(np.prod(d)) * 4 for d in dims_l)
    del Xs, ws
    return {"what": "%d independent CPRAND-MIX decompositions in one batched call (dims U[64,512], R U[4,32], "
                    "C U[0,0.9], 1%% noise, S = round(10 R ln R), paper stopping rules)" % B,
            "tensor_GB": nbytes / 1e9, "ms_per_call": ms, "decompositions_per_s": B / (ms / 1e3),
            "outer_iters_total": iters, "outer_iters_per_s": iters / (ms / 1e3),
            "phase_ms": {"setup": outs[0]["ms_setup"], "iterate": outs[0]["ms_iterate"],
                         "finish": outs[0]["ms_finish"]},
            "all_ok": all(o["status"] == cb.OK for o in outs)}


def gather_bandwidth(cb, X, dims, S=1 << 16, reps=10):
    """The fiber gather (Sec. 3.2) on its own: S sampled mode-1 fibers of the headline tensor (contiguous,
    16-byte vectors; 2^16 fibers of 1500 FP32 = 393 MB read and written per launch) and S sampled mode-3
    fibers of the standard layout (stride I_1 I_2: one 32-byte sector per element), CUDA events over
    `reps` launches each."""
    import torch
    pk, pk_src = peaks()
    out = {}
    for mode, label in ((0, "contiguous"), (len(dims) - 1, "strided")):
        Im = dims[mode]
        _, off = cb.cpr_sample_indices(dims, mode, S, seed=7, b=0, t=0, device=X.device)
        xs = torch.empty(Im * S, dtype=X.dtype, device=X.device)
        cb.cpr_gather_fibers(X, dims, mode, off, out=xs)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            cb.cpr_gather_fibers(X, dims, mode, off, out=xs)
        e1.record(stream)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / reps
        useful = Im * S * X.element_size()
        out[label] = {"mode": mode + 1, "fibers": S, "fiber_len": Im, "us_per_launch": sec * 1e6,
                      "useful_read_GBs": useful / sec / 1e9, "read_write_GBs": 2 * useful / sec / 1e9,
                      "frac_of_hbm_peak": 2 * useful / sec / 1e9 / pk["hbm_gbs"]}
        del xs
    return dict(out, peak_GBs=pk["hbm_gbs"], peak_source=pk_src,
                kernel="k_gather_contig (one warp per fiber, 16-byte vectors) / k_gather_only (strided)")


def oracle_host_views(X, dims):
    """The stored tensor on the host for the oracle, once per mode: the mode-n unfolding stored
    column-major (built on the GPU, copied down), viewed as an array indexed (i_1, ..., i_N) whose mode-n
    unfolding the oracle forms without copying.  The values stay FP32 (the oracle's arithmetic on them
    is FP64)."""
    N = len(dims)
    Xd = X.view(*dims[::-1])                       # C-order axes: mode N-1 first
    views = []
    for n in range(N):
        modes = [m for m in range(N - 1, -1, -1) if m != n] + [n]
        U = Xd.permute(*[N - 1 - m for m in modes]).contiguous().cpu().numpy()
        shapeF = [dims[n]] + [dims[m] for m in range(N) if m != n]
        U = np.reshape(U.ravel(), shapeF, order="F")  # i_n fastest, then the other modes in order
        views.append(np.moveaxis(U, 0, n))
    return views


def blas_threads(n):
    """Set the thread count of the BLAS NumPy loaded (OpenBLAS builds export a setter); returns True if
    it could be set."""
    import ctypes
    names = ("openblas_set_num_threads64_", "openblas_set_num_threads", "scipy_openblas_set_num_threads64_",
             "scipy_openblas_set_num_threads")
    libs = set()
    try:
        for ln in open("/proc/self/maps"):
            if "openblas" in ln.lower() and ".so" in ln:
                libs.add(ln.split()[-1])
    except OSError:
        return False
    ok = False
    for path in libs:
        try:
            h = ctypes.CDLL(path)
        except OSError:
            continue
        for nm in names:
            f = getattr(h, nm, None)
            if f is not None:
                f(int(n))
                ok = True
    return ok


def oracle_iterations(views, dims, w, iters, t0=0, factors=None):
    """iters outer iterations of the oracle's CPRAND (Alg. 3: per mode the sampled multi-indices, SKR,
    the fiber gather, the QR least squares; then the sampled fit), timed one by one."""
    from oracle import cp, streams
    R, S, seed = w["R"], w["S"], w["philox_seed"]
    N = len(dims)
    if factors is None:
        factors = [np.zeros((dims[0], R))] + [streams.init_factor(seed, 0, n, dims[n], R) for n in range(1, N)]
    fit_idx = streams.fit_sample_indices(seed, 0, w["P_hat"], dims)
    fit_x = views[0][tuple(fit_idx[:, m] for m in range(N))].astype(np.float64)
    normT = 1.0   # the fit's value is not used here; its cost is
    times, lam = [], None
    for t in range(t0, t0 + iters):
        a = time.perf_counter()
        for n in range(N):
            idx = streams.ls_sample_indices(seed, 0, t, n, S, dims)
            factors[n], lam = cp.cprand_update(views[n], factors, n, idx)
        cp.sampled_fit(fit_x, lam, factors, fit_idx, normT, int(np.prod(dims)))
        times.append(time.perf_counter() - a)
    return times, factors


def oracle_mix_pass(views, dims, w, slab=8):
    """One mixing pass of the oracle (the dense mode-1 product with F_1 D_1, Alg. 5) on a slab of the
    tensor (slab mode-N indices), scaled to the whole tensor."""
    from oracle import cp, mixing
    U = mixing.mixing_operators(w["philox_seed"], 0, dims[:1])[0]
    T = np.asarray(views[0][..., :slab], dtype=np.float64)
    a = time.perf_counter()
    cp.mode_product(T, U, 0)
    dt = time.perf_counter() - a
    return dt * dims[-1] / slab


def cpu_baseline(X, dims, w, iters=3):
    """The oracle as it stands on this host's cores: 3 outer iterations of its CPRAND on the headline
    tensor (the mode-n gathers read host copies of the mode-n unfoldings) and one mixing pass timed on a
    slab and scaled, with BLAS on every core and, when the BLAS thread count can be set, on one."""
    views = oracle_host_views(X, dims)
    res = {"kind": "oracle", "unit": "iters/s", "cores": os.cpu_count()}
    t_all, fac = oracle_iterations(views, dims, w, iters)
    mix_all = oracle_mix_pass(views, dims, w)
    res.update({"value": len(t_all) / sum(t_all), "iter_s": float(np.mean(t_all)), "mix_pass_s": mix_all,
                "sample": "%d outer iterations of the FP64 NumPy oracle's CPRAND on the 1500^3 tensor (iterations "
                          "1..3 of the run; host copies of the mode unfoldings) and one mode-1 mixing pass on a "
                          "1500x1500x8 slab scaled x%d, BLAS on all %d cores" % (iters, dims[-1] // 8, os.cpu_count())})
    if blas_threads(1):
        t1, _ = oracle_iterations(views, dims, w, iters)
        res["single_thread"] = {"value": len(t1) / sum(t1), "iter_s": float(np.mean(t1)),
                                "mix_pass_s": oracle_mix_pass(views, dims, w), "cores": 1}
        blas_threads(os.cpu_count())
    else:
        res["single_thread"] = {"unavailable": "the BLAS NumPy loaded has no thread-count setter"}
    del views
    return res


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on the headline workload (tensor synthesized on the GPU exactly
    as for the library's arm, then copied to the host); one step = one outer iteration of the oracle's
    CPRAND, the first `warmup` discarded."""
    if rank != 0:
        return None
    import torch
    w = WORKLOAD
    dims = tuple(w["dims"])
    torch.cuda.set_device(0)
    prob = make_workload(w, device="cuda")
    views = oracle_host_views(prob.X, dims)
    del prob
    torch.cuda.empty_cache()
    times, _ = oracle_iterations(views, dims, w, args.warmup + args.steps)
    kept = times[args.warmup:]
    value = len(kept) / sum(kept)
    mix = oracle_mix_pass(views, dims, w)
    sample = ("%d outer iterations (after %d discarded) of the FP64 NumPy oracle's CPRAND on the 1500^3 tensor, "
              "mode gathers from host unfolding copies, BLAS on %d cores; mixing pass %.1f s (slab, scaled)"
              % (len(kept), args.warmup, os.cpu_count(), mix))
    return {"impl": "reference", "metric": "ALS iters/s", "value": value, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (Sec. 4.2 recipe, seeded)",
            "config": dict(WORKLOAD, parallelism="host cores"),
            "cpu_baseline": {"value": value, "unit": "iters/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def score_assignment(true_factors, est_factors):
    """Score of eq. (score) (Sec. 4.2): mean over the true components of the product over the modes of
    the cosines with the matched estimated component, maximized over matchings; the best matching of
    the pair-score matrix by linear assignment."""
    import numpy as np
    from scipy.optimize import linear_sum_assignment
    S = None
    for A, B in zip(true_factors, est_factors):
        An = A / np.linalg.norm(A, axis=0, keepdims=True)
        Bn = B / np.linalg.norm(B, axis=0, keepdims=True)
        C = An.T @ Bn
        S = C if S is None else S * C
    rows, cols = linear_sum_assignment(-S)
    return float(np.mean(S[rows, cols]))


def exact_fit_device(X, dims, lam, factors):
    """1 - ||X - X~|| / ||X|| in FP64 on the device (X flat column-major, any order N <= 5)."""
    import torch
    N = len(dims)
    letters = "abcde"[:N]
    spec = "r," + ",".join("%sr" % c for c in letters) + "->" + letters[::-1]
    Xt = torch.einsum(spec, lam.double(), *[A.double() for A in factors]).reshape(-1)
    Xd = X.double()
    return 1.0 - torch.linalg.vector_norm(Xd - Xt).item() / torch.linalg.vector_norm(Xd).item()


def run_quality_sweep(args):
    """The recovery study of Sec. 4.2 with the parameters of its Table 1: tensors of order 3 (400^3) and
    order 4 (90^4) with R_true = 5 collinear components (C in {0.5, 0.9}) and noise eta in {0.01, 0.1};
    CPRAND-MIX and CPRAND with R in {5, 6} (S = 80, 108), three random starts each, the stopping rules
    of Sec. 4.2 (P_hat = 2^14); per cell the median and quartiles of the exact fit and of the score, the
    iterations, and the decompositions per second of the batched calls (the 6 starts of a tensor and
    method in one call)."""
    import numpy as np
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_1701_06600_gb300 import binding as cb
    from synth import make_problem
    torch.cuda.set_device(0)
    sizes = [tuple(int(v) for v in z.split("x")) for z in args.sweep_sizes.split(",")]
    cells, t_calls, n_dec = [], 0.0, 0
    for si, (N, I) in enumerate(sizes):
        dims = (I,) * N
        for ci, (C, eta) in enumerate([(0.5, 0.01), (0.5, 0.1), (0.9, 0.01), (0.9, 0.1)]):
            res = {(m, R): {"fit": [], "score": [], "iters": []} for m in ("cprand_mix", "cprand") for R in (5, 6)}
            for t in range(args.sweep_tensors):
                prob = make_problem(dims, 5, C=C, eta=eta, seed=100000 + 10000 * si + 1000 * ci + t,
                                    dtype=torch.float32, device="cuda")
                Rs = [5, 5, 5, 6, 6, 6]
                Ss = [80, 80, 80, 108, 108, 108]
                opts = [cb.cpr_default_opts(seed=7000 + t, batch_index=q, noise_eta=eta) for q in range(6)]
                for m, mix in (("cprand_mix", True), ("cprand", False)):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    outs, _ = cb.cpr_cprand_batched([prob.X] * 6, [dims] * 6, Rs, Ss, opts, mix=mix)
                    torch.cuda.synchronize()
                    t_calls += time.perf_counter() - t0
                    n_dec += 6
                    for q, o in enumerate(outs):
                        est = [A.cpu().numpy() for A in o["factors"]]
                        r = res[(m, Rs[q])]
                        r["fit"].append(exact_fit_device(prob.X, dims, o["lam"], o["factors"]))
                        r["score"].append(score_assignment(prob.factors, est))
                        r["iters"].append(o["iters"])
                del prob
            for (m, R), r in res.items():
                q = lambda v, p: float(np.percentile(v, p))
                cells.append({"order": N, "dim": I, "C": C, "eta": eta, "method": m, "R": R, "runs": len(r["fit"]),
                              "fit_q25_med_q75": [q(r["fit"], 25), q(r["fit"], 50), q(r["fit"], 75)],
                              "score_q25_med_q75": [q(r["score"], 25), q(r["score"], 50), q(r["score"], 75)],
                              "iters_median": q(r["iters"], 50)})
    return {"study": "recovery of Sec. 4.2 (Table 1 parameters): exact fit and score at termination",
            "tensors_per_cell": args.sweep_tensors, "decompositions": n_dec,
            "decompositions_per_s": n_dec / t_calls if t_calls > 0 else None,
            "seconds_in_calls": t_calls, "data": "synthetic (Sec. 4.2 recipe, seeded)", "cells": cells}




def main():
    args = parse()
    rank, world, local_rank = dist_env()
    if args.quality_sweep:
        if rank == 0:
            print(json.dumps(run_quality_sweep(args)))
        return
    if args.profile_grid:
        if rank == 0:
            print(json.dumps(profile_grid_case(args.profile_grid)))
        return
    if args.mix_shape:
        if rank == 0:
            import __graft_entry__
            __graft_entry__.build()
            from paper_1701_06600_gb300 import binding as cb
            shapes = []
            for spec in args.mix_shape:
                dims, _, dt = spec.partition(":")
                shapes.append((tuple(int(v) for v in dims.split("x")), dt or "float32"))
            print(json.dumps({"mixing_shapes": mixing_shapes(cb, reps=args.mix_reps, shapes=shapes)}))
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local_rank)
    if rank == 0 and out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
