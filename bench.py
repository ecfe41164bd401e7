#!/usr/bin/env python
"""Benchmark: FSE lost-blocks/s (and Mpix/s, % roofline) on one GB300.

Default workload: the 256-image batch -- images of uneven seeded sizes from
256x256 to 2048x1536, 5-50 % of their 4x4 (F=32, K=100) or 8x8 (F=64, K=200)
blocks lost, supports truncated at the image borders, ~2.8 M lost blocks,
both DFT classes in one call (the largest single-GPU workload).  A step is one
full pass of the method (tiling, lost-block enumeration and ordering, staging,
DFT, K iterations, model evaluation, write-back) over that input.
--workload tiled_1024 (one 1024^2 image, 16 tiles of Algorithm 1, F=64,
K=200), defects_4k (3840x2160 defect-pixel image, F=32) and plain_64 select
the other workloads.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 (launched by torch.distributed.run): every rank extrapolates its own
copy of the workload on its own GPU (replicas; the method's units are
independent, no data exchange); value = all ranks' blocks / slowest rank.
"--impl reference" times the FP64 CPU oracle on a bounded sample instead.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
SMEM_BYTES_PER_CLK_SM = 128  # shared-memory bandwidth per SM per clock
BYTES_PER_BIN_ITER = 8       # the gathered complex FP32 W(k-u) value

# DRAM bytes per launch of the dominant kernel (for the 256-image batch: per
# step, both iteration kernels) from an ncu capture of the same workload,
# reported only while the kernel source is the one that was captured.
CAPTURED_TRAFFIC = {"kernel_src_sha256_16": "85c9502f29abcf82",
                    "tiled_1024": 8358272, "defects_4k": 58633216 + 1468373,
                    "batch_256": 1298921088 + 280961056 + 3084604128 + 338152672}
CAPTURED_TRAFFIC_CLASS = {"batch_256": {"k_exec_f32_64": 1298921088 + 280961056,
                                        "k_exec_f32_32": 3084604128 + 338152672}}


def captured_traffic(workload):
    import hashlib
    src = os.path.join(ROOT, "paper_2207_00238_gb300", "csrc", "fse_kernels.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if h != CAPTURED_TRAFFIC["kernel_src_sha256_16"]:
        return None
    return CAPTURED_TRAFFIC.get(workload)


def captured_class_traffic(workload, kernel):
    if captured_traffic(workload) is None:
        return None
    return CAPTURED_TRAFFIC_CLASS.get(workload, {}).get(kernel)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed steps (default: ~6 s of steps)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batch_256")
    ap.add_argument("--mode", default="dag", choices=["dag", "levels", "per_block"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="oracle seconds per CPU-baseline leg (all cores, then one core)")
    ap.add_argument("--no-per-block", action="store_true", help="skip the per-block launch baseline")
    ap.add_argument("--arena-mb", type=int, default=4096)
    ap.add_argument("--serve-requests", type=int, default=2000,
                    help="measured requests of the serving leg (0 = skip)")
    ap.add_argument("--f64-warps", type=int, default=0, choices=[0, 2, 4, 5, 6, 8])
    ap.add_argument("--f32-layout", type=int, default=0, choices=[0, 1, 2, 3, 4])
    ap.add_argument("--no-tma", action="store_true", help="stage supports with plain loads")
    ap.add_argument("--no-graph", action="store_true", help="time direct launches instead of graph replay")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--root-window", type=int, default=-1,
                    help="FSE_OPT_ROOT_WINDOW (-1: library default)")
    ap.add_argument("--class-launch", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="FSE_OPT_CLASS_LAUNCH (-1: library default / autotuned)")
    ap.add_argument("--study", default=None, choices=[None, "overlap", "tiling"],
                    help="run a study instead of the benchmark (one JSON line per result)")
    ap.add_argument("--order", default=None, choices=[None, "phased", "raster", "independent"],
                    help="processing order override (default: the workload's, PHASED)")
    ap.add_argument("--ctas-per-sm", type=int, default=0)
    return ap.parse_args()


def workload(name):
    from paper_2207_00238_gb300 import synth
    return synth.CONFIGS[name]()


def describe(name, jobs):
    p = jobs[0]["params"]
    if len(jobs) > 1:
        return {"workload": name, "images": len(jobs), "pixels": int(sum(j["image"].size for j in jobs)),
                "blocks": sorted({j["params"]["block"] for j in jobs}),
                "fft": sorted({j["params"]["fft"] for j in jobs}), "order": p["order"]}
    d = {"workload": name, "images": len(jobs),
         "size": f"{jobs[0]['image'].shape[1]}x{jobs[0]['image'].shape[0]}" if len(jobs) == 1 else "mixed",
         "block": p["block"], "border": p["border"], "fft": p["fft"], "K": p["K"],
         "n_tiles": p["n_tiles"], "overlap": p["overlap"], "order": p["order"],
         "rho": p["rho"], "delta": p["delta"], "gamma": p["gamma"]}
    return d


def max_over_ranks(seconds, dist=None, device=None):
    """Slowest rank's time (replicas: every rank runs the whole workload)."""
    if dist is None:
        return seconds
    import torch
    t = torch.tensor([seconds], dtype=torch.float64,
                     device=device if device is not None and device.type == "cuda" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, steps, slowest_s):
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    return world * units_per_rank * steps / slowest_s


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# CPU oracle (baseline leg and reference arm)
# ---------------------------------------------------------------------------
def oracle_blocks_per_s(job, seconds, max_blocks=None, threads=0):
    """The oracle on the first blocks of one job (processing order, tile 0
    first) for about `seconds`: (blocks/s, blocks, seconds, threads used)."""
    import oracle
    oracle.build()
    p = job["params"]
    kw = dict(block=p["block"], border=p["border"], fft=p["fft"], K=p["K"], rho=p["rho"],
              delta=p["delta"], gamma=p["gamma"], order=p["order"], n_tiles=p["n_tiles"],
              overlap=p["overlap"], threads=threads)
    cores = threads if threads > 0 else oracle.threads()
    if max_blocks is None:
        probe = max(cores, 4)
        t = time.perf_counter()
        r = oracle.fse_image(job["image"], job["mask"], max_blocks=probe, **kw)
        dt = time.perf_counter() - t
        per = dt / max(r["stats"]["processed"], 1)
        max_blocks = max(probe, int(seconds / per))
    t = time.perf_counter()
    r = oracle.fse_image(job["image"], job["mask"], max_blocks=max_blocks, **kw)
    dt = time.perf_counter() - t
    n = r["stats"]["processed"]
    return n / dt, n, dt, cores


def oracle_mix_rate(jobs, class_blocks, seconds, threads=0):
    """Oracle throughput on the workload's mix of DFT classes: each class
    present is timed on the first blocks of its first job (about
    seconds / classes each) and the per-class rates r_k are combined with the
    workload's block shares f_k as 1 / sum_k f_k / r_k.  Returns
    (blocks/s, description, threads)."""
    shares = {32: class_blocks[0], 64: class_blocks[1]}
    total = sum(shares.values())
    present = [F for F in (32, 64) if shares[F] > 0]
    inv, parts, cores = 0.0, [], 0
    for F in present:
        job = next(j for j in jobs if j["params"]["fft"] == F)
        rate, n, dt, cores = oracle_blocks_per_s(job, seconds / len(present), threads=threads)
        inv += (shares[F] / total) / rate
        parts.append(f"F={F}: first {n} blocks of its first image, {dt:.1f} s, {rate:.1f} blocks/s, "
                     f"{100 * shares[F] / total:.1f} % of the workload's blocks")
    return 1.0 / inv, "; ".join(parts), cores


def class_blocks_of(jobs):
    """Lost blocks per DFT class (F=32, F=64) counted from the masks and tilings."""
    import oracle
    out = [0, 0]
    for j in jobs:
        p = j["params"]
        b = p["block"]
        rc, tiles = oracle.plan_tiles(j["image"].shape[1], j["image"].shape[0], p["n_tiles"], p["overlap"])
        for (x, y, w, h, ex, ey, ew, eh) in tiles:
            m = j["mask"][ey:ey + eh, ex:ex + ew]
            nby, nbx = -(-eh // b), -(-ew // b)
            pad = np.zeros((nby * b, nbx * b), np.uint8)
            pad[:eh, :ew] = m
            out[0 if p["fft"] == 32 else 1] += int((pad.reshape(nby, b, nbx, b).max(axis=(1, 3)) > 0).sum())
    return out


def run_reference(args, rank, world):
    if rank != 0:
        return
    jobs = workload(args.workload)
    steps = args.steps if args.steps is not None else 5
    cb = class_blocks_of(jobs)
    # ~150 s of oracle work for the whole run, whatever K and W
    per_step = max(0.1, min(30.0, 150.0 / max(steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_mix_rate(jobs, cb, per_step)
    rates, desc, cores = [], "", 0
    for _ in range(steps):
        r, desc, cores = oracle_mix_rate(jobs, cb, per_step)
        rates.append(r)
    value = len(rates) / sum(1.0 / r for r in rates)
    tot_t = steps * per_step
    sample = (f"per step: {desc}; FP64 spatial-domain oracle, {cores} threads")
    line = {"metric": "FSE lost-blocks/s", "value": value, "unit": "blocks/s", "n_gpus": world,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1000 * tot_t / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": describe(args.workload, jobs), "impl": "reference",
            "cpu_baseline": {"value": value, "unit": "blocks/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "blocks/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# serving leg: Poisson arrivals into the continuous-batching server
# ---------------------------------------------------------------------------
def serve_leg(fse, device, n_measured, n_warm=200, rate_hz=200.0, n_capacity=300, lookahead=48):
    """The serving workload through the continuous-batching server.

    Poisson leg: n_warm + n_measured fresh requests (each drawn anew: size
    log-uniform 128^2 .. 7680x4320, 1-30 % of the 8x8 blocks lost, K in
    100..200, pixels cropped from two seeded 7680x4320 images at a drawn
    position) arrive at their drawn times (mean 200/s); a producer thread builds
    each request's buffers ahead of its arrival.  Reported: achieved request
    rate, served lost blocks/s and Mpix/s, p50/p99 latency (submit ->
    completion seen by the server).
    Capacity leg: n_capacity further fresh requests, built before timing,
    submitted back to back; served lost blocks/s and Mpix/s from the first
    submit to the last completion."""
    import queue as _queue
    import threading
    from paper_2207_00238_gb300 import synth
    textures = synth.serving_textures()
    n = n_warm + n_measured
    specs = list(synth.serving_requests(textures, n_requests=n, rate_hz=rate_hz))
    ctx = fse.Context(device, arena_bytes=256 << 20)
    ctx.set_option(fse.OPT_SERVER_CLASSES, 2)  # every serving request is F = 64
    srv = fse.Server(ctx, arena_bytes=24 << 30, max_queue=4096, max_resident=256)
    try:
        ready = _queue.Queue(maxsize=lookahead)

        def producer():
            for _, spec in specs:
                ready.put(synth.materialise(textures, spec))

        tickets = [None] * n
        lat = np.zeros(n)
        got = threading.Semaphore(0)

        def waiter():
            for i in range(n):
                got.acquire()
                lat[i] = srv.wait(tickets[i], timeout_ms=300000)["exec_ms"] * 1e-3  # submit -> done

        pt = threading.Thread(target=producer, daemon=True)
        wt = threading.Thread(target=waiter, daemon=True)
        pt.start()
        wt.start()
        t0 = time.perf_counter()
        lag = 0.0
        t_meas = None
        for k, (arr, _) in enumerate(specs):
            job = ready.get()
            now = time.perf_counter() - t0
            if arr > now:
                time.sleep(arr - now)
            else:
                lag = max(lag, now - arr) if k >= n_warm else lag
            if k == n_warm:
                t_meas = time.perf_counter()
            out = np.empty_like(job["image"])
            tickets[k] = srv.submit(job["image"], job["mask"], out, job["params"])
            got.release()
        wt.join()
        t_end = time.perf_counter()
        lat = lat[n_warm:]
        meas = [sp for _, sp in specs[n_warm:]]
        px = sum(sp["W"] * sp["H"] for sp in meas)
        blocks = sum(int(sp["flags"].sum()) for sp in meas)
        wall = t_end - t_meas
        poisson = {"requests": n_measured, "warmup_requests": n_warm, "offered_rate_hz": rate_hz,
                   "achieved_rate_hz": n_measured / wall, "lost_blocks_per_s": blocks / wall,
                   "mpix_per_s": px / wall / 1e6, "p50_ms": float(np.percentile(lat, 50) * 1e3),
                   "p99_ms": float(np.percentile(lat, 99) * 1e3), "mean_ms": float(lat.mean() * 1e3),
                   "max_submit_lag_ms": lag * 1e3}
        # capacity: requests submitted back to back
        cap_specs = [sp for _, sp in synth.serving_requests(textures, n_requests=n_capacity,
                                                            seed=synth.SEED_BASE + 8)]
        jobs = [synth.materialise(textures, sp) for sp in cap_specs]
        outs = [np.empty_like(j["image"]) for j in jobs]
        t0 = time.perf_counter()
        tk = [srv.submit(j["image"], j["mask"], o, j["params"]) for j, o in zip(jobs, outs)]
        lat = np.array([srv.wait(t, timeout_ms=300000)["exec_ms"] * 1e-3 for t in tk])
        wall = time.perf_counter() - t0
        capacity = {"requests": n_capacity,
                    "lost_blocks_per_s": sum(int(sp["flags"].sum()) for sp in cap_specs) / wall,
                    "mpix_per_s": sum(sp["W"] * sp["H"] for sp in cap_specs) / wall / 1e6,
                    "seconds": wall, "p50_ms": float(np.percentile(lat, 50) * 1e3)}
    finally:
        srv.close()
        ctx.close()
    return {"poisson": poisson, "capacity": capacity,
            "requests": "fresh per request: sizes, loss flags, K and crop position drawn; pixels "
                        "cropped from two seeded 7680x4320 images; F=64, B=16, b=8"}


# ---------------------------------------------------------------------------
# studies (not part of the default run)
# ---------------------------------------------------------------------------
def paper_scale_jobs(loss):
    """6024x4024 stand-in for the paper's test images (Sec. IV) with `loss` of
    the 4x4 blocks lost (bursts and isolated), b=4, B=14, F=32, K=100."""
    from paper_2207_00238_gb300 import synth
    W, H = 6024, 4024
    rng = synth.Rng(synth.SEED_BASE + 60)
    img = synth.image(W, H, rng, structure=True)
    nb = ((W + 3) // 4) * ((H + 3) // 4)
    mask, _ = synth.block_mask(W, H, 4, int(round(loss * nb)), synth.Rng(synth.SEED_BASE + 61))
    return img, mask


def run_study(args):
    import torch
    import paper_2207_00238_gb300 as fse
    from paper_2207_00238_gb300 import synth
    fse.build()
    dev = torch.device("cuda", 0)
    ctx = fse.Context(0, arena_bytes=16 << 30)
    stream = torch.cuda.current_stream(dev).cuda_stream

    def run(img_d, msk_d, out_d, p, reps=2):
        job = fse.make_job(img_d, msk_d, out_d, p)
        st = None
        for _ in range(reps):
            st = ctx.extrapolate([job], stream=stream, stats=True)
        return st

    def psnr_all(out, img):
        d = out.astype(np.float64) - img.astype(np.float64)
        return 10 * np.log10(255.0 ** 2 / np.mean(d * d))

    def ssim_all(out, img):
        # mean SSIM (Wang, Bovik, Sheikh, Simoncelli 2004): Gaussian window
        # sigma 1.5 (11 x 11), C1 = (0.01 * 255)^2, C2 = (0.03 * 255)^2
        from scipy.ndimage import gaussian_filter
        x, y = out.astype(np.float64), img.astype(np.float64)
        g = lambda z: gaussian_filter(z, 1.5, truncate=3.5)
        mx, my = g(x), g(y)
        sxx, syy, sxy = g(x * x) - mx * mx, g(y * y) - my * my, g(x * y) - mx * my
        c1, c2 = (0.01 * 255) ** 2, (0.03 * 255) ** 2
        m = ((2 * mx * my + c1) * (2 * sxy + c2)) / ((mx * mx + my * my + c1) * (sxx + syy + c2))
        return float(m.mean())

    if args.study == "overlap":
        for loss in (0.14, 0.62):
            img, mask = paper_scale_jobs(loss)
            img_d = torch.from_numpy(img).to(dev)
            msk_d = torch.from_numpy(mask).to(dev)
            out_d = torch.empty_like(img_d)
            base = synth.params(4, 14, 32, 100)
            st = run(img_d, msk_d, out_d, dict(base, n_tiles=1, overlap=0))
            o = out_d.cpu().numpy()
            ref, ref_s = psnr_all(o, img), ssim_all(o, img)
            print(json.dumps({"study": "overlap", "loss": loss, "n_tiles": 1, "overlap": 0,
                              "psnr_db": ref, "ssim": ref_s, "lost_blocks": st["lost_blocks"],
                              "exec_ms": st["exec_ms"]}), flush=True)
            for d in (0, 1, 2, 4, 8, 16, 24, 32, 48, 64, 96):
                st = run(img_d, msk_d, out_d, dict(base, n_tiles=32, overlap=d))
                o = out_d.cpu().numpy()
                ps, ss = psnr_all(o, img), ssim_all(o, img)
                print(json.dumps({"study": "overlap", "loss": loss, "n_tiles": 32, "overlap": d,
                                  "psnr_db": ps, "delta_vs_untiled_db": ps - ref, "ssim": ss,
                                  "delta_ssim_vs_untiled": ss - ref_s,
                                  "lost_blocks": st["lost_blocks"], "exec_ms": st["exec_ms"]}),
                      flush=True)
    else:
        for W, H in ((1024, 480), (6024, 4024)):
            for N in (2, 4, 8, 16, 22, 32, 64):
                row = {"study": "tiling", "W": W, "H": H, "n_tiles": N, "overlap": 32}
                for tiling in ("alg1", "vertical"):
                    t = fse.plan_tiles(W, H, N, 32, tiling)
                    row[f"processed_over_image_{tiling}"] = float((t[:, 6] * t[:, 7]).sum()) / (W * H)
                print(json.dumps(row), flush=True)
        img, mask = paper_scale_jobs(0.62)
        img_d = torch.from_numpy(img).to(dev)
        msk_d = torch.from_numpy(mask).to(dev)
        out_d = torch.empty_like(img_d)
        for tiling in ("alg1", "vertical"):
            st = run(img_d, msk_d, out_d, synth.params(4, 14, 32, 100, n_tiles=32, overlap=32,
                                                       tiling=tiling), reps=3)
            print(json.dumps({"study": "tiling_gpu", "tiling": tiling, "n_tiles": 32, "overlap": 32,
                              "loss": 0.62, "lost_blocks": st["lost_blocks"],
                              "exec_ms": st["exec_ms"], "device_ms": st["device_ms"]}), flush=True)
    ctx.close()


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def describe_tuning(trace):
    """The autotuner's trace: the fastest candidate per class (the one it
    applied) and, for a mix, the class launch it chose."""
    best = {}
    for c, code, k, ms in trace:
        c = int(c)
        if c not in best or ms < best[c][3]:
            best[c] = (c, int(code), int(k), ms)
    out = {"candidates": len(trace), "chosen": {}}
    for c, (_, code, k, ms) in sorted(best.items()):
        if c < 0:
            out["class_launch"] = {0: "sequential", 1: "concurrent, F=64 first",
                                   2: "concurrent, F=32 first"}[code]
        else:
            out["chosen"][c] = {"layout": code // 10, "unroll": code % 10, "ctas_per_sm": k, "ms": round(ms, 4)}
    return out


def per_block_baseline(fse, ctx, cjobs, sptr, max_blocks=6000):
    """Blocks/s of the plain per-block launch (FSE_EXEC_PER_BLOCK: one kernel
    launch per lost block, in processing order) on the first jobs of the
    workload holding up to max_blocks blocks, and of the batched persistent
    launch on the same jobs."""
    sub, nb = [], 0
    for j in cjobs:
        sub.append(j)
        st = ctx.extrapolate(sub, stream=sptr, stats=True)
        nb = st["lost_blocks"]
        if nb >= max_blocks:
            break
    st_dag = ctx.extrapolate(sub, stream=sptr, stats=True)
    ctx.exec_mode("per_block")
    try:
        st_pb = ctx.extrapolate(sub, stream=sptr, stats=True)
    finally:
        ctx.exec_mode("dag")
    return {"value": st_pb["lost_blocks"] / (st_pb["device_ms"] / 1000.0), "unit": "blocks/s",
            "launches": st_pb["launches"],
            "batched_same_sample": st_dag["lost_blocks"] / (st_dag["device_ms"] / 1000.0),
            "sample": f"the first {len(sub)} images of the workload, {st_pb['lost_blocks']} lost blocks"}


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.study:
        return run_study(args)

    import torch
    import paper_2207_00238_gb300 as fse

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    fse.build()
    jobs = workload(args.workload)
    if args.order:
        for j in jobs:
            j["params"] = dict(j["params"], order=args.order)
    dev = torch.device("cuda", local)
    ctx = fse.Context(local, arena_bytes=args.arena_mb << 20)
    ctx.exec_mode(args.mode)
    if args.f64_warps:
        ctx.set_option(fse.OPT_F64_WARPS, args.f64_warps)
    if args.f32_layout:
        ctx.set_option(fse.OPT_F32_LAYOUT, args.f32_layout)
    if args.no_tma:
        ctx.set_option(fse.OPT_TMA_STAGING, 0)
    if args.ctas_per_sm:
        ctx.set_option(fse.OPT_CTAS_PER_SM, args.ctas_per_sm)
    if args.class_launch >= 0:
        ctx.set_option(fse.OPT_CLASS_LAUNCH, args.class_launch)
    if args.root_window >= 0:
        ctx.set_option(fse.OPT_ROOT_WINDOW, args.root_window)
    keep, cjobs, pix = [], [], 0
    for j in jobs:
        img = torch.from_numpy(j["image"]).to(dev)
        msk = torch.from_numpy(j["mask"]).to(dev)
        out = torch.empty_like(img)
        keep += [img, msk, out]
        cjobs.append(fse.make_job(img, msk, out, j["params"]))
        pix += img.numel()
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    tuned = None
    if (not args.no_autotune and not args.f64_warps and not args.f32_layout and not args.ctas_per_sm
            and args.class_launch < 0 and args.mode == "dag"):
        trace = ctx.autotune(cjobs, stream=sptr, reps=3)
        tuned = describe_tuning(trace)
    # one counted pass: blocks per step, bin-iterations per step (per class)
    st = ctx.extrapolate(cjobs, stream=sptr, stats=True)
    blocks, core_blocks, bins = st["lost_blocks"], st["core_lost_blocks"], st["bin_iterations"]
    cls_blocks, cls_bins = st["class_blocks"], st["class_bin_iterations"]
    launches_per_step = st["launches"]
    step_est = st["device_ms"] / 1000.0
    steps = args.steps if args.steps is not None else int(min(400, max(10, 6.0 / max(step_est, 1e-4))))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    # the iteration kernels' durations: a pass of their own without graph
    # replay (kernel-timing events are not captured into the graph)
    ctx.set_option(fse.OPT_KERNEL_TIMING, 1)
    ctx.kernel_times()
    for i in range(max(3, min(steps, 50))):
        flush.fill_(float(i))
        ctx.extrapolate(cjobs, stream=sptr, stats=False)
    torch.cuda.synchronize()
    cls_ms = ctx.class_times()
    kern_ms = ctx.kernel_times()
    ctx.set_option(fse.OPT_KERNEL_TIMING, 0)
    # the timed steps replay the call's CUDA graph (captured on the first call)
    if not args.no_graph:
        ctx.set_option(fse.OPT_USE_GRAPH, 1)
    for _ in range(args.warmup):
        ctx.extrapolate(cjobs, stream=sptr, stats=False)
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                    if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    clocks.start()
    time.sleep(0.3)
    for i in range(steps):
        flush.fill_(float(i))  # evict the inputs from L2 between steps
        starts[i].record(stream)
        ctx.extrapolate(cjobs, stream=sptr, stats=False)
        ends[i].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    ctx.set_option(fse.OPT_USE_GRAPH, 0)
    total_s = max_over_ranks(sum(step_ms) / 1000.0, dist, dev)
    value = whole_job_rate(blocks, world, steps, total_s)
    mpix = world * pix * steps / total_s / 1e6

    # roofline of the iteration kernels: algorithmic shared-memory bytes (8 B of
    # W per bin-iteration) / event-timed duration, for the call's whole
    # execution (the classes run concurrently) and per class
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    f_max = float(peaks.get("sm_max_mhz", 2070.0))
    peak_gbs = SMEM_BYTES_PER_CLK_SM * sms * f_max * 1e6 / 1e9
    kmean = statistics.mean(kern_ms) if kern_ms else float("nan")
    achieved = bins * BYTES_PER_BIN_ITER / (kmean / 1000.0) / 1e9
    names = {0: "k_exec_f32_32", 1: "k_exec_f32_64"}
    per_class = {}
    for k in (0, 1):
        if cls_blocks[k] <= 0:
            continue
        ms_k = statistics.mean(r[k] for r in cls_ms) if cls_ms else float("nan")
        ach_k = cls_bins[k] * BYTES_PER_BIN_ITER / (ms_k / 1000.0) / 1e9 if cls_bins[k] > 0 else None
        per_class[names[k]] = {"blocks_per_launch": cls_blocks[k], "bin_iterations_per_launch": cls_bins[k],
                               "kernel_ms": ms_k, "achieved": ach_k,
                               "frac": ach_k / peak_gbs if ach_k else None,
                               "traffic": captured_class_traffic(args.workload, names[k])}
    roof = {"bound": "alu", "pipe": "shared-memory (LSU) pipe, 128 B/clk/SM",
            "achieved": achieved, "peak": peak_gbs, "unit": "GB/s", "frac": achieved / peak_gbs,
            "traffic": captured_traffic(args.workload),
            "traffic_note": ("DRAM bytes per launch (ncu; for a mixed batch the sum over its class "
                             "launches); the kernel's bound is on chip"),
            "kernel": "+".join(names[k] for k in (0, 1) if cls_blocks[k] > 0),
            "kernel_ms": kmean, "bin_iterations_per_launch": bins,
            "peak_basis": f"derived: {SMEM_BYTES_PER_CLK_SM} B/clk/SM x {sms} SMs x {f_max:.0f} MHz",
            "per_class": per_class}
    if len(per_class) > 1:
        roof["per_class_note"] = ("with FSE_OPT_CLASS_LAUNCH concurrent the classes share the GPU, so a "
                                  "class's fraction counts its own launch span against the whole GPU")
    if clk:
        roof["frac_at_observed_clock"] = achieved / (SMEM_BYTES_PER_CLK_SM * sms * clk["sm_mhz"] * 1e6 / 1e9)
    # HBM side of the step: support staging and write-back are fused into the
    # iteration kernel; their algorithmic bytes per image are the image and the
    # mask read once and the output written once (3 B per pixel)
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    hbm_bytes = 3 * pix
    hbm_gbs = hbm_bytes / (statistics.mean(step_ms) / 1000.0) / 1e9
    hbm = {"algorithmic_bytes_per_step": hbm_bytes, "achieved": hbm_gbs, "peak": hbm_peak, "unit": "GB/s",
           "frac": hbm_gbs / hbm_peak, "dram_bytes_per_launch": captured_traffic(args.workload),
           "peak_basis": "measured copy bandwidth" if "hbm_gbs" in peaks else "fallback",
           "note": "staging and write-back are latency-bound parts of the on-chip-bound iteration kernel"}

    # the plain per-block launch (one launch per lost block, in processing
    # order) on a bounded sample of the workload, against the same sample in
    # the batched persistent launch
    per_block = None
    if not args.no_per_block and args.mode == "dag":
        per_block = per_block_baseline(fse, ctx, cjobs, sptr)

    # end to end through the host-buffer entry point (copies timed)
    e2e = None
    if not args.no_e2e:
        hj, hkeep = [], []
        for j in jobs:
            himg = torch.from_numpy(j["image"]).pin_memory()
            hmsk = torch.from_numpy(j["mask"]).pin_memory()
            hout = torch.empty_like(himg).pin_memory()
            hkeep += [himg, hmsk, hout]
            hj.append(fse.make_job(himg.numpy(), hmsk.numpy(), hout.numpy(), j["params"]))
        e2e_ctx = ctx  # the tuned context: a user tunes once, then calls with host buffers
        for _ in range(args.warmup):
            e2e_ctx.extrapolate_host(hj, stream=sptr)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(steps):
            e2e_ctx.extrapolate_host(hj, stream=sptr)
        torch.cuda.synchronize()
        e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
        e2e = {"value": world * blocks * steps / e2e_s, "unit": "blocks/s",
               "h2d_bytes_per_step": 2 * pix, "d2h_bytes_per_step": pix,
               "mpix_per_s": world * pix * steps / e2e_s / 1e6}

    serving = None
    if args.serve_requests > 0:
        serving = serve_leg(fse, local, args.serve_requests)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = [cls_blocks[0], cls_blocks[1]]
        v, desc, cores = oracle_mix_rate(jobs, cb, args.cpu_seconds)
        v1, desc1, _ = oracle_mix_rate(jobs, cb, args.cpu_seconds, threads=1)
        cpu = {"value": v, "unit": "blocks/s", "cores": cores, "kind": "oracle",
               "sample": f"{desc} (FP64 spatial-domain projections, {cores} threads)",
               "one_core": {"value": v1, "unit": "blocks/s", "cores": 1, "sample": desc1}}
    if rank == 0:
        cfg = describe(args.workload, jobs)
        cfg.update({"parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                    "exec_mode": args.mode, "staging": "loads" if args.no_tma else "tma where many F=32 blocks (auto)", "launch": "direct" if args.no_graph else "cuda graph replay", "autotune": tuned, "l2": "flushed between steps (256 MB write)",
                    "lost_blocks_per_step": blocks, "core_lost_blocks_per_step": core_blocks,
                    "bin_iterations_per_step": bins})
        line = {"metric": "FSE lost-blocks/s", "value": value, "unit": "blocks/s", "n_gpus": world,
                "steps": steps, "warmup": args.warmup,
                "ms_per_step": 1000 * total_s / steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": cfg, "mpix_per_s": mpix, "roofline": roof, "hbm": hbm, "cpu_baseline": cpu,
                "e2e": e2e, "clocks": clk, "gpu_launches": launches_per_step * steps,
                "plain_per_block": per_block, "serving": serving}
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
