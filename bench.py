"""Throughput of the whole hot path (views -> ORB -> matching) on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--plain-steps P]

Workload (one step = one image pair through match_pair, all stages): a
1024x768 uint8 synthetic textured pair under extreme tilt (absolute tilt 75
deg, transition tilt near 85 deg, noise sigma 2), 43 simulated views per image
(t = sqrt2^k, k <= 5, phi step 72/t), ORB with 8 levels at scale 1.2, 1000
keypoints per view, FAST threshold 20, rBRIEF-256, brute-force Hamming match of
the pooled descriptors with ratio 4/5.  Every rank processes its own pairs
(weak scaling, no collective on the data path).

The JSON line reports image pairs/s (views/s = 86 x pairs/s beside it), with
inputs resident in HBM; `e2e` is the same metric through the C ABI with the
images copied from pinned host memory and the accepted pairs copied back inside
the timed region.  `roofline` is for the stage that takes longest (the view
simulation: FP32 arithmetic bound), `rooflines` for it, the matcher (tensor
cores, fp8 dense peak) and the FAST/Harris/NMS and pyramid stages (HBM, on
their algorithmic bytes); `cpu_baseline` is the CPU oracle timed on one whole
pair with every host core (and with one).  `--impl reference` times the CPU
oracle on whole pairs as the reference arm.
"""
from __future__ import annotations

import argparse
import gc
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

H, W, KMAX, LEVELS, NFEAT, THR = 768, 1024, 5, 8, 1000, 20
LARGE_H, LARGE_W, LARGE_KMAX, LARGE_NFEAT = 3072, 4096, 6, 2000
DS = 0.5                   # scale step of the coarse stage (s = 1 + k DS)
WORKLOAD = "asift_pair_1024x768_extreme_tilt_43views_orb8x1000"
SM_COUNT = 152
POPC_PER_SM_CLK = 16       # 32-bit population count: 16 results / clock / SM
POPC_PER_PAIR = 8          # a 256-bit Hamming distance = 8 x popc(32-bit xor)


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def pair_seed(rank: int, i: int) -> int:
    """Seed of pair i of a rank: every rank processes its own pairs."""
    return 2000 + 97 * rank + i


def max_over_ranks(x: float, dist, device) -> float:
    """The largest x over the job's ranks (x itself without a process group):
    the job takes as long as its slowest rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput: each of `world` ranks processed units_per_rank
    units, the slowest of them in `seconds`."""
    return world * units_per_rank / seconds


def _pair(rank: int, i: int):
    from paper_2503_03479_gb300 import synth
    return synth.pair_extreme_tilt(seed=pair_seed(rank, i))


def _mixed_one(seed: int, index: int):
    from paper_2503_03479_gb300 import synth
    p = synth.mixed_pair(seed, index)
    return p.img1, p.img2


def _large_one(seed: int, index: int):
    """A 4096x3072 pair of the large extreme-tilt batch, the 1024x768 pair's
    recipe at this size: a 2x canonical texture seen by image 1 with absolute
    tilt t1 and by image 2 through a homography with local tilt t2 along the
    perpendicular direction, plus N(0, 2^2) noise; t1, t2 ~ U[2, 1/cos 83 deg]."""
    from paper_2503_03479_gb300 import synth
    p = synth.large_pair(seed, index, LARGE_H, LARGE_W)
    return p.img1, p.img2


def large_batch(n_pairs: int, seed: int):
    import multiprocessing as mp
    if n_pairs <= 0:
        return []
    workers = max(1, min(16, os.cpu_count() or 1, n_pairs))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.starmap(_large_one, [(seed, i) for i in range(n_pairs)])


def mixed_batch(n_pairs: int, seed: int):
    """The mixed-size batch (480x360 .. 1920x1080, absolute tilts 30-85 deg),
    generated in a spawn pool before CUDA is initialised."""
    import multiprocessing as mp
    if n_pairs <= 0:
        return []
    workers = max(1, min(16, os.cpu_count() or 1, n_pairs))
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.starmap(_mixed_one, [(seed, i) for i in range(n_pairs)])


class _Nvml:
    """Read-only NVML queries through ctypes (clocks, throttle reasons, power)."""

    SM = 1                                   # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, cuda_index: int):
        import ctypes as C
        self.C = C
        L = C.CDLL("libnvidia-ml.so.1")
        if L.nvmlInit_v2() != 0:
            raise OSError("nvmlInit failed")
        self.L = L
        self.h = C.c_void_p()
        bus = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(cuda_index)
            bus = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        except Exception:
            bus = None
        ok = bus is not None and L.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), C.byref(self.h)) == 0
        if not ok and L.nvmlDeviceGetHandleByIndex_v2(cuda_index, C.byref(self.h)) != 0:
            raise OSError("no NVML device handle")
        self._reasons = getattr(L, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            L.nvmlDeviceGetCurrentClocksThrottleReasons

    def sample(self):
        C = self.C
        sm, mx, pw, rs = C.c_uint(), C.c_uint(), C.c_uint(), C.c_ulonglong()
        self.L.nvmlDeviceGetClockInfo(self.h, self.SM, C.byref(sm))
        self.L.nvmlDeviceGetMaxClockInfo(self.h, self.SM, C.byref(mx))
        self.L.nvmlDeviceGetPowerUsage(self.h, C.byref(pw))
        self._reasons(self.h, C.byref(rs))
        return sm.value, mx.value, pw.value / 1000.0, rs.value

    def close(self):
        try:
            self.L.nvmlShutdown()
        except Exception:
            pass


class ClockSampler:
    """SM clocks and throttle reasons sampled during the timed region: NVML
    polled every 5 ms from a thread (a region of 20 steps lasts only ~60 ms),
    else nvidia-smi every 50 ms (its first line awaited before the region)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int, period_s: float = 0.005):
        self.gpu = gpu
        self.period = period_s
        self.p = None
        self.nvml = None
        self.samples = []                    # (sm MHz, max MHz, watts, reason names)
        self._buf = []
        self._first = threading.Event()
        self._stop = threading.Event()
        self._t = None
        self.source = None

    def _poll(self):
        while not self._stop.is_set():
            try:
                sm, mx, pw, rs = self.nvml.sample()
                self.samples.append((float(sm), float(mx), pw,
                                     sorted(n for b, n in _Nvml.REASONS.items() if rs & b)))
            except Exception:
                pass
            self._stop.wait(self.period)

    def _read(self):
        for l in self.p.stdout:
            if l.strip():
                self._buf.append(l)
                self._first.set()

    def __enter__(self):
        try:
            self.nvml = _Nvml(self.gpu)
            self.nvml.sample()
            self.source = "nvml, every 5 ms"
            self._t = threading.Thread(target=self._poll, daemon=True)
            self._t.start()
            return self
        except Exception:
            self.nvml = None
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.p = None
            return self
        self.source = "nvidia-smi, every 50 ms"
        self._t = threading.Thread(target=self._read, daemon=True)
        self._t.start()
        self._first.wait(timeout=5.0)
        self._start = len(self._buf)
        return self

    def __exit__(self, *a):
        if self.nvml is not None:
            self._stop.set()
            self._t.join(timeout=5)
            self.nvml.close()
            return
        if self.p is None:
            return
        n = len(self._buf)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            self.p.wait()
        self._t.join(timeout=5)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self._buf[self._start:n]:
            f = [x.strip() for x in l.split(",")]
            try:
                self.samples.append((float(f[1]), float(f[2]), float(f[3]),
                                     [nm for nm, v in zip(names, f[5:9]) if v.lower() == "active"]))
            except (ValueError, IndexError):
                continue

    def summary(self):
        if not self.samples:
            return None
        reasons = sorted({r for s in self.samples for r in s[3]})
        return {"sm_mhz": statistics.median(s[0] for s in self.samples),
                "sm_max_mhz": max(s[1] for s in self.samples), "reasons": reasons,
                "samples": len(self.samples), "power_w_max": max(s[2] for s in self.samples),
                "source": self.source}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- rooflines
FP32_LANES_PER_SM = 128    # FP32 FMA lanes per SM (one FMA = 2 flops)
FP8_PER_BF16 = 2.0         # nominal dense fp8 / bf16 tensor rate (4.5 / 2.25 PFLOP/s)


def warp_flops(v) -> float:
    """Algorithmic flops of one simulated view (Eq. (2)-(4)), multiply-add = 2:
    the 6 x 6 Lanczos-3 interpolation of the rotation at every canvas pixel
    (when phi != 0 or s != 1), the (2K+1)-tap Gaussian along the tilt axis at every canvas
    pixel and the 6-tap Lanczos-3 resampling of the tilt at every view pixel
    (both when t > 1).  Weight evaluation, staging and the mask are not counted."""
    canvas = v.Wr * v.Hr
    f = 0.0
    if v.phi_deg != 0.0 or v.s != 1.0:
        f += 36 * canvas
    if v.t > 1.0:
        f += (2 * v.K + 1) * canvas + 6 * v.Wv * v.Hv
    return 2.0 * f


def warp_roofline(views, n_images: int, ms: float, peaks: dict) -> dict:
    f_clk = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
    peak = SM_COUNT * FP32_LANES_PER_SM * 2 * f_clk / 1e12
    flops = n_images * sum(warp_flops(v) for v in views)
    return _alu_roofline(flops, ms, peak, f_clk)


def _alu_roofline(flops: float, ms: float, peak: float, f_clk: float) -> dict:
    achieved = flops / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": "warp_band_kernel (+ tilt_filter_kernel, convert_images_kernel)", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
            "flops_per_launch": flops,
            "peak_source": f"derived: {SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 FMA/clk x 2 x {f_clk/1e6:.0f} MHz"}


def match_roofline(sizes, ms: float, tensor: bool, peaks: dict) -> dict:
    """Matcher roofline over the step's pairs: `sizes` holds (n1, n2) of each
    pair the steps cycle through and `ms` is the mean stage time over those
    steps, so the work per step is the mean of n1 x n2."""
    pairs = statistics.mean(n1 * n2 for n1, n2 in sizes)
    if tensor:
        bf16 = peaks.get("bf16_tflops")
        peak = (bf16 or 1900.0) * FP8_PER_BF16
        flops = 2.0 * 256 * pairs                    # one +-1 dot product of length 256 per pair
        achieved = flops / (ms / 1e3) / 1e12
        src = (f"fp8 = measured bf16 {bf16} TFLOP/s x nominal fp8/bf16 ratio {FP8_PER_BF16}" if bf16 else
               f"fp8 = fallback bf16 1900 TFLOP/s x nominal ratio {FP8_PER_BF16}")
        return {"bound": "tensor", "kernel": "hamming_tc_kernel (+ expand_pm1_kernel, merge_kernel)",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "flops_per_launch": flops, "peak_source": src}
    f_clk = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
    peak = SM_COUNT * POPC_PER_SM_CLK * f_clk / 1e12
    achieved = pairs * POPC_PER_PAIR / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": "hamming_top2_kernel (+ merge_kernel)", "achieved": achieved,
            "peak": peak, "unit": "Tpopc/s", "frac": achieved / peak, "traffic": None,
            "peak_source": f"derived: {SM_COUNT} SMs x {POPC_PER_SM_CLK} popc/clk x {f_clk/1e6:.0f} MHz"}


def orb_level_bytes(A, views, n_levels: int):
    """Algorithmic bytes of the two HBM-bound ORB stages for one image's views:
    detect reads 1 B per pyramid pixel (every level); the pyramid reads the
    parent level's image (1 B per parent pixel) and writes the level's image
    (1 B per pixel) for every level >= 1.  A view's footprint mask is 0/1 on
    an interval of each row at every level, so its pyramid is the row hulls
    (a few bytes per row), not a second image plane."""
    det = pyr = 0
    for v in views:
        for l in range(n_levels):
            n = A.level_size(v.Wv, l) * A.level_size(v.Hv, l)
            det += n
            if l:
                pyr += A.level_size(v.Wv, l - 1) * A.level_size(v.Hv, l - 1) + n
    return det, pyr


def hbm_roofline(kernel: str, nbytes: float, ms: float, peaks: dict) -> dict:
    peak = peaks.get("hbm_gbs")
    src = "measured copy bandwidth (MEASURED_PEAKS.json)" if peak else "fallback 6800 GB/s"
    peak = peak or 6800.0
    achieved = nbytes / (ms / 1e3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "bytes_per_launch": nbytes, "peak_source": src}


def _sha256(path: str) -> str:
    import hashlib
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()


def profiled_traffic(kernel: str):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    `kernel` from the table in profiles/roofline_traffic.md, used only while
    the kernel's source file still has the sha256 recorded beside the number;
    None otherwise."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    for l in lines:
        f = [x.strip() for x in l.strip().strip("|").split("|")]
        if len(f) >= 4 and f[0] == kernel:
            src, sha, nbytes = f[1], f[2], f[3]
            try:
                if _sha256(os.path.join(ROOT, src)) == sha:
                    return float(nbytes)
            except (OSError, ValueError):
                return None
    return None


def match_engines(A, ctx, dd1, dd2, stream, reps: int = 5):
    """Times hamming_match on the pair's two pools with each engine (inputs
    and outputs in device memory, CUDA events on the stream) and checks that
    both return the same bytes."""
    import ctypes as C
    import torch
    q = torch.from_numpy(np.ascontiguousarray(dd1)).cuda()
    t = torch.from_numpy(np.ascontiguousarray(dd2)).cuda()
    nq, nt = q.shape[0], t.shape[0]
    L = ctx.L
    ws = torch.zeros(L.hamming_workspace_size(nq, nt), dtype=torch.uint8, device="cuda")
    res, outs = {}, {}
    for name, eng in (("tensor_cores", A.MATCH_TENSOR_CORES), ("cuda_cores", A.MATCH_CUDA_CORES)):
        if eng == A.MATCH_TENSOR_CORES and ctx.match_engine != A.MATCH_TENSOR_CORES:
            continue
        ctx.set_match_engine(eng)
        out = torch.zeros(max(nq, 1) * 8, dtype=torch.uint8, device="cuda")
        acc = torch.zeros(max(nq, 1), dtype=torch.uint8, device="cuda")
        nacc = torch.zeros(1, dtype=torch.int32, device="cuda")
        args = (ctx._ctx, C.c_void_p(q.data_ptr()), nq, None, C.c_void_p(t.data_ptr()), nt, None, 4, 5,
                C.c_void_p(out.data_ptr()), C.c_void_p(acc.data_ptr()), C.c_void_p(nacc.data_ptr()),
                C.c_void_p(ws.data_ptr()), ws.numel(), C.c_void_p(stream.cuda_stream))
        for _ in range(2):
            assert L.hamming_match(*args) == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        h0 = time.perf_counter()
        for _ in range(reps):
            L.hamming_match(*args)
        h1 = time.perf_counter()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name + "_host_enqueue_ms"] = (h1 - h0) * 1e3 / reps
        res[name + "_ms"] = ms
        res[name + "_tops"] = 2.0 * 256 * nq * nt / (ms / 1e3) / 1e12
        outs[name] = (out.cpu().numpy().tobytes(), int(nacc.item()))
    ctx.set_match_engine(A.MATCH_AUTO)
    if len(outs) == 2:
        res["identical"] = outs["tensor_cores"] == outs["cuda_cores"]
        res["speedup"] = res["cuda_cores_ms"] / res["tensor_cores_ms"]
    res["queries"], res["trains"] = nq, nt
    return res


# ---------------------------------------------------------------- CPU oracle
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def oracle_pair(img1, img2, threads: int):
    """The CPU oracle, as it stands, on one whole pair: the warp and ORB of
    every view of both images, the brute-force match of the pooled
    descriptors and the back-projection of the accepted pairs, run by
    `threads` host threads over the views (largest canvas first) and over
    blocks of query rows.  Every oracle call is one C function that releases
    the GIL, so the threads run in parallel.  Returns (seconds, (n1, n2),
    accepted pairs)."""
    from concurrent.futures import ThreadPoolExecutor
    import oracle as O
    pat = O.pattern()
    views = O.view_table(H, W, KMAX)
    nv = len(views)
    imgs = (img1, img2)
    order = sorted(range(2 * nv), key=lambda j: -views[j % nv].Wr * views[j % nv].Hr)

    def view_job(j):
        vo = O.warp_view(imgs[j // nv], views[j % nv])
        return j, O.orb_view(vo.u8, vo.mask, LEVELS, NFEAT, THR, pat)

    t0 = time.perf_counter()
    with ThreadPoolExecutor(threads) as ex:
        res = dict(ex.map(view_job, order))
        pools = []
        for im in (0, 1):
            outs = [res[im * nv + v] for v in range(nv)]
            pools.append((np.concatenate([o.kps for o in outs]), np.concatenate([o.desc for o in outs]),
                          np.concatenate([np.full(len(o.kps), v, np.int32) for v, o in enumerate(outs)])))
        (k1, d1, v1), (k2, d2, v2) = pools
        blocks = [b for b in np.array_split(np.arange(len(d1)), 4 * threads) if len(b)]
        ms = list(ex.map(lambda b: O.match(d1[b], d2, 4, 5), blocks))
        best = np.concatenate([m.best for m in ms]) if ms else np.zeros(0, np.int32)
        acc = np.flatnonzero(np.concatenate([m.accepted for m in ms])) if ms else np.zeros(0, np.int64)
        xy = [(O.backproject(views[v1[q]], int(k1[q]["level"]), float(k1[q]["x"]), float(k1[q]["y"])),
               O.backproject(views[v2[best[q]]], int(k2[best[q]]["level"]), float(k2[best[q]]["x"]),
                             float(k2[best[q]]["y"]))) for q in acc]
    return time.perf_counter() - t0, (len(d1), len(d2)), len(xy)


def cpu_baseline_line(p, threads: int, single: bool) -> dict:
    """The oracle on one whole pair with every host core, and (single) with one."""
    t_pool, sizes, n_acc = oracle_pair(p.img1, p.img2, threads)
    line = {"value": 1.0 / t_pool, "unit": "pairs/s", "cores": threads, "kind": "oracle",
            "sample": (f"one whole {W}x{H} pair ({sizes[0]} x {sizes[1]} pooled descriptors, {n_acc} accepted): "
                       f"warp + ORB of all {2 * len(view_table_sizes())} views and the full match, "
                       f"{threads} host threads over views and query rows"),
            "seconds": t_pool}
    if single:
        t_one, _, _ = oracle_pair(p.img1, p.img2, 1)
        line["single_thread"] = {"value": 1.0 / t_one, "unit": "pairs/s", "cores": 1, "seconds": t_one}
    return line


def view_table_sizes():
    import oracle as O
    return O.view_table(H, W, KMAX)


def run_reference(args):
    """The reference arm: the CPU oracle (there is no installable reference
    implementation: the paper ships no code), every step one whole pair
    (alternating the GPU arm's two pairs) on all host cores, on rank 0."""
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    threads = host_cores()
    pairs = [_pair(0, i) for i in range(2)]
    for i in range(args.warmup):
        oracle_pair(pairs[i % 2].img1, pairs[i % 2].img2, threads)
    times = []
    for i in range(args.steps):
        t, _, _ = oracle_pair(pairs[i % 2].img1, pairs[i % 2].img2, threads)
        times.append(t)
    tot = sum(times)
    val = args.steps / tot
    sample = (f"whole {W}x{H} pairs (the GPU arm's two pairs alternating): warp + ORB of all 86 views, the "
              f"full match and the back-projection, {threads} host threads over views and query rows")
    line = {"impl": "reference", "metric": "image pairs/s (warp+ORB+match)", "value": val, "unit": "pairs/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+int",
            "data": "synthetic", "config": {"workload": WORKLOAD, "H": H, "W": W, "views_per_image": 43,
                                            "levels": LEVELS, "features_per_view": NFEAT},
            "cpu_baseline": {"value": val, "unit": "pairs/s", "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- GPU arm
def run_ours(args):
    rank, world, local = _dist_env()
    t_gen = time.perf_counter()
    batch = mixed_batch(args.batch_pairs, 3000 + rank)
    big = large_batch(args.large_pairs, 5000 + rank)
    t_gen = time.perf_counter() - t_gen
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2503_03479_gb300 import build as B
    if rank == 0 or world == 1:
        B.build()
    if dist:
        dist.barrier()
    from paper_2503_03479_gb300 import asift as A

    ctx = A.Context(n_levels=LEVELS, n_features=NFEAT, fast_threshold=THR)
    pc = ctx.pair_cfg(kmax=KMAX)
    n_pairs = 2
    pairs = [_pair(rank, i) for i in range(n_pairs)]
    d1 = [torch.from_numpy(p.img1).cuda() for p in pairs]
    d2 = [torch.from_numpy(p.img2).cuda() for p in pairs]
    ws = ctx.match_pair_workspace((H, W), (H, W), pc)
    nv = len(A.view_table(H, W, KMAX))
    cap = nv * NFEAT
    out = torch.zeros(cap * A.PAIR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
    n_out = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")     # > 129 MB L2
    stream = torch.cuda.current_stream()

    def step(i):
        ctx.match_pair(d1[i % n_pairs], d2[i % n_pairs], pc, out, n_out, ws)

    for i in range(args.warmup):
        step(i)
        flush.zero_()
    torch.cuda.synchronize()
    if ctx.read_status(ws) != 0:
        raise RuntimeError("device status word set during warm-up")

    # ---- timed region: K steps, L2 flushed between steps (outside the events).
    # No synchronisation inside: the host builds and enqueues step i + 1 while
    # the GPU runs step i, as a caller streaming pairs would.
    # The Python garbage collector is off inside (as timeit does): a
    # collection pass would stall the enqueueing host mid-step.
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    l0 = A.launch_count()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    gc.collect()
    gc.disable()
    try:
        with ClockSampler(local) as clk:
            for i in range(args.steps):
                ev[i][0].record(stream)
                step(i)
                ev[i][1].record(stream)
                flush.zero_()
            torch.cuda.synchronize()
    finally:
        gc.enable()
    launches = A.launch_count() - l0
    if dist:
        dist.barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = sum(step_ms)
    if ctx.read_status(ws) != 0:
        raise RuntimeError("device status word set during the timed region")

    # ---- stage times: a separate profiled pass (reading the library's stage
    # events waits for each step), same steps, same flushes
    ctx.profile(True)
    stage_ms = []
    for i in range(min(args.steps, 40)):
        step(i)
        stage_ms.append(ctx.profile_read())
        flush.zero_()
    ctx.profile(False)
    t_max = max_over_ranks(ms, dist, "cuda")
    value = job_rate(world, args.steps, t_max / 1e3)

    # ---- rooflines of the two heaviest stages, timed live by the stage events
    st = {k: statistics.mean(s[k] for s in stage_ms) for k in stage_ms[0]}
    n_acc = int(n_out.item())
    # pool sizes of each pair the steps alternate over; the last pair's pools
    # feed the engine comparison below
    sizes = []
    for i in range(n_pairs):
        step(i)
        kp1, dd1, kp2, dd2, _ = ctx.inspect_pair((H, W), (H, W), pc, ws)
        sizes.append((len(kp1), len(kp2)))
    n1, n2 = sizes[-1]
    peaks = _peaks()
    clocks = clk.summary()
    views = A.view_table(H, W, KMAX)
    det_b, pyr_b = orb_level_bytes(A, views, LEVELS)
    rooflines = {"warp": warp_roofline(views, 2, st["warp"], peaks),
                 "match": match_roofline(sizes, st["match"], ctx.match_engine == A.MATCH_TENSOR_CORES, peaks),
                 "detect": hbm_roofline("detect_kernel", 2.0 * det_b, st["detect"], peaks),
                 "pyramid": hbm_roofline("pyramid_kernel", 2.0 * pyr_b, st["pyramid"], peaks)}
    for k, r in rooflines.items():
        r["traffic"] = profiled_traffic(r["kernel"].split()[0])
    dominant = max(rooflines, key=lambda k: st[k])
    roofline = dict(rooflines[dominant], stage=dominant)

    # ---- the two matcher engines on this pair's pools (device buffers, same result)
    engines = match_engines(A, ctx, dd1, dd2, stream)

    # ---- plain per-view form (same kernels, one launch per view and stage)
    plain = None
    if args.plain_steps > 0:
        pcp = ctx.pair_cfg(kmax=KMAX, per_view=True)
        wsp = ctx.match_pair_workspace((H, W), (H, W), pcp)
        for i in range(2):
            ctx.match_pair(d1[0], d2[0], pcp, out, n_out, wsp)
        torch.cuda.synchronize()
        evp = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.plain_steps)]
        for i in range(args.plain_steps):
            evp[i][0].record(stream)
            ctx.match_pair(d1[i % n_pairs], d2[i % n_pairs], pcp, out, n_out, wsp)
            evp[i][1].record(stream)
            flush.zero_()
        torch.cuda.synchronize()
        msp = sum(a.elapsed_time(b) for a, b in evp) / args.plain_steps
        plain = {"value": 1e3 / msp, "unit": "pairs/s", "ms_per_step": msp}

    # ---- batched form: the mixed-size batch in one launch per stage, CUDA graph
    batched = None
    if batch:
        b1 = [torch.from_numpy(a).cuda() for a, _ in batch]
        b2 = [torch.from_numpy(b).cuda() for _, b in batch]
        nviews = sum(len(A.view_table(*a.shape, KMAX)) + len(A.view_table(*b.shape, KMAX)) for a, b in batch)
        t0 = time.perf_counter()
        plan = A.Plan(ctx, b1, b2, kmax=KMAX)
        t_plan = time.perf_counter() - t0
        t0 = time.perf_counter()
        tuning = plan.autotune(reps=1)
        t_tune = time.perf_counter() - t0
        plan.run()
        torch.cuda.synchronize()
        if plan.status() != 0:
            raise RuntimeError("device status word set in the batched plan")
        reps = max(1, min(3, args.steps))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            plan.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1) / reps
        # the evaluation of every pair's accepted pairs, one launch per stage
        # (duplicates, RANSAC with 1024 hypotheses, inliers; the mix stores no
        # true homographies, so no precision count)
        gen_e = np.random.default_rng(6100 + rank)
        rnd_b = torch.from_numpy(gen_e.integers(0, 2 ** 32, size=(1024, 4), dtype=np.uint64)
                                 .astype(np.uint32).view(np.int32)).cuda()
        plan.evaluate(rnd=rnd_b, read=False)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(reps):
            plan.evaluate(rnd=rnd_b, read=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_eval_b = e0.elapsed_time(e1) / reps
        res_b = plan.evaluate(rnd=rnd_b)
        eval_b = {"ms": ms_eval_b, "hypotheses": 1024, "kept_pairs": int(sum(r.n_unique for r in res_b)),
                  "inliers": int(sum(r.n_inliers for r in res_b))}
        # the plain per-view form and the one-pair-per-call form on the same batch
        def per_pair(per_view):
            pcx = ctx.pair_cfg(kmax=KMAX, per_view=per_view)
            tot = 0.0
            for a, b in zip(b1, b2):
                wsx = ctx.match_pair_workspace(tuple(a.shape), tuple(b.shape), pcx)
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                ctx.match_pair(a, b, pcx, ws=wsx)
                s1.record(stream)
                torch.cuda.synchronize()
                tot += s0.elapsed_time(s1)
                ctx._ws.clear()
            return tot
        ms_plain = per_pair(True)
        ms_single = per_pair(False)
        plan.close()
        nb = len(batch)
        batched = {"pairs": nb, "views": nviews, "sizes": "480x360..1920x1080 uniform, tilts 30-85 deg",
                   "ms_per_batch": ms_b, "pairs_per_s": nb / (ms_b / 1e3), "views_per_s": nviews / (ms_b / 1e3),
                   "plain_per_view_pairs_per_s": nb / (ms_plain / 1e3),
                   "one_pair_per_call_pairs_per_s": nb / (ms_single / 1e3),
                   "batched_vs_plain": ms_plain / ms_b, "tuning": tuning,
                   "plan_create_s": t_plan, "autotune_s": t_tune, "generate_s": t_gen,
                   "evaluation": eval_b}
        del b1, b2

    # ---- large extreme-tilt batch: 4096x3072 pairs, 63 views per image, 2000 keypoints per view
    large = None
    if big:
        ctx_l = A.Context(n_levels=LEVELS, n_features=LARGE_NFEAT, fast_threshold=THR)
        g1 = [torch.from_numpy(a).cuda() for a, _ in big]
        g2 = [torch.from_numpy(b).cuda() for _, b in big]
        nv_l = len(A.view_table(LARGE_H, LARGE_W, LARGE_KMAX))
        planl = A.Plan(ctx_l, g1, g2, kmax=LARGE_KMAX)
        tun_l = planl.autotune(reps=1)
        planl.run()
        torch.cuda.synchronize()
        if planl.status() != 0:
            raise RuntimeError("device status word set in the large batch")
        cnt_l = planl.pool_counts()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps_l = 3
        e0.record(stream)
        for _ in range(reps_l):
            planl.run()
        e1.record(stream)
        torch.cuda.synchronize()
        ms_l = e0.elapsed_time(e1) / reps_l
        npl = len(big)
        pairs_desc = float(sum(int(cnt_l[2 * i]) * int(cnt_l[2 * i + 1]) for i in range(npl)))
        large = {"pairs": npl, "image": f"{LARGE_W}x{LARGE_H}", "views_per_image": nv_l,
                 "features_per_view": LARGE_NFEAT, "ms_per_batch": ms_l, "pairs_per_s": npl / (ms_l / 1e3),
                 "views_per_s": 2 * nv_l * npl / (ms_l / 1e3),
                 "descriptors_per_image_mean": float(cnt_l.mean()),
                 "hamming_pairs_per_batch": pairs_desc, "tuning": tun_l}
        planl.close()
        del g1, g2, ctx_l

    # ---- differentiable warp: 256 views of 512x512 fp32 images, forward + backward
    diff = None
    if args.diff_views > 0:
        from paper_2503_03479_gb300 import synth
        nd, HD = args.diff_views, 512
        gen = np.random.default_rng(4)
        base = [synth.texture(HD, HD, 4000 + i % 16).astype(np.float32) / 255.0 for i in range(min(nd, 16))]
        ud = torch.from_numpy(np.stack([base[i % len(base)] for i in range(nd)])).cuda()
        ts = gen.uniform(1.05, 5.7, nd)
        ph = gen.uniform(0, 180, nd)
        grid_t = np.sqrt(2.0) ** np.round(np.log(ts) / np.log(np.sqrt(2.0)))
        lay = A.warp_layout(HD, HD, grid_t, ph, 5.7)
        th = torch.from_numpy(np.stack([ts, ph, gen.uniform(-8, 8, nd), gen.uniform(-8, 8, nd)], 1)).cuda()
        vb = torch.randn(lay.total, device="cuda", generator=torch.Generator(device="cuda").manual_seed(1))
        for _ in range(2):
            A.warp_forward(ctx, ud, th, lay)
            A.warp_backward(ctx, ud, th, lay, vb)
        torch.cuda.synchronize()
        ef = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        ef[0].record(stream)
        A.warp_forward(ctx, ud, th, lay)
        ef[1].record(stream)
        A.warp_backward(ctx, ud, th, lay, vb)
        ef[2].record(stream)
        torch.cuda.synchronize()
        fms, bms = ef[0].elapsed_time(ef[1]), ef[1].elapsed_time(ef[2])
        # the parameter gradients alone (what the descent uses), and 20 steps of descent
        A.warp_backward(ctx, ud, th, lay, vb, image_grad=False)
        torch.cuda.synchronize()
        ef[0].record(stream)
        A.warp_backward(ctx, ud, th, lay, vb, image_grad=False)
        ef[1].record(stream)
        torch.cuda.synchronize()
        pms = ef[0].elapsed_time(ef[1])
        tgt = A.warp_forward(ctx, ud, th, lay)
        start = torch.stack([torch.from_numpy(grid_t).cuda(), th[:, 1], th[:, 2] * 0, th[:, 3] * 0], 1)
        A.refine(ctx, ud, tgt, lay, start, steps=2)
        torch.cuda.synchronize()
        ef[0].record(stream)
        _, dl = A.refine(ctx, ud, tgt, lay, start, steps=20)
        ef[1].record(stream)
        torch.cuda.synchronize()
        rms = ef[0].elapsed_time(ef[1])
        dl = dl.cpu().numpy()
        diff = {"views": nd, "image": f"{HD}x{HD} fp32", "fwd_ms": fms, "bwd_ms": bms,
                "bwd_params_only_ms": pms, "views_per_s_fwd_bwd": nd / ((fms + bms) / 1e3),
                "descent_20_steps_ms": rms, "descent_loss_ratio_median": float(np.median(dl[-1] / dl[0]))}
        del ud

    # ---- coarse stage (Sec. III-B): the reference's (t, phi, s) parameter
    # groups against the unwarped target, matches counted per view and the
    # best group taken on the device; nearest-neighbour views as the paper's
    # coarse stage, and the same with Lanczos-3 views
    coarse = None
    if args.coarse_steps > 0:
        coarse = {"ds": DS}
        for name, nearest in (("nearest", True), ("lanczos3", False)):
            pcc = ctx.pair_cfg(kmax=KMAX, coarse=True, ds=DS, nearest=nearest)
            wsc = ctx.match_pair_workspace((H, W), (H, W), pcc)
            vc = ctx.pair_views((H, W), pcc, 0)
            outc = torch.zeros(len(vc) * NFEAT * A.PAIR_DTYPE.itemsize, dtype=torch.uint8, device="cuda")

            def cstep(i):
                ctx.match_pair(d1[i % n_pairs], d2[i % n_pairs], pcc, outc, n_out, wsc)
                return ctx.view_counts((H, W), (H, W), pcc, wsc)

            for i in range(2):
                cstep(i)
            torch.cuda.synchronize()
            evc = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(args.coarse_steps)]
            for i in range(args.coarse_steps):
                evc[i][0].record(stream)
                cstep(i)
                evc[i][1].record(stream)
                flush.zero_()
            torch.cuda.synchronize()
            if ctx.read_status(wsc) != 0:
                raise RuntimeError("device status word set in the coarse stage")
            msc = sum(a.elapsed_time(b) for a, b in evc) / args.coarse_steps
            ctx.profile(True)
            stc = []
            for i in range(min(args.coarse_steps, 10)):
                cstep(i)
                stc.append(ctx.profile_read())
                flush.zero_()
            ctx.profile(False)
            stc = {k: statistics.mean(x[k] for x in stc) for k in stc[0]}
            best_of = []
            for i in range(n_pairs):
                counts, best = cstep(i)
                b = int(best.item())
                v = vc[b]
                best_of.append({"view": b, "t": v.t, "phi_deg": v.phi_deg, "s": v.s,
                                "matches": int(counts[b].item())})
            px = sum(v.Wv * v.Hv for v in vc)
            cline = {"pairs_per_s": 1e3 / msc, "ms_per_pair": msc, "views_reference": len(vc), "views_target": 1,
                    "view_pixels": int(px), "stage_ms": stc, "best": best_of}
            if nearest:
                cline["warp_gpix_per_s"] = px / (stc["warp"] / 1e3) / 1e9
                # the precise stage's Lanczos-4 (8 x 8) reproduction of pair 0's best group (Sec. III-C)
                bv = [vc[best_of[0]["view"]]]
                for _ in range(2):
                    ctx.views(d1[0], bv, lanczos=4)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(10):
                    ctx.views(d1[0], bv, lanczos=4)
                e1.record(stream)
                torch.cuda.synchronize()
                cline["precise_lanczos4_view"] = {"ms": e0.elapsed_time(e1) / 10, "pixels": bv[0].Wv * bv[0].Hv,
                                                 "canvas_pixels": bv[0].Wr * bv[0].Hr}
            else:
                f_clk = (peaks.get("sm_max_mhz") or 2070.0) * 1e6
                flops = sum(warp_flops(v) for v in vc)     # the target's identity view costs no arithmetic
                cline["roofline_warp"] = _alu_roofline(flops, stc["warp"],
                                                      SM_COUNT * FP32_LANES_PER_SM * 2 * f_clk / 1e12, f_clk)
            coarse[name] = cline
            del wsc, outc

    # ---- evaluation of the accepted pairs (Sec. III-C, Sec. IV-B): duplicate
    # removal, Eq. (5)-(6) precision against the pair's true homography, RANSAC
    # with 1024 hypotheses and the Eq. (7) inlier ratio
    evaluation = None
    if args.eval_hyp > 0:
        gen = np.random.default_rng(6000 + rank)
        rnd = torch.from_numpy(gen.integers(0, 2 ** 32, size=(args.eval_hyp, 4), dtype=np.uint64)
                               .astype(np.uint32).view(np.int32)).cuda()
        evaluation = {"hypotheses": args.eval_hyp, "ransac_threshold_px": 3.0, "precision_threshold_px": "sqrt(3)",
                      "pairs": []}
        for i in range(n_pairs):
            step(i)
            for _ in range(2):
                ctx.eval_pairs(out, n_out, H_true=pairs[i].H12, rnd=rnd)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            reps = 10
            e0.record(stream)
            for _ in range(reps):
                _, _, _, res = ctx.eval_pairs(out, n_out, H_true=pairs[i].H12, rnd=rnd)
            e1.record(stream)
            torch.cuda.synchronize()
            r = ctx.eval_result(res)
            evaluation["pairs"].append({
                "accepted": r.n_pairs, "unique": r.n_unique, "precision": r.r_num / max(r.n_unique, 1),
                "inlier_ratio": r.n_inliers / max(r.n_unique, 1), "ms": e0.elapsed_time(e1) / reps})

    # ---- SIFT of the precise stage (Sec. III-C) on image 1 of pair 0
    sift_line = None
    if args.sift_reps > 0:
        for _ in range(2):
            ctx.sift_raw(d1[0])
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.sift_reps):
            _, _, n_sift = ctx.sift_raw(d1[0])
        e1.record(stream)
        torch.cuda.synchronize()
        sift_line = {"image": f"{W}x{H}", "ms": e0.elapsed_time(e1) / args.sift_reps, "keypoints": int(n_sift.item())}

    # ---- end to end through the C ABI with host buffers
    h1 = [torch.from_numpy(p.img1).pin_memory() for p in pairs]
    h2 = [torch.from_numpy(p.img2).pin_memory() for p in pairs]
    hout = torch.empty(cap * A.PAIR_DTYPE.itemsize, dtype=torch.uint8).pin_memory()
    hn = torch.empty(1, dtype=torch.int32).pin_memory()
    e2e_t, host_t = [], []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        d1[0].copy_(h1[i % n_pairs], non_blocking=True)
        d2[0].copy_(h2[i % n_pairs], non_blocking=True)
        th = time.perf_counter()
        ctx.match_pair(d1[0], d2[0], pc, out, n_out, ws)
        host_t.append(time.perf_counter() - th)   # the call's host side (the GPU is idle, nothing blocks)
        hn.copy_(n_out, non_blocking=True)
        hout.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
        if i >= args.warmup:
            e2e_t.append(time.perf_counter() - t0)
    e2e = {"value": job_rate(world, 1, max_over_ranks(statistics.mean(e2e_t), dist, "cuda")), "unit": "pairs/s",
           "h2d_bytes_per_step": 2 * H * W, "d2h_bytes_per_step": int(hout.numel() + 4)}

    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baseline_line(pairs[0], host_cores(), not args.no_cpu_single)
        line = {"metric": "image pairs/s (warp+ORB+match)", "value": value, "unit": "pairs/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+int",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "H": H, "W": W, "views_per_image": nv, "levels": LEVELS,
                           "features_per_view": NFEAT, "fast_threshold": THR, "ratio": "4/5",
                           "l2": "flushed between steps (256 MB write)", "form": "batched: one launch per stage"},
                "views_per_s": value * 2 * nv,
                "stage_ms": st,
                "host_ms_per_call": statistics.median(host_t) * 1e3,
                "step_ms_median": statistics.median(step_ms), "step_ms_max": max(step_ms),
                "keypoints": [list(x) for x in sizes], "accepted": n_acc,
                "plain_per_view": plain,
                "batched_vs_plain": (value / world) / plain["value"] if plain else None,
                "batched_mixed": batched,
                "large_batched": large,
                "differentiable": diff,
                "coarse_stage": coarse,
                "evaluation": evaluation,
                "sift": sift_line,
                "roofline": roofline, "rooflines": rooflines, "match_engine": ctx.match_engine,
                "match_engines": engines,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
                "clocks": clocks}
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--plain-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-single", action="store_true", help="skip the single-threaded whole-pair oracle run")
    ap.add_argument("--batch-pairs", type=int, default=64, help="pairs in the mixed-size batched run (0: skip)")
    ap.add_argument("--large-pairs", type=int, default=8, help="pairs in the 4096x3072 batched run (0: skip)")
    ap.add_argument("--diff-views", type=int, default=256, help="views of the differentiable-warp timing (0: skip)")
    ap.add_argument("--coarse-steps", type=int, default=20, help="steps of the coarse-stage timing (0: skip)")
    ap.add_argument("--eval-hyp", type=int, default=1024, help="RANSAC hypotheses of the evaluation timing (0: skip)")
    ap.add_argument("--sift-reps", type=int, default=5, help="repetitions of the SIFT timing (0: skip)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
