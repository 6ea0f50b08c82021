"""Benchmark of the per-step contact path on the 1440-vesicle workload.

The headline (value, ms_per_step, e2e, roofline) is the FP64 form, the
paper's precision; the precision (MIXED) form is timed beside it on the same
workload and reported in config.mixed_form with its errors against the FP64
form.  One step = the whole hot path on one synthetic scene resident in HBM:
SH upsampling of X0 and X1 (p = 16 -> 32), space-time boxes, candidate
vesicle pairs (Morton grid), vertex-triangle and edge-edge contact tests,
contact volumes V and dV/dX1, and the adjoint of dV/dX1 back to the SH
coefficients.  Workload: 1440 prolate vesicles (reduced volume 0.91,
R0 = 1.34) at 58% volume fraction on a staggered lattice in a periodic cube,
step tuned to ~2 interfering neighbours per vesicle.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--single-form]
       python bench.py --impl reference ...   (the CPU oracle on a bounded sample)
Under torchrun (N > 1) every rank runs its own scene (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
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

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
# algorithmic work per exact-box primitive pair of the narrow phase (operations
# of the FP64 contact test), counted by tests/golden/make_narrow_ops.py
NARROW_OPS = os.path.join(ROOT, "tests", "golden", "narrow_ops_per_pair.json")
NARROW_STAGES = ("patch_pairs", "narrow", "pieces", "fp64")
NARROW_SRC = os.path.join(ROOT, "paper_1812_04719_gb300", "csrc", "narrow.cu")

# ncu figures of narrow_kernel (stages 1-3a), per patch pair it processes:
# smsp__inst_executed.sum (warp instructions) and dram__bytes_read.sum +
# dram__bytes_write.sum, from one capture of one launch per form on the
# 144-vesicle piece of the 58% lattice (the same cells, density and step as
# the 1440-vesicle workload).  A launch's figures are these times the patch
# pairs it processes.  They belong to the kernel as captured: when
# csrc/narrow.cu differs from the captured source (SHA-256 prefix), the
# instruction roofline and the traffic are reported as null.
NARROW_NCU = {
    "src_sha256": "92e5397a85063d40",
    # 97860990 inst, 7229952 + 889600 B over 35339 patch pairs
    "fp64": {"inst_per_patch_pair": 2769.21, "dram_bytes_per_patch_pair": 229.76},
    # 97617838 inst, 7206144 + 858880 B over 35339 patch pairs
    "mixed": {"inst_per_patch_pair": 2762.33, "dram_bytes_per_patch_pair": 228.22},
}
ISSUE_PER_SM_CLK = 4   # warp instructions an SM can issue per clock (4 schedulers)
METRIC = "vesicle-steps/s of detect+V+∇V at p=16→32, 58% vf; % of roofline vs FP64 form"
UNIT = "vesicle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"],
                    help="fp64: the FP64 form (the paper's precision; the headline); mixed: the precision form "
                         "(tensor-core 3xTF32 synthesis, FP32 vertices, FP64 detection and V/dV)")
    ap.add_argument("--single-form", action="store_true",
                    help="skip timing the other precision form beside the chosen one")
    ap.add_argument("--seed", type=int, default=None, help="scene seed (default: the workload's own)")
    ap.add_argument("--workload", default="1440", choices=["1440", "4096", "256", "64"],
                    help="1440: 58%% lattice, p=16->32 (default); 4096: 40%%, p in {8,12,16}, batched uneven "
                         "orders; 256: 50%%, p=12->24; 64: 30%% random, p=16->32")
    ap.add_argument("--cells", default=None,
                    help="smaller piece of the 58%% lattice (e.g. 6,6,2) for profiling; default: the 1440 scene")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-lcp", action="store_true", help="skip timing the contact LCP (assembly + solve)")
    ap.add_argument("--no-fidelity", action="store_true", help="skip the mesh-fidelity diagnostic")
    ap.add_argument("--no-dm", action="store_true", help="skip timing the step with minimum separation d_m > 0")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-other-workloads", action="store_true",
                    help="skip timing the 4096-vesicle (uneven orders) and 256-vesicle workloads beside the 1440 one")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU time of the oracle sample")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# algorithmic work of the dominant kernels (roofline numerators)
# ---------------------------------------------------------------------------
def synth_flops(p: int) -> int:
    """FP64 flops of one (vesicle, time) synthesis as the kernel's loops run
    them (mul + add per term; symmetric combinations)."""
    P = 2 * p
    nh = P // 2 + 1
    leg = 0
    for s in range(2 * p + 1):
        m = (s + 1) >> 1
        leg += 2 * (p + 1 - m) + 2
    leg *= 3 * nh
    four = 3 * (P + 1) * (P // 2 + 1) * (4 * p + 8)
    poles = 6 * 2 * (p + 1)
    return leg + four + poles


def fid_flops(p: int, factor: int) -> int:
    """FP64 flops of the mesh-fidelity estimate for one (vesicle, time), as
    the kernel's loops run them (mul, add = 1, fma = 2), per fine ring:
    the Legendre column recurrences (4 per (n, m)), the ring sums (an FMA
    per coefficient and field), the mesh's two lines per longitude cell and
    field (8), per longitude quadruple the odd and even partial Fourier sums
    (2 FMAs per order m and field) and their 8 combinations per field, and
    per fine point the mesh value, the difference and the squared distance
    (5 per field)."""
    P = 2 * p
    Pf = factor * P
    nl = (p + 1) * (p + 2) // 2
    nq = Pf // 2 + 1
    per_ring = 4 * nl + 6 * (p + 1) ** 2 + 24 * 2 * P + nq * (12 * p + 24) + 2 * Pf * 15
    return (Pf + 1) * per_ring


def load_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# ---------------------------------------------------------------------------
# the oracle on a bounded sample (CPU baseline / reference arm)
# ---------------------------------------------------------------------------
class OracleScene:
    """The scene prepared for the oracle once (untimed): every vesicle
    synthesized, boxes and all candidate pairs (all-pairs box test)."""

    def __init__(self, sc):
        from concurrent.futures import ThreadPoolExecutor
        import oracle as O
        O.build()
        self.O, self.sc = O, sc
        self.threads = os.cpu_count() or 1
        with ThreadPoolExecutor(self.threads) as ex:
            self.X = list(ex.map(lambda v: O.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)), range(sc.n)))
        boxes = np.stack([O.vesicle_box(X, sc.d_m) for X in self.X])
        self.pairs = O.candidate_pairs(boxes, sc.L)

    def sample(self, n_s: int, seed: int, threads: int = 0):
        """Time the oracle on n_s random vesicles: their SH synthesis plus every
        candidate pair they own (pair (i, j), i < j, is owned by i), i.e. the
        vertex-triangle and edge-edge tests, V and dV/dX1 of those pairs.
        Summed over all vesicles this is exactly one step of the scene."""
        from concurrent.futures import ThreadPoolExecutor
        O, sc = self.O, self.sc
        threads = threads or self.threads
        rng = np.random.default_rng(seed)
        S = np.sort(rng.choice(sc.n, size=min(n_s, sc.n), replace=False))
        own = self.pairs[np.isin(self.pairs[:, 0], S)]
        t0 = time.perf_counter()
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(lambda v: O.synth_vesicle(int(sc.p[v]), int(sc.P[v]), sc.coef_of(v)), S.tolist()))
        O.contacts(sc.P, self.X, own, sc.L, sc.eps * sc.dt, nthreads=threads)
        secs = time.perf_counter() - t0
        desc = (f"{len(S)} random vesicles of the {sc.n}-vesicle scene: oracle SH synthesis of X0/X1 plus "
                f"the {len(own)} candidate pairs they own (vertex-triangle and edge-edge tests, V, dV/dX1); "
                f"the all-pairs candidate search runs once beforehand, untimed")
        return len(S), secs, desc

    def sized(self, target_s: float, seed: int = 0) -> int:
        n, secs, _ = self.sample(16, seed)
        return int(max(4, min(self.sc.n, 16 * target_s / max(secs, 1e-3))))


def oracle_sample(sc, target_s: float, rng_seed: int = 0):
    """(vesicles, seconds, threads, description) of one timed oracle sample of
    about target_s seconds on all host cores, and (vesicles, seconds,
    description) of a smaller one on a single core."""
    osc = OracleScene(sc)
    n_s = osc.sized(target_s, rng_seed)
    nv, secs, desc = osc.sample(n_s, rng_seed + 1)
    # one core: about a third of the budget, scaled from the all-core rate
    n_1 = int(max(2, min(sc.n, (target_s / 3) * nv / secs / max(osc.threads, 1))))
    nv1, secs1, desc1 = osc.sample(n_1, rng_seed + 2, threads=1)
    return nv, secs, osc.threads, desc, (nv1, secs1, desc1)


def make_scene(args, seed):
    from paper_1812_04719_gb300 import scenegen as G
    if args.cells:
        return G.scene_lattice58(tuple(int(x) for x in args.cells.split(",")), seed=seed)
    return {"1440": G.scene_1440, "4096": G.scene_4096, "256": G.scene_256, "64": G.scene_64}[args.workload](seed=seed)


def default_seed(args):
    return {"1440": 3, "4096": 4, "256": 5, "64": 2}[args.workload] if args.seed is None else args.seed


# ---------------------------------------------------------------------------
def run_reference(args, rank, world):
    """The reference arm: the CPU oracle, timed on this host's cores."""
    if rank != 0:
        return
    sc = make_scene(args, default_seed(args))
    osc = OracleScene(sc)
    threads = osc.threads
    budget = max(2.0, 150.0 / max(args.steps + args.warmup, 1))
    n_s = osc.sized(budget)
    per_step = []
    total_v = 0
    desc = ""
    for k in range(args.warmup + args.steps):
        nv, t, desc = osc.sample(n_s, seed=100 + k)
        if k >= args.warmup:
            per_step.append((nv, t))
            total_v += nv
    secs = sum(t for _, t in per_step)
    value = total_v / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * secs / len(per_step),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": sc.name, "n_vesicles": sc.n, "sample": "per step: " + desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x: float, device) -> float:
    """The largest per-step time over all ranks (each rank one GPU running its
    own replica of the workload); every rank gets the same value."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(n_per_rank: int, world: int, ms_max: float) -> float:
    """Whole-job vesicle-steps/s: every rank advances its own n_per_rank
    vesicles per step; the job's step takes the slowest rank's time."""
    return n_per_rank * world / (ms_max * 1e-3)


def mixed_errors(S, sc, e_m, d_m, e_64, d_64, dev) -> dict:
    """The precision form's errors against the FP64 form on this workload and
    its stated bounds (paper_1812_04719_gb300/accuracy.py): one step of each
    form on its own synthesis, compared contact by contact."""
    import torch
    from paper_1812_04719_gb300 import accuracy as A

    def host(r):
        return {k: (v.cpu().numpy() if torch.is_tensor(v) else v) for k, v in r.items()}
    ra = host(e_m.step(d_m, grad=True))
    rb = host(e_64.step(d_64, grad=True))
    g0b = e_64.grad_x0(d_64).cpu().numpy()
    torch.cuda.synchronize(dev)
    Xa = d_m.verts.double().cpu().numpy()
    Xb = d_64.verts.cpu().numpy()
    pdelta = A.point_delta(sc.p, sc.coef_of, sc.vert_off(), Xb)
    res = A.compare(ra, Xa, rb, Xb, g0b, pdelta, sc.vert_off(), sc.L)
    keep = ("contacts_fp64", "only_mixed", "only_fp64", "V_ratio_max", "grad_ratio_max", "grad_rel_max",
            "symdiff_margin_max", "symdiff_volume", "V_pair_abs_err_sum_over_V_sum", "V_pair_rel_err_max")
    out = {k: res[k] for k in keep}
    out["max_abs_dX"] = float(np.abs(Xa - Xb).max())
    out["bounds"] = "V_ratio <= 1 (|dV_k| <= S_k delta_k); symdiff_margin <= 4; grad_ratio <= 4; pairs within bound"
    out["bounds_hold"] = bool(res["bound1_V_holds"] and res["bound2_lists_hold"] and res["bound3_grad_holds"]
                              and res["bound4_pairs_hold"])
    return out


def measure_fma_peak(S, stream, kind: int, dev) -> float:
    """GFLOP/s of the library's FMA-rate probe (kind 0 FP64, 1 FP32) on this
    GPU: best of 5 launches of about 30-40 ms, timed with CUDA events on the
    launching stream after 2 warm-up launches."""
    import torch
    sink = torch.zeros(1, dtype=torch.float64, device=dev)
    st = int(stream.cuda_stream)
    iters = 8_000 if kind == 0 else 400_000
    best = 0.0
    for k in range(7):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fl = S.stiv_peak_probe(st, kind, iters, sink.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize(dev)
        if k >= 2:
            best = max(best, fl / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def narrow_ncu_current() -> bool:
    """True when csrc/narrow.cu is the source the NARROW_NCU figures were captured on."""
    import hashlib
    with open(NARROW_SRC, "rb") as f:
        return NARROW_NCU["src_sha256"] is not None and \
            hashlib.sha256(f.read()).hexdigest()[:16] == NARROW_NCU["src_sha256"]


def kernel_roofline(S, sc, form: str, prec, stage_ms: dict, counts, peaks: dict, clk, n_sms: int):
    """Roofline of the dominant single kernel of the step (largest CUDA-event
    stage time): its work per launch over its average launch time, against
    the ceiling of the pipe that bounds it.
      narrow (narrow_kernel, stages 1-3a: integer and FP32 filter code): warp
        instructions issued (ncu count per patch pair x patch pairs) against
        the issue ceiling, 4 warp instructions per SM per clock x SMs x the
        SM clock sampled during the timed region;
      fp64 (fp64_kernel, stage 4): the FP64 operations of the contact test
        the kernel executed (counted by the kernel) against the measured FP64
        FMA rate;
      synth (FP64 form): the FP64 operations of the synthesis loops against
        the measured FP64 FMA rate."""
    dom = max(stage_ms, key=stage_ms.get)
    ms = stage_ms[dom]
    roof = {"kernel": dom, "avg_launch_ms": ms, "achieved": None, "peak": None, "frac": None, "traffic": None}
    sm_mhz = (clk or {}).get("sm_mhz") or peaks.get("sm_max_mhz", 2070.0)
    if dom == "narrow":
        fig = NARROW_NCU[form]
        units = float(counts[S.C_PATCH])
        peak = ISSUE_PER_SM_CLK * n_sms * sm_mhz * 1e6 / 1e9
        roof.update({"kernel": "narrow_kernel (stages 1-3a)", "bound": "alu", "unit": "Ginst/s", "peak": peak,
                     "peak_source": f"issue ceiling: {ISSUE_PER_SM_CLK} warp instructions per SM per clock x "
                                    f"{n_sms} SMs x {sm_mhz:.0f} MHz (SM clock sampled in the timed region)",
                     "units": units, "unit_name": "patch pairs"})
        if narrow_ncu_current() and fig["inst_per_patch_pair"]:
            inst = fig["inst_per_patch_pair"] * units
            roof["work_per_launch"] = inst
            roof["work"] = "warp instructions issued (ncu smsp__inst_executed.sum per patch pair on the " \
                           "144-vesicle piece of the lattice, times the launch's patch pairs)"
            roof["achieved"] = inst / (ms * 1e-3) / 1e9
            roof["traffic"] = fig["dram_bytes_per_patch_pair"] * units
            roof["traffic_unit"] = "bytes per launch (ncu on the 144-vesicle piece, scaled by patch pairs)"
    elif dom == "fp64":
        roof.update({"kernel": "fp64_kernel (stage 4)", "bound": "alu", "unit": "GFLOP/s", "peak": peaks["fp64_gflops"],
                     "peak_source": "FP64 FMA rate measured by the library's probe in this run",
                     "work_per_launch": float(counts[S.C_FLOPS]),
                     "work": "FP64 operations of the contact test the kernel executed, counted by it",
                     "achieved": float(counts[S.C_FLOPS]) / (ms * 1e-3) / 1e9})
    elif dom == "synth" and prec == S.STIV_FP64:
        work = float(sum(2 * synth_flops(int(p)) for p in sc.p))
        roof.update({"kernel": "synth_kernel (FP64 synthesis)", "bound": "alu", "unit": "GFLOP/s",
                     "peak": peaks["fp64_gflops"], "peak_source": "FP64 FMA rate measured by the library's probe",
                     "work_per_launch": work, "achieved": work / (ms * 1e-3) / 1e9})
    else:
        roof.update({"bound": "alu", "unit": None})
    if roof["achieved"] is not None and roof["peak"]:
        roof["frac"] = roof["achieved"] / roof["peak"]
    return roof


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_1812_04719_gb300 import build as B
    B.build()
    from paper_1812_04719_gb300 import stiv as S

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    sc = make_scene(args, default_seed(args) + rank)
    stream = torch.cuda.current_stream(dev)
    st = int(stream.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    n_sms = torch.cuda.get_device_properties(dev).multi_processor_count

    def setup(prec):
        eng = S.Stiv.for_scene(sc, precision=prec, pair_cap=8192, contact_cap=1 << 20, device=dev)
        ds = S.DeviceScene.from_scene(sc, precision=prec, device=dev)
        # size the buffers (grows on overflow), pick launch shapes, then profile
        # inside the captured graph
        eng.step(ds, grad=True)
        shapes = None if args.no_autotune else eng.autotune(ds, stream=stream)
        S.stiv_profile(eng.h, True)
        gX = torch.zeros(ds.verts.numel(), dtype=torch.float64, device=dev)
        gcoef = torch.zeros_like(ds.coef)

        def step(r_holder):
            r = eng.step(ds, grad=True, use_graph=True, stream=stream)
            b = eng.buf
            cst = b.contacts_struct()
            gX.zero_()
            S.stiv_grad_scatter(eng.h, st, ds.p.data_ptr(), cst, b.counts.data_ptr(), 0, b.grad.data_ptr(),
                                b.gves.data_ptr(), b.gvid.data_ptr(), ds.vert_off.data_ptr(), gX.data_ptr())
            S.stiv_grad_to_coef(eng.h, st, ds.n, ds.p_max, ds.p.data_ptr(), ds.coef_off.data_ptr(),
                                ds.vert_off.data_ptr(), gX.data_ptr(), gcoef.data_ptr())
            r_holder[0] = r
        return eng, ds, step, shapes

    def timed(eng, step, nsteps, clocks=None):
        holder = [None]
        for _ in range(max(args.warmup, 3)):
            flush.zero_()
            step(holder)
            torch.cuda.synchronize(dev)
            S.stiv_profile_read(eng.h)
        prof_tot = {}
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize(dev)
        if clocks:
            clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        t_wall0 = time.perf_counter()
        for k in range(nsteps):
            flush.zero_()
            ev[k][0].record(stream)
            step(holder)
            ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
            for name, (n, ms) in S.stiv_profile_read(eng.h).items():
                a = prof_tot.setdefault(name, [0, 0.0])
                a[0] += n; a[1] += ms
        torch.cuda.synchronize(dev)
        t_wall = time.perf_counter() - t_wall0
        if world > 1:
            dist.barrier()
        clk = clocks.stop() if clocks else None
        ms_mean = float(np.mean([e0.elapsed_time(e1) for e0, e1 in ev]))
        if world > 1:
            ms_mean = max_over_ranks(ms_mean, dev)
        return ms_mean, prof_tot, holder[0], t_wall, clk

    # measured arithmetic peaks of this GPU (the roofline denominators)
    peaks, peak_src = load_peaks()
    peaks = dict(peaks)
    peaks["fp64_gflops"] = measure_fma_peak(S, stream, 0, dev)
    peaks["fp32_gflops"] = measure_fma_peak(S, stream, 1, dev)

    prec = S.STIV_MIXED if args.precision == "mixed" else S.STIV_FP64
    form = "mixed" if prec == S.STIV_MIXED else "fp64"
    eng, ds, step, shapes = setup(prec)
    ms_max, prof_tot, last, t_wall, clk = timed(eng, step, args.steps, ClockSampler(local))
    counts = last["counts"]
    value = job_throughput(sc.n, world, ms_max)
    stage_ms = {k: v[1] / args.steps for k, v in prof_tot.items()}
    launches = int(sum(v[0] for v in prof_tot.values()))

    # the other precision form on the same workload, timed the same way, and
    # the precision form's errors against the FP64 form
    other = None
    if not args.single_form:
        oprec = S.STIV_FP64 if prec == S.STIV_MIXED else S.STIV_MIXED
        eng2, ds2, step2, shapes2 = setup(oprec)
        ms2, prof2, last2, _, _ = timed(eng2, step2, args.steps)
        other = {"form": "fp64" if oprec == S.STIV_FP64 else "mixed",
                 "dtype": "f64" if oprec == S.STIV_FP64 else "f32+f64",
                 "ms_per_step": ms2, "value": job_throughput(sc.n, world, ms2),
                 "stage_ms": {k: round(v[1] / args.steps, 4) for k, v in
                              sorted(prof2.items(), key=lambda x: -x[1][1])[:6]}}
        if rank == 0:
            e_m, e_64 = (eng, eng2) if prec == S.STIV_MIXED else (eng2, eng)
            d_m, d_64 = (ds, ds2) if prec == S.STIV_MIXED else (ds2, ds)
            other["mixed_errors"] = mixed_errors(S, sc, e_m, d_m, e_64, d_64, dev)
        eng2.close()

    roof = kernel_roofline(S, sc, form, prec, stage_ms, counts, peaks, clk, n_sms)

    # the other workloads of the paper's shapes, timed the same way (graph
    # replay, autotuned shapes, L2 flushed): the 4096-vesicle batch of uneven
    # orders p in {8, 12, 16} at 40% in both forms, and the 256-vesicle
    # 50% workload (p = 12 -> 24) in the FP64 form
    other_wl = None
    if args.workload == "1440" and not args.cells and not args.no_other_workloads:
        from paper_1812_04719_gb300 import scenegen as G
        other_wl = {}
        for name, mk, forms in (("4096", G.scene_4096, (S.STIV_FP64, S.STIV_MIXED)), ("256", G.scene_256, (S.STIV_FP64,))):
            sco = mk(seed=default_seed(argparse.Namespace(workload=name, seed=None)) + rank)
            rec = {"workload": sco.name}
            for fp in forms:
                eo = S.Stiv.for_scene(sco, precision=fp, pair_cap=1 << 15, contact_cap=1 << 21, device=dev)
                dso = S.DeviceScene.from_scene(sco, precision=fp, device=dev)
                eo.step(dso, grad=True)
                if not args.no_autotune:
                    eo.autotune(dso, stream=stream)
                ms_o = []
                for k in range(3 + 5):
                    flush.zero_()
                    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    ro = eo.step(dso, grad=True, use_graph=True, stream=stream)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    if k >= 3:
                        ms_o.append(e0.elapsed_time(e1))
                key = "fp64" if fp == S.STIV_FP64 else "mixed"
                rec[key] = {"ms_per_step": round(float(np.mean(ms_o)), 3),
                            "value": job_throughput(sco.n, world, float(np.mean(ms_o))),
                            "contacts": int(ro["counts"][S.C_VF] + ro["counts"][S.C_EE]),
                            "prim_pairs_tested": int(ro["counts"][S.C_PRIM])}
                eo.close()
                del dso
            other_wl[name] = rec

    # stage 4 alone: the FP64 operations it executed over its time; and the
    # narrow phase's effective rate: the FP64 contact test's operations on
    # every exact-box pair (the algorithmic count of the method's narrow
    # phase, most of which the certified FP32 cascade avoids) over the four
    # kernels' time
    fp64_ms = stage_ms.get("fp64", 0.0)
    roof_fp64 = None
    if fp64_ms > 0:
        ach = float(counts[S.C_FLOPS]) / (fp64_ms * 1e-3) / 1e9
        roof_fp64 = {"kernel": "fp64_kernel", "achieved": ach, "peak": peaks["fp64_gflops"], "unit": "GFLOP/s",
                     "frac": ach / peaks["fp64_gflops"], "avg_launch_ms": fp64_ms}
    with open(NARROW_OPS) as f:
        ops_rec = json.load(f)["workloads"]["1440" if args.cells else args.workload]
    narrow_ms = sum(stage_ms.get(k, 0.0) for k in NARROW_STAGES)
    eff_work = float(counts[S.C_PRIM]) * float(ops_rec["ops_per_prim_pair"])
    effective = {"ms": narrow_ms, "GFLOP/s": eff_work / (narrow_ms * 1e-3) / 1e9 if narrow_ms > 0 else None,
                 "work": "the FP64 contact test's operations (oracle count) on every exact-box pair; most are "
                         "decided by the certified FP32 cascade instead: an effective rate, not a fraction of a "
                         "peak"}

    # end to end through the public API: pinned host coefficients in; V per
    # pair and the gradient rows (values, vesicle and vertex ids) out into
    # pinned host buffers, every copy on the step's stream
    e2e = None
    if not args.no_e2e:
        host_coef = torch.empty(ds.coef.numel(), dtype=torch.float64, pin_memory=True)
        host_coef.copy_(torch.as_tensor(sc.coef))
        b = eng.buf
        host_out = {"V_pair": torch.empty(b.Vp.numel(), dtype=torch.float64, pin_memory=True),
                    "grad": torch.empty(b.grad.numel(), dtype=torch.float64, pin_memory=True),
                    "gves": torch.empty(b.gves.numel(), dtype=torch.int32, pin_memory=True),
                    "gvid": torch.empty(b.gvid.numel(), dtype=torch.int32, pin_memory=True)}
        e_ms = []
        bi = bo = 0
        for k in range(max(3, args.steps // 2) + 1):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ds.coef.copy_(host_coef, non_blocking=True)
            r = eng.step(ds, grad=True, use_graph=True, stream=stream)
            bo = S.NCOUNTS * 8          # the counts, read back inside step()
            with torch.cuda.stream(stream):
                for name, hbuf in host_out.items():
                    t = r[name].reshape(-1)
                    hbuf[:t.numel()].copy_(t, non_blocking=True)
                    bo += t.numel() * t.element_size()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            S.stiv_profile_read(eng.h)
            if k >= 1:
                e_ms.append(e0.elapsed_time(e1))
            bi = host_coef.numel() * 8
        e2e = {"value": sc.n * world / (float(np.mean(e_ms)) * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(bi),
               "d2h_bytes_per_step": int(bo)}

    # the contact LCP of the step (Eq. 3.7): B = J M J^T by Alg. 3 and the
    # min-map Newton solve, on the last step's contacts and gradient rows;
    # timed beside the step (the metric's step ends at dV/dX1)
    lcp_rec = None
    if not args.no_lcp:
        eng.step(ds, grad=True, use_graph=True, stream=stream)
        m_v = torch.ones(sc.n, dtype=torch.float64, device=dev)
        t_v = torch.as_tensor(1.0 / np.array([S.nverts(int(P)) for P in sc.P]), dtype=torch.float64, device=dev)
        lcp = S.ContactLCP(device=dev)
        A = lcp.assemble(eng, ds, m_v, t_v, stream=stream)
        b = eng.buf
        ms_a, ms_s = [], []
        for k in range(max(3, args.steps // 2) + 1):
            flush.zero_()
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            ev[0].record(stream)
            rc = S.lib().stiv_lcp_matrix(eng.h, st, ds.n, ds.p_max, b.pairs_struct(), b.contacts_struct(),
                                         b.counts.data_ptr(), b.Vp.data_ptr(), b.grad.data_ptr(),
                                         b.gves.data_ptr(), b.gvid.data_ptr(), m_v.data_ptr(), t_v.data_ptr(),
                                         lcp.struct())
            assert rc == S.STIV_OK, rc
            ev[1].record(stream)
            rc = S.lib().stiv_lcp_solve(eng.h, st, lcp.struct(), 1e-12, 100, 2000, lcp.lam.data_ptr(),
                                        lcp.info.data_ptr())
            assert rc == S.STIV_OK, rc
            ev[2].record(stream)
            torch.cuda.synchronize(dev)
            S.stiv_profile_read(eng.h)
            if k >= 1:
                ms_a.append(ev[0].elapsed_time(ev[1])); ms_s.append(ev[1].elapsed_time(ev[2]))
        info = lcp.info.cpu().numpy()
        cl = b.counts.cpu().numpy()
        ncon, npair = int(cl[S.C_VF] + cl[S.C_EE]), int(cl[S.C_PAIRS])
        # bytes the assembly must move at least: each contact's pair index,
        # gradient rows and their vesicle and vertex ids read once, the
        # candidate pairs and V per pair read once, B (CSR) and q written once
        lbytes = 132.0 * ncon + 20.0 * npair + 12.0 * A["nnz"] + 16.0 * A["n"]
        lach = lbytes / (float(np.mean(ms_a)) * 1e-3) / 1e9
        lcp_rec = {"rows": A["n"], "nnz": A["nnz"], "assemble_ms": round(float(np.mean(ms_a)), 4),
                   "solve_ms": round(float(np.mean(ms_s)), 4), "newton_steps": int(info[0]),
                   "max_abs_phi": float(info[1]), "status": int(info[3]),
                   "assembly_hbm_frac": round(lach / peaks["hbm_gbs"], 4)}

    # mesh fidelity of the step's meshes (Sec. 3.1.2, Fig. 6): the distance
    # between each order-2p triangle mesh and its smooth order-p surface on
    # the 4x upsampled grid; a diagnostic beside the step
    fid_rec = None
    if not args.no_fidelity:
        eng.step(ds, grad=True, use_graph=True, stream=stream)
        err = torch.zeros(ds.n, 2, dtype=torch.float64, device=dev)
        ms_f = []
        for k in range(4):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = S.lib().stiv_mesh_fidelity(eng.h, st, ds.n, ds.p_max, ds.p.data_ptr(), ds.coef_off.data_ptr(),
                                            ds.coef.data_ptr(), ds.vert_off.data_ptr(), ds.verts.data_ptr(), 4,
                                            err.data_ptr())
            assert rc == S.STIV_OK, rc
            e1.record(stream)
            torch.cuda.synchronize(dev)
            S.stiv_profile_read(eng.h)
            if k >= 1:
                ms_f.append(e0.elapsed_time(e1))
        from paper_1812_04719_gb300 import scenegen as G
        e = err.cpu().numpy()
        fwork = float(sum(2 * fid_flops(int(p), 4) for p in sc.p))
        fach = fwork / (float(np.mean(ms_f)) * 1e-3) / 1e9
        fid_rec = {"ms": round(float(np.mean(ms_f)), 3), "max_err_over_R0": float(e.max() / G.R0_PAPER),
                   "fp64_frac": round(fach / peaks["fp64_gflops"], 3)}

    # the step with minimum separation d_m > 0 (Eq. 3.1, degree six): the
    # paper's d_m = 0.009 at R0 = 1.136 (Fig. 6), scaled to this R0 and
    # inflated to (1 + 2 alpha) d_m with alpha = 0.05 (Sec. 3.1.2)
    dm_rec = None
    if not args.no_dm:
        import dataclasses
        from paper_1812_04719_gb300 import scenegen as G
        dm_val = (1.0 + 2 * 0.05) * (0.009 / 1.136) * G.R0_PAPER
        sc_dm = dataclasses.replace(sc, d_m=dm_val)
        eng_dm = S.Stiv.for_scene(sc_dm, precision=prec, pair_cap=8192, contact_cap=1 << 20, device=dev)
        ds_dm = S.DeviceScene.from_scene(sc_dm, precision=prec, device=dev)
        eng_dm.step(ds_dm, grad=True)          # sizes the buffers
        shapes_dm = None if args.no_autotune else eng_dm.autotune(ds_dm, stream=stream)
        S.stiv_profile(eng_dm.h, True)
        ms_d = []
        prof_d = {}
        for k in range(4):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rd = eng_dm.step(ds_dm, grad=True, use_graph=True, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            prof_k = S.stiv_profile_read(eng_dm.h)
            if k >= 1:
                ms_d.append(e0.elapsed_time(e1))
                for name, (n, ms) in prof_k.items():
                    prof_d[name] = prof_d.get(name, 0.0) + ms / 3
        cdm = rd["counts"]
        fp64_dm = prof_d.get("fp64", 0.0)
        dm_rec = {"d_m": dm_val, "ms_per_step": round(float(np.mean(ms_d)), 3), "contacts": int(cdm[S.C_VF] + cdm[S.C_EE]),
                  "fp64_ms": round(fp64_dm, 3),
                  "piece_levels": shapes_dm["piece_levels"] if shapes_dm else None,
                  "fp64_frac": round(float(cdm[S.C_FLOPS]) / (fp64_dm * 1e-3) / 1e9 / peaks["fp64_gflops"], 3)
                  if fp64_dm > 0 else None}
        eng_dm.close()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        nv, secs, threads, desc, one = oracle_sample(sc, args.cpu_seconds)
        cpu = {"value": nv / secs, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": desc,
               "single_core": {"value": one[0] / one[1], "unit": UNIT, "cores": 1, "sample": one[2]}}

    if rank == 0:
        cfg = {"workload": sc.name, "n_vesicles": sc.n, "p": sorted(set(int(x) for x in sc.p)),
               "P": sorted(set(int(x) for x in sc.P)), "precision": form,
               "l2": "flushed (256 MB write) before every timed step",
               "step": "upsample X0,X1 + boxes + Alg.1 pairs + VF/EE contact tests + V + dV/dX1 "
                       "+ adjoint to SH coefficients",
               "graph": "CUDA graph replay (upsample+detect+V+dV); adjoint launched after it",
               "launch_shapes": shapes,
               "candidate_pairs": int(counts[S.C_PAIRS]), "contact_pairs": int(counts[S.C_CPAIRS]),
               "contacts_vf": int(counts[S.C_VF]), "contacts_ee": int(counts[S.C_EE]),
               "prim_pairs_tested": int(counts[S.C_PRIM]), "patch_pairs": int(counts[S.C_PATCH]),
               "prim_pairs_fp64": int(counts[S.C_EXACT])}
        if other_wl is not None:
            cfg["other_workloads"] = other_wl
        if other is not None:
            key = "mixed_form" if other["form"] == "mixed" else "fp64_form"
            cfg[key] = {k: v for k, v in other.items() if k not in ("form", "stage_ms")}
            cfg[key]["speedup_mixed_over_fp64"] = (ms_max / other["ms_per_step"] if other["form"] == "mixed"
                                                   else other["ms_per_step"] / ms_max)
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64" if prec == S.STIV_FP64 else "f32+f64",
                "data": "synthetic", "gpu_launches": launches, "config": cfg,
                "roofline": roof, "cpu_baseline": cpu, "clocks": clk, "e2e": e2e,
                "peaks_measured": {"fp64_gflops": round(peaks["fp64_gflops"], 1),
                                   "fp32_gflops": round(peaks["fp32_gflops"], 1), "hbm_gbs": peaks.get("hbm_gbs"),
                                   "hbm_source": peak_src},
                "roofline_fp64_kernel": roof_fp64, "narrow_phase_effective": effective,
                "stage_ms": {k: round(v, 4) for k, v in sorted(stage_ms.items(), key=lambda x: -x[1])[:8]},
                "other_form_stage_ms": other["stage_ms"] if other else None,
                "lcp": lcp_rec, "mesh_fidelity": fid_rec, "dm_step": dm_rec, "wall_s": round(t_wall, 3)}
        print(json.dumps(line), flush=True)
    eng.close()
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
