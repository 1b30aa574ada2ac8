"""Benchmark: cone-beam FP + FDK step on the 3D short-scan workload.

Workload (one step, all on the GPU through the C ABI): 256^3 FP32 volume of
12 random ellipsoids (0.5 mm), 248 views over pi + 2 delta (short scan),
620 x 480 detector at 0.616 mm, SID 750 mm, SDD 1200 mm;
  1. ray-driven forward projection of the volume (pyro_fp_cone3d_ws: from a
     z-major copy of the volume kept in a workspace),
  2. FDK of that sinogram (pyro_fdk: cosine + Parker weights fused into the
     Shepp-Logan row filter, then the voxel-driven back-projection).
Metric: GUPS = voxel-view pairs processed per second, counting one pass of
FP and one of BP over the 256^3 x 248 problem per step (2 N^3 V units).

`value` is device time (CUDA events on the launching stream, L2 flushed
between steps, outside the timed events); `e2e` is the same step through the
public API from pinned host memory, copies included.  Under torchrun every
rank runs its own independent phantom (weak scaling, no data-path
collective); the step time is the max over ranks.

With one GPU the line also carries the other workloads as extra keys, each
with its own clock record (`--no-extras` leaves them out):
  * `configs_2d`: the 128^2 parallel-beam and 16 x 512^2 fan-beam workloads,
    GPU milliseconds beside the oracle's seconds on the host cores;
  * `fp16_storage`: the 256^3 workload with 16-bit storage (FP of an FP16
    volume, FP of the FP32 volume from an FP16 copy, FDK of an FP16
    sinogram) and each result's relative L2 against the oracle fed the FP32
    input;
  * `tv512_slice`: `--tv-steps` gradient steps of the 512^3 TV workload,
    seconds per step with FP32 storage and with an FP16 copy of the iterate;
  * `tv64_vs_oracle`: the same iteration on a 64^3 problem with that
    workload's voxel and detector pitch, the GPU iterates against the FP64
    oracle's.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload on this machine's host cores (the paper publishes no timings).

`--workload learned-init` runs the sparse-view study instead (one GPU): a
batch of 32 test phantoms, 128^3 at 1 mm, 60 views over 360 degrees, 256 x 200
detector at 1 mm; FDK -> residual CNN -> TV against plain TV from zero.  The
CNN is trained first on library-made pairs (not timed); lambda comes from a
small grid on training phantoms.  `value` is the seconds the CNN path needs
to reach the mean PSNR of 200 plain TV steps; the plain path's seconds, the
PSNRs and the fixed-budget comparison (CNN + 20 TV steps) ride along.

`--workload tv-512` times TV-regularised reconstruction (Eq. 7) at 512^3,
496 views, 1240 x 960 detector, 1 % noise: seconds per gradient step after
`--warmup` steps, FP32 against FP16 volume storage for the projector, and
the error on the central 64^3 crop.

`--workload configs` times the 2D workloads (128^2 parallel beam; a batch of
16 512^2 fan-beam phantoms) on the GPU and through the oracle.

`--workload cnn-128` times the residual CNN initialiser's forward pass on two
128^3 volumes (ms per pass) with a per-layer convolution breakdown.
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402
import torch  # noqa: E402

N, SPACING = 256, 0.5
NV, NU, SV, SU = 480, 620, 0.616, 0.616
VIEWS, SID, SDD = 248, 750.0, 1200.0
WORKLOAD = "cone-beam short-scan FDK 256^3 x 248 views, 620x480 det"
METRIC = "cone-beam BP/FP GUPS"
UNIT = "GUPS"


def geometry():
    from paper_1904_13342_gb300.geometry import ConeGeometry3D, short_scan_range

    rng_ = short_scan_range(NU * SU, SDD)
    return ConeGeometry3D((N, N, N), (SPACING,) * 3, (NV, NU), (SV, SU), VIEWS, rng_, SID, SDD)


def units_per_step() -> float:
    return 2.0 * N * N * N * VIEWS


def config(flush: str):
    return {"workload": WORKLOAD, "volume": [N, N, N], "spacing_mm": SPACING, "views": VIEWS,
            "detector": [NU, NV], "det_spacing_mm": SU, "sid_mm": SID, "sdd_mm": SDD, "filter": "shepp-logan",
            "redundancy": "parker", "step": "fp_cone3d + fdk(weights+filter, bp_cone3d)", "l2": flush}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.TemporaryFile(mode="w+")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.file.seek(0)
        rows = [[c.strip() for c in l.split(",")] for l in self.file.read().splitlines() if l.count(",") >= 8]
        note = None
        if not rows:  # a region shorter than one sampling period: one query right after it
            try:
                q = subprocess.run(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                    "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
                rows = [[c.strip() for c in l.split(",")] for l in q.stdout.splitlines() if l.count(",") >= 8]
                note = "region shorter than the 200 ms sampling period: one query right after it"
            except (OSError, subprocess.TimeoutExpired):
                rows = []
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        load = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        out = {"sm_mhz": statistics.median(load) if load else None, "sm_max_mhz": max(mx) if mx else None,
               "reasons": reasons, "samples": len(rows)}
        if note:
            out["note"] = note
        return out


def run_gpu(args):
    from paper_1904_13342_gb300 import binding as B
    from paper_1904_13342_gb300 import phantoms as ph

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    g = geometry()
    e = ph.random_ellipsoids(12, N * SPACING / 2, seed=rank)
    vol = ph.voxelize_ellipsoids(e, g.volume_shape, g.volume_spacing, device=dev, dtype=torch.float32).contiguous()
    cg = g.to_c()
    ws = torch.empty(B.lib().pyro_fdk_workspace_bytes(ctypes.byref(cg), 1), dtype=torch.uint8, device=dev)
    ws_fp = torch.empty(B.lib().pyro_fp_cone3d_workspace_bytes(ctypes.byref(cg), B.PYRO_F32), dtype=torch.uint8,
                        device=dev)
    sino_buf = torch.empty((VIEWS, NV, NU), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # 256 MB > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step(v):
        s = B.pyro_fp_cone3d_ws(v, g, workspace=ws_fp, out=sino_buf)
        return B.pyro_fdk(s, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER, workspace=ws)

    for _ in range(args.warmup):
        step(vol)
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize(dev)
    with ClockSampler(local) as clk:
        for k in range(K):
            flush.fill_(k & 0xFF)  # evict L2 between steps, outside the timed events
            e0, e1, e2, e3 = ev[k]
            e0.record(stream)
            sino = B.pyro_fp_cone3d_ws(vol, g, workspace=ws_fp, out=sino_buf)
            e1.record(stream)
            rec = B.pyro_fdk(sino, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER, workspace=ws)
            e2.record(stream)
        torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    step_ms = [ev[k][0].elapsed_time(ev[k][2]) for k in range(K)]
    fp_ms = [ev[k][0].elapsed_time(ev[k][1]) for k in range(K)]
    fdk_ms = [ev[k][1].elapsed_time(ev[k][2]) for k in range(K)]
    total_ms = sum(step_ms)
    if dist:
        t = torch.tensor([total_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    value = world * K * units_per_step() / (total_ms * 1e-3) / 1e9

    # separate per-kernel timings (outside the timed region): BP and filter alone
    sino = B.pyro_fp_cone3d_ws(vol, g, workspace=ws_fp)
    filt = torch.empty_like(sino)
    def alone(fn):
        fn()
        ts = []
        for _ in range(3):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    tk = {"bp": alone(lambda: B.pyro_bp_cone3d(sino, g, weight=B.W_INV_L2, scale=1.0)),
          "filter": alone(lambda: B.pyro_filter_rows(sino, SU * SID / SDD, B.SHEPP_LOGAN, out=filt))}

    # texture mode (the paper's fast FP mode): the volume copied into a CUDA
    # array and read with hardware trilinear filtering (8-bit weights)
    def rel_l2(a, b):
        return float(f"{float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double())):.3g}")

    texture = {}
    bp_soft = B.pyro_bp_cone3d(sino, g, weight=B.W_INV_L2, scale=1.0)
    for name, dt in (("f32", torch.float32), ("f16", torch.float16)):
        tv = B.Texture(g.volume_shape, dt, dev)
        ts = B.Texture(g.sinogram_shape, dt, dev, kind="sinogram")
        vd, sd = vol.to(dt), sino.to(dt)
        up_v, up_s = alone(lambda: tv.upload(vd)), alone(lambda: ts.upload(sd))
        fp_tex, bp_tex = torch.empty_like(sino), torch.empty_like(vol)
        fp_t = alone(lambda: B.pyro_fp_cone3d_tex(tv, g, out=fp_tex))
        bp_t = alone(lambda: B.pyro_bp_cone3d_tex(ts, g, weight=B.W_INV_L2, scale=1.0, out=bp_tex))
        texture[name] = {"fp_ms": round(fp_t, 4), "bp_ms": round(bp_t, 4), "upload_volume_ms": round(up_v, 4),
                         "upload_sinogram_ms": round(up_s, 4),
                         "arrays_MB": round((vd.numel() + sd.numel()) * vd.element_size() / 1e6, 1),
                         "fp_rel_l2_vs_software": rel_l2(fp_tex, sino), "bp_rel_l2_vs_software": rel_l2(bp_tex, bp_soft)}
        tv.close()
        ts.close()

    # end to end through the public API from pinned host memory: every step
    # copies its volume in and its reconstruction out; the copies run on
    # their own streams, double-buffered, so that step k+1's upload and step
    # k's download overlap the kernels (stream order and events keep each
    # buffer's uses apart)
    host_vol = vol.cpu().pin_memory()
    host_out = [torch.empty(vol.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    dev_in = [torch.empty_like(vol) for _ in range(2)]
    s_in, s_out = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    E = max(1, min(K, 10))
    torch.cuda.synchronize(dev)
    if dist:
        dist.barrier()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    freed = [None, None]  # the step that last read dev_in[slot] has finished with it
    a.record(stream)
    s_in.wait_event(a)
    s_out.wait_event(a)
    for e in range(E):
        slot = e & 1
        with torch.cuda.stream(s_in):
            if freed[slot] is not None:
                s_in.wait_event(freed[slot])
            dev_in[slot].copy_(host_vol, non_blocking=True)
            landed = torch.cuda.Event()
            landed.record(s_in)
        stream.wait_event(landed)
        r = step(dev_in[slot])
        done = torch.cuda.Event()
        done.record(stream)
        freed[slot] = done
        with torch.cuda.stream(s_out):
            s_out.wait_event(done)
            host_out[slot].copy_(r, non_blocking=True)
            r.record_stream(s_out)
    stream.wait_stream(s_out)
    b.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = a.elapsed_time(b)
    if dist:
        t = torch.tensor([e2e_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e = world * E * units_per_step() / (e2e_ms * 1e-3) / 1e9

    # the gather-bound view: achievable random 16-byte gather bandwidth from an
    # L2-resident 64 MB buffer (the project's probe), against the tap bytes the
    # FP (8 FP32 taps per sample) and the BP (4 taps per update) consume
    gather_gbs = gather_peak(dev, stream)
    peaks = {}
    pf = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pf):
        peaks = json.load(open(pf))
    # roofline of the dominant kernel (forward projection): FP32 issue-bound
    # gather; algorithmic work = 28 FP32 flops per trilinear sample
    samples = fp_sample_count(g)
    fp_avg_ms = statistics.mean(fp_ms)
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    achieved = samples * FLOPS_PER_SAMPLE / (fp_avg_ms * 1e-3) / 1e12
    clocks = clk.summary()
    traffic = fp_traffic_per_call()
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": round(total_ms / K, 4), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded random ellipsoid phantom)", "config": config("flushed 256 MB"),
        "e2e": {"value": round(e2e, 3), "unit": UNIT, "h2d_bytes_per_step": int(host_vol.numel() * 4),
                "d2h_bytes_per_step": int(host_out[0].numel() * 4), "steps": E,
                "copies": "pinned host buffers; H2D and D2H on their own streams, double-buffered"},
        "gpu_launches": 5 * K,  # per step: relayout, FP (two launches: 200 + 48 views), filter, BP
        "roofline": {"kernel": "fp3d_column_kernel", "bound": "alu", "achieved": round(achieved, 3),
                     "peak": round(peak_tflops, 2), "unit": "TFLOP/s", "frac": round(achieved / peak_tflops, 4),
                     "traffic": traffic,
                     "note": f"per FP call (two launches: 200 + 48 views; traffic: DRAM bytes of both, ncu); "
                             f"{samples:.4g} samples x {FLOPS_PER_SAMPLE} flop; peak = {props.multi_processor_count}"
                             f" SMs x 128 FP32 lanes x 2 x {sm_mhz:.0f} MHz"},
        "gather_view": gather_view(gather_gbs, samples, fp_avg_ms, tk["bp"]),
        "breakdown_ms": {"fp": round(fp_avg_ms, 4), "fdk": round(statistics.mean(fdk_ms), 4),
                         "bp_alone": round(tk["bp"], 4), "filter_alone": round(tk["filter"], 4)},
        "texture_mode": dict(texture, what="FP / BP through texture copies (hardware trilinear / bilinear "
                                           "filtering, 8-bit weights), timed alone"),
        "kernel_gups": {"fp": round(N ** 3 * VIEWS / (fp_avg_ms * 1e-3) / 1e9, 2),
                        "bp": round(N ** 3 * VIEWS / (tk["bp"] * 1e-3) / 1e9, 2)},
        "clocks": clocks,
    }
    if world == 1 and args.extras:
        # the other workloads, each with its own clock record
        del ws_fp, sino_buf, dev_in, host_out, sino, filt, bp_soft
        torch.cuda.empty_cache()
        out["configs_2d"] = measure_configs_2d(dev)
        out["fp16_storage"] = measure_fp16_arm(dev, g, vol, flush)
        del flush
        torch.cuda.empty_cache()
        out["tv512_slice"] = measure_tv512_slice(dev, args.tv_steps, args.tv_lambda)
        out["tv64_vs_oracle"] = measure_tv_vs_oracle(dev, args.tv_steps, args.tv_lambda)
    if rank == 0 and args.cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds, vol)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist:
        dist.destroy_process_group()


FLOPS_PER_SAMPLE = 28  # 3 position FMA (6) + 7 lerps (3 each) + 1 accumulate


def gather_peak(dev, stream) -> float:
    """GB/s of the library's random 16-byte gather probe over a 64 MB buffer
    (L2-resident after a warm-up), median of 5 runs."""
    from paper_1904_13342_gb300 import binding as B

    buf = torch.zeros(64 << 20, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1024, dtype=torch.int32, device=dev)
    threads = torch.cuda.get_device_properties(dev).multi_processor_count * 2048
    loads = 256
    B.pyro_probe_gather(buf, loads, threads, sink)
    ts = []
    for _ in range(5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        B.pyro_probe_gather(buf, loads, threads, sink)
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    return 16.0 * threads * loads / (statistics.median(ts) * 1e-3) / 1e9


def _profile_record(key):
    """A per-launch figure of the forward projector from the committed ncu
    summary (profiles/roofline_traffic.json), or None when the kernel source
    changed since the counters were taken."""
    import hashlib

    rec = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    src = os.path.join(ROOT, "paper_1904_13342_gb300", "csrc", "kernels_fp.cu")
    try:
        info = json.load(open(rec))
        if hashlib.sha256(open(src, "rb").read()).hexdigest() != info.get("source_sha256"):
            return None
        return int(info[key])
    except (OSError, ValueError, KeyError, TypeError):
        return None


def fp_traffic_per_call():
    """DRAM bytes (read + write) of one forward projection (its two launches,
    200 + 48 views), the unit the roofline's achieved rate is taken over"""
    return _profile_record("dram_bytes_per_fp_call")


def gather_view(probe_gbs, samples, fp_ms, bp_ms):
    """The gather side of the projectors.  The tap rates count every
    interpolation tap (8 FP32 per FP sample, 4 per BP update) as if gathered:
    most come from registers, shared memory (the BP's staged boxes) or L1,
    so they are effective rates, not a fraction of any bandwidth.  The bytes
    the FP moves through L2 come from the committed ncu counters (per launch,
    keyed to the kernel source) and are set against the library's random
    16-byte gather probe of an L2-resident buffer."""
    l2 = _profile_record("lts_bytes_per_fp_call")
    out = {"probe_l2_gather_GBps": round(probe_gbs, 1),
           "probe": "random 16-byte gathers from a 64 MB L2-resident buffer",
           "fp_effective_tap_rate_GBps": round(samples * 32 / (fp_ms * 1e-3) / 1e9, 1),
           "bp_effective_tap_rate_GBps": round(N ** 3 * VIEWS * 16 / (bp_ms * 1e-3) / 1e9, 1),
           "note": "tap rates are effective (taps from registers, shared memory and L1 included), not a "
                   "roofline fraction"}
    if l2 is not None:
        gbs = l2 / (fp_ms * 1e-3) / 1e9
        out.update({"fp_l2_bytes_per_call": l2, "fp_l2_GBps": round(gbs, 1),
                    "fp_l2_frac_of_probe": round(gbs / probe_gbs, 3)})
    return out


def ray_sample_estimate(beta: float, U, Vv):
    """Samples the forward projector visits on the rays through detector
    points (U, Vv) of the view at angle beta (arrays of equal shape, mm): the
    chord through the support box, divided by the sample spacing along the
    ray (dt |g| with |g| = L / SDD, L the source-to-pixel distance), in FP64."""
    import math

    L = np.sqrt(SDD ** 2 + U ** 2 + Vv ** 2)
    half = 0.5 * (N + 1) * SPACING
    c = np.array([math.cos(beta), math.sin(beta), 0.0])
    eu = np.array([-math.sin(beta), math.cos(beta), 0.0])
    S = -SID * c
    d = (SDD * c[None, None] + U[..., None] * eu[None, None] + Vv[..., None] * np.array([0, 0, 1.0])) / L[..., None]
    lo = np.full(U.shape, -np.inf)
    hi = np.full(U.shape, np.inf)
    for a in range(3):
        da = d[..., a]
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (-half - S[a]) / da
            t2 = (half - S[a]) / da
        lo = np.maximum(lo, np.where(da != 0, np.minimum(t1, t2), -np.inf))
        hi = np.minimum(hi, np.where(da != 0, np.maximum(t1, t2), np.inf))
    return np.maximum(hi - lo, 0.0) * SDD / L / (0.5 * SPACING)


def fp_sample_count(g) -> float:
    """Samples the forward projector visits (those inside the support box),
    estimated on the host in FP64 from the same ray geometry: every 15th view,
    scaled to all views."""
    ang = g.view_angles()
    nv, nu = g.detector_shape
    sv, su = g.detector_spacing
    u = (np.arange(nu) - 0.5 * (nu - 1)) * su
    v = (np.arange(nv) - 0.5 * (nv - 1)) * sv
    U, Vv = np.meshgrid(u, v)
    sub = ang[:: max(1, len(ang) // 16)]
    total = sum(float(np.sum(ray_sample_estimate(b, U, Vv))) for b in sub)
    return total * len(ang) / len(sub)


class CpuSample:
    """The oracle on a bounded sample of the workload: FP of `fv` views over
    the full volume and FDK of a `zs`-slice slab over all views.  The inputs
    (phantom, matrices, a smooth sinogram) are made once."""

    def __init__(self, vol=None):
        import oracle

        from paper_1904_13342_gb300 import phantoms as ph

        self.oracle = oracle
        self.g = g = geometry()
        if vol is None:
            e = ph.random_ellipsoids(12, N * SPACING / 2, seed=0)
            vol = ph.voxelize_ellipsoids(e, g.volume_shape, g.volume_spacing, dtype=torch.float32)
        self.vol = np.ascontiguousarray(vol.double().cpu().numpy() if torch.is_tensor(vol) else vol, np.float64)
        self.ang = g.view_angles()
        self.P = oracle.circular_pmats(self.ang, SID, SDD, (NV, NU), (SV, SU))
        # FDK of a slab: a smooth synthetic sinogram stands in for the projections
        self.y = ph.random_sinogram((VIEWS, NV, NU), 1, smooth=2)

    def run(self, fv: int, zs: int):
        o, g = self.oracle, self.g
        t0 = time.perf_counter()
        o.fp_cone3d(self.vol, g.volume_spacing, (NV, NU), self.P[:fv])
        t_fp = time.perf_counter() - t0
        kz = np.repeat(np.arange(N // 2 - zs // 2, N // 2 - zs // 2 + zs), N * N)
        jj = np.tile(np.repeat(np.arange(N), N), zs)
        ii = np.tile(np.arange(N), N * zs)
        t0 = time.perf_counter()
        o.fdk_voxels(self.y, g.volume_shape, g.volume_spacing, (SV, SU), self.ang, self.P, SID, SDD,
                     g.angular_range / VIEWS, ii, jj, kz, kind=o.SHEPP_LOGAN, redund=o.REDUND_PARKER)
        t_bp = time.perf_counter() - t0
        units = N ** 3 * fv + N * N * zs * VIEWS
        return units / (t_fp + t_bp) / 1e9, {
            "cores": o.num_threads(),
            "sample": f"oracle FP of {fv} view(s) over the 256^3 volume + FDK of a {zs}-slice slab over all 248 "
                      f"views ({units:.3g} voxel-view units, {t_fp + t_bp:.1f} s)"}


def cpu_baseline(seconds: float, vol=None):
    """About `seconds` of oracle work on all host cores (36 views + 48 slices
    take ~15 s on 16 Arm cores), then a smaller sample on one thread."""
    import oracle

    scale = max(seconds / 15.0, 0.1)
    sample = CpuSample(vol)
    v, info = sample.run(max(1, round(36 * scale)), max(2, round(48 * scale)))
    prev = oracle.set_num_threads(1)
    try:
        v1, info1 = sample.run(1, 2)
    finally:
        oracle.set_num_threads(prev)
    return {"value": round(v, 6), "unit": UNIT, "cores": info["cores"], "kind": "oracle", "sample": info["sample"],
            "single_thread": {"value": round(v1, 6), "unit": UNIT, "cores": info1["cores"], "sample": info1["sample"]}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    # each step: about 3 s of oracle work, so that --steps K --warmup W ends in minutes
    sample = CpuSample()
    vals = []
    for _ in range(args.warmup):
        sample.run(8, 10)
    info = {}
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, info = sample.run(8, 10)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = statistics.mean(vals)
    out = {"impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(wall * 1e3 / max(args.steps, 1), 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded random ellipsoid phantom)", "config": config("flushed 256 MB"),
           "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": info.get("cores"), "kind": "oracle",
                            "sample": info.get("sample")},
           "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_learned_init(args):
    from paper_1904_13342_gb300 import learned_init as LI

    dev = torch.device("cuda:0")
    setup = LI.SparseViewSetup()
    maker = LI.PairMaker(setup, dev)
    L_est = LI.lipschitz(maker)
    eps = 1e-3
    t0 = time.perf_counter()
    net, losses = LI.train_initializer(maker, list(range(1000, 1064)), steps=args.train_steps, batch=4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    grid = LI.choose_lambda(maker, list(range(1000, 1008)), [1.0, 3.0, 10.0, 30.0], 200, eps, L_est)
    lam = max(grid, key=grid.get)
    test = list(range(32))
    res = LI.ab_test(maker, net, test, lam, eps, L_est, short_iter=20, long_iter=200)
    sm = res.summary()
    value = sm["seconds_to_target"]
    line = {
        "metric": "sparse-view recon s to PSNR (CNN-initialised TV vs plain TV)",
        "value": round(value, 4) if value is not None else None,
        "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": 1, "warmup": 0,
        "dtype": "f32 (CNN bf16/f32-accumulate)", "data": "synthetic (seeded random ellipsoid phantoms)",
        "vs_baseline": None,
        "config": {"workload": "learned initializer: 32 x 128^3 (1 mm), 60 views / 360 deg, 256x200 det (1 mm), "
                               "SID 750 mm, SDD 1200 mm", "test_seeds": [0, 31], "train_seeds": [1000, 1063],
                   "train_steps": args.train_steps, "lambda": lam, "eps": eps, "lambda_grid": grid},
        "plain_tv_200_s": round(sm["seconds_plain"], 4),
        "speedup_vs_plain": round(sm["seconds_plain"] / value, 3) if value else None,
        "iters_to_target": sm["iters_to_target"],
        "psnr_db": {k: round(sm[k], 3) for k in ("psnr_fdk", "psnr_cnn", "psnr_learned", "psnr_short_tv",
                                                 "psnr_plain", "psnr_to_target")},
        "fixed_budget": {"cnn_plus_20_tv_s": round(sm["seconds_learned"], 4),
                         "tv_20_s": round(sm["seconds_short_tv"], 4)},
        "train_s": round(train_s, 2), "train_loss": [round(losses[0], 6), round(float(np.mean(losses[-50:])), 6)],
    }
    print(json.dumps(line), flush=True)


def run_tv512(args):
    """TV-regularised cone-beam reconstruction (Eq. 7) at 512^3: seconds per
    gradient step (staged FP, staged exact adjoint, TV and BB kernels), the
    forward projection with FP32 and FP16 volume storage, and the error on
    the central 64^3 crop after the steps."""
    import math

    from paper_1904_13342_gb300 import binding as B
    from paper_1904_13342_gb300 import phantoms as ph
    from paper_1904_13342_gb300.geometry import ConeGeometry3D
    from paper_1904_13342_gb300.tv import estimate_lipschitz, tv_reconstruct

    dev = torch.device("cuda:0")
    n, s = 512, 0.5
    g = ConeGeometry3D((n, n, n), (s, s, s), (960, 1240), (0.308, 0.308), 496, 2 * math.pi, 750.0, 1200.0)
    truth = ph.voxelize_ellipsoids(ph.random_ellipsoids(20, n * s / 2, seed=0), g.volume_shape, g.volume_spacing,
                                   device=dev, dtype=torch.float32)
    ws = torch.empty(B.fp_cone3d_workspace_bytes(g), dtype=torch.uint8, device=dev)
    p = B.pyro_fp_cone3d_ws(truth, g, workspace=ws)
    gen = torch.Generator(device=dev).manual_seed(1)
    p += (0.01 * float(p.abs().max())) * torch.randn(p.shape, generator=gen, device=dev)
    stream = torch.cuda.current_stream(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        return a.elapsed_time(b) / reps

    fp32_ms = timed(lambda: B.pyro_fp_cone3d_ws(truth, g, workspace=ws))
    t16 = truth.half()
    fp16_ms = timed(lambda: B.pyro_fp_cone3d_ws(t16, g, workspace=ws))
    p16 = B.pyro_fp_cone3d_ws(t16, g, workspace=ws)
    p32 = B.pyro_fp_cone3d_ws(truth, g, workspace=ws)
    fp16_rel = float(torch.linalg.norm((p16.float() - p32).double()) / torch.linalg.norm(p32.double()))
    del p16, p32, t16
    wT = torch.empty(B.fpT_cone3d_workspace_bytes(g), dtype=torch.uint8, device=dev)
    adj_ms = timed(lambda: B.pyro_fpT_cone3d_ws(p, g, workspace=wT))
    L_est = estimate_lipschitz(g, g.volume_shape, dev, iters=8)
    lam, eps = args.tv_lambda, 1e-3
    warm = tv_reconstruct(p, g, args.warmup, lam, eps, L_est=L_est)
    torch.cuda.synchronize(dev)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        a.record(stream)
        res = tv_reconstruct(p, g, args.steps, lam, eps, L_est=L_est, x0=warm.x, graph=True)
        b.record(stream)
        torch.cuda.synchronize(dev)
    step_s = a.elapsed_time(b) / 1e3 / args.steps
    c0, c1 = n // 2 - 32, n // 2 + 32
    crop = (slice(c0, c1),) * 3
    err = float(torch.linalg.norm((res.x[crop] - truth[crop]).double()) / torch.linalg.norm(truth[crop].double()))
    line = {
        "metric": "TV-regularised cone-beam reconstruction seconds per gradient step", "value": round(step_s, 4),
        "unit": "s", "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "dtype": "f32", "data": "synthetic (20 random ellipsoids, 1 % Gaussian noise on the sinogram)",
        "vs_baseline": None,
        "config": {"workload": "TV 512^3 (0.5 mm), 496 views / 360 deg, 1240x960 det (0.308 mm), SID 750, SDD 1200",
                   "lambda": lam, "eps": eps, "step": "FP + exact adjoint + TV gradient + BB step"},
        "kernel_ms": {"fp_f32": round(fp32_ms, 2), "fp_f16_storage": round(fp16_ms, 2), "adjoint": round(adj_ms, 2)},
        "fp16_storage_rel_l2": fp16_rel,
        "crop64_rel_l2_vs_phantom": round(err, 5), "total_steps": args.warmup + args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def measure_configs_2d(dev):
    """The two 2D workloads on the GPU (CUDA events, median of 10 after 3
    warm-ups) and through the FP64 oracle on the host cores (one run):
    128^2 parallel beam (180 views, 183 bins) and a batch of 16 512^2
    fan-beam phantoms (360 views, 1024 bins, SID 750, SDD 1200, step 0.25 mm).
    Units: FP samples/s, BP voxel-view updates/s (GUPS = 1e9 of them)."""
    import math

    import oracle

    from paper_1904_13342_gb300 import binding as B
    from paper_1904_13342_gb300 import phantoms as ph
    from paper_1904_13342_gb300.geometry import FanGeometry2D, ParallelGeometry2D

    stream = torch.cuda.current_stream(dev)

    def gpu_ms(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(10):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize(dev)
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    def cpu_s(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    def samples2d(g, n_img):
        """samples the projector visits: chord length / (dt |g|) summed over rays (host, FP64)"""
        ny, nx = g.volume_shape
        sy, sx = g.volume_spacing
        half = np.array([0.5 * (nx + 1) * sx, 0.5 * (ny + 1) * sy])
        u = (np.arange(g.detector_shape) - 0.5 * (g.detector_shape - 1)) * g.detector_spacing
        dt = g.step if g.step > 0 else 0.5 * min(sx, sy)
        total = 0.0
        for b in g.view_angles():
            c = np.array([math.cos(b), math.sin(b)])
            eu = np.array([-math.sin(b), math.cos(b)])
            if g.fan:
                S = -g.sid * c
                d = c[None] * g.sdd + u[:, None] * eu[None]
                gl = np.linalg.norm(d, axis=1) / g.sdd
                a = np.repeat(S[None], len(u), 0)
            else:
                d = np.repeat(c[None], len(u), 0)
                gl = np.ones(len(u))
                a = u[:, None] * eu[None]
            d = d / np.linalg.norm(d, axis=1, keepdims=True)
            lo, hi = np.full(len(u), -np.inf), np.full(len(u), np.inf)
            for ax in range(2):
                with np.errstate(divide="ignore", invalid="ignore"):
                    t1, t2 = (-half[ax] - a[:, ax]) / d[:, ax], (half[ax] - a[:, ax]) / d[:, ax]
                lo = np.maximum(lo, np.where(d[:, ax] != 0, np.minimum(t1, t2), -np.inf))
                hi = np.minimum(hi, np.where(d[:, ax] != 0, np.maximum(t1, t2), np.inf))
            total += np.sum(np.maximum(hi - lo, 0.0) / (dt * gl))
        return total * n_img

    out = {}
    # 128^2 parallel beam
    gp = ParallelGeometry2D((128, 128), (1.0, 1.0), 183, 1.0, 180, math.pi)
    img = ph.voxelize_ellipses(ph.random_ellipses(10, 64.0, seed=0), (128, 128), (1.0, 1.0), device=dev,
                               dtype=torch.float32)
    sino = B.pyro_fp_par2d(img, gp)
    ang = gp.view_angles()
    i64, s64 = img.double().cpu().numpy(), sino.double().cpu().numpy()
    ns, nb = samples2d(gp, 1), 128 * 128 * 180
    wsp = torch.empty(B.fp2d_workspace_bytes(gp, 1), dtype=torch.uint8, device=dev)
    with ClockSampler(dev.index or 0) as clk:
        t = {"fp": gpu_ms(lambda: B.pyro_fp_par2d(img, gp)),
             "fp_staged": gpu_ms(lambda: B.pyro_fp_par2d_ws(img, gp, workspace=wsp)),
             "bp": gpu_ms(lambda: B.pyro_bp_par2d(sino, gp)),
             "fbp": gpu_ms(lambda: B.pyro_fbp_par2d(sino, gp, kind=B.RAMLAK))}
    c = {"fp": cpu_s(lambda: oracle.fp_par2d(i64, (1.0, 1.0), 183, 1.0, ang)),
         "bp": cpu_s(lambda: oracle.bp_par2d(s64, (128, 128), (1.0, 1.0), 1.0, ang)),
         "fbp": cpu_s(lambda: oracle.fbp_par2d(s64, (128, 128), (1.0, 1.0), 1.0, ang))}
    out["par2d_128"] = {"workload": "2D parallel 128^2 (1 mm), 180 views over 180 deg, 183 bins",
                        "gpu_ms": {k: round(v, 4) for k, v in t.items()},
                        "fp_gsamples_per_s": round(ns / (t["fp"] * 1e-3) / 1e9, 2),
                        "bp_gups": round(nb / (t["bp"] * 1e-3) / 1e9, 2), "clocks": clk.summary(),
                        "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(),
                                         "seconds": {k: round(v, 4) for k, v in c.items()},
                                         "fp_gsamples_per_s": round(ns / c["fp"] / 1e9, 4),
                                         "bp_gups": round(nb / c["bp"] / 1e9, 4)}}
    # 16 x 512^2 fan beam
    gf = FanGeometry2D((512, 512), (0.5, 0.5), 1024, 1.0, 360, 2 * math.pi, 750.0, 1200.0, step=0.25)
    imgs = torch.stack([ph.voxelize_ellipses(ph.random_ellipses(10, 128.0, seed=s), (512, 512), (0.5, 0.5),
                                             device=dev, dtype=torch.float32) for s in range(16)])
    sf = B.pyro_fp_fan2d(imgs, gf)
    angf = gf.view_angles()
    i0, s0 = imgs[0].double().cpu().numpy(), sf[0].double().cpu().numpy()
    ns, nb = samples2d(gf, 16), 16 * 512 * 512 * 360
    wsf = torch.empty(B.fp2d_workspace_bytes(gf, 16), dtype=torch.uint8, device=dev)
    with ClockSampler(dev.index or 0) as clk:
        t = {"fp": gpu_ms(lambda: B.pyro_fp_fan2d(imgs, gf)),
             "fp_staged": gpu_ms(lambda: B.pyro_fp_fan2d_ws(imgs, gf, workspace=wsf)),
             "fpT": gpu_ms(lambda: B.pyro_fpT_fan2d(sf, gf)),
             "fpT_staged": gpu_ms(lambda: B.pyro_fpT_fan2d_ws(sf, gf, workspace=wsf)),
             "bp": gpu_ms(lambda: B.pyro_bp_fan2d(sf, gf, weight=B.W_INV_L2, scale=1.0))}
    c = {"fp": cpu_s(lambda: oracle.fp_fan2d(i0, (0.5, 0.5), 1024, 1.0, angf, 750.0, 1200.0, step=0.25)),
         "fpT": cpu_s(lambda: oracle.fpT_fan2d(s0, (512, 512), (0.5, 0.5), 1.0, angf, 750.0, 1200.0, step=0.25)),
         "bp": cpu_s(lambda: oracle.bp_fan2d(s0, (512, 512), (0.5, 0.5), 1.0, angf, 750.0, 1200.0, 2, 1.0))}
    out["fan2d_16x512"] = {"workload": "2D fan 16 x 512^2 (0.5 mm), 360 views over 360 deg, 1024 bins (1 mm), "
                                       "SID 750, SDD 1200",
                           "gpu_ms": {k: round(v, 4) for k, v in t.items()},
                           "fp_gsamples_per_s": round(ns / (t["fp"] * 1e-3) / 1e9, 2),
                           "fp_staged_gsamples_per_s": round(ns / (t["fp_staged"] * 1e-3) / 1e9, 2),
                           "fpT_gsamples_per_s": round(ns / (t["fpT"] * 1e-3) / 1e9, 2),
                           "fpT_staged_gsamples_per_s": round(ns / (t["fpT_staged"] * 1e-3) / 1e9, 2),
                           "bp_gups": round(nb / (t["bp"] * 1e-3) / 1e9, 2), "clocks": clk.summary(),
                           "cpu_baseline": {"kind": "oracle", "cores": oracle.num_threads(),
                                            "sample": "one of the 16 phantoms",
                                            "seconds": {k: round(v, 4) for k, v in c.items()},
                                            "fp_gsamples_per_s": round(ns / 16 / c["fp"] / 1e9, 4),
                                            "bp_gups": round(nb / 16 / c["bp"] / 1e9, 4)}}
    return out


def _timed_ms(dev, fn, reps=5, flush=None):
    """median CUDA-event time of fn() on the current stream after one warm-up"""
    stream = torch.cuda.current_stream(dev)
    fn()
    torch.cuda.synchronize(dev)
    ts = []
    for _ in range(reps):
        if flush is not None:
            flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def _rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(f"{np.linalg.norm(a - b) / np.linalg.norm(b):.3g}")


def measure_fp16_arm(dev, g, vol, flush):
    """The 256^3 workload with 16-bit storage: FP of the FP16 volume (FP16
    sinogram), FP of the FP32 volume from an FP16 workspace copy (FP32
    sinogram), FDK of the FP16 sinogram (FP16 volume); each against the
    oracle fed the FP32 input (end to end, storage rounding included) on
    sampled rays / voxels."""
    import oracle

    from paper_1904_13342_gb300 import binding as B

    ang = g.view_angles()
    P = oracle.circular_pmats(ang, SID, SDD, (NV, NU), (SV, SU))
    v16 = vol.half()
    ws16 = torch.empty(B.fp_cone3d_workspace_bytes(g, torch.float16), dtype=torch.uint8, device=dev)
    s16 = torch.empty((VIEWS, NV, NU), dtype=torch.float16, device=dev)
    s32 = torch.empty((VIEWS, NV, NU), dtype=torch.float32, device=dev)
    ws_fdk = torch.empty(B.lib().pyro_fdk_workspace_bytes(ctypes.byref(g.to_c()), 1), dtype=torch.uint8, device=dev)
    with ClockSampler(dev.index or 0) as clk:
        t_fp16 = _timed_ms(dev, lambda: B.pyro_fp_cone3d_ws(v16, g, workspace=ws16, out=s16), flush=flush)
        t_fp_st = _timed_ms(dev, lambda: B.pyro_fp_cone3d_ws_storage(vol, g, torch.float16, workspace=ws16, out=s32),
                            flush=flush)
        sino32 = B.pyro_fp_cone3d_ws(vol, g)
        y16 = sino32.half()
        t_fdk16 = _timed_ms(dev, lambda: B.pyro_fdk(y16, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER,
                                                     workspace=ws_fdk), flush=flush)
    rec16 = B.pyro_fdk(y16, g, kind=B.SHEPP_LOGAN, redund=B.REDUND_PARKER, workspace=ws_fdk)
    torch.cuda.synchronize(dev)
    rng = np.random.default_rng(3)
    vs, ks, ls = rng.integers(0, VIEWS, 200), rng.integers(0, NU, 200), rng.integers(0, NV, 200)
    v64 = vol.double().cpu().numpy()
    ref_rays = oracle.fp_cone3d_rays(v64, g.volume_spacing, P, vs, ks, ls)
    kk = np.repeat([N // 2, 37, N - 1], 12)
    ii, jj = rng.integers(0, N, kk.size), rng.integers(0, N, kk.size)
    fdk_vox = lambda y: oracle.fdk_voxels(y, g.volume_shape, g.volume_spacing, (SV, SU), ang, P, SID, SDD,
                                          g.angular_range / VIEWS, ii, jj, kk, kind=oracle.SHEPP_LOGAN,
                                          redund=oracle.REDUND_PARKER)
    ref_vox = fdk_vox(sino32.double().cpu().numpy())
    ref_vox16 = fdk_vox(y16.double().cpu().numpy())  # the oracle fed the FP16-rounded input
    return {"workload": WORKLOAD + ", 16-bit storage",
            "fp_f16_ms": round(t_fp16, 4), "fp_f32_volume_f16_copy_ms": round(t_fp_st, 4),
            "fdk_f16_ms": round(t_fdk16, 4),
            "fp_f16_rel_l2_vs_oracle_f32_input": _rel(s16[vs, ls, ks].double().cpu().numpy(), ref_rays),
            "fp_f16_copy_rel_l2_vs_oracle_f32_input": _rel(s32[vs, ls, ks].double().cpu().numpy(), ref_rays),
            "fdk_f16_rel_l2_vs_oracle_f32_input": _rel(rec16[kk, jj, ii].double().cpu().numpy(), ref_vox),
            "fdk_f16_rel_l2_vs_oracle_f16_rounded_input": _rel(rec16[kk, jj, ii].double().cpu().numpy(), ref_vox16),
            "gate": "2e-3 relative L2 (half storage)",
            "note": "the FDK's end-to-end error is the FP16 rounding of its input sinogram (about 1.6e-4 per "
                    "value) amplified by the ramp filter, which suppresses the projections' smooth content and "
                    "passes the white rounding noise; the kernel-only figure is against the oracle fed the same "
                    "FP16 values",
            "sample": "200 random rays, 36 voxels on three slices", "clocks": clk.summary()}


def measure_tv512_slice(dev, steps, lam, eps=1e-3):
    """A short slice of the 512^3 TV workload: `steps` gradient steps of Eq. 7
    with FP32 storage and with an FP16 copy of the iterate for the projector,
    seconds per step (after one untimed step), on the workload's geometry
    (0.5 mm, 496 views over 360 deg, 1240 x 960 at 0.308 mm, 1 % noise)."""
    import math

    from paper_1904_13342_gb300 import binding as B
    from paper_1904_13342_gb300 import phantoms as ph
    from paper_1904_13342_gb300.geometry import ConeGeometry3D
    from paper_1904_13342_gb300.tv import estimate_lipschitz, tv_reconstruct

    n, s = 512, 0.5
    g = ConeGeometry3D((n, n, n), (s, s, s), (960, 1240), (0.308, 0.308), 496, 2 * math.pi, 750.0, 1200.0)
    truth = ph.voxelize_ellipsoids(ph.random_ellipsoids(20, n * s / 2, seed=0), g.volume_shape, g.volume_spacing,
                                   device=dev, dtype=torch.float32)
    p = B.pyro_fp_cone3d_ws(truth, g)
    gen = torch.Generator(device=dev).manual_seed(1)
    p += (0.01 * float(p.abs().max())) * torch.randn(p.shape, generator=gen, device=dev)
    L_est = estimate_lipschitz(g, g.volume_shape, dev, iters=3)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": "TV 512^3 (0.5 mm), 496 views / 360 deg, 1240x960 det (0.308 mm), SID 750, SDD 1200, "
                       "1 % noise", "lambda": lam, "eps": eps, "steps_timed": steps,
           "L_est": "3 power iterations of 2 A^T A"}
    xs = {}
    for name, st in (("f32", None), ("f16_copy", torch.float16)):
        x1 = tv_reconstruct(p, g, 1, lam, eps, L_est=L_est, storage=st).x
        torch.cuda.synchronize(dev)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(dev.index or 0) as clk:
            a.record(stream)
            res = tv_reconstruct(p, g, steps, lam, eps, L_est=L_est, x0=x1, storage=st)
            b.record(stream)
            torch.cuda.synchronize(dev)
        out[f"{name}_s_per_step"] = round(a.elapsed_time(b) / 1e3 / steps, 4)
        out[f"{name}_clocks"] = clk.summary()
        xs[name] = res.x
    out["f16_copy_rel_l2_vs_f32_iterate"] = _rel(xs["f16_copy"].double().cpu().numpy(),
                                                 xs["f32"].double().cpu().numpy())
    del p, truth, xs
    torch.cuda.empty_cache()
    return out


def measure_tv_vs_oracle(dev, steps, lam, eps=1e-3):
    """Eq. 7 on a 64^3 problem with the 512^3 workload's voxel and detector
    pitch (0.5 mm voxels, 160 x 160 detector at 0.308 mm, 62 views over
    360 deg, SID 750, SDD 1200, 1 % noise): the GPU iterate after `steps`
    steps (FP32, and with an FP16 copy for the projector) against the FP64
    oracle's iterate of the same algorithm (the same L_est, from 6 oracle
    power iterations); the error the 512^3 run cannot check."""
    import oracle

    from paper_1904_13342_gb300 import phantoms as ph
    from paper_1904_13342_gb300.geometry import ConeGeometry3D
    from paper_1904_13342_gb300.tv import tv_reconstruct
    import math

    n, s, det, dsp, views = 64, 0.5, (160, 160), (0.308, 0.308), 62
    g = ConeGeometry3D((n, n, n), (s, s, s), det, dsp, views, 2 * math.pi, 750.0, 1200.0)
    ang = g.view_angles()
    P = oracle.circular_pmats(ang, 750.0, 1200.0, det, dsp)
    truth = ph.voxelize_ellipsoids(ph.random_ellipsoids(20, n * s / 2, seed=0), g.volume_shape,
                                   g.volume_spacing).numpy()
    fwd = lambda x: oracle.fp_cone3d(x, (s, s, s), det, P)
    kk, jj, ii = (a.ravel() for a in np.meshgrid(*(np.arange(n),) * 3, indexing="ij"))
    adj = lambda y: oracle.fpT_cone3d_voxels(y, (n, n, n), (s, s, s), P, ii, jj, kk).reshape(n, n, n)
    t0 = time.perf_counter()
    p = fwd(truth)
    p = np.asarray(p + 0.01 * p.max() * np.random.default_rng(1).standard_normal(p.shape), np.float32)
    p = p.astype(np.float64)
    L = oracle.lipschitz(fwd, adj, (n, n, n), iters=6)
    x_ref, _ = oracle.tv_solve(p, fwd, adj, lam, eps, steps, L)
    t_oracle = time.perf_counter() - t0
    pd = torch.from_numpy(p).float().to(dev)
    with ClockSampler(dev.index or 0) as clk:
        x32 = tv_reconstruct(pd, g, steps, lam, eps, L_est=L).x.double().cpu().numpy()
        x16 = tv_reconstruct(pd, g, steps, lam, eps, L_est=L, storage=torch.float16).x.double().cpu().numpy()
    return {"workload": "TV 64^3 (0.5 mm), 62 views / 360 deg, 160x160 det (0.308 mm), SID 750, SDD 1200, 1 % noise",
            "steps": steps, "lambda": lam, "eps": eps,
            "f32_rel_l2_vs_oracle_iterate": _rel(x32, x_ref), "f16_copy_rel_l2_vs_oracle_iterate": _rel(x16, x_ref),
            "oracle_seconds": round(t_oracle, 2), "clocks": clk.summary()}


def run_configs(args):
    out = measure_configs_2d(torch.device("cuda:0"))
    line = {"metric": "2D workloads: FP samples/s and BP GUPS, GPU against the oracle",
            "value": out["fan2d_16x512"]["bp_gups"], "unit": "GUPS (fan BP)", "higher_is_better": True, "n_gpus": 1,
            "dtype": "f32", "data": "synthetic (seeded random ellipses)", "vs_baseline": None,
            "config": {"workload": "2D parallel 128^2 x 180 views x 183 bins; fan 16 x 512^2 x 360 views x 1024 bins"},
            "results": out}
    print(json.dumps(line), flush=True)


def run_cnn128(args):
    """Forward pass of the residual CNN initialiser on two 128^3 volumes
    (BF16 activations and weights, FP32 accumulation; random-init weights of
    the network's architecture, synthetic inputs): W warm-up passes, then K
    timed passes with CUDA events, and the per-layer convolution times."""
    from paper_1904_13342_gb300 import binding as B
    from paper_1904_13342_gb300.cnn import LAYERS, ResidualCNN

    dev = torch.device("cuda:0")
    net = ResidualCNN(device="cuda", seed=0)
    g = torch.Generator().manual_seed(0)
    x = torch.rand((2, 128, 128, 128), generator=g).to(dev)
    out, acts = net.forward(x, keep=True)
    inputs = {"c0": "x16", "c1": "a0", "c2": "p1", "c3": "a2", "c4": "p2", "c5": "a4", "c6": "p3", "c7": "a6",
              "c8": "u3", "c9": "u2", "c10": "u1", "c11": "a10"}
    layers = {}
    for name, cin, cout in LAYERS:
        xin, p = acts[inputs[name]], net.params[name]
        ms = _timed_ms(dev, lambda: B.pyro_conv3d(xin, p.w16, p.b, name != "c11"), reps=5)
        vox = xin.numel() // cin
        layers[name] = {"cin": cin, "cout": cout, "size": list(xin.shape[1:4]), "ms": round(ms, 4),
                        "tflops": round(2 * 27 * cin * cout * vox / (ms * 1e-3) / 1e12, 1)}
    for _ in range(max(args.warmup, 3)):
        net.forward(x)
    torch.cuda.synchronize(dev)
    with ClockSampler(dev.index or 0) as clk:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            net.forward(x)
        b.record()
        torch.cuda.synchronize(dev)
    ms = a.elapsed_time(b) / args.steps
    line = {"metric": "residual CNN forward, ms per pass", "value": round(ms, 4), "unit": "ms",
            "higher_is_better": False, "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "dtype": "bf16 (FP32 accumulate)", "data": "synthetic (uniform random volumes, random-init weights)",
            "vs_baseline": None,
            "config": {"workload": "residual CNN initialiser forward, 2 x 128^3 volumes, 12 3x3x3 convolutions",
                       "l2": "inputs (2 x 128^3 x 16 channels, 134 MB per activation) larger than L2"},
            "layers": layers, "clocks": clk.summary()}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--workload", default="fdk-256", choices=["fdk-256", "learned-init", "tv-512", "configs", "cnn-128"])
    ap.add_argument("--train-steps", type=int, default=1000)
    ap.add_argument("--tv-lambda", type=float, default=10.0)
    ap.add_argument("--tv-steps", type=int, default=3, help="TV steps of the 512^3 slice and the 64^3 oracle check")
    ap.add_argument("--no-extras", dest="extras", action="store_false",
                    help="only the 256^3 FP + FDK line (no 2D, FP16, TV keys)")
    args = ap.parse_args()
    if args.workload == "learned-init":
        run_learned_init(args)
    elif args.workload == "tv-512":
        run_tv512(args)
    elif args.workload == "configs":
        run_configs(args)
    elif args.workload == "cnn-128":
        run_cnn128(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
