#!/usr/bin/env python
"""Benchmark: rank-k randomized SVD wall time and HBM-roofline fraction on GB300.

Default workload (N = 1): rSVD of a 200000 x 2000 FP32 matrix with planted
spectrum sigma_i = 1/i plus i.i.d. N(0, 1e-3^2) noise, k = 100, p = 10, q = 2
(2q + 2 = 6 passes over A).  A (1.6 GB) is larger than L2 (129 MB), so every
pass streams it from HBM; no extra L2 flush is needed between steps.

One step = one full rsvdgb_rsvd call (Omega, sketch, q subspace iterations
with CholeskyQR, projection, SVD of B, back-projection) through the C ABI with
A resident in HBM.  `value` is milliseconds per rSVD for the whole job (with
N ranks each factoring its own matrix: max-over-ranks time / (N * steps)).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle on the host cores (a bounded row
sample of the same workload, scaled to the full row count).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rank-k rSVD wall time and % HBM roofline, mixed/learned-q vs FP32 at equal error"

WORKLOADS = {
    "spiked200k": dict(desc="rsvd 200000x2000 fp32, sigma_i=1/i + N(0,1e-3^2) noise, k=100 p=10 q=2",
                       m=200000, n=2000, k=100, p=10, q=2, noise=1e-3),
    "spiked50k": dict(desc="rsvd 50000x2000 fp32, sigma_i=1/i + N(0,1e-3^2) noise, k=100 p=10 q=2 (profiling size)",
                      m=50000, n=2000, k=100, p=10, q=2, noise=1e-3),
    "c3bf16": dict(desc="rsvd 100000x50000 bf16, sigma=1 (i<=200), 1e-2 beyond, + N(0,1e-4^2) noise, "
                        "k=200 p=20 q=3", m=100000, n=50000, k=200, p=20, q=3, noise=1e-4, step=200,
                   dtype="bf16", cpu_rows=1000),
    "planted2k": dict(desc="rsvd 2000x1000 fp32, sigma_i=exp(-i/20), k=20 p=10 q=2",
                      m=2000, n=1000, k=20, p=10, q=2, noise=0.0),
}

# DRAM bytes (read + write) per byte of A of the FP32 tensor-core pass kernel,
# per launch, from one ncu capture (--set full, the first two launches of the
# 200000 x 2000 rSVD): the first pass (3xTF32, Y written) 1.711 GB and an
# A^T-side FP16x3 pass (panel read) 1.694 GB, for 1.6 GB of A each.
TC_PASS_TRAFFIC_PER_A_BYTE = (1.711e9 + 1.694e9) / 2 / 1.6e9

# The roofline the method's target is stated against: bytes of A per pass x
# passes at 8 TB/s (nominal HBM3e); the measured copy bandwidth is the other.
NOMINAL_HBM_TBS = 8.0

# FP32 FMA peak from unit counts: 152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz.
SIMT_FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="spiked200k")
    ap.add_argument("--prec", default="fp32")
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-rows", type=int, default=40000, help="row sample for the oracle baseline")
    ap.add_argument("--batched", type=int, default=4096, help="matrices in the batched workload (0 = skip)")
    ap.add_argument("--rpca", type=int, default=1, help="time the randomized PCA workload (0 = skip)")
    ap.add_argument("--small", type=int, default=1, help="time the 2000 x 1000 planted workload (0 = skip)")
    ap.add_argument("--rid", type=int, default=1, help="time the interpolative and CUR decompositions (0 = skip)")
    ap.add_argument("--rrpca", type=int, default=1, help="time the robust PCA workload (0 = skip)")
    ap.add_argument("--variants", type=int, default=1,
                    help="time the other precision and the learned mode on the same A (0 = skip)")
    ap.add_argument("--controller-eval", type=int, default=64,
                    help="held-out 20000x5000 matrices for the learned-(q, p) evaluation (0 = skip)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = (uuid or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            if self.uuid and self.uuid not in parts[0].lower():
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def dist_setup(n_gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value, device):
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_matrix(wl, seed, device):
    import numpy as np
    from paper_1608_02148_gb300 import inputs
    m, n = wl["m"], wl["n"]
    if wl.get("step"):
        # step spectrum on structured orthogonal factors, noise, stored BF16
        return inputs.step_noise(m, n, wl["step"], wl["noise"], seed, device=device, bf16=wl.get("dtype") == "bf16")
    if wl["noise"] > 0:
        sigma = 1.0 / np.arange(1, n + 1, dtype=np.float64)
        return inputs.spiked_noise(m, n, sigma, wl["noise"], seed, device=device)
    import torch
    return torch.from_numpy(inputs.planted(m, n, inputs.exp_spectrum(n, 1.0 / 20.0), seed)).to(device)


def run_small(rs, h, dev, stream, steps):
    """The small planted workload (2000 x 1000, sigma_i = exp(-i/20), k = 20,
    p = 10, q = 2): device time of the rSVD, and its rank-k error (the
    device's own estimate) against the planted optimum, known in closed form."""
    import numpy as np
    import torch
    from paper_1608_02148_gb300 import inputs
    wl = WORKLOADS["planted2k"]
    A = torch.from_numpy(inputs.small_planted()).to(dev)
    sigma = inputs.exp_spectrum(wl["n"], 1.0 / 20.0)
    k = wl["k"]
    opts = rs.make_opts(p=wl["p"], q=wl["q"], seed=1)
    for _ in range(3):
        rs.rsvdgb_rsvd(h, A, k, opts=opts, sync_info=False)
    n_steps = max(steps, 20)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(n_steps):
        rs.rsvdgb_rsvd(h, A, k, opts=opts, sync_info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    _, _, _, info = rs.rsvdgb_rsvd(h, A, k, opts=opts)
    opt = float(np.sqrt(np.sum(sigma[k:] ** 2)))
    err = float(np.sqrt(max(info.err2_k, 0.0)))
    return {"workload": wl["desc"], "ms": e0.elapsed_time(e1) / n_steps, "steps": n_steps, "status": info.status,
            "err_k_fro": err, "optimum_k_fro": opt, "err_ratio_vs_optimum": err / opt}


def run_batched(rs, h, dev, stream, count, steps, peaks):
    """Batched rSVD of `count` matrices, m log-uniform in [256, 4096], n in
    [64, 1024], exponential spectra with rates uniform in [0.05, 0.5];
    k = 16, p = 8, q = 1; one graph launch per step."""
    import torch
    from paper_1608_02148_gb300 import inputs
    k, p, q = 16, 8, 1
    t0 = time.perf_counter()
    mats, _ = inputs.ragged_batch(count, seed=0x160802148 + 4000, device=dev)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    call = rs.BatchedCall(mats, k)
    opts = rs.make_opts(p=p, q=q, seed=3)
    t0 = time.perf_counter()
    rs.rsvdgb_rsvd_batched(h, call, opts)  # plan, tuning, graph capture
    torch.cuda.synchronize()
    plan_s = time.perf_counter() - t0
    for _ in range(2):
        rs.rsvdgb_rsvd_batched(h, call, opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    n = max(3, steps // 2)
    l0 = rs.rsvdgb_kernel_launches()
    e0.record(stream)
    for _ in range(n):
        rs.rsvdgb_rsvd_batched(h, call, opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    launches = (rs.rsvdgb_kernel_launches() - l0) / n
    a_bytes = sum(A.numel() * 4 for A in mats)
    passes = 2 * q + 2
    roof_ms = passes * a_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    bad = sum(1 for b in range(0, count, max(1, count // 64)) if call.info(b).status != 0)
    return {"workload": f"batched rsvd of {count} matrices, m in [256,4096], n in [64,1024] log-uniform, "
                        f"exp spectra rate U[0.05,0.5], k={k} p={p} q={q}, fp32",
            "ms": ms, "matrices_per_s": count / (ms * 1e-3), "a_bytes": a_bytes, "passes_over_A": passes,
            "hbm_roofline_ms": roof_ms, "hbm_frac": roof_ms / ms, "graph_launches_per_step": 1,
            "kernels_per_step": launches, "plan_build_s": plan_s, "input_generation_s": gen_s,
            "status_nonzero_sampled": bad}


def run_rpca(rs, h, dev, stream, steps, peaks, cpu_baseline, e2e_steps):
    """Randomized PCA (Algorithm rpca, correlation PCA: centre + scale, scores
    returned) of 200000 observations x 2000 variables with heterogeneous units
    (inputs.pca_data: rank-100 factor model, loadings decaying 0.85^j, noise
    0.05, column scales log-uniform in [0.1, 10], offsets 5 spreads);
    k = 100, p = 10, q = 2: 1 statistics pass + 2q + 2 passes over A."""
    import torch
    from paper_1608_02148_gb300 import inputs
    m, n, k, p, q = 200000, 2000, 100, 10, 2
    A = inputs.pca_data(m, n, 100, seed=0x160802148 + 6000, device=dev)
    opts = rs.make_opts(p=p, q=q, seed=1)
    for _ in range(2):
        r = rs.rsvdgb_rpca(h, A, k, opts=opts, sync_info=False)
    torch.cuda.synchronize()
    info = rs._info_from(r["info"])
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    nsteps = max(3, steps)
    l0 = rs.rsvdgb_kernel_launches()
    e0.record(stream)
    for _ in range(nsteps):
        rs.rsvdgb_rpca(h, A, k, opts=opts, sync_info=False)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / nsteps
    launches = (rs.rsvdgb_kernel_launches() - l0) / nsteps
    a_bytes = m * n * 4
    passes = 2 * q + 3
    roof_ms = passes * a_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
    out = {"workload": "rpca 200000x2000 fp32 (correlation PCA, scores), rank-100 factor model + noise, "
                       "heterogeneous units and offsets, k=100 p=10 q=2",
           "ms": ms, "passes_over_A": passes, "hbm_roofline_ms": roof_ms, "hbm_frac": roof_ms / ms,
           "kernels_per_step": launches, "status": info.status,
           "explained_variance_k": float(r["eigvals"].double().sum()) / n}
    if e2e_steps > 0:
        A_host = A.cpu().pin_memory()
        rs.rsvdgb_rpca_host(h, A_host, k, opts=opts)
        ts = []
        for _ in range(e2e_steps):
            t0 = time.perf_counter()
            rs.rsvdgb_rpca_host(h, A_host, k, opts=opts)
            ts.append((time.perf_counter() - t0) * 1e3)
        out["e2e"] = {"value": statistics.median(ts), "unit": "ms", "h2d_bytes_per_step": a_bytes,
                      "d2h_bytes_per_step": 4 * (2 * k + n * k + m * k + 2 * n) + rs.INFO_BYTES}
    if cpu_baseline:
        import oracle
        oracle.build()
        rows = 20000
        A_rows = A[:rows].cpu().numpy()
        t0 = time.perf_counter()
        oracle.rpca(A_rows, k, p=p, q=q, seed=1)
        t = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": t * (m / rows) * 1e3, "unit": "ms", "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": f"oracle rpca on rows 0..{rows - 1} ({rows}x{n}), time x{m / rows:g}"}
    del A
    return out


def run_rid(rs, h, A, wl, stream, steps, peaks, cpu_baseline):
    """Algorithms rid and rcur (Sec. 7) on the benchmark matrix: rank k,
    the workload's p and q (2q + 2 passes over A), then the column-pivoted QR
    of B (and of C^T for rcur), the gathers and U = Z pinv(R)."""
    import torch
    m, n = A.shape
    k = wl["k"]
    opts = rs.make_opts(p=wl["p"], q=wl["q"], seed=2)
    out = {"workload": f"rid / rcur of the {m}x{n} benchmark matrix, k={k} p={wl['p']} q={wl['q']}"}
    a_bytes = m * n * 4
    passes = 2 * wl["q"] + 2
    for name, fn in (("rid", rs.rsvdgb_rid), ("rcur", rs.rsvdgb_rcur)):
        for _ in range(2):
            r = fn(h, A, k, opts=opts, sync_info=False)
        torch.cuda.synchronize()
        info = rs._info_from(r["info"])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        nsteps = max(3, steps // 2)
        e0.record(stream)
        for _ in range(nsteps):
            fn(h, A, k, opts=opts, sync_info=False)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / nsteps
        roof = passes * a_bytes / (peaks["hbm_gbs"] * 1e9) * 1e3
        Af = A.double()
        if name == "rid":
            err = float(torch.linalg.matrix_norm(Af - r["C"].double() @ r["Z"].double()))
        else:
            err = float(torch.linalg.matrix_norm(Af - r["C"].double() @ r["U"].double() @ r["R"].double()))
        del Af
        out[name] = {"ms": ms, "passes_over_A": passes, "hbm_roofline_ms": roof, "hbm_frac": roof / ms,
                     "status": info.status, "err_fro": err}
    if cpu_baseline:
        import oracle
        oracle.build()
        rows = 20000
        A_rows = A[:rows].cpu().numpy()
        t0 = time.perf_counter()
        oracle.rid(A_rows, k, p=wl["p"], q=wl["q"], seed=2)
        t = time.perf_counter() - t0
        out["cpu_baseline"] = {"value": t * (m / rows) * 1e3, "unit": "ms", "cores": oracle.num_threads(),
                               "kind": "oracle",
                               "sample": f"oracle rid on rows 0..{rows - 1} ({rows}x{n}), time x{m / rows:g}"}
    return out


def run_rrpca(rs, h, dev, stream, peaks):
    """Robust PCA (Algorithm rrpca) of a 20000 x 2000 matrix: rank-20 part
    plus 5 % gross corruptions (inputs.low_rank_plus_sparse), p = 10, q = 2,
    tolerance 1e-5.  One step = the whole IALM loop (host-driven); per
    iteration: one rSVD of X (2q + 2 passes over m x n) and one fused update
    pass (reads A, S, Z; writes S, Z, X)."""
    import numpy as np
    import torch
    from paper_1608_02148_gb300 import inputs
    m, n, rank, dens = 20000, 2000, 20, 0.05
    L0, S0, A64 = inputs.low_rank_plus_sparse(m, n, rank, dens, seed=0x160802148 + 7000)
    A = torch.from_numpy(A64.astype(np.float32)).to(dev)
    opts = rs.make_opts(p=10, q=2, seed=5)
    r = rs.rsvdgb_rrpca(h, A, opts=opts)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = rs.rsvdgb_rrpca(h, A, opts=opts)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    res = r["result"]
    L = r["L"].double().cpu().numpy()
    rec = float(np.linalg.norm(L - L0) / np.linalg.norm(L0))
    it = max(res.iters, 1)
    # per iteration: rSVD passes over X plus the fused update (3 reads + 3 writes of m x n)
    bytes_it = (2 * 2 + 2) * m * n * 4 + 6 * m * n * 4
    roof_ms = it * bytes_it / (peaks["hbm_gbs"] * 1e9) * 1e3
    return {"workload": f"rrpca {m}x{n} fp32, rank {rank} + {int(dens * 100)}% gross corruptions, p=10 q=2 tol=1e-5",
            "ms": ms, "iters": res.iters, "ms_per_iter": ms / it, "rank": res.rank, "err": res.err,
            "L_rel_err_vs_planted": rec, "hbm_roofline_ms": roof_ms, "hbm_frac": roof_ms / ms, "status": res.status}


def workload_config(wl, world):
    """The workload as both arms report it (no implementation keys)."""
    m, n = wl["m"], wl["n"]
    a_bytes = m * n * (2 if wl.get("dtype") == "bf16" else 4)
    return {"workload": wl["desc"], "m": m, "n": n, "k": wl["k"], "p": wl["p"], "q": wl["q"],
            "l": min(wl["k"] + wl["p"], m, n), "passes_over_A": 2 * wl["q"] + 2,
            "l2": "A (%.1f GB) larger than L2; no flush needed" % (a_bytes / 1e9),
            "parallelism": f"replicas x{world}"}


def cpu_oracle_time(A_host_rows, wl, seed_omega):
    """One timing of the FP64 oracle rSVD on a row block (callers take medians)."""
    import oracle
    t0 = time.perf_counter()
    oracle.rsvd(A_host_rows, wl["k"], p=wl["p"], q=wl["q"], seed=seed_omega)
    return time.perf_counter() - t0


def run_reference(args, wl):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    from paper_1608_02148_gb300 import inputs
    oracle.build()
    rows = min(wl["m"], 10000)
    rng_seed = 0x160802148 + 2000
    # same recipe as the GPU workload, on the host, restricted to a row block
    if wl["noise"] > 0:
        sigma = 1.0 / np.arange(1, wl["n"] + 1, dtype=np.float64)
        A = inputs.spiked_noise(rows, wl["n"], sigma, wl["noise"], rng_seed,
                                device="cpu").numpy()
    else:
        A = inputs.planted(rows, wl["n"], inputs.exp_spectrum(wl["n"], 1.0 / 20.0), rng_seed)
    scale = wl["m"] / rows
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_time(A, wl, 0)
    times = [cpu_oracle_time(A, wl, 0) * scale * 1e3 for _ in range(args.steps)]
    ms = statistics.median(times)
    cores = oracle.num_threads()
    # value: the metric on the whole workload (the sample's time x rows / sample
    # rows); ms_per_step: what each timed step actually took (the sample)
    line = {"metric": METRIC, "impl": "reference", "value": ms, "unit": "ms", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / scale, "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(wl, world),
            "implementation": {"prec": "fp64 oracle (plain C, OpenMP)", "engine": "host cores"},
            "cpu_baseline": {"value": ms, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"oracle rsvd on a {rows}x{wl['n']} row block of the workload, time x{scale:g}"},
            "value_scale": scale,
            "e2e": {"value": ms, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        return run_reference(args, wl)

    import numpy as np
    import torch
    from paper_1608_02148_gb300 import build as cuda_build
    from paper_1608_02148_gb300 import rsvdgb as rs

    world, rank, local = dist_setup(args.gpus)
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    if rank == 0 or not os.path.exists(cuda_build.LIB):
        cuda_build.build()
    barrier(world)
    stream = torch.cuda.current_stream(dev)
    h = rs.Handle(local, stream)
    peaks, peak_kind = measured_peaks()

    seed = 0x160802148 + 2000 + rank
    A = make_matrix(wl, seed, dev)
    torch.cuda.synchronize()
    m, n, k = wl["m"], wl["n"], wl["k"]
    opts = rs.make_opts(p=wl["p"], q=wl["q"], seed=rank, prec=args.prec, engine=args.engine)
    bufs = (torch.empty(k, device=dev), torch.empty(m, k, device=dev), torch.empty(n, k, device=dev),
            torch.zeros(rs.INFO_BYTES, dtype=torch.uint8, device=dev))

    for _ in range(max(args.warmup, 0)):
        rs.rsvdgb_rsvd(h, A, k, opts=opts, out=bufs, sync_info=False)
    torch.cuda.synchronize()
    info = rs._info_from(bufs[3])
    if info.status != 0:
        raise SystemExit(f"rsvd reported {info.as_dict()}")

    # ---------------- timed region (device-resident A) ----------------
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    rs.rsvdgb_profile_passes(h, True)
    launches0 = rs.rsvdgb_kernel_launches()
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        rs.rsvdgb_rsvd(h, A, k, opts=opts, out=bufs, sync_info=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    launches = rs.rsvdgb_kernel_launches() - launches0
    pass_ms, pass_n, pass_bytes = rs.rsvdgb_profile_read(h)
    rs.rsvdgb_profile_passes(h, False)
    elapsed = ev0.elapsed_time(ev1)
    elapsed = max_over_ranks(world, elapsed, dev)
    ms_per_step = elapsed / args.steps
    value = elapsed / (args.steps * world)

    passes = 2 * wl["q"] + 2
    a_bytes = m * n * (2 if A.dtype == torch.bfloat16 else 4)
    hbm = peaks["hbm_gbs"]
    roof_ms = passes * a_bytes / (hbm * 1e9) * 1e3
    pass_avg_ms = pass_ms / max(pass_n, 1)
    l = rs.rsvdgb_sketch_width(m, n, k, wl["p"])
    achieved_gbs = (pass_bytes / max(pass_n, 1)) / (pass_avg_ms * 1e-3) / 1e9
    achieved_tflops = (2.0 * m * n * l) / (pass_avg_ms * 1e-3) / 1e12
    engine = {1: "simt", 2: "tc_fp16x3", 3: "tc_tf32"}.get(info.engine, str(info.engine))
    if engine == "simt":
        roofline = {"bound": "alu", "achieved": achieved_tflops, "peak": SIMT_FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved_tflops / SIMT_FP32_PEAK_TFLOPS, "traffic": None,
                    "kernel": "simt_gemm (pass over A, FP32 FMA)",
                    "peak_source": "unit counts: 152 SM x 128 FP32 lanes x 2 flop x 2.07 GHz",
                    "hbm_view": {"achieved_gbs": achieved_gbs, "peak_gbs": hbm, "frac": achieved_gbs / hbm,
                                 "peak_source": peak_kind}}
    else:
        traffic = None
        if (TC_PASS_TRAFFIC_PER_A_BYTE is not None and args.prec == "fp32" and A.dtype == torch.float32
                and engine == "tc_fp16x3"):
            traffic = TC_PASS_TRAFFIC_PER_A_BYTE * a_bytes
        roofline = {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm, "unit": "GB/s",
                    "frac": achieved_gbs / hbm, "traffic": traffic, "peak_source": peak_kind,
                    "traffic_source": "ncu dram bytes per launch (first pass and an A^T-side pass, 200000x2000)"
                    if traffic is not None else None,
                    "kernel": ("f8_pass_kernel (E4M3 sketch and power passes, bytes of the E4M3 copy of A) and "
                               "tc_pass_kernel (FP16x3 projection, bytes of A)" if args.prec == "fp8_sketch" else
                               "tc_pass_kernel (BF16 sketch and power passes, FP16x3 projection)"
                               if args.prec == "bf16_sketch" else
                               "tc_pass_kernel (pass over A, tcgen05: the first pass 3xTF32 measuring max|A|, "
                               "the later passes scaled FP16x3)" if engine == "tc_fp16x3" else
                               "tc_pass_kernel (pass over A, tcgen05 3xTF32)"),
                    "tensor_view": {"achieved_tflops_algorithmic": achieved_tflops,
                                    "mma_products_per_k_step": 2 if A.dtype == torch.bfloat16 else 3}}

    # ---------------- the other precision at equal error (same A, same Omega) ----------------
    variants = {}
    others = [x for x in ("fp32", "bf16_sketch", "fp8_sketch") if x != args.prec]
    err_main = float(np.sqrt(max(info.err2_k, 0.0)))
    variants = {args.prec: {"ms": ms_per_step, "err_k_fro": err_main}}
    for other in others:
        try:
            if not args.variants:
                raise RuntimeError("skipped (--variants 0)")
            o2 = rs.make_opts(p=wl["p"], q=wl["q"], seed=rank, prec=other, engine=args.engine)
            for _ in range(2):
                rs.rsvdgb_rsvd(h, A, k, opts=o2, out=bufs, sync_info=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nv = max(3, args.steps // 2)
            for _ in range(nv):
                rs.rsvdgb_rsvd(h, A, k, opts=o2, out=bufs, sync_info=False)
            e1.record(stream)
            torch.cuda.synchronize()
            info2 = rs._info_from(bufs[3])
            err_other = float(np.sqrt(max(info2.err2_k, 0.0)))
            variants[other] = {"ms": e0.elapsed_time(e1) / nv, "err_k_fro": err_other,
                               "err_ratio_vs_" + args.prec: err_other / err_main if err_main > 0 else None,
                               "status": info2.status}
        except Exception as exc:  # a variant the build does not serve
            variants[other] = {"unavailable": str(exc)}

    # ---------------- the other test matrices of Sec. 2.3 on the same A ----------------
    if args.variants:
        for sd, power in (("unif", "subspace"), ("rademacher", "subspace"), ("normal", "lu")):
            name = f"{args.prec}_omega_{sd}" if power == "subspace" else f"{args.prec}_power_{power}"
            try:
                o4 = rs.make_opts(p=wl["p"], q=wl["q"], seed=rank, prec=args.prec, engine=args.engine, sdist=sd,
                                  power=power)
                for _ in range(2):
                    rs.rsvdgb_rsvd(h, A, k, opts=o4, out=bufs, sync_info=False)
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                nv = max(3, args.steps // 2)
                e0.record(stream)
                for _ in range(nv):
                    rs.rsvdgb_rsvd(h, A, k, opts=o4, out=bufs, sync_info=False)
                e1.record(stream)
                torch.cuda.synchronize()
                info4 = rs._info_from(bufs[3])
                err_main = float(np.sqrt(max(info.err2_k, 0.0)))
                err4 = float(np.sqrt(max(info4.err2_k, 0.0)))
                variants[name] = {
                    "ms": e0.elapsed_time(e1) / nv, "err_k_fro": err4,
                    "err_ratio_vs_" + args.prec: err4 / err_main if err_main > 0 else None}
            except Exception as exc:
                variants[name] = {"unavailable": str(exc)}

    # ---------------- learned (q, p) on the same A: the packaged controller ----------------
    ctl_path = os.path.join(ROOT, "paper_1608_02148_gb300", "controller_default.bin")
    if os.path.exists(ctl_path) and args.variants:
        try:
            rs.rsvdgb_controller_load(h, ctl_path)
            o3 = rs.make_opts(p=wl["p"], q=wl["q"], seed=rank, prec=args.prec, engine=args.engine,
                              q_mode="learned")
            for _ in range(2):
                rs.rsvdgb_rsvd(h, A, k, opts=o3, out=bufs, sync_info=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nv = max(3, args.steps // 2)
            for _ in range(nv):
                rs.rsvdgb_rsvd(h, A, k, opts=o3, out=bufs, sync_info=False)
            e1.record(stream)
            torch.cuda.synchronize()
            info3 = rs._info_from(bufs[3])
            err_main = float(np.sqrt(max(info.err2_k, 0.0)))
            err3 = float(np.sqrt(max(info3.err2_k, 0.0)))
            variants["learned_" + args.prec] = {
                "ms": e0.elapsed_time(e1) / nv, "err_k_fro": err3, "q_used": info3.q_used,
                "p_used": info3.p_used, "passes_over_A": 2 * info3.q_used + 2,
                "err_ratio_vs_" + args.prec: err3 / err_main if err_main > 0 else None}
        except Exception as exc:
            variants["learned_" + args.prec] = {"unavailable": str(exc)}

    # ---------------- learned (q, p) against fixed p = 10, q = 2 on held-out planted matrices ----------------
    controller = None
    if args.controller_eval > 0 and rank == 0 and os.path.exists(ctl_path):
        try:
            from paper_1608_02148_gb300 import controller_train as ct
            rs.rsvdgb_controller_load(h, ctl_path)
            t0 = time.perf_counter()
            controller = ct.evaluate(h, args.controller_eval, seed=0x160802148 + 5000 + 7777)
            controller["target"] = "||A - U S V^T||_F <= 1.05 x optimum + 1e-4 ||A||_F"
            controller["seconds"] = time.perf_counter() - t0
        except Exception as exc:
            controller = {"unavailable": str(exc)}

    # ---------------- batched workload: 4096 ragged matrices, one graph launch ----------------
    batched = None
    if args.batched > 0 and rank == 0:
        try:
            batched = run_batched(rs, h, dev, stream, args.batched, args.steps, peaks)
        except Exception as exc:
            batched = {"unavailable": str(exc)}

    # ---------------- the small planted workload (2000 x 1000) ----------------
    small = None
    if args.small > 0 and rank == 0:
        try:
            small = run_small(rs, h, dev, stream, args.steps)
        except Exception as exc:
            small = {"unavailable": str(exc)}

    # ---------------- interpolative and CUR decompositions (Algorithms rid, rcur) ----------------
    rid = None
    if args.rid > 0 and rank == 0 and A.dtype == torch.float32:
        try:
            rid = run_rid(rs, h, A, wl, stream, args.steps, peaks, world == 1 and not args.no_cpu_baseline)
        except Exception as exc:
            rid = {"unavailable": str(exc)}

    # ---------------- robust PCA (Algorithm rrpca) ----------------
    rrpca = None
    if args.rrpca > 0 and rank == 0 and args.workload == "spiked200k":
        try:
            rrpca = run_rrpca(rs, h, dev, stream, peaks)
        except Exception as exc:
            rrpca = {"unavailable": str(exc)}

    # ---------------- randomized PCA (Algorithm rpca) ----------------
    rpca = None
    if args.rpca > 0 and rank == 0 and args.workload == "spiked200k":
        try:
            rpca = run_rpca(rs, h, dev, stream, args.steps, peaks, world == 1 and not args.no_cpu_baseline,
                            args.e2e_steps)
        except Exception as exc:
            rpca = {"unavailable": str(exc)}

    # ---------------- end to end through the host-buffer entry point ----------------
    e2e = None
    if args.e2e_steps > 0:
        A_host = A.cpu().pin_memory()
        outs = (torch.empty(k, pin_memory=True), torch.empty(m, k, pin_memory=True),
                torch.empty(n, k, pin_memory=True))
        rs.rsvdgb_rsvd_host(h, A_host, k, opts=opts, out=outs)
        ts = []
        for _ in range(args.e2e_steps):
            barrier(world)
            t0 = time.perf_counter()
            rs.rsvdgb_rsvd_host(h, A_host, k, opts=opts, out=outs)
            ts.append((time.perf_counter() - t0) * 1e3)
        e2e_ms = max_over_ranks(world, statistics.median(ts), dev)
        e2e = {"value": e2e_ms / world, "unit": "ms", "h2d_bytes_per_step": a_bytes,
               "d2h_bytes_per_step": 4 * (k + m * k + n * k) + rs.INFO_BYTES}
        del A_host

    # ---------------- CPU oracle baseline (rank 0, N = 1 only) ----------------
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        rows = min(wl.get("cpu_rows", args.cpu_rows), m)
        if A.dtype == torch.bfloat16:  # the oracle reads BF16 bit patterns
            A_rows = A[:rows].view(torch.int16).cpu().numpy().view(np.uint16)
        else:
            A_rows = A[:rows].cpu().numpy()
        reps = [cpu_oracle_time(A_rows, wl, 0) for _ in range(5)]
        t = statistics.median(reps)
        cpu = {"value": t * (m / rows) * 1e3, "unit": "ms", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": f"oracle rsvd on rows 0..{rows - 1} of the same A ({rows}x{n}), median of 5, "
                         f"time x{m / rows:g}",
               "sample_s": [round(x, 4) for x in reps]}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16-stored A, f32 arithmetic" if A.dtype == torch.bfloat16 else "f32",
                "data": "synthetic",
                "config": workload_config(wl, world),
                "implementation": {"prec": args.prec, "engine": engine, "engine_requested": args.engine},
                "hbm_roofline": {"time_ms": roof_ms, "frac_of_step": roof_ms / ms_per_step,
                                 "peak_gbs": hbm, "peak_source": peak_kind},
                "hbm_roofline_nominal": {"time_ms": passes * a_bytes / (NOMINAL_HBM_TBS * 1e12) * 1e3,
                                         "frac_of_step": passes * a_bytes / (NOMINAL_HBM_TBS * 1e12) * 1e3
                                         / ms_per_step,
                                         "peak_gbs": NOMINAL_HBM_TBS * 1e3,
                                         "pass_kernel_frac": achieved_gbs / (NOMINAL_HBM_TBS * 1e3)
                                         if achieved_gbs else None,
                                         "peak_source": "nominal HBM3e (bytes of A per pass x passes / 8 TB/s)"},
                "roofline": roofline,
                "pass_kernels": {"launches": pass_n, "avg_ms": pass_avg_ms, "share_of_step":
                                 pass_ms / max(elapsed, 1e-9) if world == 1 else None},
                "variants": variants,
                "controller": controller,
                "batched": batched,
                "small_planted": small,
                "rpca": rpca,
                "rid": rid,
                "rrpca": rrpca,
                "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
                "info": info.as_dict()}
        print(json.dumps(line), flush=True)
    h.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
