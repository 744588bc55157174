"""Benchmark of the hot path: Y = Z X (Algorithm 1) and Psi = Z^H Phi (Algorithm 2) on the
Tucker-compressed coupling matrix of the 96^3-voxel, 1024-segment, 16-RHS workload
("precision": 2 mm voxels, 8-loop cylindrical coil, HOSVD tol 1e-6, complex64 storage).

One step = one Z X plus one Z^H Phi on 16 right-hand sides.  Metric = algorithmic TFLOP/s of
the step (Table III count, complex MAC = 8 flops, summed over both products), with the step
time and the relative error against the FP64 oracle on sampled outputs.  Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl zbc|reference] [--prec auto|...]

Multi-GPU: replicas only (each rank runs the whole workload; no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "precision"
METRIC = "Z·x and Z^H·v time (s) & TFLOP/s, batched TC vs plain FP32, rel err <= 1e-5"
UNIT = "TFLOP/s"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank_ms(ms, ws, device):
    """Max over ranks of a per-rank time: the job ends with its slowest rank."""
    if ws == 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_tflops(flops_per_rank, ms, ws):
    """Aggregate throughput of ws replicas, each doing flops_per_rank in the job's time ms."""
    return ws * flops_per_rank / (ms * 1e-3) / 1e12


# ---------------------------------------------------------------------------------------------
# workload construction on the GPU (assembly + HOSVD through the C ABI)
# ---------------------------------------------------------------------------------------------

def build_handle(w, zbc, torch, batch_cols=256):
    g, s = w.grid, w.segments
    ds = zbc.DeviceSegments(s)
    h = None
    t0 = time.time()
    for c0 in range(0, s.m, batch_cols):
        cols = torch.arange(c0, min(s.m, c0 + batch_cols), dtype=torch.int32, device="cuda")
        Z = zbc.colmajor(3 * g.nv, cols.numel(), torch.complex128)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cols, Z)
        h, st = zbc.tucker_compress(Z, g, w.tol, append_to=h)
        del Z
    torch.cuda.synchronize()
    return h, time.time() - t0


def algorithmic_flops(h, w, p):
    """Real flops of one product by the complexity count of Table III (complex MAC = 8 flops):
    per stored tensor the mode products of the decompression (n1 r1 r2 r3 + n1 n2 r2 r3 +
    n_v r3 complex MACs), plus the contraction with the p right-hand sides (q n_v M p MACs)."""
    ranks, _, _ = h.export()
    inf = h.info()
    n1, n2, n3 = w.grid.shape
    nv = n1 * n2 * n3
    r = np.asarray(ranks, dtype=np.float64).reshape(-1, 3)
    r1, r2, r3 = r[:, 0], r[:, 1], r[:, 2]
    dec = float((n1 * r1 * r2 * r3 + n1 * n2 * r2 * r3 + nv * r3).sum())
    return 8.0 * dec + 8.0 * inf.q * nv * inf.M * p


# ---------------------------------------------------------------------------------------------
# clocks sampling
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={CLOCK_QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------------------------
# oracle checks on sampled outputs
# ---------------------------------------------------------------------------------------------

def sampled_errors(tens, w, X, Phi, Ys, Psis, seed=2, nrows=512, ncols=12):
    """Relative errors of each path's Y (dict name -> array) on nrows sampled rows and of each
    path's Psi on ncols sampled columns, against the FP64 oracle."""
    from oracle import products, tucker
    g = w.grid
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(3 * g.nv, size=nrows, replace=False))
    Yo = products.matvec_rows(tens, g.shape, X, rows)
    cols = np.sort(rng.choice(len(tens), size=min(ncols, len(tens)), replace=False))
    Po = np.stack([tucker.decompress_column(tens[j], g.shape).conj() @ Phi for j in cols])
    ey = {n: float(np.linalg.norm(Y[rows] - Yo) / np.linalg.norm(Yo)) for n, Y in Ys.items()}
    ep = {n: float(np.linalg.norm(P[cols] - Po) / np.linalg.norm(Po)) for n, P in Psis.items()}
    return ey, ep


# ---------------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on a bounded sample
# ---------------------------------------------------------------------------------------------

def oracle_sample_rate(tens, w, X, Phi, F_total, budget_s=15.0):
    """Time the oracle's Algorithms 1 and 2 over a growing prefix of the columns until about
    budget_s of CPU work; return (TFLOP/s scaled to the full workload, columns used)."""
    from oracle import products
    M = len(tens)
    ncol = 4
    t_used, used = 0.0, 0
    while True:
        sub = tens[:ncol]
        t0 = time.perf_counter()
        products.matvec(sub, w.grid.shape, X[:ncol])
        products.rmatvec(sub, w.grid.shape, Phi)
        dt = time.perf_counter() - t0
        t_used, used = dt, ncol
        if dt > budget_s / 3 or ncol >= M:
            break
        ncol = min(M, ncol * 2)
    t_full = t_used * M / used
    return F_total / t_full / 1e12, used, t_used


# ---------------------------------------------------------------------------------------------

def time_steps(fn, steps, flush, torch, stream):
    times = []
    for _ in range(steps):
        flush()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    return times


def mode1_gemm_flops(h, w, p, forward=False):
    """Real tensor-core flops of the mode-1 form's GEMMs, 3 fp16 products (hi.hi, hi.lo, lo.hi)
    per real MAC.  Adjoint: per group of 128 (column, rank) rows of one component, M = 128,
    K = 2 n1p (n1 rounded up to 8, whatever the i1 tiling), N = 2 n2 n3 P per pass of
    P in {1, 2, 4, 8, 16} right-hand sides.  Forward: per block of 128 (i23, s) rows and i1 tile
    (ceil(n1 / 96) tiles of n1t = n1 / tiles rounded up to 16), M = 128, N = 2 n1t, K = 2 x the
    component's rows rounded up to chunks of 32, passes of P in {4, 8, 16}."""
    g = w.grid
    ranks = h.export()[0]                      # (M, q, 3)
    n1, n2n3 = g.shape[0], g.shape[1] * g.shape[2]
    if forward:
        P = 4 if p <= 4 else 8 if p <= 8 else 16
        nsc = -(-p // P)
        blocks = -(-n2n3 // (128 // P)) * nsc
        rows = sum(-(-int(ranks[:, k, 0].sum()) // 32) * 32 for k in range(ranks.shape[1]))
        ntile1 = -(-n1 // 96)
        n1t = -(-(-(-n1 // ntile1)) // 16) * 16
        return 2.0 * 128 * (2 * n1t * ntile1) * (2 * rows) * 3 * blocks
    groups = sum(-(-int(ranks[:, k, 0].sum()) // 128) for k in range(ranks.shape[1]))
    P = 1 << max(0, (min(p, 16) - 1).bit_length())
    nsc = -(-p // P)
    n1p = -(-n1 // 8) * 8                     # i1 tiles of 160 beyond 224 split K, not add to it
    return 2.0 * 128 * (2 * n1p) * (2 * n2n3 * P * nsc) * 3 * groups


def run_zbc(args):
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_06393_gb300 import inputs, zbc

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = inputs.workload(WORKLOAD)
    if args.columns:
        w = inputs.scaled_workload(WORKLOAD, w.grid.shape, m=args.columns)
    g = w.grid
    p = w.p
    h, t_build = build_handle(w, zbc, torch)
    inf = h.info()
    log(f"[bench] handle built in {t_build:.1f}s: M={inf.M} max_rank={inf.max_rank} pool={inf.pool_bytes/2**20:.1f} MiB")
    F1 = algorithmic_flops(h, w, p)
    F = 2.0 * F1

    X = inputs.cn01((w.segments.m, p), seed=0).astype(np.complex64)
    Phi = inputs.cn01((3 * g.nv, p), seed=1).astype(np.complex64)
    Xd, Phid = zbc.to_colmajor(X), zbc.to_colmajor(Phi)
    Yd = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psid = zbc.colmajor(w.segments.m, p, torch.complex64)
    flushbuf = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def flush():
        flushbuf.fill_(1)

    names = {zbc.FP32_SIMT: "fp32_simt", zbc.TF32X3: "tf32x3", zbc.BF16X3: "bf16x3", zbc.TC2: "tc2",
             zbc.TC_MODE1: "tc_mode1"}

    def available(fn, a, b, codes):
        out = [zbc.FP32_SIMT]
        for code in codes:
            try:
                fn(h, a, b, code)
                out.append(code)
            except zbc.ZbcError:
                pass
        return [c for c in out if args.prec in ("auto", names[c])] or [zbc.FP32_SIMT]

    fwd_codes = available(zbc.zbc_matvec, Xd, Yd, (zbc.TF32X3, zbc.BF16X3, zbc.TC2, zbc.TC_MODE1))
    adj_codes = available(zbc.zbc_rmatvec, Phid, Psid, (zbc.TC_MODE1,))
    tens, _ = h.tensors()
    nt = max(3, args.steps // 2)
    # every form's output is kept for the oracle check (rank 0, with the CPU baseline); all of
    # them meet the 1e-5 relative tolerance in the parity tests, so the fastest is timed
    fwd, adj, Ys, Psis = {}, {}, {}, {}
    for code in fwd_codes:
        for _ in range(args.warmup):
            zbc.zbc_matvec(h, Xd, Yd, code)
        torch.cuda.synchronize()
        Ys[names[code]] = zbc.from_colmajor(Yd)
        t = statistics.median(time_steps(lambda: zbc.zbc_matvec(h, Xd, Yd, code), nt, flush, torch, stream))
        fwd[names[code]] = dict(code=code, ms=t)
        log(f"[bench] forward {names[code]}: {t:.3f} ms")
    for code in adj_codes:
        for _ in range(args.warmup):
            zbc.zbc_rmatvec(h, Phid, Psid, code)
        torch.cuda.synchronize()
        Psis[names[code]] = zbc.from_colmajor(Psid)
        t = statistics.median(time_steps(lambda: zbc.zbc_rmatvec(h, Phid, Psid, code), nt, flush, torch, stream))
        adj[names[code]] = dict(code=code, ms=t)
        log(f"[bench] adjoint {names[code]}: {t:.3f} ms")

    # the step runs what the library's autotuner picks (ZBC_AUTO after zbc_tune for this p)
    tune = zbc.zbc_tune(h, p)
    log(f"[bench] zbc_tune: {tune}")
    if args.prec == "auto":
        fv = min((k for k in tune if k.startswith("fwd_")), key=lambda k: tune[k])
        av = min((k for k in tune if k.startswith("adj_")), key=lambda k: tune[k])
        fwd_head = "fp32_simt" if "simt" in fv else ("tc_mode1" if fv == "fwd_mode1" else fv[4:])
        adj_head = "fp32_simt" if "simt" in av else "tc_" + av[4:]
        fcode = acode = zbc.AUTO
        variant = {"forward": fv, "adjoint": av}
    else:
        fwd_head = min(fwd, key=lambda n: fwd[n]["ms"])
        adj_head = min(adj, key=lambda n: adj[n]["ms"])
        fcode, acode = fwd[fwd_head]["code"], adj[adj_head]["code"]
        variant = {"forward": fwd_head, "adjoint": adj_head}
    for _ in range(args.warmup):
        zbc.zbc_matvec(h, Xd, Yd, fcode)
        zbc.zbc_rmatvec(h, Phid, Psid, acode)
    torch.cuda.synchronize()
    Ys["step"], Psis["step"] = zbc.from_colmajor(Yd), zbc.from_colmajor(Psid)
    # each product's main kernel timed alone (the roofline's dominant-kernel figure)
    fwd_ms = statistics.median(time_steps(lambda: zbc.zbc_matvec(h, Xd, Yd, fcode), nt, flush, torch, stream))
    adj_ms = statistics.median(time_steps(lambda: zbc.zbc_rmatvec(h, Phid, Psid, acode), nt, flush, torch, stream))

    def step():
        zbc.zbc_matvec(h, Xd, Yd, fcode)
        zbc.zbc_rmatvec(h, Phid, Psid, acode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clk = ClockSampler(local)
    clk.start()
    l0 = zbc.kernel_launches()
    times = time_steps(step, args.steps, flush, torch, stream)
    launches = zbc.kernel_launches() - l0
    torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    clocks = clk.stop()
    ms = slowest_rank_ms(np.mean(times), ws, "cuda")
    value = whole_job_tflops(F, ms, ws)

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
    Phih = torch.from_numpy(np.ascontiguousarray(Phi.T)).pin_memory()
    Yh = torch.empty(Yd.shape, dtype=Yd.dtype).pin_memory()
    Psih = torch.empty(Psid.shape, dtype=Psid.dtype).pin_memory()

    # the copies run on a second stream where the data flow allows: Phi's upload beside the
    # forward product, Y's download beside the adjoint; the step ends when every copy has
    copy_stream = torch.cuda.Stream()

    def e2e_step():
        main = torch.cuda.current_stream()
        copy_stream.wait_stream(main)            # the previous step is done with Phi and Y
        with torch.cuda.stream(copy_stream):
            Phid.copy_(Phih, non_blocking=True)
        phi_ready = copy_stream.record_event()
        Xd.copy_(Xh, non_blocking=True)
        zbc.zbc_matvec(h, Xd, Yd, fcode)
        copy_stream.wait_stream(main)
        with torch.cuda.stream(copy_stream):
            Yh.copy_(Yd, non_blocking=True)
        main.wait_event(phi_ready)
        zbc.zbc_rmatvec(h, Phid, Psid, acode)
        Psih.copy_(Psid, non_blocking=True)
        main.wait_stream(copy_stream)

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    te = time_steps(e2e_step, max(3, args.steps // 2), flush, torch, stream)
    e2e_ms = slowest_rank_ms(np.mean(te), ws, "cuda")
    h2d = Xh.numel() * 8 + Phih.numel() * 8
    d2h = Yh.numel() * 8 + Psih.numel() * 8

    # roofline of the dominant kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    # the dominant kernel: the slower of the two products' main kernels
    dom_fwd = fwd_ms >= adj_ms
    dom_name, dom_ms = (fwd_head, fwd_ms) if dom_fwd else (adj_head, adj_ms)
    kern = ("matvec" if dom_fwd else "rmatvec") + {"fp32_simt": "_simt_kernel", "tc_mode1": "_mode1_kernel",
                                                   "tc2": "_tc2_kernel"}.get(dom_name, "_tc_kernel")
    if dom_name == "fp32_simt":
        sm_count = torch.cuda.get_device_properties(local).multi_processor_count
        mx = (clocks or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = sm_count * 128 * 2 * mx * 1e6 / 1e12
        roof = {"bound": "alu", "achieved": F1 / (dom_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x {mx:.0f} MHz",
                "kernel": kern, "traffic": None}
    else:
        # real tensor-core products per real MAC of the split: BF16x3 6, TF32x3 3 at half the bf16
        # rate (= 6), fp16 hi/lo (TC_MODE1) 3
        mult = 3.0 if dom_name == "tc_mode1" else 6.0
        bf = peaks.get("bf16_tflops", 1900.0)
        peak = bf / mult
        roof = {"bound": "tensor", "achieved": F1 / (dom_ms * 1e-3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                "peak_source": f"measured bf16 {bf} TFLOP/s / {mult:.0f} real products per split MAC",
                "kernel": kern, "traffic": None}
        if dom_name == "tc_mode1":
            # the mode-1 form's own GEMM (3 fp16 products per real MAC)
            gf = mode1_gemm_flops(h, w, p, forward=dom_fwd)
            roof["gemm"] = {"tflops": gf / (dom_ms * 1e-3) / 1e12, "peak": bf,
                            "frac": gf / (dom_ms * 1e-3) / 1e12 / bf,
                            "counts": ("forward: 2 x 128 (i23, s) rows x 2 n1f x 2 (rank rows) x 3 products per block"
                                       if dom_fwd else
                                       "adjoint: 2 x 128 (column, rank) rows x 2 n1p x 2 (n2 n3 p) x 3 products per group")}
    # DRAM bytes per launch of the dominant kernel on this workload, from a one-pass ncu capture
    # (dram__bytes_read.sum + dram__bytes_write.sum) of this command; only for the full workload
    # and the kernel version it was taken on
    measured_traffic = {("rmatvec_simt_kernel", "adj_simt9"): 3.313e9 + 0.059e9,
                        ("rmatvec_simt_kernel", "adj_simt6"): 3.222e9 + 0.003e9,
                        ("matvec_tc_kernel", "fwd_tf32x3"): 2.9106e9 + 0.3299e9,
                        ("matvec_tc_kernel", "tf32x3"): 2.9106e9 + 0.3299e9,
                        ("matvec_mode1_kernel", "fwd_mode1"): 2.9775e9 + 0.3334e9,
                        ("matvec_mode1_kernel", "tc_mode1"): 2.9775e9 + 0.3334e9,
                        ("rmatvec_mode1_kernel", "adj_mode1"): 3.8657e9 + 0.0406e9,
                        ("rmatvec_mode1_kernel", "tc_mode1"): 3.8657e9 + 0.0406e9}
    dom_variant = variant["forward"] if dom_fwd else variant["adjoint"]
    if not args.columns:
        roof["traffic"] = measured_traffic.get((kern, dom_variant))
    roof["frac"] = roof["achieved"] / roof["peak"]

    cpu = None
    ey, ep = {}, {}
    if rank == 0 and not args.no_cpu_baseline:
        ey, ep = sampled_errors(tens, w, X, Phi, Ys, Psis)
        log(f"[bench] sampled relative errors vs the FP64 oracle: forward {ey} adjoint {ep}")
        rate, used, t_used = oracle_sample_rate(tens, w, X.astype(np.complex128), Phi.astype(np.complex128), F)
        cpu = {"value": rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"FP64 oracle Algorithms 1+2 over {used} of {inf.M} columns ({t_used:.1f}s), "
                         f"scaled linearly to all columns"}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64", "data": "synthetic",
        "config": {"workload": f"precision: 96^3 voxels (2 mm), 8-loop coil, {w.segments.m} segments, 298.2 MHz, "
                               "HOSVD tol 1e-6, complex64 Tucker storage, p=16",
                   "forward": fwd_head, "adjoint": adj_head, "variant": variant, "M": inf.M, "max_rank": inf.max_rank, "l2": "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas x{ws}"},
        "rel_err": {"y": ey.get("step"), "psi": ep.get("step"), "vs": "FP64 oracle, sampled outputs"},
        "tune_ms": tune,
        "paths": {"forward": {n: {"ms": v["ms"], "rel_err": ey.get(n), "tflops": F1 / (v["ms"] * 1e-3) / 1e12}
                              for n, v in fwd.items()},
                  "adjoint": {n: {"ms": v["ms"], "rel_err": ep.get(n), "tflops": F1 / (v["ms"] * 1e-3) / 1e12}
                              for n, v in adj.items()}},
        "e2e": {"value": whole_job_tflops(F, e2e_ms, ws), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
        "gpu_launches": launches,
        "roofline": roof,
        "clocks": clocks,
        "cpu_baseline": cpu,
        "setup_s": t_build,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_compression(args):
    """Compression benchmark of the learned workload (128^3 voxels, 2 mm, 4096 random segments,
    tol 1e-6): truncated HOSVD against the MLP-width randomized Tucker with HOSVD fallback, on the
    same assembled columns.  The MLP is first trained on the HOSVD ranks of other columns of the
    workload.  Prints one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_06393_gb300 import inputs, zbc

    w = inputs.workload("learned")
    g, s = w.grid, w.segments
    ntrain, ntest, batch = 512, args.columns or 512, 128
    perm = np.random.default_rng(7).permutation(s.m)
    train, test = perm[:ntrain], perm[ntrain:ntrain + ntest]
    ds = zbc.DeviceSegments(s)
    feats_all = inputs.rank_features(g, s)

    def assemble(cols):
        cd = torch.from_numpy(np.asarray(cols, dtype=np.int32)).cuda()
        Z = zbc.colmajor(3 * g.nv, len(cols), torch.complex64)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cd, Z)
        return Z

    def ranks_of(h):
        r, _, _ = h.export()
        return r.reshape(-1, 9)

    # 1. HOSVD ranks of the training columns -> MLP targets log(rank)
    rt = []
    for b0 in range(0, ntrain, batch):
        Z = assemble(train[b0:b0 + batch])
        h, _ = zbc.tucker_compress(Z, g, w.tol)
        rt.append(ranks_of(h))
        del h, Z
    T = torch.from_numpy(np.log(np.concatenate(rt).astype(np.float32))).cuda()
    X = torch.from_numpy(feats_all[train]).cuda()
    model = zbc.Mlp(inputs.mlp_init_params(0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = model.train(X, T, 3000, 1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    loss = hist.cpu().numpy()

    # 2. the test columns, both ways
    lmax = 64
    sk = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=11)]
    t_h = t_r = 0.0
    nf = nt = 0
    err_h = err_r = 0.0
    rk_h, rk_r, exact = [], [], 0
    for b0 in range(0, ntest, batch):
        cols = test[b0:b0 + batch]
        Z = assemble(cols)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh, sh = zbc.tucker_compress(Z, g, w.tol)
        torch.cuda.synchronize()
        t_h += time.perf_counter() - t0
        t0 = time.perf_counter()
        widths = model.widths(torch.from_numpy(feats_all[cols]).cuda(), g, oversample=4)
        hr, sr = zbc.tucker_compress_randomized(Z, g, w.tol, widths, sk, lmax)
        torch.cuda.synchronize()
        t_r += time.perf_counter() - t0
        nf += sr.n_fallback
        nt += sr.n_tensors
        err_h, err_r = max(err_h, sh.max_rel_err), max(err_r, sr.max_rel_err)
        a, b = ranks_of(hh), ranks_of(hr)
        rk_h.append(a)
        rk_r.append(b)
        exact += int(np.sum(np.all(a == b, axis=1)))
        del hh, hr, Z
    rk_h, rk_r = np.concatenate(rk_h), np.concatenate(rk_r)
    line = {
        "metric": "Tucker compression time per column, HOSVD vs MLP-width randomized (fallback rate)",
        "value": 1e3 * t_r / ntest, "unit": "ms/column", "higher_is_better": False, "n_gpus": 1,
        "data": "synthetic", "dtype": "c64 input, FP64 factorisation",
        "config": {"workload": "learned: 128^3 voxels (2 mm), 4096 random 5 mm segments, 298.2 MHz, tol 1e-6",
                   "train_columns": ntrain, "test_columns": ntest, "batch": batch, "sketch_lmax": lmax,
                   "oversample": 4, "mlp_steps": 3000, "mlp_lr": 1e-3},
        "hosvd_ms_per_column": 1e3 * t_h / ntest,
        "randomized_ms_per_column": 1e3 * t_r / ntest,
        "speedup": t_h / t_r if t_r > 0 else None,
        "fallback_rate": nf / max(1, nt),
        "max_rel_err": {"hosvd": err_h, "randomized": err_r, "tol": w.tol},
        "mean_rank": {"hosvd": float(rk_h.mean()), "randomized": float(rk_r.mean())},
        "columns_with_equal_ranks": exact / max(1, len(rk_h)),
        "mlp": {"train_s": t_train, "loss_first": float(loss[0]), "loss_last": float(loss[-1])},
    }
    print(json.dumps(line), flush=True)


def cross_cpu_baseline(w, cols, tol, checks):
    """The FP64 oracle's fibre cross (entries evaluated voxel by voxel from the Green's function,
    as cross_tucker_assemble does) on a bounded sample of columns: ms per column."""
    from oracle import cross_tucker as xt
    g, s = w.grid, w.segments
    t0 = time.perf_counter()
    for e in cols:
        for k in range(3):
            src = xt.green_source(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, int(e), k,
                                  mask_radius=g.mask_radius)
            G, Us, _ = xt.cross_tucker(src, g.shape, tol)
            xt.check_error(src, G, Us, g.shape, checks)
    return 1e3 * (time.perf_counter() - t0) / len(cols)


def run_cross(args):
    """Compression from fibres (3D cross-Tucker; end of Sec. II.B.1 and Sec. V) against column
    assembly + truncated HOSVD, on columns of the bench workload (96^3 voxels, 2 mm, 298.2 MHz,
    tol 1e-6): time per column, tensor entries evaluated per tensor against n_v, the check-fibre
    error and the true error of both models against the assembled column (each handle decompressed
    on the GPU as Z~ I with the FP32 forward product).  Prints one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_06393_gb300 import inputs, zbc

    w = inputs.workload("precision")
    g, s = w.grid, w.segments
    tol = 1e-6
    ncols = args.columns or 128
    batch = min(64, ncols)
    cols = (np.arange(ncols) * (s.m // ncols)).astype(np.int32)
    ds = zbc.DeviceSegments(s)
    chk = inputs.cross_check_fibres(g.shape, 24, seed=13)
    nv = g.nv

    def assemble(cb):
        cd = torch.from_numpy(cb).cuda()
        Z = zbc.colmajor(3 * nv, len(cb), torch.complex64)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cd, Z)
        return Z

    def true_err(h, Z, nb):
        X = zbc.to_colmajor(np.eye(nb, dtype=np.complex64))
        Y = zbc.colmajor(3 * nv, nb, torch.complex64)
        zbc.zbc_matvec(h, X, Y, zbc.FP32_SIMT)
        zbc.zbc_product_status(h)
        d = (Y - Z).reshape(nb, 3, nv)
        ref = Z.reshape(nb, 3, nv)
        e = torch.linalg.vector_norm(d, dim=2) / torch.linalg.vector_norm(ref, dim=2)
        return float(e.max())

    # warm-up: one small batch each way (allocations, first launches)
    Z = assemble(cols[:2])
    zbc.tucker_compress(Z, g, tol)
    zbc.cross_tucker_assemble(g, ds, w.freq_hz, cols[:2], tol, checks=chk)
    torch.cuda.synchronize()
    t_h = t_x = 0.0
    eh = ex = echk = 0.0
    entries = 0
    rk_h, rk_x = [], []
    for b0 in range(0, ncols, batch):
        cb = cols[b0:b0 + batch]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Z = assemble(cb)
        hh, _ = zbc.tucker_compress(Z, g, tol)
        torch.cuda.synchronize()
        t_h += time.perf_counter() - t0
        t0 = time.perf_counter()
        hx, _, xs = zbc.cross_tucker_assemble(g, ds, w.freq_hz, cb, tol, checks=chk)
        torch.cuda.synchronize()
        t_x += time.perf_counter() - t0
        entries += xs.entries
        echk = max(echk, xs.max_check_err)
        eh = max(eh, true_err(hh, Z, len(cb)))
        ex = max(ex, true_err(hx, Z, len(cb)))
        rk_h.append(hh.export()[0].reshape(-1, 3))
        rk_x.append(hx.export()[0].reshape(-1, 3))
        del hh, hx, Z
    rk_h, rk_x = np.concatenate(rk_h), np.concatenate(rk_x)
    line = {
        "metric": "Tucker compression time per column: from fibres (cross) vs assembly + HOSVD",
        "value": 1e3 * t_x / ncols, "unit": "ms/column", "higher_is_better": False, "n_gpus": 1,
        "data": "synthetic", "dtype": "f64 factorisation (HOSVD input c64)",
        "config": {"workload": "precision: 96^3 voxels (2 mm), 8 loops x 128 segments, 298.2 MHz, tol 1e-6",
                   "columns": ncols, "batch": batch, "check_fibres": len(chk),
                   "cross": {"sweeps": 2, "s0": 8, "over": 4, "rmax": 64}},
        "hosvd_ms_per_column": 1e3 * t_h / ncols,
        "entries_per_tensor": entries / (3 * ncols),
        "n_v": nv,
        "max_check_err": echk,
        "max_true_err": {"cross": ex, "hosvd": eh, "tol": tol},
        "mean_rank": {"cross": float(rk_x.mean()), "hosvd": float(rk_h.mean())},
        "max_rank_diff": int(np.abs(rk_x - rk_h).max()),
        "column_bytes": {"assembled_c64": 3 * nv * 8, "fibres_f64": int(16 * entries / ncols)},
    }
    if not args.no_cpu_baseline:
        sample = cols[:: max(1, ncols // 4)][:4]
        line["cpu_baseline"] = {"value": cross_cpu_baseline(w, sample, tol, chk), "unit": "ms/column",
                                "cores": os.cpu_count(), "kind": "oracle",
                                "sample": f"{len(sample)} of the {ncols} columns (3 tensors each), same checks"}
    print(json.dumps(line), flush=True)


def run_batching(args):
    """Batching benchmark of the ACA workload (160 x 160 x 128 voxels at 1.5 mm, 16 loops x 256
    segments, ACA tol 1e-6, Tucker 3e-6): for p = 1 .. 128 right-hand sides, the tuned forward and
    adjoint products (ZBC_AUTO after zbc_tune), then the whole mixed batch (one product pair per
    p) eagerly and as one replayed CUDA graph.  Prints one JSON line."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    from paper_2103_06393_gb300 import inputs, zbc

    w = inputs.workload("batching")
    g, s = w.grid, w.segments
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, ast, piv = zbc.aca_compress(g, zbc.DeviceSegments(s), w.freq_hz, w.tol, 400, zbc.ACA_DENSE_U)
    torch.cuda.synchronize()
    t_aca = time.perf_counter() - t0
    inf = h.info()
    ranks, _, _ = h.export()
    r = np.asarray(ranks, dtype=np.float64).reshape(-1, 3)
    n1, n2, n3 = g.shape
    nv = n1 * n2 * n3
    dec = float((n1 * r[:, 0] * r[:, 1] * r[:, 2] + n1 * n2 * r[:, 1] * r[:, 2] + nv * r[:, 2]).sum())
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ps = [1, 2, 4, 8, 16, 32, 64, 128]
    per_p, bufs = {}, []
    for p in ps:
        F = 2 * (8.0 * dec + 8.0 * 3 * nv * inf.M * p + 8.0 * inf.M * inf.m * p)
        X = zbc.to_colmajor(inputs.cn01((inf.m, p), seed=p).astype(np.complex64))
        Phi = zbc.to_colmajor(inputs.cn01((3 * nv, p), seed=100 + p).astype(np.complex64))
        Y = zbc.colmajor(3 * nv, p, torch.complex64)
        Psi = zbc.colmajor(inf.m, p, torch.complex64)
        tune = zbc.zbc_tune(h, p)

        def pair(X=X, Y=Y, Phi=Phi, Psi=Psi):
            zbc.zbc_matvec(h, X, Y, zbc.AUTO)
            zbc.zbc_rmatvec(h, Phi, Psi, zbc.AUTO)

        for _ in range(3):
            pair()
        ms = statistics.median(time_steps(pair, 5, lambda: flush.fill_(1), torch, stream))
        fv = min((k for k in tune if k.startswith("fwd_")), key=lambda k: tune[k])
        av = min((k for k in tune if k.startswith("adj_")), key=lambda k: tune[k])
        per_p[str(p)] = {"ms": ms, "tflops": F / (ms * 1e-3) / 1e12, "forward": fv, "adjoint": av,
                         "fwd_ms": tune[fv], "adj_ms": tune[av]}
        bufs.append(pair)
        log(f"[bench] batching p={p}: {ms:.3f} ms ({per_p[str(p)]['tflops']:.1f} TFLOP/s, {fv}, {av})")

    def mixed():
        for f in bufs:
            f()

    for _ in range(2):
        mixed()
    torch.cuda.synchronize()
    eager = statistics.median(time_steps(mixed, 3, lambda: flush.fill_(1), torch, stream))
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        mixed()
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        mixed()
    graph.replay()
    torch.cuda.synchronize()
    replay = statistics.median(time_steps(graph.replay, 3, lambda: flush.fill_(1), torch, stream))
    zbc.zbc_product_status(h)
    Ftot = sum(v["tflops"] * v["ms"] * 1e-3 * 1e12 for v in per_p.values())
    line = {
        "metric": "mixed-batch Z x and Z^H v throughput (p = 1..128), ACA storage, graph-captured",
        "value": Ftot / (replay * 1e-3) / 1e12, "unit": "TFLOP/s", "higher_is_better": True, "n_gpus": 1,
        "data": "synthetic", "dtype": "c64",
        "config": {"workload": "batching: 160x160x128 voxels (1.5 mm, masked beyond r = 0.157 m), 16 loops x 256 "
                               "segments, ACA tol 1e-6 (dense U, Tucker 3e-6)", "rhs": ps,
                   "l2": "flushed (256 MiB write) between steps"},
        "aca": {"rank": int(ast.rank), "converged": int(ast.converged), "seconds": t_aca, "M": inf.M,
                "max_tucker_rank": inf.max_rank},
        "per_p": per_p,
        "mixed_batch_ms": {"eager": eager, "graph": replay},
        "gpu_launches_per_batch": None,
    }
    l0 = zbc.kernel_launches()
    mixed()
    torch.cuda.synchronize()
    line["gpu_launches_per_batch"] = zbc.kernel_launches() - l0
    print(json.dumps(line), flush=True)


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import greens, products, tucker
    from paper_2103_06393_gb300 import inputs

    w = inputs.workload(WORKLOAD)
    g, s = w.grid, w.segments
    p = w.p
    # the reference arm runs the FP64 oracle on a bounded sample of columns per step
    ncols = 4
    X = inputs.cn01((s.m, p), seed=0)
    Phi = inputs.cn01((3 * g.nv, p), seed=1)
    Z = greens.assemble_columns(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, np.arange(ncols))
    tens = tucker.compress_columns(Z, g.shape, 3, w.tol)
    ranks = np.array([[U.shape[1] for U in t[1]] for tj in tens for t in tj])
    F_sample = 2.0 * products.flops(ranks, g.shape, 3, ncols, p)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        products.matvec(tens, g.shape, X[:ncols])
        products.rmatvec(tens, g.shape, Phi)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    dt = float(np.mean(times))
    value = F_sample / dt / 1e12
    ms = 1e3 * dt * s.m / ncols   # the full step, extrapolated linearly in the columns
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "precision: 96^3 voxels (2 mm), 8-loop coil, 1024 segments, 298.2 MHz, "
                               "HOSVD tol 1e-6, complex128 Tucker storage, p=16", "path": "FP64 CPU oracle"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": f"{ncols} of {s.m} columns per step, scaled linearly"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zbc", choices=["zbc", "reference"])
    ap.add_argument("--prec", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cross", action="store_true",
                    help="compression from fibres (cross-Tucker) vs assembly + HOSVD instead of the products")
    ap.add_argument("--compression", action="store_true",
                    help="compression benchmark (HOSVD vs learned randomized Tucker) instead of the products")
    ap.add_argument("--batching", action="store_true",
                    help="mixed right-hand-side batches on the ACA workload (tuned forms, CUDA graph)")
    ap.add_argument("--columns", type=int, default=0,
                    help="keep only the first N segments (smaller case for profiler captures)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cross:
        run_cross(args)
        return
    if args.compression:
        run_compression(args)
    elif args.batching:
        run_batching(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_zbc(args)


if __name__ == "__main__":
    main()
