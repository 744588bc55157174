"""Benchmark of the hot path: Y = Z X (Algorithm 1) and Psi = Z^H Phi (Algorithm 2) on the
compressed coupling matrix.

Default workload ("large"): 320 x 320 x 256 voxels at 1 mm, a 32-loop cylindrical coil with 2048
segments at 298.2 MHz, each column stored in Tucker form at tol 1e-5 by the certified fixed-width
randomized Tucker (HOSVD fallback; complex64 storage; Algorithm 3's ACA does not compress this
coil's coupling matrix at that tolerance), 32 right-hand sides.  One step = one Z X plus one
Z^H Phi.  Metric = algorithmic TFLOP/s of the step (Table III count, complex MAC = 8 flops, summed
over both products), with the step time and the relative error against the FP64 oracle on sampled
outputs.  The line also carries, under "extra", the 96^3 / 1024-segment / 16-RHS workload
("precision"), the compression comparison of the 128^3 workload ("learned": HOSVD against the
randomized Tucker with learned and with fixed widths) and the mixed right-hand-side batches of the
160 x 160 x 128 workload ("batching"), each started only inside --extras-budget seconds.
Prints ONE JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl zbc|reference]
                  [--workload large|precision] [--no-extras] [--prec auto|...]
                  [--columns N] [--n3 N] [--extras-budget S]

Multi-GPU: replicas only (each rank runs the whole workload; no collective on the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

T_START = time.time()
ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Z·x and Z^H·v time (s) & TFLOP/s, batched TC vs plain FP32, rel err <= 1e-5"
UNIT = "TFLOP/s"
CLOCK_QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
# column-wise randomized Tucker of the large grids: width, sketch columns, sketch seed
TK_WIDTH, TK_LMAX, SKETCH_SEED = 32, 32, 31


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


def table3_flops(ranks, shape, q, M, p, m_aca=0):
    """Real flops of one product by the complexity count of Table III (complex MAC = 8 flops):
    per stored tensor the mode products of the decompression in the order x1, x2, x3
    (n1 r1 r2 r3 + n1 n2 r2 r3 + n_v r3 complex MACs), the contraction with the p right-hand
    sides (q n_v M p MACs) and, for ACA storage (m_aca = m columns of Z), the product with V
    (r_c m p MACs).  ranks: (r1, r2, r3) per stored tensor, any array shape ending in 3."""
    n1, n2, n3 = shape
    nv = n1 * n2 * n3
    r = np.asarray(ranks, dtype=np.float64).reshape(-1, 3)
    r1, r2, r3 = r[:, 0], r[:, 1], r[:, 2]
    dec = float((n1 * r1 * r2 * r3 + n1 * n2 * r2 * r3 + nv * r3).sum())
    return 8.0 * dec + 8.0 * q * nv * M * p + 8.0 * M * m_aca * p


def algorithmic_flops(h, shape, p):
    """table3_flops of one product on handle h (ACA storage adds its r_c m p term)."""
    ranks, _, _ = h.export()
    inf = h.info()
    return table3_flops(ranks, shape, inf.q, inf.M, p, inf.m if inf.has_v else 0)


def algorithmic_bytes(inf, shape, p):
    """Bytes one product must move at least: the compressed storage (cores, factors, V) read
    once, X (or Psi) and Y (or Phi), complex64."""
    n1, n2, n3 = shape
    return float(inf.pool_bytes + inf.v_bytes + 8 * inf.m * p + 8 * inf.q * n1 * n2 * n3 * p)


def rel_errors(got, ref):
    """Reading C11: per right-hand side (column) ||got - ref||_2 / ||ref||_2; returns
    {"max": the largest over right-hand sides (the 1e-5 criterion), "fro": the Frobenius value}."""
    got, ref = np.asarray(got), np.asarray(ref)
    per = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    return {"max": float(per.max()), "fro": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}


# ---------------------------------------------------------------------------------------------
# clocks, timing, peaks, recorded traffic
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    def __init__(self, gpu_index=0):
        self.proc = None
        self.path = None
        self.idx = gpu_index

    def start(self):
        try:
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


def measured_peaks(torch):
    """TF32 tensor-core and FP32 CUDA-core rates of this GPU, measured with torch.matmul (8192^2
    operands, best of 6): the denominators of the TF32x3 and FP32 SIMT forms."""
    out = {}
    a = torch.randn(8192, 8192, device="cuda")
    b = torch.randn(8192, 8192, device="cuda")
    old = torch.backends.cuda.matmul.allow_tf32
    for name, tf32 in (("tf32_tflops", True), ("fp32_tflops", False)):
        torch.backends.cuda.matmul.allow_tf32 = tf32
        best = float("inf")
        for _ in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            torch.matmul(a, b)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = 2.0 * 8192 ** 3 / (best * 1e-3) / 1e12
    torch.backends.cuda.matmul.allow_tf32 = old
    del a, b
    return out


KERNEL_SOURCES = {"matvec_mode1_kernel": "products_mode1_fwd.cu", "rmatvec_mode1_kernel": "products_mode1.cu",
                  "matvec_simt_kernel": "products_simt.cu", "rmatvec_simt_kernel": "products_simt.cu",
                  "matvec_tc_kernel": "products_tc.cu", "matvec_tc2_kernel": "products_tc2.cu",
                  "matvec_dc_kernel": "products_dc.cu"}


def source_sha16(kernel):
    """Hash of the source file that defines a product kernel (the traffic record's validity key)."""
    f = KERNEL_SOURCES.get(kernel)
    path = os.path.join(ROOT, "paper_2103_06393_gb300", "csrc", f) if f else None
    if not path or not os.path.exists(path):
        return None
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def recorded_traffic(kernel, workload):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of `kernel` on
    `workload`, from profiles/traffic.txt, only while that record's source hash matches the
    kernel's current source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    sha = source_sha16(kernel)
    if not sha or not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) >= 4 and not line.startswith("#") and f[0] == kernel and f[1] == workload and f[2] == sha:
            return float(f[3])
    return None


# ---------------------------------------------------------------------------------------------
# workload construction on the GPU (through the C ABI)
# ---------------------------------------------------------------------------------------------

def build_precision(w, zbc, torch, batch_cols=256):
    """Column assembly + HOSVD of every column (Sec. III.A)."""
    g, s = w.grid, w.segments
    ds = zbc.DeviceSegments(s)
    h = None
    t0 = time.time()
    for c0 in range(0, s.m, batch_cols):
        cols = torch.arange(c0, min(s.m, c0 + batch_cols), dtype=torch.int32, device="cuda")
        Z = zbc.colmajor(3 * g.nv, cols.numel(), torch.complex128)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cols, Z)
        h, _ = zbc.tucker_compress(Z, g, w.tol, append_to=h)
        del Z
    torch.cuda.synchronize()
    return h, time.time() - t0, {"method": f"assembly + HOSVD at tol {w.tol:g}"}


def build_randomized(w, zbc, torch, inputs, batch_bytes=10 << 30):
    """Column assembly (complex64) + the certified fixed-width randomized Tucker of every column
    (HOSVD fallback per tensor), in batches of about batch_bytes of assembled columns.  (Algorithm
    3 at these grids' ACA tolerances does not compress their coils' coupling matrices: its stopping
    term stays near 5e-3 after ~200 iterations, the residual columns as large as the columns.)"""
    g, s = w.grid, w.segments
    ds = zbc.DeviceSegments(s)
    sk = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, TK_LMAX, seed=SKETCH_SEED)]
    model = zbc.rank_model(sk, TK_LMAX, fixed_width=TK_WIDTH)
    batch = max(1, min(s.m, batch_bytes // (3 * g.nv * 8)))
    h, fb, err = None, 0, 0.0
    torch.cuda.synchronize()
    t0 = time.time()
    for c0 in range(0, s.m, batch):
        cols = torch.arange(c0, min(s.m, c0 + batch), dtype=torch.int32, device="cuda")
        Z = zbc.colmajor(3 * g.nv, cols.numel(), torch.complex64)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cols, Z)
        h, st = zbc.tucker_compress(Z, g, w.tol, method=zbc.RANDOMIZED_FIXED, model=model, append_to=h)
        fb += st.n_fallback
        err = max(err, st.max_rel_err)
        del Z
    torch.cuda.synchronize()
    return h, time.time() - t0, {"method": f"assembly (complex64) + randomized Tucker of width {TK_WIDTH} at tol "
                                           f"{w.tol:g}, HOSVD fallback", "columns": s.m, "batch": batch,
                                 "fallback_tensors": fb, "max_rel_err": err}


# ---------------------------------------------------------------------------------------------
# oracle legs (rank 0): sampled parity and the CPU baseline
# ---------------------------------------------------------------------------------------------

def _psi_part(args):
    """Worker of the spawn pool: the oracle's Algorithm 2 on a chunk of stored columns, for the
    right-hand sides held in the .npy file `path` (memory-mapped)."""
    tens, shape, path = args
    from oracle import products
    Phi = np.load(path, mmap_mode="r")
    return products.rmatvec(tens, shape, np.asarray(Phi, dtype=np.complex128))


def oracle_psi_columns(tens, shape, Phi_s, procs):
    """Psi' = U^H Phi_s over every stored column with the oracle, the columns spread over `procs`
    processes started with spawn."""
    import multiprocessing as mp
    fd, path = tempfile.mkstemp(suffix=".npy")
    os.close(fd)
    try:
        np.save(path, np.ascontiguousarray(Phi_s))
        procs = max(1, min(procs, len(tens)))
        chunks = [tens[i::procs] for i in range(procs)]
        with mp.get_context("spawn").Pool(procs) as pool:
            parts = pool.map(_psi_part, [(c, shape, path) for c in chunks if c])
    finally:
        os.unlink(path)
    out = np.zeros((len(tens), Phi_s.shape[1]), dtype=np.complex128)
    for i, part in enumerate(parts):
        out[i::procs] = part
    return out


def sampled_errors(tens, V, shape, X, Phi, Ys, Psis, rows, psi_cols, psi_rhs, procs):
    """Relative errors (per right-hand side ||got - ref|| / ||ref||, max and Frobenius) of each path's sampled Y rows (Ys: name -> rows x p) and of
    the sampled entries of Psi (Psis: name -> m x p) against the FP64 oracle on the handle's own
    tensors: Y rows by element-wise Tucker evaluation (matvec_rows on X' = V^H X for ACA storage),
    the columns psi_rhs of Psi by the oracle's Algorithm 2 over every stored column (then V Psi')."""
    from oracle import products
    X = X.astype(np.complex128)
    Xp = X if V is None else V.astype(np.complex128).conj().T @ X
    Yo = products.matvec_rows(tens, shape, Xp, rows)
    if V is None:      # Psi[j, :] needs column j's tensors only
        Po = oracle_psi_columns([tens[j] for j in psi_cols], shape, Phi[:, psi_rhs], procs)
    else:              # Psi = V Psi' needs every stored column
        Po = (V.astype(np.complex128) @ oracle_psi_columns(tens, shape, Phi[:, psi_rhs], procs))[psi_cols]
    ey = {n: rel_errors(Y, Yo) for n, Y in Ys.items()}
    ep = {n: rel_errors(P[np.ix_(psi_cols, psi_rhs)], Po) for n, P in Psis.items()}
    return ey, ep


def oracle_baseline(tens, V, shape, X, Phi, slab_planes, budget_s=20.0):
    """The oracle's Algorithms 1 and 2 (plain FP64 NumPy, one process) timed on a bounded sample:
    the first K stored columns on the first `slab_planes` i3 planes, K doubled until about a third
    of budget_s; scaled linearly to all columns and planes.  Returns (seconds of the full step,
    K, sample seconds)."""
    from oracle import products
    n1, n2, n3 = shape
    sub = (n1, n2, slab_planes)
    nvs, nv = n1 * n2 * slab_planes, n1 * n2 * n3
    rows = np.concatenate([k * nv + np.arange(nvs) for k in range(3)])
    Phis = Phi[rows].astype(np.complex128)
    M = len(tens)
    X = X.astype(np.complex128)
    Xp = X if V is None else V.astype(np.complex128).conj().T @ X
    k = 1
    while True:
        part = [[(G, [Us[0], Us[1], Us[2][:slab_planes]]) for (G, Us, *_r) in tj] for tj in tens[:k]]
        t0 = time.perf_counter()
        products.matvec(part, sub, Xp[:k])
        products.rmatvec(part, sub, Phis)
        dt = time.perf_counter() - t0
        if dt > budget_s / 3 or k >= M:
            break
        k = min(M, 2 * k)
    return dt * (M / k) * (n3 / slab_planes), k, dt


# ---------------------------------------------------------------------------------------------
# the products on one workload
# ---------------------------------------------------------------------------------------------

NAMES = {0: "fp32_simt", 1: "tf32x3", 2: "bf16x3", 4: "tc2", 5: "tc_mode1", 6: "tc_dc"}
TUNE_HEAD = {"fwd_simt6": "fp32_simt", "fwd_simt9": "fp32_simt", "fwd_tf32x3": "tf32x3", "fwd_bf16x3": "bf16x3",
             "fwd_tc2": "tc2", "fwd_mode1": "tc_mode1", "fwd_dc": "tc_dc", "adj_simt6": "fp32_simt",
             "adj_simt9": "fp32_simt", "adj_mode1": "tc_mode1"}


def measure_products(h, w, zbc, torch, X, Phi, args, ws, local, nrows, npsi):
    """Every product form timed alone, the tuned step (ZBC_AUTO after zbc_tune), the step end to
    end through host buffers and the outputs kept for the oracle checks."""
    g = w.grid
    p = X.shape[1]
    inf = h.info()
    F1 = algorithmic_flops(h, g.shape, p)
    F = 2.0 * F1
    Xd, Phid = zbc.to_colmajor(X), zbc.to_colmajor(Phi)
    Yd = zbc.colmajor(3 * g.nv, p, torch.complex64)
    Psid = zbc.colmajor(inf.m, p, torch.complex64)
    flushbuf = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    rng = np.random.default_rng(2)
    rows = np.sort(rng.choice(3 * g.nv, size=min(nrows, 3 * g.nv), replace=False))
    rows_d = torch.from_numpy(rows).cuda()
    psi_rhs = np.sort(rng.choice(p, size=min(p, 4), replace=False))
    psi_cols = np.sort(rng.choice(inf.m, size=min(inf.m, max(1, npsi // len(psi_rhs))), replace=False))

    def flush():
        flushbuf.fill_(1)

    fwd_codes = [zbc.FP32_SIMT]
    for code in (zbc.TF32X3, zbc.BF16X3, zbc.TC2, zbc.TC_MODE1, zbc.TC_DC):
        try:
            zbc.zbc_matvec(h, Xd, Yd, code)
            fwd_codes.append(code)
        except zbc.ZbcError:
            pass
    adj_codes = [zbc.FP32_SIMT]
    try:
        zbc.zbc_rmatvec(h, Phid, Psid, zbc.TC_MODE1)
        adj_codes.append(zbc.TC_MODE1)
    except zbc.ZbcError:
        pass
    fwd_codes = [c for c in fwd_codes if args.prec in ("auto", NAMES[c])] or [zbc.FP32_SIMT]
    adj_codes = [c for c in adj_codes if args.prec in ("auto", NAMES[c])] or [zbc.FP32_SIMT]
    nt = max(3, args.steps // 2)
    fwd, adj, Ys, Psis = {}, {}, {}, {}

    def time_form(call):
        """Median time of one form: args.warmup untimed calls and nt timed ones; a form whose first
        call takes more than half a second gets one untimed and two timed calls (the other forms'
        figures, not the step's)."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        call()
        torch.cuda.synchronize()
        slow = time.perf_counter() - t0 > 0.5
        for _ in range(0 if slow else args.warmup - 1):
            call()
        return statistics.median(time_steps(call, 2 if slow else nt, flush, torch, stream))

    for code in fwd_codes:
        t = time_form(lambda: zbc.zbc_matvec(h, Xd, Yd, code))
        zbc.zbc_product_status(h)
        Ys[NAMES[code]] = zbc.from_colmajor_rows(Yd, rows_d)
        fwd[NAMES[code]] = t
        log(f"[bench] {w.name} forward {NAMES[code]}: {t:.3f} ms")
    for code in adj_codes:
        t = time_form(lambda: zbc.zbc_rmatvec(h, Phid, Psid, code))
        zbc.zbc_product_status(h)
        Psis[NAMES[code]] = zbc.from_colmajor(Psid)
        adj[NAMES[code]] = t
        log(f"[bench] {w.name} adjoint {NAMES[code]}: {t:.3f} ms")

    # the step runs what the library's autotuner picks (ZBC_AUTO after zbc_tune for this p)
    tune = zbc.zbc_tune(h, p)
    log(f"[bench] {w.name} zbc_tune: {tune}")
    fv = min((k for k in tune if k.startswith("fwd_")), key=lambda k: tune[k])
    av = min((k for k in tune if k.startswith("adj_")), key=lambda k: tune[k])
    if args.prec == "auto":
        fwd_head, adj_head, fcode, acode = TUNE_HEAD[fv], TUNE_HEAD[av], zbc.AUTO, zbc.AUTO
    else:
        fwd_head, adj_head = min(fwd, key=fwd.get), min(adj, key=adj.get)
        inv = {v: k for k, v in NAMES.items()}
        fcode, acode, fv, av = inv[fwd_head], inv[adj_head], fwd_head, adj_head
    for _ in range(args.warmup):
        zbc.zbc_matvec(h, Xd, Yd, fcode)
        zbc.zbc_rmatvec(h, Phid, Psid, acode)
    zbc.zbc_product_status(h)
    Ys["step"], Psis["step"] = zbc.from_colmajor_rows(Yd, rows_d), zbc.from_colmajor(Psid)
    # each product timed alone (its main kernel dominates the call: the roofline's figure)
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
    zbc.zbc_product_status(h)
    ms = slowest_rank_ms(np.mean(times), ws, "cuda")
    out = {"F1": F1, "ms": ms, "value": whole_job_tflops(F, ms, ws), "launches": launches, "clocks": clocks,
           "fwd_head": fwd_head, "adj_head": adj_head, "variant": {"forward": fv, "adjoint": av}, "tune": tune,
           "fwd_ms": fwd_ms, "adj_ms": adj_ms, "fwd": fwd, "adj": adj, "p": p}

    # end to end through the public API with host buffers (pinned), copies inside the timed region
    if not args.no_e2e:
        Xh = torch.from_numpy(np.ascontiguousarray(X.T)).pin_memory()
        Phih = torch.from_numpy(np.ascontiguousarray(Phi.T)).pin_memory()
        Yh = torch.empty(Yd.shape, dtype=Yd.dtype).pin_memory()
        Psih = torch.empty(Psid.shape, dtype=Psid.dtype).pin_memory()
        # the copies run on a second stream where the data flow allows: Phi's upload beside the
        # forward product, Y's download beside the adjoint; the step ends when every copy has.
        # X goes up first: host-to-device copies share one copy engine in issue order, so an X
        # upload issued after Phi's would hold the forward back for the whole of Phi's upload.
        copy_stream = torch.cuda.Stream()

        def e2e_step():
            main = torch.cuda.current_stream()
            Xd.copy_(Xh, non_blocking=True)
            copy_stream.wait_stream(main)            # the previous step is done with Phi and Y
            with torch.cuda.stream(copy_stream):
                Phid.copy_(Phih, non_blocking=True)
            phi_ready = copy_stream.record_event()
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
        out["e2e"] = {"value": whole_job_tflops(F, e2e_ms, ws), "unit": UNIT,
                      "h2d_bytes_per_step": Xh.numel() * 8 + Phih.numel() * 8,
                      "d2h_bytes_per_step": Yh.numel() * 8 + Psih.numel() * 8, "ms_per_step": e2e_ms}
        del Xh, Phih, Yh, Psih
    del Xd, Phid, Yd, Psid, flushbuf
    torch.cuda.empty_cache()
    out["Ys"], out["Psis"] = Ys, Psis
    out["samples"] = (rows, psi_cols, psi_rhs)
    return out


def roofline(inf, w, res, peaks, measured):
    """Roofline of the dominant kernel: the slower of the two products' main kernels.  achieved =
    Table III flops of one product / that product's CUDA-event time; peak = the measured rate of
    the unit the form computes on."""
    F1 = res["F1"]
    dom_fwd = res["fwd_ms"] >= res["adj_ms"]
    name = res["fwd_head"] if dom_fwd else res["adj_head"]
    dom_ms = res["fwd_ms"] if dom_fwd else res["adj_ms"]
    kern = ("matvec" if dom_fwd else "rmatvec") + {"fp32_simt": "_simt_kernel", "tc_mode1": "_mode1_kernel",
                                                   "tc2": "_tc2_kernel", "tc_dc": "_dc_kernel"}.get(name, "_tc_kernel")
    achieved = F1 / (dom_ms * 1e-3) / 1e12
    bf = peaks.get("bf16_tflops", 1905.6)
    if name == "fp32_simt":
        peak, bound = measured["fp32_tflops"], "alu"
        src = "measured FP32 CUDA-core rate (torch.matmul FP32 in this run)"
    elif name == "tf32x3":
        peak, bound = measured["tf32_tflops"] / 3.0, "tensor"
        src = "measured TF32 rate (torch.matmul in this run) / 3 split products per real MAC"
    elif name in ("tc_mode1", "tc2", "tc_dc"):
        peak, bound = bf / 3.0, "tensor"
        src = f"measured bf16 {bf} TFLOP/s (MEASURED_PEAKS.json) / 3 fp16 split products per real MAC"
    else:
        peak, bound = bf / 6.0, "tensor"
        src = f"measured bf16 {bf} TFLOP/s (MEASURED_PEAKS.json) / 6 bf16 split products per real MAC"
    b1 = algorithmic_bytes(inf, w.grid.shape, res["p"])
    return {"bound": bound, "achieved": achieved, "peak": peak, "unit": UNIT, "frac": achieved / peak,
            "peak_source": src, "kernel": kern, "kernel_ms": dom_ms, "algorithmic_bytes": b1,
            "algorithmic_gbs": b1 / (dom_ms * 1e-3) / 1e9, "traffic": recorded_traffic(kern, w.name)}


def describe(w, inf):
    g = w.grid
    if w.aca:
        return (f"{w.name}: {g.n1}x{g.n2}x{g.n3} voxels ({g.h * 1e3:g} mm), {w.segments.m} segments, 298.2 MHz, "
                f"column-wise Tucker at tol {w.tol:g} (randomized, width {TK_WIDTH}, HOSVD fallback; ACA at this "
                f"tolerance does not compress the coil's coupling matrix), complex64 Tucker storage, p={w.p}")
    return (f"{w.name}: {g.n1}x{g.n2}x{g.n3} voxels ({g.h * 1e3:g} mm), {w.segments.m} segments, 298.2 MHz, "
            f"HOSVD tol {w.tol:g}, complex64 Tucker storage, p={w.p}")


def run_workload(name, args, zbc, torch, inputs, ws, rank, local, peaks, measured, baseline=True):
    """Build the named workload's handle, measure its products and (rank 0) check them against the
    oracle and time the oracle.  Returns the JSON fields of this workload."""
    w = inputs.workload(name)
    if args.columns or args.n3:
        n1, n2, n3 = w.grid.shape
        w = inputs.scaled_workload(name, (n1, n2, args.n3 or n3), m=args.columns or None)
    g = w.grid
    if w.aca:
        h, t_build, build = build_randomized(w, zbc, torch, inputs)
    else:
        h, t_build, build = build_precision(w, zbc, torch)
    inf = h.info()
    log(f"[bench] {name}: handle built in {t_build:.1f}s: M={inf.M} max_rank={inf.max_rank} "
        f"pool={inf.pool_bytes / 2 ** 20:.1f} MiB {build}")
    X = inputs.cn01_columns_c64(w.segments.m, w.p, seed=0)
    Phi = inputs.cn01_columns_c64(3 * g.nv, w.p, seed=1)
    big = 3 * g.nv * w.p * 8 > (4 << 30)
    res = measure_products(h, w, zbc, torch, X, Phi, args, ws, local, nrows=4096 if big else 512,
                           npsi=64 if big else 48)
    tb, vb, fb = h.memory_bytes()
    out = {
        "config": {"workload": describe(w, inf), "forward": res["fwd_head"], "adjoint": res["adj_head"],
                   "variant": res["variant"], "M": inf.M, "max_rank": inf.max_rank, "p": w.p,
                   "l2": ("inputs larger than L2, and " if big else "") + "flushed (256 MiB write) between steps",
                   "parallelism": f"replicas x{ws}"},
        "value": res["value"], "ms_per_step": res["ms"], "gpu_launches": res["launches"], "clocks": res["clocks"],
        "tune_ms": res["tune"], "roofline": roofline(inf, w, res, peaks, measured), "setup_s": t_build,
        "build": build,
        "memory": {"table2_tucker_bytes": tb, "table2_v_bytes": vb, "dense_c64_bytes": fb,
                   "device_bytes": h.device_bytes()},
        "paths": {"forward": {n: {"ms": t, "tflops": res["F1"] / (t * 1e-3) / 1e12} for n, t in res["fwd"].items()},
                  "adjoint": {n: {"ms": t, "tflops": res["F1"] / (t * 1e-3) / 1e12} for n, t in res["adj"].items()}},
    }
    if "e2e" in res:
        out["e2e"] = res["e2e"]
    if rank == 0 and not args.no_cpu_baseline:
        tens, V = h.tensors()
        rows, psi_cols, psi_rhs = res["samples"]
        t0 = time.time()
        ey, ep = sampled_errors(tens, V, g.shape, X, Phi, res["Ys"], res["Psis"], rows, psi_cols, psi_rhs,
                                max(1, min(16, os.cpu_count() or 1)))
        log(f"[bench] {name}: oracle checks in {time.time() - t0:.1f}s: forward {ey} adjoint {ep}")
        for d, e in (("forward", ey), ("adjoint", ep)):
            for n in out["paths"][d]:
                out["paths"][d][n]["rel_err"] = e.get(n)
        out["rel_err"] = {"y": ey.get("step"), "psi": ep.get("step"),
                          "vs": f"FP64 oracle on the handle's tensors: {len(rows)} sampled rows of Y and "
                                f"{len(psi_cols) * len(psi_rhs)} sampled entries of Psi; max = largest per-RHS "
                                "relative L2 error (the 1e-5 criterion), fro = Frobenius"}
        if baseline:
            slab = max(1, g.n3 // 16)
            t_full, k, t_s = oracle_baseline(tens, V, g.shape, X, Phi, slab)
            out["cpu_baseline"] = {"value": 2.0 * res["F1"] / t_full / 1e12, "unit": UNIT, "cores": 1,
                                   "kind": "oracle", "extrapolated": True, "sample_s": t_s,
                                   "sample": f"FP64 oracle Algorithms 1+2 (one process) on {k} of {inf.M} stored "
                                             f"columns over {slab} of {g.n3} i3 planes ({t_s:.1f}s), scaled "
                                             "linearly to all columns and planes"}
    del h
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------------
# the bench line
# ---------------------------------------------------------------------------------------------

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
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    measured = measured_peaks(torch)
    log(f"[bench] measured peaks: {measured}")
    head = run_workload(args.workload, args, zbc, torch, inputs, ws, rank, local, peaks, measured)
    line = {
        "metric": METRIC, "value": head.pop("value"), "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head.pop("ms_per_step"), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64", "data": "synthetic",
    }
    line.update(head)
    line["peaks_measured"] = dict(measured, source="torch.matmul 8192^3 in this run, best of 6")
    if not args.no_extras and ws == 1 and not args.columns and not args.n3:
        # the other workloads ride along as sub-objects, each started only while the run is inside
        # its time budget (a skipped one says so)
        extra = {}
        jobs = []
        if args.workload != "precision":
            jobs.append(("precision", lambda: dict(run_workload("precision", args, zbc, torch, inputs, ws, rank, local,
                                                                peaks, measured, baseline=False), unit=UNIT)))
        jobs += [("learned", lambda: compression(zbc, torch, inputs)),
                 ("batching", lambda: batching(zbc, torch, inputs))]
        for name, job in jobs:
            used = time.time() - T_START
            if used > args.extras_budget:
                extra[name] = {"skipped": f"time budget: {used:.0f} s used of {args.extras_budget:.0f} s "
                                          "when this workload was due (--extras-budget)"}
                continue
            t0 = time.time()
            try:
                extra[name] = job()
            except Exception as ex:  # a failed ride-along is reported, the headline line stands
                log(f"[bench] {name} failed: {ex!r}")
                extra[name] = {"error": repr(ex)}
                torch.cuda.empty_cache()
            extra[name]["wall_s"] = time.time() - t0
        line["extra"] = extra
    line["wall_s"] = time.time() - T_START
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------------------------------------
# batching: mixed right-hand-side counts on the ACA workload (160 x 160 x 128)
# ---------------------------------------------------------------------------------------------

def batching(zbc, torch, inputs):
    """Batching workload (160 x 160 x 128 voxels at 1.5 mm, 16 loops x 256 segments, column-wise
    Tucker at tol 1e-6 by the fixed-width randomized Tucker): for p = 1 .. 128 right-hand sides the
    tuned forward and adjoint products (ZBC_AUTO after zbc_tune), then the whole mixed batch (one
    product pair per p) eagerly and as one replayed CUDA graph."""
    w = inputs.workload("batching")
    g = w.grid
    h, t_aca, build = build_randomized(w, zbc, torch, inputs)
    inf = h.info()
    log(f"[bench] batching: handle in {t_aca:.1f}s {build}")
    nv = g.nv
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    ps = [1, 2, 4, 8, 16, 32, 64, 128]
    per_p, bufs = {}, []
    ranks = h.export()[0]
    for p in ps:
        F = 2 * table3_flops(ranks, g.shape, 3, inf.M, p, inf.m if inf.has_v else 0)
        X = zbc.to_colmajor(inputs.cn01_columns_c64(inf.m, p, seed=p))
        Phi = zbc.to_colmajor(inputs.cn01_columns_c64(3 * nv, p, seed=100 + p))
        Y = zbc.colmajor(3 * nv, p, torch.complex64)
        Psi = zbc.colmajor(inf.m, p, torch.complex64)
        tune = zbc.zbc_tune(h, p)

        def pair(X=X, Y=Y, Phi=Phi, Psi=Psi):
            zbc.zbc_matvec(h, X, Y, zbc.AUTO)
            zbc.zbc_rmatvec(h, Phi, Psi, zbc.AUTO)

        pair()
        ms = statistics.median(time_steps(pair, 3, lambda: flush.fill_(1), torch, stream))
        fv = min((k for k in tune if k.startswith("fwd_")), key=lambda k: tune[k])
        av = min((k for k in tune if k.startswith("adj_")), key=lambda k: tune[k])
        per_p[str(p)] = {"ms": ms, "tflops": F / (ms * 1e-3) / 1e12, "forward": fv, "adjoint": av,
                         "fwd_ms": tune[fv], "adj_ms": tune[av]}
        bufs.append(pair)
        log(f"[bench] batching p={p}: {ms:.3f} ms ({per_p[str(p)]['tflops']:.1f} TFLOP/s, {fv}, {av})")

    def mixed():
        for f in bufs:
            f()

    mixed()
    torch.cuda.synchronize()
    eager = statistics.median(time_steps(mixed, 2, lambda: flush.fill_(1), torch, stream))
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
    replay = statistics.median(time_steps(graph.replay, 2, lambda: flush.fill_(1), torch, stream))
    zbc.zbc_product_status(h)
    l0 = zbc.kernel_launches()
    mixed()
    torch.cuda.synchronize()
    launches = zbc.kernel_launches() - l0
    Ftot = sum(v["tflops"] * v["ms"] * 1e-3 * 1e12 for v in per_p.values())
    out = {
        "metric": "mixed-batch Z x and Z^H v throughput (p = 1..128), column-wise Tucker storage, graph-captured",
        "value": Ftot / (replay * 1e-3) / 1e12, "unit": "TFLOP/s",
        "config": {"workload": describe(w, inf) + f"; voxels with max(|x|, |y|) > {g.mask_box:.4f} m masked", "rhs": ps},
        "build": dict(build, seconds=t_aca),
        "per_p": per_p, "mixed_batch_ms": {"eager": eager, "graph": replay}, "gpu_launches_per_batch": launches,
    }
    del h, bufs, graph
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------------------------
# compression: HOSVD against the randomized Tucker with learned and with fixed widths
# ---------------------------------------------------------------------------------------------

def compression(zbc, torch, inputs, ntrain=256, ntest=256, batch=128):
    """Compression of the learned workload (128^3 voxels, 2 mm, 4096 random segments, tol 1e-6):
    the MLP is trained on the GPU on HOSVD ranks of ntrain columns, then ntest other columns are
    compressed by (a) truncated HOSVD, (b) the randomized Tucker with the MLP's widths, (c) the
    randomized Tucker with one fixed width for every tensor, the training set's largest rank + 4
    (the method without the network), and (d) a fixed width equal to the MLP's mean width (the
    same sketch budget spread evenly); (b) also with 8 instead of 4 oversampling columns.  Time per
    column, fallback rate, errors, mean ranks."""
    w = inputs.workload("learned")
    g, s = w.grid, w.segments
    perm = np.random.default_rng(7).permutation(s.m)
    train, test = perm[:ntrain], perm[ntrain:ntrain + ntest]
    ds = zbc.DeviceSegments(s)
    feats_all = inputs.rank_features(g, s)
    lmax = 64
    sk = [zbc.to_colmajor(o) for o in inputs.mode_sketches(g, lmax, seed=11)]

    def assemble(cols):
        cd = torch.from_numpy(np.asarray(cols, dtype=np.int32)).cuda()
        Z = zbc.colmajor(3 * g.nv, len(cols), torch.complex64)
        zbc.vsie_assemble_columns(g, ds, w.freq_hz, cd, Z)
        return Z

    def ranks_of(h):
        return h.export()[0].reshape(-1, 9)

    rt = []
    for b0 in range(0, ntrain, batch):
        Z = assemble(train[b0:b0 + batch])
        h, _ = zbc.tucker_compress(Z, g, w.tol)
        rt.append(ranks_of(h))
        del h, Z
    rt = np.concatenate(rt)
    T = torch.from_numpy(np.log(rt.astype(np.float32))).cuda()
    model = zbc.Mlp(inputs.mlp_init_params(0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = model.train(torch.from_numpy(feats_all[train]).cuda(), T, 3000, 1e-3).cpu().numpy()
    t_train = time.perf_counter() - t0
    fixed_max = int(rt.max()) + 4
    mean_learned = float(model.widths(torch.from_numpy(feats_all[test]).cuda(), g, oversample=4).mean())
    fixed_mean = int(round(mean_learned))
    models = {"fixed_max": zbc.rank_model(sk, lmax, fixed_width=fixed_max),
              "fixed_mean": zbc.rank_model(sk, lmax, fixed_width=fixed_mean)}
    res = {k: {"s": 0.0, "fallback": 0, "tensors": 0, "err": 0.0, "ranks": []}
           for k in ("hosvd", "learned", "learned_os8", "fixed_max", "fixed_mean")}
    for b0 in range(0, ntest, batch):
        cols = test[b0:b0 + batch]
        Z = assemble(cols)
        feats = torch.from_numpy(feats_all[cols]).cuda()
        for k in res:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if k == "hosvd":
                hh, st = zbc.tucker_compress(Z, g, w.tol)
            elif k.startswith("learned"):
                os_ = 8 if k == "learned_os8" else 4
                hh, st = zbc.tucker_compress(Z, g, w.tol, method=zbc.RANDOMIZED_LEARNED,
                                             model=zbc.rank_model(sk, lmax, mlp=model, features=feats, oversample=os_))
            else:
                hh, st = zbc.tucker_compress(Z, g, w.tol, method=zbc.RANDOMIZED_FIXED, model=models[k])
            torch.cuda.synchronize()
            res[k]["s"] += time.perf_counter() - t0
            res[k]["fallback"] += st.n_fallback
            res[k]["tensors"] += st.n_tensors
            res[k]["err"] = max(res[k]["err"], st.max_rel_err)
            res[k]["ranks"].append(ranks_of(hh))
            del hh
        del Z
    out = {
        "metric": "Tucker compression time per column: HOSVD vs randomized (learned / fixed widths), fallback rate",
        "value": 1e3 * res["learned"]["s"] / ntest, "unit": "ms/column", "higher_is_better": False,
        "config": {"workload": "learned: 128^3 voxels (2 mm), 4096 random 5 mm segments, 298.2 MHz, tol 1e-6",
                   "train_columns": ntrain, "test_columns": ntest, "batch": batch, "sketch_lmax": lmax,
                   "oversample": 4, "mlp_steps": 3000, "mlp_lr": 1e-3, "fixed_max_width": fixed_max,
                   "fixed_mean_width": fixed_mean, "learned_mean_width": mean_learned},
        "mlp": {"train_s": t_train, "loss_first": float(hist[0]), "loss_last": float(hist[-1])},
    }
    for k, r in res.items():
        rk = np.concatenate(r["ranks"])
        out[k] = {"ms_per_column": 1e3 * r["s"] / ntest, "fallback_rate": r["fallback"] / max(1, r["tensors"]),
                  "max_rel_err": r["err"], "mean_rank": float(rk.mean())}
    return out


# ---------------------------------------------------------------------------------------------
# compression from fibres (3D cross-Tucker) against assembly + HOSVD
# ---------------------------------------------------------------------------------------------

def cross_cpu_baseline(w, cols, tol, checks):
    """The FP64 oracle's fibre cross (entries evaluated voxel by voxel from the Green's function,
    as cross_tucker_assemble does) on a bounded sample of columns: ms per column."""
    from oracle import cross_tucker as xt
    g, s = w.grid, w.segments
    t0 = time.perf_counter()
    for e in cols:
        for k in range(3):
            src = xt.green_source(g.shape, g.h, s.centre, s.tangent, s.length, w.freq_hz, int(e), k,
                                  mask_radius=g.mask_radius, mask_box=g.mask_box)
            G, Us, _ = xt.cross_tucker(src, g.shape, tol)
            xt.check_error(src, G, Us, g.shape, checks)
    return 1e3 * (time.perf_counter() - t0) / len(cols)


def run_cross(args):
    """Compression from fibres (3D cross-Tucker; end of Sec. II.B.1 and Sec. V) against column
    assembly + truncated HOSVD, on columns of the 96^3 workload (2 mm, 298.2 MHz, tol 1e-6): time
    per column, tensor entries evaluated per tensor against n_v, the check-fibre error and the true
    error of both models against the assembled column (each handle decompressed on the GPU as Z~ I
    with the FP32 forward product).  Prints one JSON line."""
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
                                "cores": 1, "kind": "oracle",
                                "sample": f"{len(sample)} of the {ncols} columns (3 tensors each), same checks"}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# reference arm: the FP64 oracle on a bounded sample of the same workload
# ---------------------------------------------------------------------------------------------

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    from oracle import greens, products, tucker
    from paper_2103_06393_gb300 import inputs

    w = inputs.workload(args.workload)
    g, s = w.grid, w.segments
    p = w.p
    n1, n2, n3 = g.shape
    # a bounded sample of the workload: a few of its columns assembled and compressed by the
    # oracle itself on the first `planes` i3 planes; each step runs Algorithms 1 and 2 on them
    planes = max(2, n3 // 32) if w.aca else n3
    sub = (n1, n2, planes)
    ncols = 2 if w.aca else 4
    tol = w.tol
    t0 = time.perf_counter()
    cols = np.linspace(0, s.m - 1, ncols).round().astype(int)
    Z = greens.assemble_columns(sub, g.h, s.centre, s.tangent, s.length, w.freq_hz, cols)
    tens = tucker.compress_columns(Z, sub, 3, tol)
    del Z
    t_setup = time.perf_counter() - t0
    X = inputs.cn01((ncols, p), seed=0)
    Phi = inputs.cn01((3 * n1 * n2 * planes, p), seed=1)
    ranks = np.array([[U.shape[1] for U in t[1]] for tj in tens for t in tj])
    F_sample = 2.0 * products.flops(ranks, sub, 3, ncols, p)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        products.matvec(tens, sub, X)
        products.rmatvec(tens, sub, Phi)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    dt = float(np.mean(times))
    value = F_sample / dt / 1e12
    scale = n3 / planes
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * dt * scale, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128", "data": "synthetic", "impl": "reference", "extrapolated": True,
        "sample_ms_per_step": 1e3 * dt,
        "config": {"workload": f"{w.name}: {n1}x{n2}x{n3} voxels, {s.m} segments, 298.2 MHz, p={p}",
                   "path": "FP64 CPU oracle (Algorithms 1 and 2), one process",
                   "sample": f"{ncols} columns assembled and HOSVD-compressed (tol {tol:g}) by the oracle on "
                             f"{planes} of {n3} i3 planes ({t_setup:.1f}s setup)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "extrapolated": True,
                         "sample": f"{ncols} columns on {planes} of {n3} i3 planes per step; ms_per_step is "
                                   f"the sample's time x {scale:.0f} (all planes, the sample's columns)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="zbc", choices=["zbc", "reference"])
    ap.add_argument("--workload", default="large", choices=["large", "precision"])
    ap.add_argument("--prec", default="auto")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--extras-budget", type=float, default=700.0,
                    help="seconds since the start after which the ride-along workloads are skipped")
    ap.add_argument("--no-extras", action="store_true",
                    help="only the headline workload (no precision / batching / learned sub-objects)")
    ap.add_argument("--cross", action="store_true",
                    help="compression from fibres (cross-Tucker) vs assembly + HOSVD instead of the products")
    ap.add_argument("--columns", type=int, default=0,
                    help="keep only N segments (smaller case for profiler captures; no extras)")
    ap.add_argument("--n3", type=int, default=0,
                    help="keep only N planes of i3 (smaller case for profiler captures; no extras)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cross:
        run_cross(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_zbc(args)


if __name__ == "__main__":
    main()
