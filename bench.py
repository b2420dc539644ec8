#!/usr/bin/env python
"""TSQR benchmark: rows/s of tsqr_factor + tsqr_form_q on a tall-skinny matrix.

Default workload: FP64, m = 4,194,304 x n = 64, iid N(0, 1) entries, leaf
height 256, binary tree.  One step = restore A from a pristine device copy
(the factorisation overwrites A), tsqr_refactor (leaf QRs, tree, signs) and
tsqr_form_q (the thin Q).  Inputs (2.1 GB each) are larger than L2, so no L2
flush is needed between steps.

Prints one JSON line (rank 0).  Also reports:
  roofline      the dominant kernel's algorithmic FLOP rate against the FP64
                ALU peak (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz), timed with
                CUDA events the library records on the launching stream;
  cpu_baseline  the CPU oracle (plain Householder QR + form Q) on a bounded
                row sample, on this host's cores;
  e2e           the same step through the public API with host buffers:
                A read from pinned host memory by the leaf kernel, factor,
                form Q stored into pinned host memory, R back to the host
                (with each timed step's span, and the copy engines' pinned
                rates measured alone);
  variants      the mixed-precision form (FP32 storage, FP64 reflectors) on
                the same shape.
`--impl reference` times the CPU oracle alone (the reference arm).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSQR rows/s & CAQR GFLOP/s vs roofline at stated backward error, FP64 vs mixed"
FP64_PEAK_GFLOPS = 152 * 2 * 2 * 2.07  # SMs x DFMA/clk x flop/FMA x GHz = 1258.6 GFLOP/s


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=4194304)
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--leaf-rows", type=int, default=0, help="0 = the library default")
    p.add_argument("--arity", type=int, default=0, help="0 = the library default")
    p.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU time of the oracle sample")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--variants", default="mixed,hybrid,rec,lstsq,caqr,caqr_mixed,batched,grad",
                   help="comma list of extra measurements")
    p.add_argument("--caqr-leaf-rows", type=int, default=0)
    p.add_argument("--caqr-arity", type=int, default=0, help="0 = the library default")
    p.add_argument("--caqr-n", type=int, default=8192, help="square CAQR size for the CAQR variant")
    p.add_argument("--caqr-b", type=int, default=64)
    p.add_argument("--batched-count", type=int, default=2048, help="matrices in the batched variant")
    p.add_argument("--batched-autotune", type=int, default=1, help="0: default tile and arity, no autotuner")
    p.add_argument("--peaks", action="store_true",
                   help="compile and run bench_peaks.cu (FP64 / FP32 FMA and DMMA throughput probes) and exit")
    return p.parse_args()


def run_peaks():
    """FP64 FMA, FP32 FMA and DMMA rates of this GPU (bench_peaks.cu), printed as its own lines."""
    import tempfile

    exe = os.path.join(tempfile.mkdtemp(prefix="bench_peaks"), "bench_peaks")
    subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(ROOT, "bench_peaks.cu")], check=True)
    subprocess.run([exe], check=True)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# --------------------------------------------------------------- CPU oracle --
def oracle_rows_per_s(m_full: int, n: int, target_s: float, seed: int = 2000):
    """Time the CPU oracle (factor + thin Q) on a row sample of the workload."""
    import oracle
    from paper_0808_2664_gb300 import inputs

    oracle.build()
    ms = 8192
    while True:
        A = inputs.gaussian(ms, n, seed)
        t0 = time.perf_counter()
        oracle.qr(A)
        dt = time.perf_counter() - t0
        if dt >= target_s / 4 or ms >= m_full:
            break
        ms = min(m_full, int(ms * max(2.0, min(8.0, target_s / max(dt, 1e-3)))))
    return ms / dt, ms, dt, oracle.num_threads()


def reference_arm(args, world, rank):
    if rank != 0:
        return
    import oracle

    oracle.build()
    from paper_0808_2664_gb300 import inputs

    # Size one step so that warmup + steps stay within a few minutes.
    rate, ms, dt, cores = oracle_rows_per_s(args.m, args.n, target_s=4.0)
    per_step = max(8192, min(args.m, int(rate * 8.0)))
    A = inputs.gaussian(per_step, args.n, 2000)
    for _ in range(args.warmup):
        oracle.qr(A)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.qr(A)
    t = time.perf_counter() - t0
    value = per_step * args.steps / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": "rows/s", "cores": cores, "kind": "oracle",
                         "sample": f"{per_step} x {args.n} rows per step of the {args.m} x {args.n} workload"},
        "e2e": {"value": value, "unit": "rows/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


L2_BYTES = 129 * 2**20  # GB300 L2


def workload_config(args, dtype="f64"):
    nbytes = args.m * args.n * (8 if dtype == "f64" else 4)
    l2 = (f"inputs ({nbytes / 1e9:.1f} GB) larger than L2; no flush" if nbytes > L2_BYTES else
          f"inputs ({nbytes / 1e6:.1f} MB) fit in L2; no flush (warm-L2 figures)")
    return {"workload": f"tsqr_factor+form_q {dtype} m={args.m} n={args.n} gaussian",
            "m": args.m, "n": args.n, "leaf_rows": args.leaf_rows, "arity": args.arity, "l2": l2}


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r.split(",") for r in getattr(self, "out", "").strip().splitlines() if r.count(",") >= 8]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------- ours --
def run_variant(tq, torch, args, dtype, steps, warmup, seed, timing=False, flags=0, m=None, n=None):
    """tsqr_refactor + tsqr_form_q per step on an m x n N(0, 1) matrix.  The timed
    steps run without the library's stage events; with timing=True a second pass
    of the same steps records them (per-stage device times for the roofline)."""
    m, n = m or args.m, n or args.n
    dev = torch.device("cuda")
    from paper_0808_2664_gb300 import inputs

    A0 = inputs.gaussian_device(m, n, seed, dtype=dtype).t()  # column-major m x n
    A = tq.colmajor(m, n, dtype, dev)
    Q = tq.colmajor(m, n, dtype, dev)
    R = tq.colmajor(n, n, dtype, dev)
    q = tq.tsqr_q_create(m, n, dtype, dev, leaf_rows=args.leaf_rows, arity=args.arity, flags=flags)
    stream = torch.cuda.current_stream()

    def step():
        A.copy_(A0)
        q.refactor(A, R)
        q.form_q(Q)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_total = e0.elapsed_time(e1)
    # The restore copy of A, timed alone, so that the kernels' share is known.
    c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0.record(stream)
    for _ in range(steps):
        A.copy_(A0)
    c1.record(stream)
    torch.cuda.synchronize()
    copy_ms = c0.elapsed_time(c1) / steps
    stages = None
    if timing:
        q.set_timing(True)
        for _ in range(steps):
            step()
        torch.cuda.synchronize()
        stages = q.stage_times()
        q.set_timing(False)
    status = q.sync_status()
    # Backward error and orthogonality of the last step, in FP64 on the device.
    A64, Q64, R64 = A0.double(), Q.double(), R.double()
    berr = (torch.linalg.norm(A64 - Q64 @ R64) / torch.linalg.norm(A64)).item()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device=dev) - Q64.t() @ Q64).item()
    info = q.info()
    del A64, Q64, R64
    return {"ms_total": ms_total, "stages": stages, "status": status, "berr": berr, "orth": orth, "info": info,
            "q": q, "A0": A0, "A": A, "Q": Q, "R": R, "copy_ms": copy_ms}


def caqr_run(tq, torch, args, steps, warmup, dtype=None, upd=None):
    """Square CAQR, U[-1, 1] entries, panel width b: GFLOP/s of 4n^3/3 and the update's roofline.

    dtype float64 -> FP64 throughout; float32 -> FP32 storage with FP64
    reflector generation and FP32 (upd = PREC_FP32) or 3xBF16 tensor-core
    (upd = UPDATE_BF16X3) trailing updates."""
    dtype = dtype or torch.float64
    upd = tq.PREC_FP64 if upd is None else upd
    n, b = args.caqr_n, args.caqr_b
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(3001)
    A0 = (torch.rand((n, n), generator=g, dtype=torch.float64, device=dev) * 2 - 1).to(dtype).t()
    A = tq.colmajor(n, n, dtype, dev)
    q = tq.caqr_q_create(n, n, b, dtype, dev, update_precision=upd, leaf_rows=args.caqr_leaf_rows,
                          arity=args.caqr_arity)
    stream = torch.cuda.current_stream()

    def step():
        A.copy_(A0)
        q.refactor(A)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # Per-stage times come from a second pass with the library's stage
    # events on, so that recording them does not touch the timed steps.
    q.set_timing(True)
    for _ in range(steps):
        step()
    torch.cuda.synchronize()
    st = q.stage_times()
    q.set_timing(False)
    Q = q.form_q().double()
    R = torch.triu(A).double()
    A64 = A0.double()
    berr = (torch.linalg.norm(A64 - Q @ R) / torch.linalg.norm(A64)).item()
    orth = torch.linalg.norm(torch.eye(n, dtype=torch.float64, device=dev) - Q.t() @ Q).item()
    flops = 4.0 * n ** 3 / 3.0
    upd_ms = st["leaf_apply"][0] / steps
    upd_flops = sum(4.0 * (n - j) * b * (n - j - b) for j in range(0, n, b))
    eps = {tq.PREC_FP64: 2.0 ** -52, tq.PREC_FP32: 2.0 ** -23, tq.UPDATE_BF16X3: 2.0 ** -16,
           tq.UPDATE_TF32X3: 2.0 ** -18}[upd]
    if upd in (tq.UPDATE_BF16X3, tq.UPDATE_TF32X3):
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"] if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1900.0
        tf32 = upd == tq.UPDATE_TF32X3
        if tf32:
            peak *= 1.1 / 2.25  # the measured BF16 peak times the nominal dense TF32 / BF16 ratio
        ach = 3 * upd_flops / (upd_ms / 1e3) / 1e12
        # C (FP32) is read twice and written once per panel: 12 bytes per element.
        upd_bytes = sum(12.0 * (n - j) * (n - j - b) for j in range(0, n, b))
        roof = {"bound": "tensor", "kernel": "split3_update_kernel<%s> (tcgen05, 3 %s products per FP32 product)"
                % (("true", "TF32") if tf32 else ("false", "BF16")),
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": "MEASURED_PEAKS.json bf16_tflops" + (" x 1.1 / 2.25 (nominal TF32 / BF16)" if tf32 else ""),
                "hbm_achieved_gbs": upd_bytes / (upd_ms / 1e3) / 1e9,
                "note": "achieved counts the 3 BF16 products; at b = 64 the update is bound neither by the "
                        "tensor pipe nor by HBM but by each CTA's serial stage / MMA / epilogue steps; the "
                        "CAQR total is set by the panel chain (leaf and tree factor of each panel)"}
    elif upd == tq.PREC_FP32:
        ach = upd_flops / (upd_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "leaf_apply_kernel<float> (trailing update)", "achieved": ach,
                "peak": 152 * 128 * 2 * 2.07e9 / 1e12, "unit": "TFLOP/s",
                "frac": ach / (152 * 128 * 2 * 2.07e9 / 1e12)}
    else:
        ach = upd_flops / (upd_ms / 1e3) / 1e12
        roof = {"bound": "alu", "kernel": "leaf_apply_kernel<double> (trailing update)", "achieved": ach,
                "peak": FP64_PEAK_GFLOPS / 1e3, "unit": "TFLOP/s", "frac": ach / (FP64_PEAK_GFLOPS / 1e3)}
    return {"value": flops / (ms / 1e3) / 1e9, "unit": "GFLOP/s", "ms_per_step": ms, "n": n, "b": b,
            "storage": str(dtype).replace("torch.", ""),
            "update_precision": {tq.PREC_FP64: "fp64", tq.PREC_FP32: "fp32", tq.UPDATE_BF16X3: "3xbf16",
                                 tq.UPDATE_TF32X3: "3xtf32"}[upd],
            "backward_error": berr, "orthogonality": orth,
            # FP64: 10 n eps sqrt(m); FP32 storage: c sqrt(n) eps with c = 2 (FP32 products) or
            # 1 (3xBF16 / 3xTF32 products), orthogonality n eps32 (the tests' bounds).
            "tolerance": (10 * n * eps * n ** 0.5 if upd == tq.PREC_FP64 else
                          (2.0 if upd == tq.PREC_FP32 else 1.0) * n ** 0.5 * eps),
            "orthogonality_tolerance": 10 * n * eps * n ** 0.5 if upd == tq.PREC_FP64 else n * 2.0 ** -23,
            "status": q.sync_status(), "update_roofline": roof,
            "stage_ms_per_step": {k: v[0] / steps for k, v in st.items()}}


def batched_run(tq, torch, args, steps, warmup, count=2048, autotune=True):
    """2048 uneven FP32 matrices (m log-uniform in [1024, 65536], n in {16, 32, 64}):
    one persistent graph-replayed launch (autotuned) vs a loop over the plain path."""
    from paper_0808_2664_gb300 import inputs

    dev = torch.device("cuda")
    sh = inputs.batched_shapes(count, 4000)
    total = sum(m * n for m, n in sh)
    g = torch.Generator(device=dev)
    g.manual_seed(4000)
    buf0 = torch.randn(total, generator=g, dtype=torch.float32, device=dev)
    buf = torch.empty_like(buf0)
    As, off = [], 0
    for m, n in sh:
        As.append(buf[off:off + m * n].view(n, m).t())
        off += m * n
    buf.copy_(buf0)
    b = tq.Batch(As, autotune=autotune)
    info = b.info()

    def timed(run, k, w):
        for _ in range(w):
            buf.copy_(buf0)
            run()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(k):
            buf.copy_(buf0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            tot += e0.elapsed_time(e1)
        return tot / k

    ms_batch = timed(lambda: b.factor(graph=True), steps, warmup)
    status = b.sync_status()
    handles = [tq.tsqr_q_create(m, n, torch.float32, dev) for m, n in sh]
    Rs = [tq.colmajor(n, n, torch.float32, dev) for _, n in sh]

    def loop():
        for h, A, R in zip(handles, As, Rs):
            h.refactor(A, R)

    ms_loop = timed(loop, max(2, steps // 2), 1)
    # Accuracy of the FP32-storage R against the FP64 path on a sample of matrices.
    errs = []
    buf.copy_(buf0)
    b.factor(graph=True)
    torch.cuda.synchronize()
    for i in range(0, count, count // 16):
        A64 = buf0[sum(m * n for m, n in sh[:i]):][: sh[i][0] * sh[i][1]].view(sh[i][1], sh[i][0]).t().double()
        R64, _ = tq.tsqr_factor(tq.as_colmajor(A64.clone()), keep_q=False)
        errs.append((torch.linalg.norm(b.R[i].double() - R64) / torch.linalg.norm(R64)).item())
    for h in handles:
        h.destroy()
    algo_bytes = 2.0 * total * 4 + sum(n * n * 4 for _, n in sh)
    flops = sum(2.0 * m * n * n for m, n in sh)
    gbs = algo_bytes / (ms_batch / 1e3) / 1e9
    hbm = measured_hbm()
    res = {"value": count / (ms_batch / 1e3), "unit": "matrices/s", "ms_per_step": ms_batch,
           "loop_plain_path_ms": ms_loop, "speedup_vs_loop": ms_loop / ms_batch, "count": count,
           "elements": total, "tile_kb": info["tile_kb"], "arity": info["arity"], "work_items": info["items"],
           "gflops": flops / (ms_batch / 1e3) / 1e9,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm},
           "max_rel_err_r_vs_fp64_path_sample16": max(errs), "tolerance": 10 * 64 * 2.0 ** -23 * 65536 ** 0.5,
           "status": status}
    b.destroy()
    return res


def grad_run(tq, torch, dtype, steps, warmup, m=1 << 20, n=128):
    """Differentiable TSQR forward + backward at m x n (dQ, dR iid N(0, 1))."""
    from paper_0808_2664_gb300 import autograd as tqa
    from paper_0808_2664_gb300 import inputs

    A = inputs.gaussian_device(m, n, 5555, dtype=dtype).t()
    g = torch.Generator(device="cuda")
    g.manual_seed(5556)
    dQ = torch.randn((n, m), generator=g, dtype=dtype, device="cuda").t()
    dR = tq.as_colmajor(torch.triu(torch.randn((n, n), generator=g, dtype=dtype, device="cuda")))
    res = {}
    for recompute in (False, True):
        def step():
            Q, R = tqa.qr_forward(A)
            if recompute:
                del Q, R
                Q, R = tqa.qr_forward(A)
            return tqa.qr_backward(Q, R, dQ, dR)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        torch.cuda.reset_peak_memory_stats()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            dA = step()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        res["recompute" if recompute else "store"] = {"ms_per_step": ms,
                                                      "torch_peak_bytes": torch.cuda.max_memory_allocated()}
    # Gradient check against the device forward by central differences is in the tests; here the
    # forward's backward error on the last step.
    Q, R = tqa.qr_forward(A)
    Q64, R64, A64 = Q.double(), R.double(), A.double()
    berr = (torch.linalg.norm(A64 - Q64 @ R64) / torch.linalg.norm(A64)).item()
    res.update({"m": m, "n": n, "dtype": str(dtype).replace("torch.", ""), "forward_backward_error": berr,
                "flops_fwd_bwd": 4.0 * m * n * n + 6.0 * m * n * n})
    return res


def lstsq_run(tq, torch, args, steps, warmup, k=16):
    """Least squares (Section 1) for k right-hand sides: tsqr_refactor + tsqr_lstsq per step
    (leaves, tree, Q^T B through the tree, back substitution, residual norms)."""
    m, n = args.m, args.n
    from paper_0808_2664_gb300 import inputs

    dev = torch.device("cuda")
    A0 = inputs.gaussian_device(m, n, 6100).t()
    B0 = inputs.gaussian_device(m, k, 6101).t()
    A, B = tq.colmajor(m, n, torch.float64, dev), tq.colmajor(m, k, torch.float64, dev)
    X = tq.colmajor(n, k, torch.float64, dev)
    R = tq.colmajor(n, n, torch.float64, dev)
    q = tq.tsqr_q_create(m, n, torch.float64, dev)

    def step():
        A.copy_(A0)
        B.copy_(B0)
        q.refactor(A, R)
        return q.lstsq(R, B, X)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        _, rn = step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    # Optimality check on the device: the residual is orthogonal to range(A).
    Ad, Bd = A0.double(), B0.double()
    res = Ad @ X - Bd
    ortho = (torch.linalg.norm(Ad.t() @ res) / (torch.linalg.norm(Ad) * torch.linalg.norm(res))).item()
    rn_err = (torch.linalg.norm(torch.linalg.norm(res, dim=0) - rn) / torch.linalg.norm(rn)).item()
    status = q.sync_status()
    q.destroy()
    return {"value": m / (ms / 1e3), "unit": "rows/s", "ms_per_step": ms, "k": k,
            "normal_equations_residual": ortho, "residual_norm_rel_err": rn_err,
            "tolerance": 10 * n * 2.0 ** -52 * m ** 0.5, "status": status}


def measured_hbm():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except Exception:
        return 6800.0


def e2e_run(tq, torch, args, q, steps, warmup):
    """Public API with host buffers (tsqr_factor_form_host), each step inside the timed region: A
    read from pinned host memory by the leaf kernel, factor, form Q into pinned host memory, R to
    the host."""
    m, n = args.m, args.n
    dtype = torch.float64
    from paper_0808_2664_gb300 import inputs

    Ah = torch.empty((n, m), dtype=dtype, pin_memory=True)
    Ah.copy_(inputs.gaussian_device(m, n, 77, dtype=dtype).cpu())
    Ah = Ah.t()
    Qh = torch.empty((n, m), dtype=dtype, pin_memory=True).t()
    Rh = torch.empty((n, n), dtype=dtype, pin_memory=True).t()
    A = tq.colmajor(m, n, dtype)
    Q = tq.colmajor(m, n, dtype)
    R = tq.colmajor(n, n, dtype)
    stream = torch.cuda.current_stream()

    def step():
        # One library call: pinned host A in (read by the leaf kernel over the host link), host Q
        # and R out (Q stored by the form kernels straight into the pinned Q_host).
        q.factor_form_host(Ah, Qh, Rh, A, None, R)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    # One event between consecutive steps on the same stream: the total is the first to the
    # last, and the per-step spans show whether the copies stalled in some steps.
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    evs[0].record(stream)
    for i in range(steps):
        step()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [round(evs[i].elapsed_time(evs[i + 1]), 3) for i in range(steps)]
    es = 8
    # Plain pinned copies of the same buffers, each alone: the end-to-end step cannot beat
    # max(H2D, device work) + max(D2H, form) when the copies overlap only their own phase.
    def copy_gbs(fn):
        fn()
        torch.cuda.synchronize()
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(3):
            fn()
        c1.record(stream)
        torch.cuda.synchronize()
        return 3 * m * n * es / (c0.elapsed_time(c1) / 1e3) / 1e9

    h2d = copy_gbs(lambda: A.copy_(Ah, non_blocking=True))
    d2h = copy_gbs(lambda: Qh.copy_(Q, non_blocking=True))
    return {"value": m * steps / (ms / 1e3), "unit": "rows/s", "h2d_bytes_per_step": m * n * es,
            "d2h_bytes_per_step": m * n * es + n * n * es, "ms_per_step": ms / steps, "step_ms": step_ms,
            "pinned_h2d_gbs": h2d, "pinned_d2h_gbs": d2h, "host_cpus": sorted(os.sched_getaffinity(0))[:1] +
            sorted(os.sched_getaffinity(0))[-1:], "gpu_numa_node": _gpu_numa_node(torch)}


def dist_run(tq, torch, dist, args, rank, world):
    """Row-slab TSQR across the ranks (Section 2.1 parallel TSQR): each rank holds an m x n slab;
    one step = restore the slab, local TSQR, all_gather of the packed R triangles, the stacked
    triangles' structured QR, and this rank's block of the thin Q.  Timed between barriers with a
    device synchronize on both sides; the max over ranks.  The end-to-end form adds the pinned
    H2D copy of the slab and the D2H copies of Q_local and R to every step."""
    from paper_0808_2664_gb300 import distributed as D
    from paper_0808_2664_gb300 import inputs

    m, n = args.m, args.n
    dev = torch.device("cuda", torch.cuda.current_device())
    A0 = inputs.gaussian_device(m, n, 2200 + rank).t()
    A = tq.colmajor(m, n, torch.float64, dev)
    Q = tq.colmajor(m, n, torch.float64, dev)
    dt = D.DistTsqr(m, n, torch.float64, dev)

    def timed(step, k, w):
        for _ in range(w):
            step()
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(k):
            step()
        e1.record()
        torch.cuda.synchronize()
        dist.barrier()
        t = torch.tensor([e0.elapsed_time(e1) / k], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return t.item()

    def step():
        A.copy_(A0)
        dt.factor(A, Q)

    ms = timed(step, args.steps, args.warmup)
    Ah = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    Ah.copy_(A0)
    Qh = torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
    Rh = torch.empty((n, n), dtype=torch.float64, pin_memory=True)

    def step_host():
        A.copy_(Ah, non_blocking=True)
        _, R = dt.factor(A, Q)
        Qh.copy_(Q, non_blocking=True)
        Rh.copy_(R, non_blocking=True)

    ms_e2e = timed(step_host, max(3, args.steps // 2), 2)
    # Accuracy of the distributed factors on this rank's slab: A_p = Q_p R.
    A64 = A0.double()
    berr = (torch.linalg.norm(A64 - Q @ dt.R) / torch.linalg.norm(A64)).item()
    dt.destroy()
    return {"ms_per_step": ms, "slab_backward_error": berr,
            "e2e": {"value": world * m / (ms_e2e / 1e3), "unit": "rows/s", "h2d_bytes_per_step": m * n * 8,
                    "d2h_bytes_per_step": m * n * 8 + n * n * 8}}


def _gpu_numa_node(torch):
    """NUMA node of the current GPU from sysfs (None if unknown)."""
    try:
        p = torch.cuda.get_device_properties(torch.cuda.current_device())
        bus = f"{int(p.pci_domain_id):04x}:{int(p.pci_bus_id):02x}:{int(p.pci_device_id):02x}.0"
    except Exception:
        return None
    for cand in (bus,):
        path = f"/sys/bus/pci/devices/{cand}/numa_node"
        if os.path.exists(path):
            try:
                v = int(open(path).read().strip())
                return v if v >= 0 else None
            except (OSError, ValueError):
                return None
    return None


def _bind_to_gpu_node(torch):
    """Run on the host cores of the GPU's NUMA node, so that pinned buffers are allocated
    there and host-device copies do not cross sockets (no-op when the node is unknown)."""
    node = _gpu_numa_node(torch)
    if node is None:
        return
    try:
        spec = open(f"/sys/devices/system/node/node{node}/cpulist").read().strip()
    except OSError:
        return
    cpus = set()
    for part in spec.split(","):
        if "-" in part:
            a, b = part.split("-")
            cpus.update(range(int(a), int(b) + 1))
        elif part:
            cpus.add(int(part))
    cpus &= os.sched_getaffinity(0)
    if cpus:
        os.sched_setaffinity(0, cpus)


def ours(args, world, rank, local):
    import torch

    import paper_0808_2664_gb300 as tq

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    tq._lib.lib()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    dres = None
    with ClockSampler(local) as clk:
        r = run_variant(tq, torch, args, torch.float64, args.steps, args.warmup, seed=2000 + rank, timing=True)
        if dist:
            dres = dist_run(tq, torch, dist, args, rank, world)
    ms_step = r["ms_total"] / args.steps
    if dist:
        ms_step = dres["ms_per_step"]  # row-slab TSQR across the ranks, max over ranks
    m, n = args.m, args.n
    value = world * m / (ms_step / 1e3)

    # Roofline of the dominant kernel (per-launch averages from the stage events).
    st = r["stages"]
    info = r["info"]
    nl, h = info["leaves"], info["leaf_rows"]
    leaf_flops = 2.0 * m * n * n - nl * 2.0 * n ** 3 / 3.0  # Householder count per leaf, summed
    cands = {}
    for stage, (tot, launches) in st.items():
        if stage in ("leaf_factor", "leaf_apply") and launches:
            cands[stage] = tot / launches
    dom = max(cands, key=cands.get)
    dom_ms = cands[dom]
    achieved = leaf_flops / (dom_ms / 1e3) / 1e12
    peak = FP64_PEAK_GFLOPS / 1e3
    kernel_name = {"leaf_factor": "leaf_factor_kernel<double>", "leaf_apply": "leaf_apply_kernel<double> (form)"}[dom]
    # DRAM traffic of the leaf-factor launch: one ncu capture of this kernel (n = 64, h = 416) at
    # m = 524,288 read + wrote 567.3 MB; A, Y and the per-leaf R/T scale with the rows.
    traffic = None
    if dom == "leaf_factor" and n == 64 and h == 416:
        traffic = 567.3e6 / 524288 * m
    roofline = {"bound": "alu", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": traffic,
                "peak_source": "derived FP64 FMA peak: 152 SMs x 2 DFMA/clk x 2 x 2.07 GHz (probe measured 1.19-1.26)",
                "stage_ms_per_launch": {k: (v[0] / v[1] if v[1] else 0.0) for k, v in st.items()}}
    launches = int(sum(v[1] for v in st.values()))

    e2e = None
    if dist:
        e2e = dres["e2e"]
    elif not args.no_e2e:
        _bind_to_gpu_node(torch)
        e2e = e2e_run(tq, torch, args, r["q"], steps=max(3, args.steps // 2), warmup=2)
        e2e["value"] *= world

    variants = {}
    # At N > 1 the line measures the row-slab exchange; the single-GPU variants run at N = 1.
    want = set() if (args.no_variants or world > 1) else set(args.variants.split(","))
    del r["A0"], r["A"], r["Q"]
    torch.cuda.empty_cache()
    if "mixed" in want:
        ks = max(3, args.steps)
        v = run_variant(tq, torch, args, torch.float32, ks, 3, seed=3000 + rank, timing=True)
        lf_ms = v["stages"]["leaf_factor"][0] / max(1, v["stages"]["leaf_factor"][1])
        la_ms = v["stages"]["leaf_apply"][0] / max(1, v["stages"]["leaf_apply"][1])
        hbm = measured_hbm()
        # Leaf factor: reads A and writes Y (2 m n 4 bytes per launch); form: reads Y's slots and
        # Y, writes Q (2 m n 4 bytes).
        lf_gbs = 2.0 * m * n * 4 / (lf_ms / 1e3) / 1e9
        variants["mixed_fp32_storage_fp64_reflectors"] = {
            "value": world * m / (v["ms_total"] / ks / 1e3), "unit": "rows/s",
            "ms_per_step": v["ms_total"] / ks, "restore_copy_ms": v["copy_ms"], "backward_error": v["berr"],
            "orthogonality": v["orth"], "tolerance": 10 * n * 2.0 ** -23 * m ** 0.5, "status": v["status"],
            "roofline": {"bound": "hbm", "kernel": "leaf_factor_kernel<float>", "achieved": lf_gbs, "peak": hbm,
                         "unit": "GB/s", "frac": lf_gbs / hbm,
                         "form_kernel_gbs": 2.0 * m * n * 4 / (la_ms / 1e3) / 1e9},
            "stage_ms_per_launch": {k2: (x[0] / x[1] if x[1] else 0.0) for k2, x in v["stages"].items()}}
        del v
        torch.cuda.empty_cache()
    if "hybrid" in want:
        ks = max(3, args.steps // 2)
        v = run_variant(tq, torch, args, torch.float64, ks, 2, seed=2000 + rank, timing=True,
                        flags=tq.FLAG_HYBRID_TREE)
        ch = v["q"].chains()
        variants["hybrid_tree_fp64"] = {
            "value": world * m / (v["ms_total"] / ks / 1e3), "unit": "rows/s", "ms_per_step": v["ms_total"] / ks,
            "chains": ch["chains"], "leaves_per_chain": ch["leaves_per_chain"], "levels": v["info"]["levels"],
            "leaf_rows": v["info"]["leaf_rows"], "backward_error": v["berr"], "orthogonality": v["orth"],
            "tolerance": 10 * n * 2.0 ** -52 * m ** 0.5, "status": v["status"],
            "stage_ms_per_step": {k2: x[0] / ks for k2, x in v["stages"].items()}}
        del v
        torch.cuda.empty_cache()
        mf = 65536
        v = run_variant(tq, torch, args, torch.float64, 3, 1, seed=2100 + rank, flags=tq.FLAG_FLAT_TREE, m=mf)
        variants["flat_tree_fp64_m65536"] = {
            "value": world * mf / (v["ms_total"] / 3 / 1e3), "unit": "rows/s", "ms_per_step": v["ms_total"] / 3,
            "backward_error": v["berr"], "orthogonality": v["orth"], "status": v["status"],
            "note": "one CTA streams every leaf (sequential TSQR): a latency reference, not a throughput form"}
        del v
        torch.cuda.empty_cache()
    if "rec" in want:
        for dt, name in ((torch.float64, "recursive_leaf_fp64"), (torch.float32, "recursive_leaf_fp32")):
            ks = max(3, args.steps // 2)
            v = run_variant(tq, torch, args, dt, ks, 2, seed=2300 + rank, timing=True, flags=tq.FLAG_RECURSIVE_LEAF)
            variants[name] = {
                "value": world * m / (v["ms_total"] / ks / 1e3), "unit": "rows/s", "ms_per_step": v["ms_total"] / ks,
                "leaf_rows": v["info"]["leaf_rows"], "levels": v["info"]["levels"], "backward_error": v["berr"],
                "orthogonality": v["orth"], "status": v["status"],
                "stage_ms_per_launch": {k2: (x[0] / x[1] if x[1] else 0.0) for k2, x in v["stages"].items()}}
            del v
            torch.cuda.empty_cache()
    if "lstsq" in want:
        variants["lstsq_fp64_k16"] = lstsq_run(tq, torch, args, steps=max(3, args.steps // 2), warmup=2)
        torch.cuda.empty_cache()
    if "caqr" in want:
        variants["caqr_fp64"] = caqr_run(tq, torch, args, steps=3, warmup=3)
        torch.cuda.empty_cache()
    if "caqr_mixed" in want:
        variants["caqr_fp32_update"] = caqr_run(tq, torch, args, 3, 3, torch.float32, tq.PREC_FP32)
        torch.cuda.empty_cache()
        variants["caqr_3xbf16_update"] = caqr_run(tq, torch, args, 3, 3, torch.float32, tq.UPDATE_BF16X3)
        torch.cuda.empty_cache()
        variants["caqr_3xtf32_update"] = caqr_run(tq, torch, args, 3, 3, torch.float32, tq.UPDATE_TF32X3)
        torch.cuda.empty_cache()
    if "batched" in want:
        variants[f"batched_fp32_{args.batched_count}"] = batched_run(
            tq, torch, args, steps=5, warmup=3, count=args.batched_count, autotune=bool(args.batched_autotune))
        torch.cuda.empty_cache()
    if "grad" in want:
        variants["grad_fp64_1Mx128"] = grad_run(tq, torch, torch.float64, steps=3, warmup=3)
        variants["grad_fp32_1Mx128"] = grad_run(tq, torch, torch.float32, steps=3, warmup=3)

    # The CPU oracle runs after every GPU measurement, so that its host
    # threads never share the cores with the timed host-buffer pipeline.
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        rate, ms, dt, cores = oracle_rows_per_s(args.m, args.n, args.cpu_seconds)
        cpu = {"value": rate, "unit": "rows/s", "cores": cores, "kind": "oracle",
               "sample": f"{ms} x {args.n} rows (factor + thin Q) of the {args.m} x {args.n} workload, {dt:.1f} s"}
        import oracle as _oracle
        _oracle.set_num_threads(1)
        try:
            r1, ms1, dt1, _ = oracle_rows_per_s(args.m, args.n, args.cpu_seconds)
        finally:
            _oracle.set_num_threads(cores)
        cpu["single_thread"] = {"value": r1, "unit": "rows/s", "cores": 1,
                                "sample": f"{ms1} x {args.n} rows of the same workload, {dt1:.1f} s"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "rows/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": dict(workload_config(args), leaves=nl, levels=info["levels"], leaf_rows=h, arity=info["arity"],
                           parallelism=(f"{world} row slabs of {m} rows, one all_gather of packed R, structured "
                                        "top factorisation on every rank" if world > 1 else "1 GPU")),
            "single_gpu_ms_per_step": r["ms_total"] / args.steps,
            "backward_error": r["berr"], "orthogonality": r["orth"],
            "tolerance": 10 * n * 2.0 ** -52 * m ** 0.5, "device_status": r["status"],
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk.summary(), "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.peaks:
        run_peaks()
        return
    world, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, world, rank)
        return
    ours(args, world, rank, local)


if __name__ == "__main__":
    main()
