"""SAQ encode benchmark: encoded vectors/s on one GB300 (or N replicas).

A step is one full pass of the encode hot path (projection GEMM, per-segment
initial quantization, code adjustment, factors and bit-packing) over the whole
batch of the workload, inputs resident in HBM.  Default workload: 1,000,000
vectors of d = 960 drawn with a power-law spectrum (alpha = 0.8) under a
seeded random rotation, 4 bits/dim on average, 6 adjustment rounds, FP32
projection.  The batch (3.84 GB) is larger than L2, so no flush is needed
between steps.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on the host cores on a bounded sample of the same workload.
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
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import paper_2509_12086_gb300 as P  # noqa: E402
from paper_2509_12086_gb300 import synth  # noqa: E402

METRIC = "SAQ encoded vectors/s at d=960 4b/dim, FP32 vs BF16; ingest p50/p99 latency"
UNIT = "vectors/s"


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per row of one
# launch of each encode kernel, from ncu captures of one launch each on the
# 65,536-row case of the default workload.  Both kernels stream their rows, so
# a launch's traffic is proportional to its rows.  A figure is reported only while the
# kernel's source file is the one that was captured (SHA-1 below).
NCU_TRAFFIC = {
    "projection": {"src": "k_tc.cu", "sha1": "957519d74ad2b945597249c6b3734e933f4f3071",
                   "workload": "c2_d960", "precision": "fp32",
                   "bytes_per_row": (258402304 + 211736064) / 65536},
    "quantize_adjust_pack": {"src": "k_caq1.cu", "sha1": "ca5627b928766d09ea89518c720662654251fdcb",
                             "workload": "c2_d960", "precision": "fp32",
                             "bytes_per_row": (1558764544 + 35263744) / 65536},
}


def traffic_per_launch(kind, workload, precision, rows_per_launch):
    e = NCU_TRAFFIC.get(kind)
    if not e or e["workload"] != workload or e["precision"] != precision:
        return None
    with open(os.path.join(ROOT, "paper_2509_12086_gb300", "csrc", e["src"]), "rb") as f:
        if hashlib.sha1(f.read()).hexdigest() != e["sha1"]:
            return None
    return e["bytes_per_row"] * rows_per_launch


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            j = json.load(f)
        return {"hbm_gbs": j["hbm_gbs"], "bf16_tflops": j["bf16_tflops"],
                "bf16_tflops_sustained": j.get("bf16_tflops_sustained", j["bf16_tflops"]),
                "sm_max_mhz": j.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def ready(self, timeout_s=5.0):
        """Wait for nvidia-smi's first sample, then drop what came before the
        timed region."""
        t0 = time.perf_counter()
        while self.proc is not None and not self.lines and time.perf_counter() - t0 < timeout_s:
            time.sleep(0.01)
        self.lines.clear()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    elif torch.cuda.is_available():
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x, device="cuda"):
    """Slowest rank's time: the whole job ends when the last replica ends."""
    if world <= 1:
        return x
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(rank):
    """Each rank encodes its own batch (weak scaling); seeds differ by rank."""
    return synth.SEED_DATA + 7919 * rank


def workload_desc(w, name, precision, plan, code_bytes):
    return {"workload": "%s: N=%d d=%d power-law alpha=%.1f under a seeded random rotation, "
                        "%.0f b/dim avg, r=%d, %s projection" % (
                            name, w["n"], w["d"], w["alpha"], w["avg_bits"], w["rounds"],
                            precision),
            "n": w["n"], "d": w["d"], "alpha": w["alpha"], "avg_bits": w["avg_bits"],
            "rounds": w["rounds"], "precision": precision, "plan": plan,
            "code_bytes": code_bytes,
            "l2": "inputs (%.2f GB) larger than L2 (129 MB): no flush" % (w["n"] * w["d"] * 4 / 1e9)}


def cpu_baseline(w, X_dev, target_s=12.0, chunk=100000, one_core_s=3.0):
    """The FP64 oracle as it stands, on the host cores, on a bounded sample of
    the same workload: the rows it encodes in about `target_s` seconds, in
    chunks of `chunk` rows (model fitted on 50,000 rows, not timed); beside it
    the same oracle on one core, for about `one_core_s` seconds."""
    import oracle as O
    fit_rows = min(w["n"], 50000)
    Xf = X_dev[:fit_rows].cpu().numpy()
    mo = O.fit(Xf, w["avg_bits"])
    probe = Xf[:2000]
    t0 = time.perf_counter()
    O.encode(probe, mo, rounds=w["rounds"])
    per = (time.perf_counter() - t0) / probe.shape[0]
    ns = int(min(w["n"], max(2000, target_s / max(per, 1e-9))))
    dt = 0.0
    enc = None
    for r0 in range(0, ns, chunk):
        Xs = X_dev[r0:min(ns, r0 + chunk)].cpu().numpy()
        t0 = time.perf_counter()
        e = O.encode(Xs, mo, rounds=w["rounds"])
        dt += time.perf_counter() - t0
        if enc is None:
            enc = e
    cores = O.max_threads()
    ns1 = int(min(ns, max(200, one_core_s / max(per * cores, 1e-9))))
    try:
        one = cpu_baseline_one_core(mo, X_dev[:ns1].cpu().numpy(), w["rounds"])
    except (subprocess.SubprocessError, OSError, ValueError) as e:
        # the one-core figure is context beside the all-core baseline: a host
        # where the pinned child fails still gets its bench line
        one = {"value": None, "error": "%s: %s" % (type(e).__name__, str(e)[:200])}
    return {"value": ns / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d rows of the workload in chunks of %d (oracle fit on %d rows, not timed): "
                      "FP64 projection + CAQ + factors, %.1f s" % (ns, chunk, fit_rows, dt),
            "one_core": one}, mo, enc


_ONE_CORE = r"""
import os, pickle, sys, time
os.sched_setaffinity(0, {min(os.sched_getaffinity(0))})
sys.path.insert(0, sys.argv[1])
import oracle as O
with open(sys.argv[2], "rb") as f:
    mo, X, rounds = pickle.load(f)
t0 = time.perf_counter()
O.encode(X, mo, rounds=rounds, nthreads=1)
print(time.perf_counter() - t0, O.max_threads())
"""


def cpu_baseline_one_core(mo, X, rounds):
    """The same oracle on one core: a child process pinned to one CPU, with one
    OpenMP thread and one BLAS thread, on the first rows of the sample."""
    import pickle
    import tempfile
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    with tempfile.TemporaryDirectory() as td:
        path = os.path.join(td, "sample.pkl")
        with open(path, "wb") as f:
            pickle.dump((mo, X, rounds), f)
        out = subprocess.run([sys.executable, "-c", _ONE_CORE, ROOT, path], env=env,
                             capture_output=True, text=True, timeout=600, check=True)
    dt, threads = out.stdout.split()[-2:]
    dt = float(dt)
    return {"value": X.shape[0] / dt, "unit": UNIT, "cores": 1, "omp_threads": int(threads),
            "sample": "%d rows of the workload, one pinned CPU, one OpenMP and one BLAS thread, "
                      "%.1f s" % (X.shape[0], dt)}


def form_accuracy(m_forms, mo, enc, X_dev, rows=2000, nq=100, alpha=0.8):
    """Part of the CPU-baseline leg: the error of each projection form
    against the oracle's FP64 encode of the first `rows` rows of the sample
    that leg timed.  The library encodes the same rows with the oracle's
    model (imported, so rotations and plan are the same) in each form;
    reported: code agreement, mean quantization error eps against the
    oracle's, the largest per-vector |eps difference|, and the mean relative
    error of the library's distance estimates for `nq` queries (exact
    distances in FP64 on the GPU) beside that of the oracle's codes run
    through the same estimator."""
    import oracle as O
    ns = min(rows, enc.codes.shape[0])
    Xs = X_dev[:ns].contiguous()
    Q = synth.queries(nq, X_dev.shape[1], alpha, device=X_dev.device)
    X64, Q64 = Xs.double(), Q.double()
    exact = ((Q64 * Q64).sum(1)[:, None] + (X64 * X64).sum(1)[None, :] - 2.0 * Q64 @ X64.T)

    def rel_err(m, codes, factors):
        est = m.estimate_dist(codes, factors, Q).double()
        return float(((est - exact).abs() / exact.clamp_min(1e-300)).mean())

    eps_o = O.quant_error(enc.factors[:ns], mo)
    codes_o = torch.from_numpy(O.pack(enc.codes[:ns], mo)).to(X_dev.device)
    fac_o = torch.from_numpy(enc.factors[:ns].astype(np.float32)).to(X_dev.device)
    out = {}
    for prec in m_forms:
        m = P.saq_model_create(mo.d, mo.mean, mo.W, mo.plan, mo.sig2, rounds=6, precision=prec)
        c, f = m.encode(Xs)
        cu = O.unpack(c.cpu().numpy(), mo)
        eps = O.quant_error(f.cpu().numpy().astype(np.float64), mo)
        out[prec] = {"code_agreement": float((cu == enc.codes[:ns]).mean()),
                     "mean_eps": float(eps.mean()), "oracle_mean_eps": float(eps_o.mean()),
                     "max_abs_eps_diff": float(np.abs(eps - eps_o).max()),
                     "mean_rel_dist_err": rel_err(m, c, f),
                     "oracle_codes_mean_rel_dist_err": rel_err(m, codes_o, fac_o),
                     "sample": "%d rows x %d queries of the workload, oracle model imported"
                               % (ns, nq)}
        del m
    return out


# Algorithmic lane operations of quantize / adjust / pack (Eq. find_nearest_code,
# Algorithm 1, factors, bit-planes), per coordinate:
#   initial code: fma, floor, two clamps; I, |o|^2 and |u|^2 accumulations   7
#   one trial of a round: o*S, T = o*S - u*I, o*(o*S), |T|*I + o^2*S,
#     comparison with I^2, range check                                      6
#   an accepted move: I, S, I^2, the code                                   4
#   packing: extract and insert one bit per bit-plane                       2 per plane
ALU_INIT, ALU_TRIAL, ALU_ACCEPT, ALU_PACK = 7, 6, 4, 2


def alu_ops_per_vector(enc, mo, rounds):
    """Lane operations and round lane-steps (coordinate trials) per vector,
    counted from the oracle's accept statistics: a vector-segment runs rounds
    through its first round without an accept."""
    ops, steps = 0.0, 0.0
    for j, (off, l, b) in enumerate(mo.kept):
        a = enc.accepts[:, j, :rounds]
        zero = a == 0
        ran = np.where(zero.any(axis=1), zero.argmax(axis=1) + 1, rounds)
        ops += l * (ALU_INIT + ALU_PACK * b) + l * ALU_TRIAL * ran.mean()
        ops += ALU_ACCEPT * a.sum(axis=1).mean()
        steps += l * ran.mean()
    return ops, steps


def tf32_peak(dev, stream):
    """Measured cuBLAS TF32 GEMM rate (8192^3, FP32 operands), TFLOP/s."""
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = True
    try:
        a = torch.randn(8192, 8192, device=dev)
        b = torch.randn(8192, 8192, device=dev)
        for _ in range(3):
            torch.mm(a, b)
        t = time_events(lambda: torch.mm(a, b), 10, stream)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del a, b
    return 2.0 * 8192 ** 3 / t / 1e12


def run_reference(args):
    # the oracle runs on the host cores of rank 0 alone: no process group, no GPU
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    w = dict(synth.WORKLOADS[args.workload])
    # model fitted on 50,000 rows (not timed); each step encodes a chunk of
    # ref_rows further rows, the chunk size of the CPU baseline
    X = synth.power_law(min(w["n"], 50000 + args.ref_rows), w["d"], w["alpha"]).numpy()
    mo = O.fit(X[:50000], w["avg_bits"])
    sample = X[50000:50000 + args.ref_rows] if X.shape[0] > 50000 else X[:args.ref_rows]
    for _ in range(args.warmup):
        O.encode(sample[:500], mo, rounds=w["rounds"])
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.encode(sample, mo, rounds=w["rounds"])
    dt = time.perf_counter() - t0
    value = sample.shape[0] * args.steps / dt
    cfg = workload_desc(w, args.workload, "fp64 (oracle)", mo.plan, mo.code_bytes)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": dt * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": cfg,
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.max_threads(),
                            "kind": "oracle",
                            "sample": "%d rows per step, oracle fit on 50000 rows" % sample.shape[0]},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def time_events(fn, iters, stream):
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    start.record(stream)
    for _ in range(iters):
        fn()
    stop.record(stream)
    torch.cuda.synchronize()
    return start.elapsed_time(stop) / 1e3 / iters


def run_ours(args):
    world, rank, local = dist_setup()
    pk = peaks()
    w = dict(synth.WORKLOADS[args.workload])
    if args.n:
        w["n"] = args.n
    n, d = w["n"], w["d"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    # each rank encodes its own batch (weak scaling, no collective on the data path)
    X = synth.power_law(n, d, w["alpha"], seed=replica_seed(rank), device=dev)
    m = P.saq_fit(X, avg_bits=w["avg_bits"], rounds=w["rounds"], precision=args.precision)
    codes, factors = m.alloc_outputs(n, dev)

    def step():
        m.encode(X, codes, factors)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    clk.ready()
    l0 = P.saq_kernel_launch_count()
    P.saq_kernel_timing(True)
    t_dev = time_events(step, args.steps, stream) * args.steps
    launches = P.saq_kernel_launch_count() - l0
    clocks = clk.stop()
    # each launch's device time inside the timed steps (events on its own stream)
    ktimes = P.saq_kernel_times()
    P.saq_kernel_timing(False)
    torch.cuda.synchronize()
    barrier(world)
    t_max = max_over_ranks(world, t_dev)
    value = n * world * args.steps / t_max

    # kernel times per step from the timed region (each chunk of rows is
    # projected, then quantized, on the caller's stream)
    (ms_p, l_p), (ms_q, l_q) = ktimes["projection"], ktimes["quantize_adjust_pack"]
    t_proj = ms_p / 1e3 / args.steps
    t_caq = ms_q / 1e3 / args.steps
    # the same kernels alone (serial), in the encode's own data layout; the
    # kernel timer separates k_caq1 from the v_max pass this form adds
    rows = min(n, 262144)
    O_buf, nrm = m.project_interleaved(X[:rows])
    c2, f2 = m.alloc_outputs(rows, dev)
    m.quantize_interleaved(O_buf, nrm, c2, f2)
    torch.cuda.synchronize()
    P.saq_kernel_timing(True)
    for _ in range(3):
        m.project_interleaved(X[:rows])
        m.quantize_interleaved(O_buf, nrm, c2, f2)
    torch.cuda.synchronize()
    ka = P.saq_kernel_times()
    P.saq_kernel_timing(False)
    t_proj_alone = ka["projection"][0] / 1e3 / 3 * n / rows
    t_caq_alone = ka["quantize_adjust_pack"][0] / 1e3 / 3 * n / rows
    del O_buf, c2, f2
    plan = m.plan
    dk = m.d_kept
    flops = 2.0 * n * d * dk
    bytes_alg = n * (4.0 * d + m.code_bytes + 4.0 * m.factor_count)
    if args.precision in ("fp32_simt",) or not tc_enabled(m):
        sm_mhz = pk["sm_max_mhz"]
        fp32_peak = 152 * 128 * 2 * sm_mhz * 1e6 / 1e12  # FP32 FMA pipe, TFLOP/s
        proj_roof = {"bound": "alu", "achieved": flops / t_proj / 1e12, "peak": fp32_peak,
                     "unit": "TFLOP/s", "frac": flops / t_proj / 1e12 / fp32_peak,
                     "traffic": None,
                     "peak_source": "152 SMs x 128 FP32 lanes x 2 x %.0f MHz" % sm_mhz}
    else:
        pkv = pk["bf16_tflops_sustained"]
        proj_roof = {"bound": "tensor", "achieved": flops / t_proj / 1e12, "peak": pkv,
                     "unit": "TFLOP/s", "frac": flops / t_proj / 1e12 / pkv, "traffic": None,
                     "peak_source": "%s bf16 sustained" % pk["source"]}
        if args.precision == "fp32":
            # FP32 operands reach the tensor cores as TF32 or as a split into
            # FP16 pairs (three products here): the fraction of the measured
            # TF32 GEMM rate is the other yardstick
            tf = tf32_peak(dev, stream)
            proj_roof["tf32_peak_measured"] = tf
            proj_roof["frac_of_tf32"] = flops / t_proj / 1e12 / tf
    caq_bytes = n * (4.0 * dk + m.code_bytes + 4.0 * m.factor_count)
    caq_roof = {"bound": "hbm", "achieved": caq_bytes / t_caq / 1e9, "peak": pk["hbm_gbs"],
                "unit": "GB/s", "frac": caq_bytes / t_caq / 1e9 / pk["hbm_gbs"], "traffic": None,
                "peak_source": "%s hbm copy" % pk["source"]}
    # per launch, like `achieved` (algorithmic bytes or flops of one launch's rows)
    proj_roof["traffic"] = traffic_per_launch("projection", args.workload, args.precision,
                                              n / max(l_p / args.steps, 1))
    caq_roof["traffic"] = traffic_per_launch("quantize_adjust_pack", args.workload, args.precision,
                                             n / max(l_q / args.steps, 1))
    caq_roof["algorithmic_bytes_per_launch"] = caq_bytes / max(l_q / args.steps, 1)
    if caq_roof["traffic"] is not None:
        # the DRAM bytes the launches actually move (each adjustment round
        # re-reads the segment's rows and codes) over their time
        gbs = caq_roof["traffic"] * (l_q / args.steps) / t_caq / 1e9
        caq_roof["dram_traffic_gbs"] = gbs
        caq_roof["dram_traffic_frac"] = gbs / pk["hbm_gbs"]
    if t_proj >= t_caq:
        roof, dom = proj_roof, "projection"
    else:
        roof, dom = caq_roof, "quantize_adjust_pack"
    roof = dict(roof)
    roof["kernel"] = dom
    step_roof = 1.0 / max(flops / n / (pk["bf16_tflops"] * 1e12), bytes_alg / n / (pk["hbm_gbs"] * 1e9))

    # end to end through the host-buffer API: H2D of the rows, D2H of codes+factors
    e2e = None
    if not args.no_e2e:
        ne = min(n, args.e2e_rows)
        Xh = X[:ne].cpu().pin_memory()
        ch = torch.empty((ne, max(m.code_bytes, 1)), dtype=torch.uint8).pin_memory()
        fh = torch.empty((ne, m.factor_count), dtype=torch.float32).pin_memory()
        m.encode_host(Xh, ch, fh)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            m.encode_host(Xh, ch, fh)
        dt = (time.perf_counter() - t0) / args.e2e_steps
        dt = max_over_ranks(world, dt)
        # the host link's own rate on this machine: the same rows copied alone
        scratch = torch.empty((ne, d), dtype=torch.float32, device=dev)
        scratch.copy_(Xh, non_blocking=True)
        t_copy = time_events(lambda: scratch.copy_(Xh, non_blocking=True), 3, stream)
        del scratch
        h2d_gbs = ne * d * 4 / t_copy / 1e9
        e2e = {"value": ne * world / dt, "unit": UNIT, "h2d_bytes_per_step": ne * d * 4,
               "d2h_bytes_per_step": ne * (m.code_bytes + 4 * m.factor_count),
               "rows_per_step": ne, "h2d_gbs_measured": h2d_gbs,
               "frac_of_copy_in_bound": (ne / dt) / (ne / t_copy)}
        del Xh, ch, fh

    # the precision forms on the same batch (BF16 / FP8 projection, FP32 quantization)
    forms = {}
    if not args.no_forms:
        for prec in ("bf16", "fp8"):
            m.set_precision(prec)
            for _ in range(2):
                step()
            barrier(world)
            t = max_over_ranks(world, time_events(step, max(3, args.steps // 2), stream))
            forms[prec] = {"value": n * world / t, "unit": UNIT, "ms_per_step": t * 1e3,
                           "tensor_cores": m.tensor_cores}
        m.set_precision(args.precision)

    # distance estimation on the encoded batch (Sec. 3.2 estimator, b-bit
    # prefixes, Sec. 4.3 multi-stage bounds): query-vector pairs per second
    # (rank 0 alone, no collectives: a failure is reported in its field and
    # the headline line still prints)
    est = None
    if not args.no_estimator and rank == 0:
        try:
            ne, nqe = min(n, 100000), 100
            Qe = synth.queries(nqe, d, w["alpha"]).to(dev)
            ce, fe = codes[:ne], factors[:ne]
            est = {"n": ne, "nq": nqe}
            for name, fn in (("estimate", lambda: m.estimate_dist(ce, fe, Qe)),
                             ("prefix_2bit", lambda: m.estimate_dist(ce, fe, Qe, prefix_bits=2)),
                             ("staged_m2", lambda: m.estimate_staged(ce, fe, Qe, 2.0))):
                fn()
                t = time_events(fn, 3, stream)
                est[name + "_pairs_per_s"] = ne * nqe / t
            del Qe
        except Exception as e:  # noqa: BLE001
            est = {"error": "%s: %s" % (type(e).__name__, str(e)[:200])}

    # serving form: Poisson stream of insert requests over three collections
    ingest = None
    if not args.no_ingest and rank == 0:
        try:
            ingest = serving_run(args, dev)
        except Exception as e:  # noqa: BLE001
            ingest = {"error": "%s: %s" % (type(e).__name__, str(e)[:200])}

    cpu = None
    alu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, mo, enc = cpu_baseline(w, X)
        # the same leg: each projection form's error against the oracle
        try:
            acc = form_accuracy(["fp32"] + list(forms), mo, enc, X, alpha=w["alpha"])
            for prec, a in acc.items():
                if prec in forms:
                    forms[prec]["accuracy_vs_oracle"] = a
            cpu["fp32_accuracy_vs_oracle"] = acc.get("fp32")
        except Exception as e:  # noqa: BLE001
            cpu["accuracy_error"] = "%s: %s" % (type(e).__name__, str(e)[:200])
        if mo.plan == plan:
            ops, steps = alu_ops_per_vector(enc, mo, w["rounds"])
            # the step's own instruction ceiling at the quantize kernel's
            # occupancy (32 warps per SM), B of the plan's longest segment
            bits = max(mo.kept, key=lambda k: k[1])[2]
            ceil = P.saq_quantize_step_ceiling(32, bits)
            sm_mhz = clocks.get("sm_mhz") or pk["sm_max_mhz"]
            alu_peak = 152 * 128 * sm_mhz * 1e6 / 1e12
            alu = {"bound": "alu", "kernel": "quantize_adjust_pack",
                   "ops_per_vector": ops, "achieved": ops * n / t_caq / 1e12, "peak": alu_peak,
                   "unit": "Tops/s", "frac": ops * n / t_caq / 1e12 / alu_peak,
                   "peak_source": "152 SMs x 128 lanes x %.0f MHz (one op per lane per clock)" % sm_mhz,
                   "counted_from": "oracle accept statistics of the cpu_baseline sample",
                   "round_lane_steps_per_vector": steps,
                   "step_ceiling_lane_steps_per_s": ceil,
                   "frac_of_step_ceiling": steps * n / t_caq / ceil,
                   "step_ceiling_source": "saq_quantize_step_ceiling(32 warps/SM, B=%d): the "
                                          "adjustment step on register-resident data" % bits}

    if rank == 0:
        cfg = workload_desc(w, args.workload, args.precision, plan, m.code_bytes)
        cfg["parallelism"] = "replicas x%d (independent batches)" % world
        out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": max(3, args.warmup),
               "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "data": "synthetic",
               # projection operands of the form (FP32 accumulation; quantize,
               # adjust and factors in FP32 in every form)
               "dtype": {"bf16": "bf16", "fp8": "e4m3"}.get(args.precision, "f32"),
               "config": cfg, "roofline": roof,
               "kernels_ms_per_step": {"projection": t_proj * 1e3,
                                       "quantize_adjust_pack": t_caq * 1e3,
                                       "launches_per_step": {"projection": l_p / args.steps,
                                                             "quantize_adjust_pack": l_q / args.steps}},
               "kernels_ms_per_step_alone": {"projection": t_proj_alone * 1e3,
                                             "quantize_adjust_pack": t_caq_alone * 1e3},
               "alu_roofline": alu,
               "other_kernel_roofline": caq_roof if dom == "projection" else proj_roof,
               "step_roofline_vectors_per_s": step_roof,
               "step_roofline_frac": value / world / step_roof,
               "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": int(launches),
               "clocks": clocks, "precision_forms": forms, "estimator": est, "ingest": ingest}
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def serving_run(args, dev):
    """Continuous-batching ingest (include/saq.h saq_ingest_*): three resident
    collections (d = 128 / 960 at 4 b/dim, d = 1536 at 2 b/dim, alpha 0.8),
    requests of log-uniform size in [1, 65536] rows (2M vectors in all).  The
    service's capacity on this mix is measured first (all requests submitted
    at once, copies included, median of three passes after one warm-up pass;
    at about 7 GB of FP32 rows per pass it is bound by the host-to-device
    copies); then the same requests
    arrive as a Poisson stream at a load factor of that capacity, three runs
    per load factor.  HBM budget 40 GB.  Projection in BF16 (the serving
    configuration); the same requests through the FP32 projection are
    reported beside it (capacity and the headline load factor)."""
    rng = np.random.default_rng(2024)
    specs = [(128, 4.0), (960, 4.0), (1536, 2.0)]
    models = []
    for d, bits in specs:
        Xf = synth.power_law(100_000, d, 0.8, seed=17 + d, device=dev)
        models.append(P.saq_fit(Xf, avg_bits=bits, precision=args.ingest_precision))
    total = args.ingest_vectors
    sizes, colls = [], []
    while sum(sizes) < total:
        sizes.append(int(np.exp(rng.uniform(0.0, np.log(65536.0)))))
        colls.append(int(rng.integers(0, 3)))
    # request rows in page-locked host memory (generated on the GPU)
    reqs = []
    for i, (nr, c) in enumerate(zip(sizes, colls)):
        Xr = synth.power_law(nr, specs[c][0], 0.8, seed=5000 + i, device=dev).cpu().pin_memory()
        m = models[c]
        cb = torch.empty((nr, max(m.code_bytes, 1)), dtype=torch.uint8).pin_memory()
        fb = torch.empty((nr, m.factor_count), dtype=torch.float32).pin_memory()
        reqs.append((c, Xr, cb, fb))
    svc = P.Ingest(models, hbm_budget_bytes=40 << 30, max_batch_rows=65536, slots=4)
    # warm-up: every request once (the first copies out of freshly pinned
    # host pages run at a fraction of the link's rate)
    for t in [svc.submit(c, Xr, cb, fb) for c, Xr, cb, fb in reqs]:
        svc.wait(t, timeout_ms=120000)
    # capacity of the service on this request mix: everything submitted at
    # once, the median of three passes
    def capacity_of():
        sat = []
        for _ in range(3):
            t0 = time.perf_counter()
            tk = [svc.submit(c, Xr, cb, fb) for c, Xr, cb, fb in reqs]
            for t in tk:
                svc.wait(t, timeout_ms=120000)
            sat.append(time.perf_counter() - t0)
        return sum(sizes) / float(np.median(sat))
    capacity = capacity_of()
    # Poisson arrivals at load factors rho of that capacity (the headline
    # figures are those of --ingest-load; 0.5 and 0.95 are reported beside)
    def poisson(rho, seed, capacity=capacity):
        rate = rho * capacity / float(np.mean(sizes))  # requests / s
        gaps = np.random.default_rng(seed).exponential(1.0 / rate, size=len(sizes))
        b0 = svc.stats()["batches"]
        tickets = []
        t0 = time.perf_counter()
        due = t0
        for (c, Xr, cb, fb), g in zip(reqs, gaps):
            due += g
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            tickets.append(svc.submit(c, Xr, cb, fb))
        lats = np.array([svc.wait(t, timeout_ms=120000)[2] for t in tickets])
        wall = time.perf_counter() - t0
        return {"load_factor": rho, "arrival_rate_per_s": rate,
                "vectors_per_s": sum(sizes) / wall, "wall_s": wall,
                "p50_ms": float(np.percentile(lats, 50) * 1e3),
                "p99_ms": float(np.percentile(lats, 99) * 1e3), "max_ms": float(lats.max() * 1e3),
                "batches": int(svc.stats()["batches"] - b0)}
    # each load factor three times (a run lasts 0.05-0.1 s, so one hiccup of
    # the host can decide it): the run with the median p99, and all three
    def median_run(rho, seed, capacity=capacity):
        runs = sorted((poisson(rho, seed + 100 * k, capacity) for k in range(3)),
                      key=lambda r: r["p99_ms"])
        out = dict(runs[1])
        out["runs_p50_p99_ms"] = [[r["p50_ms"], r["p99_ms"]] for r in runs]
        return out
    head = median_run(args.ingest_load, 2025)
    others = {("%.2f" % rho): median_run(rho, 2026 + k)
              for k, rho in enumerate((0.5, 0.95)) if abs(rho - args.ingest_load) > 1e-9}
    st = svc.stats()
    batch_stats = {k: st[k] for k in ("batches", "mixed_batches", "deferred_batches",
                                      "peak_bytes_in_flight")}
    svc.close()
    # the same requests through the FP32 projection, beside
    fp32 = None
    if args.ingest_precision != "fp32":
        for m in models:
            m.set_precision("fp32")
        svc = P.Ingest(models, hbm_budget_bytes=40 << 30, max_batch_rows=65536, slots=4)
        for t in [svc.submit(c, Xr, cb, fb) for c, Xr, cb, fb in reqs[:30]]:
            svc.wait(t, timeout_ms=120000)
        cap32 = capacity_of()
        fp32 = {"saturation_vectors_per_s": cap32}
        fp32.update(median_run(args.ingest_load, 2125, cap32))
        svc.close()
    out = {"requests": len(sizes), "vectors": int(sum(sizes)), "saturation_vectors_per_s": capacity,
           "projection": args.ingest_precision}
    out.update(head)
    out.update({"other_loads": others, "slots": 4, "max_batch_rows": 65536, "hbm_budget_gb": 40,
                "collections": "d128@4b, d960@4b, d1536@2b (alpha 0.8)",
                "batch_stats": batch_stats, "fp32_projection": fp32})
    return out


def tc_enabled(m):
    # the library reports the projection kind through its precision setting;
    # the tensor-core path is used for fp32/bf16/fp8 when available
    return m.tensor_cores


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2_d960", choices=list(synth.WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=list(P.PRECISIONS))
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--e2e-rows", type=int, default=1_000_000)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--ref-rows", type=int, default=100000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true")
    ap.add_argument("--no-ingest", action="store_true")
    ap.add_argument("--no-estimator", action="store_true")
    ap.add_argument("--ingest-vectors", type=int, default=2_000_000)
    ap.add_argument("--ingest-load", type=float, default=0.8)
    ap.add_argument("--ingest-precision", default="bf16", choices=["fp32", "bf16", "fp8"])
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
