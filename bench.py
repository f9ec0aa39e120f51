"""Benchmark: exact QFT on 27 qubits (complex64 ket) through the C-ABI
library, in amplitude-gate updates per second.

One step = the whole hot path over one ket: the 391-gate QFT (H, controlled
phases, qubit-reversal swaps) applied to a seeded Gaussian 27-qubit ket as
fused dense blocks on the tensor cores (BF16x3 split, FP32 accumulation;
blocks of up to 6 qubits by default, --block 7 for the 7-qubit kernel),
followed by the FP64 norm of the result taken by the last block's
write-back. updates/s = gates x 2^n / step time. The ket (1 GiB) is larger
than L2, so no flush is needed between steps.

Also reported on the same box: the plain per-gate FP64 (complex128) path on
the same circuit (the in-run GPU baseline), fused SIMT and FP64 passes, the
other block sizes and splits, the 30-qubit 5x6 grid random circuit (10
layers), the roofline of the dominant kernel against the measured HBM copy
bandwidth, the end-to-end number with host buffers, and the FP64 CPU oracle
on a bounded sample.

--impl reference times the CPU oracle instead (the oracle is the reference
for this build: there is no reference implementation to install).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_QUBITS = 27


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the per-gate FP64, grid and CPU legs")
    ap.add_argument("--block", type=int, default=6, choices=[6, 7],
                    help="largest tensor-core block of the timed plans (6: k_tc_pipe, 7: the 7-qubit kernel)")
    ap.add_argument("--workload", default="qft27",
                    help="qft27 (default: the 27-qubit QFT on tensor-core blocks), "
                         "{qft,grid}<n>_{tc,tc7,tf32,tc128,simt} (one circuit on complex64 BF16x3 6- or 7-qubit, "
                         "or 3xTF32, or complex128, tensor-core blocks, or fused SIMT passes; "
                         "gates27: the per-gate kernels on a 27-qubit complex64 ket, low and high qubits; "
                         "profiling workloads), or appendix_a (the paper's fidelity-model validation in full)")
    return ap.parse_args()


def dist_init(n):
    """N > 1: one process per GPU under torchrun (NCCL; gloo where no CUDA
    device is present). The GPUs run independent replicas: no data-path
    collective, only the barrier and the max of the step times."""
    if n <= 1:
        return 0, 1
    import torch
    import torch.distributed as dist
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return dist.get_rank(), dist.get_world_size()


def max_over_ranks(x, world):
    """The largest value of x over all ranks (the job's time is its slowest
    replica's)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(world, units_per_rank, ms_per_step):
    """Whole-job throughput: every replica processes units_per_rank per step."""
    return world * units_per_rank / (ms_per_step * 1e-3)


# ------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
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
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle

def cpu_model():
    """Host CPU model name (lscpu's, else /proc/cpuinfo's; Arm hosts may list
    only a part number there)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            k, _, v = ln.partition(":")
            if k.strip().lower() == "model name" and v.strip():
                return v.strip()
    except Exception:
        pass
    try:
        names, parts = [], []
        for ln in open("/proc/cpuinfo"):
            k, _, v = ln.partition(":")
            k = k.strip().lower()
            if k in ("model name", "cpu model"):
                names.append(v.strip())
            elif k == "cpu part":
                parts.append(v.strip())
        if names:
            return names[0]
        if parts:
            return f"Arm CPU part {parts[0]}"
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


_ORACLE_INPUTS = {}


def oracle_sample(n_gates=16, n=N_QUBITS, seed=0, all_cores=False):
    """The FP64 CPU oracle on the first n_gates gates of the 27-qubit QFT on a
    Gaussian ket: the one-thread build, or the all-core build (the same C
    loops with OpenMP pragmas). Returns (updates/s, seconds, gates, threads)."""
    import oracle
    from paper_2304_14969_gb300 import workloads as W
    g = W.qft_circuit(n)[:n_gates]
    key = (n, seed)
    if key not in _ORACLE_INPUTS:
        _ORACLE_INPUTS.clear()
        _ORACLE_INPUTS[key] = W.gaussian_state(n, seed)
    x = _ORACLE_INPUTS[key]
    oracle.use_all_cores(all_cores)
    try:
        threads = oracle.threads()
        t0 = time.perf_counter()
        oracle.apply_circuit(x, g)
        dt = time.perf_counter() - t0
    finally:
        oracle.use_all_cores(False)
    return len(g) * (1 << n) / dt, dt, len(g), threads


def main_config(world, blocks=5, block=6):
    """The workload both arms report (the 27-qubit QFT on a Gaussian
    complex64 ket, on tensor-core blocks in this implementation)."""
    return {"workload": "qft27_gaussian_c64_tc_bf16x3", "n_qubits": N_QUBITS, "gates": 391, "blocks": blocks,
            "max_block": block,
            "path": f"fused <={block}-qubit blocks on tensor cores (BF16x3 split, FP32 accumulation)",
            "ket_bytes": 8 << N_QUBITS, "l2": "ket (1 GiB) larger than L2",
            "parallelism": "replicas" if world > 1 else "single"}


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (all-core build) on the host's
    cores, each step the first 16 gates of the 27-qubit QFT on the same
    Gaussian ket, in the same metric."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals, secs = [], []
    ng, threads = 16, 1
    for i in range(args.warmup + args.steps):
        v, dt, ng, threads = oracle_sample(n_gates=16, all_cores=True)
        if i >= args.warmup:
            vals.append(v)
            secs.append(dt)
    value = float(np.median(vals))
    sample = (f"first {ng} gates of the 27-qubit QFT on a Gaussian ket per step, FP64 oracle (all-core build, "
              f"{threads} threads, {cpu_model()}, nproc {os.cpu_count()})")
    line = {
        "impl": "reference", "metric": "amplitude-gate updates/s", "value": value, "unit": "updates/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * float(np.median(secs)), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(main_config(1), sample=sample),
        "cpu_baseline": {"value": value, "unit": "updates/s", "cores": threads, "kind": "oracle", "sample": sample,
                         "cpu_model": cpu_model(), "nproc": os.cpu_count()},
        "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ------------------------------------------------------------ GPU legs

def traffic_from_profiles(kernel):
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        e = d.get(kernel)
        if not e:
            return None
        src = os.path.join(ROOT, "paper_2304_14969_gb300", "csrc", e["source"])
        import hashlib
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
        return e["bytes_per_launch"] if h == e.get("source_sha") else None
    except Exception:
        return None


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.workload == "appendix_a":
        run_appendix_a()
        return
    if args.workload == "gates27":
        run_gates(args)
        return
    if args.workload != "qft27":
        run_grid_tc(args)
        return
    import torch
    rank, world = dist_init(args.gpus)
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    from paper_2304_14969_gb300 import build, qsim as Q
    from paper_2304_14969_gb300 import workloads as W
    build.build()
    Q.lib()
    n = N_QUBITS
    N = 1 << n
    gates = W.qft_circuit(n)
    ng = len(gates)
    circ = Q.Circuit(n, gates)
    stream = torch.cuda.Stream()
    sp = stream.cuda_stream
    # ket in a torch-owned device buffer, wrapped by the library
    x = W.gaussian_state(n, rank)
    x64 = torch.from_numpy(x.astype(np.complex64))
    host_in = torch.empty(N, dtype=torch.complex64).pin_memory()
    host_in.copy_(x64)
    host_out = torch.empty(N, dtype=torch.complex64).pin_memory()
    dev = torch.empty(N, dtype=torch.complex64, device="cuda")
    st = Q.State(n, Q.QSIM_C64, stream=sp, dev_ptr=dev.data_ptr())
    import ctypes as C
    Q.qsim_upload(st.h, C.c_void_p(host_in.data_ptr()))
    # The QFT leaves the ket bit-reversed (its swaps are relabels, Table I);
    # a second plan starts from that layout, so consecutive steps alternate
    # between the two plans and no step moves data for the relabel.
    # Fused blocks of <= 6 (or 7) qubits on the tensor cores (BF16x3 split,
    # FP32 accumulation in TMEM, controlled phases deferred into per-group
    # phases).
    mb = 7 if args.block == 7 else 0
    kernel = "k_tc_pipe7" if args.block == 7 else "k_tc_pipe"
    plans = [Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=mb)]
    plans[0].execute(st)
    plans.append(Q.Plan(circ, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=st, max_block=mb))
    plans[1].execute(st)
    info = plans[0].info()
    nrm = C.c_double()
    turn = [0]

    def step():
        # the plan, then the FP64 norm of the result (taken by the last
        # block's write-back; syncs)
        nrm.value = plans[turn[0]].execute_norm(st)
        turn[0] ^= 1

    for _ in range(args.warmup):
        step()
    # ---- timed region: K steps, events on the library's stream
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        clocks = ClockSampler(local)
        clocks.start()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        for k in range(args.steps):
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    # kernel timing for the roofline: the plan's launches back to back
    # (no host synchronisation between executions), events on the stream
    kt = max(10, args.steps // 4)
    with torch.cuda.stream(stream):
        torch.cuda.synchronize()
        ka, kz = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ka.record(stream)
        for _ in range(kt):
            plans[turn[0]].execute(st)
            turn[0] ^= 1
        kz.record(stream)
        torch.cuda.synchronize()
    pass_ms = [ka.elapsed_time(kz) / kt]
    total_ms = max_over_ranks(sum(step_ms), world)
    ms_per_step = total_ms / args.steps
    value = job_value(world, ng * N, ms_per_step)
    npass = info["passes"]
    launch_ms = float(np.mean(pass_ms)) / npass
    alg_bytes = 2 * 8 * N                   # one read + one write of the ket per pass
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    peak = peaks.get("hbm_gbs", 6800.0)

    # ---- end to end through the public API with pinned host buffers: every
    # step uploads its input ket, runs the QFT and downloads the result in
    # logical order; `depth` kets on as many streams, so one step's download
    # overlaps the next ones' uploads and transforms (the host link carries
    # both directions at once). Wall-clock over all steps, after every
    # stream drained; the pipeline depth (2 or 3) with the lower time is
    # reported, both are recorded.
    e2e_steps = max(6, min(args.steps, 12))
    extra_kets = [Q.State(n, Q.QSIM_C64, stream=torch.cuda.Stream().cuda_stream) for _ in range(2)]
    extra_outs = [torch.empty(N, dtype=torch.complex64).pin_memory() for _ in range(2)]
    kets_all, outs_all = [st] + extra_kets, [host_out] + extra_outs

    def e2e_run(depth):
        kets, outs = kets_all[:depth], outs_all[:depth]

        def e2e_step(k):
            s_ = kets[k % depth]
            Q.qsim_upload(s_.h, C.c_void_p(host_in.data_ptr()))
            plans[0].execute(s_)
            Q.qsim_download_async(s_.h, C.c_void_p(outs[k % depth].data_ptr()))

        for k in range(depth):
            e2e_step(k)
        for s_ in kets:
            Q.qsim_synchronize(s_.h)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(e2e_steps):
            e2e_step(k)
        for s_ in kets:
            Q.qsim_synchronize(s_.h)
        return (time.perf_counter() - t0) * 1e3 / e2e_steps

    e2e_by_depth = {d: e2e_run(d) for d in (2, 3)}
    e2e_depth = min(e2e_by_depth, key=e2e_by_depth.get)
    e2e_ms = e2e_by_depth[e2e_depth]
    for s_ in extra_kets:
        s_.close()
    e2e_val = job_value(world, ng * N, max_over_ranks(e2e_ms, world))
    phases = e2e_phases(Q, C, torch, plans[0], st, stream, host_in, host_out)
    parity = headline_parity(Q, W, plans, st, n)

    extras = {}
    if rank == 0 and not args.no_extras:
        extras = extra_legs(Q, W, C, torch, circ, x, n, ng, plans)
    if rank != 0:
        return
    cpu = {}
    if not args.no_extras:
        # the oracle as it stands on the host's cores (all-core build), and
        # its one-thread build beside it
        v, dt, k, thr = oracle_sample(n_gates=64, all_cores=True)
        v1, dt1, k1, _ = oracle_sample(n_gates=8)
        cpu = {"value": v, "unit": "updates/s", "cores": thr, "kind": "oracle",
               "sample": f"first {k} gates of the 27-qubit QFT on a Gaussian ket, FP64 oracle, all-core build "
                         f"({thr} threads, {dt:.1f} s)",
               "cpu_model": cpu_model(), "nproc": os.cpu_count(),
               "one_thread": {"value": v1, "unit": "updates/s", "cores": 1,
                              "sample": f"first {k1} gates, one-thread build ({dt1:.1f} s)"}}
    line = {
        "metric": "amplitude-gate updates/s", "value": value, "unit": "updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": main_config(world, npass, args.block),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_from_profiles(kernel),
                     "kernel": kernel, "alg_bytes_per_launch": alg_bytes,
                     "launch_ms": launch_ms, "peak_source": "measured hbm_gbs" if peaks else "fallback"},
        "e2e": {"value": e2e_val, "unit": "updates/s", "h2d_bytes_per_step": 8 * N, "d2h_bytes_per_step": 8 * N,
                "ms_per_step": e2e_ms,
                "pipeline": f"{e2e_depth} kets on {e2e_depth} streams: upload, QFT, download in logical order",
                "ms_per_step_by_depth": e2e_by_depth, "phases_one_stream": phases},
        "infidelity": parity,
        "gpu_launches": args.steps * npass,   # timed steps (the kernel-timing loop is outside the step region)
        "clocks": clk,
        "cpu_baseline": cpu,
        "norm_check": nrm.value,   # after every step so far ran on the same ket (repeated transforms)
    }
    line.update(extras)
    if "per_gate_fp64" in extras:
        line["speedup_vs_per_gate_fp64"] = extras["per_gate_fp64"]["ms"] / float(np.mean(pass_ms))
    print(json.dumps(line))
    st.close()


def _chunked_fidelity(y, ref_fn, N, chunk=1 << 24):
    """1 - |<y|ref>|^2 / (<y|y><ref|ref>) in FP64, with ref produced chunk by
    chunk by ref_fn(start, stop) (keeps host memory small at 2^27)."""
    ip = 0j
    ny = nr = 0.0
    for a in range(0, N, chunk):
        b = min(N, a + chunk)
        yy = y[a:b].astype(np.complex128)
        rr = ref_fn(a, b)
        ip += np.vdot(yy, rr)
        ny += float(np.vdot(yy, yy).real)
        nr += float(np.vdot(rr, rr).real)
    return 1.0 - abs(ip) ** 2 / (ny * nr)


def headline_parity(Q, W, plans, st, n):
    """The timed path's error, measured beside the headline: the bench's two
    plans applied to a basis ket |x>, every output of the first against
    Eq. (dft)'s closed form y_k = 2^(-n/2) exp(2 pi i x k / 2^n), the second
    (the QFT applied again) against QFT^2 |x> = |-x mod 2^n>."""
    N = 1 << n
    x = W.basis_index(n, 27)
    Q.qsim_set_basis(st.h, x)
    n0 = plans[0].execute_norm(st)
    y = st.download()

    def cf(a, b):
        ks = np.arange(a, b, dtype=np.int64)
        return np.exp(2j * np.pi * ((x * ks) % N).astype(np.float64) / N) / np.sqrt(N)

    f0 = _chunked_fidelity(y, cf, N)
    n1 = plans[1].execute_norm(st)
    y = st.download().astype(np.complex128)
    j = (N - x) % N
    f1 = 1.0 - abs(y[j]) ** 2 / float(np.vdot(y, y).real)
    return {"input": f"basis |x>, x = {x}", "infidelity_first_plan_vs_closed_form": f0,
            "infidelity_second_plan_vs_closed_form": f1, "fused_norms": [n0, n1], "bound": 1e-6,
            "within_bound": bool(f0 <= 1e-6 and f1 <= 1e-6)}


def e2e_phases(Q, C, torch, plan, st, stream, host_in, host_out, reps=4):
    """Device time of each phase of one end-to-end step on one stream (CUDA
    events): upload of the input ket from pinned memory, the plan, the
    download in logical order (permutation and copy to pinned memory)."""
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    acc = np.zeros(3)
    for r in range(reps + 1):
        ev[0].record(stream)
        Q.qsim_upload(st.h, C.c_void_p(host_in.data_ptr()))
        ev[1].record(stream)
        plan.execute(st)
        ev[2].record(stream)
        Q.qsim_download_async(st.h, C.c_void_p(host_out.data_ptr()))
        ev[3].record(stream)
        Q.qsim_synchronize(st.h)
        if r:
            acc += [ev[k].elapsed_time(ev[k + 1]) for k in range(3)]
    acc /= reps
    gb = host_in.numel() * host_in.element_size() / 1e9
    # the host link itself: a 1 GiB copy each way alone and both at once on
    # two streams (copy engines, pinned buffers), the floor of an e2e step
    dev_a = torch.empty_like(host_in, device="cuda")
    dev_b = torch.empty_like(host_in, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def link(h2d, d2h):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if h2d:
            with torch.cuda.stream(s1):
                dev_a.copy_(host_in, non_blocking=True)
        if d2h:
            with torch.cuda.stream(s2):
                host_out.copy_(dev_b, non_blocking=True)
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) * 1e3

    for _ in range(2):
        link(True, True)
    h2d_ms = min(link(True, False) for _ in range(3))
    d2h_ms = min(link(False, True) for _ in range(3))
    both_ms = min(link(True, True) for _ in range(3))
    del dev_a, dev_b
    return {"upload_ms": acc[0], "plan_ms": acc[1], "download_ms": acc[2], "upload_gbs": gb / (acc[0] * 1e-3),
            "download_gbs": gb / (acc[2] * 1e-3),
            "link": {"h2d_ms": h2d_ms, "d2h_ms": d2h_ms, "both_ms": both_ms, "h2d_gbs": gb / (h2d_ms * 1e-3),
                     "d2h_gbs": gb / (d2h_ms * 1e-3), "both_gbs_total": 2 * gb / (both_ms * 1e-3)}}


def time_plan(Q, C, plan, st, reps):
    """Device time of plan executions (events on the ket's stream)."""
    import torch
    s = torch.cuda.Stream()
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.execute(st)
    Q.qsim_synchronize(st.h)
    torch.cuda.synchronize()
    a.record()
    for _ in range(reps):
        plan.execute(st)
    z.record()
    Q.qsim_synchronize(st.h)
    torch.cuda.synchronize()
    return a.elapsed_time(z) / reps


def run_gates(args):
    """Per-gate kernels (A2-A4) and the all-qubit Bloch reduction (A11) on a
    27-qubit complex64 ket (1 GiB, larger than L2), each gate on high and on
    low qubits (where a 32-byte sector
    holds 4 amplitudes and a gate touching every other run of them reads
    whole sectors anyway): device time per call (CUDA events), algorithmic
    bytes and GB/s. The profiling workload for their DRAM traffic."""
    import ctypes as C
    import torch
    from paper_2304_14969_gb300 import build, qsim as Q
    build.build()
    Q.lib()
    n = N_QUBITS
    N = 1 << n
    B = 8
    st = Q.State(n, Q.QSIM_C64)
    Q.qsim_set_basis(st.h, 12345)
    h = np.ascontiguousarray(np.array([1, 0, 1, 0, 1, 0, -1, 0], dtype=np.float64) / np.sqrt(2))
    x = np.ascontiguousarray(np.array([0, 0, 1, 0, 1, 0, 0, 0], dtype=np.float64))
    fsim = np.zeros((4, 4), dtype=np.complex128)
    fsim[0, 0] = 1
    fsim[1, 2] = fsim[2, 1] = -1j
    fsim[3, 3] = np.exp(-1j * np.pi / 6)
    f2 = np.ascontiguousarray(fsim.ravel().view(np.float64))
    ctl = (C.c_int * 1)(5)
    hp = h.ctypes.data_as(C.c_void_p)
    r3 = np.zeros(3 * n)
    cases = [
        ("H q20", lambda: Q.qsim_apply_gate(st.h, hp, 20, None, 0, 0), 2 * B * N),
        ("H q1", lambda: Q.qsim_apply_gate(st.h, hp, 1, None, 0, 0), 2 * B * N),
        ("CX c5 t20", lambda: Q.qsim_apply_gate(st.h, x.ctypes.data_as(C.c_void_p), 20, ctl, 1, 1), B * N),
        ("CP q3 q22", lambda: Q.qsim_apply_cphase(st.h, 3, 22, 0.3), 2 * B * N // 4),
        ("CP q0 q1", lambda: Q.qsim_apply_cphase(st.h, 0, 1, 0.3), 2 * B * N // 4),
        ("CP q20 q24", lambda: Q.qsim_apply_cphase(st.h, 20, 24, 0.3), 2 * B * N // 4),
        ("fSim q7 q19", lambda: Q.qsim_apply_2q(st.h, f2.ctypes.data_as(C.c_void_p), 7, 19), 2 * B * N),
        # all 27 Bloch vectors: three tiled passes, each one read of the ket (synchronises)
        ("Bloch all", lambda: Q.qsim_bloch_all(st.h, r3.ctypes.data_as(C.c_void_p)), 3 * B * N),
    ]
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    peak = peaks.get("hbm_gbs", 6800.0)
    out = {}
    for name, fn, by in cases:
        for _ in range(args.warmup):
            fn()
        Q.qsim_synchronize(st.h)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(args.steps):
            fn()
        z.record()
        Q.qsim_synchronize(st.h)
        torch.cuda.synchronize()
        ms = a.elapsed_time(z) / args.steps
        out[name] = {"ms": ms, "alg_bytes": by, "gbs": by / (ms * 1e-3) / 1e9, "frac_of_hbm": by / (ms * 1e-3) / 1e9 / peak}
    st.close()
    print(json.dumps({"workload": "gates27", "n_qubits": n, "ket_bytes": B * N, "steps": args.steps, "cases": out}))


def run_grid_tc(args):
    """One grid circuit or QFT on tensor-core blocks or fused SIMT passes
    (profiling workload)."""
    import ctypes as C
    import torch
    from paper_2304_14969_gb300 import build, qsim as Q
    from paper_2304_14969_gb300 import workloads as W
    build.build()
    Q.lib()
    fam = "qft" if args.workload.startswith("qft") else "grid"
    n = int(args.workload[len(fam):].split("_")[0])
    simt = args.workload.endswith("_simt")
    k7 = args.workload.endswith("_tc7")
    c128 = args.workload.endswith("_tc128")
    tf32 = args.workload.endswith("_tf32")
    dt, es = (Q.QSIM_C128, 16) if c128 else (Q.QSIM_C64, 8)
    prec_kw = {} if simt else {"prec": Q.QSIM_PREC_BF16X6 if c128 else Q.QSIM_PREC_3XTF32 if tf32
                               else Q.QSIM_PREC_BF16X3}
    if k7:
        prec_kw["max_block"] = 7
    if fam == "grid":
        rows, cols = W.grid_shape(n)
        g = W.grid_rcs_circuit(rows, cols, 10, seed=0, n=n)
    else:
        g = W.qft_circuit(n)
    circ = Q.Circuit(n, g)
    st = Q.State(n, dt)
    # plans for both qubit maps the state alternates between (a QFT with
    # relabelled swaps leaves the ket bit-reversed), so no step permutes
    plans = [Q.Plan(circ, dtype=dt, state=st, **prec_kw)]
    plans[0].execute(st)
    plans.append(Q.Plan(circ, dtype=dt, state=st, **prec_kw))
    k = 1
    for _ in range(args.warmup):
        plans[k % 2].execute(st)
        k += 1
    Q.qsim_synchronize(st.h)
    import torch
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record()
    for _ in range(args.steps):
        plans[k % 2].execute(st)
        k += 1
    z.record()
    Q.qsim_synchronize(st.h)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / args.steps
    nb = plans[0].info()["passes"]
    N = 1 << n
    print(json.dumps({"metric": "amplitude-gate updates/s", "value": len(g) * N / (ms * 1e-3), "unit": "updates/s",
                      "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                      "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                      "data": "synthetic",
                      "config": {"workload": f"{fam}{n}_" + ("c128_tc_bf16x6" if c128 else "c64_fused_simt" if simt
                                                             else "c64_tc_3xtf32" if tf32 else
                                                             "c64_tc_bf16x3_k7" if k7 else "c64_tc_bf16x3"),
                                 "n_qubits": n, "gates": len(g), "launches_per_step": nb},
                      "roofline": {"bound": "hbm", "kernel": "k_fused_pass" if simt else
                                   "k_tc_pipe7" if k7 else "k_tc_pipe",
                                   "achieved": 2 * es * N / (ms / nb * 1e-3) / 1e9}}))


def c128_tc_leg(Q, C, torch, circ, x, n, ng, sref, peaks, fused_ms, per_gate_ms, reps=6):
    """Complex128 ket through BF16X6 tensor-core blocks: device time (two
    plans alternated, as the QFT leaves the ket bit-reversed), HBM rate per
    block, and infidelity against sref, the per-gate FP64 result of the same
    circuit on the same input (x, or |0...0> when x is None)."""
    N = 1 << n
    st = Q.State(n, Q.QSIM_C128)
    if x is None:
        Q.qsim_set_basis(st.h, 0)
    else:
        st.upload(x)
    tps = [Q.Plan(circ, dtype=Q.QSIM_C128, prec=Q.QSIM_PREC_BF16X6, state=st)]
    tps[0].execute(st)
    ip = (C.c_double * 2)()
    na, nb = C.c_double(), C.c_double()
    Q.qsim_inner_product(sref.h, st.h, ip)
    Q.qsim_norm(sref.h, C.byref(na))
    Q.qsim_norm(st.h, C.byref(nb))
    infid = 1.0 - (ip[0] ** 2 + ip[1] ** 2) / (na.value * nb.value)
    tps.append(Q.Plan(circ, dtype=Q.QSIM_C128, prec=Q.QSIM_PREC_BF16X6, state=st))
    tps[1].execute(st)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Q.qsim_synchronize(st.h)
    torch.cuda.synchronize()
    a.record()
    for r in range(reps):
        tps[r % 2].execute(st)
    z.record()
    Q.qsim_synchronize(st.h)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / reps
    nbk = tps[0].info()["passes"]
    achieved = 2 * 16 * N / (ms / nbk * 1e-3) / 1e9
    st.close()
    r = {"updates_per_s": ng * N / (ms * 1e-3), "ms": ms, "blocks": nbk, "kernel": "k_tc_pipe (complex128)",
         "hbm_gbs_per_block": achieved, "frac_of_hbm": achieved / peaks.get("hbm_gbs", 6800.0),
         "infidelity_vs_per_gate_fp64": infid, "speedup_vs_per_gate_fp64": per_gate_ms / ms,
         "alg_bytes_per_block": 2 * 16 * N}
    if n == 27 and circ.n == 27:
        # ncu DRAM traffic per launch of the QFT-27 blocks (profiles/traffic.json)
        r["traffic_per_block"] = traffic_from_profiles("k_tc_pipe_c128")
    if fused_ms:
        r["speedup_vs_fused_fp64"] = fused_ms / ms
    return r


def extra_legs(Q, W, C, torch, circ, x, n, ng, plans):
    out = {}
    N = 1 << n
    # plain per-gate FP64 path on the same circuit
    s128 = Q.State(n, Q.QSIM_C128)
    s128.upload(x)
    o = Q.qsim_run_opts(mode=0, relabel_swaps=1)
    Q.qsim_run_circuit(s128.h, circ.ptr(), C.byref(o))
    Q.qsim_synchronize(s128.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q.qsim_upload(s128.h, x.ctypes.data_as(C.c_void_p))
    Q.qsim_synchronize(s128.h)
    t0 = time.perf_counter()
    Q.qsim_run_circuit(s128.h, circ.ptr(), C.byref(o))
    Q.qsim_synchronize(s128.h)
    pg = time.perf_counter() - t0
    out["per_gate_fp64"] = {"updates_per_s": ng * N / pg, "ms": pg * 1e3, "dtype": "c128"}
    # the headline path (first plan of the timed steps) on the same Gaussian
    # input, against the per-gate FP64 result: the infidelity of the speedup
    ref = s128.download()
    sh = Q.State(n, Q.QSIM_C64)
    sh.upload(x)
    plans[0].execute_norm(sh)
    yh = sh.download()
    sh.close()
    out["per_gate_fp64"]["infidelity_of_headline_path"] = _chunked_fidelity(yh, lambda a, b: ref[a:b], N)
    del ref, yh
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    # fused c128
    s = Q.State(n, Q.QSIM_C128)
    s.upload(x)
    p = Q.Plan(circ, dtype=Q.QSIM_C128)
    p.execute(s)
    Q.qsim_synchronize(s.h)
    t0 = time.perf_counter()
    for _ in range(3):
        p.execute(s)
    Q.qsim_synchronize(s.h)
    f128 = (time.perf_counter() - t0) / 3
    out["fused_fp64"] = {"updates_per_s": ng * N / f128, "ms": f128 * 1e3, "dtype": "c128",
                         "passes": p.info()["passes"]}
    s.close()
    # the same QFT on complex128 tensor-core blocks (BF16X6: three BF16
    # slices per operand, six products, FP32 accumulation), against the
    # per-gate FP64 result
    out["qft27_c128_tc_bf16x6"] = c128_tc_leg(Q, C, torch, circ, x, n, ng, s128, peaks, out["fused_fp64"]["ms"],
                                              out["per_gate_fp64"]["ms"])
    s128.close()
    # the same QFT as fused SIMT passes (complex64, 2^13-amplitude tiles)
    ssim = Q.State(n, Q.QSIM_C64)
    ssim.upload(x)
    sps = [Q.Plan(circ, dtype=Q.QSIM_C64, state=ssim)]
    sps[0].execute(ssim)
    sps.append(Q.Plan(circ, dtype=Q.QSIM_C64, state=ssim))
    sps[1].execute(ssim)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    Q.qsim_synchronize(ssim.h)
    torch.cuda.synchronize()
    a.record()
    for r in range(10):
        sps[r % 2].execute(ssim)
    z.record()
    Q.qsim_synchronize(ssim.h)
    torch.cuda.synchronize()
    ms = a.elapsed_time(z) / 10
    npp = sps[0].info()["passes"]
    out["qft27_c64_fused_simt"] = {"updates_per_s": ng * N / (ms * 1e-3), "ms": ms, "passes": npp,
                                   "kernel": "k_fused_pass", "hbm_gbs_per_pass": 2 * 8 * N / (ms / npp * 1e-3) / 1e9}
    ssim.close()
    # larger QFTs on tensor-core blocks (complex64, 8 GiB and 64 GiB kets,
    # basis-state input prepared on the device)
    for nn, mbk in ((30, 0), (30, 7), (33, 0)):
        key = f"qft{nn}_c64_tc_bf16x3" + ("_k7" if mbk else "")
        try:
            cc = Q.Circuit(nn, W.qft_circuit(nn))
            sb = Q.State(nn, Q.QSIM_C64)
            Q.qsim_set_basis(sb.h, 1)
            bps = [Q.Plan(cc, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=sb, max_block=mbk)]
            bps[0].execute(sb)
            bps.append(Q.Plan(cc, dtype=Q.QSIM_C64, prec=Q.QSIM_PREC_BF16X3, state=sb, max_block=mbk))
            bps[1].execute(sb)
            reps = 6 if nn == 30 else 2
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            Q.qsim_synchronize(sb.h)
            torch.cuda.synchronize()
            a.record()
            for r in range(reps):
                bps[r % 2].execute(sb)
            z.record()
            Q.qsim_synchronize(sb.h)
            torch.cuda.synchronize()
            ms = a.elapsed_time(z) / reps
            nb_ = bps[0].info()["passes"]
            nrm = C.c_double()
            Q.qsim_norm(sb.h, C.byref(nrm))
            ngg = len(cc.gates)
            out[key] = {
                "updates_per_s": ngg * (1 << nn) / (ms * 1e-3), "ms": ms, "blocks": nb_,
                "kernel": "k_tc_pipe7" if mbk else "k_tc_pipe",
                "hbm_gbs_per_block": 2 * 8 * (1 << nn) / (ms / nb_ * 1e-3) / 1e9,
                "ket_gib": 8 * (1 << nn) / 2 ** 30, "norm": nrm.value}
            sb.close()
            del bps
        except Exception as e:   # e.g. not enough device memory on a smaller part
            out[key] = {"error": str(e)[:200]}
    # the same QFT on tensor-core blocks (deferred phases as per-group
    # pre-diagonals), agreement with the fused SIMT result
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    sref = Q.State(n, Q.QSIM_C64)
    sref.upload(x)
    Q.Plan(circ, dtype=Q.QSIM_C64, state=sref).execute(sref)
    for prec, name, mbk in ((Q.QSIM_PREC_BF16X3, "bf16x3", 0), (Q.QSIM_PREC_BF16X3, "bf16x3_k7", 7),
                            (Q.QSIM_PREC_3XTF32, "3xtf32", 0)):
        stc = Q.State(n, Q.QSIM_C64)
        stc.upload(x)
        tp = Q.Plan(circ, dtype=Q.QSIM_C64, prec=prec, state=stc, max_block=mbk)
        tp.execute(stc)
        ip = (C.c_double * 2)()
        na, nb = C.c_double(), C.c_double()
        Q.qsim_inner_product(sref.h, stc.h, ip)
        Q.qsim_norm(sref.h, C.byref(na))
        Q.qsim_norm(stc.h, C.byref(nb))
        # timing: alternate the two layouts as in the main leg
        tps = [Q.Plan(circ, dtype=Q.QSIM_C64, prec=prec, state=stc, max_block=mbk)]
        tps[0].execute(stc)
        tps.append(Q.Plan(circ, dtype=Q.QSIM_C64, prec=prec, state=stc, max_block=mbk))
        tps[1].execute(stc)
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        Q.qsim_synchronize(stc.h)
        torch.cuda.synchronize()
        a.record()
        for r in range(6):
            tps[r % 2].execute(stc)
        z.record()
        Q.qsim_synchronize(stc.h)
        torch.cuda.synchronize()
        ms = a.elapsed_time(z) / 6
        nbk = tps[0].info()["passes"]
        achieved = 2 * 8 * N / (ms / nbk * 1e-3) / 1e9
        kn = {"bf16x3": "k_tc_pipe", "bf16x3_k7": "k_tc_pipe7", "3xtf32": "k_tc_pipe (3xTF32)"}[name]
        out[f"qft27_c64_tc_{name}"] = {"updates_per_s": ng * N / (ms * 1e-3), "ms": ms, "blocks": nbk,
                                       "kernel": kn, "hbm_gbs_per_block": achieved,
                                       "frac_of_hbm": achieved / peaks.get("hbm_gbs", 6800.0),
                                       "infidelity_vs_simt": 1.0 - (ip[0] ** 2 + ip[1] ** 2) / (na.value * nb.value)}
        stc.close()
    sref.close()
    # grid random circuit, 5x6, 10 layers, complex64 fused
    g = W.grid_rcs_circuit(5, 6, 10, seed=0)
    gc = Q.Circuit(30, g)
    gp = Q.Plan(gc, dtype=Q.QSIM_C64)
    sg = Q.State(30, Q.QSIM_C64)
    gp.execute(sg)
    Q.qsim_synchronize(sg.h)
    t0 = time.perf_counter()
    for _ in range(3):
        gp.execute(sg)
    Q.qsim_synchronize(sg.h)
    tg = (time.perf_counter() - t0) / 3
    gi = gp.info()
    out["grid30_c64_fused"] = {"updates_per_s": len(g) * (1 << 30) / tg, "ms": tg * 1e3, "passes": gi["passes"],
                               "hbm_gbs": gi["passes"] * 2 * 8 * (1 << 30) / tg / 1e9}
    # the same circuit on tensor-core blocks (BF16x3 and 3xTF32 splits)
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    for prec, name, mbk in ((Q.QSIM_PREC_BF16X3, "bf16x3", 0), (Q.QSIM_PREC_BF16X3, "bf16x3_k7", 7),
                            (Q.QSIM_PREC_3XTF32, "3xtf32", 0)):
        tp = Q.Plan(gc, dtype=Q.QSIM_C64, prec=prec, max_block=mbk)
        st2 = Q.State(30, Q.QSIM_C64)
        ms = time_plan(Q, C, tp, st2, 3)
        nb = tp.info()["passes"]
        achieved = 2 * 8 * (1 << 30) / (ms / nb * 1e-3) / 1e9
        # agreement with the SIMT result from |0...0> (both complex64)
        Q.qsim_set_basis(sg.h, 0)
        gp.execute(sg)
        Q.qsim_set_basis(st2.h, 0)
        tp.execute(st2)
        ip = (C.c_double * 2)()
        Q.qsim_inner_product(sg.h, st2.h, ip)
        na, nb2 = C.c_double(), C.c_double()
        Q.qsim_norm(sg.h, C.byref(na))
        Q.qsim_norm(st2.h, C.byref(nb2))
        out[f"grid30_c64_tc_{name}"] = {
            "updates_per_s": len(g) * (1 << 30) / (ms * 1e-3), "ms": ms, "blocks": nb,
            "kernel": {"bf16x3": "k_tc_pipe", "bf16x3_k7": "k_tc_pipe7", "3xtf32": "k_tc_pipe (3xTF32)"}[name],
            "hbm_gbs_per_block": achieved,
            "frac_of_hbm": achieved / peaks.get("hbm_gbs", 6800.0),
            "infidelity_vs_simt": 1.0 - (ip[0] ** 2 + ip[1] ** 2) / (na.value * nb2.value)}
        st2.close()
    sg.close()
    # the plain per-gate FP64 path on the grid circuit (one run)
    s128 = Q.State(30, Q.QSIM_C128)
    o = Q.qsim_run_opts(mode=0, relabel_swaps=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    Q.qsim_run_circuit(s128.h, gc.ptr(), C.byref(o))
    Q.qsim_synchronize(s128.h)
    pg = time.perf_counter() - t0
    out["grid30_per_gate_fp64"] = {"updates_per_s": len(g) * (1 << 30) / pg, "ms": pg * 1e3, "dtype": "c128"}
    best = min(out[k]["ms"] for k in out if k.startswith("grid30_c64"))
    out["grid30_speedup_vs_per_gate_fp64"] = pg * 1e3 / best
    out["grid30_c128_tc_bf16x6"] = c128_tc_leg(Q, C, torch, gc, None, 30, len(g), s128, peaks, None, pg * 1e3)
    s128.close()
    out["rows"] = rows_leg(Q, W, C, torch)
    out["batch512"] = batch_leg(Q, W, C)
    out["batch512_tc"] = batch_leg(Q, W, C, path=2)
    out["approx54_grid"] = approx_leg(Q, W, W.grid_rcs_circuit(6, 9, 7, seed=0), budget_gib=80.0)
    pf = W.paper_random_circuit(6, 9, 7, seed=0)
    out["approx54_paper_family"] = approx_leg(Q, W, pf, budget_gib=80.0)
    out["approx54_paper_family_full_hbm"] = approx_leg(Q, W, pf, budget_gib=240.0, p_start=0.45, time_cap_s=60.0)
    # the same sweep with the learned proposal schedule (MLP trained here on
    # exhaustive-mode traces of 20-qubit circuits of the same family)
    h, out["mlp_training"] = train_proposal_mlp(Q, W, C)
    out["mlp_gain_20_28_qubits"] = mlp_gain_leg(Q, W, h)
    out["approx54_paper_family_mlp"] = approx_leg(Q, W, pf, budget_gib=80.0, mlp=h)
    out["appendix_a_validation"] = appa_leg(Q, W, C, seeds=10, time_cap_s=60.0)
    out["qft54_zero_factorized"] = qft_zero_factorized_leg(Q, W)
    Q.qsim_mlp_destroy(h)
    return out


def rows_leg(Q, W, C, torch, n=27):
    """Each remaining hot-path row on its own, on a 27-qubit complex64 ket
    (1 GiB, larger than L2): device time per call with CUDA events (reductions
    include their host synchronisation), algorithmic bytes, GB/s and the
    fraction of the measured HBM peak; MLP inference / training latency."""
    peaks = {}
    pp = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pp):
        peaks = json.load(open(pp))
    peak = peaks.get("hbm_gbs", 6800.0)
    N = 1 << n
    B = 8
    st = Q.State(n, Q.QSIM_C64)
    Q.qsim_set_basis(st.h, 12345)
    other = Q.State(n, Q.QSIM_C64)
    Q.qsim_set_basis(other.h, 12345)
    h = np.ascontiguousarray(np.array([1, 0, 1, 0, 1, 0, -1, 0], dtype=np.float64) / np.sqrt(2))
    x = np.ascontiguousarray(np.array([0, 0, 1, 0, 1, 0, 0, 0], dtype=np.float64))
    fsim = np.zeros((4, 4), dtype=np.complex128)
    fsim[0, 0] = 1
    fsim[1, 2] = fsim[2, 1] = -1j
    fsim[3, 3] = np.exp(-1j * np.pi / 6)
    f2 = np.ascontiguousarray(fsim.ravel().view(np.float64))
    ctl = (C.c_int * 1)(5)
    r3 = (C.c_double * (3 * n))()
    ip = (C.c_double * 2)()
    d = C.c_double()

    def timed(fn, reps=10):
        fn()
        Q.qsim_synchronize(st.h)
        torch.cuda.synchronize()
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        z.record()
        Q.qsim_synchronize(st.h)
        torch.cuda.synchronize()
        return a.elapsed_time(z) / reps

    cases = [
        ("A2 1-qubit gate (H, qubit 20)", lambda: Q.qsim_apply_gate(st.h, h.ctypes.data_as(C.c_void_p), 20, None, 0, 0),
         2 * B * N),
        ("A2 controlled X (control 5, target 20)",
         lambda: Q.qsim_apply_gate(st.h, x.ctypes.data_as(C.c_void_p), 20, ctl, 1, 1), 2 * B * N // 2),
        ("A3 controlled phase (qubits 3, 22)", lambda: Q.qsim_apply_cphase(st.h, 3, 22, 0.3), 2 * B * N // 4),
        ("A4 dense 2-qubit fSim (qubits 7, 19)", lambda: Q.qsim_apply_2q(st.h, f2.ctypes.data_as(C.c_void_p), 7, 19),
         2 * B * N),
        ("A8 FP64 norm", lambda: Q.qsim_norm(st.h, C.byref(d)), B * N),
        ("A9 P(q = 1), qubit 11", lambda: Q.qsim_measure_prob(st.h, 11, C.byref(d)), B * N),
        ("A10 FP64 inner product", lambda: Q.qsim_inner_product(st.h, other.h, ip), 2 * B * N),
    ]
    out = {}
    for name, fn, by in cases:
        ms = timed(fn)
        out[name] = {"ms": ms, "bytes": by, "gbs": by / (ms * 1e-3) / 1e9, "frac_of_hbm": by / (ms * 1e-3) / 1e9 / peak}
    # A11: Bloch vectors of all 27 qubits (tiled passes over the ket)
    ms = timed(lambda: Q.qsim_bloch_all(st.h, r3), reps=3)
    by = 3 * B * N   # three tiled passes, one read of the ket each
    out["A11 Bloch vectors, all 27 qubits"] = {"ms": ms, "bytes": by, "gbs": by / (ms * 1e-3) / 1e9,
                                               "frac_of_hbm": by / (ms * 1e-3) / 1e9 / peak}
    st.close()
    other.close()
    # A19 / A20: proposal MLP (12 -> 64 -> 64 -> 1)
    hm = C.c_void_p()
    Q.qsim_mlp_create(12, 64, 1, C.byref(hm))
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    X = np.ascontiguousarray(np.random.default_rng(0).normal(size=(10000, 12)), dtype=np.float32)
    Y = np.ascontiguousarray((X[:, 0] > 0).astype(np.float32))
    lg = np.zeros(10000, dtype=np.float32)
    loss = C.c_float()
    t0 = time.perf_counter()
    for _ in range(50):
        Q.qsim_mlp_infer(hm, fp(X), 64, 1, fp(lg))
    out["A19 MLP inference, 64 candidates (BF16 weights), host call"] = {"us": (time.perf_counter() - t0) / 50 * 1e6}
    t0 = time.perf_counter()
    for _ in range(20):
        Q.qsim_mlp_train_step(hm, fp(X), fp(Y), 10000, C.c_float(3e-3), C.byref(loss))
    out["A20 MLP training step, 10000 rows (fwd + bwd + Adam), host call"] = {
        "ms": (time.perf_counter() - t0) / 20 * 1e3}
    Q.qsim_mlp_destroy(hm)
    return out


def batch_leg(Q, W, C, path=0):
    """512 seeded circuits (n ~ U{10..24}, depth ~ U{4..20}, QFT / grid 50/50)
    replayed from a CUDA graph: a persistent launch for the circuits on fused
    SIMT passes, grouped launches per block round for those on tensor-core
    blocks. path 0: per qubit count the autotuner's choice (tile width, or
    tensor cores; one representative circuit timed alone per qubit count);
    path 2: tensor cores for every circuit with n >= 13."""
    import tempfile
    specs = W.batch_circuits(512, seed=0)
    circs = [Q.Circuit(sp["n"], sp["gates"]) for sp in specs]
    with tempfile.TemporaryDirectory() as d:
        cache = os.path.join(d, "tune.jsonl")
        tuned = {}
        for sp, c in zip(specs, circs):
            if sp["n"] in tuned or sp["kind"] != "grid":
                continue
            best = Q.qsim_run_opts()
            sec = C.c_double()
            Q.qsim_autotune(c.ptr(), Q.QSIM_C64, cache.encode(), C.byref(best), C.byref(sec))
            tuned[sp["n"]] = "tc" if best.prec == Q.QSIM_PREC_BF16X3 else best.tile_qubits
        arr = (C.POINTER(Q.qsim_circuit) * len(circs))(*[C.pointer(c.c) for c in circs])
        o = Q.qsim_batch_opts(use_graph=1, path=path, tune_cache=cache.encode())
        h = C.c_void_p()
        Q.qsim_batch_create(C.cast(arr, C.c_void_p), len(circs), C.byref(o), C.byref(h))
    info = np.zeros(8, dtype=np.int64)
    Q.qsim_batch_info(h, info.ctypes.data_as(C.c_void_p))
    secs, lat = [], np.zeros(len(circs))
    for r in range(5):
        Q.qsim_batch_reset(h)
        sec = C.c_double()
        Q.qsim_batch_run(h, C.byref(sec), lat.ctypes.data_as(C.c_void_p))
        if r >= 2:
            secs.append(sec.value)
    Q.qsim_batch_destroy(h)
    t = float(np.median(secs))
    upd = sum(len(sp["gates"]) * (1 << sp["n"]) for sp in specs)
    return {"circuits": len(specs), "seconds": t, "circuits_per_s": len(specs) / t, "updates_per_s": upd / t,
            "latency_p50_ms": float(np.percentile(lat, 50)) * 1e3,
            "latency_p99_ms": float(np.percentile(lat, 99)) * 1e3, "work_items": int(info[1]),
            "ctas": int(info[2]), "arena_bytes": int(info[3]), "graph": bool(info[6]),
            "tensor_core_circuits": int(info[7]),
            "fastest_alone": {str(k): v for k, v in sorted(tuned.items())}}


def approx_leg(Q, W, g, budget_gib=80.0, time_cap_s=40.0, p_start=1.0, mlp=None):
    """The paper's Fig. 3 protocol on a 54-qubit, 7-layer circuit: p from
    p_start downward in steps of 0.025 until the memory budget is exceeded
    (or one run exceeds the time cap); F model of the last completed run.
    With mlp, the learned proposal schedule (top 4; exhaustive every 8
    entangling gates and on subsystems of 20 qubits or more) replaces the
    exhaustive checks."""
    runs = []
    p = p_start
    kw = {} if mlp is None else {"schedule": Q.QSIM_SCHED_MLP, "mlp": mlp, "top_m": 4, "fallback_every": 8,
                                 "exhaustive_from": 20}
    while p > -1e-9:
        try:
            r, _, _, _ = Q.approx_run(54, g, round(p, 3), budget=budget_gib * 2 ** 30, **kw)
        except Q.QsimError as e:
            runs.append({"p": round(p, 3), "status": "budget" if e.status == 5 else str(e)})
            break
        runs.append({"p": round(p, 3), "F": r.fidelity_model, "seconds": r.seconds, "rounds": r.n_rounds,
                     "peak_gib": r.peak_bytes / 2 ** 30, "max_subsystem_qubits": r.max_subsystem_qubits,
                     "bloch_passes": r.n_bloch_passes})
        if r.seconds > time_cap_s:
            break
        p -= 0.025
    done = [x for x in runs if "F" in x]
    return {"qubits": 54, "layers": 7, "budget_gib": budget_gib,
            "schedule": "exhaustive" if mlp is None else "mlp top-4; exhaustive every 8 gates and from 20 qubits",
            "min_p": done[-1]["p"] if done else None, "F_at_min_p": done[-1]["F"] if done else None,
            "seconds_total": sum(x["seconds"] for x in done),
            "bloch_passes_total": sum(x["bloch_passes"] for x in done), "runs": runs}


# App. A of the paper: RMSE of the fidelity model against the exact fidelity,
# per width x depth set (its Table II, 100 circuits per set there)
APPA_SETS = ((6, 6), (12, 6), (18, 6), (12, 12), (18, 12), (18, 18), (15, 15), (19, 10))
APPA_PAPER_RMSE = {(6, 6): 0.067, (12, 6): 0.054, (18, 6): 0.044, (12, 12): 0.039, (18, 12): 0.025,
                   (18, 18): 0.018, (15, 15): 0.024, (19, 10): 0.025}


def appa_leg(Q, W, C, seeds=3, time_cap_s=90.0):
    """For each set: `seeds` circuits of the paper's family (width w on a
    grid of ceil(sqrt(w)) columns), p = 0, 0.025, ..., 1; F model of the
    approximate run (complex128) against F_exact = |<psi_approx|psi_exact>|^2
    with psi_exact from the per-gate FP64 path. Seeds are added round-robin
    over the sets until the time cap."""
    t0 = time.perf_counter()
    res = {s: [] for s in APPA_SETS}
    ps = [round(0.025 * i, 3) for i in range(41)]
    for seed in range(seeds):
        for (w, d) in APPA_SETS:
            if time.perf_counter() - t0 > time_cap_s:
                break
            rows, cols = W.grid_shape(w)
            g = W.paper_random_circuit(rows, cols, d, seed=1000 * w + d * 10 + seed, n=w)
            se = Q.State(w, Q.QSIM_C128)
            se.run(Q.Circuit(w, g), mode=Q.QSIM_MODE_PER_GATE)
            ex = se.download()
            se.close()
            for p in ps:
                r, st, _, _ = Q.approx_run(w, g, p, dtype=Q.QSIM_C128, want_state=True)
                fe = abs(np.vdot(st, ex)) ** 2 / (np.vdot(st, st).real * np.vdot(ex, ex).real)
                res[(w, d)].append((r.fidelity_model, float(fe)))
    out = {"sets": [], "p_grid": "0..1 step 0.025", "dtype": "c128", "seconds": time.perf_counter() - t0}
    allr = []
    for (w, d), obs in res.items():
        if not obs:
            continue
        r2 = [(a - b) ** 2 for a, b in obs]
        allr += r2
        out["sets"].append({"width": w, "depth": d, "circuits": len(obs) // len(ps), "observations": len(obs),
                            "rmse": float(np.sqrt(np.mean(r2))), "mean_F": float(np.mean([a for a, _ in obs])),
                            "mean_F_exact": float(np.mean([b for _, b in obs])),
                            "paper_rmse_100_circuits": APPA_PAPER_RMSE[(w, d)]})
    out["observations"] = len(allr)
    out["rmse_overall"] = float(np.sqrt(np.mean(allr))) if allr else None
    out["paper_rmse_overall"] = 0.039
    return out


def qft_zero_factorized_leg(Q, W, n=54):
    """QFT of |0...0> on 54 qubits through the approximate mode with p = 0
    (exact separation only): the ket stays factorised (2-qubit subsystems at
    most), where a state vector would take 2^54 x 16 bytes. Also with the
    unobservable optimisation (Sec. II.B): every controlled phase meets a
    qubit in |0> and is removed, so nothing is ever composed."""
    out = {}
    for unobs in (0, 1):
        r, _, _, _ = Q.approx_run(n, W.qft_circuit(n), 0.0, dtype=Q.QSIM_C128, tau=1e-13, unobservable=unobs)
        out["unobservable_on" if unobs else "unobservable_off"] = {
            "seconds": r.seconds, "F": r.fidelity_model, "rounds": r.n_rounds, "exact_separations": r.n_exact,
            "checks": r.n_checks, "gates_removed_or_reduced": r.n_unobservable,
            "max_subsystem_qubits": r.max_subsystem_qubits, "peak_bytes": r.peak_bytes}
    return {"qubits": n, "gates": len(W.qft_circuit(n)), "state_vector_bytes": 16 * 2 ** n, **out}


def run_appendix_a():
    """The paper's App. A protocol in full: 100 circuits per width x depth
    set, 41 values of p each (32,800 observations); one JSON line."""
    import ctypes as C
    from paper_2304_14969_gb300 import build, qsim as Q
    from paper_2304_14969_gb300 import workloads as W
    build.build()
    Q.lib()
    print(json.dumps({"workload": "appendix_a_validation", **appa_leg(Q, W, C, seeds=100, time_cap_s=1e9)}))


def train_proposal_mlp(Q, W, C):
    """Proposal MLP (12 -> 64 -> 64 -> 1) trained on the GPU on traces of the
    exhaustive approximate mode: paper-family circuits (U3 + C/A Pauli) on
    4x5, 4x6, 5x5 and 4x7 grids (20 to 28 qubits), 7 layers, p from 0.3 to
    0.7. Returns (handle, training summary)."""
    X, Y = [], []
    t0 = time.perf_counter()
    shapes = ((4, 5), (4, 6), (5, 5), (4, 7))
    for si, (rows, cols) in enumerate(shapes):
        for seed in range(3 if rows * cols < 28 else 2):
            g = W.paper_random_circuit(rows, cols, 7, seed=200 + 10 * si + seed)
            for p in (0.3, 0.4, 0.5, 0.6, 0.7):
                _, _, (f, l), _ = Q.approx_run(rows * cols, g, p, trace_cap=20000)
                X.append(f)
                Y.append(l)
    t_traces = time.perf_counter() - t0
    X = np.ascontiguousarray(np.concatenate(X), dtype=np.float32)
    Y = np.ascontiguousarray(np.concatenate(Y), dtype=np.float32)
    h = C.c_void_p()
    Q.qsim_mlp_create(12, 64, 7, C.byref(h))
    loss = C.c_float()
    fp = lambda a: a.ctypes.data_as(C.POINTER(C.c_float))
    t0 = time.perf_counter()
    first = None
    for _ in range(400):
        Q.qsim_mlp_train_step(h, fp(X), fp(Y), len(X), C.c_float(3e-3), C.byref(loss))
        first = loss.value if first is None else first
    t_train = time.perf_counter() - t0
    return h, {"qubits": [r * c for r, c in shapes], "trace_rows": int(len(X)), "positive_fraction": float(Y.mean()),
               "traces_seconds": t_traces, "train_steps": 400, "train_seconds": t_train, "loss_first": first,
               "loss_last": loss.value}


def mlp_gain_leg(Q, W, h):
    """The learned schedule against the exhaustive one on held-out
    paper-family circuits of 20, 24 and 28 qubits (7 layers), at equal p:
    wall time, Bloch reductions, roundings and F model of each (summed over
    the circuits). An MLP round scores, selects and checks on the device
    with one host synchronisation, as an exhaustive round does, and skips
    the Bloch reductions when nothing is proposed."""
    out = []
    for rows, cols in ((4, 5), (4, 6), (4, 7)):
        n = rows * cols
        gs = [W.paper_random_circuit(rows, cols, 7, seed=900 + s) for s in range(2)]
        for p in (0.2, 0.4, 0.6):
            row = {"qubits": n, "p": p}
            for name, kw in (("exhaustive", {}), ("mlp", {"schedule": Q.QSIM_SCHED_MLP, "mlp": h, "top_m": 4,
                                                          "fallback_every": 8})):
                sec = passes = rounds = 0
                logF = 0.0
                for g in gs:
                    r, _, _, _ = Q.approx_run(n, g, p, **kw)
                    sec += r.seconds
                    passes += r.n_bloch_passes
                    rounds += r.n_rounds
                    logF += float(np.log(max(r.fidelity_model, 1e-300)))
                row[name] = {"seconds": sec, "bloch_passes": passes, "rounds": rounds,
                             "F_geomean": float(np.exp(logF / len(gs)))}
            row["wall_time_gain"] = row["exhaustive"]["seconds"] / max(row["mlp"]["seconds"], 1e-12)
            out.append(row)
    return out


if __name__ == "__main__":
    main()
