#!/usr/bin/env python
"""Benchmark of the state-vector gate engine on the 30-qubit complex128 workload.

One step is one pass of the whole hot path over one batch of synthetic input:
  P1  single-gate sweep, plain per-gate path: H(t), RZ(t), CNOT(24, t) and a
      Haar U4 on (t, t+1 mod 30) for t = 0..29 (120 gates) applied to a seeded
      Gaussian 30-qubit state (restored from a device copy at the start of
      the step);
  P2  a 10-layer RY/RZ + CNOT-ladder ansatz from |0..0> on the fused tile path
      (890 gates), then <TFIM> = <sum Z_i Z_i+1 + 0.5 sum X_i>;
  P3  the 30-qubit QFT of a seeded basis state on the fused path (480 gates).
Metric: gates/s (1490 gates per step) with the step's algorithmic HBM GB/s.
The same line carries the metric's other two parts: the step run again in
complex64 (its gates/s, and its energy and states against complex128's), and
the adjoint gradient's time over one forward pass on the 24-qubit, 8-layer,
384-parameter TFIM circuit in both precisions, with a central-difference check.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload (one sweep gate per step) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

METRIC = "gates/s & HBM GB/s at 30q c128 vs 8 TB/s; adjoint/forward time; c64 vs c128"
UNIT = "gates/s"
N_QUBITS = 30
WORKLOAD = ("30-qubit complex128 state (16 GiB): P1 single-gate sweep H/RZ/CNOT(24,t)/U4(t,t+1) over t=0..29 on a "
            "seeded Gaussian state (plain path, 120 gates); P2 10-layer RY+RZ+CNOT-ladder ansatz from |0> (fused, "
            "890 gates) + TFIM expectation; P3 30-qubit QFT of a seeded basis state (fused, 480 gates)")


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# ranks: one process per GPU, independent replicas
# ---------------------------------------------------------------------------
class Ranks:
    """The processes of a torchrun launch (RANK / WORLD_SIZE / LOCAL_RANK).
    The path does not shard: each rank runs a full replica, and ranks share
    only a barrier around the timed region and the slowest rank's time."""

    def __init__(self, backend: str):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        if self.world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self) -> None:
        if self.dist is not None:
            self.dist.barrier()

    def max(self, x: float, device: str) -> float:
        """The largest x over all ranks."""
        if self.dist is None:
            return float(x)
        import torch
        t = torch.tensor([float(x)], device=device, dtype=torch.float64)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self) -> None:
        if self.dist is not None:
            self.dist.destroy_process_group()
            self.dist = None


def replicas_value(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of `world` replicas that each processed
    `units_per_rank` units, timed by the slowest rank."""
    return units_per_rank * world / seconds


# ---------------------------------------------------------------------------
# the workload
# ---------------------------------------------------------------------------
class Workload:
    def __init__(self, n: int, psi_host, dtype: str = "c128"):
        import torch

        import paper_2508_13615_gb300 as L
        self.L = L
        self.n = n
        self.dtype = dtype
        self.sweep = W.sweep_30q(n)
        self.ansatz = W.ansatz(n, 10, 3)
        self.qft = W.qft(n)
        self.x = W.basis_index(n, 4)
        self.tfim = W.tfim(n)
        self.ans_ops = L.OpArray(self.ansatz.ops)
        self.qft_ops = L.OpArray(self.qft.ops)
        self.terms = L.PauliArray(self.tfim)
        self.sweep_calls = []
        for _, c in self.sweep:
            op = c.ops[0]
            p = op.matrix if op.name in ("U2", "U4") else (c.params if len(c.params) else ())
            self.sweep_calls.append((op.name, op.wires, p))
        self.gates = len(self.sweep) + len(self.ansatz.ops) + len(self.qft.ops)
        self.sv = L.StateVector(n, dtype)
        self.saved = torch.empty_like(self.sv.tensor)
        self.psi_host = psi_host
        L.lqs_sv_copy_from_host(self.sv.h, psi_host)
        self.saved.copy_(self.sv.tensor)
        torch.cuda.synchronize()
        self.energy = None

    def precompile(self, arith) -> int:
        """Compiles the fused segments and Pauli passes of P2 and P3 (host only)."""
        L = self.L
        k = sum(L.lqs_jit_precompile(self.n, self.dtype, c.ops, c.params, arith) for c in (self.ansatz, self.qft))
        return k + L.lqs_jit_precompile_expval(self.n, self.dtype, self.tfim, False, arith)

    def close(self) -> None:
        self.sv.close()
        self.saved = None

    def input_bytes(self) -> int:
        b = self.psi_host.nbytes
        b += sum(np.asarray(p).nbytes for _, _, p in self.sweep_calls if len(p))
        b += self.ansatz.params.nbytes + self.qft.params.nbytes
        return b

    def p1(self, h=None):
        L = self.L
        h = self.sv.h if h is None else h
        for name, wires, p in self.sweep_calls:
            L.lqs_apply_gate(h, name, wires, p)

    def p2p3(self, h=None):
        L = self.L
        h = self.sv.h if h is None else h
        L.lqs_sv_set_basis(h, 0)
        L.lqs_apply_fused(h, self.ans_ops, self.ansatz.params, None)
        self.energy, _ = L.lqs_expval(h, self.terms)
        L.lqs_sv_set_basis(h, self.x)
        L.lqs_apply_fused(h, self.qft_ops, self.qft.params, None)

    def step(self):
        self.sv.tensor.copy_(self.saved)
        self.p1()
        self.p2p3()


class E2EPipeline:
    """The step end to end through the C ABI with host buffers.

    Every step copies its input state from pinned host memory, runs P1 on it
    and reads P1's output state back into pinned host memory, then runs P2
    (the energy is read back to the host by lqs_expval) and P3 on a second
    state and reads P3's output state back as well.  Uploads and read-backs
    run on streams of their own into alternating device buffers, so step
    i+1's upload and step i's read-backs overlap step i's compute; all of
    their bytes still cross inside the timed region (the first upload and the
    last read-back are fully exposed)."""

    def __init__(self, wl: Workload, out_p1, out_p3):
        import torch
        L = wl.L
        self.wl, self.out_p1, self.out_p3 = wl, out_p1, out_p3
        self.sc, self.sh, self.sd = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        self.buf = [torch.empty_like(wl.sv.tensor) for _ in range(2)]
        self.wbuf = [torch.empty_like(wl.sv.tensor) for _ in range(2)]
        # one library handle per (buffer, stream) it is used on
        self.comp = [L.StateVector(wl.n, wl.dtype, tensor=b, stream=self.sc) for b in self.buf]
        self.up = [L.StateVector(wl.n, wl.dtype, tensor=b, stream=self.sh) for b in self.buf]
        self.down = [L.StateVector(wl.n, wl.dtype, tensor=b, stream=self.sd) for b in self.buf]
        self.work = [L.StateVector(wl.n, wl.dtype, tensor=b, stream=self.sc) for b in self.wbuf]
        self.work_down = [L.StateVector(wl.n, wl.dtype, tensor=b, stream=self.sd) for b in self.wbuf]
        torch.cuda.synchronize()

    def d2h_bytes_per_step(self) -> int:
        return int(self.out_p1.nbytes) + int(self.out_p3.nbytes) + 8  # two states and the energy

    def run(self, steps: int) -> None:
        import torch
        L, wl = self.wl.L, self.wl
        up = [torch.cuda.Event() for _ in range(steps)]
        p1 = [torch.cuda.Event() for _ in range(steps)]
        p3 = [torch.cuda.Event() for _ in range(steps)]
        down = [torch.cuda.Event() for _ in range(steps)]
        down3 = [torch.cuda.Event() for _ in range(steps)]

        def upload(i):
            if i >= 2:  # the buffer is free once step i-2's read-back is done
                self.sh.wait_event(down[i - 2])
            L.lqs_sv_copy_from_host(self.up[i % 2].h, wl.psi_host)
            up[i].record(self.sh)

        upload(0)
        for i in range(steps):
            if i + 1 < steps:
                upload(i + 1)
            self.sc.wait_event(up[i])
            wl.p1(self.comp[i % 2].h)
            p1[i].record(self.sc)
            self.sd.wait_event(p1[i])
            L.lqs_sv_copy_to_host_async(self.down[i % 2].h, self.out_p1)
            down[i].record(self.sd)
            if i >= 2:  # the work buffer is free once step i-2's P3 read-back is done
                self.sc.wait_event(down3[i - 2])
            wl.p2p3(self.work[i % 2].h)
            p3[i].record(self.sc)
            self.sd.wait_event(p3[i])
            L.lqs_sv_copy_to_host_async(self.work_down[i % 2].h, self.out_p3)
            down3[i].record(self.sd)
        for s in (self.sc, self.sh, self.sd):
            s.synchronize()

    def close(self) -> None:
        for sv in self.comp + self.up + self.down + self.work + self.work_down:
            sv.close()
        self.buf = self.wbuf = None


# A secondary, derived arithmetic figure for the double-float kernels (it is
# not a chip peak): 152 SMs x 128 FP32 lanes x 2.07 GHz = 40.3 T FP32
# instructions/s, divided by the FP32 instructions this code's double-float
# complex128 gate math spends per float64-equivalent flop.  A real 2x2 update
# costs 32 FP32 instructions per amplitude (6 flops): each of the two real
# outputs is two products with their exact error terms (8), one TwoSum (6)
# and two error additions.  That is 5.33 instructions per flop, so the
# derived figure is 40.3 / 5.33 = 7.6 TFLOP/s float64-equivalent.  Native
# complex64 math is 2 flops per FMA lane-cycle.
FP32_INSTR_PEAK = 152 * 128 * 2.07e9
DF_INSTR_PER_FLOP = 32.0 / 6.0
ALU_PEAK_TFLOPS = {"df": FP32_INSTR_PEAK / DF_INSTR_PER_FLOP / 1e12, "f32": 2 * FP32_INSTR_PEAK / 1e12,
                   "f64": 1.25}


def sources_digest(paths) -> str:
    """sha256 (first 16 hex digits) of the listed repository files, in order.
    A traffic figure from an ncu capture is valid only while the sources of
    the captured kernel are the ones it was taken from."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(p.encode() + b"\0" + f.read())
    return h.hexdigest()[:16]


# The sources that make each captured kernel family (the kernel, the headers
# it includes and the host code that plans and launches it).
SEG_SOURCES = ("paper_2508_13615_gb300/csrc/jit.cu", "paper_2508_13615_gb300/csrc/jit_dev.cuh",
               "paper_2508_13615_gb300/csrc/tile.cuh", "paper_2508_13615_gb300/csrc/arith.cuh",
               "paper_2508_13615_gb300/csrc/fused_reg.cu")
BLOCK_SOURCES = ("paper_2508_13615_gb300/csrc/block_tc.cu", "paper_2508_13615_gb300/csrc/tile.cuh")
DENSE_SOURCES = ("paper_2508_13615_gb300/csrc/gate_kernels.cu", "paper_2508_13615_gb300/csrc/arith.cuh",
                 "paper_2508_13615_gb300/csrc/gates.cu")

# DRAM read + write per launch of each captured kernel family, from one ncu
# capture on a smaller state, scaled to a launch at the benchmark's size by the
# units processed (the state size: a pass moves every amplitude once).  Each
# entry names the profile summary it comes from and the digest of the sources
# at capture time; `traffic` is null whenever the sources have changed since.
TRAFFIC = {
    "k_fused_reg_jit/df": {"read": 268.581632e6, "write": 207.311360e6, "capture_qubits": 24,
                           "source": "profiles/compiled_segment_ansatz_24q_c128.md",
                           "files": SEG_SOURCES, "sha": "532d9ed60565e781"},
    "k_block_tc": {"read": 537.046528e6, "write": 475.009792e6, "capture_qubits": 26,
                   "source": "profiles/k_block_tc_tf32x3_26q_c64.md", "files": BLOCK_SOURCES, "sha": "38c07247c2d88ac4"},
}


def traffic_of(name: str, n: int):
    """(bytes per launch at n qubits or None, details) for a kernel family."""
    t = TRAFFIC.get(name)
    if t is None:
        return None, {}
    scaled = (t["read"] + t["write"]) * float(1 << (n - t["capture_qubits"]))
    now = sources_digest(t["files"])
    info = {"traffic_source": f"{t['source']} ({t['capture_qubits']} q capture x 2^({n}-{t['capture_qubits']}))",
            "traffic_sources_sha": now}
    if t["sha"] != now:
        info["traffic_last_capture"] = scaled
        info["traffic_note"] = ("the kernel's sources changed after the capture (digest "
                                f"{t['sha']} at capture, {now} now): retake it")
        return None, info
    return scaled, info


def roofline(records, pk, n):
    """The dominant kernel family (by device time) against the measured HBM
    copy peak: achieved = its algorithmic bytes per launch / its average
    launch time.  The double-float arithmetic figure derived from this code's
    own instruction count is reported beside it under `alu_derived`."""
    fam = {}
    for name, ms, b, f in records:
        d = fam.setdefault(name, [0, 0.0, 0.0, 0.0])
        d[0] += 1
        d[1] += ms
        d[2] += b
        d[3] += f
    total = sum(d[1] for d in fam.values()) or 1.0
    name, (cnt, ms, b, f) = max(fam.items(), key=lambda kv: kv[1][1])
    hbm = float(pk.get("hbm_gbs", 6800.0))
    gbs = b / (ms * 1e-3) / 1e9
    tfl = f / (ms * 1e-3) / 1e12
    arith = name.split("/")[-1] if "/" in name else "f32"
    alu_peak = ALU_PEAK_TFLOPS.get(arith, ALU_PEAK_TFLOPS["f32"])
    traffic, tinfo = traffic_of(name, n)
    out = {"kernel": name, "bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm,
           "peak_source": ("MEASURED_PEAKS.json hbm_gbs (measured copy); frac is of measured" if "hbm_gbs" in pk
                           else "fallback 6.8 TB/s; frac is of fallback"),
           "traffic": traffic, **tinfo,
           "launches": cnt, "share": ms / total, "bytes_per_launch": b / cnt, "ms_per_launch": ms / cnt,
           "frac_of_nominal_8TBps": gbs / 8000.0,
           "alu_derived": {
               "achieved_f64eq_tflops": tfl, "figure_tflops": alu_peak, "frac": tfl / alu_peak,
               "basis": (f"derived from this code's own instruction count, not a chip peak: 152 SMs x 128 FP32 "
                         f"lanes x 2.07 GHz / {DF_INSTR_PER_FLOP:.2f} FP32 instructions per float64-equivalent "
                         f"flop of its double-float arithmetic; flops are the gates' algorithmic flops")
               if arith == "df" else "derived from unit counts and clocks"}}
    fams = {k: {"launches": v[0], "ms": round(v[1], 3), "share": round(v[1] / total, 4),
                "GBps": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] else None} for k, v in fam.items()}
    return out, fams


def cpu_baseline_sample(psi_host, sweep_calls_circ, budget_s=15.0):
    """The oracle as it stands, on the host cores, applying sweep gates in place
    to the 30-qubit host state until about `budget_s` seconds of work."""
    import oracle
    th = oracle.max_threads()
    done, t0 = 0, time.perf_counter()
    n = int(psi_host.size).bit_length() - 1
    while True:
        _, c = sweep_calls_circ[done % len(sweep_calls_circ)]
        oracle.apply_op(psi_host, n, c.ops[0], c.params)
        done += 1
        if time.perf_counter() - t0 >= budget_s:
            break
    dt = time.perf_counter() - t0
    # the same oracle on one thread: one sweep gate
    oracle.set_threads(1)
    try:
        _, c = sweep_calls_circ[done % len(sweep_calls_circ)]
        t1 = time.perf_counter()
        oracle.apply_op(psi_host, n, c.ops[0], c.params)
        dt1 = time.perf_counter() - t1
    finally:
        oracle.set_threads(th)
    return {"value": done / dt, "unit": UNIT, "cores": th, "kind": "oracle",
            "sample": f"{done} gates of the P1 sweep applied in place to the 30-qubit complex128 state by the CPU "
                      f"oracle (general matrix update, OpenMP {th} threads), {dt:.1f} s",
            "one_thread": {"value": 1.0 / dt1, "unit": UNIT,
                           "sample": f"one P1 sweep gate ({c.ops[0].name}) by the same oracle on one thread, "
                                     f"{dt1:.1f} s"}}


def host_state(n: int, pinned: bool):
    import torch
    if pinned:
        t = torch.empty(1 << n, dtype=torch.complex128, pin_memory=True)
        a = t.numpy()
    else:
        t = None
        a = np.empty(1 << n, dtype=np.complex128)
    W.gaussian_state(n, 2, out=a)
    return t, a


def run_reference(args):
    """--impl reference: the CPU oracle on the same workload, one sweep gate per step."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    n = args.n
    _, psi = host_state(n, pinned=False)
    sweep = W.sweep_30q(n)
    th = oracle.max_threads()
    for i in range(args.warmup):
        _, c = sweep[i % len(sweep)]
        oracle.apply_op(psi, n, c.ops[0], c.params)
    t0 = time.perf_counter()
    for i in range(args.steps):
        _, c = sweep[(args.warmup + i) % len(sweep)]
        oracle.apply_op(psi, n, c.ops[0], c.params)
    dt = time.perf_counter() - t0
    v = args.steps / dt
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD + "; reference arm: the CPU oracle applies one P1 sweep gate per step",
                   "n_qubits": n,
                   "units": ("this arm counts single P1 sweep gates (H, RZ, CNOT(24,t), U4 on the 30-qubit state, "
                             "one gate per step, general matrix update); the GPU arm counts all 1490 gates of its "
                             "step (120 plain P1 gates, 890 fused P2 gates, 480 fused P3 gates), so the two arms "
                             "do not time the same gate mix")},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": th, "kind": "oracle",
                         "sample": f"{args.steps} P1 sweep gates on the {n}-qubit state"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)


# ---------------------------------------------------------------------------
# secondary configurations (one JSON line each; not part of the default run)
# ---------------------------------------------------------------------------
def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def adjoint_leg(steps: int, warmup: int, n: int = 24, layers: int = 8):
    """24 qubits, 8-layer ansatz (384 parameters), TFIM: adjoint gradient time
    over forward time (fused forward + expectation), complex128 and complex64,
    each timed with CUDA events on the launching stream (median of the timed
    repetitions); central differences (h = 1e-6) on a sample of parameters
    (complex128), and the complex64 gradient against the complex128 one."""
    import torch
    import paper_2508_13615_gb300 as L
    c = W.ansatz(n, layers, 6)
    terms = W.tfim(n)
    ops = L.OpArray(c.ops)
    pa = L.PauliArray(terms)
    out = {"n_qubits": n, "layers": layers, "params": c.n_params, "observable": "TFIM sum Z_iZ_i+1 + 0.5 sum X_i",
           "forward": "fused ansatz (compiled segments) + expectation (compiled Pauli passes)",
           "adjoint": "lambda = H psi + compiled reverse sweep (psi and lambda in registers)",
           "timing": "CUDA events on the launching stream, median"}
    old = L.lqs_jit_info()["mode"]
    L.lqs_set_jit(L.LQS_JIT_ON)
    g128 = None
    try:
        for dtype in ("c128", "c64"):
            ar = L.LQS_ARITH_DF if dtype == "c128" else L.LQS_ARITH_AUTO
            t_jit = time.perf_counter()
            L.lqs_jit_precompile(n, dtype, c.ops, c.params, ar)
            L.lqs_jit_precompile_adjoint(n, dtype, c.ops, c.params, ar)
            L.lqs_jit_precompile_expval(n, dtype, terms, False, ar)
            L.lqs_jit_precompile_expval(n, dtype, terms, True, ar)
            jit_s = time.perf_counter() - t_jit
            sv = L.StateVector(n, dtype)
            st = torch.cuda.current_stream()

            def fwd():
                L.lqs_sv_set_basis(sv.h, 0)
                L.lqs_apply_fused(sv.h, ops, c.params, None)
                return L.lqs_expval(sv.h, pa)[0]

            for _ in range(warmup):
                fwd()
                L.lqs_adjoint_grad(sv.h, ops, c.params, pa)
            tf, ta = [], []
            for _ in range(max(steps, 3)):
                e0, e1 = _events()
                e0.record(st)
                fwd()
                e1.record(st)
                torch.cuda.synchronize()
                tf.append(e0.elapsed_time(e1))
                e0.record(st)
                g, e = L.lqs_adjoint_grad(sv.h, ops, c.params, pa)
                e1.record(st)
                torch.cuda.synchronize()
                ta.append(e0.elapsed_time(e1))
            # device time per kernel family of one forward and one adjoint call
            parts = {}
            for key, fn in (("forward", fwd), ("adjoint", lambda: L.lqs_adjoint_grad(sv.h, ops, c.params, pa))):
                if key == "adjoint":
                    fwd()
                L.lqs_profile_start()
                fn()
                fam = {}
                for name, ms, _, _ in L.lqs_profile_stop():
                    fam[name] = round(fam.get(name, 0.0) + ms, 3)
                parts[key] = fam
            rec = {"forward_ms": statistics.median(tf), "adjoint_ms": statistics.median(ta),
                   "adjoint_over_forward": statistics.median(ta) / statistics.median(tf), "energy": e,
                   "kernel_ms": parts, "compile_wall_s": round(jit_s, 2)}
            if dtype == "c128":
                h = 1e-6
                fd = []
                for k in (0, 7, 100, 383 % c.n_params):
                    vals = []
                    for sgn in (1, -1):
                        p = c.params.copy()
                        p[k] += sgn * h
                        L.lqs_sv_set_basis(sv.h, 0)
                        L.lqs_apply_fused(sv.h, ops, p, None)
                        vals.append(L.lqs_expval(sv.h, pa)[0])
                    fd.append(abs((vals[0] - vals[1]) / (2 * h) - g[k]))
                rec["fd_params_checked"] = [0, 7, 100, 383 % c.n_params]
                rec["max_abs_adjoint_minus_fd"] = max(fd)
                g128 = g
            else:
                rec["max_abs_grad_c64_minus_c128"] = float(np.max(np.abs(g - g128)))
            out[dtype] = rec
            sv.close()
    finally:
        L.lqs_set_jit(old)
    return out


def config_adjoint24(args):
    """The adjoint/forward measurement alone (it is also part of the default line)."""
    rec = adjoint_leg(args.steps, args.warmup)
    rec["config"] = "adjoint24"
    rec["metric"] = "adjoint/forward time"
    print(json.dumps(rec), flush=True)


def config_precision32(args):
    """32 qubits, 20-layer ansatz: complex64 (32 GiB) vs complex128 (64 GiB) on the
    fused path; <sum Z_i Z_i+1> in float64 for both, and the complex64 state's
    relative L2 distance from the complex128 one."""
    import torch
    import paper_2508_13615_gb300 as L
    n = args.n if args.n != N_QUBITS else 32
    c = W.ansatz(n, 20, 5)
    terms = W.zz_chain(n)
    ops = L.OpArray(c.ops)
    res = {"config": "precision32", "n_qubits": n, "layers": 20, "gates": len(c.ops),
           "timing": "second application (the segment kernels are compiled before the first), CUDA events"}
    svs = {}
    L.lqs_set_jit(L.LQS_JIT_ON)
    for dtype in ("c128", "c64"):
        L.lqs_jit_precompile(n, dtype, c.ops, c.params, L.LQS_ARITH_DF if dtype == "c128" else L.LQS_ARITH_AUTO)
        sv = L.StateVector(n, dtype)
        st = torch.cuda.current_stream()
        L.lqs_sv_set_basis(sv.h, 0)
        L.lqs_apply_fused(sv.h, ops, c.params, None)
        e0, e1 = _events()
        e0.record(st)
        L.lqs_sv_set_basis(sv.h, 0)
        L.lqs_apply_fused(sv.h, ops, c.params, None)
        e1.record(st)
        torch.cuda.synchronize()
        e, _ = L.lqs_expval(sv.h, terms)
        res[dtype] = {"forward_ms": e0.elapsed_time(e1), "energy_zz": e,
                      "passes": L.lqs_plan_fused(n, dtype, c.ops)[0]}
        svs[dtype] = sv
    d2, nb = L.lqs_sv_distance(svs["c64"].h, svs["c128"].h)
    res["abs_energy_c64_minus_c128"] = abs(res["c64"]["energy_zz"] - res["c128"]["energy_zz"])
    res["rel_l2_c64_vs_c128"] = math.sqrt(d2 / nb)
    for sv in svs.values():
        sv.close()
    print(json.dumps(res), flush=True)


def config_batch256(args):
    """256 circuits, n ~ U{10..20}, 4..12 ansatz layers, TFIM, complex64: one
    persistent launch (forward + energy + adjoint gradients) against a loop
    that runs the circuits one at a time through the same library."""
    import torch
    import paper_2508_13615_gb300 as L
    circs = W.batch_circuits(256, 7)
    terms = [W.tfim(c.n_qubits) for c in circs]
    # arguments marshalled once, as the loop below does for its calls
    t_m = time.perf_counter()
    B = L.BatchItems(circs, terms)
    marshal_s = time.perf_counter() - t_m
    t_first = time.perf_counter()
    B.run("c64")  # first call: plans built and cached, buffers grown
    first_s = time.perf_counter() - t_first
    t_tune = time.perf_counter()
    tuned = B.autotune("c64", repeats=1)  # tile shape per qubit count
    tune_s = time.perf_counter() - t_tune
    for _ in range(2):
        B.run("c64")
    torch.cuda.synchronize()
    tb = []
    for _ in range(max(args.steps, 3)):
        t0 = time.perf_counter()
        B.run("c64")
        tb.append(time.perf_counter() - t0)
    # device time of the batch's kernels in one call (the rest of the call is host work)
    L.lqs_profile_start()
    t0 = time.perf_counter()
    B.run("c64")
    prof_wall = time.perf_counter() - t0
    kern = {}
    for name, ms, _, _ in L.lqs_profile_stop():
        kern[name] = round(kern.get(name, 0.0) + ms, 3)
    # new parameters, same structures (the next step of a variational loop): written in place
    for c, p in zip(circs, B.params):
        c.params = (c.params + 0.1) % (2 * np.pi)
        p[:] = c.params
    t0 = time.perf_counter()
    e, g = B.run("c64")
    new_params_s = time.perf_counter() - t0
    e, g = np.array(e), [np.array(x) for x in g]

    # the loop baseline: same library, one circuit at a time, with its
    # arguments marshalled once and one state per qubit count reused
    ops = [L.OpArray(c.ops) for c in circs]
    pas = [L.PauliArray(t) for t in terms]
    svs = {n: L.StateVector(n, "c64") for n in sorted({c.n_qubits for c in circs})}

    def loop():
        es, gs = [], []
        for c, oa, pa in zip(circs, ops, pas):
            h = svs[c.n_qubits].h
            L.lqs_sv_set_basis(h, 0)
            L.lqs_apply_fused(h, oa, c.params, None)
            gg, ee = L.lqs_adjoint_grad(h, oa, c.params, pa)
            es.append(ee)
            gs.append(gg)
        return es, gs

    loop()
    loop()  # structures used twice: the segment compiler's automatic mode has compiled them now
    torch.cuda.synchronize()
    jit0 = L.lqs_jit_info()
    tl = []
    for _ in range(2):
        t0 = time.perf_counter()
        el, gl = loop()
        tl.append(time.perf_counter() - t0)
    jit1 = L.lqs_jit_info()
    # per qubit count: one pass of the loop over that count's circuits
    per_n = {}
    for nq in sorted({c.n_qubits for c in circs}):
        idx = [i for i, c in enumerate(circs) if c.n_qubits == nq]
        t0 = time.perf_counter()
        for i in idx:
            h = svs[nq].h
            L.lqs_sv_set_basis(h, 0)
            L.lqs_apply_fused(h, ops[i], circs[i].params, None)
            L.lqs_adjoint_grad(h, ops[i], circs[i].params, pas[i])
        per_n[nq] = round(time.perf_counter() - t0, 4)
    err_e = max(abs(a - b) for a, b in zip(e, el))
    err_g = max(float(np.max(np.abs(a - b))) if len(a) else 0.0 for a, b in zip(g, gl))
    print(json.dumps({"config": "batch256", "circuits": len(circs), "dtype": "c64",
                      "gates": sum(len(c.ops) for c in circs), "params": sum(c.n_params for c in circs),
                      "marshal_once_s": marshal_s, "first_call_s": first_s, "autotune_s": tune_s,
                      "qubit_counts_tuned": tuned,
                      "one_call_kernel_ms": kern, "one_call_wall_s": prof_wall,
                      "batched_new_params_s": new_params_s,
                      "batched_s": statistics.median(tb), "loop_s": statistics.median(tl),
                      "speedup": statistics.median(tl) / statistics.median(tb),
                      "loop_s_per_qubit_count": per_n,
                      "loop_compiled_during_timing": jit1["compiled"] - jit0["compiled"],
                      "loop_compile_s_during_timing": jit1["compile_seconds"] - jit0["compile_seconds"],
                      "max_abs_energy_batched_minus_loop": err_e, "max_abs_grad_batched_minus_loop": err_g}),
          flush=True)


def config_sweep30(args):
    """Dedicated vs general kernels over every target at 30 qubits complex128
    (Sec. 3.1, Fig. 3c / 4c on one GPU): X by the permutation kernel against X as
    a dense 2x2; CNOT(24, t) by the permutation kernel against a dense 4x4."""
    import torch
    import paper_2508_13615_gb300 as L
    n = args.n
    sv = L.StateVector(n, "c128")
    L.lqs_sv_set_basis(sv.h, 0)
    st = torch.cuda.current_stream()
    Xm = np.array([[0, 1], [1, 0]], dtype=complex)
    CN = np.eye(4, dtype=complex)[[0, 1, 3, 2]]

    def t_of(fn, reps=3):
        fn()
        ts = []
        for _ in range(reps):
            e0, e1 = _events()
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    rows = []
    S = (1 << n) * 16
    for t in range(n):
        c = 24 if t != 24 else 0
        rows.append({"t": t,
                     "x_dedicated_ms": t_of(lambda: L.lqs_apply_gate(sv.h, "X", (t,))),
                     "x_general_ms": t_of(lambda: L.lqs_apply_matrix(sv.h, (t,), Xm)),
                     "cnot_dedicated_ms": t_of(lambda: L.lqs_apply_gate(sv.h, "CNOT", (c, t))),
                     "cnot_general_ms": t_of(lambda: L.lqs_apply_matrix(sv.h, (c, t), CN))})
    sv.close()
    print(json.dumps({"config": "sweep30", "n_qubits": n, "state_bytes": S, "rows": rows}), flush=True)


def config_universal30(args):
    """The universal circuit of Sec. 3.2 (Fig. 6a: 2 n^2 gates, phase gates
    and CNOT ladders) at 30 qubits complex128: fused (compiled segments)
    against the plain per-gate path."""
    import torch
    import paper_2508_13615_gb300 as L
    n = args.n
    c = W.universal(n)
    L.lqs_set_jit(L.LQS_JIT_ON)
    L.lqs_jit_precompile(n, "c128", c.ops, c.params, L.LQS_ARITH_DF)
    sv = L.StateVector(n, "c128")
    st = torch.cuda.current_stream()
    ops = L.OpArray(c.ops)

    def t_of(fn, reps=3):
        L.lqs_sv_set_basis(sv.h, 1)
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            L.lqs_sv_set_basis(sv.h, 1)
            e0, e1 = _events()
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    ms_fused = t_of(lambda: L.lqs_apply_fused(sv.h, ops, c.params, None))
    ms_plain = t_of(lambda: sv.apply(c, fused=False), reps=1)
    passes = L.lqs_plan_fused(n, "c128", c.ops)[0]
    print(json.dumps({"config": "universal30", "n_qubits": n, "dtype": "c128", "gates": len(c.ops),
                      "fused_ms": ms_fused, "fused_passes": passes, "fused_gates_per_s": len(c.ops) / (ms_fused * 1e-3),
                      "plain_ms": ms_plain, "plain_gates_per_s": len(c.ops) / (ms_plain * 1e-3),
                      "speedup_fused": ms_plain / ms_fused}), flush=True)
    sv.close()


def config_fusedplain30(args):
    """The three circuit families of the 30-qubit step (P2 ansatz, P3 QFT) and
    the universal circuit of Sec. 3.2, complex128: the fused path (compiled
    segments) against the plain per-gate path, with the HBM passes of each
    (plain: one kernel launch per lowered gate)."""
    import torch
    import paper_2508_13615_gb300 as L
    n = args.n
    L.lqs_set_jit(L.LQS_JIT_ON)
    sv = L.StateVector(n, "c128")
    st = torch.cuda.current_stream()
    rows = []
    for name, c, basis in (("ansatz_10_layers", W.ansatz(n, 10, 3), 0), ("qft", W.qft(n), W.basis_index(n, 4)),
                           ("universal", W.universal(n), 1)):
        L.lqs_jit_precompile(n, "c128", c.ops, c.params, L.LQS_ARITH_DF)
        ops = L.OpArray(c.ops)

        def run(fused):
            L.lqs_sv_set_basis(sv.h, basis)
            if fused:
                L.lqs_apply_fused(sv.h, ops, c.params, None)
            else:
                sv.apply(c, fused=False)

        def t_of(fused, reps):
            run(fused)
            torch.cuda.synchronize()
            ts = []
            for _ in range(reps):
                k0 = L.lqs_kernel_launches()
                e0, e1 = _events()
                e0.record(st)
                run(fused)
                e1.record(st)
                torch.cuda.synchronize()
                ts.append((e0.elapsed_time(e1), L.lqs_kernel_launches() - k0 - 1))  # less the set_basis launch
            return statistics.median(t for t, _ in ts), ts[-1][1]

        ms_f, launches_f = t_of(True, 3)
        ms_p, launches_p = t_of(False, 1)
        rows.append({"circuit": name, "gates": len(c.ops), "fused_ms": ms_f, "fused_launches": launches_f,
                     "plain_ms": ms_p, "plain_launches": launches_p, "speedup_fused": ms_p / ms_f,
                     "pass_ratio": launches_p / max(launches_f, 1)})
    print(json.dumps({"config": "fusedplain30", "n_qubits": n, "dtype": "c128", "rows": rows}), flush=True)
    sv.close()


def config_tcblock30(args):
    """Dense 32x32 blocks on the tensor cores at 30 qubits complex64: one
    block pass (tcgen05 3xTF32) against the same run of gates on the fused
    path (40 Haar U4 gates on neighbouring pairs of qubits 0..4, compiled
    segments, block extraction off), with the block's matrix formed on the
    host from the gates; and the same gates with the planner's extraction on."""
    import torch
    import paper_2508_13615_gb300 as L
    n = args.n
    pk = peaks()
    L.lqs_set_jit(L.LQS_JIT_ON)
    sv = L.StateVector(n, "c64")
    st = torch.cuda.current_stream()
    c = W.Circuit(n)
    U = np.eye(32, dtype=np.complex128)
    for g in range(40):
        q = (g * 3) % 4  # pairs (q, q + 1) inside qubits 0..4
        M = W.haar_unitary(4, 61, g)
        c.add("U4", (q + 1, q), matrix=M)
        # M acts on (qubit q+1, qubit q) as (most, least) significant local bits
        T = M.reshape(2, 2, 2, 2)
        op = np.zeros((32, 32), dtype=np.complex128)
        for k in range(32):
            e = np.zeros(32, dtype=np.complex128)
            e[k] = 1
            t = e.reshape(2, 2, 2, 2, 2)  # axes: qubit 4, 3, 2, 1, 0
            ax = (4 - (q + 1), 4 - q)
            r = np.tensordot(T, t, axes=([2, 3], list(ax)))
            r = np.moveaxis(r, [0, 1], list(ax))
            op[:, k] = r.reshape(32)
        U = op @ U
    L.lqs_jit_precompile(n, "c64", c.ops, c.params, L.LQS_ARITH_AUTO)

    def t_of(fn, reps=5):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            e0, e1 = _events()
            e0.record(st)
            fn()
            e1.record(st)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return statistics.median(ts)

    L.lqs_sv_set_basis(sv.h, 0)
    L.lqs_apply_fused(sv.h, L.OpArray([W.Op("H", (q,)) for q in range(n)]), np.zeros(1), None)
    ref = sv.tensor.clone()
    ms_block = t_of(lambda: L.lqs_apply_block(sv.h, 5, U))
    ops = L.OpArray(c.ops)
    alu = {"tc_blocks": -1}  # the gates on the compiled fused path (no block extraction)
    ms_fused = t_of(lambda: L.lqs_apply_fused(sv.h, ops, c.params, alu))
    ms_auto = t_of(lambda: L.lqs_apply_fused(sv.h, ops, c.params, None))  # the planner extracts the block
    # one application each from the same input, compared
    sv.tensor.copy_(ref)
    L.lqs_apply_block(sv.h, 5, U)
    a = sv.tensor.clone()
    sv.tensor.copy_(ref)
    L.lqs_apply_fused(sv.h, ops, c.params, alu)
    diff = float((a - sv.tensor).abs().max().item())
    scale = float(sv.tensor.abs().max().item())
    # the same 40 gates on a window of five high qubits (12..16): the planner
    # swaps the window onto qubits 0..4 around the block (relabelling SWAPs)
    win = (12, 13, 14, 15, 16)
    cw = W.Circuit(n)
    for op in c.ops:
        cw.ops.append(W.Op(op.name, tuple(win[q] for q in op.wires), op.pidx, op.matrix, op.inverse))
    cw.params = c.params
    L.lqs_jit_precompile(n, "c64", cw.ops, cw.params, L.LQS_ARITH_AUTO)
    wops = L.OpArray(cw.ops)
    ms_wfused = t_of(lambda: L.lqs_apply_fused(sv.h, wops, cw.params, alu))
    ms_wauto = t_of(lambda: L.lqs_apply_fused(sv.h, wops, cw.params, None))
    L.lqs_profile_start()
    L.lqs_apply_fused(sv.h, wops, cw.params, None)
    wrecs = L.lqs_profile_stop()
    sv.tensor.copy_(ref)
    L.lqs_apply_fused(sv.h, wops, cw.params, None)
    wa = sv.tensor.clone()
    sv.tensor.copy_(ref)
    L.lqs_apply_fused(sv.h, wops, cw.params, alu)
    wdiff = float((wa - sv.tensor).abs().max().item())
    window = {"qubits": list(win), "fused_ms": ms_wfused, "with_block_extraction_ms": ms_wauto,
              "speedup": ms_wfused / ms_wauto, "launches": [r[0] for r in wrecs],
              "max_abs_diff_block_vs_fused": wdiff}
    S = (1 << n) * 8
    gbs = 2 * S / (ms_block * 1e-3) / 1e9
    flops = ((1 << n) // 32) * 64 * 64 * 2 * 3  # per row of 32 amplitudes: a 64 x 64 real product, three times
    print(json.dumps({
        "config": "tcblock30", "n_qubits": n, "dtype": "c64", "state_bytes": S,
        "block": "32x32 complex on qubits 0..4, tcgen05.mma kind::tf32, 3xTF32",
        "block_ms": ms_block, "block_gbs": gbs,
        "roofline": {"bound": "hbm", "achieved": gbs, "peak": pk["hbm_gbs"], "unit": "GB/s",
                     "frac": gbs / pk["hbm_gbs"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured copy)",
                     # DRAM read + write of one launch at 26 qubits (ncu), scaled by the units of n qubits
                     "traffic": traffic_of("k_block_tc", n)[0], **traffic_of("k_block_tc", n)[1]},
        "tensor_tflops": flops / (ms_block * 1e-3) / 1e12,
        "fused_gates": len(c.ops), "fused_ms": ms_fused, "fused_with_block_extraction_ms": ms_auto,
        "speedup_vs_fused": ms_fused / ms_block,
        "max_abs_diff_block_vs_fused": diff, "max_abs_amplitude": scale, "window": window}), flush=True)
    sv.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_QUBITS)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-c64", action="store_true", help="skip the complex64 run of the step")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the 24-qubit adjoint/forward measurement")
    ap.add_argument("--tune", action="store_true",
                    help="let lqs_autotune_fused pick the tile shapes first (measured: +0.4%% for 45 s of tuning)")
    ap.add_argument("--config", default="main",
                    choices=["main", "adjoint24", "precision32", "batch256", "sweep30", "tcblock30", "universal30",
                             "fusedplain30"],
                    help="secondary measurements (one JSON line each); the default is the headline run")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config != "main":
        import torch
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        {"adjoint24": config_adjoint24, "precision32": config_precision32, "batch256": config_batch256,
         "sweep30": config_sweep30, "tcblock30": config_tcblock30, "universal30": config_universal30,
         "fusedplain30": config_fusedplain30}[args.config](args)
        return

    import torch
    ranks = Ranks("nccl")
    world, rank, local = ranks.world, ranks.rank, ranks.local
    torch.cuda.set_device(local)
    barrier = ranks.barrier

    import paper_2508_13615_gb300 as L
    pk = peaks()
    n = args.n
    pin_t, psi_host = host_state(n, pinned=True)
    wl = Workload(n, psi_host)
    st = torch.cuda.current_stream()
    # Fused segments run as compiled straight-line kernels: compile the
    # workload's structures once, ahead of the warm-up (host only, parallel).
    L.lqs_set_jit(L.LQS_JIT_ON)
    t_jit = time.perf_counter()
    n_jit = wl.precompile(L.LQS_ARITH_DF)
    jit_s = time.perf_counter() - t_jit
    # The tile shape per circuit structure, chosen once by the library's
    # autotuner (lqs_apply_fused then uses it); the autotuner uses the state as
    # scratch, and every step starts from the saved input.
    t_tune = time.perf_counter()
    tuned = {}
    if args.tune:
        for name, c, ops in (("ansatz", wl.ansatz, wl.ans_ops), ("qft", wl.qft, wl.qft_ops)):
            tuned[name] = L.lqs_autotune_fused(wl.sv.h, ops, c.params, repeats=1)
    tune_s = time.perf_counter() - t_tune

    for _ in range(args.warmup):
        wl.step()
    torch.cuda.synchronize()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = L.lqs_kernel_launches()
    jit0 = L.lqs_jit_info()
    L.lqs_profile_start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        wl.step()
    e1.record(st)
    torch.cuda.synchronize()
    records = L.lqs_profile_stop()
    launches = L.lqs_kernel_launches() - launches0
    jit1 = L.lqs_jit_info()
    clk = clocks.stop()
    barrier()
    ms = ranks.max(e0.elapsed_time(e1), "cuda")
    ms_step = ms / args.steps
    value = replicas_value(wl.gates, world, ms_step * 1e-3)
    bytes_step = sum(r[2] for r in records) / args.steps
    roof, fams = roofline(records, pk, n)

    # The same step in complex64 (float32 gate math; norms, energies and
    # distances accumulated in float64), from the complex128 input rounded to
    # complex64, timed the same way; then its results against complex128's.
    c64 = None
    if not args.no_c64:
        psi64 = psi_host.astype(np.complex64)
        wl64 = Workload(n, psi64, "c64")
        t_jit = time.perf_counter()
        n_jit64 = wl64.precompile(L.LQS_ARITH_AUTO)
        jit64_s = time.perf_counter() - t_jit
        for _ in range(args.warmup):
            wl64.step()
        torch.cuda.synchronize()
        barrier()
        clocks64 = ClockSampler(local)
        clocks64.start()
        L.lqs_profile_start()
        e0.record(st)
        for _ in range(args.steps):
            wl64.step()
        e1.record(st)
        torch.cuda.synchronize()
        rec64 = L.lqs_profile_stop()
        clk64 = clocks64.stop()
        barrier()
        ms64 = ranks.max(e0.elapsed_time(e1), "cuda") / args.steps
        roof64, fams64 = roofline(rec64, pk, n)
        # P2 energy and the P3 output state (both states hold P3's result now)
        d2, nb = L.lqs_sv_distance(wl64.sv.h, wl.sv.h)
        e128_p2, e64_p2 = wl.energy, wl64.energy
        # P1's output state from the same input in both precisions
        wl.sv.tensor.copy_(wl.saved)
        wl64.sv.tensor.copy_(wl64.saved)
        wl.p1()
        wl64.p1()
        d2p1, nbp1 = L.lqs_sv_distance(wl64.sv.h, wl.sv.h)
        torch.cuda.synchronize()
        c64 = {"value": replicas_value(wl64.gates, world, ms64 * 1e-3), "unit": UNIT, "ms_per_step": ms64,
               "c64_over_c128_speed": ms_step / ms64,
               "arith": "complex64 storage, float32 gate math; norms, energies, distances accumulated in float64",
               "gb_per_s_algorithmic": sum(r[2] for r in rec64) / args.steps / (ms64 * 1e-3) / 1e9,
               "roofline": {k: roof64[k] for k in ("kernel", "bound", "achieved", "peak", "unit", "frac", "share",
                                                   "ms_per_launch")},
               "kernels": fams64, "clocks": clk64,
               "segment_compiler": {"structures_compiled": n_jit64, "compile_wall_s": round(jit64_s, 2)},
               "energy_tfim_ansatz_c64": e64_p2, "abs_energy_c64_minus_c128": abs(e64_p2 - e128_p2),
               "rel_l2_c64_vs_c128_p1_state": math.sqrt(d2p1 / nbp1),
               "rel_l2_c64_vs_c128_p3_state": math.sqrt(d2 / nb),
               "input": "the complex128 input rounded to complex64 (relative L2 rounding about 3e-8)"}
        wl64.close()
        del psi64

    # adjoint gradient over the forward pass (24 qubits, 8 layers, 384 params)
    adj = None if args.no_adjoint else adjoint_leg(args.steps, args.warmup)

    e2e = None
    if not args.no_e2e:
        out_p1 = torch.empty(1 << n, dtype=torch.complex128, pin_memory=True)
        out_p3 = torch.empty(1 << n, dtype=torch.complex128, pin_memory=True)
        o1, o3 = out_p1.numpy(), out_p3.numpy()
        pipe = E2EPipeline(wl, o1, o3)
        pipe.run(1)  # warm (scratch buffers of the new states)
        barrier()
        t0 = time.perf_counter()
        pipe.run(args.steps)
        et = ranks.max(time.perf_counter() - t0, "cuda")
        d2h = pipe.d2h_bytes_per_step()
        pipe.close()
        stride = max(1, o1.size // 4096)
        s1, s3 = o1[::stride].copy(), o3[::stride].copy()
        # one more step with nothing overlapped, timed part by part (after the measured ones)
        parts = {}
        for key, fn in (("h2d", lambda: L.lqs_sv_copy_from_host(wl.sv.h, wl.psi_host)), ("p1", wl.p1),
                        ("d2h_p1", lambda: L.lqs_sv_copy_to_host(wl.sv.h, o1)), ("p2p3", wl.p2p3),
                        ("d2h_p3", lambda: L.lqs_sv_copy_to_host(wl.sv.h, o3))):
            torch.cuda.synchronize()
            tp = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            parts[key] = round(1e3 * (time.perf_counter() - tp), 1)
        e2e = {"value": replicas_value(wl.gates * args.steps, world, et), "unit": UNIT,
               "h2d_bytes_per_step": wl.input_bytes(), "d2h_bytes_per_step": d2h,
               "ms_per_step": 1e3 * et / args.steps, "parts_ms_sequential_step": parts,
               "pipelined_result_matches_sequential":
                   bool(np.array_equal(s1, o1[::stride]) and np.array_equal(s3, o3[::stride])),
               "path": "lqs_sv_copy_from_host (pinned) -> P1 -> lqs_sv_copy_to_host_async (P1 state) -> P2 (expval "
                       "to host) -> P3 -> lqs_sv_copy_to_host_async (P3 state); copies on their own streams, "
                       "overlapping the previous and next step's compute"}

    cpu = None
    if rank == 0 and world == 1:
        # the GPU work is done; the oracle runs in place on the pinned input buffer
        cpu = cpu_baseline_sample(psi_host, wl.sweep, args.cpu_budget)

    if rank == 0:
        rec = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "arith": "complex128 storage, double-float (2 x fp32) gate math",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_qubits": n, "state_gib": (1 << n) * 16 / 2 ** 30,
                       "gates_per_step": wl.gates, "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (16 GiB state vs 129 MB L2); no flush needed"},
            "gb_per_s_algorithmic": bytes_step / (ms_step * 1e-3) / 1e9,
            "hbm_frac_of_8TBps": bytes_step / (ms_step * 1e-3) / 8e12,
            "hbm_frac_of_measured": bytes_step / (ms_step * 1e-3) / 1e9 / float(pk.get("hbm_gbs", 6800.0)),
            "energy_tfim_ansatz": wl.energy,
            "autotuned": {"configs": tuned, "wall_s": round(tune_s, 2)} if tuned else None,
            "segment_compiler": {"mode": "on", "structures_compiled": n_jit, "compile_wall_s": round(jit_s, 2),
                                 "compiled_launches_timed": jit1["launches"] - jit0["launches"],
                                 "compiled_during_timed": jit1["compiled"] - jit0["compiled"],
                                 "failed": jit1["failed"]},
            "roofline": roof, "kernels": fams, "gpu_launches": int(launches), "clocks": clk,
            "c64": c64, "adjoint24": adj,
            "e2e": e2e, "cpu_baseline": cpu,
        }
        print(json.dumps(rec), flush=True)
    ranks.close()


if __name__ == "__main__":
    main()
