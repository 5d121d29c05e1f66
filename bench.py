#!/usr/bin/env python
"""Benchmark of the batched fifth-order Taylor update on one or more GB300s.

Workload (the 14-qubit configuration the headline metric is quoted on):
8192 complex64 states of 14 qubits (7 spatial orbitals, 6 electrons,
Bravyi-Kitaev, strongly correlated synthetic integrals), each prepared from
the Hartree-Fock state by three Taylor updates and then updated in place,
once per step, with its own pool generator (204 spin-conserving singles and
doubles) and angle.  One step = one launch of the support-only update over
all 8192 states: each state's generator support (D/2 rows for a single,
D/8 for a double) is read and written in place, rows off the support are
left as they are (every term of the series past the first vanishes there),
and each state's float64 squared norm is carried (about 0.83 GB of DRAM
traffic per step, larger than L2).  The full-state kernel, which streams
all 2 GiB, is reported beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own 8192 states (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Taylor-5 state updates/s at 14 qubits"
UNIT = "updates/s"
N_SPATIAL, N_ELECTRONS, MAPPING = 7, 6, 1      # 14 qubits, BK
NQ = 2 * N_SPATIAL
D = 1 << NQ
FALLBACK_HBM_GBS = 6800.0
CSRC = os.path.join(ROOT, "paper_2606_29692_gb300", "csrc")
# committed ncu summaries: (file, sources whose hash the summary records)
PROFILE_SUPPORT = (os.path.join(ROOT, "profiles", "taylor5_support_c64_14q.md"),
                   [os.path.join(CSRC, f) for f in ("support.cu", "pair.cuh", "grad.cuh", "dev.cuh")])
PROFILE_PAIR = (os.path.join(ROOT, "profiles", "taylor5_pair_c64_14q.md"),
                [os.path.join(CSRC, f) for f in ("evolve_kernels.cu", "pair.cuh", "dev.cuh")])


def workload_config(n_states):
    return {
        "workload": (f"batched Taylor-5: {n_states} complex64 states, 14 qubits "
                     "(7 spatial orbitals, 6 electrons), Bravyi-Kitaev, strongly correlated "
                     "synthetic integrals (seed 2), pool of 204 singles+doubles, per-state op "
                     "and angle N(0,0.1) (seed 3), states prepared by 3 updates from HF"),
        "n_states": n_states,
        "n_qubits": NQ,
        "pool_size": 204,
        "mapping": "BK",
        "state_precision": "complex64 (float32 products), float64 norm reduction",
        "l2_policy": "inputs larger than L2 (1 GiB of states; each step moves about 0.83 GB of support "
                     "lines and sectors, in place)",
        "norm": "float64 squared norm per state, carried across steps",
    }


# ------------------------------------------------------------------ helpers

def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(sources):
    h = hashlib.sha256()
    for f in sources:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(profile, n_states, layout=None):
    """DRAM bytes per launch from a committed ncu summary, if the kernel's
    sources still hash to the value the summary records and, when the
    summary names the states' memory layout, the run uses the same one."""
    path, sources = profile
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_state:\s*([0-9.eE+]+)", txt)
    h = re.search(r"kernel_source_sha:\s*([0-9a-f]+)", txt)
    if not m or not h or h.group(1) != kernel_source_hash(sources):
        return None
    lay = re.search(r"state_layout:\s*(\w+)", txt)
    if lay and layout is not None and lay.group(1) != layout:
        return None
    return float(m.group(1)) * n_states


def measure_link(src_h, src_d, nbytes=512 << 20, reps=3):
    """Copy rates of the host link: pinned host -> device, device -> pinned
    host, and both at once on two streams (the ceiling for a step whose
    reads and writes cross the link together).  Reads src_h and src_d only."""
    import torch
    hs = src_h.view(torch.uint8).reshape(-1)[:nbytes]
    ds = src_d.view(torch.uint8).reshape(-1)[:nbytes]
    nbytes = min(hs.numel(), ds.numel())
    hs, ds = hs[:nbytes], ds[:nbytes]
    hb = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    db = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    cur = torch.cuda.current_stream()

    def run(h2d, d2h):
        best = float("inf")
        for i in range(reps + 1):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(cur)
            for s, on in ((s1, h2d), (s2, d2h)):
                s.wait_stream(cur)
                if on:
                    with torch.cuda.stream(s):
                        (db.copy_(hs, non_blocking=True) if s is s1 else hb.copy_(ds, non_blocking=True))
            cur.wait_stream(s1)
            cur.wait_stream(s2)
            e1.record(cur)
            torch.cuda.synchronize()
            if i:
                best = min(best, e0.elapsed_time(e1) / 1e3)
        return best

    t_in, t_out, t_both = run(True, False), run(False, True), run(True, True)
    return {"bytes": nbytes, "h2d_gbs": nbytes / t_in / 1e9, "d2h_gbs": nbytes / t_out / 1e9,
            "bidir_gbs": 2 * nbytes / t_both / 1e9, "note": "cudaMemcpyAsync from and to pinned host memory"}


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-i", str(self.gpu_id), "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        for l in self.lines:
            parts = [p.strip() for p in l.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(self.NAMES, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------- CPU oracle timing

_ORACLE_CACHE = {}


def _oracle_setup(idx):
    """Oracle-side inputs of a worker's sample states (cached per process)."""
    key = tuple(idx)
    if key in _ORACLE_CACHE:
        return _ORACLE_CACHE[key]
    import synth
    from oracle import adapt, evolve, pauli
    exc, pps = pauli.pool_pauli(N_SPATIAL, N_ELECTRONS, MAPPING)
    prep_k, prep_th, k, th = synth.t5_batch(8192, len(exc))
    cache = {}

    def A(j):
        if j not in cache:
            cache[j] = pauli.pauli_to_csr(pps[j])
        return cache[j]

    states = []
    for b in idx:
        psi = adapt.hf_state(NQ, N_ELECTRONS, MAPPING)
        for j in range(prep_k.shape[1]):
            psi = evolve.taylor5(A(int(prep_k[b, j])), psi, prep_th[b, j])
        states.append((psi, A(int(k[b])), float(th[b])))
    _ORACLE_CACHE[key] = states
    return states


def _oracle_worker(args):
    """Oracle Taylor-5 updates on a slice of sample states for ~`seconds`."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    idx, seconds = args
    from oracle import evolve
    states = _oracle_setup(idx)
    n = 0
    t0 = time.perf_counter()
    while True:
        for psi, A, th in states:
            evolve.taylor5(A, psi, th)
            n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el


RATE_OPS = ((0, 0.1), (101, -0.07), (203, 0.05))    # (pool index, angle) applied to HF


def _oracle_rate_worker(args):
    """Oracle energies or gradient sweeps of one 14-qubit state for ~`seconds`."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    kind, seconds = args
    import synth
    from oracle import adapt, evolve
    if "rates" not in _ORACLE_CACHE:
        ints, ne = synth.config2()
        sysm = adapt.build_system(ints, ne, MAPPING)
        psi = adapt.hf_state(NQ, ne, MAPPING)
        for k, th in RATE_OPS:
            psi = evolve.taylor5(sysm.pool[k], psi, th)
        _ORACLE_CACHE["rates"] = (sysm, psi)
    sysm, psi = _ORACLE_CACHE["rates"]
    n = 0
    t0 = time.perf_counter()
    while True:
        if kind == "energy":
            adapt.energy(sysm.H, psi)
        elif kind == "gradients":
            adapt.gradients(sysm.H, sysm.pool, psi)
        else:
            evolve.taylor5(sysm.pool[RATE_OPS[0][0]], psi, 0.1)
        n += 1
        el = time.perf_counter() - t0
        if el >= seconds:
            return n, el


def oracle_rates(seconds=3.0):
    """The oracle's energies/s, gradient sweeps/s and updates/s at 14 qubits:
    one core, and all cores (one spawn worker per core, each on its own copy)."""
    cores = os.cpu_count() or 1
    out = {"cores": cores, "workload": "one 14-qubit BK state (Hartree-Fock after three updates), "
                                       "config-2 integrals, complex128 SciPy CSR"}
    with mp.get_context("spawn").Pool(cores) as p:
        for kind in ("energy", "gradients", "update"):
            n1, t1 = p.map(_oracle_rate_worker, [(kind, seconds)])[0]
            res = p.map(_oracle_rate_worker, [(kind, seconds)] * cores)
            out[kind] = {"one_core_per_s": n1 / t1,
                         "all_cores_per_s": sum(r[0] for r in res) / max(r[1] for r in res)}
    return out


def measure_adapt_step(tq, ctx, steps=10):
    """tq_adapt_step with the exact line search (theta = NaN), one state, ten
    consecutive iterations from Hartree-Fock, at 14 and 18 qubits: wall
    time per call (each call synchronises) and the kernels' split."""
    import synth
    out = {"workload": "ADAPT iterations with the line search from Hartree-Fock, complex64 state, BK, "
                       "14 q (config-2 integrals) and 18 q (9 orbitals, 8 electrons, seed 2012)"}
    for nq_, ints, ne in ((14,) + synth.config2(),
                          (18, synth.integrals(9, synth.SEED_CATALOGUE_BASE + 12), synth.electrons_for(9))):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, MAPPING, tq.TQ_C64)
        pool = tq.build_pool(ctx, ints.n_spatial, ne, MAPPING)
        st = tq.State(ctx, nq_, tq.TQ_C64)
        tq.state_set_hf(st, ne, MAPPING)
        tq.adapt_step(ctx, ham, pool, st, 0.0, float("nan"))          # warm
        tq.state_set_hf(st, ne, MAPPING)
        ctx.trace(True)
        t0 = time.perf_counter()
        energies, chosen = [], []
        for _ in range(steps):
            r_ = tq.adapt_step(ctx, ham, pool, st, 0.0, float("nan"))
            energies.append(r_["energy"])
            chosen.append(r_["selected"])
        t = (time.perf_counter() - t0) / steps
        rep = ctx.trace_report()
        ctx.trace(False)
        roof = adapt_kernel_rooflines(tq, ctx, ham, pool, ints.n_spatial, ne, chosen, rep, steps)
        # the same iterations as one call: the first step launched, the rest
        # replayed from a captured graph (no host round trip between steps)
        tq.state_set_hf(st, ne, MAPPING)
        tq.adapt_run(ctx, ham, pool, st, 0.0, steps)                   # warm
        tq.state_set_hf(st, ne, MAPPING)
        t0 = time.perf_counter()
        res, _ = tq.adapt_run(ctx, ham, pool, st, 0.0, steps)
        tr = (time.perf_counter() - t0) / steps
        # the same iterations with the H passes over the CSR (8 lanes per row)
        ctx.set_spmv_schedule(8)
        tq.state_set_hf(st, ne, MAPPING)
        ctx.trace(True)
        t0 = time.perf_counter()
        csr_e = [tq.adapt_step(ctx, ham, pool, st, 0.0, float("nan"))["energy"] for _ in range(steps)]
        tc = (time.perf_counter() - t0) / steps
        rep_c = ctx.trace_report()
        ctx.trace(False)
        ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)
        out[f"{nq_}q_csr"] = {"ms_per_step": 1e3 * tc, "kernel_ms_per_step": {k_: v[1] / steps for k_, v in rep_c.items()},
                              "same_trajectory": [abs(a_ - b_) < 1e-6 for a_, b_ in zip(csr_e, energies)].count(True)}
        out[f"{nq_}q"] = {"ms_per_step": 1e3 * t, "ms_per_step_graph_run": 1e3 * tr, "nnz": ham.nnz, "pool": pool.M,
                          "rooflines": roof,
                          "kernel_ms_per_step": {k_: v[1] / steps for k_, v in rep.items()},
                          "energy_first_last": [energies[0], energies[-1]],
                          "graph_run_same_energies": [r_["energy"] for r_ in res] == energies}
    return out


_L2_RATE = {}


def l2_rate(tq, ctx):
    """The device's measured L2 read rate (bytes/s), once per process."""
    if "v" not in _L2_RATE:
        _L2_RATE["v"] = tq.l2_read_rate(ctx, 32 << 20, 64)
    return _L2_RATE["v"]


def adapt_kernel_rooflines(tq, ctx, ham, pool, n_spatial, ne, chosen, rep, steps):
    """Achieved bytes over time for the ADAPT step's gradient and line-search
    kernels, against the HBM copy peak and the measured L2 read rate.

    Gradients (k_pool_grad): every generator's support rows, each reading
    H psi at the row (float32 pairs for complex64) and psi at its partner:
    sum_k |S_k| (8 + 8) bytes in complex64; both vectors stay in L2.
    Line search (k_line_support): the CSR rows of the chosen generator's
    support (8 bytes per row of offsets and diagonal, 8 per entry of column
    and value in complex64) and psi (8 bytes per amplitude, read once at
    best); the gathers land in L2."""
    import numpy as np
    peak, _ = peaks()
    l2 = l2_rate(tq, ctx) / 1e9
    nq_ = 2 * n_spatial
    D_ = 1 << nq_
    f = tq.pool_support_forms(n_spatial, ne, MAPPING)
    supp = float(sum(D_ >> int(m) for m in f["m"]))
    out = {"peak_hbm_gbs": peak, "l2_read_gbs": l2}
    n_g, ms_g = rep.get("pool_gradients", (0, float("nan")))
    if n_g:
        b = supp * 16
        s_ = ms_g / n_g * 1e-3
        out["pool_gradients"] = {"kernel": "k_pool_grad", "bytes_per_sweep": b, "ms": 1e3 * s_,
                                 "achieved_gbs": b / s_ / 1e9, "frac_hbm": b / s_ / 1e9 / peak,
                                 "frac_l2": b / s_ / 1e9 / l2}
    n_l, ms_l = rep.get("line_support", (0, float("nan")))
    if n_l:
        rp, _, _, _ = tq.ham_csr(ham)
        rowptr = _dev_to_host(rp, D_ + 1, "<i4").astype(np.int64)
        rows = support_rows(tq, n_spatial, ne, MAPPING, ks=sorted(set(chosen)))
        per_k = {}
        for k_, r_ in rows.items():
            nnz_s = int((rowptr[r_ + 1] - rowptr[r_]).sum())
            per_k[k_] = 16.0 * r_.size + 8.0 * nnz_s + 8.0 * D_
        b = float(np.mean([per_k[k_] for k_ in chosen]))
        s_ = ms_l / n_l * 1e-3
        out["line_search"] = {"kernel": "k_line_support", "mean_bytes_per_step": b, "ms": 1e3 * s_,
                              "achieved_gbs": b / s_ / 1e9, "frac_hbm": b / s_ / 1e9 / peak,
                              "frac_l2": b / s_ / 1e9 / l2}
    return out


def measure_rates(tq, ctx, reps=200):
    """Energies/s and gradient sweeps/s through the public API (one state per
    call, result read back on the host) at 14 qubits, beside the oracle's."""
    import synth
    ints, ne = synth.config2()
    out = {"workload": "one 14-qubit BK state (Hartree-Fock after three updates), config-2 integrals; "
                       "tq_energy / tq_pool_gradients with host results (each call synchronises)"}
    pool = tq.build_pool(ctx, ints.n_spatial, ne, MAPPING)
    for prec, name in ((tq.TQ_C64, "c64"), (tq.TQ_C128, "c128")):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, MAPPING, prec)
        st = tq.State(ctx, NQ, prec)
        tq.state_set_hf(st, ne, MAPPING)
        for k, th in RATE_OPS:
            tq.evolve_taylor5(ctx, pool, k, th, st)
        for _ in range(5):
            tq.energy(ctx, ham, st)
            tq.pool_gradients(ctx, ham, pool, st)
        t0 = time.perf_counter()
        for _ in range(reps):
            tq.energy(ctx, ham, st)
        te = time.perf_counter() - t0
        t0 = time.perf_counter()
        for _ in range(reps):
            tq.pool_gradients(ctx, ham, pool, st)
        tg = time.perf_counter() - t0
        out[name] = {"energies_per_s": reps / te, "gradient_sweeps_per_s": reps / tg}
    return out


def cpu_oracle_rate(seconds=12.0, states_per_core=4, cores=None, pool=None):
    cores = cores or os.cpu_count() or 1
    jobs = [(list(range(c * states_per_core, (c + 1) * states_per_core)), seconds) for c in range(cores)]
    if pool is None:
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as p:
            res = p.map(_oracle_worker, jobs)
    else:
        res = pool.map(_oracle_worker, jobs)
    n = sum(r[0] for r in res)
    t = max(r[1] for r in res)
    return n / t, cores, n, t


# --------------------------------------------------------------- GPU arm

def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import paper_2606_29692_gb300 as tq
    import synth

    from paper_2606_29692_gb300 import dist as tqd

    torch.cuda.set_device(local_rank)
    tqd.init("nccl", torch.device("cuda", local_rank))
    S = args.states
    ctx = tq.Context(local_rank)
    pool_nat = tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, MAPPING)
    # the states' memory layout: BK with its basis index carried by an
    # invertible GF(2) map (linear) or a qubit order (sector) chosen so that
    # the pool's supports fill the lowest index bits (32-byte sectors), or
    # BK's own order; every result is the same up to the index map
    if args.layout == "linear":
        lrows = tq.pool_sector_basis(N_SPATIAL, N_ELECTRONS, MAPPING, args.layout_bits)
        mp_run = tq.mapping_linear(MAPPING, lrows)
        index_map = tq.linear_index(lrows)
        layout_desc = {"kind": "linear", "rows": [int(r) for r in lrows],
                       "note": "Bravyi-Kitaev with basis index r stored at r' = M r over GF(2), bit i of r' the "
                               "parity of r over rows[i] (tq_mapping_linear, rows from tq_pool_sector_basis): "
                               "the same encoding's results, the pool's supports packed into 32-byte sectors"}
    elif args.layout == "sector":
        order = tq.pool_sector_order(N_SPATIAL, N_ELECTRONS, MAPPING, args.layout_bits)
        mp_run = tq.mapping_relabelled(MAPPING, order)
        index_map = tq.relabel_index(order)
        layout_desc = {"kind": "sector", "bit_of_qubit": [int(o) for o in order],
                       "note": "Bravyi-Kitaev with qubit k stored at index bit bit_of_qubit[k] "
                               "(tq_mapping_relabelled, order from tq_pool_sector_order)"}
    else:
        mp_run = MAPPING
        index_map = np.arange(D)
        layout_desc = {"kind": "natural", "note": "Bravyi-Kitaev's own qubit order"}
    pool = pool_nat if mp_run == MAPPING else tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, mp_run)
    # every rank updates its own batch of S states (weak scaling, no exchange)
    prep_k, prep_th, k, th = synth.t5_batch(S, pool.M, seed=tqd.rank_seed(synth.SEED_T5_BATCH, rank))
    hf = tq.hf_index(NQ, N_ELECTRONS, mp_run)
    psi = torch.zeros((S, D), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    dn = torch.ones(S, dtype=torch.float64, device="cuda")       # ||HF||^2, carried from here on
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch_support(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                        torch.as_tensor(prep_th[:, j].copy()).cuda(), dn)
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    # the CUDA context's L2 fetch granularity (32 or 64 bytes: the update's
    # reads are runs of support rows) and the schedule are the fastest pair
    # of the sixteen on this batch (untimed, before warm-up)
    fetch_default = ctx.l2_fetch()

    applied = [0]   # launches of the timed update on the batch (the fidelity check replays them)

    def step():
        tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, dn)
        applied[0] += 1

    # the clock sampler starts now, so that it samples under load and the GPU
    # never idles between the tuning, the warm-up and the timed region (a
    # GPU left idle for a fraction of a second runs its next launches slower)
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        gpu_id = str(local_rank)
    clocks = ClockSampler(gpu_id)
    clocks.start()
    tune = {}
    for fetch in ([args.l2_fetch] if args.l2_fetch else [32, 64]):
        ctx.set_l2_fetch(fetch)
        for occ in ([args.ctas_per_sm] if args.ctas_per_sm >= 0 else [0, 3, 2]):
            ctx.set_support_occupancy(tq.TQ_C64, occ)
            for cand in ([args.pair_schedule] if args.pair_schedule else [4, -1, -2, -4, -8]):
                ctx.set_support_schedule(tq.TQ_C64, cand)
                step()
                tune[(fetch, occ, cand)] = time_launches(step, 10)
    best_fetch, best_occ, upt = min(tune, key=tune.get)
    tune_ms = {f"{f_}B/{o_ or 'max'}cta/{c_}": v for (f_, o_, c_), v in tune.items()}
    ctx.set_support_schedule(tq.TQ_C64, upt)
    ctx.set_support_occupancy(tq.TQ_C64, best_occ)
    ctx.set_l2_fetch(best_fetch)

    barrier = tqd.barrier

    def max_over_ranks(x):
        return tqd.max_over_ranks(x, device="cuda")

    # untimed steps until the sampler has three samples under load (at most 2 s)
    t_wait = time.time() + 2.0
    while clocks.proc is not None and len(clocks.lines) < 3 and time.time() < t_wait:
        for _ in range(20):
            step()
        torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    # the timed region: K steps, one launch each, no per-launch events (a
    # recorded event between launches adds a few microseconds of gap)
    launches0 = ctx.launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    launches = ctx.launches() - launches0
    t_local = e0.elapsed_time(e1) / 1e3
    t = max_over_ranks(t_local)
    value = tqd.weak_scaling_value(S, world, args.steps, t)
    # every step is one launch of the update kernel, so its average duration
    # over the timed region is the region's time over K (gaps included)
    assert launches == args.steps, (launches, args.steps)
    sup_s = t_local / args.steps
    # beside it, untimed: the same launches bracketed one by one by events
    ctx.trace(True)
    for _ in range(min(args.steps, 20)):
        step()
    rep = ctx.trace_report()
    ctx.trace(False)
    sup_n, sup_ms = rep.get("taylor5_support", (0, float("nan")))
    sup_traced_s = sup_ms / max(sup_n, 1) / 1e3
    # the access pattern's own floor: the same launch (schedule, L2 fetch,
    # occupancy, state queue) with the update taken out, every support row
    # written back as read; timed back to back like the steps
    for _ in range(3):
        tq.evolve_taylor5_batch_support_touch(ctx, pool, psi, dk, dn)
    touch_s = time_launches(lambda: tq.evolve_taylor5_batch_support_touch(ctx, pool, psi, dk, dn),
                            max(args.steps, 20)) / 1e3
    ctx.set_l2_fetch(0)
    # algorithmic bytes: each support amplitude read and written once, the
    # carried norm read and written once; the touched 32-byte sectors and
    # 128-byte lines are the floors the memory system can reach
    rows = support_rows(tq, N_SPATIAL, N_ELECTRONS, mp_run)
    n_rows = np.array([r.size for r in rows], dtype=np.float64)[k]
    n_sect = np.array([np.unique(r >> 2).size for r in rows], dtype=np.float64)[k]
    n_line = np.array([np.unique(r >> 4).size for r in rows], dtype=np.float64)[k]
    alg_bytes = float((16 * n_rows).sum() + 16 * S)
    sector_bytes = float((64 * n_sect).sum() + 16 * S)
    line_bytes = float((128 * n_line + 32 * n_sect).sum())      # reads by line, writes by sector
    peak, peak_src = peaks()
    achieved = alg_bytes / sup_s / 1e9
    traffic = profiled_traffic(PROFILE_SUPPORT, S, args.layout)

    # end to end: the same update on states in pinned host memory, through
    # the host-memory entry point (the kernel reads and writes each state's
    # support sectors over the host link; k, theta and the norms are copied)
    psi_h = torch.empty((S, D), dtype=torch.complex64).pin_memory()
    psi_h.copy_(psi)
    k_h = torch.as_tensor(k).pin_memory()
    th_h = torch.as_tensor(th).pin_memory()
    n_h = dn.cpu().pin_memory()
    e2e_steps = max(1, min(args.steps, 20))
    e2e_tune = {}
    for fetch in (32, 64, 128):
        ctx.set_l2_fetch(fetch)
        for cand in (-1, -2, -4, -8, 1, 2, 4):
            ctx.set_support_schedule(tq.TQ_C64, cand)
            tq.evolve_taylor5_batch_support_host(ctx, pool, psi_h, k_h, th_h, n_h)
            t0 = time.perf_counter()
            for _ in range(3):
                tq.evolve_taylor5_batch_support_host(ctx, pool, psi_h, k_h, th_h, n_h)
            e2e_tune[(fetch, cand)] = (time.perf_counter() - t0) / 3
    e2e_fetch, e2e_sched = min(e2e_tune, key=e2e_tune.get)
    ctx.set_l2_fetch(e2e_fetch)
    ctx.set_support_schedule(tq.TQ_C64, e2e_sched)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        tq.evolve_taylor5_batch_support_host(ctx, pool, psi_h, k_h, th_h, n_h)
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    ctx.set_l2_fetch(0)
    e2e = {"value": world * S * e2e_steps / t_e2e, "unit": UNIT,
           "h2d_bytes_per_step": float(32 * n_sect.sum()) + S * (4 + 8 + 8),
           "d2h_bytes_per_step": float(32 * n_sect.sum()) + S * 8,
           "bytes_note": "support sectors read and written in place by the kernel over the host link "
                         "(32-byte sectors), plus k, theta and the norms copied",
           "schedule": e2e_sched, "l2_fetch_bytes": e2e_fetch,
           "ms_per_step_by_fetch_and_schedule": {f"{f_}B/{c_}": 1e3 * v for (f_, c_), v in e2e_tune.items()},
           "api": "tq_evolve_taylor5_batch_support_host (states in pinned host memory)"}
    # the full-state host path for comparison: whole states copied in and out
    tq.evolve_taylor5_batch_host(ctx, pool, psi_h, k_h, th_h, n_h)     # warm
    t0 = time.perf_counter()
    for _ in range(3):
        tq.evolve_taylor5_batch_host(ctx, pool, psi_h, k_h, th_h, n_h)
    t_full = max_over_ranks(time.perf_counter() - t0)
    e2e["full_copy_path"] = {"value": world * S * 3 / t_full, "api": "tq_evolve_taylor5_batch_host "
                             "(whole states copied in and out on 3 streams, full-state kernel)",
                             "h2d_bytes_per_step": S * D * 8 + S * 12, "d2h_bytes_per_step": S * D * 8 + S * 8}
    # the host link's own copy rates: the roofline of both host paths
    link = measure_link(psi_h, psi)
    e2e_bytes = e2e["h2d_bytes_per_step"] + e2e["d2h_bytes_per_step"]
    full_bytes = e2e["full_copy_path"]["h2d_bytes_per_step"] + e2e["full_copy_path"]["d2h_bytes_per_step"]
    link["frac"] = e2e_bytes / (t_e2e / e2e_steps) / 1e9 / link["bidir_gbs"]
    link["full_copy_frac"] = full_bytes / (t_full / 3) / 1e9 / link["bidir_gbs"]
    link["frac_note"] = ("the step's bytes over the link at the two-way copy rate, over the measured step "
                         "time; the support path moves sectors by kernel loads and stores, not by copies")
    e2e["link"] = link
    finite = bool(torch.isfinite(dn).all().item()) and float(dn.min().item()) > 0.5
    extra = {}
    if rank == 0 and world == 1 and args.fidelity_samples > 0:
        idx = np.linspace(0, S - 1, args.fidelity_samples).astype(np.int64).tolist()
        # the oracle's BK order: amplitude b of the oracle is at relabel[b]
        extra["headline_vs_oracle"] = headline_fidelity(psi, dn, idx, S, tqd.rank_seed(synth.SEED_T5_BATCH, rank),
                                                        applied[0], index_map)
    if rank == 0 and args.layout != "natural":
        extra["natural_layout"] = measure_layout(tq, ctx, pool_nat, MAPPING, "BK's own qubit order", S, k, th,
                                                 prep_k, prep_th, sup_s)
    if rank == 0 and args.layout == "linear":
        order = tq.pool_sector_order(N_SPATIAL, N_ELECTRONS, MAPPING, args.layout_bits)
        mp_o = tq.mapping_relabelled(MAPPING, order)
        extra["qubit_order_layout"] = measure_layout(
            tq, ctx, tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, mp_o), mp_o,
            "BK with its qubits reordered for sector fill (tq_pool_sector_order)", S, k, th, prep_k, prep_th, sup_s)
        extra["grouped_layout"] = measure_grouped_layout(tq, ctx, pool, psi, dn, k, th, sup_s,
                                                         mapping=mp_run)
    pool = pool_nat   # the other sections use BK's own qubit order
    if rank == 0 and not args.headline_only:
        extra["precision_vs_oracle"] = measure_precision(tq, ctx)
        extra["m0_8q_step"] = measure_m0(tq, ctx)
        extra["m1_12q_trajectories"] = measure_m1(tq, ctx)
        extra["general_update"] = measure_general_update(tq, ctx)
        extra["fp64_single_instance"] = measure_fp64_single(tq, ctx, pool, k, th)
        extra["full_state"] = measure_full_state(tq, ctx, pool, S)
        extra["rates_14q"] = measure_rates(tq, ctx)
        extra["adapt_step"] = measure_adapt_step(tq, ctx)
        extra["c128_batched"] = measure_c128_batched(tq, ctx, pool)
        extra["spmv"] = measure_spmv(tq, ctx, args.spmv_qubits)
        extra["trajectories"] = measure_trajectories(tq, ctx, args.traj)
        extra["sector"] = measure_sector(tq, ctx)
        extra["families"] = measure_families(tq)
        extra["vqe"] = measure_vqe(tq, ctx)
        extra["io"] = measure_io(tq, ctx)
        if args.serve_seconds > 0:
            extra["serving"] = measure_serving_process(local_rank, args.serve_seconds, args.serve_rate,
                                                       args.serve_sweep)
    out = None
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64",
            "data": "synthetic",
            "config": dict(workload_config(S),
                           qubit_layout=layout_desc,
                           schedule={"support_pairs_per_thread": upt,
                                                         "ms_per_launch_by_schedule": tune_ms,
                                                         "l2_fetch_bytes": best_fetch,
                                                         "ctas_per_sm": best_occ or "as many as fit",
                                                         "l2_fetch_default": fetch_default}),
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": "k_taylor5_support<float>",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "sector_bytes_per_launch": sector_bytes,
                         "sector_frac": sector_bytes / sup_s / 1e9 / peak,
                         "line_read_sector_write_bytes_per_launch": line_bytes,
                         "line_frac": line_bytes / sup_s / 1e9 / peak,
                         # the ncu DRAM bytes of the committed capture over this run's launch time
                         "traffic_gbs": traffic / sup_s / 1e9 if traffic is not None else None,
                         "traffic_frac": traffic / sup_s / 1e9 / peak if traffic is not None else None,
                         # the full-state byte model (2 D 8 bytes per update):
                         # its roofline in updates/s, and this step against it
                         "full_state_roofline_updates_per_s": peak * 1e9 / (2 * D * 8),
                         "value_over_full_state_roofline": value / (peak * 1e9 / (2 * D * 8) * world),
                         "kernel_ms_per_launch": sup_s * 1e3,
                         "kernel_ms_per_launch_note": "the timed region's CUDA-event time over its K launches "
                                                      "(one launch per step, gaps included)",
                         "kernel_ms_per_launch_event_bracketed": sup_traced_s * 1e3,
                         "touch_floor_ms_per_launch": touch_s * 1e3,
                         "update_over_touch_floor": sup_s / touch_s,
                         "touch_floor_note": "the same launch with the update taken out (every support row read "
                                             "and written back unchanged, tq_evolve_taylor5_batch_support_touch): "
                                             "the floor the access pattern sets",
                         "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured"
                         else "fallback"},
            "e2e": e2e,
            "gpu_launches": launches,
            "kernels": {"taylor5_support": {"launches": launches, "ms": t_local * 1e3}},
            "clocks": clk,
            "norms_finite": finite,
        }
        out.update(extra)
    return out


def time_launches(fn, reps):
    """Milliseconds per call of fn (one kernel launch each) on the current
    stream: one CUDA-event pair around reps calls, no per-launch events."""
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_layout(tq, ctx, pool, mapping, label, n_states, k, th, prep_k, prep_th, s_headline, reps=50):
    """The headline batch in another memory layout (mapping: BK's own order
    or another relabelling): the same states, generators and angles, the
    same support-only kernel, every schedule timed at 32-byte L2 fetches
    and the fastest kept."""
    import numpy as np
    import torch
    hf = tq.hf_index(NQ, N_ELECTRONS, mapping)
    psi = torch.zeros((n_states, D), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    dn = torch.ones(n_states, dtype=torch.float64, device="cuda")
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch_support(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                        torch.as_tensor(prep_th[:, j].copy()).cuda(), dn)
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    ctx.set_l2_fetch(32)
    per = {}
    for occ in (0, 3, 2):
        ctx.set_support_occupancy(tq.TQ_C64, occ)
        for ppt in (4, -1, -2, -4):
            ctx.set_support_schedule(tq.TQ_C64, ppt)
            for _ in range(3):
                tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, dn)
            per[(occ, ppt)] = time_launches(lambda: tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, dn),
                                            reps)
    ctx.set_l2_fetch(0)
    ctx.set_support_occupancy(tq.TQ_C64, 0)
    best = min(per, key=per.get)
    ms = per[best]
    rows = support_rows(tq, N_SPATIAL, N_ELECTRONS, mapping)
    n_rows = np.array([r.size for r in rows], dtype=np.float64)[k]
    n_sect = np.array([np.unique(r >> 2).size for r in rows], dtype=np.float64)[k]
    alg = float((16 * n_rows).sum() + 16 * n_states)
    sect = float((64 * n_sect).sum() + 16 * n_states)
    peak, _ = peaks()
    return {"workload": f"the headline batch in {label}",
            "ctas_per_sm": best[0] or "as many as fit", "pairs_per_thread": best[1],
            "ms_per_launch": ms, "ms_by_schedule": {f"{o_ or 'max'}cta/{p_}": v for (o_, p_), v in per.items()},
            "updates_per_s": n_states / (ms * 1e-3),
            "algorithmic_bytes_per_launch": alg, "sector_bytes_per_launch": sect,
            "frac": alg / (ms * 1e-3) / 1e9 / peak, "sector_frac": sect / (ms * 1e-3) / 1e9 / peak,
            "headline_layout_speedup": ms / (s_headline * 1e3)}


def measure_grouped_layout(tq, ctx, pool, psi, dn, k, th, s_flat, mapping, reps=50):
    """The headline batch with the states that take the same generator
    interleaved in groups of four (tq_evolve_taylor5_batch_grouped): a
    support row of a group is one whole 32-byte sector holding that row of
    its four states.  The same states, generators and angles in the same
    qubit layout; a generator's last group is filled up with theta = 0
    copies of one of its states.  One launch is checked against the
    per-state support update (bit-identical amplitudes) before timing."""
    import numpy as np
    import torch
    G = tq.TQ_GROUP_C64
    S = int(k.size)
    slot_state, slot_theta, group_k = [], [], []
    for kk in np.unique(k):
        idx = np.flatnonzero(k == kk)
        pad = (-idx.size) % G
        slot_state.extend(idx.tolist() + [int(idx[-1])] * pad)
        slot_theta.extend(th[idx].tolist() + [0.0] * pad)
        group_k.extend([int(kk)] * ((idx.size + pad) // G))
    n_groups = len(group_k)
    sel = torch.as_tensor(np.asarray(slot_state, dtype=np.int64)).cuda()
    dth = torch.as_tensor(np.asarray(slot_theta, dtype=np.float64)).cuda()
    dkg = torch.as_tensor(np.asarray(group_k, dtype=np.int32)).cuda()
    dks = torch.as_tensor(np.repeat(np.asarray(group_k, dtype=np.int32), G)).cuda()
    ref = psi.index_select(0, sel)
    n_ref = dn.index_select(0, sel)
    gpsi = ref.view(n_groups, G, D).permute(0, 2, 1).contiguous()
    n_g = n_ref.clone()
    tq.evolve_taylor5_batch_support(ctx, pool, ref, dks, dth, n_ref)
    tq.evolve_taylor5_batch_grouped(ctx, pool, gpsi, dkg, dth, n_g)
    back = gpsi.permute(0, 2, 1).reshape(n_groups * G, D)
    identical = bool(torch.equal(torch.view_as_real(back), torch.view_as_real(ref)))
    norm_dev = float(((n_g - n_ref).abs() / n_ref).max().item())
    del ref, back
    fetch0 = ctx.l2_fetch()
    per = {}
    for fetch in (32, 64):
        ctx.set_l2_fetch(fetch)
        for lanes in (1, 2, 4):
            for ppt in (1, 2, 4):
                ctx.set_grouped_schedule(tq.TQ_C64, lanes, ppt)
                for _ in range(3):
                    tq.evolve_taylor5_batch_grouped(ctx, pool, gpsi, dkg, dth, n_g)
                per[(fetch, lanes, ppt)] = time_launches(
                    lambda: tq.evolve_taylor5_batch_grouped(ctx, pool, gpsi, dkg, dth, n_g), reps)
    ctx.set_l2_fetch(fetch0)
    best = min(per, key=per.get)
    ctx.set_grouped_schedule(tq.TQ_C64, best[1], best[2])
    ms = per[best]
    finite = bool(torch.isfinite(n_g).all().item())
    del gpsi
    torch.cuda.empty_cache()
    rows = support_rows(tq, N_SPATIAL, N_ELECTRONS, mapping)
    n_rows = np.array([r.size for r in rows], dtype=np.float64)
    alg = float((16 * n_rows[k]).sum() + 16 * S)                       # the real states' rows and norms
    touched = float((64 * n_rows[np.asarray(group_k)]).sum() + 16 * n_groups * G)   # padding included
    peak, _ = peaks()
    return {"workload": f"the headline batch ({S} complex64 14-qubit states, same generators and angles, same "
                        f"qubit layout) grouped by generator: {n_groups} groups of {G} interleaved states, "
                        f"{n_groups * G - S} theta = 0 fill states",
            "kernel": "k_taylor5_grouped<float>", "api": "tq_evolve_taylor5_batch_grouped",
            "l2_fetch_bytes": best[0], "lanes_per_row": best[1], "pairs_per_lane": best[2],
            "ms_by_fetch_lanes_and_pairs": {f"{f_}B/{l_}/{p_}": v for (f_, l_, p_), v in per.items()},
            "ms_per_launch": ms, "updates_per_s": S / (ms * 1e-3),
            "algorithmic_bytes_per_launch": alg, "touched_sector_bytes_per_launch": touched,
            "frac": alg / (ms * 1e-3) / 1e9 / peak, "sector_frac": touched / (ms * 1e-3) / 1e9 / peak,
            "speedup_over_one_state_per_vector": s_flat * 1e3 / ms,
            "amplitudes_identical_to_per_state_update": identical,
            "max_rel_norm_deviation_from_per_state_update": norm_dev, "norms_finite": finite,
            "note": "applies when several states take the same generator in one step (a pool scan, "
                    "a line search, trajectories that agree); not the headline layout"}


def measure_full_state(tq, ctx, pool, n_states, reps=50):
    """The same batch with the full-state pair kernel, which streams every
    amplitude of every state (2 D 8 bytes per update) and recomputes each
    norm from scratch."""
    import torch

    import synth
    prep_k, prep_th, k, th = synth.t5_batch(n_states, pool.M, seed=synth.SEED_T5_BATCH)
    hf = tq.hf_index(NQ, N_ELECTRONS, MAPPING)
    psi = torch.zeros((n_states, D), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                torch.as_tensor(prep_th[:, j].copy()).cuda())
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    dn = torch.zeros(n_states, dtype=torch.float64, device="cuda")
    upt, _ = tq.autotune_pair(ctx, pool, tq.TQ_C64, n_states=min(n_states, 2048))
    for _ in range(3):
        tq.evolve_taylor5_batch(ctx, pool, psi, dk, dth, dn)
    ctx.trace(True)
    for _ in range(reps):
        tq.evolve_taylor5_batch(ctx, pool, psi, dk, dth, dn)
    rep = ctx.trace_report()
    ctx.trace(False)
    n_l, ms = rep["taylor5_pair"]
    nr, nrms = rep.get("norm_reduce", (1, 0.0))
    ms /= n_l
    peak, _ = peaks()
    alg = 2.0 * D * 8 * n_states
    gbs = alg / (ms * 1e-3) / 1e9
    return {"workload": f"the headline batch ({n_states} complex64 14-qubit states) with the full-state kernel",
            "kernel": "k_taylor5_pair<float>", "units_per_thread": upt, "ms_per_launch": ms,
            "norm_reduce_ms": nrms / nr, "updates_per_s": n_states / ((ms + nrms / nr) * 1e-3),
            "algorithmic_bytes_per_launch": alg, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
            "traffic": profiled_traffic(PROFILE_PAIR, n_states)}


def measure_c128_batched(tq, ctx, pool, n_states=4096, reps=20):
    """The complex128 form of the headline update, batched: n_states 14-qubit
    states (1 GiB, larger than L2), each its own generator and angle."""
    import numpy as np
    import torch

    import synth
    D = 1 << NQ
    rng = np.random.default_rng(synth.SEED_T5_BATCH)
    k = torch.as_tensor(rng.integers(0, pool.M, size=n_states).astype(np.int32)).cuda()
    th = torch.as_tensor(rng.normal(0.0, 0.1, size=n_states)).cuda()
    g = torch.Generator("cuda").manual_seed(6)
    psi = torch.randn(n_states, D, dtype=torch.complex128, device="cuda", generator=g)
    psi /= torch.linalg.vector_norm(psi, dim=1, keepdim=True)
    n2 = torch.zeros(n_states, dtype=torch.float64, device="cuda")
    for _ in range(3):
        tq.evolve_taylor5_batch(ctx, pool, psi, k, th, n2, prec=tq.TQ_C128)
    ctx.trace(True)
    for _ in range(reps):
        tq.evolve_taylor5_batch(ctx, pool, psi, k, th, n2, prec=tq.TQ_C128)
    rep = ctx.trace_report()
    ctx.trace(False)
    n_l, ms = rep["taylor5_pair"]
    ms /= n_l
    nr, nrms = rep.get("norm_reduce", (1, 0.0))
    peak, _ = peaks()
    alg = 2.0 * D * 16
    # the support-only form of the same update (norm carried), every schedule
    per = {}
    for ppt in (1, 2, 4, 8, -1, -2, -4, -8):
        ctx.set_support_schedule(tq.TQ_C128, ppt)
        for _ in range(3):
            tq.evolve_taylor5_batch_support(ctx, pool, psi, k, th, n2, prec=tq.TQ_C128)
        ctx.trace(True)
        for _ in range(reps):
            tq.evolve_taylor5_batch_support(ctx, pool, psi, k, th, n2, prec=tq.TQ_C128)
        rep = ctx.trace_report()
        ctx.trace(False)
        ns, sms_ = rep["taylor5_support"]
        nc, ncms = rep.get("norm_carry", (1, 0.0))
        per[ppt] = sms_ / ns + ncms / nc
    ppt = min(per, key=per.get)
    ctx.set_support_schedule(tq.TQ_C128, ppt)
    sup_ms = per[ppt]
    # both kernels are bound by the float64 pipe: 12 float64 operations per
    # pair (c5 psi + s5 A psi: 4 multiplies and 4 FMAs; |psi|^2: 4 FMAs),
    # against the device's measured float64 FMA rate
    fma_rate = tq.fp64_fma_rate(ctx)
    rows = support_rows(tq, N_SPATIAL, N_ELECTRONS, MAPPING)
    n_pairs = np.array([r.size // 2 for r in rows], dtype=np.float64)[k.cpu().numpy()]
    ops_sup = 12.0 * float(n_pairs.sum())
    ops_full = 12.0 * n_states * (D // 2)
    fp64 = {"peak_lane_ops_per_s": fma_rate, "peak_tflops": 2 * fma_rate / 1e12,
            "peak_source": "tq_fp64_fma_rate (independent float64 FMA chains, this run)",
            "ops_per_pair": 12,
            "support": {"lane_ops_per_launch": ops_sup, "achieved_lane_ops_per_s": ops_sup / (sup_ms * 1e-3),
                        "frac": ops_sup / (sup_ms * 1e-3) / fma_rate},
            "full_state": {"lane_ops_per_launch": ops_full, "achieved_lane_ops_per_s": ops_full / (ms * 1e-3),
                           "frac": ops_full / (ms * 1e-3) / fma_rate}}
    return {"workload": f"{n_states} complex128 states, 14 qubits, own generator and angle each",
            "kernel": "k_taylor5_pair<double>", "ms_per_launch": ms, "norm_reduce_ms": nrms / nr,
            "updates_per_s": n_states / ((ms + nrms / nr) * 1e-3),
            "achieved_gbs": alg * n_states / (ms * 1e-3) / 1e9, "hbm_frac": alg * n_states / (ms * 1e-3) / 1e9 / peak,
            "support": {"kernel": "k_taylor5_support<double>", "pairs_per_thread": ppt, "ms_per_update_launch": sup_ms,
                        "ms_by_schedule": {str(p_): v for p_, v in per.items()},
                        "updates_per_s": n_states / (sup_ms * 1e-3)},
            "fp64_roofline": fp64}


def _parity(v):
    import numpy as np
    v = v.astype(np.uint64)
    for sh in (32, 16, 8, 4, 2, 1):
        v = v ^ (v >> np.uint64(sh))
    return (v & np.uint64(1)).astype(np.int64)


def support_rows(tq, n_spatial, n_electrons, mapping, ks=None):
    """Per generator, the rows its support-only update reads and writes
    (pair representatives and partners), from the library's support form;
    a list over the pool, or a dict over `ks` when given."""
    import numpy as np

    def insert_zero(v, b):
        return ((v >> b) << (b + 1)) | (v & ((1 << b) - 1))

    N = 2 * n_spatial
    f = tq.pool_support_forms(n_spatial, n_electrons, mapping)
    x = tq.pauli_pool(n_spatial, n_electrons, mapping)[0]
    out = [] if ks is None else {}
    for k in (range(x.size) if ks is None else ks):
        m = int(f["m"][k])
        r = insert_zero(np.arange(1 << (N - m - 1), dtype=np.int64), int(f["rep_pos"][k]))
        for p in f["pivots"][k, :m]:
            r = insert_zero(r, int(p))
        for i, p in enumerate(f["pivots"][k, :m]):
            r = r | ((((int(f["target"][k]) >> i) & 1) ^ _parity(r & int(f["masks"][k, i]))) << int(p))
        rows = np.concatenate([r, r ^ int(x[k])])
        if ks is None:
            out.append(rows)
        else:
            out[k] = rows
    return out


def measure_support(tq, ctx, pool, n_states, reps=50):
    """The headline update with the support-only kernel: the same 8192
    complex64 14-qubit states, generators and angles; only each generator's
    support rows are read and written (in place), the norm carried."""
    import numpy as np
    import torch

    import synth
    D = 1 << NQ
    prep_k, prep_th, k, th = synth.t5_batch(n_states, pool.M, seed=synth.SEED_T5_BATCH)
    hf = tq.hf_index(NQ, N_ELECTRONS, MAPPING)
    psi = torch.zeros((n_states, D), dtype=torch.complex64, device="cuda")
    psi[:, hf] = 1.0
    dn = torch.ones(n_states, dtype=torch.float64, device="cuda")
    for j in range(prep_k.shape[1]):
        tq.evolve_taylor5_batch_support(ctx, pool, psi, torch.as_tensor(prep_k[:, j].copy()).cuda(),
                                        torch.as_tensor(prep_th[:, j].copy()).cuda(), dn)
    dk = torch.as_tensor(k).cuda()
    dth = torch.as_tensor(th).cuda()
    fetch0 = ctx.l2_fetch()
    per = {}
    for fetch in (0, 32):
        ctx.set_l2_fetch(fetch)
        for ppt in (1, 2, 4, 8, -1, -2, -4, -8):
            ctx.set_support_schedule(tq.TQ_C64, ppt)
            for _ in range(3):
                tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, dn)
            ctx.trace(True)
            for _ in range(reps):
                tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, dn)
            rep = ctx.trace_report()
            ctx.trace(False)
            n_l, ms = rep["taylor5_support"]
            nc, ncms = rep.get("norm_carry", (1, 0.0))
            per[(fetch, ppt)] = (ms / n_l, ncms / nc)
    best_f, best = min(per, key=lambda fp: per[fp][0] + per[fp][1])
    ctx.set_support_schedule(tq.TQ_C64, best)
    # the same launch without the norm (the finish's share of the time)
    ctx.set_l2_fetch(best_f)
    ctx.trace(True)
    for _ in range(reps):
        tq.evolve_taylor5_batch_support(ctx, pool, psi, dk, dth, None)
    rep = ctx.trace_report()
    ctx.trace(False)
    n_l, ms_nn = rep["taylor5_support"]
    ms_no_norm = ms_nn / n_l
    ctx.set_l2_fetch(0)
    ms, ncms = per[(best_f, best)]
    rows = support_rows(tq, N_SPATIAL, N_ELECTRONS, MAPPING)
    n_rows = np.array([r.size for r in rows], dtype=np.float64)
    n_sect = np.array([np.unique(r >> 2).size for r in rows], dtype=np.float64)   # 32-byte sectors
    alg = float((2 * 8 * n_rows[k]).sum() + 16 * n_states)          # amplitudes in + out, norm in + out
    sect = float((2 * 32 * n_sect[k]).sum() + 16 * n_states)
    peak, _ = peaks()
    gbs = alg / (ms * 1e-3) / 1e9
    return {"workload": f"{n_states} complex64 states of 14 qubits (the headline batch), own generator and angle "
                        "each, support rows only, norm carried",
            "kernel": "k_taylor5_support<float>", "pairs_per_thread": best,
            "l2_fetch_bytes": best_f or fetch0, "l2_fetch_default": fetch0,
            "ms_by_fetch_and_schedule": {f"{f or fetch0}B/{p}": v[0] + v[1] for (f, p), v in per.items()},
            "ms_per_launch": ms, "norm_carry_ms": ncms, "ms_per_launch_without_norm": ms_no_norm,
            "updates_per_s": n_states / ((ms + ncms) * 1e-3),
            "algorithmic_bytes_per_launch": alg, "sector_bytes_per_launch": sect,
            "mean_support_rows": float(n_rows[k].mean()), "achieved_gbs": gbs, "peak_gbs": peak,
            "frac": gbs / peak, "sector_gbs": sect / (ms * 1e-3) / 1e9,
            "sector_frac": sect / (ms * 1e-3) / 1e9 / peak,
            "norms_finite": bool(torch.isfinite(dn).all().item())}


def measure_fp64_single(tq, ctx, pool, k, th, reps=2000):
    """The plain float64 single-instance form: one 14-qubit complex128 state
    per call, renormalised after each update (as the ADAPT step does)."""
    import torch
    st = tq.State(ctx, NQ, tq.TQ_C128)
    tq.state_set_hf(st, N_ELECTRONS, MAPPING)
    for i in range(20):
        tq.evolve_taylor5(ctx, pool, int(k[i]), float(th[i]), st, renormalize=True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    kl = [int(x) for x in k[:reps]]
    tl = [float(x) for x in th[:reps]]
    n = len(kl)
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    l0 = ctx.launches()
    e0.record()
    t0 = time.perf_counter()
    for i in range(reps):
        tq.evolve_taylor5(ctx, pool, kl[i % n], tl[i % n], st, renormalize=True, stream=stream)
    host_s = time.perf_counter() - t0     # the host's issue time (the GPU runs behind it)
    e1.record()
    torch.cuda.synchronize()
    launches = (ctx.launches() - l0) / reps
    ms = e0.elapsed_time(e1) / reps
    # the kernel alone (CUDA events around each launch)
    ctx.trace(True)
    for i in range(200):
        tq.evolve_taylor5(ctx, pool, kl[i % n], tl[i % n], st, renormalize=True)
    rep = ctx.trace_report()
    ctx.trace(False)
    kn = "taylor5_single" if "taylor5_single" in rep else "taylor5_pair"
    # the device time per update without the per-call launch: 100 calls
    # captured in one CUDA graph, replayed
    graph_us = None
    try:
        g = torch.cuda.CUDAGraph()
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.graph(g, stream=side):
            for i in range(100):
                tq.evolve_taylor5(ctx, pool, kl[i % n], tl[i % n], st, renormalize=True, stream=side)
        g.replay()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(20):
            g.replay()
        e1.record()
        torch.cuda.synchronize()
        graph_us = 1e3 * e0.elapsed_time(e1) / 2000
    except Exception as exc:   # capture not possible here: report it, keep the rest
        graph_us = f"unavailable: {exc}"
    return {"workload": "one 14-qubit complex128 state, evolve_taylor5 with renormalisation per call, "
                        "back-to-back calls on one stream from Python",
            "updates_per_s": 1e3 / ms, "us_per_update": ms * 1e3,
            "host_issue_us_per_call": 1e6 * host_s / reps,
            "launches_per_update": launches, "kernel": kn,
            "kernel_us_per_update": 1e3 * sum(v[1] for v in rep.values()) / 200,
            "kernel_us_per_update_note": "CUDA events around each launch (their own overhead included)",
            "device_us_per_update_graph": graph_us,
            "device_us_per_update_graph_note": "100 calls captured in one CUDA graph and replayed: the kernel's "
                                               "device time with no per-call launch"}


def measure_spmv(tq, ctx, nq):
    """Energy (fused SpMV + float64 dots) on a Hamiltonian larger than L2, every schedule timed."""
    import numpy as np
    import torch

    import synth
    n = nq // 2
    ne = synth.electrons_for(n)
    ints = synth.integrals(n, synth.SEED_CATALOGUE_BASE + 12)
    t0 = time.perf_counter()
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, 1, tq.TQ_C64)
    build_s = time.perf_counter() - t0
    D = 1 << nq
    st = tq.State(ctx, nq, tq.TQ_C64)
    tq.state_set_hf(st, ne, 1)
    pool = tq.build_pool(ctx, n, ne, 1)
    for k in range(0, pool.M, max(1, pool.M // 8)):
        tq.evolve_taylor5(ctx, pool, k, 0.1, st, renormalize=True)
    best, _ = tq.autotune_spmv(ctx, ham, st)
    reps = 20

    def timed(sched):
        ctx.set_spmv_schedule(sched)
        for _ in range(3):
            tq.energy(ctx, ham, st)
        ctx.trace(True)
        for _ in range(reps):
            e = tq.energy(ctx, ham, st)
        rep = ctx.trace_report()
        ctx.trace(False)
        n_l, t = rep["energy_xell" if sched == tq.TQ_SPMV_XELL else "energy_csr"]
        return t / n_l, e

    per_sched = {}
    for sched in (4, 8, 16, 32, tq.TQ_SPMV_XELL):
        per_sched["xell" if sched == tq.TQ_SPMV_XELL else f"csr_lanes_{sched}"] = timed(sched)[0]
    ms, e = timed(best)
    nb, npairs = tq.ham_xell(ham)[:2]
    # what the method must move (CSR of float32 values, float64 diagonal, state in, w out)
    alg = 4 * (D + 1) + 8 * ham.nnz + 8 * D + 8 * D + 16 * D
    # what the chosen layout moves
    if best == tq.TQ_SPMV_XELL:
        layout = 4 * (nb + 1) + (4 + 8 * 4) * npairs + 8 * D + 8 * D + 16 * D
        kernel = "k_energy_xell_tma<float,float>"
    else:
        layout = alg
        kernel = f"k_energy_csr<float,float,{best}>"
    peak, _ = peaks()
    gbs = alg / (ms * 1e-3) / 1e9
    # the matrix-free energy (each row's terms evaluated from the X-mask
    # groups, no matrix stored): one float64 add per term and row and two
    # FMAs per off-diagonal group and row, against the measured FMA rate
    tq.energy_matrix_free(ctx, ham, st)
    ctx.trace(True)
    for _ in range(3):
        e_mf = tq.energy_matrix_free(ctx, ham, st)
    rep = ctx.trace_report()
    ctx.trace(False)
    n_mf, t_mf = rep["energy_matrix_free"]
    ms_mf = t_mf / n_mf
    terms = float(D) * ham.n_pauli
    g_off = ham.n_xgroups - 1                     # the groups less the diagonal (x = 0) one
    fp64_ops = terms + 2.0 * D * g_off
    fma_rate = tq.fp64_fma_rate(ctx)
    mf = {"kernel": "k_energy_mf<float>", "ms_per_energy": ms_mf, "pauli_terms": ham.n_pauli,
          "x_mask_groups": ham.n_xgroups, "term_evaluations": terms,
          "term_evaluations_per_s": terms / (ms_mf * 1e-3), "fp64_lane_ops": fp64_ops,
          "bound": "fp64 (an add per term and row, two FMAs per group and row)",
          "fp64_peak_lane_ops_per_s": fma_rate, "fp64_frac": fp64_ops / (ms_mf * 1e-3) / fma_rate,
          "energy_abs_diff_vs_stored_layout": abs(e_mf - e)}
    return {"workload": f"energy of a {nq}-qubit BK Hamiltonian (synthetic, {n} orbitals, "
                        f"{ne} electrons), complex64 state, float32 off-diagonal values + float64 diagonal",
            "kernel": kernel, "schedule": "xell" if best == tq.TQ_SPMV_XELL else f"csr_lanes_{best}",
            "nnz": ham.nnz, "xell_pairs": npairs, "hamiltonian_bytes": ham.device_bytes,
            "build_s": build_s, "ms_per_energy": ms, "ms_per_schedule": per_sched,
            "algorithmic_bytes": alg, "layout_bytes": layout, "achieved_gbs": gbs,
            "layout_gbs": layout / (ms * 1e-3) / 1e9, "peak_gbs": peak, "frac": gbs / peak,
            "energy": e, "l2_policy": "Hamiltonian larger than L2", "matrix_free": mf}


def measure_sector(tq, ctx, n_states=65536, reps=20):
    """Batched Taylor-5 and energies in the sector-restricted basis.

    The 14-qubit workload of the headline (7 orbitals, 6 electrons, BK,
    strongly correlated) restricted to its Hartree-Fock sector (3 alpha + 3
    beta electrons: 1225 amplitudes instead of 16384); n_states complex64
    states, each with its own generator and angle (inputs larger than L2)."""
    import numpy as np
    import torch

    import synth
    ints, ne = synth.config2()
    n = ints.n_spatial
    na, nb = (ne + 1) // 2, ne // 2
    mp = 1
    pool = tq.build_pool_sector(ctx, n, ne, mp, na, nb)
    dim = pool.dim
    rng = np.random.default_rng(synth.SEED_T5_BATCH)
    k = torch.as_tensor(rng.integers(0, pool.M, size=n_states).astype(np.int32)).cuda()
    th = torch.as_tensor(rng.normal(0.0, 0.1, size=n_states)).cuda()
    g = torch.Generator("cuda").manual_seed(5)
    psi = torch.randn(n_states, dim, dtype=torch.complex64, device="cuda", generator=g)
    psi /= torch.linalg.vector_norm(psi, dim=1, keepdim=True)
    n2 = torch.zeros(n_states, dtype=torch.float64, device="cuda")
    for _ in range(3):
        tq.evolve_taylor5_batch(ctx, pool, psi, k, th, n2)
    ctx.trace(True)
    for _ in range(reps):
        tq.evolve_taylor5_batch(ctx, pool, psi, k, th, n2)
    rep = ctx.trace_report()
    ctx.trace(False)
    n_l, ms = rep["taylor5_sector"]
    ms /= n_l
    nr, nrms = rep.get("norm_reduce", (1, 0.0))      # the shared-memory update finishes norms itself
    # every amplitude read and written once (the state goes through shared
    # memory); the generator tables (int32 + int8 per row and op) stay in L2
    alg = 2.0 * dim * 8
    peak, _ = peaks()
    gbs = alg * n_states / (ms * 1e-3) / 1e9
    out = {"workload": f"{n_states} complex64 states of the 14-qubit BK Hamiltonian's ({na}, {nb}) sector "
                       f"({dim} amplitudes), own generator and angle each",
           "kernel": "k_taylor5_sector_smem<float>", "ms_per_launch": ms, "norm_reduce_ms": nrms / nr,
           "updates_per_s": n_states / ((ms + nrms / nr) * 1e-3),
           "algorithmic_bytes_per_update": alg, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
           "norms_finite": bool(torch.isfinite(n2).all().item())}
    # energies: 14 and 18 qubits in their Hartree-Fock sectors
    for nq_, seed in ((14, None), (18, synth.SEED_CATALOGUE_BASE + 12)):
        ints_ = ints if seed is None else synth.integrals(nq_ // 2, seed)
        ne_ = ne if seed is None else synth.electrons_for(nq_ // 2)
        a_, b_ = (ne_ + 1) // 2, ne_ // 2
        ham = tq.build_hamiltonian_sector(ctx, ints_.h, ints_.g, ints_.e_const, mp, tq.TQ_C64, a_, b_)
        st = tq.State(ctx, nq_, tq.TQ_C64, sector=(a_, b_))
        tq.state_set_hf(st, ne_, mp)
        tq.autotune_spmv(ctx, ham, st)
        for _ in range(3):
            tq.energy(ctx, ham, st)
        ctx.trace(True)
        for _ in range(reps):
            tq.energy(ctx, ham, st)
        r = ctx.trace_report()
        ctx.trace(False)
        nl, t = r["energy_csr"]
        out[f"energy_{nq_}q"] = {"dim": ham.dim, "nnz": ham.nnz, "ms_per_energy": t / nl}
    ctx.set_spmv_schedule(tq.TQ_SPMV_XELL)
    return out


def measure_vqe(tq, ctx, reps=20):
    """ADAPT-VQE with re-optimised angles: one energy + adjoint gradient of a
    20-factor ansatz at 14 qubits (c64 and c128; the oracle timed beside it),
    and a whole run on the 12-qubit workload (BK, eps 1e-3, c128)."""
    import numpy as np

    import synth
    out = {}
    ints, ne = synth.config2()
    n = ints.n_spatial
    rng = np.random.default_rng(11)
    pool = tq.build_pool(ctx, n, ne, 1)
    ops = rng.integers(0, pool.M, size=20).astype(np.int32)
    th = rng.normal(0, 0.2, size=20)
    for name, prec in (("c64", tq.TQ_C64), ("c128", tq.TQ_C128)):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, 1, prec)
        st = tq.State(ctx, 2 * n, prec)
        tq.state_set_hf(st, ne, 1)
        for _ in range(3):
            tq.ansatz_energy_grad(ctx, ham, pool, st, ops, th)
        t0 = time.perf_counter()
        for _ in range(reps):
            tq.ansatz_energy_grad(ctx, ham, pool, st, ops, th)
        out[f"energy_grad_20_ops_14q_{name}_ms"] = 1e3 * (time.perf_counter() - t0) / reps
    # the oracle on the same 20-factor evaluation (one host thread)
    from oracle import adapt as oadapt, vqe as ovqe
    sysm = oadapt.build_system(ints, ne, 1)
    psi0 = oadapt.hf_state(2 * n, ne, 1)
    t0 = time.perf_counter()
    ovqe.energy_and_gradient(sysm, list(ops), th, psi0)
    out["oracle_energy_grad_20_ops_14q_ms"] = 1e3 * (time.perf_counter() - t0)
    # a whole run
    ints1, ne1 = synth.config1()
    ham = tq.build_hamiltonian(ctx, ints1.h, ints1.g, ints1.e_const, 1, tq.TQ_C128)
    pool1 = tq.build_pool(ctx, ints1.n_spatial, ne1, 1)
    st = tq.State(ctx, 2 * ints1.n_spatial, tq.TQ_C128)
    tq.state_set_hf(st, ne1, 1)
    t0 = time.perf_counter()
    ops1, th1, en1 = tq.adapt_vqe(ctx, ham, pool1, st, 1e-3, max_ops=20, gtol=1e-6)
    out["adapt_vqe_12q"] = {"seconds": time.perf_counter() - t0, "operators": int(ops1.size),
                            "final_energy": float(en1[-1]) if en1.size else None}
    out["workload"] = ("energy + adjoint gradient of a 20-factor Taylor-5 ansatz of the 14-qubit BK "
                       "Hamiltonian from HF; ADAPT-VQE (BFGS on every angle) on the 12-qubit BK workload")
    return out


def measure_io(tq, ctx):
    """FCIDUMP read of 13 orbitals and a checkpoint of a 24-qubit complex64 state."""
    import os
    import tempfile

    import synth
    out = {}
    with tempfile.TemporaryDirectory() as d:
        ints = synth.integrals(13, 7)
        path = os.path.join(d, "FCIDUMP")
        tq.write_fcidump(path, ints.h, ints.g, 0.0, 12)
        t0 = time.perf_counter()
        tq.read_fcidump(path)
        out["fcidump_13_orbitals_read_ms"] = 1e3 * (time.perf_counter() - t0)
        st = tq.State(ctx, 24, tq.TQ_C64)
        tq.state_set_hf(st, 12, tq.TQ_BK)
        sp = os.path.join(d, "state.bin")
        t0 = time.perf_counter()
        tq.state_save(st, sp)
        t1 = time.perf_counter()
        tq.state_load(st, sp)
        t2 = time.perf_counter()
        mb = (1 << 24) * 8 / 1e6
        out["checkpoint_24q_c64"] = {"mbytes": mb, "save_gbs": mb / 1e3 / (t1 - t0), "load_gbs": mb / 1e3 / (t2 - t1)}
    return out


def measure_families(tq):
    """Algorithm 1 (commuting families) on the 18-qubit pool, both relations (host)."""
    out = {}
    for name, mode in (("full", tq.TQ_COMMUTE_FULL), ("qubit_wise", tq.TQ_COMMUTE_QWC)):
        t0 = time.perf_counter()
        fam, _, k = tq.pool_families_host(9, 8, tq.TQ_BK, mode)
        out[name] = {"pool_size": int(fam.size), "families": k, "ms": 1e3 * (time.perf_counter() - t0)}
    return {"workload": "pool of 9 orbitals, 8 electrons, BK (560 generators)", **out}


def measure_serving_process(device, seconds, rate, sweep=""):
    """The request loop measured in a process of its own (as a server runs):
    `bench.py --section serving` on the same device, its JSON line parsed."""
    env = dict(os.environ, LOCAL_RANK=str(device), RANK="0", WORLD_SIZE="1")
    cmd = [sys.executable, os.path.join(ROOT, "bench.py"), "--section", "serving",
           "--serve-seconds", str(seconds), "--serve-rate", str(rate), "--serve-sweep", sweep]
    r = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=seconds + 900)
    if r.returncode != 0:
        return {"error": f"serving process exited {r.returncode}: {r.stderr.strip()[-300:]}"}
    out = json.loads(r.stdout.strip().splitlines()[-1])
    out["process"] = "own process (bench.py --section serving)"
    return out


def _serve_stream(tq, srv, arr, pools_m, n_cat, timeout_s):
    """Submits a timed arrival list from a thread while polling completions;
    returns latency and throughput figures."""
    import numpy as np
    lag = []
    ticks0 = srv.stats()["ticks"]

    def submitter():
        start = time.perf_counter()
        for i, a in enumerate(arr):
            dt = start + a.t - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            lag.append(time.perf_counter() - start - a.t)
            srv.submit(a.kind, a.session, a.op % pools_m[a.session % n_cat], a.theta, i)

    th = threading.Thread(target=submitter)
    th.start()
    got = []
    deadline = time.perf_counter() + timeout_s
    while len(got) < len(arr) and time.perf_counter() < deadline:
        got += srv.poll(5000)
    th.join()
    ticks = srv.stats()["ticks"] - ticks0
    if not got:
        return {"requests": len(arr), "completed": 0}
    lat = np.array([c["t_done"] - c["t_submit"] for c in got]) * 1e3
    span = max(c["t_done"] for c in got) - min(c["t_submit"] for c in got)
    by_kind = {}
    for name, kind in (("evolve", 0), ("energy", 1), ("gradients", 2)):
        lk = np.array([c["t_done"] - c["t_submit"] for c in got if c["kind"] == kind]) * 1e3
        if lk.size:
            by_kind[name] = {"n": int(lk.size), "p50_ms": float(np.percentile(lk, 50)),
                             "p99_ms": float(np.percentile(lk, 99))}
    return {"requests": len(arr), "completed": len(got),
            "failed": int(sum(c["status"] != 0 for c in got)),
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "throughput_rps": len(got) / span,
            "ticks": ticks, "mean_batch": len(got) / max(1, ticks),
            "submit_lag_p99_ms": float(np.percentile(np.array(lag) * 1e3, 99)),
            "by_kind": by_kind}


def measure_serving(tq, device, seconds, rate, sweep=(), sweep_seconds=5.0):
    """Poisson request stream into the continuous-batching request loop, then
    (same server, same resident sessions) a sweep of offered rates up to
    saturation: it stops once p99 passes 10 ms, a request fails or the
    achieved rate falls below 80 % of the offered one."""
    import synth
    ctx = tq.Context(device)                  # the server owns this context
    srv = tq.Server(ctx, tq.TQ_C64, hbm_budget=16 << 30, max_batch=1024)
    cat = synth.catalogue()
    pools_m = []
    t0 = time.perf_counter()
    for n, ne, mp_, seed in cat:
        ints = synth.integrals(n, seed)
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp_, tq.TQ_C64)
        pool = tq.build_pool(ctx, n, ne, mp_)
        srv.add_hamiltonian(ham, pool)
        pools_m.append(pool.M)
    n_sessions = 256
    for j in range(n_sessions):
        n, ne, mp_, _ = cat[j % len(cat)]
        srv.add_session(j % len(cat), ne, mp_)
    build_s = time.perf_counter() - t0
    srv.start()
    out = {"workload": (f"Poisson arrivals at {rate:.0f}/s for {seconds:.0f} s, 50% evolve / 30% energy / "
                        "20% gradients, 256 resident sessions over 16 resident Hamiltonians and pools of "
                        "12-18 qubits (synthetic, seeds 2000+j), complex64 with float64 reductions")}
    if seconds > 0:
        out.update(_serve_stream(tq, srv, synth.arrivals(rate, seconds, n_sessions), pools_m, len(cat),
                                 seconds + 60))
    sw = []
    for r_ in sweep:
        res = _serve_stream(tq, srv, synth.arrivals(r_, sweep_seconds, n_sessions), pools_m, len(cat),
                            sweep_seconds + 30)
        res = {"offered_rps": r_, "seconds": sweep_seconds, **res}
        sw.append(res)
        if (res.get("completed", 0) < res["requests"] or res.get("failed", 0) > 0 or res["p99_ms"] > 10.0
                or res["throughput_rps"] < 0.8 * r_):
            break
    if sw:
        out["sweep"] = sw
        out["sweep_note"] = ("the same server and sessions, one Poisson stream per offered rate; mean_batch is "
                             "requests per tick of the loop")
    srv.stop()
    out["build_s"] = build_s
    return out


def measure_trajectories(tq, ctx, n_traj):
    """Independent ADAPT trajectories of 10-16 qubits, one graph replay per run."""
    import numpy as np
    import torch

    import synth
    trajs = synth.trajectories(n_traj)
    t0 = time.perf_counter()
    hams, pools = [], []
    for tr in trajs:
        ints = synth.integrals(tr.n_spatial, tr.seed)
        hams.append(tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, tr.mapping, tq.TQ_C64))
        pools.append(tq.build_pool(ctx, tr.n_spatial, tr.n_electrons, tr.mapping))
    b = tq.Batch(ctx, hams, pools, [t.n_electrons for t in trajs], [t.mapping for t in trajs],
                 [t.thetas for t in trajs], 1e-3)
    build_s = time.perf_counter() - t0
    lpr, _ = b.autotune()
    b.run(use_graph=True)          # warm: captures the graph
    torch.cuda.synchronize()
    runs = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(runs):
        b.run(use_graph=True)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / runs
    res = b.results()
    iters = sum(r["n_iter"] for r in res)
    # one more, untimed run without the graph, traced per kernel
    ctx.trace(True)
    b.run(use_graph=False)
    split = ctx.trace_report()
    ctx.trace(False)
    # the energy passes' algorithmic bytes: per pass the Hamiltonian in the
    # chosen layout (XOR-ELL: block offsets, 4-byte masks, 8 float32 values
    # per pair; CSR: offsets, columns, values) plus the float64 diagonal,
    # psi read and w = H psi written (float32 pairs)
    e_bytes = 0.0
    for r_, h_ in zip(res, hams):
        D_ = 1 << h_.n_qubits
        if lpr == tq.TQ_SPMV_XELL:
            nb_, np_, _, _, _ = tq.ham_xell(h_)
            hb = 4.0 * (nb_ + 1) + np_ * (4 + 8 * 4)
        else:
            hb = 4.0 * (D_ + 1) + 8.0 * h_.nnz
        e_bytes += r_["n_iter"] * (hb + D_ * (8 + 8 + 8))
    peak, _ = peaks()
    e_ms = split.get("batch_energy", (1, float("nan")))[1]
    return {"workload": f"{n_traj} ADAPT trajectories, qubits uniform over 10-16, JW/BK 50/50, "
                        "own integrals (seeds 1000+i), angle lists of 1-30 from N(0,0.1), eps 1e-3, "
                        "complex64 with float64 reductions",
            "build_s": build_s, "lanes_per_row": lpr, "ms_per_run": ms,
            "iterations_per_run": iters, "iterations_per_s": iters / (ms * 1e-3),
            "converged": int(sum(r["converged"] for r in res)),
            "graph_launches_per_run": 4 * max(len(t.thetas) for t in trajs) + 1,
            "kernel_ms_untimed_direct_run": {k: round(v[1], 3) for k, v in split.items()},
            "energy_roofline": {"layout": "XOR-ELL" if lpr == tq.TQ_SPMV_XELL else f"CSR, {lpr} lanes per row",
                                "bytes_per_run": e_bytes, "ms": e_ms,
                                "achieved_gbs": e_bytes / (e_ms * 1e-3) / 1e9,
                                "frac": e_bytes / (e_ms * 1e-3) / 1e9 / peak}}


# ------------------------------------------- precision against the oracle

def _dev_to_host(ptr, n, typestr):
    """Copy n elements at a device pointer into a numpy array."""
    import numpy as np
    import torch

    class _A:
        __cuda_array_interface__ = {"shape": (int(n),), "typestr": typestr, "data": (int(ptr), False),
                                    "version": 3}
    if n == 0:
        return np.zeros(0, dtype=np.dtype(typestr))
    t = torch.as_tensor(_A(), device="cuda")
    torch.cuda.synchronize()
    return t.cpu().numpy().copy()


def _fid(a, b):
    import numpy as np
    return float(abs(np.vdot(a, b)) ** 2 / (np.vdot(a, a).real * np.vdot(b, b).real))


def _oracle_headline_worker(args):
    """The oracle's states for sampled members of the headline batch: each
    prepared from HF by its three rotations, then its own update applied
    n_apply times (the number of launches the bench ran on the batch)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    idx, n_states, seed, n_apply = args
    import synth
    from oracle import adapt, evolve, pauli
    exc, pps = pauli.pool_pauli(N_SPATIAL, N_ELECTRONS, MAPPING)
    prep_k, prep_th, k, th = synth.t5_batch(n_states, len(exc), seed=seed)
    out = []
    for b in idx:
        psi = adapt.hf_state(NQ, N_ELECTRONS, MAPPING)
        for j in range(prep_k.shape[1]):
            psi = evolve.taylor5(pauli.pauli_to_csr(pps[int(prep_k[b, j])]), psi, prep_th[b, j])
        A = pauli.pauli_to_csr(pps[int(k[b])])
        for _ in range(n_apply):
            psi = evolve.taylor5(A, psi, th[b])
        out.append(psi)
    return out


def headline_fidelity(psi, dn, idx, n_states, seed, n_apply, relabel):
    """The headline batch's sampled states against the oracle after the
    same updates: fidelity, relative L2 error and the carried norm's error.
    relabel[b] is the index of the oracle's basis state b in the GPU layout."""
    import numpy as np
    cores = min(len(idx), os.cpu_count() or 1)
    chunks = [list(idx[i::cores]) for i in range(cores)]
    with mp.get_context("spawn").Pool(cores) as p:
        res = p.map(_oracle_headline_worker, [(c, n_states, seed, n_apply) for c in chunks])
    ref = {}
    for c, r in zip(chunks, res):
        for b, v in zip(c, r):
            ref[b] = v
    fids, rels, nerr = [], [], []
    got = psi[list(idx)].cpu().numpy()[:, relabel].astype(np.complex128)
    norms = dn[list(idx)].cpu().numpy()
    carry = []
    for i, b in enumerate(idx):
        o = ref[b]
        fids.append(_fid(got[i], o))
        rels.append(float(np.linalg.norm(got[i] - o) / np.linalg.norm(o)))
        nerr.append(abs(float(norms[i]) - float(np.vdot(o, o).real)) / float(np.vdot(o, o).real))
        own = float(np.vdot(got[i], got[i]).real)
        carry.append(abs(float(norms[i]) - own) / own)
    return {"sampled_states": len(idx), "updates_per_state": n_apply + 3,
            "min_fidelity": min(fids), "max_one_minus_fidelity": max(1.0 - f for f in fids),
            "max_rel_l2": max(rels), "max_norm2_rel_err_vs_oracle": max(nerr),
            "max_carried_norm2_rel_err_vs_own_state": max(carry),
            "reference": "oracle (complex128 SciPy CSR chain of Eqs. (7)-(8)) after the same 3 preparation "
                         "and n_apply timed updates of each sampled state, no renormalisation"}


def measure_precision(tq, ctx, steps=12):
    """Each result of the complex64 form against the float64 oracle, on the
    14-qubit BK workload (strongly correlated integrals, pool of 204): ADAPT
    steps with the line search from HF run on the GPU in complex64 and in
    complex128.  After every step the oracle takes the GPU's operator and
    angle (teacher forcing) from its own complex128 state; the step's
    energy, gradient maximum and angle are compared with the oracle's at that
    state, and the GPU state after the update with the oracle's."""
    import numpy as np

    import synth
    from oracle import adapt as oadapt
    from oracle import evolve as oevolve
    ints, ne = synth.config2()
    sysm = oadapt.build_system(ints, ne, MAPPING)
    out = {"workload": "ADAPT with the line search from HF, 14 q BK, config-2 integrals (seed 2), pool of 204; "
                       "oracle teacher-forced with the GPU's operator and angle",
           "steps": steps}
    pool = tq.build_pool(ctx, ints.n_spatial, ne, MAPPING)
    for prec, name in ((tq.TQ_C64, "c64"), (tq.TQ_C128, "c128")):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, MAPPING, prec)
        st = tq.State(ctx, NQ, prec)
        tq.state_set_hf(st, ne, MAPPING)
        psi_o = oadapt.hf_state(NQ, ne, MAPPING)
        rows = []
        for it in range(steps):
            e_o, _ = oadapt.energy(sysm.H, psi_o)
            g_o = oadapt.gradients(sysm.H, sysm.pool, psi_o)
            k_o, gmax_o = oadapt.select(g_o, oadapt.FP64 if prec == tq.TQ_C128 else oadapt.C64)
            r = tq.adapt_step(ctx, ham, pool, st, 0.0, float("nan"))
            k = r["selected"]
            th_o = oadapt.line_search(oadapt.line_search_coefficients(sysm.H, sysm.pool[k], psi_o))
            psi_o = oevolve.normalise(oevolve.taylor5(sysm.pool[k], psi_o, r["theta"]))
            got = st.numpy().astype(np.complex128)
            e_after = tq.energy(ctx, ham, st)
            rows.append({"step": it, "selected": k, "oracle_selected": k_o,
                         "selection_tie": bool(abs(abs(g_o[k]) - gmax_o) <= 1e-5),
                         "energy_err_ha": r["energy"] - e_o, "max_grad_err": r["max_grad"] - gmax_o,
                         "theta_err": r["theta"] - th_o,
                         "state_fidelity": _fid(got, psi_o),
                         "state_rel_l2": float(np.linalg.norm(got - psi_o) / np.linalg.norm(psi_o)),
                         "energy_after_err_ha": e_after - oadapt.energy(sysm.H, psi_o)[0]})
        out[name] = {"per_step": rows,
                     "max_abs_energy_err_ha": max(abs(x["energy_err_ha"]) for x in rows),
                     "max_abs_energy_after_err_ha": max(abs(x["energy_after_err_ha"]) for x in rows),
                     "min_state_fidelity": min(x["state_fidelity"] for x in rows),
                     "max_abs_theta_err": max(abs(x["theta_err"]) for x in rows),
                     "selections_equal_or_tied": sum(x["selected"] == x["oracle_selected"] or x["selection_tie"]
                                                     for x in rows),
                     "final_energy": rows[-1]["energy_after_err_ha"] + oadapt.energy(sysm.H, psi_o)[0]}
    out["c64_minus_c128_final_energy_ha"] = out["c64"]["final_energy"] - out["c128"]["final_energy"]
    out["bounds"] = {"c64_energy_ha": 1e-6, "c64_fidelity": 0.999999, "c128_energy_ha": 1e-10}
    return out


def measure_m0(tq, ctx, reps=200):
    """The plain method at 8 qubits (JW, complex128, one ADAPT step from HF at
    theta = 0.05): the GPU step and the oracle's, timed, and the result
    against the dense exponential (eigendecomposition of the 256 x 256
    generator)."""
    import numpy as np

    import synth
    from oracle import adapt as oadapt
    from oracle import evolve as oevolve
    ints, ne = synth.config0()
    mp_ = 0
    th = 0.05
    sysm = oadapt.build_system(ints, ne, mp_)
    psi0 = oadapt.hf_state(8, ne, mp_)
    ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp_, tq.TQ_C128)
    pool = tq.build_pool(ctx, ints.n_spatial, ne, mp_)
    st = tq.State(ctx, 8, tq.TQ_C128)
    for _ in range(10):
        tq.state_set_hf(st, ne, mp_)
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3, th)
    t0 = time.perf_counter()
    for _ in range(reps):
        tq.state_set_hf(st, ne, mp_)
        r = tq.adapt_step(ctx, ham, pool, st, 1e-3, th)
    t_gpu = (time.perf_counter() - t0) / reps
    got = st.numpy()
    n_o = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < 1.0:
        ref, psi_ref = oadapt.adapt_step(sysm, psi0, 1e-3, theta=th)
        n_o += 1
    t_o = (time.perf_counter() - t0) / n_o
    ex = oevolve.expm_dense(sysm.pool[r["selected"]], th) @ psi0
    ex = ex / np.linalg.norm(ex)
    return {"workload": "config 0: 8 qubits (4 orbitals, 4 electrons, seed 0), JW, complex128, one ADAPT step "
                        "from HF at theta = 0.05 (energy, 26 gradients, selection, Taylor-5, renormalisation)",
            "gpu_ms_per_step": 1e3 * t_gpu, "gpu_api": "tq_state_set_hf + tq_adapt_step (host result, synchronous)",
            "oracle_ms_per_step": 1e3 * t_o, "oracle_cores": 1,
            "selected": r["selected"], "oracle_selected": ref.selected,
            "energy_err_vs_oracle_ha": r["energy"] - ref.energy,
            "state_rel_l2_vs_oracle": float(np.linalg.norm(got - psi_ref) / np.linalg.norm(psi_ref)),
            "state_err_vs_dense_expm": float(np.linalg.norm(got - ex)),
            "truncation_bound": th ** 6 / 720,
            "fidelity_vs_dense_expm": _fid(got, ex),
            "energy_after_vs_dense_expm_ha": tq.energy(ctx, ham, st) - oadapt.energy(sysm.H, ex)[0]}


def measure_m1(tq, ctx, n_iter=20):
    """The plain method at 12 qubits: 20 ADAPT iterations (eps = 1e-3, line
    search) from HF under JW and BK, on the GPU in complex128 and in
    complex64 with float64 reductions (one tq_adapt_run call each), and the
    oracle's float64 trajectory, all timed."""
    import numpy as np

    import synth
    from oracle import adapt as oadapt
    ints, ne = synth.config1()
    out = {"workload": "config 1: 12 qubits (6 orbitals, 8 electrons, seed 1), pool of 92, 20 ADAPT iterations "
                       "from HF, eps 1e-3, line-search angles"}
    for mp_, mname in ((0, "JW"), (1, "BK")):
        sysm = oadapt.build_system(ints, ne, mp_)
        t0 = time.perf_counter()
        res_o, psi_o = oadapt.trajectory(sysm, oadapt.hf_state(12, ne, mp_), 1e-3, n_iter=n_iter)
        t_o = time.perf_counter() - t0
        e_o = [r.energy for r in res_o]
        row = {"oracle": {"seconds": t_o, "cores": 1, "iterations": len(res_o),
                          "final_energy": oadapt.energy(sysm.H, psi_o)[0]}}
        pool = tq.build_pool(ctx, ints.n_spatial, ne, mp_)
        for prec, pname in ((tq.TQ_C128, "fp64"), (tq.TQ_C64, "c64")):
            ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, mp_, prec)
            st = tq.State(ctx, 12, prec)
            tq.state_set_hf(st, ne, mp_)
            tq.adapt_run(ctx, ham, pool, st, 1e-3, n_iter)       # warm (captures its graph)
            tq.state_set_hf(st, ne, mp_)
            t0 = time.perf_counter()
            res, done = tq.adapt_run(ctx, ham, pool, st, 1e-3, n_iter)
            t = time.perf_counter() - t0
            e = [x["energy"] for x in res[:done]]
            m = min(len(e), len(e_o))
            row[pname] = {"seconds": t, "ms_per_iteration": 1e3 * t / max(done, 1), "iterations": done,
                          "final_energy": tq.energy(ctx, ham, st),
                          "same_selections_as_oracle": sum(res[i]["selected"] == res_o[i].selected
                                                           for i in range(m)),
                          "max_abs_energy_diff_vs_oracle_ha": float(np.max(np.abs(np.array(e[:m]) -
                                                                                   np.array(e_o[:m])))),
                          "speedup_vs_oracle": t_o / t}
        row["c64_minus_fp64_final_energy_ha"] = row["c64"]["final_energy"] - row["fp64"]["final_energy"]
        out[mname] = row
    return out


def measure_general_update(tq, ctx, reps=100):
    """The general-operator fused Taylor-5 (tq_evolve_taylor5_csr: any CSR
    operator, the state held in a thread-block cluster's shared memory, each
    of the five products behind a cluster barrier) and the one-launch
    single-state update of a pool generator (tq_evolve_taylor5), 14 qubits."""
    import synth
    ints, ne = synth.config2()
    peak, _ = peaks()
    pool = tq.build_pool(ctx, ints.n_spatial, ne, MAPPING)
    D_ = 1 << NQ
    out = {"workload": "one 14-qubit state (HF after three updates), config-2 BK operators"}
    for prec, name, vb in ((tq.TQ_C64, "c64", 4), (tq.TQ_C128, "c128", 8)):
        ham = tq.build_hamiltonian(ctx, ints.h, ints.g, ints.e_const, MAPPING, prec)
        st = tq.State(ctx, NQ, prec)
        tq.state_set_hf(st, ne, MAPPING)
        for k, th in RATE_OPS:
            tq.evolve_taylor5(ctx, pool, k, th, st)
        sb = 8 if prec == tq.TQ_C64 else 16
        res = {}
        rp, cl, vl, nnz = tq.pool_csr(ctx, pool, 101, prec)
        hrp, hcl, hvl, _ = tq.ham_csr(ham)
        for oname, (orp, ocl, ovl, onnz, th) in (("pool_generator_101", (rp, cl, vl, nnz, 0.07)),
                                                 ("hamiltonian_offdiagonal", (hrp, hcl, hvl, ham.nnz, 0.01))):
            for _ in range(5):
                tq.evolve_taylor5_csr(ctx, NQ, orp, ocl, ovl, th, st, renormalize=True)
            ctx.trace(True)
            for _ in range(reps):
                tq.evolve_taylor5_csr(ctx, NQ, orp, ocl, ovl, th, st, renormalize=True)
            rep = ctx.trace_report()
            ctx.trace(False)
            n_l, ms = rep.get("taylor5_csr", (1, float("nan")))
            ms /= n_l
            csr_b = 4 * (D_ + 1) + (4 + vb) * onnz
            alg = 2 * D_ * sb + csr_b
            res[oname] = {"nnz": int(onnz), "ms_per_update": ms, "algorithmic_bytes": alg,
                          "bytes_note": "state in and out once + the CSR once from HBM (it is re-read 4 more "
                                        "times from L2, not counted)",
                          "achieved_gbs": alg / (ms * 1e-3) / 1e9, "frac": alg / (ms * 1e-3) / 1e9 / peak,
                          "csr_l2_gbs": 5 * csr_b / (ms * 1e-3) / 1e9}
        # the one-launch single-state update (pool generator, renormalised)
        l0 = ctx.launches()
        ctx.trace(True)
        for i in range(reps):
            tq.evolve_taylor5(ctx, pool, RATE_OPS[i % 3][0], 0.01, st, renormalize=True)
        rep = ctx.trace_report()
        ctx.trace(False)
        launches = (ctx.launches() - l0) / reps
        kname = "taylor5_single" if "taylor5_single" in rep else "taylor5_pair"
        n_l, ms = rep[kname]
        ms /= n_l
        res["single_state_pool_update"] = {"kernel": kname, "launches_per_update": launches,
                                           "ms_per_update": ms, "algorithmic_bytes": 2 * D_ * sb,
                                           "achieved_gbs": 2 * D_ * sb / (ms * 1e-3) / 1e9,
                                           "frac": 2 * D_ * sb / (ms * 1e-3) / 1e9 / peak}
        out[name] = res
    out["peak_gbs"] = peak
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--states", type=int, default=8192)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--headline-only", action="store_true",
                    help="skip the SpMV, trajectory-batch and request-loop measurements")
    ap.add_argument("--section", choices=["spmv", "trajectories", "serving", "sector", "vqe", "c128", "support",
                                              "full_state", "adapt", "precision", "m0", "m1", "general",
                                              "fp64_single"], default=None,
                    help="run one secondary measurement alone and print its JSON (profiling)")
    ap.add_argument("--spmv-qubits", type=int, default=18)
    ap.add_argument("--traj", type=int, default=256)
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="length of the request-loop measurement (0 skips it)")
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--serve-sweep", type=str, default="2000,4000,8000,12000,16000,24000,32000",
                    help="offered rates (requests/s) of the saturation sweep, comma-separated ('' skips)")
    ap.add_argument("--l2-fetch", type=int, default=0, choices=[0, 32, 64, 128],
                    help="L2 fetch granularity of the headline (0 = tuned)")
    ap.add_argument("--ctas-per-sm", type=int, default=-1,
                    help="resident CTAs per SM of the headline update (-1 = tuned, 0 = as many as fit)")
    ap.add_argument("--layout", choices=["linear", "sector", "natural"], default="linear",
                    help="states in BK with the index carried by a GF(2) map chosen for sector fill (linear), "
                         "with its qubits reordered for it (sector), or in BK's own order")
    ap.add_argument("--layout-bits", type=int, default=14,
                    help="index bits the sector-packing map fills (tq_pool_sector_basis / tq_pool_sector_order)")
    ap.add_argument("--fidelity-samples", type=int, default=64,
                    help="headline states checked against the oracle after the run (0 skips)")
    ap.add_argument("--pair-schedule", type=int, default=0,
                    help="support pairs per thread of the update (0 = autotune)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)

    if args.impl == "reference":
        if rank != 0:
            return 0
        return run_reference(args, world)

    if args.section:
        if rank != 0:
            return 0
        import torch

        import paper_2606_29692_gb300 as tq
        torch.cuda.set_device(local_rank)
        ctx = tq.Context(local_rank)
        if args.section == "spmv":
            print(json.dumps(measure_spmv(tq, ctx, args.spmv_qubits)))
        elif args.section == "trajectories":
            print(json.dumps(measure_trajectories(tq, ctx, args.traj)))
        elif args.section == "sector":
            print(json.dumps(measure_sector(tq, ctx)))
        elif args.section == "vqe":
            print(json.dumps(measure_vqe(tq, ctx)))
        elif args.section == "adapt":
            print(json.dumps(measure_adapt_step(tq, ctx)))
        elif args.section == "full_state":
            print(json.dumps(measure_full_state(tq, ctx, tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, MAPPING), 8192)))
        elif args.section == "support":
            print(json.dumps(measure_support(tq, ctx, tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, MAPPING), 8192)))
        elif args.section == "precision":
            print(json.dumps(measure_precision(tq, ctx)))
        elif args.section == "m0":
            print(json.dumps(measure_m0(tq, ctx)))
        elif args.section == "m1":
            print(json.dumps(measure_m1(tq, ctx)))
        elif args.section == "general":
            print(json.dumps(measure_general_update(tq, ctx)))
        elif args.section == "fp64_single":
            import synth
            pool = tq.build_pool(ctx, N_SPATIAL, N_ELECTRONS, MAPPING)
            _, _, k_, th_ = synth.t5_batch(8192, pool.M)
            print(json.dumps(measure_fp64_single(tq, ctx, pool, k_, th_)))
        elif args.section == "c128":
            import synth
            ints, ne = synth.config2()
            print(json.dumps(measure_c128_batched(tq, ctx, tq.build_pool(ctx, ints.n_spatial, ne, MAPPING))))
        else:
            sweep = [float(x) for x in args.serve_sweep.split(",") if x.strip()]
            print(json.dumps(measure_serving(tq, local_rank, args.serve_seconds, args.serve_rate, sweep)))
        return 0

    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            rate, cores, n, t = cpu_oracle_rate(args.cpu_seconds)
            out["cpu_baseline"] = {
                "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": (f"{n} oracle updates (scipy CSR complex128, 5 SpMV + Eq. (8) sum) of "
                           f"{4 * cores} states of the same workload, {cores} spawn workers, "
                           f"{t:.1f} s")}
            if "rates_14q" in out:
                out["rates_14q"]["oracle"] = oracle_rates(seconds=2.0)
        else:
            out["cpu_baseline"] = None
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def run_reference(args, world):
    """The oracle timed on the host cores on the same metric (reference arm)."""
    cores = os.cpu_count() or 1
    per_step = max(1.0, min(6.0, 150.0 / max(1, args.steps + args.warmup)))
    rates = []
    with mp.get_context("spawn").Pool(cores) as pool:
        for i in range(args.warmup + args.steps):
            rate, c, n, t = cpu_oracle_rate(per_step, states_per_core=2, cores=cores, pool=pool)
            if i >= args.warmup:
                rates.append((n, t))
    n = sum(r[0] for r in rates)
    t = sum(r[1] for r in rates)
    value = n / t
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
        "data": "synthetic", "config": workload_config(args.states),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": (f"each step: {per_step:.1f} s of oracle updates (scipy CSR complex128) "
                                    f"on {2 * cores} states of the workload across {cores} spawn workers")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
