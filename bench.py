"""Benchmark: MTP energy + force evaluation on the 1,024,000-atom level-16 BCC
workload (3 species, r_cut 5.0 A, ~26 neighbours per atom), FP32-mixed, one
GPU.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one mtp_compute_efv call (site energies, forces, virial) on the
prebuilt neighbour list; the neighbour build is timed separately and reported
as nbr_build_ms.  With N > 1 (torchrun) every rank evaluates its own replica of
the workload (independent configurations, no exchange) and the value is the sum.
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
sys.path.insert(0, ROOT)

METRIC = "MTP E+F atom-steps/s, 1M atoms lev16, FP32-mixed vs FP64; % HBM roofline"
UNIT = "atom-steps/s"
WORKLOAD = "bcc-80x80x80 (1,024,000 atoms), MTP level 16, 3 species, n_q 8, r_cut 5.0 A, sigma 0.08 A"
POTENTIAL = "bcc-l16-s3"
CELLS = (80, 80, 80)
SM_COUNT = 152
FP32_LANES = 128
# DRAM read + write per atom of efv_kernel<MtpLevel16, float, 0> from the
# latest ncu capture in profiles/efv_kernel_bcc70_l16_mixed.md (686,000 atoms;
# traffic scales with the atom count).  Set to None whenever that kernel changes.
EFV_TRAFFIC_BYTES_PER_ATOM = (184.299520e6 + 11.423744e6) / 686000


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), d.get("sm_max_mhz", 2070.0), "measured"
    return 6800.0, 2070.0, "fallback"


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    return rank, world


def max_over_ranks(ms, world, device="cuda"):
    """The slowest rank's time per step: every rank evaluates its own replica
    (weak scaling, no exchange on the data path), so the job's step ends when
    the last rank's does.  One all-reduce of one number, outside the timed region."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, n_atoms_per_rank, ms):
    """Whole-job atom-steps/s: the atoms of all replicas per slowest step."""
    return world * n_atoms_per_rank / (ms * 1e-3)


def _workload(cells=CELLS):
    import synth
    return synth.crystal("bcc", tuple(cells), 3.16, 0.08, 3, 2)


def _flops_per_atom(level, n_q, n_mu, nbar, sweep_all=True):
    """FP32 flops per atom of one E+F evaluation (geometry, radial functions
    and derivatives, monomials, moments, contraction and its reverse, pair
    adjoint, force/virial accumulation), counted from the generated code.
    With sweep_all (the algorithmic count of the roofline) the neighbour sweeps
    cover every Cartesian moment component, as the method is written; without
    it, the count of the code the kernel runs, whose sweeps cover only the
    components with a z-exponent of at most 1 (the rest follow per atom from
    |rhat| = 1).  Recomputation in the second neighbour sweep is not counted."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2510_00193_gb300"))
    import basisgen
    fc = basisgen.flop_counts(basisgen.Level(level), sweep_all=sweep_all)
    q = n_q
    radial_f = 4 + 2 * n_mu + (q - 2) * (3 + 2 * n_mu) + n_mu
    radial_d = (q - 2) * (4 + 2 * n_mu) + 1 + 4 * n_mu
    geom, accum = 28, 24
    per_pair = geom + radial_f + fc["monomials"] + fc["moments"] + radial_d + fc["pair_adjoint"] + accum
    return per_pair * nbar + fc["contract"], fc


class ClockSampler:
    """nvidia-smi clock and throttle samples while the timed region runs."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "mtp_bench_clocks_%d.csv" % os.getpid())

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        loaded = sorted(sm)[len(sm) // 2:] if sm else []
        return {"sm_mhz": statistics.median(loaded) if loaded else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(st, n_sample, seed=3):
    """Oracle E+F throughput on a bounded sample of centre atoms: the sampled
    centres' neighbour rows are built first (outside the timer), then the
    oracle's evaluation of their site energies with force and virial
    contributions is timed, so the cost per atom does not depend on the
    sample size.  Returns (atom-steps/s, seconds, threads used, host cores)."""
    import numpy as np
    import torch

    from oracle import mtp as O
    from tests.helpers import BinnedCandidates, oracle_rows, pot_dict

    model = O.load_model(pot_dict(POTENTIAL))
    g = np.random.default_rng(seed)
    centres = np.sort(g.choice(st.n, n_sample, replace=False))
    cands = BinnedCandidates(st, 5.5)
    rows = [oracle_rows(st, 5.0, c, cands(c)) for c in centres]
    nl = (np.concatenate([np.full(len(r[0]), c) for c, r in zip(centres, rows)]),
          np.concatenate([r[0] for r in rows]), np.concatenate([r[1] for r in rows]))
    t0 = time.perf_counter()
    O.evaluate(model, st.x, st.z, st.cell, nl, want=("e", "f", "w"), atoms=centres)
    dt = time.perf_counter() - t0
    return n_sample / dt, dt, torch.get_num_threads(), os.cpu_count()


MIXED_KAPPA = 64.0
MIXED_BOUND = ("|dE_i| <= 1e-5 eV + 64 u a_i and |dF_k| <= 1e-4 eV/A + 64 u A_k / A, u = 2^-24, "
               "a_i = sum_alpha |xi_alpha B_alpha(i)|, A_k = a_k + sum over neighbours j of k of a_j; "
               "*_bound_use = max over atoms of error / bound")


def mixed_conditioning(P, torch, pot, nl, x, z, cell, pot_name):
    """a_i = sum_alpha |xi_alpha B_alpha(i)| (from the FP64 basis rows) and
    A_k = a_k + sum over the neighbours j of k of a_j, the conditioning of the
    site energies and forces that scales the mixed-precision error bound."""
    with open(os.path.join(ROOT, "potentials", pot_name + ".json")) as fh:
        xi = torch.tensor(json.load(fh)["xi"], dtype=torch.float64, device="cuda").abs()
    n = x.shape[0]
    rows = P.mtp_compute_basis_rows(pot, nl, x, z, cell)
    a = (rows.abs() * xi).sum(1)
    del rows
    off, j, _ = nl.to_tensors()
    ii = torch.repeat_interleave(torch.arange(n, device="cuda"), off[1:] - off[:-1])
    A = a.clone().index_add_(0, ii, a[j.long()])
    return {"a": a, "A": A}


def fma_peaks(P, local):
    """Measured FMA throughput of this GPU (FP32 and FP64), with the SM clock
    sampled while the probe kernels ran."""
    with ClockSampler(local) as clk:
        fp32 = max(P.mtp_probe_fma(P.PROBE_FP32, 4096, 4)["flops_per_s"] for _ in range(3))
        fp64 = max(P.mtp_probe_fma(P.PROBE_FP64, 256, 4)["flops_per_s"] for _ in range(3))
    return {"fp32_tflops": fp32 / 1e12, "fp64_tflops": fp64 / 1e12, "clocks": clk.summary(),
            "how": "mtp_probe_fma: 152 x 4 blocks of 256 threads, 8 independent fma chains per thread, "
                   "CUDA events, best of 3"}


def run_grade(P, torch, args):
    """Extrapolation grade on the 500,000-atom BCC workload (50 x 50 x 100 cells,
    sigma 0.15 A, level 16, one species), neighbourhood and configuration mode."""
    import synth
    with open(os.path.join(ROOT, "potentials", "bcc-l16-s1-active.json")) as fh:
        act = json.load(fh)
    m = act["m"]
    st = synth.crystal("bcc", (50, 50, args.grade_cells), 3.16, 0.15, 1, 5)
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", "bcc-l16-s1.json"))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    a_inv = torch.tensor(act["a_inv"], dtype=torch.float64, device="cuda").reshape(m, m)
    a_cfg = torch.tensor(act["a_inv_cfg"], dtype=torch.float64, device="cuda").reshape(m, m)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    res = {"workload": "bcc-50x50x%d (%d atoms), level 16, 1 species, sigma 0.15 A; active sets by MaxVol"
                       % (args.grade_cells, st.n), "unit": UNIT}
    flops_fp64 = 2.0 * st.n * m * m
    for name, method in (("tensor", P.MTP_GRADE_TENSOR), ("fp64", P.MTP_GRADE_FP64)):
        out = P.mtp_compute_grade(pot, nl, x, z, st.cell, a_inv=a_inv, a_inv_cfg=a_cfg, method=method)
        torch.cuda.synchronize()
        steps = 3
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(steps):
            out = P.mtp_compute_grade(pot, nl, x, z, st.cell, a_inv=a_inv, a_inv_cfg=a_cfg, method=method, out=out)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        flags = out["flags"].cpu().numpy()
        res[name] = {"value": st.n / (ms * 1e-3), "ms_per_step": ms, "gamma_max": out["gamma_max"],
                     "gamma_cfg": out["gamma_cfg"], "n_ambiguous": out["n_ambiguous"],
                     "n_rechecked": out["n_rechecked"], "n_selected": int((flags & 1).sum()),
                     "n_break": int((flags & 2).sum() // 2)}
        if name == "tensor":
            res["flags_tensor"] = flags
    res["flags_identical"] = bool((res.pop("flags_tensor") == flags).all())
    res["value"] = res["tensor"]["value"]
    res["ms_per_step"] = res["tensor"]["ms_per_step"]
    res["product_flops_fp64_equivalent"] = flops_fp64
    res["mma_flops_executed"] = 2.0 * 28 * 128 * 128 * 128 * ((st.n + 127) // 128)
    res["tc_kernel"] = time_tc_kernel(P, torch)
    res["maxvol"] = time_maxvol(P, torch)
    return res


def time_maxvol(P, torch):
    """Active-set selection for the neighbourhood grade: MaxVol (delta 0.01)
    over the FP64 basis rows of every atom of a 20^3-cell BCC box (16,000
    atoms, sigma 0.05 A, level 16), from the first m rows of a seeded
    permutation of the pool; basis rows and MaxVol both on the device."""
    import numpy as np

    import synth
    st = synth.crystal("bcc", (20, 20, 20), 3.16, 0.05, 1, 5, sub=8)
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", "bcc-l16-s1.json"))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    rows = P.mtp_compute_basis_rows(pot, nl, x, z, st.cell)
    torch.cuda.synchronize()
    init = np.random.default_rng(20251005).permutation(st.n)[:pot.m]
    t0 = time.perf_counter()
    sel, _, swaps = P.mtp_maxvol(rows, init, delta=0.01)
    ms = 1e3 * (time.perf_counter() - t0)
    return {"pool_rows": st.n, "m": pot.m, "swaps": swaps, "ms": ms, "ms_per_swap": ms / max(1, swaps)}


def time_tc_kernel(P, torch, rows=262144, reps=5):
    """The tensor-core grade kernel alone (through the C-ABI verification hook)
    on random BF16 slices of one full 262,144-row chunk: device time per
    launch and executed MMA throughput against the measured BF16 peak."""
    g = torch.Generator(device="cuda").manual_seed(20251009)
    tiles = (rows + 127) // 128
    xs = torch.randint(-128, 129, (tiles * 7 * 128 * 128,), device="cuda", generator=g, dtype=torch.int32)
    ys = torch.randint(-128, 129, (2 * 7 * 64 * 128,), device="cuda", generator=g, dtype=torch.int32)
    # integers -> BF16 bit patterns (exact: at most 8 significant bits)
    to_bf16 = lambda t: (t.to(torch.float32).view(torch.int32) >> 16).to(torch.int16)
    xs, ys = to_bf16(xs), to_bf16(ys)
    fexp = torch.zeros(128, dtype=torch.int32, device="cuda")
    erow = torch.zeros(rows, dtype=torch.int32, device="cuda")
    P.mtp_grade_tc_selftest(xs, ys, fexp, erow, rows)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(reps):
        e0.record()
        P.mtp_grade_tc_selftest(xs, ys, fexp, erow, rows)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = min(times)
    flops = 2.0 * 28 * 128 * 128 * 128 * tiles
    peak = 1881.0
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            peak = json.load(fh).get("bf16_tflops", peak)
    return {"rows": rows, "ms": ms, "mma_tflops": flops / (ms * 1e-3) / 1e12, "bf16_peak_tflops": peak,
            "frac": flops / (ms * 1e-3) / 1e12 / peak}


def run_small(P, torch, args):
    """Small systems (the paper's block-parallel regime, ~2,000 atoms per GPU):
    level-16 BCC boxes of 2,000 and 16,000 atoms (3 species, sigma 0.08 A) and
    a level-20 FCC box of 2,048 atoms (4 species), mixed precision, one thread
    per atom against one warp per atom, and the tuner's choice."""
    import synth
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", POTENTIAL + ".json"))
    out = {}
    for cells in (10, 20):
        st = synth.crystal("bcc", (cells,) * 3, 3.16, 0.08, 3, 2)
        x = torch.tensor(st.x, device="cuda")
        z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
        nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        res = {}
        for name, variant in (("thread_per_atom", 1), ("warp_per_atom", 2)):
            P.mtp_set_efv_variant(pot, variant)
            o = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
            for _ in range(5):
                P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED, out=o)
            reps = 50
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=P.MTP_MIXED, out=o)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            res[name] = {"ms": ms, "atom_steps_per_s": st.n / (ms * 1e-3)}
        P.mtp_set_efv_variant(pot, 0)
        res["tuner"] = P.mtp_efv_tune(pot, nl, x, z, st.cell, precision=P.MTP_MIXED)
        out["%d_atoms" % st.n] = res
    # level 20 (interpreted contraction): 2,048-atom FCC, 4 species, the
    # differentiation recipe at small size
    pot20 = P.Potential.from_file(os.path.join(ROOT, "potentials", "fcc-l20-s4.json"))
    st = synth.crystal("fcc", (8, 8, 8), 3.6, 0.1, 4, 3)
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    nl = P.mtp_build_neighbors(pot20, x, st.cell, st.pbc)
    res = {}
    for name, variant in (("thread_per_atom_three_kernels", 1), ("warp_per_atom", 2)):
        P.mtp_set_efv_variant(pot20, variant)
        o = P.mtp_compute_efv(pot20, nl, x, z, st.cell, precision=P.MTP_MIXED)
        for _ in range(3):
            P.mtp_compute_efv(pot20, nl, x, z, st.cell, precision=P.MTP_MIXED, out=o)
        reps = 20
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            P.mtp_compute_efv(pot20, nl, x, z, st.cell, precision=P.MTP_MIXED, out=o)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        res[name] = {"ms": ms, "atom_steps_per_s": st.n / (ms * 1e-3)}
    P.mtp_set_efv_variant(pot20, 0)
    res["tuner"] = P.mtp_efv_tune(pot20, nl, x, z, st.cell, precision=P.MTP_MIXED)
    out["level20_%d_atoms" % st.n] = res
    return out


def run_batch(P, torch, args):
    """4096 periodic configurations of 8..256 atoms (2 species, level 16,
    random triclinic cells at 0.085 atoms/A^3, 1.9 A minimum separation):
    energies, forces, virials and dE/dtheta in one persistent launch replayed
    from a CUDA graph, against one mtp_compute_efv launch per configuration."""
    import numpy as np

    import synth
    structs = synth.random_gas_batch(4096, 8, 256, 0.085, 1.9, 2, 4)
    off = np.concatenate([[0], np.cumsum([st.n for st in structs])]).astype(np.int64)
    x = torch.tensor(np.concatenate([st.x for st in structs]), device="cuda")
    z = torch.tensor(np.concatenate([st.z for st in structs]).astype(np.int32), device="cuda")
    cells = np.stack([st.cell for st in structs])
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", "gas-l16-s2.json"))
    b = P.Batch(pot, off, cells, x)
    chosen = P.mtp_batch_tune(pot, b, x, z, P.MTP_MIXED, True)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        out = P.mtp_compute_batch(pot, b, x, z, precision=P.MTP_MIXED, dtheta=True, stream=s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        P.mtp_compute_batch(pot, b, x, z, precision=P.MTP_MIXED, dtheta=True, out=out, stream=s)
    reps = 20
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(s):          # replay() launches on the current stream
        for _ in range(3):
            g.replay()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    torch.cuda.synchronize()
    ms_graph = e0.elapsed_time(e1) / reps
    # the same launch without the graph, for reference
    e0.record()
    for _ in range(reps):
        P.mtp_compute_batch(pot, b, x, z, precision=P.MTP_MIXED, dtheta=True, out=out)
    e1.record()
    torch.cuda.synchronize()
    ms_direct = e0.elapsed_time(e1) / reps
    # one launch sequence per configuration (mtp_compute_efv, same precision and outputs)
    nls = []
    for st in structs:
        xs = torch.tensor(st.x, device="cuda")
        nls.append((xs, torch.tensor(st.z, device="cuda"), P.mtp_build_neighbors(pot, xs, st.cell, st.pbc), st.cell))
    outs = [P.mtp_compute_efv(pot, nl, xs, zs, cell, precision=P.MTP_MIXED, dtheta=True) for xs, zs, nl, cell in nls]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record()
    for (xs, zs, nl, cell), o in zip(nls, outs):
        P.mtp_compute_efv(pot, nl, xs, zs, cell, precision=P.MTP_MIXED, dtheta=True, out=o)
    e1.record()
    host_ms = 1e3 * (time.perf_counter() - t0)
    torch.cuda.synchronize()
    ms_each = e0.elapsed_time(e1)
    n_atoms = int(off[-1])
    return {"workload": "4096 random triclinic periodic gases, 8..256 atoms (%d in all), level 16, 2 species"
                        % n_atoms,
            "atoms_per_block": chosen, "ms_per_batch": ms_graph, "ms_per_batch_without_graph": ms_direct,
            "per_config_launches_host_ms": host_ms,
            "configs_per_s": 4096 / (ms_graph * 1e-3), "atom_steps_per_s": n_atoms / (ms_graph * 1e-3),
            "per_config_launches_ms": ms_each, "speedup_vs_per_config": ms_each / ms_graph,
            "outputs": "energies, forces, virials, dE/dtheta per configuration (mixed precision)"}


def run_diff(P, torch, args):
    """256,000-atom FCC (40^3 cells, a = 3.6 A, sigma 0.1 A), 4 species, level 20,
    n_q 10, r_cut 5.5 A: forward (energy), backward (forces and dE/dtheta) and
    double backward (directional derivative of dE/dtheta for a force-matching
    loss), FP64 and mixed; mixed errors against FP64 are reported."""
    import synth
    st = synth.crystal("fcc", (40, 40, 40), 3.6, 0.1, 4, 3)
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", "fcc-l20-s4.json"))
    x = torch.tensor(st.x, device="cuda")
    z = torch.tensor(st.z, device="cuda")
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    v = torch.tensor(synth.target_forces(st.n, 3), device="cuda")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            r = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, r

    res = {"workload": "fcc-40x40x40 (256,000 atoms), level 20, 4 species, n_q 10, r_cut 5.5 A, sigma 0.1 A"}
    outs = {}
    for name, prec, reps in (("mixed", P.MTP_MIXED, 3), ("fp64", P.MTP_FP64, 1)):
        ms_e, _ = timed(lambda: P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=prec), reps)
        ms_b, o = timed(lambda: P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=prec, dtheta=True), reps)
        ms_t, t = timed(lambda: P.mtp_compute_efv_tangent(pot, nl, x, z, st.cell, v, precision=prec), reps)
        outs[name] = (o, t)
        res[name] = {"efv_ms": ms_e, "efv_dtheta_ms": ms_b, "double_backward_ms": ms_t,
                     "atom_steps_per_s": st.n / (ms_e * 1e-3)}
    (om, tm), (od, td) = outs["mixed"], outs["fp64"]
    import numpy as np
    cond = mixed_conditioning(P, torch, pot, nl, x, z, st.cell, "fcc-l20-s4")
    de = (om["e_atom"] - od["e_atom"]).abs()
    dfa = (om["forces"] - od["forces"]).abs().max(1).values
    res["mixed_errors_vs_fp64"] = {
        "e_atom_max_abs": float(de.max()),
        "force_rms": float(((om["forces"] - od["forces"]) ** 2).mean().sqrt()),
        "force_max_abs": float(dfa.max()),
        "e_total_per_atom_abs": float((om["e_total"] - od["e_total"]).abs().item() / st.n),
        "bound": MIXED_BOUND,
        "e_atom_bound_use": float((de / (1e-5 + MIXED_KAPPA * 2.0 ** -24 * cond["a"])).max()),
        "force_bound_use": float((dfa / (1e-4 + MIXED_KAPPA * 2.0 ** -24 * cond["A"])).max()),
        "dtheta_max_rel": float((om["dtheta"] - od["dtheta"]).abs().max() / od["dtheta"].abs().max()),
        "dtheta_tan_max_rel": float((tm["dtheta_tan"] - td["dtheta_tan"]).abs().max()
                                    / td["dtheta_tan"].abs().max())}
    del np
    return res


MD_MASSES = (183.84, 95.95, 50.94)   # amu of the three species (W, Mo, V: BCC metals near a = 3.16 A)


def run_md(P, torch, st, pot, z, args):
    """Molecular dynamics on the headline workload as the paper benchmarks its
    pair styles: runs of 100 velocity-Verlet steps, the best of five, each run
    from the same start (FP32-mixed forces, 300 K Maxwell-Boltzmann
    velocities, skin 0.3 A, displacements checked every step and the skin
    list rebuilt when an atom has moved more than half the skin, the list
    filtered to the exact list every step).  The paper's runs take 1 fs steps
    with fitted potentials; the synthetic random-coefficient potential is not
    a stable model (forces of ~4 eV/A RMS on this structure and hundreds of
    eV/A on its worst atoms, which then leave the skin within a few 0.1 fs
    steps), so the step here is 0.01 fs and the 100 steps need no rebuild.
    The cost of a step does not depend on dt: atom-steps/s is the comparable
    figure.  The skin-list rebuild is timed separately, and the per-step cost
    with one rebuild every 20 steps is derived from the two."""
    import numpy as np
    kb, mvv2e = 8.617333e-5, 1.0364269e-4
    m = np.asarray(MD_MASSES)[st.z]
    g = np.random.default_rng(20251002)
    v0 = g.normal(size=(st.n, 3)) * np.sqrt(kb * 300.0 / (m * mvv2e))[:, None]
    v0 -= (m[:, None] * v0).sum(0) / m.sum()
    steps, rebuild_every, skin, dt = 100, -1, 0.3, 1e-5
    x0 = torch.tensor(st.x, device="cuda")
    v0 = torch.tensor(v0, device="cuda")
    x, v = x0.clone(), v0.clone()
    md = P.MD(pot, x, st.cell, st.pbc, skin=skin)
    f0 = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_MIXED)["forces"]
    f = f0.clone()
    e_pot = torch.empty(steps, dtype=torch.float64, device="cuda")
    e_kin = torch.empty(steps, dtype=torch.float64, device="cuda")
    md.run(x, v, z, MD_MASSES, dt, 5, f, rebuild_every=rebuild_every, precision=P.MTP_MIXED)   # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    drift = None
    rebuilds = []
    for rep in range(5):
        x.copy_(x0)
        v.copy_(v0)
        f.copy_(f0)
        md.rebuild(x)
        torch.cuda.synchronize()
        r0 = md.rebuilds()
        e0.record()
        md.run(x, v, z, MD_MASSES, dt, steps, f, rebuild_every=rebuild_every, precision=P.MTP_MIXED,
               e_pot=e_pot, e_kin=e_kin)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
        rebuilds.append(md.rebuilds() - r0)
        if rep == 0:
            et = (e_pot + e_kin).cpu().numpy()
            drift = float(abs(et[-1] - et[0]) / st.n)
    ms = min(times) / steps
    t0 = time.perf_counter()
    md.rebuild(x)
    rebuild_ms = 1e3 * (time.perf_counter() - t0)
    # the same steps replayed from a CUDA graph of 10 steps (no synchronisation
    # inside; the displacement check runs between replays every 20 steps,
    # outside the graph).  A rebuild may move the list buffers, which a
    # captured graph holds by address, so a caller that rebuilds captures
    # again; these 0.01 fs steps need no rebuild (checked).
    x.copy_(x0)
    v.copy_(v0)
    f.copy_(f0)
    md.rebuild(x)
    gs = torch.cuda.Stream()
    with torch.cuda.stream(gs):
        md.run(x, v, z, MD_MASSES, dt, 10, f, rebuild_every=0, precision=P.MTP_MIXED, stream=gs)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gs):
        md.run(x, v, z, MD_MASSES, dt, 10, f, rebuild_every=0, precision=P.MTP_MIXED, stream=gs)
    x.copy_(x0)
    v.copy_(v0)
    f.copy_(f0)
    md.rebuild(x)
    torch.cuda.synchronize()
    g_times = []
    with torch.cuda.stream(gs):
        for rep in range(3):
            t0 = time.perf_counter()
            for k in range(steps // 10):
                graph.replay()
                if k % 2 == 1:
                    md.status(stream=gs)     # displacement check (synchronises; raises if stale)
            gs.synchronize()
            g_times.append(1e3 * (time.perf_counter() - t0))
    graph_ms = min(g_times) / steps
    del graph
    return {"workload": "bcc-80x80x80 (1,024,000 atoms), level 16, 3 species (%.2f, %.2f, %.2f amu), 300 K"
                        % MD_MASSES,
            "integrator": "velocity Verlet (NVE), dt 0.01 fs, mixed-precision forces",
            "steps_per_run": steps, "runs": 5, "skin_A": skin,
            "neighbour_policy": "displacements checked every step, skin list rebuilt beyond skin/2",
            "rebuilds_per_run": rebuilds,
            "ms_per_step_best_of_5": ms, "ms_per_step_median": sorted(times)[2] / steps,
            "atom_steps_per_s": st.n / (ms * 1e-3), "ns_per_day_at_1fs": 86400 / (ms * 1e-3) * 1e-6,
            "skin_list_rebuild_ms": rebuild_ms,
            "ms_per_step_with_a_rebuild_every_20_steps": ms + rebuild_ms / 20,
            "graph_replay_ms_per_step": graph_ms,
            "graph_replay_ms_per_step_with_a_rebuild_every_20_steps": graph_ms + rebuild_ms / 20,
            "graph_note": "10-step CUDA graphs (rebuild_every = 0); the displacement check between replays every "
                          "20 steps; host wall clock per step, best of 3 runs of %d steps; the rebuild figure adds "
                          "the measured skin-list rebuild / 20" % steps,
            "total_energy_change_per_atom_eV": drift}


def run_md_graded(P, torch, args):
    """MD with the extrapolation grade every 10 steps (paper Sec. 2.3): the
    500,000-atom grade workload (BCC 50 x 50 x 100, sigma 0.15 A, level 16,
    one species, its MaxVol active set), 100 velocity-Verlet steps of 0.01 fs
    at 300 K with mixed-precision forces and the tensor-core grade."""
    import numpy as np

    import synth
    with open(os.path.join(ROOT, "potentials", "bcc-l16-s1-active.json")) as fh:
        act = json.load(fh)
    m = act["m"]
    st = synth.crystal("bcc", (50, 50, args.grade_cells), 3.16, 0.15, 1, 5)
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", "bcc-l16-s1.json"))
    masses = (183.84,)
    kb, mvv2e = 8.617333e-5, 1.0364269e-4
    g = np.random.default_rng(20251003)
    v0 = g.normal(size=(st.n, 3)) * np.sqrt(kb * 300.0 / (masses[0] * mvv2e))
    v0 -= v0.mean(0)
    x = torch.tensor(st.x, device="cuda")
    v = torch.tensor(v0, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    a_inv = torch.tensor(act["a_inv"], dtype=torch.float64, device="cuda").reshape(m, m)
    md = P.MD(pot, x, st.cell, st.pbc, skin=0.3)
    f = P.mtp_compute_efv(pot, md.nlist(), x, z, st.cell, precision=P.MTP_MIXED)["forces"]
    sel = torch.zeros(st.n, dtype=torch.uint8, device="cuda")
    md.set_grade(a_inv, 10, 2.0, 1e30, P.MTP_GRADE_TENSOR, sel)
    md.run(x, v, z, masses, 1e-5, 10, f, rebuild_every=-1, precision=P.MTP_MIXED)   # warm-up (sizes scratch)
    torch.cuda.synchronize()
    steps = 100
    t0 = time.perf_counter()
    status = md.run(x, v, z, masses, 1e-5, steps, f, rebuild_every=-1, precision=P.MTP_MIXED)
    torch.cuda.synchronize()
    ms = 1e3 * (time.perf_counter() - t0) / steps
    info = md.info()
    md.set_grade(None, 0)
    t0 = time.perf_counter()
    md.run(x, v, z, masses, 1e-5, steps, f, rebuild_every=-1, precision=P.MTP_MIXED)
    torch.cuda.synchronize()
    ms_plain = 1e3 * (time.perf_counter() - t0) / steps
    return {"workload": "bcc-50x50x%d (%d atoms), level 16, 1 species, sigma 0.15 A, 300 K, dt 0.01 fs"
                        % (args.grade_cells, st.n),
            "grade_every": 10, "tau_sel": 2.0, "steps": steps, "status": int(status),
            "ms_per_step": ms, "ms_per_step_without_grade": ms_plain,
            "atom_steps_per_s": st.n / (ms * 1e-3), "grade_evals": info["grade_evals"],
            "gamma_max_last": info["gamma_max_last"], "n_selected_last": info["n_selected_last"],
            "atoms_selected_during_run": int((sel & 1).sum().item()),
            "timing": "host wall clock around the run (the grade synchronises every 10 steps, the "
                      "displacement check every step)"}


def run_reference(args):
    rank, world = _dist()
    if rank != 0:
        return
    st = _workload()
    rates = []
    n_sample = 48
    for _ in range(args.warmup):
        oracle_rate(st, 8)
    t_total = 0.0
    for k in range(args.steps):
        r, dt, threads, cores = oracle_rate(st, n_sample, seed=100 + k)
        rates.append(r)
        t_total += dt
    value = n_sample * args.steps / t_total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "precision": "fp64 (oracle)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
                         "sample": "%d random centre atoms of the workload per step (E_i and their force and "
                                   "virial contributions; neighbour rows built outside the timer)" % n_sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_ours(args):
    import numpy as np
    import torch

    import paper_2510_00193_gb300 as P

    rank, world = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    st = _workload((args.cells,) * 3)
    pot = P.Potential.from_file(os.path.join(ROOT, "potentials", POTENTIAL + ".json"))
    x = torch.tensor(st.x, dtype=torch.float64, device="cuda")
    z = torch.tensor(st.z, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()
    peaks = fma_peaks(P, local)

    # neighbour list (timed separately)
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nl = P.mtp_build_neighbors(pot, x, st.cell, st.pbc, nlist=nl)
    torch.cuda.synchronize()
    nbr_ms = 1e3 * (time.perf_counter() - t0)
    n_atoms, n_pairs = nl.info()
    nbar = n_pairs / n_atoms

    def timed(precision, steps, warmup):
        out = P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision)
        for _ in range(warmup):
            P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision, out=out)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        ev[0].record(stream)
        for k in range(steps):
            P.mtp_compute_efv(pot, nl, x, z, st.cell, precision=precision, out=out)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        per = [ev[k].elapsed_time(ev[k + 1]) for k in range(steps)]
        return out, per

    with ClockSampler(local) as clk:
        out, per = timed(P.MTP_MIXED, args.steps, args.warmup)
    clocks = clk.summary()
    ms = max_over_ranks(sum(per) / len(per), world)
    value = job_rate(world, n_atoms, ms)

    # FP64 path for the mixed/FP64 ratio (a few steps)
    ms64 = None
    mixed_err = None
    if not args.no_fp64:
        out64, per64 = timed(P.MTP_FP64, max(2, min(3, args.steps)), 1)
        ms64 = max_over_ranks(sum(per64) / len(per64), world)
        # errors of the mixed path against the FP64 path (which matches the oracle to 1e-12)
        de = (out["e_atom"] - out64["e_atom"]).abs()
        df = out["forces"] - out64["forces"]
        cond = mixed_conditioning(P, torch, pot, nl, x, z, st.cell, POTENTIAL)
        mixed_err = {"e_atom_max_abs_eV": float(de.max()),
                     "bound": MIXED_BOUND,
                     "e_atom_bound_use": float((de / (1e-5 + MIXED_KAPPA * 2.0 ** -24 * cond["a"])).max()),
                     "force_bound_use": float((df.abs().max(1).values
                                               / (1e-4 + MIXED_KAPPA * 2.0 ** -24 * cond["A"])).max()),
                     "e_total_per_atom_abs_eV": float((out["e_total"] - out64["e_total"]).abs().item() / n_atoms),
                     "force_rms_eV_per_A": float((df * df).mean().sqrt()),
                     "force_max_abs_eV_per_A": float(df.abs().max()),
                     "virial_max_rel": float((out["virial"] - out64["virial"]).abs().max()
                                             / out64["virial"].abs().max()),
                     "targets": "1e-5 eV/atom, 1e-4 eV/A RMS"}
        del out64

    # end to end through the public API: pinned host positions in, forces and energy out
    xh = torch.tensor(st.x, dtype=torch.float64).pin_memory()
    zh = torch.tensor(st.z, dtype=torch.int32).pin_memory()
    fh = torch.empty((n_atoms, 3), dtype=torch.float64).pin_memory()
    eh = torch.empty(1, dtype=torch.float64).pin_memory()
    xd = torch.empty_like(x)
    zd = torch.empty_like(z)
    e2e_steps = 0 if args.no_e2e else args.steps
    for k in range(args.warmup + e2e_steps):
        if k == args.warmup:
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
        xd.copy_(xh, non_blocking=True)
        zd.copy_(zh, non_blocking=True)
        o = P.mtp_compute_efv(pot, nl, xd, zd, st.cell, precision=P.MTP_MIXED, out=out)
        fh.copy_(o["forces"], non_blocking=True)
        eh.copy_(o["e_total"], non_blocking=True)
    e2e_ms = None
    if e2e_steps:
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(e0.elapsed_time(e1) / e2e_steps, world)
    # the same with the neighbour list rebuilt from each step's positions (a
    # caller whose positions change between calls; the build synchronises)
    e2e_nb_ms = None
    if e2e_steps:
        nl2 = P.mtp_build_neighbors(pot, x, st.cell, st.pbc)
        nb_steps = max(3, e2e_steps // 4)
        for k in range(args.warmup + nb_steps):
            if k == args.warmup:
                torch.cuda.synchronize()
                e0.record(stream)
            xd.copy_(xh, non_blocking=True)
            zd.copy_(zh, non_blocking=True)
            nl2 = P.mtp_build_neighbors(pot, xd, st.cell, st.pbc, nlist=nl2)
            o = P.mtp_compute_efv(pot, nl2, xd, zd, st.cell, precision=P.MTP_MIXED, out=out)
            fh.copy_(o["forces"], non_blocking=True)
            eh.copy_(o["e_total"], non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_nb_ms = max_over_ranks(e0.elapsed_time(e1) / nb_steps, world)
        del nl2
    h2d = xh.numel() * 8 + zh.numel() * 4
    d2h = fh.numel() * 8 + 8

    grade = None if args.no_grade else run_grade(P, torch, args)
    batch = None if args.no_batch else run_batch(P, torch, args)
    small = None if args.no_batch else run_small(P, torch, args)
    diff = None if args.no_diff else run_diff(P, torch, args)
    md = None
    md_graded = None
    if not args.no_md:
        try:
            md = run_md(P, torch, st, pot, z, args)
        except P.MtpError as err:   # e.g. MTP_ERR_STALE_LIST: reported, the headline stands
            md = {"error": str(err)}
        try:
            md_graded = run_md_graded(P, torch, args)
        except P.MtpError as err:
            md_graded = {"error": str(err)}

    hbm_gbs, max_mhz, peak_src = _peaks()
    flops_atom, fc = _flops_per_atom(pot.level, pot.n_q, pot.n_mu, nbar)
    flops_atom_run, _ = _flops_per_atom(pot.level, pot.n_q, pot.n_mu, nbar, sweep_all=False)
    peak_tflops = peaks["fp32_tflops"]
    achieved_tflops = flops_atom * n_atoms / (ms * 1e-3) / 1e12
    executed_tflops = flops_atom_run * n_atoms / (ms * 1e-3) / 1e12
    bytes_atom = 16 + 8 * nbar + 24 + 8      # fixed-point position, (j, image) per pair, force, site energy
    hbm_achieved = bytes_atom * n_atoms / (ms * 1e-3) / 1e9

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        r, dt, threads, cores = oracle_rate(st, args.cpu_sample)
        cpu = {"value": r, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
               "sample": "%d random centre atoms of the workload (E_i with their force and virial "
                         "contributions; neighbour rows built outside the timer), %.1f s" % (args.cpu_sample, dt)}
    if rank == 0:
        workload = WORKLOAD if args.cells == CELLS[0] else WORKLOAD.replace("80x80x80 (1,024,000", "%dx%dx%d (%d" % (
            args.cells, args.cells, args.cells, n_atoms))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "precision": "mixed (FP32 arithmetic, FP64 accumulation)",
                       "l2": "inputs larger than L2 (neighbour list %.0f MB)" % (n_pairs * 8 / 1e6),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "mean_neighbours": round(nbar, 3)},
            "fp64": ({"value": job_rate(world, n_atoms, ms64), "unit": UNIT, "ms_per_step": ms64}
                     if ms64 else None),
            "mixed_over_fp64": (ms64 / ms) if ms64 else None,
            "mixed_errors_vs_fp64": mixed_err,
            "nbr_build_ms": nbr_ms,
            "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops, "unit": "TFLOP/s",
                         "frac": achieved_tflops / peak_tflops,
                         "traffic": (EFV_TRAFFIC_BYTES_PER_ATOM * n_atoms
                                     if EFV_TRAFFIC_BYTES_PER_ATOM and args.cells == CELLS[0] else None),
                         "peak_source": "measured (FP32 fma probe on this GPU, %s; SM clock %s MHz during the "
                                        "probe; nominal %.1f TFLOP/s = 152 SMs x 128 lanes x 2 x %.0f MHz)"
                                        % (peaks["how"], peaks["clocks"].get("sm_mhz"),
                                           SM_COUNT * FP32_LANES * 2 * max_mhz * 1e-6, max_mhz),
                         "flops_per_atom": flops_atom,
                         "flops_per_atom_note": "algorithmic: every Cartesian moment component swept per pair",
                         "executed_flops_per_atom": flops_atom_run,
                         "executed_tflops": executed_tflops,
                         "executed_frac": executed_tflops / peak_tflops},
            "fma_peaks_measured": peaks,
            "hbm": {"achieved": hbm_achieved, "peak": hbm_gbs, "unit": "GB/s", "frac": hbm_achieved / hbm_gbs,
                    "bytes_per_atom": bytes_atom, "peak_source": peak_src},
            "grade": grade,
            "batch": batch,
            "small_systems": small,
            "differentiation": diff,
            "md": md,
            "md_with_grade": md_graded,
            "cpu_baseline": cpu,
            "ms_per_step_median": statistics.median(per),
            "ms_per_step_min": min(per),
            "e2e": ({"value": job_rate(world, n_atoms, e2e_ms), "unit": UNIT, "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h} if e2e_ms else None),
            "e2e_with_neighbor_build": ({"value": job_rate(world, n_atoms, e2e_nb_ms), "unit": UNIT,
                                         "ms_per_step": e2e_nb_ms, "h2d_bytes_per_step": h2d,
                                         "d2h_bytes_per_step": d2h} if e2e_nb_ms else None),
            "gpu_launches": 3 * args.steps,   # fixed-point pass, energy/force kernel, FP64 force conversion
            "clocks": clocks,
        }
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-sample", type=int, default=256)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 comparison steps")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end steps")
    ap.add_argument("--no-grade", action="store_true", help="skip the extrapolation-grade workload")
    ap.add_argument("--grade-cells", type=int, default=100,
                    help="BCC cells along c of the grade box (50 x 50 x this; 100: the 500,000-atom workload)")
    ap.add_argument("--no-batch", action="store_true", help="skip the 4096-configuration batch workload")
    ap.add_argument("--no-diff", action="store_true", help="skip the level-20 differentiation workload")
    ap.add_argument("--no-md", action="store_true", help="skip the molecular-dynamics runs")
    ap.add_argument("--cells", type=int, default=CELLS[0], help="BCC cells per edge (80: the 1,024,000-atom "
                    "workload; smaller values only for profiling captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
