#!/usr/bin/env python
"""Benchmark of fast WQ/DWQ formation (arXiv 2211.06427) on one GB300 per rank.

Workload (default): the degree-4, 64^3-element gyroid mesh (sin6x cos6y + sin6y cos6z +
sin6z cos6x < 0.3 in [0,1]^3) with a log-normal B-spline coefficient field, Laplace
stiffness, octree depth 3.  Weight tables, classification and the CSR pattern are built once
(reported as setup_ms).  One step = one formation of the matrix values (coefficient at the
quadrature points, interior rows, cut-element matrices, cut rows), replayed from a CUDA
graph, in the mixed form (interior rows on the tensor cores in 3xTF32, cut-cell moments in
double).  Metric: nonzeros formed per second, median over the timed steps, next to the plain
FP64 GPU path on the same mesh, with the per-row error of both against the CPU oracle, the
degree sweep p = 2..6 and the paper's three-way comparison (DWQ / Hybrid / Standard Gauss).

Multi-GPU: meshes are formed independently, so N ranks run N replicas (weak scaling, no
collective on the data path); `value` = nnz of all replicas / max time.
`--impl reference` times the CPU oracle (C row oracle, all host cores) on bounded row samples
of the same workload.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2211_06427_gb300 import synthetic  # noqa: E402

METRIC = "nonzeros formed/s vs plain FP64 GPU path, p=2..6, at stated error; % roofline"
DTYPES = {"fp64": "f64", "fp32": "f32", "fp32_m64": "f32+f64", "tf32": "tf32", "tf32x3": "tf32x3",
          "tf32x3_m64": "tf32x3+f64", "bf16": "bf16"}
# per-row error bars the tests hold each precision to (relative Frobenius norm per row)
BARS = {"fp64": 1e-12, "fp32": 5e-5, "fp32_m64": 5e-5, "tf32x3": 5e-5, "tf32x3_m64": 5e-5, "tf32": 4e-3,
        "bf16": 1.5e-2}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="sfa", choices=["sfa", "reference"])
    ap.add_argument("--p", type=int, default=4)
    ap.add_argument("--n-el", type=int, default=64)
    ap.add_argument("--prec", default="tf32x3_m64", choices=list(DTYPES))
    ap.add_argument("--op", default="stiffness", choices=["mass", "stiffness"])
    ap.add_argument("--geometry", default="gyroid", choices=["gyroid", "full"])
    ap.add_argument("--batch-c5", action="store_true",
                    help="time the 64-mesh batch (one graph launch) against one FP64 call per mesh")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fp64-ref", action="store_true", help="skip the FP64 GPU comparison")
    ap.add_argument("--no-sweep", action="store_true", help="skip the degree sweep and the three-way table")
    ap.add_argument("--no-errors", action="store_true", help="skip the per-row error against the oracle")
    ap.add_argument("--sample-rows", type=int, default=600, help="rows of the oracle error sample")
    return ap.parse_args()


def workload(p, n_el, geometry):
    if geometry == "gyroid":
        return synthetic.c3_gyroid_64(p, n_el=n_el)
    return synthetic.c3_full_64(p, n_el=n_el)


def workload_name(p, n_el, geometry, op):
    g = "gyroid" if geometry == "gyroid" else "full cube"
    return f"{g} {n_el}^3, p={p}, {op}, log-normal B-spline c, octree depth 3"


# ------------------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part")):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ------------------------------------------------------------------------------------
# CPU legs: the C row oracle (oracle/sfrow.c, FP64, row loop + sum factorisation) in worker
# processes started with `spawn` before the first GPU call.  They return the oracle's rows
# for the per-row error statement and time the CPU baseline; nothing here feeds the GPU path.
_ORACLES = {}


def _desc_of(key):
    if key[0] == "plane":
        _, p, h = key
        return dict(synthetic.paper_plane(p, h), coef="analytic")
    p, n_el, geometry = key
    return workload(p, n_el, geometry)


def _oracle(key):
    """(OracleMesh, RowOracle) of a workload, built once per worker process."""
    if key not in _ORACLES:
        from oracle.formation import OracleMesh
        from oracle.sfrow import RowOracle
        om = OracleMesh(_desc_of(key))
        _ORACLES[key] = (om, RowOracle(om))
    return _ORACLES[key]


def _sample_rows(om, n, seed):
    """A seeded sample of active rows in the mesh's interior/cut proportions."""
    g = om.geo
    rng = np.random.default_rng(seed)
    ints = np.nonzero(g.fclass == 1)[0]
    cuts = np.nonzero(g.fclass == 2)[0]
    ni = int(round(n * len(ints) / max(1, len(ints) + len(cuts))))
    ni = min(ni, len(ints))
    rows = np.concatenate([rng.choice(ints, ni, replace=False),
                           rng.choice(cuts, min(n - ni, len(cuts)), replace=False)])
    return np.sort(rows).astype(np.int64), ni


def oracle_rows_job(key, op, nrows, seed, threads):
    """The oracle's values on a seeded row sample: {rows, lengths, values (concatenated)}."""
    om, ro = _oracle(key)
    rows, ni = _sample_rows(om, nrows, seed)
    ref = ro.rows(op, rows, threads=threads)
    return {"rows": rows, "lengths": np.array([len(ref[int(i)]) for i in rows]),
            "values": np.concatenate([ref[int(i)] for i in rows]), "n_interior": ni, "n_cut": len(rows) - ni}


def cpu_baseline_job(key, op, rows_all, rows_one, seed):
    """Time the oracle (C rows, FP64) on all host cores and on one core, on seeded samples in
    the mesh's row proportions; rules and boxes of the sample are prepared first, untimed."""
    om, ro = _oracle(key)
    cores = os.cpu_count() or 1
    out = {"cores": cores, "cpu": cpu_model()}
    for label, n, th, s in (("all", rows_all, cores, seed), ("one", rows_one, 1, seed + 1)):
        rows, ni = _sample_rows(om, n, s)
        ro._prepare_boxes(rows)
        t0 = time.perf_counter()
        ref = ro.rows(op, rows, threads=th)
        dt = time.perf_counter() - t0
        nnz = int(sum(len(v) for v in ref.values()))
        out[label] = {"nnz": nnz, "seconds": dt, "rows": len(rows), "interior": ni, "cut": len(rows) - ni,
                      "threads": th}
    return out


def row_error_stats(vals, rowptr, res):
    """max / median relative Frobenius error per row of GPU values against the oracle rows."""
    errs = []
    off = 0
    for i, n in zip(res["rows"], res["lengths"]):
        a, b = int(rowptr[i]), int(rowptr[i + 1])
        if b - a != n:
            raise RuntimeError("pattern length differs from the oracle's")
        ref = res["values"][off:off + n]
        off += n
        got = np.asarray(vals[a:b], dtype=np.float64)
        errs.append(float(np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)))
    return {"max_row_err": max(errs), "median_row_err": float(np.median(errs)), "rows": len(errs),
            "interior_rows": int(res["n_interior"]), "cut_rows": int(res["n_cut"])}


def run_reference(args):
    """The CPU oracle (C rows, FP64, all host cores) as it stands, on bounded row samples of
    the bench workload: each step forms a fresh seeded sample of rows."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    key = (args.p, args.n_el, args.geometry)
    om, ro = _oracle(key)
    cores = os.cpu_count() or 1
    nrows = max(8, args.sample_rows)
    for w in range(args.warmup):
        rows, _ = _sample_rows(om, nrows // 4, 1000 + w)
        ro.rows(args.op, rows, threads=cores)
    tot_nnz, tot_t = 0, 0.0
    for s in range(args.steps):
        rows, ni = _sample_rows(om, nrows, s)
        ro._prepare_boxes(rows)
        t0 = time.perf_counter()
        ref = ro.rows(args.op, rows, threads=cores)
        tot_t += time.perf_counter() - t0
        tot_nnz += int(sum(len(v) for v in ref.values()))
    value = tot_nnz / tot_t
    sample = (f"C row oracle (FP64, row loop + sum factorisation), {nrows} rows per step in the mesh's "
              f"interior/cut proportions, fresh seeded sample each step; geometry, rules and boxes untimed")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot_t / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_name(args.p, args.n_el, args.geometry, args.op), "p": args.p,
                   "n_el": args.n_el, "op": args.op},
        "cpu_baseline": {"value": value, "unit": "nnz/s", "cores": cores, "kind": "oracle-sf", "sample": sample,
                         "cpu": cpu_model()},
        "e2e": {"value": value, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------
# Algorithmic work per launch (the roofline numerators).
def moment_flops(p, n_pieces):
    """Cut-cell moments by sum factorisation over each octree piece's (p+1)^3 Gauss points:
    NB Q^3 + NB^2 Q^2 + NB^3 Q multiply-adds per piece (Q = p+1 points, NB = 2p+1 moments per
    direction), two FLOPs each."""
    q, nb = p + 1, 2 * p + 1
    return 2.0 * n_pieces * (nb * q ** 3 + nb * nb * q * q + nb ** 3 * q)


def elemmat_work(p, stiff, info):
    """FLOPs of one cut-element-matrix launch for a polynomial (B-spline or constant)
    coefficient, as the kernel performs them, split by precision:
    accumulation (the moment precision): per element the coefficient's Bernstein block
    3 Q^4 MAC, per piece M3 additions into its slot, per nonempty slot M3^2 MAC, per group
    M3^3 MAC (M3 = 3p+1 degree-3p moments per direction);
    maps (the value precision): per element the correlation with the coefficient NB^3 Q^3 MAC
    and the element-matrix expansion NT Q^2 NB^3 + c Q^4 NB^2 + c2 Q^6 NB MAC ((NT, c, c2) =
    (2, 3, 2) for stiffness, (1, 1, 1) for mass); Q = p+1, NB = 2p+1."""
    q, nb, m3 = p + 1, 2 * p + 1, 3 * p + 1
    ne = info["n_cut_elements"]
    acc = 2.0 * (ne * 3 * q ** 4 + info["moment_slots"] * m3 ** 2 + info["moment_groups"] * m3 ** 3) + \
        info["n_pieces"] * m3
    nt, c, c2 = (2, 3, 2) if stiff else (1, 1, 1)
    maps = 2.0 * ne * (nb ** 3 * q ** 3 + nt * q * q * nb ** 3 + c * q ** 4 * nb * nb + c2 * q ** 6 * nb)
    return acc, maps


def cutrows_flops(p, stiff, info):
    """Cut rows, from the classification's work counts: per (row, inside element outside the
    box) three sum-factorised Gauss stages, 7 Q^4 MAC for stiffness (3 Q^4 mass); per (row, cut
    element) Q^3 additions of an element-matrix row; per DWQ box NB NT m_f m_s m_t +
    NB^2 c2 m_s m_t + NB^3 c3 m_t MAC (NT = 2, c2 = 3, c3 = 2 for stiffness, 1 each for mass)."""
    q, nb = p + 1, 2 * p + 1
    nt, c2, c3 = (2, 3, 2) if stiff else (1, 1, 1)
    mac = ((7 if stiff else 3) * q ** 4 * info["cut_gauss_pairs"] + nb * nt * info["box_points_fst"] +
           nb * nb * c2 * info["box_points_st"] + nb ** 3 * c3 * info["box_points_t"])
    return 2.0 * mac + q ** 3 * info["cut_elem_pairs"]


# Non-tensor arithmetic peaks from unit counts and the maximum SM clock (2070 MHz):
# 152 SMs x 128 FP32 lanes x 2 FLOP per FMA; FP64 at the nominal 1.25 TFLOP/s.
SM_COUNT, FP32_LANES, MAX_SM_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * MAX_SM_MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = 1.25
FP32_SRC = "derived: 152 SMs x 128 FP32 lanes x 2 x 2070 MHz"
FP64_SRC = "nominal GB300 FP64 1.25 TFLOP/s"


def load_dram_per_unit():
    """DRAM bytes (read + write) per unit of work, from ncu captures of smaller cases of the
    same workloads (profiles/dram_per_unit.json); traffic grows with the units a launch
    processes, so a full launch is the per-unit figure times its units."""
    try:
        return json.load(open(os.path.join(ROOT, "profiles", "dram_per_unit.json")))["kernels"]
    except Exception:
        return {}


def dram_traffic(table, kernel, p, op, prec, units):
    e = table.get(kernel)
    if not e or [p, op, prec] != e["shape"] or units is None:
        return None
    return e["bytes_per_unit"] * units


# ------------------------------------------------------------------------------------
def _pool(workers):
    import concurrent.futures as cf
    import multiprocessing as mp
    try:
        return cf.ProcessPoolExecutor(max_workers=workers, mp_context=mp.get_context("spawn"))
    except Exception:
        return None


def _timed(fn, steps, warmup, stream, flush):
    """CUDA-event milliseconds of `steps` calls of fn on `stream`, L2 flushed (untimed) before
    each, after `warmup` untimed calls."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev = []
    for k in range(steps):
        flush.fill_(float(k))
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        ev.append((a, b))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def _result(fut, timeout=1800):
    if fut is None:
        return None
    try:
        return fut.result(timeout=timeout)
    except Exception as e:  # reported, never silently replaced
        return {"failed": f"{type(e).__name__}: {e}"}


def _err(vals, rowptr, res):
    if res is None or "failed" in res:
        return res
    return row_error_stats(vals.cpu().numpy(), rowptr, res)


def tensor_peak(prec, peaks):
    """Peak of the interior contractions (TFLOP/s): TF32 from the measured bf16 rate at the
    nominal dense ratio 1.1 / 2.25, divided by the passes of the split products."""
    bf16 = peaks.get("bf16_tflops", 1900.0)
    tf32 = bf16 * 1.1 / 2.25
    return {"tf32": tf32, "tf32x3": tf32 / 3, "tf32x3_m64": tf32 / 3, "bf16": bf16}.get(prec)


def kernel_rooflines(args, mesh, prec, ms4, peaks, dram, world):
    """Roofline objects of the four stages from their serialised device times."""
    info = mesh.info
    p, stiff = args.p, args.op == "stiffness"
    vsize = 8 if prec == "fp64" else 4
    hbm = peaks.get("hbm_gbs", 6800.0)
    hsrc = "measured hbm_gbs" if "hbm_gbs" in peaks else "fallback 6.8 TB/s"
    mom64 = prec in ("fp64", "fp32_m64", "tf32x3_m64")
    ne = mesh.desc["n_el"]
    nsup = np.prod([e * (p + 1) for e in ne])                      # Gauss superset grid
    nq = np.prod([2 * (p + 1) + 2 * max(0, e - 2) for e in ne])    # weighted-quadrature grid
    out = {}
    units = {"coefficient": (float(nsup + nq) * vsize, "hbm", None),
             "interior_rows": (info["nnz_interior"] * vsize, "hbm", info["nnz_interior"]),
             "cut_element_matrices": (moment_flops(p, info["n_pieces"]), "alu", info["n_cut_elements"]),
             "cut_rows": (cutrows_flops(p, stiff, info), "alu", info["n_cut_rows"])}
    names = {"coefficient": "k_coef", "interior_rows": "k_interior_tc3" if prec in ("tf32", "tf32x3", "tf32x3_m64", "bf16") else "k_interior_reg",
             "cut_element_matrices": "k_cut_elemmat", "cut_rows": "k_cut_rows"}
    for (stage, (work, bound, unit_count)), t in zip(units.items(), ms4):
        if t <= 0:
            continue
        if stage == "cut_element_matrices" and mesh.desc.get("coef") in ("bspline", "const"):
            # two pipes: the accumulation in the moment precision, the maps in the value one
            acc, maps = elemmat_work(p, stiff, info)
            pa = FP64_PEAK_TFLOPS if mom64 else FP32_PEAK_TFLOPS
            pm = FP64_PEAK_TFLOPS if prec == "fp64" else FP32_PEAK_TFLOPS
            t_min = acc / (pa * 1e12) + maps / (pm * 1e12)
            work = acc + maps
            ach, peak = work / (t / 1e3) / 1e12, work / t_min / 1e12
            out[stage] = {"bound": "alu", "kernel": "k_cut_elemmat_b3p", "achieved": ach, "peak": peak,
                          "unit": "TFLOP/s", "frac": ach / peak,
                          "peak_source": f"{FP64_SRC if mom64 else FP32_SRC} for the accumulation "
                                         f"({acc / 1e9:.2f} GFLOP), {FP64_SRC if prec == 'fp64' else FP32_SRC} "
                                         f"for the maps ({maps / 1e9:.2f} GFLOP); peak = work / sum of the two "
                                         f"times at peak",
                          "traffic": dram_traffic(dram, "k_cut_elemmat_b3p", p, args.op, prec, unit_count),
                          "algorithmic_per_launch": work, "serial_ms": t, "share_of_serial": t / sum(ms4)}
            continue
        if bound == "hbm":
            ach, peak, unit, src = work / (t / 1e3) / 1e9, hbm, "GB/s", hsrc
        else:
            f64 = mom64 if stage == "cut_element_matrices" else prec == "fp64"
            ach = work / (t / 1e3) / 1e12
            peak, unit = (FP64_PEAK_TFLOPS, "TFLOP/s") if f64 else (FP32_PEAK_TFLOPS, "TFLOP/s")
            src = FP64_SRC if f64 else FP32_SRC
        out[stage] = {"bound": bound, "kernel": names[stage], "achieved": ach, "peak": peak, "unit": unit,
                      "frac": ach / peak, "peak_source": src,
                      "traffic": dram_traffic(dram, names[stage], p, args.op, prec, unit_count),
                      "algorithmic_per_launch": work, "serial_ms": t, "share_of_serial": t / sum(ms4)}
    return out


def run_c5(args):
    """64 independent meshes (n_el ~ U{8..48}, p ~ U{2..5}, 1-8 balls, analytic c): the whole
    batch formed by one graph launch (tiles autotuned per degree) against one call per mesh
    in FP64 and in the batch's precision.  Setup (tables, classification) is untimed."""
    import torch
    from paper_2211_06427_gb300 import sfa
    torch.cuda.set_device(0)
    descs = synthetic.c5_batch()
    meshes = [sfa.Mesh(d) for d in descs]
    nnz = sum(m.nnz for m in meshes)
    stream = torch.cuda.current_stream()
    prec = args.prec if args.prec != "fp64" else "fp32"
    tuned = {}
    for m, d in zip(meshes, descs):
        if (d["p"], prec) not in tuned:
            m.autotune(args.op, prec)
            tuned[(d["p"], prec)] = sfa.get_tuning(d["p"], args.op, prec)
    outs = [torch.empty(max(m.nnz, 1), dtype=torch.float32, device="cuda") for m in meshes]
    outs64 = [torch.empty(max(m.nnz, 1), dtype=torch.float64, device="cuda") for m in meshes]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    t_batch = float(np.median(_timed(lambda: sfa.form_batched(meshes, args.op, prec, outs=outs), args.steps,
                                     args.warmup, stream, flush)))
    t_single = float(np.median(_timed(lambda: [m.form(args.op, prec, out=o) for m, o in zip(meshes, outs)],
                                      args.steps, args.warmup, stream, flush)))
    t_fp64 = float(np.median(_timed(lambda: [m.form(args.op, "fp64", out=o) for m, o in zip(meshes, outs64)],
                                    max(1, args.steps // 2), 1, stream, flush)))
    line = {"metric": "nonzeros formed/s, 64-mesh batch", "value": nnz / (t_batch / 1000.0), "unit": "nnz/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_batch,
            "higher_is_better": True, "dtype": DTYPES[prec], "data": "synthetic",
            "config": {"workload": "C5: 64 meshes, n_el ~ U{8..48}, p ~ U{2..5}, 1-8 balls, analytic c, depth 3",
                       "op": args.op, "precision": prec, "nnz": nnz,
                       "tuning": {f"p={p}": list(v) for (p, _), v in sorted(tuned.items())}},
            "one_call_per_mesh_ms": t_single, "fp64_one_call_per_mesh_ms": t_fp64,
            "speedup_vs_fp64_per_mesh": t_fp64 / t_batch, "speedup_vs_same_precision_per_mesh": t_single / t_batch}
    print(json.dumps(line), flush=True)


def sweep_and_variants(args, sfa, stream, flush, futs, head):
    """Degree sweep p = 2..6 on the bench geometry (mixed form and FP64, nnz/s and per-row error)
    and the paper's three-way comparison (Sec. 3.1: DWQ / Hybrid Gauss / Standard Gauss) on its
    own plane geometry at h = 32, mass matrix, FP64 and the mixed form."""
    import torch
    sweep = []
    for p in range(2, 7):
        if p == args.p:
            sweep.append(head)
            continue
        m = sfa.Mesh(workload(p, args.n_el, args.geometry))
        rowptr = m.pattern()[0].cpu().numpy()
        v = torch.empty(max(1, m.nnz), dtype=torch.float32, device="cuda")
        v64 = torch.empty(max(1, m.nnz), dtype=torch.float64, device="cuda")
        tm = float(np.median(_timed(lambda: sfa.form_batched([m], args.op, args.prec, outs=[v]), 5, 2, stream,
                                    flush)))
        t64 = float(np.median(_timed(lambda: sfa.form_batched([m], args.op, "fp64", outs=[v64]), 3, 1, stream,
                                     flush)))
        res = _result(futs.get(("sweep", p)))
        sweep.append({"p": p, "nnz": m.nnz, "ms": tm, "nnz_per_s": m.nnz / (tm / 1e3), "fp64_ms": t64,
                      "fp64_nnz_per_s": m.nnz / (t64 / 1e3), "speedup_vs_fp64": t64 / tm,
                      "error": _err(v, rowptr, res), "fp64_error": _err(v64, rowptr, res)})
        m.close()
        del v, v64
        torch.cuda.empty_cache()
    three = []
    for p in range(2, 7):
        m = sfa.Mesh(dict(synthetic.paper_plane(p, 32), coef="analytic"))
        row = {"p": p, "nnz": m.nnz}
        for prec in ("fp64", args.prec):
            v = torch.empty(max(1, m.nnz), dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
            for variant in ("dwq", "hybrid", "gauss"):
                t = float(np.median(_timed(lambda: m.form("mass", prec, out=v, variant=variant), 5, 1, stream,
                                           flush)))
                row[f"{variant}_{prec}_ms"] = t
            row[f"hybrid_over_dwq_{prec}"] = row[f"hybrid_{prec}_ms"] / row[f"dwq_{prec}_ms"]
            row[f"gauss_over_dwq_{prec}"] = row[f"gauss_{prec}_ms"] / row[f"dwq_{prec}_ms"]
        three.append(row)
        m.close()
    return sweep, three


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.batch_c5:
        run_c5(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    # CPU oracle legs in spawned workers, started before the first GPU call: one worker for
    # the bench workload (its error sample, then the timed CPU baseline), others for the sweep
    head_key = (args.p, args.n_el, args.geometry)
    cores = os.cpu_count() or 1
    futs, head_pool, sweep_pool = {}, None, None
    if rank == 0 and world == 1 and not (args.no_errors and args.no_cpu_baseline):
        head_pool = _pool(1)
        if head_pool and not args.no_errors:
            futs["head"] = head_pool.submit(oracle_rows_job, head_key, args.op, args.sample_rows, 11,
                                            max(1, cores // 2))
        if not args.no_errors and not args.no_sweep:
            sweep_pool = _pool(max(1, min(4, cores // 4)))
            if sweep_pool:
                for p in range(2, 7):
                    if p != args.p:
                        futs[("sweep", p)] = sweep_pool.submit(oracle_rows_job, (p, args.n_el, args.geometry),
                                                               args.op, 150, 20 + p, max(1, cores // 8))
    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2211_06427_gb300 import sfa

    desc = workload(args.p, args.n_el, args.geometry)
    stream = torch.cuda.current_stream()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MiB > L2
    mesh = sfa.Mesh(desc, setup=False)
    setup_ms = []
    for k in range(3):  # tables + classification (synchronises inside), host wall clock
        flush.fill_(float(k))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mesh.build_tables()
        mesh.classify()
        torch.cuda.synchronize()
        setup_ms.append(1e3 * (time.perf_counter() - t0))
    nnz, info = mesh.nnz, mesh.info
    rowptr = mesh.pattern()[0].cpu().numpy()
    vdtype = torch.float64 if args.prec == "fp64" else torch.float32
    vals = torch.empty(max(1, nnz), dtype=vdtype, device="cuda")

    def step():  # one formation, replayed from the CUDA graph the library captured for it
        sfa.form_batched([mesh], args.op, args.prec, outs=[vals])

    l0 = sfa.launch_count()
    step()  # captures the graph
    torch.cuda.synchronize()
    per_step = sfa.launch_count() - l0  # kernels in the graph, launched by every replay
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms = _timed(step, args.steps, 0, stream, flush)
    if dist:
        dist.barrier()
    ms = float(np.median(step_ms))
    if dist:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    value = world * nnz / (ms / 1000.0)
    clocks = clk.summary()

    # per-stage device times with the stages serialised (the roofline denominators)
    prof = [mesh.form_profile(args.op, args.prec, out=vals)[1] for _ in range(3)]
    ms4 = [float(np.median([pr[k] for pr in prof])) for k in range(4)]
    step()
    torch.cuda.synchronize()
    head = {"p": args.p, "nnz": nnz, "ms": ms, "nnz_per_s": nnz / (ms / 1e3)}
    if "head" in futs:
        head["error"] = _err(vals, rowptr, _result(futs["head"]))

    # the plain FP64 GPU path on the same mesh (the metric's comparison)
    fp64_ref = None
    if args.prec != "fp64" and not args.no_fp64_ref:
        vals64 = torch.empty(max(1, nnz), dtype=torch.float64, device="cuda")
        t64 = _timed(lambda: sfa.form_batched([mesh], args.op, "fp64", outs=[vals64]), 5, 1, stream, flush)
        m64 = float(np.median(t64))
        fp64_ref = {"ms_per_step": m64, "value": nnz / (m64 / 1000.0), "unit": "nnz/s", "steps": len(t64)}
        if "head" in futs:
            fp64_ref["error"] = _err(vals64, rowptr, _result(futs["head"]))
        head.update(fp64_ms=m64, fp64_nnz_per_s=fp64_ref["value"], speedup_vs_fp64=m64 / ms,
                    fp64_error=fp64_ref.get("error"))
        del vals64
        torch.cuda.empty_cache()

    # end to end through the host-buffer entry point: coefficients in, values out, every step
    e2e = None
    if not args.no_e2e:
        coef_h = torch.as_tensor(desc["coef_bspline"]).pin_memory() if desc["coef"] == "bspline" else None
        vals_h = torch.empty(nnz, dtype=vdtype).pin_memory()
        e_ms = _timed(lambda: mesh.form_host(args.op, args.prec, coef_h, vals_h), args.steps, 2, stream, flush)
        em = float(np.median(e_ms))
        if dist:
            t = torch.tensor([em], device="cuda", dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            em = float(t.item())
        e2e = {"value": world * nnz / (em / 1000.0), "unit": "nnz/s",
               "h2d_bytes_per_step": int(coef_h.numel() * 8) if coef_h is not None else 0,
               "d2h_bytes_per_step": int(nnz * vals_h.element_size()), "ms_per_step": em,
               "call": "sfa_form_host (host coefficients in, host values out, synchronous)"}

    sweep, three = (None, None)
    if not args.no_sweep and rank == 0:
        sweep, three = sweep_and_variants(args, sfa, stream, flush, futs, head)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    roofs = kernel_rooflines(args, mesh, args.prec, ms4, peaks, load_dram_per_unit(), world)
    dominant = max(roofs, key=lambda k: roofs[k]["serial_ms"]) if roofs else None
    # whole matrix: achieved nnz/s against the slower of the value stream over HBM and the
    # stage-3 floor of the contractions (8 (p+1) FLOP per nonzero for stiffness, 4 (p+1) mass)
    vsize = 8 if args.prec == "fp64" else 4
    fpn = (8 if args.op == "stiffness" else 4) * (args.p + 1)
    cpeak = tensor_peak(args.prec, peaks) or (FP64_PEAK_TFLOPS if args.prec == "fp64" else FP32_PEAK_TFLOPS)
    hbm_nnz = peaks.get("hbm_gbs", 6800.0) * 1e9 / vsize
    bound_nnz = min(hbm_nnz, cpeak * 1e12 / fpn)
    roof_matrix = {"achieved_nnz_per_s": value / world, "bound_nnz_per_s": bound_nnz,
                   "frac": value / world / bound_nnz,
                   "bound": "hbm" if hbm_nnz <= cpeak * 1e12 / fpn else "compute",
                   "model": f"min(HBM {vsize} B/nnz, contraction peak {cpeak:.1f} TFLOP/s / {fpn} FLOP/nnz)"}

    cpu = None
    if head_pool and not args.no_cpu_baseline:
        for k, f in futs.items():  # the oracle jobs finish before the CPU timing starts
            _result(f)
        if sweep_pool:
            sweep_pool.shutdown(wait=True)
            sweep_pool = None
        res = _result(head_pool.submit(cpu_baseline_job, head_key, args.op, 4000, 300, 77))
        if res and "failed" not in res:
            a, o = res["all"], res["one"]
            cpu = {"value": a["nnz"] / a["seconds"], "unit": "nnz/s", "cores": a["threads"], "kind": "oracle-sf",
                   "cpu": res["cpu"], "nproc": res["cores"],
                   "sample": (f"C row oracle (FP64, row loop + sum factorisation): {a['rows']} rows "
                              f"({a['interior']} interior, {a['cut']} cut, mesh proportions), "
                              f"{a['nnz']} nnz in {a['seconds']:.2f} s on {a['threads']} threads; "
                              f"geometry, rules and boxes untimed"),
                   "one_core": {"value": o["nnz"] / o["seconds"], "unit": "nnz/s", "rows": o["rows"],
                                "seconds": o["seconds"]}}
        else:
            cpu = {"value": None, "unit": "nnz/s", "cores": cores, "kind": "oracle-sf", "sample": str(res)}
    for pl in (head_pool, sweep_pool):
        if pl:
            pl.shutdown(wait=False, cancel_futures=True)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "nnz/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "ms_per_step_mean": float(np.mean(step_ms)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": DTYPES[args.prec],
            "data": "synthetic",
            "config": {"workload": workload_name(args.p, args.n_el, args.geometry, args.op), "p": args.p,
                       "n_el": args.n_el, "op": args.op, "precision": args.prec, "variant": "dwq", "nnz": nnz,
                       "interior_rows": info["n_interior_rows"], "cut_rows": info["n_cut_rows"],
                       "box_rows": info["n_box_rows"], "cut_elements": info["n_cut_elements"],
                       "pieces": info["n_pieces"],
                       "l2": "flushed between steps (256 MiB write, outside the timed events)",
                       "parallelism": f"replicas{world}",
                       "step": "one formation (sfa_form replayed from its CUDA graph); tables, classification "
                               "and pattern built once (setup_ms)"},
            "setup_ms": float(np.median(setup_ms)),
            "stages_ms_serial": dict(zip(["coefficient", "interior_rows", "cut_element_matrices", "cut_rows"], ms4)),
            "error": {"precision": args.prec, "bar": BARS[args.prec], **(head.get("error") or {})},
            "fp64_gpu": fp64_ref,
            "speedup_vs_fp64_gpu": (value / world / fp64_ref["value"]) if fp64_ref else None,
            "sweep": sweep, "paper_three_way": three,
            "roofline": roofs.get(dominant), "roofline_dominant_stage": dominant, "rooflines": roofs,
            "roofline_interior": roofs.get("interior_rows"), "roofline_matrix": roof_matrix,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(per_step * args.steps), "gpu_launches_per_step": int(per_step),
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
