"""Per-cell DRAM traffic of a collide kernel, from an ncu capture, as an
entry of the traffic table the benchmark reads (profiles/traffic.json).

Run right after the capture, on the machine that made it:

  ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum \\
      --clock-control none -k regex:k_collide -s 2 -c 1 --csv --log-file cap.csv \\
      python -m paper_1505_02037_gb300.profile_step --storage f32 --n 128 --variant P1-reread
  python -m paper_1505_02037_gb300.traffic_table cap.csv \\
      --key k_collide:gauge3d-256-f32:P1-reread --cells 2097152 --out traffic_new.json \\
      --captured-on "D3Q19 FP32 128^3 gauge wave, one launch" --command "<the ncu line>"

The entry records the hash of the kernel sources as they are when this
script runs, beside the capture: an entry's hash is therefore never newer
than its counters, and the benchmark ignores an entry whose hash differs
from the sources it runs (the kernel changed since the counters were taken).
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))

# Sources the collide-and-stream kernels of the 3D lattice are built from.
COLLIDE_SOURCES = ("collide_tma.cuh", "dispatch.h", "instantiate.cuh",
                   "kernels.cuh", "lattice.cuh", "physics.cuh", "inst_q19_s0.cu",
                   "inst_q19_s1.cu", "inst_q19_s2.cu", "inst_q19_s3.cu", "inst_q19_s4.cu")
# Sources the 37-field collide kernel is built from.
AD_SOURCES = ("ad.cuh", "ad_q19_f32.cu", "dispatch.h", "kernels.cuh", "lattice.cuh",
              "physics.cuh")
# Sources of the batched ensemble kernel.
BATCH_SOURCES = ("batch.cu", "dispatch.h", "kernels.cuh", "lattice.cuh", "physics.cuh")


def source_hash(files=COLLIDE_SOURCES) -> str:
    h = hashlib.sha256()
    d = os.path.join(HERE, "csrc")
    for n in sorted(files):
        with open(os.path.join(d, n), "rb") as f:
            h.update(n.encode() + f.read())
    return h.hexdigest()[:16]


def read_ncu_csv(path, kernel_substring):
    """Per-launch metrics {name: value} of the launches whose kernel name
    contains kernel_substring, from ncu --csv output (one row per metric)."""
    launches = {}
    with open(path, newline="") as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for row in csv.DictReader(lines):
        if kernel_substring not in row.get("Kernel Name", ""):
            continue
        key = row["ID"]
        unit = row.get("Metric Unit", "")
        v = float(row["Metric Value"].replace(",", ""))
        # bytes as bytes, durations in milliseconds
        scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1e-6,
                 "ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0}.get(unit, 1.0)
        launches.setdefault(key, {})[row["Metric Name"]] = v * scale
    return list(launches.values())


def main(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("csv")
    p.add_argument("--key", required=True)
    p.add_argument("--kernel", default="k_collide")
    p.add_argument("--cells", type=int, required=True)
    p.add_argument("--sources", default="collide", choices=["collide", "ad", "batch"])
    p.add_argument("--captured-on", required=True)
    p.add_argument("--command", required=True)
    p.add_argument("--out", required=True)
    p.add_argument("--flops-per-cell", type=float, default=None)
    a = p.parse_args(argv)
    files = {"collide": COLLIDE_SOURCES, "ad": AD_SOURCES, "batch": BATCH_SOURCES}[a.sources]
    rows = read_ncu_csv(a.csv, a.kernel)
    if not rows:
        print(f"no launch of {a.kernel} in {a.csv}")
        return 2
    m = rows[-1]
    rd = m["dram__bytes_read.sum"] / a.cells
    wr = m["dram__bytes_write.sum"] / a.cells
    entry = {"source_hash": source_hash(files), "dram_bytes_per_cell": round(rd + wr, 1),
             "dram_read_bytes_per_cell": round(rd, 1), "dram_write_bytes_per_cell": round(wr, 1),
             "launch_ms_under_ncu": round(m.get("gpu__time_duration.sum", float("nan")), 4),
             "captured_on": a.captured_on, "command": a.command}
    if a.flops_per_cell is not None:
        entry["fp64_flops_per_cell"] = a.flops_per_cell
    ops = {k: m.get(f"smsp__sass_thread_inst_executed_op_{k}_pred_on.sum")
           for k in ("dadd", "dmul", "dfma")}
    if all(v is not None for v in ops.values()):
        # FP64 flops with a fused multiply-add counted as two
        entry["fp64_instructions_per_cell"] = round(sum(ops.values()) / a.cells, 1)
        entry["fp64_flops_per_cell"] = round((ops["dadd"] + ops["dmul"] + 2 * ops["dfma"]) /
                                             a.cells, 1)
    table = {}
    if os.path.exists(a.out):
        with open(a.out) as f:
            table = json.load(f)
    table[a.key] = entry
    with open(a.out, "w") as f:
        json.dump(table, f, indent=1)
    print(json.dumps({a.key: entry}))
    return 0


if __name__ == "__main__":
    sys.exit(main())
