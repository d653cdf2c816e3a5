"""Short text summaries of Nsight Compute output (the figures the profiles
and the roofline use).

    python -m paper_2502_11129_b300.ncu_summary launches launches.csv
        per kernel of an `ncu --metrics gpu__time_duration.sum --csv` launch
        list: launches, total device time and share.  Per-launch times under
        ncu are cold-cache and serialised: compare shares, not absolutes.

    python -m paper_2502_11129_b300.ncu_summary capture prof.ncu-rep
        the headline counters of one captured launch (`ncu --set full`):
        duration, DRAM bytes, issue activity, pipe use, occupancy and the
        warp stall breakdown (cycles per issued instruction).
"""
from __future__ import annotations

import collections
import csv
import io
import subprocess
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
         "s": 1e3, "second": 1e3}

CAPTURE_METRICS = [
    "gpu__time_duration.sum",
    "launch__grid_size",
    "launch__block_size",
    "launch__registers_per_thread",
    "launch__shared_mem_per_block_dynamic",
    "launch__occupancy_limit_registers",
    "launch__occupancy_limit_shared_mem",
    "sm__warps_active.avg.per_cycle_active",
    "smsp__issue_active.avg.pct_of_peak_sustained_active",
    "smsp__inst_executed.sum",
    "smsp__thread_inst_executed_per_inst_executed.ratio",
    "sm__pipe_fma_cycles_active.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fma.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_alu.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_fp64.avg.pct_of_peak_sustained_active",
    "sm__inst_executed_pipe_lsu.avg.pct_of_peak_sustained_active",
    "sm__pipe_tensor_cycles_active.avg.pct_of_peak_sustained_active",
    "dram__bytes_read.sum",
    "dram__bytes_write.sum",
    "gpu__dram_throughput.avg.pct_of_peak_sustained_elapsed",
    "l1tex__t_sector_hit_rate.pct",
    "lts__t_sector_hit_rate.pct",
    "l1tex__data_bank_conflicts_pipe_lsu_mem_shared.sum",
]
STALL_PREFIX = "smsp__average_warps_issue_stalled_"
STALL_SUFFIX = "_per_issue_active.ratio"


def launches(path: str) -> str:
    rows = list(csv.reader(open(path)))
    h = [i for i, r in enumerate(rows) if r and r[0] == "ID"][0]
    hdr = rows[h]
    ki, mi, vi, ui = (hdr.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    tot = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[h + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        name = r[ki].split("(")[0]
        tot[name][0] += 1
        tot[name][1] += float(r[vi].replace(",", "")) * SCALE[r[ui]]
    total = sum(v[1] for v in tot.values())
    out = [f"{'launches':>8} {'total ms':>10} {'share':>7}  kernel"]
    for k, (n, t) in sorted(tot.items(), key=lambda x: -x[1][1]):
        out.append(f"{n:8d} {t:10.3f} {100 * t / total:6.2f}%  {k}")
    return "\n".join(out)


def capture(path: str) -> str:
    raw = subprocess.run(["ncu", "-i", path, "--page", "raw", "--csv"], check=True, capture_output=True,
                         text=True).stdout
    rows = list(csv.reader(io.StringIO(raw)))
    hdr, units = rows[0], rows[1]
    out = []
    for r in rows[2:]:
        name = r[hdr.index("Kernel Name")] if "Kernel Name" in hdr else "?"
        out.append(f"kernel: {name.split('(')[0]}")
        for k in CAPTURE_METRICS:
            if k in hdr:
                i = hdr.index(k)
                out.append(f"  {k} = {r[i]} {units[i]}".rstrip())
        stalls = []
        for i, k in enumerate(hdr):
            if k.startswith(STALL_PREFIX) and k.endswith(STALL_SUFFIX):
                try:
                    v = float(r[i])
                except ValueError:
                    continue
                if v >= 0.05:
                    stalls.append((v, k[len(STALL_PREFIX):-len(STALL_SUFFIX)]))
        out.append("  warp stalls (cycles per issued instruction): " +
                   ", ".join(f"{n} {v:.2f}" for v, n in sorted(stalls, reverse=True)))
    return "\n".join(out)


def main(argv):
    if len(argv) != 3 or argv[1] not in ("launches", "capture"):
        print(__doc__)
        return 2
    print(launches(argv[2]) if argv[1] == "launches" else capture(argv[2]))
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv))
