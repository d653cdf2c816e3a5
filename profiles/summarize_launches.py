"""Summarise an ncu --csv launch list (gpu__time_duration.sum) per kernel.

usage: python profiles/summarize_launches.py launches.csv
Prints launches, total device time and share per kernel.  Per-launch times
under ncu are cold-cache and serialised: compare shares, not absolutes.
"""
import collections
import csv
import sys

SCALE = {"ns": 1e-6, "nsecond": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0,
         "s": 1e3, "second": 1e3}


def main(path):
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
    T = sum(v[1] for v in tot.values())
    print(f"{'launches':>8} {'total ms':>10} {'share':>7}  kernel")
    for k, (n, t) in sorted(tot.items(), key=lambda x: -x[1][1]):
        print(f"{n:8d} {t:10.3f} {100 * t / T:6.2f}%  {k}")


if __name__ == "__main__":
    main(sys.argv[1])
