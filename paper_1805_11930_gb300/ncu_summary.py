"""Per-kernel summary of an ncu launch list.

    python -m paper_1805_11930_gb300.ncu_summary launches.csv [more.csv ...]

Reads the CSV that `ncu --metrics gpu__time_duration.sum --csv --log-file`
writes (one row per captured launch) and prints, per kernel name (template
arguments kept, parameter list dropped), the number of launches, the summed
device time, its share of the total and the mean time per launch, largest
share first.  ncu serialises launches and runs them with cold caches, so the
shares are the meaningful figures, not the absolute times.
"""
import collections
import csv
import sys

_UNIT_NS = {"nsecond": 1.0, "ns": 1.0, "usecond": 1e3, "us": 1e3, "msecond": 1e6, "ms": 1e6, "second": 1e9, "s": 1e9}


def kernel_times(path):
    """{kernel: [launches, total ns]} from one ncu CSV launch list."""
    with open(path, newline="") as fh:
        rows = list(csv.reader(fh))
    head = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    h = rows[head]
    ki, mi, vi, ui = (h.index(k) for k in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    out = collections.defaultdict(lambda: [0, 0.0])
    for r in rows[head + 1:]:
        if len(r) <= vi or r[mi] != "gpu__time_duration.sum":
            continue
        ns = float(r[vi].replace(",", "")) * _UNIT_NS.get(r[ui], 1.0)
        name = r[ki].split("(")[0].replace("void ", "").replace("dgmg::<unnamed>::", "").replace("dgmg::", "")
        out[name][0] += 1
        out[name][1] += ns
    return out


def summary(paths):
    tot = collections.defaultdict(lambda: [0, 0.0])
    for p in paths:
        for k, (c, ns) in kernel_times(p).items():
            tot[k][0] += c
            tot[k][1] += ns
    T = sum(v[1] for v in tot.values()) or 1.0
    lines = [f"launches {sum(v[0] for v in tot.values())}  total {T / 1e6:.3f} ms",
             f"{'share':>7} {'launches':>8} {'total ms':>10} {'ms/launch':>10}  kernel"]
    for k, (c, ns) in sorted(tot.items(), key=lambda x: -x[1][1]):
        lines.append(f"{ns / T * 100:6.2f}% {c:8d} {ns / 1e6:10.3f} {ns / 1e6 / c:10.4f}  {k}")
    return "\n".join(lines)


if __name__ == "__main__":
    print(summary(sys.argv[1:]))
