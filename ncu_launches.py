"""Per-kernel totals of an ncu launch list (``--metrics gpu__time_duration.sum --csv``).

Usage: python ncu_launches.py launches.csv
Prints one row per kernel: launches, total device time and share of the total.
"""
import collections
import csv
import sys


def summarise(path):
    with open(path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    rows = list(csv.DictReader(lines))
    agg = collections.defaultdict(lambda: [0, 0.0])
    for r in rows:
        if r.get("Metric Name") != "gpu__time_duration.sum":
            continue
        # namespaces first: "(anonymous namespace)" holds a parenthesis too
        name = r["Kernel Name"]
        for pre in ("(anonymous namespace)::", "<unnamed>::", "adc::"):
            name = name.replace(pre, "")
        name = name.split("(")[0]
        scale = {"ns": 1e-6, "us": 1e-3, "usecond": 1e-3, "ms": 1.0, "msecond": 1.0}.get(r["Metric Unit"], 1e-6)
        a = agg[name]
        a[0] += 1
        a[1] += float(r["Metric Value"].replace(",", "")) * scale
    return agg


if __name__ == "__main__":
    agg = summarise(sys.argv[1])
    tot = sum(v[1] for v in agg.values())
    print(f"{'kernel':44s} {'launches':>8s} {'total ms':>10s} {'share':>7s}")
    for k, v in sorted(agg.items(), key=lambda x: -x[1][1]):
        print(f"{k[:44]:44s} {v[0]:8d} {v[1]:10.2f} {100 * v[1] / tot:6.2f}%")
    print(f"{'total':44s} {sum(v[0] for v in agg.values()):8d} {tot:10.2f}")
