"""Summarises an ncu launch list (--metrics gpu__time_duration.sum --csv) per kernel:
launches, total device time and share.  Usage: python profiles/summarize_launches.py FILE.csv"""
import csv
import re
import sys
from collections import defaultdict


def main(path):
    rows = list(csv.reader(open(path)))
    hdr = None
    for i, r in enumerate(rows):
        if "Kernel Name" in r and "Metric Name" in r:
            hdr, rows = r, rows[i + 1:]
            break
    k_name, k_metric, k_val, k_unit = (hdr.index(x) for x in ("Kernel Name", "Metric Name", "Metric Value", "Metric Unit"))
    tot = defaultdict(float)
    cnt = defaultdict(int)
    for r in rows:
        if len(r) <= k_val or r[k_metric] != "gpu__time_duration.sum":
            continue
        name = re.sub(r"\(.*", "", r[k_name]).replace("void ", "").strip()
        name = re.sub(r"<unnamed>::|\(anonymous namespace\)::", "", name)
        v = float(r[k_val].replace(",", ""))
        unit = r[k_unit]
        v *= {"ns": 1e-6, "usecond": 1e-3, "us": 1e-3, "msecond": 1.0, "ms": 1.0, "nsecond": 1e-6}.get(unit, 1.0)
        tot[name] += v
        cnt[name] += 1
    all_ms = sum(tot.values())
    print(f"{'kernel':70s} {'launches':>9s} {'total ms':>11s} {'share':>7s}")
    for name in sorted(tot, key=lambda n: -tot[n]):
        print(f"{name[:70]:70s} {cnt[name]:9d} {tot[name]:11.3f} {100 * tot[name] / all_ms:6.2f}%")
    print(f"{'all':70s} {sum(cnt.values()):9d} {all_ms:11.3f}")


if __name__ == "__main__":
    main(sys.argv[1])
