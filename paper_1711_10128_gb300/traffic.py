"""Record the DRAM traffic of a kernel family from an ncu capture.

The bench reports `roofline.traffic`, the DRAM bytes one launch of the
dominant kernel family moves, as the DRAM-bytes-per-algorithmic-byte ratio
measured by ncu times the launch's algorithmic bytes.  This script computes
that ratio from the raw page of an ncu report (`ncu -i REPORT --page raw
--csv`) for the launches whose kernel name matches a pattern, given the
algorithmic bytes of those launches, and stores it in profiles/traffic.json
under "<workload>/<family>" together with the sha256 of the kernel sources it
was measured on; the bench withdraws the figure (reports null) as soon as any
of those sources changes.

Usage:
  python -m paper_1711_10128_gb300.traffic RAW.csv WORKLOAD FAMILY KERNEL_REGEX ALG_BYTES_PER_LAUNCH \\
      SOURCE [SOURCE ...] --command "the ncu command line"
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "profiles", "traffic.json")


def _num(s):
    return float(s.replace(",", "")) if s not in ("", "n/a") else None


def launches(raw_csv, kernel_regex):
    """(kernel name, dram read bytes, dram write bytes, duration ns) of every
    matching launch in an ncu raw CSV page."""
    rows = list(csv.reader(open(raw_csv)))
    hdr, units = rows[0], rows[1]
    col = {h: i for i, h in enumerate(hdr)}
    scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0, "usecond": 1e3,
             "msecond": 1e6, "ns": 1.0, "us": 1e3, "ms": 1e6}
    out = []
    for r in rows[2:]:
        name = r[col["Kernel Name"]]
        if not re.search(kernel_regex, name):
            continue
        vals = []
        for m in ("dram__bytes_read.sum", "dram__bytes_write.sum", "gpu__time_duration.sum"):
            v = _num(r[col[m]])
            vals.append(None if v is None else v * scale.get(units[col[m]], 1.0))
        out.append((name, *vals))
    return out


def sources_sha(sources):
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("raw_csv")
    ap.add_argument("workload")
    ap.add_argument("family")
    ap.add_argument("kernel_regex")
    ap.add_argument("alg_bytes", type=float, help="algorithmic bytes of one captured launch")
    ap.add_argument("sources", nargs="+")
    ap.add_argument("--command", required=True)
    a = ap.parse_args()
    ls = launches(a.raw_csv, a.kernel_regex)
    if not ls:
        raise SystemExit("no launch matches")
    caps = [{"kernel": n, "dram_read": r, "dram_write": w, "duration_us": t / 1e3,
             "dram_per_algorithmic_byte": (r + w) / a.alg_bytes} for n, r, w, t in ls]
    ratio = sum(c["dram_per_algorithmic_byte"] for c in caps) / len(caps)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    data[f"{a.workload}/{a.family}"] = {
        "dram_per_algorithmic_byte": ratio, "algorithmic_bytes_per_launch": a.alg_bytes, "captures": caps,
        "command": a.command, "sources": a.sources, "sha256": sources_sha(a.sources)}
    json.dump(data, open(OUT, "w"), indent=1)
    print(f"{a.workload}/{a.family}: {ratio:.4f} DRAM bytes per algorithmic byte over {len(caps)} launch(es)")


if __name__ == "__main__":
    main()
