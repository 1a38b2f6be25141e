"""DRAM traffic and launch list of the solver's kernel families from one ncu capture.

The bench reports `roofline.traffic`, the DRAM bytes one launch of the
dominant kernel family moves, as the DRAM-bytes-per-algorithmic-byte ratio
that ncu measured for that family times the launch's algorithmic bytes.  This
script computes those ratios.  It reads two files made by the same command:

  * the raw page of an ncu capture of every kernel the command launches
    (`ncu --metrics gpu__time_duration.sum,dram__bytes_read.sum,dram__bytes_write.sum
    --csv --page raw --log-file RAW.csv python bench.py --profile-solves N ...`);
  * the JSON line the same command prints without ncu (the library profiler's
    launches and algorithmic bytes per kernel family for those N solves).

Every ncu launch is assigned to the profiler family its kernel belongs to
(template arguments name the precision, the matvec's scaled form and the
streaming pass's kind); for a family whose launch counts agree, the ratio
sum(DRAM bytes) / sum(algorithmic bytes) goes to profiles/traffic.json under
"<workload>/<family>", with the sha256 of the kernel sources it was measured
on: the bench withdraws the figure (reports null) once any of them changes.
With --launches-md it also writes the launch list (per kernel family:
launches, total device time, share) as a Markdown summary.

Usage:
  python -m paper_1711_10128_gb300.traffic RAW.csv PROFILE.json --command "the ncu command" \\
      [--plain "the command without ncu"] [--launches-md profiles/launches_<workload>_mixed.md]
"""
from __future__ import annotations

import argparse
import csv
import glob
import hashlib
import json
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
OUT = os.path.join(ROOT, "profiles", "traffic.json")
CSRC = os.path.join("paper_1711_10128_gb300", "csrc")
TS_KINDS = ["ts_project", "ts_inner", "ts_update_project", "ts_update_norm", "ts_update", "ts_rotate", "ts_resid",
            "ts_dot"]
SCALE = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0, "usecond": 1e3, "msecond": 1e6,
         "ns": 1.0, "us": 1e3, "ms": 1e6, "second": 1e9, "s": 1e9}


def _flag(s):
    return s.strip() in ("1", "true", "(bool)1")


def family_of(name):
    """The library profiler's family of a kernel (by its demangled name), or
    None for kernels outside the families (setup, conversions, reductions)."""
    suffix = lambda prec: "_f64" if prec == "double" else ""
    m = re.search(r"ts_kernel<(float|double),\s*(?:\(int\))?(\d+),", name)
    if m:
        return TS_KINDS[int(m.group(2))] + suffix(m.group(1))
    m = re.search(r"(?:sell_spmv_kernel|dia_spmv_kernel|\bspmv_kernel)<(float|double),\s*((?:\(bool\))?\w+)", name)
    if m:
        return ("spmv_scaled" if _flag(m.group(2)) else "spmv") + suffix(m.group(1))
    if "rotate_tc_kernel" in name:
        return "ts_rotate"
    if "rr_kernel" in name:
        return "rayleigh_ritz"
    return None


METRICS = ("gpu__time_duration.sum", "dram__bytes_read.sum", "dram__bytes_write.sum")


def read_launches(raw_csv):
    """(kernel name, family, duration ns, dram read bytes, dram write bytes)
    for every launch of an ncu CSV (the raw page: a row per launch; or the
    details page: a row per launch and metric); missing metrics are None."""
    rows = list(csv.reader(open(raw_csv)))
    start = next(i for i, r in enumerate(rows) if "Kernel Name" in r)
    hdr = rows[start]
    col = {h: i for i, h in enumerate(hdr)}
    if "Metric Name" in col:   # details page
        per = {}
        for r in rows[start + 1:]:
            if len(r) != len(hdr) or r[col["Metric Name"]] not in METRICS:
                continue
            key = r[col["ID"]]
            e = per.setdefault(key, {"name": r[col["Kernel Name"]]})
            v = r[col["Metric Value"]].replace(",", "")
            e[r[col["Metric Name"]]] = float(v) * SCALE.get(r[col["Metric Unit"]], 1.0) if v not in ("", "n/a") else None
        out = []
        for key in sorted(per, key=int):
            e = per[key]
            out.append((e["name"], family_of(e["name"]), *[e.get(m) for m in METRICS]))
        return out
    units = rows[start + 1]
    out = []
    for r in rows[start + 2:]:
        if len(r) != len(hdr):
            continue
        vals = []
        for m in METRICS:
            if m not in col or r[col[m]] in ("", "n/a"):
                vals.append(None)
                continue
            vals.append(float(r[col[m]].replace(",", "")) * SCALE.get(units[col[m]], 1.0))
        name = r[col["Kernel Name"]]
        out.append((name, family_of(name), *vals))
    return out


def sources():
    return sorted(os.path.relpath(p, ROOT) for p in glob.glob(os.path.join(ROOT, CSRC, "*"))
                  if p.endswith((".cu", ".cuh", ".h")))


def sources_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()


def launch_table(launches, commands, workload, solves):
    tot = sum(t for _, _, t, _, _ in launches if t) or 1.0
    by = {}
    for name, fam, t, _, _ in launches:
        short = re.sub(r"\(.*$", "", name).replace("void ", "").replace("trplk::", "")
        short = short.replace("(anonymous namespace)::", "").replace("<unnamed>::", "")
        e = by.setdefault(short, [fam or "-", 0, 0.0])
        e[1] += 1
        e[2] += t or 0.0
    lines = [f"# Launch list: {workload}, {solves} mixed solve(s)", "",
             "Every kernel launched by the command below, with its device time "
             "(`gpu__time_duration.sum`, one pass; launches serialised and cold-cache under the profiler, so "
             "compare shares, not absolute times).  Commands, from the repository root:", "", "```", *commands,
             "```", "",
             "| kernel | family | launches | total us | share |", "|---|---|---:|---:|---:|"]
    for short, (fam, n, t) in sorted(by.items(), key=lambda kv: -kv[1][2]):
        lines.append(f"| `{short}` | {fam} | {n} | {t / 1e3:.1f} | {t / tot:.4f} |")
    fams = {}
    for _, fam, t, _, _ in launches:
        fams[fam or "other"] = fams.get(fam or "other", 0.0) + (t or 0.0)
    lines += ["", "By family:", "", "| family | share |", "|---|---:|"]
    for fam, t in sorted(fams.items(), key=lambda kv: -kv[1]):
        lines.append(f"| {fam} | {t / tot:.4f} |")
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("raw_csv")
    ap.add_argument("profile_json")
    ap.add_argument("--command", required=True, help="the ncu capture command")
    ap.add_argument("--plain", help="the same command without ncu, whose output is PROFILE.json")
    ap.add_argument("--launches-md")
    a = ap.parse_args()
    launches = read_launches(a.raw_csv)
    prof = json.loads(open(a.profile_json).read().strip().splitlines()[-1])
    workload = prof["workload"]
    files = sources()
    sha = sources_sha(files)
    data = json.load(open(OUT)) if os.path.exists(OUT) else {}
    for fam, ent in prof["families"].items():
        if ent["algorithmic_bytes"] <= 0:
            continue
        mine = [l for l in launches if l[1] == fam]
        if not mine or any(l[3] is None or l[4] is None for l in mine):
            continue
        if len(mine) != ent["launches"]:
            print(f"{fam}: {len(mine)} ncu launches against {ent['launches']} profiled; not recorded")
            continue
        dram = sum(l[3] + l[4] for l in mine)
        ratio = dram / ent["algorithmic_bytes"]
        data[f"{workload}/{fam}"] = {
            "dram_per_algorithmic_byte": ratio, "launches": len(mine), "dram_bytes": dram,
            "algorithmic_bytes": ent["algorithmic_bytes"], "solves": prof["solves"], "command": a.command,
            "sources": files, "sha256": sha}
        print(f"{workload}/{fam}: {ratio:.4f} DRAM bytes per algorithmic byte over {len(mine)} launches")
    json.dump(data, open(OUT, "w"), indent=1)
    if a.launches_md:
        cmds = ([f"{a.plain} > {a.profile_json}"] if a.plain else []) + [
            a.command,
            f"python -m paper_1711_10128_gb300.traffic {a.raw_csv} {a.profile_json} --command '<the ncu line>' "
            f"--launches-md {a.launches_md}"]
        open(a.launches_md, "w").write(launch_table(launches, cmds, workload, prof["solves"]))
        print("wrote", a.launches_md)


if __name__ == "__main__":
    main()
