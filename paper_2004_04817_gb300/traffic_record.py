"""Write profiles/traffic_<kernel>.json from an ncu report: the DRAM bytes
of one launch (dram__bytes_read.sum + dram__bytes_write.sum) and a hash of
the kernel's sources, so bench.py reports the figure only while the kernel
is unchanged.

  python -m paper_2004_04817_gb300.traffic_record <report.ncu-rep> <kernel> <launch> <src>...
"""
import csv
import hashlib
import io
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def main():
    rep, kernel, launch = sys.argv[1], sys.argv[2], int(sys.argv[3])
    srcs = sys.argv[4:]
    out = subprocess.run(["ncu", "-i", rep, "--page", "raw", "--csv"], capture_output=True,
                         text=True, check=True).stdout
    rows = list(csv.reader(io.StringIO(out)))
    hdr, units, data = rows[0], rows[1], rows[2:]
    d = dict(zip(hdr, data[launch]))
    scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}
    tot = 0.0
    for m in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
        tot += float(d[m]) * scale[units[hdr.index(m)]]
    h = hashlib.sha1()
    for src in srcs:
        with open(os.path.join(ROOT, src), "rb") as f:
            h.update(f.read())
    rec = {"kernel": kernel, "report": os.path.basename(rep), "launch": launch,
           "dram_bytes_per_launch": tot, "sources": srcs, "sources_sha1": h.hexdigest(),
           "duration": d.get("gpu__time_duration.sum")}
    with open(os.path.join(ROOT, "profiles", f"traffic_{kernel}.json"), "w") as f:
        json.dump(rec, f, indent=1)
    print(rec)


if __name__ == "__main__":
    main()
