"""Measure cuFFT plane-transform times for the planner's candidate grid sizes and write them
to csrc/fft_table.inc (run on the target GPU; the library must be built).

Candidates: n = 32 m for 4 <= m <= 512 with m 11-smooth (FFT-friendly multiples of the uv
tile).  For each n the batched 2-D C2C (FP32) and Z2Z (FP64) cuFFT transforms, the library's
double-float FFT (FP64 planes) and the library's FP32 FFT (sizes an implementation does not
support get 0) are timed through the library's wg_fft_time entry point with ~1-2 GiB of planes
per batch.  --columns re-measures only some of the four columns (c2c, z2z, df64, f32), and
--min-n / --max-n only the sizes in that range, keeping the other entries of the existing table.  The planner uses the
table to pick, for each oversampling factor, the fastest size >= sigma * n and to price the
FFT stage in its cost model (Sec. 4.1).

usage: python -m paper_2010_10122_gb300.calibrate_fft [--max-n 16384] [--out PATH]
"""
import argparse
import os
import sys
import time


def smooth(m, primes=(2, 3, 5, 7, 11)):
    for p in primes:
        while m % p == 0:
            m //= p
    return m == 1


COLUMNS = ("c2c", "z2z", "df64", "f32")
# (precision, bytes per complex value, impl of wg_fft_time) per column
KINDS = (("f32", 8, 1), ("f64", 16, 1), ("f64", 16, 2), ("f32", 8, 4))


def read_table(path):
    """{n: [c2c, z2z, df64, f32]} from a table file (missing columns read as 0)."""
    old = {}
    if os.path.exists(path):
        for ln in open(path):
            ln = ln.strip()
            if ln.startswith("{"):
                v = [float(x) for x in ln.strip("{},").split(",")]
                old[int(v[0])] = (v[1:] + [0.0] * 4)[:4]
    return old


def table_plan(old, cols, min_n, max_n):
    """Rows of the new table in size order: (n, [column -> measure?]).  Sizes are n = 32 m, m
    11-smooth, up to max_n, plus every size the old table has beyond it; a column is re-measured
    only when it is selected and n lies in [min_n, max_n] (or the old table lacks n)."""
    top = max([max_n] + list(old))
    out = []
    for m in range(4, top // 32 + 1):
        if not smooth(m):
            continue
        n = 32 * m
        if n > max_n and n not in old:
            continue
        measure = [not ((name not in cols or n < min_n or n > max_n) and n in old)
                   for name in COLUMNS]
        out.append((n, measure))
    return out


def format_table(rows, device_name):
    lines = [f"// cuFFT batched 2-D plane transform times on {device_name}, measured by\n",
             "// paper_2010_10122_gb300/calibrate_fft.py: {n, ms per plane C2C, ms per plane Z2Z, "
             "ms per plane double-float, ms per plane library FP32}\n"]
    for n, a, b, c, d in rows:
        lines.append(f"{{{n}, {a:.6g}, {b:.6g}, {c:.6g}, {d:.6g}}},\n")
    return "".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--max-n", type=int, default=16384)
    ap.add_argument("--min-n", type=int, default=0)
    ap.add_argument("--columns", default=",".join(COLUMNS))
    ap.add_argument("--out", default=os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                                  "csrc", "fft_table.inc"))
    args = ap.parse_args()
    cols = args.columns.split(",")
    old = read_table(args.out)
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from paper_2010_10122_gb300 import _build
    _build.build()
    import paper_2010_10122_gb300 as wg
    import torch
    rows = []
    t0 = time.time()
    for n, measure in table_plan(old, cols, args.min_n, args.max_n):
        out = [n]
        for c, (prec, b, impl) in enumerate(KINDS):
            if not measure[c]:
                out.append(old[n][c])
                continue
            batch = max(1, min(64, int((1.5 * 2**30) // (n * n * b))))
            reps = 3 if n * n * b * batch > 2**28 else 6
            try:
                out.append(wg.fft_time(n, prec, batch=batch, reps=reps, impl=impl))
            except wg.WgridError:   # a size this implementation does not support
                out.append(0.0)
        rows.append(out)
        print(f"n={n:6d} c2c {out[1]*1e3:9.2f} us/plane  z2z {out[2]*1e3:10.2f} us/plane  "
              f"df64 {out[3]*1e3:10.2f} us/plane  f32 {out[4]*1e3:10.2f} us/plane", flush=True)
    with open(args.out, "w") as f:
        f.write(format_table(rows, torch.cuda.get_device_name(0)))
    print(f"wrote {len(rows)} sizes to {args.out} in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
