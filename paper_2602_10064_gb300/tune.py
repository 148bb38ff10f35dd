"""Autotuner for the FFT pass kernels of the slice path.

Every FFT pass kernel (spreading row pass, potential and band-limit column passes, the row
passes that form t, the multislice row and column passes) comes in variants: radix-16 or
radix-8 plans (512 and 1024 points), 16 or 32 elements per thread (three- or two-pass
transforms), two or three resident CTAs per SM, and for the column passes twice the columns
per CTA.  No single choice is best for all of them: on GB300 the
radix-8 plans speed up the 1024-point row passes, and three CTAs per SM speed up the
spreading pass but slow down the multislice row pass.

This script builds the library once per variant (TACAW_TUNE_FORCE), times every kernel class
at every transform length on representative runs with the library's own CUDA-event profiler,
and writes csrc/tuning_table.h with the fastest variant per (kernel, length).  A variant
replaces the default only when it is at least 2% faster.  Results of different variants agree
to FP32 rounding (the radix schedule changes the rounding order); the parity tests hold for
every variant.

    python -m paper_2602_10064_gb300.tune [--out PATH] [--variants 0 1 ... 14]

Needs a GPU.  Synthetic inputs come from the repository's `workloads` module.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)

# kernel class (library profiler name) -> KernelId in k_slices.cu
KERNEL_IDS = {"splat_row": 0, "col_pot": 1, "row_pot_t": 2, "row_vt": 3, "col_t": 4, "row_tout": 5,
              "slice_row": 8, "slice_col": 9}
# classes whose kernels take the column-width bit (variant & 4); the others ignore it
COLUMN_CLASSES = {"col_pot", "col_t", "slice_col"}
N_KERNELS = 10
LENGTHS = (32, 64, 128, 256, 512, 1024, 96, 192, 384, 768, 1152)
MIN_GAIN = 0.02


def cases():
    """(name, transform length, workload factory): runs whose kernel mix matches the hot path
    at each length (plane waves, and a probe scan for the full-t row pass)."""
    sys.path.insert(0, ROOT)
    import workloads
    return [
        ("diamond-128", 128, lambda: workloads.diamond_si(n_frames=512, grid=128, n_slices=8, seed=11)),
        ("diamond-256", 256, lambda: workloads.diamond_si(n_frames=256, grid=256, n_slices=20, seed=12,
                                                           reps=(4, 4, 2))),
        ("scan-256", 256, lambda: workloads.config3(n_frames=16, seed=13)),
        ("rocksalt-512", 512, lambda: workloads.config2(n_frames=128, seed=14)),
        ("diamond-1024", 1024, lambda: workloads.config4(n_frames=64, seed=15)),
        ("diamond-768", 768, lambda: workloads.diamond_si(n_frames=64, grid=768, n_slices=20, seed=16,
                                                           reps=(8, 8, 2))),
        ("minimal-example-1152", 1152, lambda: workloads.minimal_example_si(n_frames=16, seed=17)),
    ]


def measure(steps: int = 3) -> dict:
    """Per (kernel class, length): milliseconds per run, summed over the cases of that length."""
    import torch

    import paper_2602_10064_gb300 as T
    out = {}
    ctx = T.Context(0)
    st = torch.cuda.current_stream()
    for name, n, make in cases():
        w = make()
        ctx.load_form_factors(w.form_Z, w.form_coef)
        params, probe = T.params_of(w), T.probe_of(w)
        pos = torch.from_numpy(w.pos).cuda()
        Z = torch.from_numpy(w.Z).cuda()
        S = torch.empty((w.n_probes, w.n_frames, w.ny, w.nx), dtype=torch.float32, device="cuda")

        def run():
            T.tacaw_run(ctx.h, params, pos, Z, w.n_atoms, w.n_frames, probe, T.DFT_BF16X3, T.REDUCE_NONE, S, st)

        def transmission(V):
            ctx.transmission(params, V)

        run()
        V = ctx.build_potential(params, pos[: min(8, w.n_frames)], Z)
        transmission(V)
        torch.cuda.synchronize()
        best = {}
        for fn in (run, lambda: transmission(V)):
            for _ in range(steps):
                T.tacaw_profile_begin(ctx.h)
                fn()
                torch.cuda.synchronize()
                prof = T.tacaw_profile_end(ctx.h)
                cur = {}
                for cls, (ms, _n, _b, _f) in prof.items():
                    if cls in KERNEL_IDS:
                        cur[cls] = cur.get(cls, 0.0) + ms
                for cls, ms in cur.items():
                    key = f"{cls}@{n}"
                    best[key] = min(best.get(key, float("inf")), ms)
        for key, ms in best.items():
            out[key] = out.get(key, 0.0) + ms
        del pos, Z, S, V
    ctx.check()
    ctx.close()
    return out


def choose(results: dict) -> list:
    """table[kernel][length index]: the fastest variant, kept at 0 unless MIN_GAIN faster."""
    table = [[0] * len(LENGTHS) for _ in range(N_KERNELS)]
    keys = set().union(*(r.keys() for r in results.values()))
    for key in sorted(keys):
        cls, n = key.split("@")
        if 0 not in results or key not in results[0]:
            continue
        base = results[0][key]
        v_best, t_best = 0, base
        for v, r in results.items():
            if (v & 4) and cls not in COLUMN_CLASSES:
                continue
            if key in r and r[key] < t_best:
                v_best, t_best = v, r[key]
        if v_best != 0 and t_best > (1.0 - MIN_GAIN) * base:
            v_best = 0
        table[KERNEL_IDS[cls]][LENGTHS.index(int(n))] = v_best
    return table


def header(table: list, results: dict) -> str:
    names = {v: k for k, v in KERNEL_IDS.items()}
    rows = []
    for k in range(N_KERNELS):
        rows.append("    {" + ", ".join(str(x) for x in table[k]) + "},  // " + names.get(k, "probe (not tuned)"))
    lines = [
        "// Variant of each FFT pass kernel per transform length (see Tuned in k_slices.cu).",
        "// Written by paper_2602_10064_gb300/tune.py from CUDA-event timings of every variant on GB300",
        "// (variant & 1: radix-8 plans; & 2: more resident threads; & 4: wide column CTAs; & 8: 32 elements",
        "// per thread); ms per variant:",
    ]
    for key in sorted(set().union(*(r.keys() for r in results.values()))):
        lines.append("//   " + key + ": " + ", ".join(f"v{v} {r[key]:.2f}" for v, r in sorted(results.items())
                                                  if key in r))
    lines += ["#pragma once", "", "namespace tacaw {", "",
              "// transform lengths of the columns of kTunedVariant",
              "constexpr int kTunedLengths[11] = {" + ", ".join(str(n) for n in LENGTHS) + "};",
              "",
              "// [kernel][index of N in kTunedLengths]",
              "constexpr int kTunedVariant[10][11] = {"] + rows + ["};", "",
              "constexpr int tuned_variant(int kernel, int n) {",
              "  for (int l = 0; l < 11; ++l)",
              "    if (kTunedLengths[l] == n) return (kernel >= 0 && kernel < 10) ? kTunedVariant[kernel][l] : 0;",
              "  return 0;",
              "}", "", "}  // namespace tacaw", ""]
    return "\n".join(lines)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=os.path.join(PKG, "csrc", "tuning_table.h"))
    # bit 1 (radix-8 plans) has no effect together with bit 8 (32 elements per thread)
    ap.add_argument("--variants", type=int, nargs="*", default=[v for v in range(16) if not (v & 8 and v & 1)])
    ap.add_argument("--measure", type=int, default=None, help=argparse.SUPPRESS)
    args = ap.parse_args()
    if args.measure is not None:
        sys.path.insert(0, ROOT)
        from paper_2602_10064_gb300 import _build
        _build.build()
        print(json.dumps(measure()))
        return
    results = {}
    for v in args.variants:
        env = dict(os.environ, TACAW_NVCC_DEFINES=f"-DTACAW_TUNE_FORCE={v}")
        r = subprocess.run([sys.executable, "-m", "paper_2602_10064_gb300.tune", "--measure", str(v)], cwd=ROOT,
                           env=env, capture_output=True, text=True)
        if r.returncode != 0:
            raise SystemExit(f"variant {v} failed:\n{r.stdout[-2000:]}\n{r.stderr[-4000:]}")
        results[v] = json.loads(r.stdout.strip().splitlines()[-1])
        print(f"variant {v}: " + ", ".join(f"{k} {ms:.2f}" for k, ms in sorted(results[v].items())), flush=True)
    table = choose(results)
    with open(args.out, "w") as fh:
        fh.write(header(table, results))
    print(f"wrote {args.out}")


if __name__ == "__main__":
    main()
