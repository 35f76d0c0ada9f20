"""The 1024x1024 cylinder contact-angle sweep run to steady state (Sec. 3.2), on the GPU through the
library, in FP32 storage and in FP64 storage side by side.

Seven droplet-on-cylinder cases (cylinder radius 160, droplet radius 200, lambda from the paper's
correlation for theta = 30 ... 150 degrees; the same cases and seeds as the benchmark's headline
workload) step `steps` times in each storage mode.  Every `check` steps the study reads the
contact angles and the diagnostics of all cases.  The FP64 run equals the CPU oracle to about
1e-10 after 100 steps (the GPU parity tests), so at this size, where the oracle would need days, it
stands in for it.  Per case and storage mode the records give:
  * theta and its change over the last check interval;
  * the largest spurious current max |u| (Fig. 10), over all fluid nodes;
  * the relative mass drift of each component since the start;
and per case |theta_FP32 - theta_FP64|.

    python -m paper_2505_22256_gb300.study_sweep [--steps 50000] [--check 5000] [--storage f32,f64]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

from . import lbm, scenarios as S


def run(steps: int, check: int, storage: str, n: int = 1024, seed: int = 2, angles=(30, 50, 70, 90, 110, 130, 150),
        **overrides) -> list[dict]:
    """Step the sweep in one storage mode and return one record per case."""
    if check < 1 or steps < check:
        raise ValueError("need steps >= check >= 1")
    cases = S.lambda_sweep_cylinder(n=n, seed=seed, angles=angles)
    for sc in cases:
        for k, v in overrides.items():
            setattr(sc, k, v)
    lat = lbm.Lattice(cases, storage)
    try:
        d0 = lat.diagnostics_all()
        hist = []
        done = 0
        t0 = time.perf_counter()
        while done < steps:
            k = min(check, steps - done)
            lat.step(k)
            done += k
            hist.append((done, lat.contact_angle_all()[0]))
        lat.sync()
        wall = time.perf_counter() - t0
        d1 = lat.diagnostics_all(allow_unstable=True)
    finally:
        lat.close()
    out = []
    for k, sc in enumerate(cases):
        th = float(hist[-1][1][k])
        prev = float(hist[-2][1][k]) if len(hist) > 1 else float("nan")
        out.append({
            "case": sc.name, "storage": storage, "lambda": sc.lam, "steps": steps,
            "target_theta": angles[k], "theta": th if th == th else None,
            "dtheta_last": abs(th - prev) if th == th and prev == prev else None,
            "theta_history": [[s, float(t[k])] for s, t in hist],
            "umax": d1[k]["umax"],
            "mass_drift_A": (d1[k]["mass_A"] - d0[k]["mass_A"]) / d0[k]["mass_A"],
            "mass_drift_B": (d1[k]["mass_B"] - d0[k]["mass_B"]) / d0[k]["mass_B"],
            "unstable": bool(d1[k]["unstable"]), "wall_s_all_cases": wall,
        })
    return out


def table(rows: list[dict]) -> str:
    """Markdown table: one line per case, the storage modes side by side."""
    by = {}
    for r in rows:
        by.setdefault(r["case"], {})[r["storage"]] = r
    modes = sorted({r["storage"] for r in rows}, key=lambda m: ("f32", "f16", "bf16", "f64").index(m))
    f = lambda v, spec: "—" if v is None or v != v else format(v, spec)
    head = ["target θ", "λ"]
    for m in modes:
        head += [f"θ {m}", f"Δθ last interval {m}", f"max \\|u\\| {m}", f"mass drift A / B {m}"]
    if "f32" in modes and "f64" in modes:
        head.append("\\|θ f32 − θ f64\\|")
    lines = ["| " + " | ".join(head) + " |", "|" + "---|" * len(head)]
    for case, d in by.items():
        r0 = next(iter(d.values()))
        cells = [f"{r0['target_theta']:.0f}", f"{r0['lambda']:.4f}"]
        for m in modes:
            r = d.get(m)
            if r is None:
                cells += ["—"] * 4
                continue
            cells += [f(r["theta"], ".2f"), f(r["dtheta_last"], ".3f"), f"{r['umax']:.2e}",
                      f"{r['mass_drift_A']:.1e} / {r['mass_drift_B']:.1e}"]
        if "f32" in modes and "f64" in modes:
            a, b = d.get("f32", {}).get("theta"), d.get("f64", {}).get("theta")
            cells.append(f(abs(a - b) if a is not None and b is not None else None, ".3f"))
        lines.append("| " + " | ".join(cells) + " |")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=50000)
    ap.add_argument("--check", type=int, default=5000)
    ap.add_argument("--storage", default="f32,f64", help="comma-separated storage modes")
    ap.add_argument("--n", type=int, default=1024, help="lattice side (geometry scales with it)")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    rows = []
    for m in args.storage.split(","):
        rows += run(args.steps, args.check, m, n=args.n)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
