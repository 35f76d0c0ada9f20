"""Immiscible displacement in a porous medium (the shape of Sec. 3.4), on the GPU through the library.

The 4096x2048 porous medium of disks (porosity 0.6) starts filled with component B; a velocity inlet
at x = 0 injects A (rho_in = 1.0 for A, 0.03 for B, u_in = 0.005) and an outflow boundary closes
x = nx - 1.  Every `check` steps the study reads the diagnostics and the fields and records:
  * the mass of each component, and the change of A's mass per step since the start next to the
    source the inlet rule adds, rho_in,A u_in H per step (H = fluid rows of the inlet column).  The
    rule adds exactly that per step once the flow through the inlet column is steady; the mass
    balance also holds what leaves or enters through the outflow column, whose copied populations
    leave the pressure level free (dissolved A leaves with B, and B enters when the medium's
    resistance raises the pressure);
  * the A saturation (share of fluid nodes where rho_A > rho_B) and the front: the largest x at
    which any fluid node is A-dominated, and the first time that front reaches the outlet column
    (breakthrough), with the saturation then.

    python -m paper_2505_22256_gb300.study_displacement [--steps 200000] [--check 20000]
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np

from . import lbm, scenarios as S


def case(nx: int = 4096, ny: int = 2048, seed: int = 4):
    """The benchmark's porous workload (keep-out band scaled with the width)."""
    keep = max(8, 64 * nx // 4096)
    return S.porous_disks(nx=nx, ny=ny, keep_out=(keep, keep), seed=seed)


def snapshot(sc, rA: np.ndarray, rB: np.ndarray) -> dict:
    """Saturation and front of one state (fields of the case, [ny][nx])."""
    fluid = sc.solid == 0
    a_dom = fluid & (rA > rB)
    cols = np.nonzero(a_dom.any(axis=0))[0]
    return {"saturation_A": float(a_dom.sum() / fluid.sum()), "front_x": int(cols.max()) if len(cols) else -1}


def run(sc, steps: int, check: int, storage: str = "f32") -> list[dict]:
    """Step the case and return one record per check."""
    if check < 1 or steps < check:
        raise ValueError("need steps >= check >= 1")
    inlet_rows = int((sc.solid[:, 0] == 0).sum())
    inflow = sc.rho_in[0] * sc.u_in * inlet_rows  # prescribed mass of A per step
    lat = lbm.Lattice(sc, storage)
    rows = []
    try:
        d0 = lat.diagnostics()
        done, t0 = 0, time.perf_counter()
        breakthrough = None
        while done < steps:
            k = min(check, steps - done)
            lat.step(k)
            done += k
            d = lat.diagnostics(allow_unstable=True)
            rA, rB, _, _ = lat.fields()
            snap = snapshot(sc, rA, rB)
            if breakthrough is None and snap["front_x"] == sc.nx - 1:
                breakthrough = {"step": done, "saturation_A": snap["saturation_A"]}
            rows.append({"case": sc.name, "storage": storage, "step": done, "mass_A": d["mass_A"], "mass_B": d["mass_B"],
                         "dmass_A_per_step": (d["mass_A"] - d0["mass_A"]) / done, "inflow_A_per_step": inflow,
                         "dmass_B_per_step": (d["mass_B"] - d0["mass_B"]) / done, "umax": d["umax"],
                         **snap, "breakthrough": breakthrough, "unstable": bool(d["unstable"]),
                         "wall_s": time.perf_counter() - t0})
    finally:
        lat.close()
    return rows


def table(rows: list[dict]) -> str:
    lines = ["| step | mass A | mass B | ΔM_A per step (measured) | ρ_in u_in H (inlet) | ratio | ΔM_B per step "
             "| A saturation | front x | max \\|u\\| |", "|---|---|---|---|---|---|---|---|---|---|"]
    for r in rows:
        lines.append(f"| {r['step']:,} | {r['mass_A']:.6e} | {r['mass_B']:.6e} | {r['dmass_A_per_step']:.5f} "
                     f"| {r['inflow_A_per_step']:.5f} | {r['dmass_A_per_step'] / r['inflow_A_per_step']:.4f} "
                     f"| {r['dmass_B_per_step']:.5f} | {r['saturation_A']:.4f} | {r['front_x']} "
                     f"| {r['umax']:.2e}{' (unstable)' if r['unstable'] else ''} |")
    bt = rows[-1]["breakthrough"] if rows else None
    lines.append("")
    lines.append("breakthrough: " + ("not reached" if bt is None else
                                     f"step {bt['step']:,}, A saturation {bt['saturation_A']:.4f}"))
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=200000)
    ap.add_argument("--check", type=int, default=20000)
    ap.add_argument("--size", default="4096x2048")
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--u-in", type=float, default=None, help="inlet velocity (default 0.005)")
    ap.add_argument("--outlet", default="copy", choices=["copy", "pressure"],
                    help="outflow rule: copy from column nx-2, or the Zou-He density condition holding "
                         "the initial densities of the B-filled medium (0.03, 1.0)")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    nx, ny = map(int, args.size.split("x"))
    sc = case(nx, ny)
    if args.u_in is not None:
        sc.u_in = args.u_in
    sc.outlet = args.outlet
    rows = run(sc, args.steps, args.check, args.storage)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
