"""Original against improved solid-fluid scheme (Sec. 3.2; Figs. 6, 10 and 11), on the GPU through
the library.

Both schemes step the paper's 300x350 droplet-on-cylinder case for each target angle (lambda
from the correlation of Fig. 7; the original scheme uses G_w1 = lambda G_w2 everywhere).  Every
`check` steps the study reads the fields, the contact angles and the diagnostics of all cases.
For each case the table then gives:
  * theta, and its change over the last check interval;
  * the largest change of |u| at any node over that interval (the convergence measure of
    Sec. 3.1);
  * the largest spurious current max |u| (Fig. 10), over all fluid nodes and over those more
    than three nodes from the solid (the free interface alone);
  * the smallest and largest component density (Fig. 11);
  * the wall layer: the median rho_A over first-layer fluid nodes where B dominates.  Where B wets
    the wall that layer holds A at about its dissolved density; a film of A along the wall (the
    mass-transfer layer of Fig. 6) raises it;
  * whether the droplet still touches the cylinder (any first-layer node where A dominates).

    python -m paper_2505_22256_gb300.study_schemes [--steps 60000] [--check 10000] [--storage f32]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import lbm, scenarios as S

# D2Q9 neighbour offsets (ex, ey)
_NEIGHBOURS = ((1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1))


def first_layer(solid: np.ndarray) -> np.ndarray:
    """Fluid nodes with at least one solid D2Q9 neighbour, on a lattice periodic in x and y."""
    s = solid.astype(bool)
    touch = np.zeros_like(s)
    for ex, ey in _NEIGHBOURS:
        touch |= np.roll(s, shift=(-ey, -ex), axis=(0, 1))  # s[y + ey, x + ex] at (y, x)
    return ~s & touch


def near_solid(solid: np.ndarray, margin: int = 3) -> np.ndarray:
    """Nodes within `margin` nodes of a solid node in both x and y (periodic), solid included."""
    s = solid.astype(bool)
    out = np.zeros_like(s)
    for dy in range(-margin, margin + 1):
        for dx in range(-margin, margin + 1):
            out |= np.roll(s, shift=(dy, dx), axis=(0, 1))
    return out


def wall_layer(solid: np.ndarray, rA: np.ndarray, rB: np.ndarray) -> tuple[float, float]:
    """(median rho_A over the first-layer nodes where rho_B > rho_A, share of first-layer nodes
    where rho_A >= rho_B).  The median is NaN when A covers the whole layer."""
    m = first_layer(solid)
    a, b = rA[m], rB[m]
    bdom = b > a
    med = float(np.median(a[bdom])) if bdom.any() else float("nan")
    return med, float(np.mean(~bdom))


def run(cases: list, steps: int, check: int, storage: str = "f32") -> list[dict]:
    """Step every case `steps` times and return one record per case (see the module text)."""
    if check < 1 or steps < check:
        raise ValueError("need steps >= check >= 1")
    lat = lbm.Lattice(cases, storage)
    try:
        prev_u, prev_th = None, None
        done = 0
        while done < steps:
            n = min(check, steps - done)
            lat.step(n)
            done += n
            fields = lat.fields_all()
            th = lat.contact_angle_all()[0]
            diag = lat.diagnostics_all(allow_unstable=True)
            u = [np.hypot(f[2], f[3]) for f in fields]
            du = [float("nan")] * len(cases) if prev_u is None else \
                [float(np.max(np.abs(a - b))) for a, b in zip(u, prev_u)]
            dth = [float("nan")] * len(cases) if prev_th is None else list(np.abs(th - prev_th))
            prev_u, prev_th = u, th
    finally:
        lat.close()
    out = []
    for k, sc in enumerate(cases):
        rA, rB = fields[k][0], fields[k][1]
        layer, a_share = wall_layer(sc.solid, rA, rB)
        far = ~near_solid(sc.solid)
        d = diag[k]
        out.append({
            "case": sc.name, "scheme": sc.scheme, "target_theta": sc.extra.get("target_theta"),
            "lambda": sc.lam, "steps": steps, "theta": None if th[k] != th[k] else float(th[k]),
            "dtheta_last": dth[k], "du_last": du[k], "umax": d["umax"],
            "umax_off_wall": float(np.max(np.hypot(fields[k][2], fields[k][3])[far])),
            "rho_min": min(d["rhoA_min"], d["rhoB_min"]), "rho_max": max(d["rhoA_max"], d["rhoB_max"]),
            "wall_layer_rhoA": layer, "attached": a_share > 0.0, "unstable": bool(d["unstable"]),
        })
    return out


def table(rows: list[dict]) -> str:
    """Markdown table of the records."""
    head = ("| scheme | target θ | λ | θ | Δθ (last interval) | max Δ\\|u\\| (last interval) | max \\|u\\| "
            "| max \\|u\\| off the wall | ρ min | ρ max | wall layer ρ_A | attached |\n"
            "|---|---|---|---|---|---|---|---|---|---|---|---|")
    lines = [head]
    f = lambda v, spec: "—" if v is None or v != v else format(v, spec)
    for r in rows:
        lines.append(f"| {r['scheme']} | {f(r['target_theta'], '.0f')} | {r['lambda']:.4f} | {f(r['theta'], '.1f')} "
                     f"| {f(r['dtheta_last'], '.2f')} | {f(r['du_last'], '.1e')} | {r['umax']:.2e} "
                     f"| {r['umax_off_wall']:.2e} "
                     f"| {r['rho_min']:.4f} | {r['rho_max']:.4f} | {f(r['wall_layer_rhoA'], '.4f')} "
                     f"| {'yes' if r['attached'] else 'no'}{' (unstable)' if r['unstable'] else ''} |")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=60000)
    ap.add_argument("--check", type=int, default=10000)
    ap.add_argument("--storage", default="f32", choices=["f32", "f64", "f16", "bf16"])
    ap.add_argument("--angles", default="30,50,70,90,110,130,150")
    ap.add_argument("--paper-params", action="store_true",
                    help="densities 1.02 / 0.05, nu = 0.17 and G_w2 = G_12 as stated in Sec. 3.2")
    ap.add_argument("--gw2", type=float, default=-1.0, help="override G_w2 (>= 0)")
    ap.add_argument("--gw2-is-g", action="store_true", help="G_w2 = G_12 (the paper's choice)")
    ap.add_argument("--G", type=float, default=None, help="override G_12")
    ap.add_argument("--second-layer", default="psi_and_solid", choices=["psi_and_solid", "psi"],
                    help="what a non-fluid second-layer stencil site takes from x + sign(e) (Table 1)")
    ap.add_argument("--adhesion-stencil", default="e8", choices=["e8", "d2q9"],
                    help="stencil of the adhesion sum of Eq. 9 (d2q9: as printed, first layer)")
    ap.add_argument("--json", default=None, help="also write the records to this file")
    args = ap.parse_args(argv)
    angles = tuple(int(a) for a in args.angles.split(","))
    cases = S.scheme_study(angles, paper_params=args.paper_params, Gw2=None if args.gw2_is_g else args.gw2,
                           second_layer=args.second_layer, adhesion_stencil=args.adhesion_stencil)
    if args.G is not None:
        for sc in cases:
            sc.G = args.G
    rows = run(cases, args.steps, args.check, args.storage)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
