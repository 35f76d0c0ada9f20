"""Static contact angles on a sphere in 3-D (Sec. 3.5; Fig. 16), on the GPU through the library.

The case is the paper's 200x200x280 periodic box: a solid sphere of radius 50 at (100, 100, 100)
and a droplet of A of radius 45 at (100, 100, 180).  The paper's three strength coefficients are
lambda = 0.38, 1 and 2.1, for which it reports theta of about 45, 90 and 146 deg.  Each case steps
in intervals, and after each interval the study fits the contact angle.  The table gives the final
angle, its change over the last interval, max |u| and the density extrema.  --adhesion-stencil d3q19
takes the adhesion sum of Eq. 9 as printed (first layer, D3Q19 weights) and --gw2-is-g sets
G_w2 = G_AB, the paper's choice.

    python -m paper_2505_22256_gb300.study_sphere3d [--steps 30000] [--interval 5000] [--n 200]
        [--adhesion-stencil e8|d3q19] [--gw2-is-g]
"""
from __future__ import annotations

import argparse
import json
import sys

from . import lbm3d, scenarios as S

PAPER_THETA = {0.38: 45.0, 1.0: 90.0, 2.1: 146.0}


def case(lam: float, n: int = 200, second_layer: str = "psi_and_solid", adhesion_stencil: str = "e8",
         gw2_is_g: bool = False):
    sc = S.sphere_droplet_3d(lam=lam) if n == 200 else S.sphere_droplet_3d_small(n, lam=lam)
    sc.second_layer = second_layer
    sc.adhesion_stencil = adhesion_stencil
    if gw2_is_g:
        sc.Gw2 = sc.G
    return sc


def run(lams=(0.38, 1.0, 2.1), steps: int = 30000, interval: int = 5000, storage: str = "f32",
        n: int = 200, second_layer: str = "psi_and_solid", adhesion_stencil: str = "e8",
        gw2_is_g: bool = False) -> list[dict]:
    """One record per lambda."""
    if interval < 1 or steps < interval:
        raise ValueError("need steps >= interval >= 1")
    out = []
    for lam in lams:
        sc = case(lam, n, second_layer, adhesion_stencil, gw2_is_g)
        lat = lbm3d.Lattice3(sc.solid, sc.rhoA0, sc.rhoB0, sc.params(), storage)
        try:
            angles = []
            done = 0
            while done < steps:
                k = min(interval, steps - done)
                lat.step(k)
                done += k
                angles.append(lat.contact_angle(sc.sphere)[0])
            d = lat.diagnostics(allow_unstable=True)
        finally:
            lat.close()
        out.append({
            "lambda": lam, "adhesion_stencil": adhesion_stencil, "G_w2": sc.Gw2, "paper_theta": PAPER_THETA.get(lam), "n": n, "steps": steps, "theta": angles[-1],
            "dtheta_last": abs(angles[-1] - angles[-2]) if len(angles) > 1 else float("nan"), "history": angles,
            "umax": d["umax"], "rhoA_min": d["rhoA_min"], "rhoA_max": d["rhoA_max"],
            "rhoB_min": d["rhoB_min"], "rhoB_max": d["rhoB_max"], "unstable": bool(d["unstable"]),
        })
    return out


def table(rows: list[dict]) -> str:
    f = lambda v, spec: "—" if v is None or v != v else format(v, spec)
    lines = ["| λ | θ (paper) | θ | Δθ (last interval) | max \\|u\\| | ρ_A min / max | ρ_B min / max |",
             "|---|---|---|---|---|---|---|"]
    for r in rows:
        lines.append(f"| {r['lambda']:g} | {f(r['paper_theta'], '.0f')} | {f(r['theta'], '.1f')} "
                     f"| {f(r['dtheta_last'], '.2f')} | {r['umax']:.2e} | {r['rhoA_min']:.4f} / {r['rhoA_max']:.4f} "
                     f"| {r['rhoB_min']:.4f} / {r['rhoB_max']:.4f}{' (unstable)' if r['unstable'] else ''} |")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--steps", type=int, default=30000)
    ap.add_argument("--interval", type=int, default=5000)
    ap.add_argument("--n", type=int, default=200, help="200: the paper's box; else the geometry scaled to n")
    ap.add_argument("--storage", default="f32", choices=["f32", "f64"])
    ap.add_argument("--lambdas", default="0.38,1,2.1")
    ap.add_argument("--second-layer", default="psi_and_solid", choices=["psi_and_solid", "psi"])
    ap.add_argument("--adhesion-stencil", default="e8", choices=["e8", "d3q19"])
    ap.add_argument("--gw2-is-g", action="store_true", help="G_w2 = G_AB (the paper's choice)")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    rows = run(tuple(float(v) for v in args.lambdas.split(",")), args.steps, args.interval, args.storage, args.n,
               args.second_layer, args.adhesion_stencil, args.gw2_is_g)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
