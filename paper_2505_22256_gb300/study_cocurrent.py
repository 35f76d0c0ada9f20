"""Two-layer co-current flow (Sec. 3.1; Figs. 3 and 4), on the GPU through the library.

Fluid A fills the central half of a 50x100 channel and fluid B the two outer quarters, with the
same viscosity (nu = 0.17) and densities.  Poiseuille flow is driven by the body acceleration
g = 1e-6 on both components between walls at rest.  Couette flow is driven by the walls sliding at
-/+0.005.  Every target angle (lambda from the correlation of Fig. 7) runs under both flows.  The
study steps all cases until u_x changes by less than 1e-5 at every node over 10,000 steps (the
criterion of Sec. 3.1).  It then reports the relative L2 error of the x-averaged profile u_x(y)
against two profiles:
  * analytic: both fluids have the same viscosity and main density, so Eq. 13 reduces to the
    parabola u = g s (H - s) / (2 nu), and the Couette profile is the straight line from -U to U.
    Here s = y + 1/2 and H = ny: the walls lie half a cell outside the first and last rows;
  * balance: the steady momentum balance d/dy(rho nu du/dy) + rho g = 0 with the simulated total
    density rho(y), solved by central differences with the wall velocity mirrored about the wall.
    It isolates the diffuse interface, where the mixture density dips, from the lattice numerics.

    python -m paper_2505_22256_gb300.study_cocurrent [--max-steps 400000] [--storage f32]
"""
from __future__ import annotations

import argparse
import json
import sys

import numpy as np

from . import lbm, scenarios as S

INTERVAL = 10000   # steps between the profiles the convergence test compares
TOL = 1e-5         # largest change of u_x over INTERVAL steps at convergence


def cases(angles=(45, 90, 135), paper_params: bool = False, gw2: float | None = -1.0,
          second_layer: str = "psi_and_solid", adhesion_stencil: str = "e8") -> list:
    """Poiseuille then Couette channels, one per target angle.  gw2 >= 0 (or None: G_w2 = G)
    overrides G_w2; second_layer picks the Table 1 reading, adhesion_stencil that of Eq. 9."""
    extra = {k: S.PAPER_SEC32[k] for k in ("rho_m", "rho_d", "G", "Gw2")} if paper_params else {}
    if gw2 is None or gw2 >= 0:
        extra["Gw2"] = gw2
    out = []
    for flow, make in (("poiseuille", S.poiseuille_channel), ("couette", S.couette_channel)):
        for k, th in enumerate(angles):
            sc = make(lam=S.lambda_for_angle(th), seed=40 + 10 * k + (flow == "couette"), **extra)
            sc.name = f"{flow}_theta{th}_{sc.name}"
            sc.second_layer = second_layer
            sc.adhesion_stencil = adhesion_stencil
            sc.extra.update(flow=flow, target_theta=float(th))
            out.append(sc)
    return out


def analytic_profile(sc) -> np.ndarray:
    """u_x(y) of one fluid of the same viscosity filling the channel."""
    nu = (sc.tau[0] - 0.5) / 3.0
    s = np.arange(sc.ny) + 0.5
    if sc.extra["flow"] == "poiseuille":
        return sc.g[0] * s * (sc.ny - s) / (2.0 * nu)
    lo, hi = sc.u_wall
    return lo + (hi - lo) * s / sc.ny


def balance_profile(sc, rho: np.ndarray) -> np.ndarray:
    """u_x(y) from nu [rho_{j+1/2}(u_{j+1} - u_j) - rho_{j-1/2}(u_j - u_{j-1})] + rho_j g = 0, with
    face densities the mean of their two nodes and ghost rows u_{-1} = 2 u_lo - u_0,
    u_{ny} = 2 u_hi - u_{ny-1} (the wall velocity half a cell outside the first and last rows)."""
    nu = (sc.tau[0] - 0.5) / 3.0
    n = sc.ny
    lo, hi = sc.u_wall
    g = sc.g[0]
    rf = 0.5 * (rho[1:] + rho[:-1])               # faces j + 1/2, j = 0 .. n-2
    rlo, rhi = rho[0], rho[-1]                    # wall faces take the adjacent node's density
    A = np.zeros((n, n))
    b = -rho * g / nu
    for j in range(n):
        wm = rlo if j == 0 else rf[j - 1]
        wp = rhi if j == n - 1 else rf[j]
        A[j, j] = -(wm + wp)
        if j > 0:
            A[j, j - 1] = wm
        else:  # u_{-1} = 2 lo - u_0
            A[j, j] -= wm
            b[j] -= 2.0 * wm * lo
        if j < n - 1:
            A[j, j + 1] = wp
        else:  # u_n = 2 hi - u_{n-1}
            A[j, j] -= wp
            b[j] -= 2.0 * wp * hi
    return np.linalg.solve(A, b)


def rel_l2(u: np.ndarray, ref: np.ndarray) -> float:
    return float(np.sqrt(np.sum((u - ref) ** 2) / np.sum(ref ** 2)))


def run(cs: list, max_steps: int = 400000, storage: str = "f32", interval: int = INTERVAL) -> list[dict]:
    """Step every case until all have converged (or max_steps) and return one record per case."""
    lat = lbm.Lattice(cs, storage)
    try:
        prev = None
        steps = 0
        conv = [None] * len(cs)
        while steps < max_steps:
            lat.step(interval)
            steps += interval
            fields = lat.fields_all()
            ux = [f[2] for f in fields]
            if prev is not None:
                for k in range(len(cs)):
                    if conv[k] is None and float(np.max(np.abs(ux[k] - prev[k]))) < TOL:
                        conv[k] = steps
            prev = ux
            if all(c is not None for c in conv):
                break
        diag = lat.diagnostics_all(allow_unstable=True)
    finally:
        lat.close()
    out = []
    for k, sc in enumerate(cs):
        rA, rB, ux_k = fields[k][0], fields[k][1], fields[k][2]
        u = ux_k.mean(axis=1)
        rho = (rA + rB).mean(axis=1)
        ua = analytic_profile(sc)
        ub = balance_profile(sc, rho)
        out.append({
            "case": sc.name, "flow": sc.extra["flow"], "target_theta": sc.extra["target_theta"], "lambda": sc.lam,
            "converged_at": conv[k], "steps": steps, "eps_analytic": rel_l2(u, ua), "eps_balance": rel_l2(u, ub),
            "u_peak": float(np.max(np.abs(u))), "u_peak_analytic": float(np.max(np.abs(ua))),
            "rho_min": float(rho.min()), "unstable": bool(diag[k]["unstable"]),
        })
    return out


def table(rows: list[dict]) -> str:
    lines = ["| flow | target θ | λ | converged at | ε vs analytic | ε vs momentum balance | peak \\|u_x\\| "
             "(analytic) | ρ min (x-mean) |", "|---|---|---|---|---|---|---|---|"]
    for r in rows:
        conv = "not within %d" % r["steps"] if r["converged_at"] is None else f"{r['converged_at']:,}"
        lines.append(f"| {r['flow']} | {r['target_theta']:.0f} | {r['lambda']:.4f} | {conv} "
                     f"| {100 * r['eps_analytic']:.2f} % | {100 * r['eps_balance']:.2f} % "
                     f"| {r['u_peak']:.3e} ({r['u_peak_analytic']:.3e}) | {r['rho_min']:.3f} |")
    return "\n".join(lines)


def main(argv=None) -> int:
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--storage", default="f32", choices=["f32", "f64"])
    ap.add_argument("--angles", default="45,90,135")
    ap.add_argument("--paper-params", action="store_true",
                    help="densities 1.02 / 0.05 and G_w2 = G_12 as stated in Sec. 3.1")
    ap.add_argument("--gw2", type=float, default=-1.0, help="override G_w2 (>= 0)")
    ap.add_argument("--gw2-is-g", action="store_true", help="G_w2 = G_12 (the paper's choice)")
    ap.add_argument("--second-layer", default="psi_and_solid", choices=["psi_and_solid", "psi"])
    ap.add_argument("--adhesion-stencil", default="e8", choices=["e8", "d2q9"],
                    help="stencil of the adhesion sum of Eq. 9 (d2q9: as printed, first layer)")
    ap.add_argument("--json", default=None)
    args = ap.parse_args(argv)
    angles = tuple(int(a) for a in args.angles.split(","))
    gw2 = None if args.gw2_is_g else args.gw2
    rows = run(cases(angles, args.paper_params, gw2, args.second_layer, args.adhesion_stencil), args.max_steps,
               args.storage)
    print(table(rows))
    if args.json:
        with open(args.json, "w") as fh:
            json.dump(rows, fh, indent=1)
    return 0


if __name__ == "__main__":
    sys.exit(main())
