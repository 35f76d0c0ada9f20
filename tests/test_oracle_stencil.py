"""Pins for the oracle's stencil: E8 weights (Sec. 2.4), Table 1's node correspondence, the
second-layer reconstruction, the wall list and the force sums (brute force on tiny grids)."""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _box_offsets():
    return [(dx, dy) for dy in range(-2, 3) for dx in range(-2, 3) if (dx, dy) != (0, 0)]


def _moment(w, a, b):
    return sum(w[dx * dx + dy * dy] * Fraction(dx) ** a * Fraction(dy) ** b for dx, dy in _box_offsets())


# ---------------------------------------------------------------------------------------------
# P1: weights
# ---------------------------------------------------------------------------------------------
def test_e8_weights_match_published_values():
    w = oracle.e8_weights()
    for q, num, den in _read("e8_weights.txt"):
        assert w[int(q)] == Fraction(int(num), int(den))


def test_e8_weights_isotropy_identities():
    """Moment identities of 8th-order isotropy, evaluated from the 5x5 box enumerated here."""
    w = oracle.e8_weights()
    assert _moment(w, 2, 0) == 1 and _moment(w, 0, 2) == 1
    assert _moment(w, 4, 0) == Fraction(12, 7) == 3 * _moment(w, 2, 2)
    assert _moment(w, 6, 0) == Fraction(32, 7) == 5 * _moment(w, 4, 2)
    assert _moment(w, 8, 0) == 16 == 7 * _moment(w, 6, 2)
    assert _moment(w, 4, 4) == Fraction(48, 35) == Fraction(3, 5) * _moment(w, 6, 2)
    for a in range(0, 9):
        for b in range(0, 9):
            if (a % 2 or b % 2) and a + b <= 9:
                assert _moment(w, a, b) == 0, (a, b)


def test_e8_offset_table_covers_the_5x5_box():
    offs = oracle.e8_offsets()
    assert sorted(offs) == sorted(_box_offsets())
    # first layer in the D2Q9 order: axes (1,0),(0,1),(-1,0),(0,-1) then diagonals
    assert offs[:8] == [(1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
    assert all(max(abs(dx), abs(dy)) == 2 for dx, dy in offs[8:])
    # pairs (e, -e) sit two apart within each group of four (the force sums rely on it)
    for n in range(0, 24, 4):
        for j in range(2):
            a, b = offs[n + j], offs[n + j + 2]
            assert a == (-b[0], -b[1])


# ---------------------------------------------------------------------------------------------
# P12: Table 1 -- second-layer node n takes the information of first-layer node m = sign(e_n)
# ---------------------------------------------------------------------------------------------
def test_table1_correspondence_is_sign_of_offset():
    offs = oracle.e8_offsets()
    rows = _read("table1_node_correspondence.txt")
    assert len(rows) == 16
    for n, m in rows:
        n, m = int(n), int(m)
        ex, ey = offs[n - 1]
        assert offs[m - 1] == (int(np.sign(ex)), int(np.sign(ey))), (n, m)
        # ranges printed in Table 1
        assert m == (n - 8 if n <= 16 else n - 12 if n <= 20 else n - 16)


# ---------------------------------------------------------------------------------------------
# P11: brute force on tiny grids
# ---------------------------------------------------------------------------------------------
def _weights_float():
    return {int(q): int(a) / int(b) for q, a, b in _read("e8_weights.txt")}


def _bf_forces(cfg, solid, rhoA, rhoB):
    """Independent loop over the 5x5 box of each fluid node: cohesion (Eq. 8, other component,
    E8 weights), adhesion (Eq. 9 with the local parameter of Eq. 12 / constant G_w1), body force;
    second-layer sites that are not in-array fluid nodes take the value of x + sign(e): its density
    and its solid switch, or (second_layer "psi") its density while the site keeps its own switch.
    With adhesion_stencil "d2q9" the adhesion sum is Eq. 9 as printed: the eight first neighbours
    with the lattice weights 1/9 (axes) and 1/36 (diagonals) times their solid switch."""
    W = _weights_float()
    ny, nx = solid.shape
    Gw2 = cfg.G if cfg.Gw2 is None else cfg.Gw2

    def site(X, Y):
        if not 0 <= X < nx:
            if cfg.bc_x != "periodic":
                return None
            X %= nx
        if not 0 <= Y < ny:
            if cfg.bc_y != "periodic":
                return None
            Y %= ny
        return X, Y

    def first(x, y, dx, dy):
        X = x + dx
        if cfg.bc_x == "open":
            X = min(max(X, 0), nx - 1)
        p = site(X, y + dy)
        if p is None or solid[p[1], p[0]]:
            return 0.0, 0.0, 1.0
        return rhoA[p[1], p[0]], rhoB[p[1], p[0]], 0.0

    FA = np.zeros((2, ny, nx))
    FB = np.zeros((2, ny, nx))
    for y in range(ny):
        for x in range(nx):
            if solid[y, x]:
                continue
            gA = np.zeros(2)
            gB = np.zeros(2)
            a = np.zeros(2)
            for dy in range(-2, 3):
                for dx in range(-2, 3):
                    if dx == 0 and dy == 0:
                        continue
                    w = W[dx * dx + dy * dy]
                    if max(abs(dx), abs(dy)) == 2:
                        p = site(x + dx, y + dy)
                        if p is not None and not solid[p[1], p[0]]:
                            vA, vB, s = rhoA[p[1], p[0]], rhoB[p[1], p[0]], 0.0
                        else:
                            vA, vB, s = first(x, y, int(np.sign(dx)), int(np.sign(dy)))
                            if cfg.second_layer == "psi":  # the site's own switch
                                s = first(x, y, dx, dy)[2]
                    else:
                        vA, vB, s = first(x, y, dx, dy)
                    e = np.array([dx, dy], float)
                    gA += w * vA * e
                    gB += w * vB * e
                    a += w * s * e
            if cfg.adhesion_stencil == "d2q9":
                a = np.zeros(2)
                for dy in (-1, 0, 1):
                    for dx in (-1, 0, 1):
                        if dx or dy:
                            wi = 1.0 / 9.0 if abs(dx) + abs(dy) == 1 else 1.0 / 36.0
                            a += wi * first(x, y, dx, dy)[2] * np.array([dx, dy], float)
            rA, rB = rhoA[y, x], rhoB[y, x]
            if cfg.scheme == "improved":
                re = (rA - rB) / (rA + rB)
                lam, d = cfg.lam, cfg.delta
                s1 = 2 * lam / (1 + lam)
                if re > d:
                    h = lam
                elif re > 0:
                    h = s1 + 2 * (lam * lam - lam) / (d * (1 + lam)) * re + (lam - lam * lam) / (d * d * (1 + lam)) * re * re
                elif re > -d:
                    h = s1 + 2 * (lam - 1) / (d * (1 + lam)) * re + (lam - 1) / (d * d * (1 + lam)) * re * re
                else:
                    h = 1.0
                GA = Gw2 * h
            else:
                GA = cfg.lam * Gw2
            g = np.array(cfg.g, float)
            FA[:, y, x] = -cfg.G * rA * gB - GA * rA * a + rA * g
            FB[:, y, x] = -cfg.G * rB * gA - Gw2 * rB * a + rB * g
    return FA, FB


def _pillar_case(nx=8, ny=8, block=None):
    solid = np.zeros((ny, nx), np.uint8)
    if block is None:
        solid[3, 3] = 1
    else:
        (x0, x1), (y0, y1) = block
        solid[y0:y1, x0:x1] = 1
    return solid


@pytest.mark.parametrize("adhesion_stencil", ["e8", "d2q9"])
@pytest.mark.parametrize("second_layer", ["psi_and_solid", "psi"])
@pytest.mark.parametrize("scheme,lam", [("improved", 0.4), ("improved", 1.7), ("original", 0.6)])
@pytest.mark.parametrize("geom", ["pillar", "block_walls", "open_x"])
def test_forces_match_brute_force(scheme, lam, geom, second_layer, adhesion_stencil):
    rng = np.random.default_rng(7)
    if geom == "pillar":
        solid = _pillar_case()
        cfg = oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic", scheme=scheme, lam=lam,
                            G=1.2, g=(1e-3, -2e-3), nthreads=1)
    elif geom == "block_walls":
        solid = _pillar_case(9, 8, ((2, 5), (3, 6)))
        solid[5, 7] = 1
        cfg = oracle.Config(nx=9, ny=8, bc_x="periodic", bc_y="wall", scheme=scheme, lam=lam, G=1.2,
                            Gw2=0.7, nthreads=1)
    else:
        solid = _pillar_case(10, 7)
        solid[0, :] = 1
        cfg = oracle.Config(nx=10, ny=7, bc_x="open", bc_y="wall", scheme=scheme, lam=lam, G=1.2,
                            nthreads=1)
    cfg.second_layer = second_layer
    cfg.adhesion_stencil = adhesion_stencil
    ny, nx = solid.shape
    rA = rng.uniform(0.02, 1.1, (ny, nx)) * (1 - solid)
    rB = rng.uniform(0.02, 1.1, (ny, nx)) * (1 - solid)
    # a state whose densities are exactly these: all mass in the rest population
    f = np.zeros((2, 9, ny, nx))
    f[0, 0] = rA
    f[1, 0] = rB
    FA, FB = oracle.forces(cfg, solid, f)
    bA, bB = _bf_forces(cfg, solid, rA, rB)
    np.testing.assert_allclose(FA, bA, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(FB, bB, rtol=1e-12, atol=1e-14)


def _entry(node, subst, seff, ax, ay, nx, x, y):
    k = np.nonzero(node == y * nx + x)[0]
    assert len(k) == 1, (x, y)
    k = k[0]
    return int(subst[k]), int(seff[k]), ax[k], ay[k]


def _bits(*nodes):
    """Mask with the bits of the given 1-based stencil node numbers."""
    m = 0
    for n in nodes:
        m |= 1 << (n - 1)
    return m


def test_wall_list_single_pillar_by_hand():
    """8x8 fully periodic, one solid node at (3,3): the wall list is the 24 nodes around it."""
    solid = _pillar_case()
    cfg = oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    expect = sorted((3 + dy) * 8 + (3 + dx) for dy in range(-2, 3) for dx in range(-2, 3)
                    if (dx, dy) != (0, 0))
    assert node.tolist() == expect
    W = _weights_float()
    # (3,4): pillar is first-layer node 4 (0,-1)
    assert _entry(node, subst, seff, ax, ay, 8, 3, 4) == (0, _bits(4), 0.0, -W[1])
    # (3,5): pillar is second-layer node 12 (0,-2): replaced by first-layer node 4 = (3,4), fluid
    assert _entry(node, subst, seff, ax, ay, 8, 3, 5) == (_bits(12), 0, 0.0, 0.0)
    # (5,5): pillar is node 15 (-2,-2) -> node 7 (-1,-1) = (4,4), fluid
    assert _entry(node, subst, seff, ax, ay, 8, 5, 5) == (_bits(15), 0, 0.0, 0.0)
    # (5,4): pillar is knight node 19 (-2,-1) -> node 7 (-1,-1) = (4,3), fluid
    assert _entry(node, subst, seff, ax, ay, 8, 5, 4) == (_bits(19), 0, 0.0, 0.0)
    # (4,5): pillar is knight node 23 (-1,-2) -> node 7 = (3,4), fluid
    assert _entry(node, subst, seff, ax, ay, 8, 4, 5) == (_bits(23), 0, 0.0, 0.0)
    # (2,2): pillar is first-layer diagonal node 5 (1,1)
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 8, 2, 2)
    assert (sm, em) == (0, _bits(5)) and a_x == pytest.approx(W[2]) and a_y == pytest.approx(W[2])


def test_wall_list_single_pillar_psi_only_by_hand():
    """The same pillar when a replaced second-layer node copies psi only: the solid site itself
    stays in the adhesion sum, so seff gains the replaced node and a(x) its w e term."""
    solid = _pillar_case()
    cfg = oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic", second_layer="psi")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    W = _weights_float()
    assert _entry(node, subst, seff, ax, ay, 8, 3, 4) == (0, _bits(4), 0.0, -W[1])  # first layer: unchanged
    # (3,5): node 12 = (0,-2) replaced, counted as solid: a = w(4) (0,-2)
    assert _entry(node, subst, seff, ax, ay, 8, 3, 5) == (_bits(12), _bits(12), 0.0, -2 * W[4])
    # (5,5): node 15 = (-2,-2): a = w(8) (-2,-2)
    assert _entry(node, subst, seff, ax, ay, 8, 5, 5) == (_bits(15), _bits(15), -2 * W[8], -2 * W[8])
    # (5,4): knight node 19 = (-2,-1): a = w(5) (-2,-1)
    assert _entry(node, subst, seff, ax, ay, 8, 5, 4) == (_bits(19), _bits(19), -2 * W[5], -W[5])
    # the substitution masks (which sites take psi from x + sign(e)) do not depend on the reading
    _, subst0, _, _, _ = oracle.wall_list(oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic"), solid)
    np.testing.assert_array_equal(subst, subst0)


def test_wall_list_block_by_hand():
    """8x8 fully periodic with a 3x3 solid block at x, y in [2, 4]."""
    solid = _pillar_case(8, 8, ((2, 5), (2, 5)))
    cfg = oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    W = _weights_float()
    # fluid nodes within two cells (Chebyshev, on the torus) of the block: all but column 7 and row 7
    near = [(x, y) for y in range(8) for x in range(8) if not solid[y, x] and x != 7 and y != 7]
    assert node.tolist() == sorted(y * 8 + x for x, y in near)
    # (3,5) right above the block's middle column
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 8, 3, 5)
    assert sm == _bits(12, 23, 24)
    assert em == _bits(4, 7, 8, 12, 23, 24)
    assert a_x == pytest.approx(0.0, abs=1e-15)
    assert a_y == pytest.approx(-(W[1] + 2 * W[2] + 2 * W[4] + 4 * W[5]))
    # (3,6): (0,-2) = (3,4) is solid -> copied from (3,5), fluid; (+-1,-2), (+-2,-2) solid or
    # fluid per the block: (2,4),(4,4) solid -> from (2,5),(4,5) fluid; (1,4),(5,4) fluid
    sm, em, _, _ = _entry(node, subst, seff, ax, ay, 8, 3, 6)
    assert sm == _bits(12, 23, 24) and em == 0


def test_wall_list_counts_outside_of_wall_direction():
    """Rows outside the array along a wall direction count as solid; periodic ones do not."""
    solid = np.zeros((10, 6), np.uint8)
    cfg = oracle.Config(nx=6, ny=10, bc_x="periodic", bc_y="wall")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    rows = sorted(set((node // 6).tolist()))
    assert rows == [0, 1, 8, 9]
    W = _weights_float()
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 6, 2, 0)
    # y = -1 and y = -2 are outside: layer 1 below solid, layer 2 below copied from layer 1
    assert em == _bits(4, 7, 8, 12, 19, 20, 15, 16, 23, 24)
    assert sm == _bits(12, 15, 16, 19, 20, 23, 24)
    assert a_y == pytest.approx(-(W[1] + 2 * W[2] + 2 * W[4] + 6 * W[5] + 4 * W[8]))


# ---------------------------------------------------------------------------------------------
# Eq. 9 as printed: D2Q9 weights over the first layer (adhesion_stencil = "d2q9")
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("second_layer", ["psi_and_solid", "psi"])
def test_wall_list_single_pillar_d2q9_adhesion_by_hand(second_layer):
    """The 8x8 pillar under the printed Eq. 9: a(x) = sum_i w_i s(x + e_i) e_i with w = 1/9 on the
    axes and 1/36 on the diagonals.  Only the eight first neighbours of the pillar feel it, whatever
    the second-layer reading; the substitution masks (cohesion) are unchanged."""
    solid = _pillar_case()
    cfg = oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic", second_layer=second_layer,
                        adhesion_stencil="d2q9")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    # (3,4): the pillar is first-layer node 4 = e_4 = (0,-1): a = (1/9) (0,-1)
    assert _entry(node, subst, seff, ax, ay, 8, 3, 4) == (0, _bits(4), 0.0, -1.0 / 9.0)
    # (2,3): pillar at e_1 = (1,0)
    assert _entry(node, subst, seff, ax, ay, 8, 2, 3) == (0, _bits(1), 1.0 / 9.0, 0.0)
    # (2,2): pillar at e_5 = (1,1): a = (1/36) (1,1)
    assert _entry(node, subst, seff, ax, ay, 8, 2, 2) == (0, _bits(5), 1.0 / 36.0, 1.0 / 36.0)
    # (4,2): pillar at e_6 = (-1,1)
    assert _entry(node, subst, seff, ax, ay, 8, 4, 2) == (0, _bits(6), -1.0 / 36.0, 1.0 / 36.0)
    # second-layer nodes of the pillar: still in the wall list (cohesion substitution), no adhesion
    assert _entry(node, subst, seff, ax, ay, 8, 3, 5) == (_bits(12), 0, 0.0, 0.0)
    assert _entry(node, subst, seff, ax, ay, 8, 5, 5) == (_bits(15), 0, 0.0, 0.0)
    assert _entry(node, subst, seff, ax, ay, 8, 5, 4) == (_bits(19), 0, 0.0, 0.0)
    _, subst_e8, _, _, _ = oracle.wall_list(oracle.Config(nx=8, ny=8, bc_x="periodic", bc_y="periodic"), solid)
    np.testing.assert_array_equal(subst, subst_e8)


def test_flat_wall_d2q9_adhesion_vector():
    """Outside a walled y: the first row sees e_4, e_7, e_8 solid, a_y = -(1/9 + 2/36) = -1/6 (the
    D2Q9 first moment sum_(e_y < 0) w_i e_y); the second row sees no solid first neighbour."""
    solid = np.zeros((10, 6), np.uint8)
    cfg = oracle.Config(nx=6, ny=10, bc_x="periodic", bc_y="wall", adhesion_stencil="d2q9")
    node, subst, seff, ax, ay = oracle.wall_list(cfg, solid)
    assert sorted(set((node // 6).tolist())) == [0, 1, 8, 9]
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 6, 2, 0)
    assert em == _bits(4, 7, 8) and a_x == 0.0 and a_y == pytest.approx(-1.0 / 6.0, abs=1e-16)
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 6, 2, 9)
    assert em == _bits(2, 5, 6) and a_y == pytest.approx(1.0 / 6.0, abs=1e-16)
    sm, em, a_x, a_y = _entry(node, subst, seff, ax, ay, 6, 2, 1)
    assert em == 0 and a_x == 0.0 and a_y == 0.0 and sm == _bits(12, 23, 24, 15, 16)


def test_d2q9_adhesion_force_next_to_a_wall_by_hand():
    """Uniform densities, no cohesion (G = 0): the only force at a first-row node is the adhesion
    of Eq. 9, F_k = -G_w,k rho_k a = G_w,k rho_k / 6 along +y (original scheme, G_w1 = lambda G_w2);
    nodes further out feel nothing."""
    nx, ny = 6, 9
    solid = np.zeros((ny, nx), np.uint8)
    cfg = oracle.Config(nx=nx, ny=ny, bc_x="periodic", bc_y="wall", scheme="original", G=0.0, lam=0.5,
                        Gw2=0.3, adhesion_stencil="d2q9", nthreads=1)
    f = np.zeros((2, 9, ny, nx))
    f[0, 0] = 0.8
    f[1, 0] = 0.1
    FA, FB = oracle.forces(cfg, solid, f)
    assert np.all(FA[0] == 0.0) and np.all(FB[0] == 0.0)
    np.testing.assert_allclose(FA[1, 0], 0.5 * 0.3 * 0.8 / 6.0, rtol=1e-14)
    np.testing.assert_allclose(FB[1, 0], 0.3 * 0.1 / 6.0, rtol=1e-14)
    np.testing.assert_allclose(FA[1, -1], -0.5 * 0.3 * 0.8 / 6.0, rtol=1e-14)
    assert np.all(FA[1, 1:-1] == 0.0) and np.all(FB[1, 1:-1] == 0.0)
