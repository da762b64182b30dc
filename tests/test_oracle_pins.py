"""Pins of the CPU oracle against the paper's definitions (no GPU needed).

Each test compares the oracle with something other than itself: global
topology computed by connected-component labelling, brute-force distances,
explicit unions of Euclidean discs, closed forms that hold for topologically
trivial shapes, invariants, and hand-worked examples under tests/golden/.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from paper_1603_09337_gb300 import synth
from tests import _brute as B

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --- simple points (Sec. 2, T and Tbar) -------------------------------------

OFFS = [(0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1), (1, 0), (1, 1)]  # (dy, dx): E..SE


def code_image(code: int, centre: int = 1) -> np.ndarray:
    img = np.zeros((7, 7), np.uint8)
    img[3, 3] = centre
    for k, (dy, dx) in enumerate(OFFS):
        img[3 + dy, 3 + dx] = (code >> k) & 1
    return img


@pytest.mark.parametrize("conn", [8, 4])
def test_lut_equals_global_definition_on_all_codes(conn):
    """Every neighbour configuration, placed alone on a background, is simple
    for the LUT iff removing the centre keeps the global component counts
    (Sec. 2 definition of a simple point)."""
    lut = oracle.simple_lut(conn)
    for code in range(256):
        assert lut[code] == B.globally_simple(code_image(code), 3, 3, conn), code


@pytest.mark.parametrize("conn", [8, 4])
def test_lut_in_random_images(conn):
    """Inside random images, removable object points and addable background
    points are exactly the LUT-simple ones."""
    lut = oracle.simple_lut(conn)
    for seed in range(12):
        X = synth.small_random(seed, 11, 9, density_permille=350 + 30 * seed)
        P = np.pad(X, 1)
        for y in range(9):
            for x in range(11):
                code = 0
                for k, (dy, dx) in enumerate(OFFS):
                    code |= int(P[y + 1 + dy, x + 1 + dx]) << k
                assert lut[code] == B.globally_simple(X, y, x, conn), (seed, y, x)


def test_lut_duality():
    """(4,8)-simplicity of a code is (8,4)-simplicity of its complement."""
    l8, l4 = oracle.simple_lut(8), oracle.simple_lut(4)
    for c in range(256):
        assert l4[c] == l8[(~c) & 0xFF]


# --- distance transform (Sec. 4.1) ------------------------------------------

EDT_CASES = [(1, 1), (1, 17), (17, 1), (5, 7), (32, 32), (31, 33), (40, 23)]


@pytest.mark.parametrize("h,w", EDT_CASES)
@pytest.mark.parametrize("outside", [False, True])
def test_edt_equals_brute_force(h, w, outside):
    for seed, dens in [(1, 20), (2, 150), (3, 500), (4, 950)]:
        F = synth.small_random(seed * 97 + h * 7 + w, w, h, dens)
        np.testing.assert_array_equal(oracle.edt(F, outside), B.edt_brute(F, outside))


def test_edt_edge_cases():
    z = np.zeros((9, 13), np.uint8)
    assert (oracle.edt(z) == oracle.INF).all()          # no feature: infinite
    assert (oracle.edt(np.ones_like(z)) == 0).all()     # all feature: zero
    d = oracle.edt(z, outside_is_feature=True)           # only the outside
    yy, xx = np.mgrid[0:9, 0:13]
    near = np.minimum.reduce([xx + 1, 13 - xx, yy + 1, 9 - yy])
    np.testing.assert_array_equal(d, near.astype(np.int64) ** 2)
    one = z.copy()
    one[4, 6] = 1
    np.testing.assert_array_equal(oracle.edt(one), (yy - 4) ** 2 + (xx - 6) ** 2)


# --- erosion / dilation by Euclidean balls (Sec. 2) --------------------------

@pytest.mark.parametrize("r", [1, 2, 3, 5, 7])
def test_masks_equal_disc_unions(r):
    for seed in range(4):
        S = synth.shapes_image(seed, 45, 38, 4, 3, 12, n_holes=1, hole_lo=2, hole_hi=4,
                               jitter=1, noise_permille=40)
        np.testing.assert_array_equal(oracle.dilate(S, r), B.dilate_union(S, r))
        np.testing.assert_array_equal(oracle.erode(S, r), B.erode_union(S, r))


# --- thinning / thickening invariants (Sec. 2) --------------------------------

def _prio_thin(Z):
    return oracle.edt(1 - Z, outside_is_feature=True)


@pytest.mark.parametrize("conn", [8, 4])
def test_thin_invariants(conn):
    """W within H(Z,W) within Z; same topology; no simple point left in the
    result outside W (the thinning is ultimate)."""
    for seed in range(6):
        Z = synth.shapes_image(seed, 24, 20, 3, 3, 8, n_holes=1, hole_lo=1, hole_hi=2,
                               jitter=1, noise_permille=30)
        Wc = synth.small_random(seed + 100, 24, 20, 60) & Z
        res = oracle.thin(Z, Wc, _prio_thin(Z), conn)
        assert ((Wc <= res) & (res <= Z)).all()
        assert B.component_counts(res, conn) == B.component_counts(Z, conn)
        for y, x in np.argwhere((res == 1) & (Wc == 0)):
            assert not B.globally_simple(res, y, x, conn), (seed, y, x)


@pytest.mark.parametrize("conn", [8, 4])
def test_ultimate_thinning_of_a_simply_connected_set_is_one_point(conn):
    """With W empty, a set that is one component with a connected complement
    thins down to a single point (2D: such a set is reducible to a point by
    simple deletions, and the thinning stops only when no point is simple)."""
    used = 0
    for seed in range(12):
        Z = synth.shapes_image(seed + 300, 30, 26, 1 + seed % 2, 3, 9, n_holes=0, jitter=0,
                               noise_permille=0)
        if B.component_counts(Z, conn) != (1, 1):
            continue
        used += 1
        res = oracle.thin(Z, np.zeros_like(Z), _prio_thin(Z), conn)
        assert res.sum() == 1 and (res <= Z).all()
    assert used >= 3


@pytest.mark.parametrize("conn", [8, 4])
def test_thicken_invariants(conn):
    """Y within *H(Y,V) within Y cup V; same topology; no point of V left that
    could still be added."""
    for seed in range(6):
        Y = synth.shapes_image(seed + 50, 24, 20, 3, 3, 8, n_holes=1, hole_lo=1, hole_hi=2,
                               jitter=1, noise_permille=30)
        V = synth.small_random(seed + 200, 24, 20, 700)
        res = oracle.thicken(Y, V, oracle.edt(Y), conn)
        assert ((Y <= res) & (res <= (Y | V))).all()
        assert B.component_counts(res, conn) == B.component_counts(Y, conn)
        for y, x in np.argwhere((res == 0) & (V == 1)):
            assert not B.globally_simple(res, y, x, conn), (seed, y, x)


def _sweep_python(S, K, prio, remove, conn, rng):
    """Tiny pure-Python restatement of the sweep order with the points of each
    subfield visited in a random order (which must not matter: points of one
    subfield are never 8-adjacent)."""
    lut = oracle.simple_lut(conn)
    S = S.copy()
    h, w = S.shape

    def cand(y, x):
        return (S[y, x] and not K[y, x]) if remove else (not S[y, x] and K[y, x])

    levels = sorted({int(prio[y, x]) for y in range(h) for x in range(w) if cand(y, x)})
    for lv in levels:
        while True:
            changed = False
            for sy in (0, 1):
                for sx in (0, 1):
                    pts = [(y, x) for y in range(sy, h, 2) for x in range(sx, w, 2)]
                    rng.shuffle(pts)
                    for y, x in pts:
                        if not cand(y, x) or prio[y, x] > lv:
                            continue
                        code = 0
                        for k, (dy, dx) in enumerate(OFFS):
                            yy, xx = y + dy, x + dx
                            if 0 <= yy < h and 0 <= xx < w and S[yy, xx]:
                                code |= 1 << k
                        if lut[code]:
                            S[y, x] = 0 if remove else 1
                            changed = True
            if not changed:
                break
    return S


def test_sweep_order_within_subfield_is_irrelevant():
    rng = np.random.default_rng(5)
    for seed in range(5):
        Z = synth.shapes_image(seed + 300, 18, 14, 3, 2, 6, jitter=1, noise_permille=50)
        Wc = synth.small_random(seed + 7, 18, 14, 80) & Z
        pr = _prio_thin(Z)
        np.testing.assert_array_equal(oracle.thin(Z, Wc, pr), _sweep_python(Z, Wc, pr, True, 8, rng))
        V = synth.small_random(seed + 9, 18, 14, 600)
        pr = oracle.edt(Z)
        np.testing.assert_array_equal(oracle.thicken(Z, V, pr),
                                      _sweep_python(Z, V, pr, False, 8, rng))


def _read_golden(path):
    blocks, cur, key = [], None, None
    for line in open(path):
        line = line.rstrip("\n")
        if line.startswith("#") or not line.strip():
            key = None if line.startswith("#") else key
            continue
        if line.startswith("name:"):
            cur = {"name": line.split(":", 1)[1].strip()}
            blocks.append(cur)
        elif line.split(":")[0] in ("op", "cite", "rmax"):
            k, v = line.split(":", 1)
            cur[k] = v.strip()
        elif line in ("input:", "expected:", "swapped:"):
            key = line[:-1]
            cur[key] = []
        else:
            cur[key].append(line)
    return blocks


def test_hand_worked_examples():
    blocks = _read_golden(os.path.join(GOLDEN, "sweep_examples.txt"))
    assert len(blocks) >= 4
    for b in blocks:
        grid = np.array([list(r) for r in b["input"]])
        exp = (np.array([list(r) for r in b["expected"]]) == "#").astype(np.uint8)
        S = (grid == "#").astype(np.uint8)
        if b["op"] == "thin":
            res = oracle.thin(S, np.zeros_like(S), B.edt_brute(1 - S, True))
        else:
            V = ((grid == "v") | (grid == "#")).astype(np.uint8)
            res = oracle.thicken(S, V, B.edt_brute(S))
        np.testing.assert_array_equal(res, exp, err_msg=b["name"])


def _grid(rows):
    return (np.array([list(r) for r in rows]) == "#").astype(np.uint8)


def test_hand_worked_hasf1_order():
    """HASF_1 = HF_1 o HC_1 (cutting first): on the worked example the filter
    gives the hand-derived image, and the operators applied the other way
    round give the other hand-derived image."""
    blocks = _read_golden(os.path.join(GOLDEN, "hasf1_order.txt"))
    assert blocks
    for b in blocks:
        assert b["op"] == "hasf"
        X, want, other = _grid(b["input"]), _grid(b["expected"]), _grid(b["swapped"])
        r = int(b["rmax"])
        assert (want != other).any()
        np.testing.assert_array_equal(oracle.hasf(X, r), want, err_msg=b["name"])
        np.testing.assert_array_equal(oracle.hf(oracle.hc(X, r), r), want, err_msg=b["name"])
        np.testing.assert_array_equal(oracle.hc(oracle.hf(X, r), r), other, err_msg=b["name"])


# --- cutting, filling, HASF (Sec. 2, eqs. (i), (ii)) ---------------------------

def _trivial_shapes():
    """Convex blobs plus non-convex unions (L / T / cross shapes, pairs of
    overlapping ellipses), whose openings and closings differ from them."""
    out = []
    for seed in range(60):
        rng = synth.SplitMix64(seed + 900)
        img = np.zeros((48, 52), np.uint8)
        kind = seed % 4
        if kind == 0:
            img[rng.randint(6, 12):rng.randint(30, 40), rng.randint(6, 12):rng.randint(30, 44)] = 1
        elif kind == 1:
            a, b = rng.randint(6, 15), rng.randint(6, 15)
            u, v = rng.direction(16)
            synth._paint_ellipse(img, 26, 24, a, b, u, v, 1)
        elif kind == 2:   # two bars: L, T or cross shapes
            y0, x0 = rng.randint(6, 16), rng.randint(6, 16)
            img[y0:y0 + rng.randint(5, 9), x0:rng.randint(34, 46)] = 1
            x1 = rng.randint(x0, 30)
            img[rng.randint(4, y0):rng.randint(32, 44), x1:x1 + rng.randint(5, 9)] = 1
        else:             # two overlapping ellipses (a waist to fill)
            for cx in (18, 34):
                a, b = rng.randint(7, 12), rng.randint(7, 12)
                u, v = rng.direction(16)
                synth._paint_ellipse(img, cx + rng.randint(-2, 2), 24 + rng.randint(-3, 3),
                                     a, b, u, v, 1)
        out.append(img)
    return out


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_cutting_is_opening_on_trivial_shapes(r):
    """When X, eps_r(X) and the opening gamma_r(X) are each one component with
    a connected complement, every step of (i) preserves topology, so (2D,
    Ronse) the ultimate thinning reaches eps_r(X) and the thickening reaches
    gamma_r(X): HC_r(X) is the plain opening by B_r."""
    used = changed = 0
    for X in _trivial_shapes():
        E, G = B.erode_union(X, r), B.opening(X, r)
        if not (B.is_simply_connected(X) and E.any() and B.is_simply_connected(E)
                and B.is_simply_connected(G)):
            continue
        used += 1
        changed += int((G != X).any())
        np.testing.assert_array_equal(oracle.hc(X, r), G)
    assert used >= 20 and changed >= 10


@pytest.mark.parametrize("r", [1, 2, 3, 4])
def test_filling_is_closing_on_trivial_shapes(r):
    """Dual of the above for (ii): when X, delta_r(X) and eps_r(delta_r(X)) cup X
    are simply connected, HF_r(X) = eps_r(delta_r(X)) cup X (the closing,
    joined with X where the box border cuts the closing)."""
    used = changed = 0
    for X in _trivial_shapes():
        Dl = B.dilate_union(X, r)
        Wx = B.erode_union(Dl, r) | X
        if not (B.is_simply_connected(X) and B.is_simply_connected(Dl)
                and B.is_simply_connected(Wx)):
            continue
        used += 1
        changed += int((Wx != X).any())
        np.testing.assert_array_equal(oracle.hf(X, r), Wx)
    assert used >= 20 and changed >= 10


def _spur_shapes():
    """A block with 2-4 spurs (width 1-3, length 3-8) and 1-3 notches (width
    1-3, depth 2-6) on its sides: features of every size from 1 to 3, so
    that openings and closings of different radii, and their order, matter."""
    out = []
    for seed in range(48):
        rng = synth.SplitMix64(seed + 7000)
        img = np.zeros((56, 60), np.uint8)
        y0, x0 = rng.randint(10, 16), rng.randint(10, 16)
        y1, x1 = rng.randint(36, 44), rng.randint(38, 48)
        img[y0:y1, x0:x1] = 1
        for val, count in ((1, rng.randint(2, 5)), (0, rng.randint(1, 4))):
            for _ in range(count):
                wd = rng.randint(1, 3)
                ln = rng.randint(3, 8) if val else rng.randint(2, 6)
                side = rng.randint(0, 3)
                if side < 2:
                    p = rng.randint(x0 + 2, x1 - 6)
                    ys = (slice(y0 - ln, y0) if side == 0 else slice(y1, y1 + ln)) if val else \
                         (slice(y0, y0 + ln) if side == 0 else slice(y1 - ln, y1))
                    img[ys, p:p + wd] = val
                else:
                    p = rng.randint(y0 + 2, y1 - 6)
                    xs = (slice(x0 - ln, x0) if side == 2 else slice(x1, x1 + ln)) if val else \
                         (slice(x0, x0 + ln) if side == 2 else slice(x1 - ln, x1))
                    img[p:p + wd, xs] = val
        out.append(img)
    return out


def _alternating(X, steps):
    """The classical alternating filter by explicit disc unions: for each
    ("open" | "close", r) in order, gamma_r(Y) = delta_r(eps_r(Y)) or
    phi_r(Y) = eps_r(delta_r(Y)) cup Y.  None unless every step meets the
    conditions under which HC_r = gamma_r and HF_r = phi_r (the sets involved
    are each one component with a connected complement; see the two tests
    above)."""
    Y = X.copy()
    for kind, r in steps:
        if kind == "open":
            E, G = B.erode_union(Y, r), B.opening(Y, r)
            if not (B.is_simply_connected(Y) and E.any() and B.is_simply_connected(E)
                    and B.is_simply_connected(G)):
                return None
            Y = G
        else:
            Wx = B.erode_union(B.dilate_union(Y, r), r) | Y
            if not (B.is_simply_connected(Y) and B.is_simply_connected(B.dilate_union(Y, r))
                    and B.is_simply_connected(Wx)):
                return None
            Y = Wx
    return Y.astype(np.uint8)


@pytest.mark.parametrize("n", [2, 3])
def test_hasf_is_the_alternating_filter_on_trivial_shapes(n):
    """HASF_n = HF_n o HC_n o ... o HF_1 o HC_1 (Sec. 2), read right to left:
    radii ascending, cutting before filling.  Where every intermediate set is
    one component with a connected complement, each HC_r is the opening and
    each HF_r the closing cup Y, so HASF_n(X) is the alternating sequential
    filter phi_n gamma_n ... phi_1 gamma_1 (X) computed by disc unions.  The
    shapes are chosen so that the other orders (filling first, or radii
    descending) give other images: a filter composed that way fails here."""
    used = swapped_differs = descending_differs = 0
    for X in _spur_shapes():
        want = _alternating(X, [(k, r) for r in range(1, n + 1) for k in ("open", "close")])
        if want is None:
            continue
        used += 1
        np.testing.assert_array_equal(oracle.hasf(X, n), want)
        sw = _alternating(X, [(k, r) for r in range(1, n + 1) for k in ("close", "open")])
        de = _alternating(X, [(k, r) for r in range(n, 0, -1) for k in ("open", "close")])
        swapped_differs += sw is not None and bool((sw != want).any())
        descending_differs += de is not None and bool((de != want).any())
    assert used >= 30 and swapped_differs >= 10 and descending_differs >= 10, \
        (used, swapped_differs, descending_differs)


def test_open_and_closed_image_is_a_fixed_point():
    """Separated large discs that every opening and closing by B_r, r <= 3,
    leaves unchanged are left unchanged by HASF_3."""
    used = 0
    for seed in range(12):
        rng = synth.SplitMix64(seed + 4000)
        X = np.zeros((96, 96), np.uint8)
        for cx, cy in [(24, 24), (72, 24), (24, 72), (72, 72)]:
            rad = rng.randint(9, 16)
            synth._paint_ellipse(X, cx + rng.randint(-3, 3), cy + rng.randint(-3, 3),
                                 rad, rad, 1, 0, 1)
        if not all((B.opening(X, r) == X).all() and (B.closing(X, r) == X).all()
                   for r in (1, 2, 3)):
            continue
        used += 1
        np.testing.assert_array_equal(oracle.hasf(X, 3), X)
    assert used >= 3


@pytest.mark.parametrize("conn", [8, 4])
def test_hasf_invariants(conn):
    """HASF keeps the component counts of X and of its complement, keeps C and
    never adds a point of D."""
    for seed in range(4):
        X = synth.shapes_image(seed + 77, 64, 56, 5, 4, 14, n_holes=2, hole_lo=2, hole_hi=4,
                               jitter=2, noise_permille=50)
        C = synth.constraint_points(seed, X, 10)
        Dm = synth.small_random(seed + 5, 64, 56, 30) & (1 - X)
        out = oracle.hasf(X, 3, C=C, D=Dm, conn=conn)
        assert B.component_counts(out, conn) == B.component_counts(X, conn)
        assert (out >= C).all()
        assert not (out & Dm).any()


def test_hasf_trivial_cases():
    for h, w in [(1, 1), (1, 9), (9, 1), (2, 2), (5, 7)]:
        z = np.zeros((h, w), np.uint8)
        np.testing.assert_array_equal(oracle.hasf(z, 3), z)
        o = np.ones((h, w), np.uint8)
        out = oracle.hasf(o, 3)
        assert B.component_counts(out) == B.component_counts(o)
    # an isolated pixel is not simple, so noise points survive as points
    X = np.zeros((9, 9), np.uint8)
    X[4, 4] = 1
    np.testing.assert_array_equal(oracle.hasf(X, 2), X)


def test_rmax_zero_is_identity():
    X = synth.shapes_image(3, 30, 20, 3, 3, 8)
    np.testing.assert_array_equal(oracle.hasf(X, 0), X)


# ---- run to stability (the unbounded radius of Table 1, read as "until a step
# changes nothing") ----------------------------------------------------------

def test_stable_stops_at_once_on_an_open_and_closed_image():
    """Separated large discs left unchanged by the opening and the closing by
    B_1 are a fixed point of step 1, so the run stops there with X itself."""
    used = 0
    for seed in range(12):
        rng = synth.SplitMix64(seed + 4000)
        X = np.zeros((96, 96), np.uint8)
        for cx, cy in [(24, 24), (72, 24), (24, 72), (72, 72)]:
            rad = rng.randint(9, 16)
            synth._paint_ellipse(X, cx + rng.randint(-3, 3), cy + rng.randint(-3, 3),
                                 rad, rad, 1, 0, 1)
        if not ((B.opening(X, 1) == X).all() and (B.closing(X, 1) == X).all()):
            continue
        used += 1
        out, r = oracle.hasf_stable(X, 64)
        assert r == 1
        np.testing.assert_array_equal(out, X)
    assert used >= 3


@pytest.mark.parametrize("conn", [8, 4])
def test_stable_stops_at_the_first_step_that_changes_nothing(conn):
    """The run's radius r is the first one whose step leaves the image as it
    was: HASF_r(X) = HASF_{r-1}(X) and HASF_s(X) != HASF_{s-1}(X) for s < r;
    the output is HASF_r(X)."""
    seen = 0
    for seed in range(6):
        X = synth.shapes_image(seed + 900, 56, 48, 4, 4, 12, n_holes=2, hole_lo=2, hole_hi=4,
                               jitter=1, noise_permille=40)
        C = synth.constraint_points(seed, X, 6)
        out, r = oracle.hasf_stable(X, 16, C=C, conn=conn)
        assert r >= 1
        seen += r > 1
        prev = (X != 0).astype(np.uint8)
        for s in range(1, r + 1):
            cur = oracle.hasf(X, s, C=C, conn=conn)
            assert (s == r) == bool((cur == prev).all()), f"seed {seed} step {s}"
            prev = cur
        np.testing.assert_array_equal(out, prev)
    assert seen >= 3


def test_stable_reports_the_cap():
    """A run capped before its fixed point returns 0 and HASF_cap(X)."""
    X = synth.shapes_image(931, 56, 48, 4, 4, 12, n_holes=2, hole_lo=2, hole_hi=4, jitter=1,
                           noise_permille=40)
    out_full, r = oracle.hasf_stable(X, 16)
    assert r >= 2
    out, r1 = oracle.hasf_stable(X, r - 1)
    assert r1 == 0
    np.testing.assert_array_equal(out, oracle.hasf(X, r - 1))
