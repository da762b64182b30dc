"""Pins of the 3D oracle ((26, 6) adjacency) against definitions it does not
share code with: topological numbers from scipy's component labelling,
global counts of components, cavities and the Euler characteristic, a
brute-force distance map, invariants and a hand-worked thinning."""
from __future__ import annotations

import numpy as np
import pytest
from scipy import ndimage

import oracle

S26 = np.ones((3, 3, 3), bool)
S6 = ndimage.generate_binary_structure(3, 1)


def cube_of(code: int) -> np.ndarray:
    """Code bit (dz+1)*9 + (dy+1)*3 + (dx+1) -> array [dz+1, dy+1, dx+1]."""
    return np.array([(code >> i) & 1 for i in range(27)], bool).reshape(3, 3, 3)


L1 = np.abs(np.indices((3, 3, 3)) - 1).sum(axis=0)
N26 = L1 > 0
N18 = (L1 > 0) & (L1 <= 2)
N6 = L1 == 1


def simple_by_labels(code: int) -> bool:
    c = cube_of(code)
    obj = c & N26
    _, t26 = ndimage.label(obj, S26)
    bg = ~c & N18
    lab, _ = ndimage.label(bg, S6)
    t6 = len(set(lab[N6 & bg].tolist()) - {0})
    return t26 == 1 and t6 == 1


def test_simple3d_equals_topological_numbers():
    """The oracle's test is T26 = 1 and T6 = 1 computed by scipy's labelling,
    on 20,000 random neighbourhoods of every density and a few structured ones."""
    rng = np.random.default_rng(3)
    codes = []
    for dens in (0.1, 0.3, 0.5, 0.7, 0.9):
        bits = rng.random((4000, 27)) < dens
        codes += [int(sum(1 << i for i in range(27) if b[i])) for b in bits]
    codes += [0, (1 << 27) - 1, 1 << 14, ((1 << 27) - 1) & ~(1 << 14)]
    mism = [c for c in codes if oracle.simple3d(c) != simple_by_labels(c)]
    assert not mism, f"{len(mism)} codes differ, e.g. {mism[:3]}"


def euler26(X: np.ndarray) -> int:
    """Euler characteristic of the union of the closed unit cubes of X."""
    P = np.pad(X.astype(bool), 1)
    d, h, w = P.shape
    def cells(axes):
        # a cell of dimension len(axes) spanned along `axes` from a lattice
        # point is in the complex if any voxel sharing it is in X
        sl = []
        acc = None
        shifts = [(0, 1) if a not in axes else (0,) for a in range(3)]
        for oz in shifts[0]:
            for oy in shifts[1]:
                for ox in shifts[2]:
                    v = P[oz:d - 1 + oz, oy:h - 1 + oy, ox:w - 1 + ox]
                    acc = v if acc is None else (acc | v)
        return int(acc.sum())
    V = cells(())
    E = sum(cells((a,)) for a in range(3))
    F = sum(cells(ax) for ax in ((0, 1), (0, 2), (1, 2)))
    C = int(X.astype(bool).sum())
    return V - E + F - C


def counts(X: np.ndarray):
    _, n26 = ndimage.label(X.astype(bool), S26)
    _, n6 = ndimage.label(~np.pad(X.astype(bool), 1), S6)   # the outside frame included
    return n26, n6, euler26(X)


def code_at(X, z, y, x):
    P = np.pad(X.astype(np.uint8), 1)
    c = P[z:z + 3, y:y + 3, x:x + 3].reshape(-1)
    return int(sum(int(c[i]) << i for i in range(27)))


def test_simple_deletion_preserves_topology():
    """Deleting a voxel the oracle calls simple keeps the number of
    26-components of X, of 6-components of its complement and the Euler
    characteristic; deleting an isolated or an interior voxel does not."""
    rng = np.random.default_rng(7)
    checked = 0
    for t in range(25):
        X = (rng.random((5, 5, 6)) < 0.55).astype(np.uint8)
        base = counts(X)
        for z, y, x in zip(*np.nonzero(X)):
            code = code_at(X, z, y, x)
            Y = X.copy()
            Y[z, y, x] = 0
            if oracle.simple3d(code):
                assert counts(Y) == base
                checked += 1
            elif (code & ~(1 << 13)) == 0 or (code | (1 << 13)) == (1 << 27) - 1:
                assert counts(Y) != base
    assert checked > 300


def test_edt3d_equals_brute_force():
    rng = np.random.default_rng(11)
    for t in range(6):
        d, h, w = 5 + t % 3, 6, 7 - t % 2
        F = rng.random((d, h, w)) < 0.15
        for outside in (False, True):
            for r in (1, 2, 3):
                got = oracle.edt3d(F, r, outside)
                Z, Y, Xc = np.indices((d, h, w))
                best = np.full((d, h, w), r * r + 1, np.int64)
                for fz, fy, fx in zip(*np.nonzero(F)):
                    best = np.minimum(best, (Z - fz) ** 2 + (Y - fy) ** 2 + (Xc - fx) ** 2)
                if outside:
                    edge = np.minimum.reduce([Z + 1, d - Z, Y + 1, h - Y, Xc + 1, w - Xc]) ** 2
                    best = np.minimum(best, edge)
                best = np.minimum(best, r * r + 1)
                np.testing.assert_array_equal(got, best)


def balls(seed, d, h, w, n, rlo, rhi, noise):
    rng = np.random.default_rng(seed)
    Z, Y, Xc = np.indices((d, h, w))
    X = np.zeros((d, h, w), np.uint8)
    for _ in range(n):
        cz, cy, cx = rng.integers(0, d), rng.integers(0, h), rng.integers(0, w)
        rr = rng.integers(rlo, rhi + 1)
        X |= ((Z - cz) ** 2 + (Y - cy) ** 2 + (Xc - cx) ** 2 <= rr * rr).astype(np.uint8)
    flip = rng.random((d, h, w)) < noise
    return (X ^ flip).astype(np.uint8)


def test_hasf3d_invariants():
    """HASF keeps the 26-components of X, the 6-components of its complement
    and the Euler characteristic, keeps C and never adds D."""
    for seed in range(3):
        X = balls(seed, 12, 13, 14, 4, 2, 5, 0.04)
        rng = np.random.default_rng(seed + 50)
        C = X & (rng.random(X.shape) < 0.03)
        D = (1 - X) & (rng.random(X.shape) < 0.05)
        out = oracle.hasf3d(X, 2, C=C, D=D)
        assert counts(out) == counts(X)
        assert (out >= C).all()
        assert not (out & D).any()
        assert (out != X).any()


def test_operators3d_are_ultimate():
    """After H(S, K) no voxel of S minus K is simple; after *H(S, K) no voxel
    of K minus S is (at radius r with r^2 above every priority)."""
    X = balls(21, 9, 10, 11, 3, 2, 4, 0.03)
    rng = np.random.default_rng(5)
    K = X & (rng.random(X.shape) < 0.1)
    T = oracle.operator3d(X, K, 9, True)
    assert ((T <= X) & (T >= K)).all()
    for z, y, x in zip(*np.nonzero(T & (1 - K))):
        assert not oracle.simple3d(code_at(T, z, y, x))
    V = np.ones_like(X)
    G = oracle.operator3d(X, V, 9, False)
    assert (G >= X).all()
    for z, y, x in zip(*np.nonzero(V & (1 - G))):
        assert not oracle.simple3d(code_at(G, z, y, x))


def test_ultimate_thinning_of_a_box_is_one_voxel():
    """A solid box (collapsible) thinned with nothing kept ends as one voxel."""
    rng = np.random.default_rng(23)
    for _ in range(4):
        d, h, w = (int(v) for v in rng.integers(2, 7, size=3))
        X = np.zeros((d + 2, h + 2, w + 3), np.uint8)
        X[1:1 + d, 1:1 + h, 1:1 + w] = 1
        T = oracle.operator3d(X, np.zeros_like(X), 6, True)
        assert T.sum() == 1 and (T <= X).all()


def test_hand_worked_thinning_of_a_2x2x2_block():
    """H(block, empty) of the block (0..1)^3: every voxel has priority 1; the
    round visits subfields (x, y, z) parities (0,0,0), (1,0,0), (0,1,0),
    (1,1,0), (0,0,1), (1,0,1), (0,1,1), (1,1,1), one voxel each, and each is
    simple when its turn comes (the rest stays one 26-component whose
    background is one 6-component) except the last, then isolated: the result
    is the voxel (1, 1, 1)."""
    X = np.zeros((3, 3, 3), np.uint8)
    X[:2, :2, :2] = 1
    got = oracle.operator3d(X, np.zeros_like(X), 3, True)
    want = np.zeros_like(X)
    want[1, 1, 1] = 1
    np.testing.assert_array_equal(got, want)


def test_trivial_volumes():
    E = np.zeros((4, 5, 6), np.uint8)
    np.testing.assert_array_equal(oracle.hasf3d(E, 3), E)
    P = E.copy()
    P[2, 2, 3] = 1
    np.testing.assert_array_equal(oracle.hasf3d(P, 3), P)   # an isolated voxel stays


# ---- the composition of the filter: radii ascending, cutting before filling ----

def _ball_offsets(r):
    s = range(-r, r + 1)
    return [(a, b, c) for a in s for b in s for c in s if a * a + b * b + c * c <= r * r]


def _shift3(S, dz, dy, dx):
    """out[z, y, x] = S[z + dz, y + dy, x + dx], background outside the box."""
    d, h, w = S.shape
    out = np.zeros_like(S)
    z0, z1, y0, y1 = max(0, -dz), min(d, d - dz), max(0, -dy), min(h, h - dy)
    x0, x1 = max(0, -dx), min(w, w - dx)
    if z0 < z1 and y0 < y1 and x0 < x1:
        out[z0:z1, y0:y1, x0:x1] = S[z0 + dz:z1 + dz, y0 + dy:y1 + dy, x0 + dx:x1 + dx]
    return out


def _dilate3(S, r):
    """Union of the balls B_r centred on S, kept inside the box."""
    out = np.zeros(S.shape, bool)
    for o in _ball_offsets(r):
        out |= _shift3(S != 0, *o)
    return out


def _erode3(S, r):
    """Voxels whose whole ball B_r lies in S (outside = background)."""
    out = np.ones(S.shape, bool)
    for o in _ball_offsets(r):
        out &= _shift3(S != 0, *o)
    return out


def _trivial3(S):
    """One 26-component, one 6-component of the complement, no tunnel
    (Euler characteristic 1)."""
    return counts(S) == (1, 1, 1)


def _alternating3(X, steps):
    """gamma_r = dilation of the erosion, phi_r = erosion of the dilation cup Y,
    by explicit ball unions, in the given order; None unless every set involved
    is topologically trivial (then the thinning / thickening of each operator
    has nothing to stop it short of its constraint set on these shapes)."""
    Y = X != 0
    for kind, r in steps:
        if kind == "open":
            E = _erode3(Y, r)
            G = _dilate3(E, r)
            if not (_trivial3(Y) and E.any() and _trivial3(E) and _trivial3(G)):
                return None
            Y = G
        else:
            Dl = _dilate3(Y, r)
            Wx = _erode3(Dl, r) | Y
            if not (_trivial3(Y) and _trivial3(Dl) and _trivial3(Wx)):
                return None
            Y = Wx
    return Y.astype(np.uint8)


def _box_shapes(n):
    """A box with 2-4 slabs (width 1-3, length 2-3) on its faces and 1-2
    notches (width 1-2, depth 1-2) cut into them."""
    out = []
    for s in range(n):
        rng = np.random.default_rng(300 + s)
        X = np.zeros((16, 17, 18), np.uint8)
        lo = [int(v) for v in rng.integers(4, 6, size=3)]
        hi = [int(v) for v in rng.integers(11, 13, size=3)]
        X[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = 1
        for val, count in ((1, int(rng.integers(2, 5))), (0, int(rng.integers(1, 3)))):
            for _ in range(count):
                wd = int(rng.integers(1, 4 if val else 3))
                ln = int(rng.integers(2, 4) if val else rng.integers(1, 3))
                ax, side = int(rng.integers(0, 3)), int(rng.integers(0, 2))
                sl = []
                for a in range(3):
                    if a != ax:
                        p = int(rng.integers(lo[a] + 1, hi[a] - wd))
                        sl.append(slice(p, p + wd))
                    elif val:
                        sl.append(slice(lo[a] - ln, lo[a]) if side == 0 else slice(hi[a], hi[a] + ln))
                    else:
                        sl.append(slice(lo[a], lo[a] + ln) if side == 0 else slice(hi[a] - ln, hi[a]))
                X[tuple(sl)] = val
        out.append(X)
    return out


def test_hasf3d_is_the_alternating_filter_on_boxes():
    """HASF_2 = HF_2 o HC_2 o HF_1 o HC_1 (the 2D formula of Sec. 2 carried to
    volumes): on boxes with slabs and notches whose every intermediate set is
    topologically trivial, the filter equals the alternating sequential filter
    phi_2 gamma_2 phi_1 gamma_1 by ball unions; filling first, or radii
    descending, gives other volumes on these shapes."""
    used = swapped_differs = descending_differs = 0
    for X in _box_shapes(24):
        want = _alternating3(X, [("open", 1), ("close", 1), ("open", 2), ("close", 2)])
        if want is None:
            continue
        used += 1
        np.testing.assert_array_equal(oracle.hasf3d(X, 2), want)
        sw = _alternating3(X, [("close", 1), ("open", 1), ("close", 2), ("open", 2)])
        de = _alternating3(X, [("open", 2), ("close", 2), ("open", 1), ("close", 1)])
        swapped_differs += sw is not None and bool((sw != want).any())
        descending_differs += de is not None and bool((de != want).any())
    assert used >= 15 and swapped_differs >= 8 and descending_differs >= 8, \
        (used, swapped_differs, descending_differs)
