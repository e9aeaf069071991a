"""Pins of the oracle's tagging (connected components), near-contact test
(Steps 1 and 3) and recolouring (Step 4) against brute force, the paper's
worked example (figure fig:criterion) and the method's invariants."""
import itertools
import json
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def neighbours(shape, conn):
    nz, ny, nx = shape
    offs = [o for o in itertools.product((-1, 0, 1), repeat=3) if any(o)]
    if conn == 6:
        offs = [o for o in offs if sum(map(abs, o)) == 1]
    return offs


def brute_components(mask, conn):
    """Canonical labels by reachability closure of the periodic adjacency
    matrix, numbered by each component's smallest linear index."""
    shape = mask.shape
    nz, ny, nx = shape
    N = mask.size
    A = np.eye(N, dtype=bool)
    flat = mask.ravel()
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        x = (k * ny + j) * nx + i
        if not flat[x]:
            continue
        for dk, dj, di in neighbours(shape, conn):
            y = (((k + dk) % nz) * ny + (j + dj) % ny) * nx + (i + di) % nx
            if flat[y]:
                A[x, y] = A[y, x] = True
    R = A.copy()
    while True:
        R2 = (R.astype(np.int32) @ R.astype(np.int32)) > 0
        if np.array_equal(R2, R):
            break
        R = R2
    lab = np.zeros(N, dtype=np.int32)
    n = 0
    for x in range(N):
        if flat[x] and lab[x] == 0:
            n += 1
            lab[R[x] & flat] = n
    return lab.reshape(shape), n


@pytest.mark.parametrize("conn", [6, 26])
def test_label_brute_force(oracle, conn):
    rng = np.random.default_rng(21 + conn)
    for t in range(12):
        shape = tuple(int(v) for v in rng.integers(2, 7, size=3))
        c = rng.random(shape) * (rng.random(shape) < rng.uniform(0.2, 0.6))
        lab, n = oracle.label(c, 0.0, conn)
        want, nw = brute_components(c > 0, conn)
        assert n == nw
        assert np.array_equal(lab, want)


def test_label_wraps_periodic(oracle):
    c = np.zeros((6, 6, 6))
    c[2, 2, 0] = c[2, 2, 5] = 1.0   # neighbours through the x wrap
    c[0, 4, 4] = c[5, 4, 4] = 0.3   # neighbours through the z wrap
    lab, n = oracle.label(c)
    assert n == 2
    assert lab[0, 4, 4] == lab[5, 4, 4] == 1
    assert lab[2, 2, 0] == lab[2, 2, 5] == 2


def brute_near_contact_map(c, w, tau):
    nz, ny, nx = c.shape
    out = np.zeros(c.shape, dtype=np.uint8)
    for k, j, i in itertools.product(range(nz), range(ny), range(nx)):
        if c[k, j, i] > tau:
            continue
        for d in itertools.product(range(-w, w + 1), repeat=3):
            if not any(d):
                continue
            a = c[(k + d[0]) % nz, (j + d[1]) % ny, (i + d[2]) % nx]
            b = c[(k - d[0]) % nz, (j - d[1]) % ny, (i - d[2]) % nx]
            if a > tau and b > tau:
                out[k, j, i] = 1
                break
    return out


def test_near_contact_brute_force(oracle):
    rng = np.random.default_rng(31)
    for t in range(6):
        shape = tuple(int(v) for v in rng.integers(3, 9, size=3))
        c = rng.random(shape) * (rng.random(shape) < 0.15)
        for w in (1, 2):
            assert np.array_equal(oracle.near_contact_map(c, w), brute_near_contact_map(c, w, 0.0))


def load_criterion_panel(name, margin=5):
    meta = json.load(open(os.path.join(GOLDEN, "criterion.json")))[name]
    rows = open(os.path.join(GOLDEN, meta["grid"])).read().split()
    nrows, ncols = len(rows), len(rows[0])
    ci = np.zeros((1, nrows + 2 * margin, ncols + 2 * margin))
    cj = np.zeros_like(ci)
    for r, line in enumerate(rows):
        for col, ch in enumerate(line):
            if ch == "i":
                ci[0, r + margin, col + margin] = 1.0
            elif ch == "j":
                cj[0, r + margin, col + margin] = 1.0
    centre = (0, meta["centre_row"] + margin, meta["centre_col"] + margin)
    return meta, ci, cj, centre


@pytest.mark.parametrize("panel", ["left", "right"])
def test_worked_example_criterion(oracle, panel):
    """Figure fig:criterion: left, Steps 1 and 3 hold at the grey centre cell;
    right, Step 1 holds and Step 3 does not."""
    meta, ci, cj, centre = load_criterion_panel(panel)
    cmap = oracle.near_contact_map(ci, 2)
    assert bool(cmap[centre]) == meta["step1"]
    lab, n = oracle.label(ci)
    pairs = oracle.near_pairs(ci, lab, 2)
    assert (len(pairs) > 0) == meta["step3"]
    if panel == "right":
        assert n == 1


def test_worked_example_recolour(oracle):
    """Left panel of fig:criterion: the drop that moves is tag 2, which touches
    field j, so it cannot take field j and a third field is created."""
    meta, ci, cj, centre = load_criterion_panel("left")
    c = np.zeros((3,) + ci.shape)
    c[0] = ci
    c[1] = cj
    c2, na, nm, st, moves = oracle.recolour(c, 2)
    assert st == 0 and nm == 1 and na == 3
    assert moves[0].tolist() == [0, 2, 2]
    lab, _ = oracle.label(ci)
    assert np.array_equal(c2[2] > 0, lab == 2)
    assert np.array_equal(c2[1], c[1])


def cube(c, f, lo, size, val=1.0):
    k, j, i = lo
    c[f, k:k + size, j:j + size, i:i + size] = val


def test_recolour_invariants(oracle):
    rng = np.random.default_rng(41)
    for t in range(4):
        K = 4
        shape = (16, 16, 16)
        c = np.zeros((K,) + shape)
        # drops of random cubes in field 0, some touching-close
        for _ in range(7):
            lo = tuple(int(v) for v in rng.integers(0, 13, size=3))
            cube(c, 0, lo, 3, rng.uniform(0.5, 1.0))
        c[0] *= rng.random(shape) > 0.1
        c2, na, nm, st, moves = oracle.recolour(c, 1)
        total0 = c.sum(axis=0)
        total1 = c2.sum(axis=0)
        np.testing.assert_allclose(total1, total0, atol=1e-15, rtol=0)
        if st == 0:
            for f in range(na):
                lab, _ = oracle.label(c2[f])
                assert len(oracle.near_pairs(c2[f], lab, 2)) == 0
        # per-field volume changes are the moved drops' volumes
        lab0, _ = oracle.label(c[0])
        moved = np.zeros(K)
        for fi, lb, tg in moves:
            v = c[0][lab0 == lb].sum()
            moved[tg] += v
            moved[fi] -= v
        np.testing.assert_allclose(c2.sum(axis=(1, 2, 3)) - c.sum(axis=(1, 2, 3)), moved,
                                   atol=1e-12)


def test_recolour_hand_case(oracle):
    """Three 2-cell cubes in a row with 2-cell gaps: pairs (1,2) and (2,3);
    (1,2) marks tag 2 as moving and (2,3) is then skipped, so only the middle
    cube moves, to field 1."""
    c = np.zeros((3, 6, 6, 16))
    cube(c, 0, (2, 2, 1), 2)
    cube(c, 0, (2, 2, 5), 2)
    cube(c, 0, (2, 2, 9), 2)
    c2, na, nm, st, moves = oracle.recolour(c, 1)
    assert st == 0 and nm == 1 and na == 2
    assert moves[0].tolist() == [0, 2, 1]
    assert c2[1, 2, 2, 5] == 1.0 and c2[0, 2, 2, 5] == 0.0
    assert c2[0, 2, 2, 9] == 1.0


def test_recolour_no_free_field(oracle):
    c = np.zeros((1, 6, 6, 12))
    cube(c, 0, (2, 2, 1), 2)
    cube(c, 0, (2, 2, 5), 2)
    c2, na, nm, st, moves = oracle.recolour(c, 1)
    assert st == -4 and nm == 0 and na == 1
    assert np.array_equal(c2, c)
