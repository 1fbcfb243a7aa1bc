"""Pins for the CPU oracle (oracle/), independent of the oracle's own code.

Each check is something the paper's definition (Section 2, Eq. 1) or plain
mathematics fixes, chosen so that a plausible slip in the oracle -- a dropped
neighbour, a wrong index, a wrong start/end rule, |x-y| instead of (x-y)^2, a
transposed query/reference, a wrong tie order in the walk-back -- fails one:

* brute force: the minimum over every warp path, enumerated explicitly;
* closed forms: N = 1, M = 1, an exact cut of the reference;
* invariants: prefix of the last row, monotone cost as the reference grows,
  common shift, power-of-two scaling, orientation;
* worked examples derived by hand (tests/golden/worked_examples.json);
* FP64 central differences of the cost against the walk-back path gradient.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2403_06931_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


# --------------------------------------------------------------- brute force --

def brute_force_last_row(x, y):
    """Minimum path cost ending at each column of the last row, by enumeration.

    Every warp path starts at some (0, s), moves by (1,0), (0,1) or (1,1), and
    ends at some (n-1, e); each path is generated once and its cost summed
    cell by cell.  No recurrence is used: minima are taken over whole paths.
    """
    n, m = len(x), len(y)
    best = [None] * m

    def extend(i, j, acc):
        acc = acc + (x[i] - y[j]) ** 2
        if i == n - 1 and (best[j] is None or acc < best[j]):
            best[j] = acc
        if i + 1 < n:
            extend(i + 1, j, acc)
        if j + 1 < m:
            extend(i, j + 1, acc)
        if i + 1 < n and j + 1 < m:
            extend(i + 1, j + 1, acc)

    for s in range(m):
        extend(0, s, 0)
    return best


SHAPES = [(n, m) for n in range(1, 6) for m in range(1, 6)] + [(6, 4), (4, 6), (2, 7), (7, 2), (6, 6)]


@pytest.mark.parametrize("n,m", SHAPES)
def test_brute_force_integer_exact(oracle_mod, n, m):
    rng = np.random.default_rng(1000 * n + m)
    for _ in range(3):
        x = [int(v) for v in rng.integers(-4, 5, size=n)]
        y = [int(v) for v in rng.integers(-4, 5, size=m)]
        bf = brute_force_last_row(x, y)
        c64, e64, row64 = oracle_mod.forward(np.array(x, dtype=np.int64), np.array(y, dtype=np.int64), last_row=True)
        cf, ef, rowf = oracle_mod.forward(np.array(x, dtype=np.float64), np.array(y, dtype=np.float64), last_row=True)
        assert list(row64) == bf
        assert [float(v) for v in rowf] == [float(v) for v in bf]
        assert c64 == min(bf) and e64 == bf.index(min(bf))
        assert cf == min(bf) and ef == bf.index(min(bf))


@pytest.mark.parametrize("n,m", [(3, 3), (4, 5), (5, 4), (6, 6)])
def test_brute_force_float(oracle_mod, n, m):
    rng = np.random.default_rng(7 * n + m)
    for _ in range(3):
        x = rng.standard_normal(n)
        y = rng.standard_normal(m)
        bf = brute_force_last_row(list(x), list(y))
        _, _, row = oracle_mod.forward(x, y, last_row=True)
        np.testing.assert_allclose(row, bf, rtol=1e-12, atol=1e-14)


# --------------------------------------------------------------- closed forms --

def test_single_sample_query(oracle_mod):
    rng = np.random.default_rng(3)
    y = rng.standard_normal(257)
    x = np.array([0.37])
    c, e = oracle_mod.forward(x, y)
    d2 = (0.37 - y) ** 2
    assert c == d2.min() and e == int(np.argmin(d2))


def test_single_sample_reference(oracle_mod):
    rng = np.random.default_rng(4)
    x = rng.standard_normal(91)
    y = np.array([-0.2])
    c, e = oracle_mod.forward(x, y)
    assert e == 0
    assert math.isclose(c, float(np.sum((x + 0.2) ** 2)), rel_tol=1e-13)


@pytest.mark.parametrize("o,n", [(0, 50), (123, 200), (700, 300)])
def test_exact_cut_has_zero_cost(oracle_mod, o, n):
    w = inputs.tiny(B=1, N=n, M=1000, seed=11)
    y = w.ref.astype(np.float64)
    x = y[o:o + n].copy()
    c, e, row = oracle_mod.forward(x, y, last_row=True)
    assert c == 0.0
    assert row[o + n - 1] == 0.0
    assert e <= o + n - 1 and row[e] == 0.0


def test_tied_minimum_takes_smallest_end(oracle_mod):
    # x = [1]: last row is (1 - y_j)^2 with exact zeros at j = 2 and j = 5
    y = np.array([3.0, 0.0, 1.0, 2.0, -1.0, 1.0])
    c, e = oracle_mod.forward(np.array([1.0]), y)
    assert c == 0.0 and e == 2
    c, e = oracle_mod.forward(np.array([1], dtype=np.int64), y.astype(np.int64))
    assert c == 0 and e == 2


# ----------------------------------------------------------------- invariants --

def test_last_row_prefix_and_monotone_growth(oracle_mod):
    rng = np.random.default_rng(5)
    x = rng.standard_normal(40)
    y = rng.standard_normal(600)
    _, _, full = oracle_mod.forward(x, y, last_row=True)
    prev = math.inf
    for k in (1, 7, 39, 40, 41, 100, 333, 600):
        c, e, row = oracle_mod.forward(x, y[:k], last_row=True)
        assert np.array_equal(row, full[:k])
        assert c <= prev
        prev = c


def test_common_shift_integer_exact(oracle_mod):
    rng = np.random.default_rng(6)
    x = rng.integers(-50, 50, size=30)
    y = rng.integers(-50, 50, size=200)
    a = oracle_mod.forward(x, y, last_row=True)
    b = oracle_mod.forward(x + 1234, y + 1234, last_row=True)
    assert a[0] == b[0] and a[1] == b[1] and np.array_equal(a[2], b[2])


def test_common_shift_float(oracle_mod):
    rng = np.random.default_rng(7)
    x = rng.standard_normal(30)
    y = rng.standard_normal(200)
    a = oracle_mod.forward(x, y, last_row=True)
    b = oracle_mod.forward(x + 0.75, y + 0.75, last_row=True)
    np.testing.assert_allclose(a[2], b[2], rtol=1e-12)


def test_power_of_two_scaling_is_quadratic(oracle_mod):
    rng = np.random.default_rng(8)
    x = rng.standard_normal(25)
    y = rng.standard_normal(150)
    a = oracle_mod.forward(x, y, last_row=True)
    b = oracle_mod.forward(4.0 * x, 4.0 * y, last_row=True)
    assert b[0] == 16.0 * a[0] and b[1] == a[1]
    assert np.array_equal(b[2], 16.0 * a[2])


def test_orientation_query_vs_reference(oracle_mod):
    # the query must be the rows: a one-sample query matches anywhere in y,
    # while a one-sample reference forces every query sample onto it
    x = np.array([0.0])
    y = np.array([5.0, 0.0, 5.0])
    assert oracle_mod.forward(x, y)[0] == 0.0
    assert oracle_mod.forward(y, x)[0] == 50.0


# ----------------------------------------------------------- worked examples --

def _golden_cases():
    with open(GOLDEN) as f:
        return json.load(f)["cases"]


@pytest.mark.parametrize("case", _golden_cases(), ids=lambda c: c["name"])
def test_worked_examples(oracle_mod, case):
    x = np.array(case["x"], dtype=np.int64)
    y = np.array(case["y"], dtype=np.int64)
    D = np.array(case["D"], dtype=np.int64)
    c, e, row = oracle_mod.forward(x, y, last_row=True)
    assert c == case["cost"] and e == case["end"]
    assert list(row) == list(D[-1])
    cf, ef, rowf = oracle_mod.forward(x.astype(np.float64), y.astype(np.float64), last_row=True)
    assert cf == case["cost"] and ef == case["end"] and list(rowf) == list(D[-1].astype(float))
    # every row of the hand matrix is the last row of the query's prefix
    for i in range(len(x)):
        _, _, r = oracle_mod.forward(x[:i + 1], y, last_row=True)
        assert list(r) == list(D[i])
    cells, margins = oracle_mod.walkback(x, y, case["end"])
    assert cells.tolist() == case["path"]
    assert margins.tolist() == [float(v) for v in case["margins"]]
    assert oracle_mod.path_is_valid(cells, len(x), len(y), case["end"])
    assert oracle_mod.path_cost(x, y, cells) == case["cost"]
    gx, gy = oracle_mod.path_gradient(x, y, cells)
    assert gx.tolist() == [float(v) for v in case["gradient_x"]]
    assert gy.tolist() == [float(v) for v in case["gradient_y"]]


def test_path_helpers_reject_invalid_paths(oracle_mod):
    ok = [[2, 4], [1, 3], [1, 2], [0, 1]]
    assert oracle_mod.path_is_valid(ok, 3, 5, 4)
    assert not oracle_mod.path_is_valid(ok, 3, 5, 3)                       # wrong end
    assert not oracle_mod.path_is_valid([[2, 4], [1, 2], [0, 1]], 3, 5, 4)  # jump of two columns
    assert not oracle_mod.path_is_valid([[2, 4], [1, 3], [1, 2]], 3, 5, 4)  # never reaches row 0
    assert not oracle_mod.path_is_valid([[2, 4], [1, 3], [0, 3], [0, 2]], 3, 5, 4)  # runs on in row 0
    lo, hi = oracle_mod.intervals_from_cells(ok, 3)
    assert lo.tolist() == [1, 2, 4] and hi.tolist() == [1, 3, 4]
    assert oracle_mod.cells_from_intervals(lo, hi).tolist() == ok


def test_walkback_path_cost_equals_min_cost(oracle_mod):
    w = inputs.tiny(B=6, N=40, M=500, seed=21)
    for q in range(w.B):
        x = w.query(q).astype(np.float64)
        y = w.ref.astype(np.float64)
        c, e = oracle_mod.forward(x, y)
        cells, _ = oracle_mod.walkback(x, y, e)
        assert oracle_mod.path_is_valid(cells, len(x), len(y), e)
        assert math.isclose(oracle_mod.path_cost(x, y, cells), c, rel_tol=1e-12)


# ------------------------------------------------------ finite differences --

def _stable_fd(oracle_mod, x, y, which, k, h, cells):
    """Central difference of the cost in x[k] (or y[k]); None if the walk-back
    path changes at either perturbed point (the cost is then not one quadratic
    piece over [-h, h] and the difference is not a derivative)."""
    out = []
    for s in (+1.0, -1.0):
        xp, yp = x.copy(), y.copy()
        (xp if which == "x" else yp)[k] += s * h
        c, e = oracle_mod.forward(xp, yp)
        cp, _ = oracle_mod.walkback(xp, yp, e)
        if cp.shape != cells.shape or not np.array_equal(cp, cells):
            return None
        out.append(c)
    return (out[0] - out[1]) / (2.0 * h)


def test_gradient_matches_central_differences(oracle_mod):
    """8 x 64 vs 512 subset, h = 1e-4, elements where the path is stable."""
    w = inputs.grad_subset()
    y = w.ref.astype(np.float64)
    h = 1e-4
    rng = np.random.default_rng(9)
    checked = skipped = 0
    for q in range(w.B):
        x = w.query(q).astype(np.float64)
        c, e = oracle_mod.forward(x, y)
        cells, _ = oracle_mod.walkback(x, y, e)
        gx, gy = oracle_mod.path_gradient(x, y, cells, g=1.0)
        scale = max(np.abs(gx).max(), np.abs(gy).max(), 1e-12)
        on_path = np.unique(cells[:, 1])
        off_path = np.setdiff1d(np.arange(len(y)), on_path)
        ys = np.concatenate([on_path, rng.choice(off_path, size=min(16, len(off_path)), replace=False)])
        for which, ks in (("x", range(len(x))), ("y", ys)):
            for k in ks:
                fd = _stable_fd(oracle_mod, x, y, which, int(k), h, cells)
                if fd is None:
                    skipped += 1
                    continue
                an = (gx if which == "x" else gy)[int(k)]
                assert abs(fd - an) <= 1e-6 * scale + 1e-8, (q, which, k, fd, an)
                checked += 1
    assert checked > 10 * skipped and checked > 500


# --------------------------------------------------------------- integer mode --

def test_int_and_double_oracles_agree_on_int8_codes(oracle_mod):
    w = inputs.paper_i8(B=6, N=60, M=1500)
    c_i, e_i = oracle_mod.forward_batch(w.ref, w.queries)
    c_f, e_f = oracle_mod.forward_batch(w.ref.astype(np.float64), w.queries.astype(np.float64))
    assert c_i.dtype == np.int64
    assert np.array_equal(c_i.astype(np.float64), c_f) and np.array_equal(e_i, e_f)


def test_batch_driver_matches_single_calls(oracle_mod):
    w = inputs.ragged_fp32(B=5, n_lo=3, n_hi=40, M=300)
    costs, ends = oracle_mod.forward_batch(w.ref, w.queries, offsets=w.offsets, threads=3)
    for q in range(w.B):
        c, e = oracle_mod.forward(w.query(q), w.ref)
        assert costs[q] == c and ends[q] == e


def test_oracle_rejects_bad_sizes(oracle_mod):
    with pytest.raises(ValueError):
        oracle_mod.forward(np.zeros(0), np.zeros(4))
    with pytest.raises(ValueError):
        oracle_mod.walkback(np.zeros(3), np.zeros(4), 4)


# ------------------------------------------------------- interval form --

def test_interval_helpers_agree_with_cell_helpers(oracle_mod):
    w = inputs.tiny(B=5, N=30, M=400, seed=31)
    y = w.ref.astype(np.float64)
    for q in range(w.B):
        x = w.query(q).astype(np.float64)
        c, e = oracle_mod.forward(x, y)
        cells, _ = oracle_mod.walkback(x, y, e)
        lo, hi = oracle_mod.intervals_from_cells(cells, len(x))
        assert oracle_mod.intervals_are_valid(lo, hi, len(y), e)
        assert math.isclose(oracle_mod.intervals_cost(x, y, lo, hi), oracle_mod.path_cost(x, y, cells),
                            rel_tol=1e-11)
        gx, gy = oracle_mod.intervals_gradient(x, y, lo, hi, g=0.7)
        hx, hy = oracle_mod.path_gradient(x, y, cells, g=0.7)
        np.testing.assert_allclose(gx, hx, rtol=1e-10, atol=1e-10)
        np.testing.assert_allclose(gy, hy, rtol=1e-10, atol=1e-10)


def test_interval_validity_rejects_bad_runs(oracle_mod):
    assert oracle_mod.intervals_are_valid([1, 2, 4], [1, 3, 4], 5, 4)
    assert not oracle_mod.intervals_are_valid([1, 2, 4], [1, 3, 4], 5, 3)   # wrong end
    assert not oracle_mod.intervals_are_valid([1, 3, 4], [1, 3, 4], 5, 4)   # jump of two columns
    assert oracle_mod.intervals_are_valid([1, 2, 3], [1, 3, 4], 5, 4)       # up step from (2,3) to (1,3)
    assert not oracle_mod.intervals_are_valid([1, 2, 2], [1, 3, 4], 5, 4)   # run overlaps previous row
    assert not oracle_mod.intervals_are_valid([1, 2, 4], [1, 1, 4], 5, 4)   # lo > hi
    assert not oracle_mod.intervals_are_valid([1, 2, 4], [1, 3, 5], 5, 5)   # outside the matrix


# --------------------------------------------------- z-normalisation (Eq. 2) --

def test_znorm_textbook_example(oracle_mod):
    # the classic population example: mean 5, population standard deviation 2
    z = oracle_mod.znormalize([2, 4, 4, 4, 5, 5, 7, 9])
    assert np.array_equal(z, [-1.5, -0.5, -0.5, -0.5, 0.0, 0.0, 1.0, 2.0])
    z3 = oracle_mod.znormalize([1, 2, 3])
    s = np.sqrt(2.0 / 3.0)                       # population, not the sample sqrt(1)
    assert np.allclose(z3, [-1 / s, 0.0, 1 / s], rtol=0, atol=1e-15)


def test_znorm_moments_and_library(oracle_mod):
    x = np.random.default_rng(3).standard_normal(1000) * 3.0 + 1.5
    z = oracle_mod.znormalize(x)
    assert abs(z.mean()) < 1e-12 and abs(np.mean(z * z) - 1.0) < 1e-12
    assert np.allclose(z, (x - x.mean()) / x.std(ddof=0), rtol=1e-13, atol=1e-13)


def test_znorm_affine_invariance(oracle_mod):
    x = np.random.default_rng(4).standard_normal(257)
    z = oracle_mod.znormalize(x)
    assert np.allclose(oracle_mod.znormalize(3.0 * x + 7.0), z, rtol=0, atol=1e-12)
    assert np.allclose(oracle_mod.znormalize(-2.0 * x + 1.0), -z, rtol=0, atol=1e-12)


def test_znorm_degenerate_series(oracle_mod):
    assert np.array_equal(oracle_mod.znormalize([4.25] * 9), np.zeros(9))   # zero spread: centred only
    assert np.array_equal(oracle_mod.znormalize([-3.0]), [0.0])
    assert oracle_mod.znormalize(np.zeros(0)).size == 0


def test_znorm_is_two_pass(oracle_mod):
    # a large common offset: the centred second moment keeps the digits that
    # a one-pass E[x^2] - E[x]^2 would cancel away
    noise = np.random.default_rng(5).standard_normal(4000)
    z = oracle_mod.znormalize(1e9 + noise)
    assert np.allclose(z, oracle_mod.znormalize(noise), rtol=0, atol=1e-6)


def test_znorm_batch_layouts(oracle_mod):
    v = np.random.default_rng(6).standard_normal(30)
    u = oracle_mod.znormalize_batch(v, N=10)
    assert np.array_equal(u[10:20], oracle_mod.znormalize(v[10:20]))
    offs = np.array([0, 3, 3, 17, 30])
    r = oracle_mod.znormalize_batch(v, offsets=offs)
    assert np.array_equal(r[3:17], oracle_mod.znormalize(v[3:17])) and np.array_equal(r[17:], oracle_mod.znormalize(v[17:]))


# ------------------------------------------- derivative of the normalisation --

def _central(f, x, k, h):
    xp, xm = x.copy(), x.copy()
    xp[k] += h
    xm[k] -= h
    return (f(xp) - f(xm)) / (2.0 * h)


def test_znorm_vjp_matches_central_differences_of_a_smooth_loss(oracle_mod):
    """d/dx of L(znorm(x)) for a smooth L (a weighted sum plus half the
    squares, so dL/dz = w + z), against FP64 central differences."""
    rng = np.random.default_rng(21)
    for n in (2, 5, 37, 400):
        x = rng.standard_normal(n) * 3.0 + 7.0
        w = rng.standard_normal(n)
        loss = lambda v: float(np.dot(w, oracle_mod.znormalize(v)) + 0.5 * np.sum(oracle_mod.znormalize(v) ** 2))  # noqa: E731
        gx = oracle_mod.znormalize_vjp(x, w + oracle_mod.znormalize(x))
        for k in range(min(n, 12)):
            fd = _central(loss, x, k, 1e-5)
            assert abs(fd - gx[k]) <= 1e-6 * max(1.0, np.abs(gx).max()), (n, k, fd, gx[k])


def test_znorm_vjp_invariants(oracle_mod):
    """Eq. 2 is invariant to a shift and a positive scale of x, so its
    derivative is orthogonal to the all-ones vector and to x itself; a
    gradient along z or along ones has no effect (z is normalised)."""
    rng = np.random.default_rng(22)
    x = rng.standard_normal(50) * 2.0 - 1.0
    g = rng.standard_normal(50)
    gx = oracle_mod.znormalize_vjp(x, g)
    assert abs(gx.sum()) <= 1e-12 * np.abs(gx).max() * 50
    assert abs(np.dot(gx, x)) <= 1e-11 * np.abs(gx).max() * np.abs(x).sum()
    z = oracle_mod.znormalize(x)
    assert np.abs(oracle_mod.znormalize_vjp(x, z)).max() <= 1e-12
    assert np.abs(oracle_mod.znormalize_vjp(x, np.ones(50))).max() <= 1e-12
    # zero spread: only centred, so the derivative removes the mean
    c = np.full(8, 3.5)
    assert np.allclose(oracle_mod.znormalize_vjp(c, np.arange(8.0)), np.arange(8.0) - 3.5, atol=1e-15)


def test_cost_of_normalised_query_gradient_matches_central_differences(oracle_mod):
    """The path gradient with respect to z = znorm(x), carried to x by the
    normalisation's derivative, against central differences of
    cost(ref, znorm(x)) where the path is stable."""
    w = inputs.grad_subset()
    y = w.ref.astype(np.float64)
    h = 1e-6
    checked = 0
    for q in range(3):
        x = w.query(q).astype(np.float64) * 1.7 + 0.3   # raw, not normalised
        z = oracle_mod.znormalize(x)
        c, e = oracle_mod.forward(z, y)
        cells, _ = oracle_mod.walkback(z, y, e)
        gz, _ = oracle_mod.path_gradient(z, y, cells, g=1.0)
        gx = oracle_mod.znormalize_vjp(x, gz)

        def cost_on_path(v):
            zz = oracle_mod.znormalize(v)
            cc, ee = oracle_mod.forward(zz, y)
            cp, _ = oracle_mod.walkback(zz, y, ee)
            return cc if cp.shape == cells.shape and np.array_equal(cp, cells) else None

        for k in range(0, len(x), 4):
            xp, xm = x.copy(), x.copy()
            xp[k] += h
            xm[k] -= h
            fp, fm = cost_on_path(xp), cost_on_path(xm)
            if fp is None or fm is None:
                continue
            fd = (fp - fm) / (2.0 * h)
            assert abs(fd - gx[k]) <= 1e-5 * max(1.0, np.abs(gx).max()), (q, k, fd, gx[k])
            checked += 1
    assert checked >= 24


# ---------------------------------------------------------------------------
# Reference codebook (Section 8): the fit in FP64, the encoding decided in
# float32, then the exact integer DP on the codes.

def test_codebook_fit_closed_forms(oracle_mod):
    y = np.tile([-1.0, 1.0], 500)                  # mean 0, population spread 1
    lo, step = oracle_mod.codebook_fit(y, sigmas=4.0)
    assert lo == -4.0 and step == 8.0 / 256.0
    lo3, step3 = oracle_mod.codebook_fit(y, sigmas=3.0)
    assert lo3 == -3.0 and step3 == 6.0 / 256.0
    # a constant reference: the constant lands at code 128 with unit steps
    assert oracle_mod.codebook_fit(np.full(7, 2.5)) == (2.5 - 128.0, 1.0)
    # population, not sample, spread: [0, 2] has S = 1
    assert oracle_mod.codebook_fit(np.array([0.0, 2.0]), sigmas=1.0) == (0.0, 2.0 / 256.0)


def test_codebook_fit_is_affine_equivariant(oracle_mod):
    y = np.cumsum(np.random.default_rng(3).standard_normal(5000))
    lo, step = oracle_mod.codebook_fit(y)
    lo2, step2 = oracle_mod.codebook_fit(4.0 * y - 7.0)
    assert abs(lo2 - (4.0 * lo - 7.0)) <= 1e-9 * abs(lo2) and abs(step2 - 4.0 * step) <= 1e-12 * step2


def test_codebook_encode_bins_and_clamps(oracle_mod):
    lo, inv = -4.0, 32.0                            # step 1/32: bin edges exact in float32
    k = np.arange(256)
    edges = (lo + k / 32.0).astype(np.float32)      # a bin's lower edge belongs to it
    centres = (lo + (k + 0.5) / 32.0).astype(np.float32)
    assert np.array_equal(oracle_mod.codebook_encode(edges, lo, inv), k)
    assert np.array_equal(oracle_mod.codebook_encode(centres, lo, inv), k)
    below = np.array([-4.0001, -10.0, -1e30], dtype=np.float32)
    above = np.array([4.0, 4.5, 1e30], dtype=np.float32)
    assert (oracle_mod.codebook_encode(below, lo, inv) == 0).all()
    assert (oracle_mod.codebook_encode(above, lo, inv) == 255).all()
    # monotone, and equal to the exact floor away from bin edges
    x = np.sort(np.random.default_rng(4).uniform(-5.0, 5.0, 20000).astype(np.float32))
    c = oracle_mod.codebook_encode(x, lo, inv)
    assert (np.diff(c.astype(np.int64)) >= 0).all()
    exact = np.clip(np.floor((x.astype(np.float64) - lo) * inv), 0, 255)
    far = np.abs((x.astype(np.float64) - lo) * inv - np.round((x.astype(np.float64) - lo) * inv)) > 1e-3
    assert np.array_equal(c[far], exact[far].astype(np.uint8))


def test_codebook_encode_decides_in_float32(oracle_mod):
    # (x - lo) rounds to float32 before the product: a value just below a bin
    # edge whose difference rounds up onto the edge takes the upper bin, as the
    # library's float32 arithmetic does
    lo, inv = np.float32(-3.0), np.float32(64.0)
    x = np.nextafter(np.float32(1.0), np.float32(0.0))       # 1 - 2^-24
    assert np.float32(x - lo) == np.float32(4.0)             # 4 - 2^-24 rounds to 4
    assert oracle_mod.codebook_encode(np.array([x]), lo, inv)[0] == 255   # floor(256) clamped
    x2 = np.float32(0.5) - np.float32(2.0 ** -25)            # exact: 0.5 - 2^-25
    assert np.float32(x2 - lo) == np.float32(3.5)            # 3.5 - 2^-25 rounds to 3.5
    # exact arithmetic would give floor(224 - 2^-19) = 223
    assert oracle_mod.codebook_encode(np.array([x2], np.float32), lo, inv)[0] == 224


def test_codebook_pipeline_exact_cut(oracle_mod):
    # codes of an exact cut of the reference are the cut of the codes: cost 0 at its end
    y = inputs.znorm(np.cumsum(np.random.default_rng(5).standard_normal(3000))).astype(np.float32)
    lo, step = oracle_mod.codebook_fit(y)
    lo32, inv32 = np.float32(lo), np.float32(1.0 / step)
    cy = oracle_mod.codebook_encode(y, lo32, inv32).astype(np.int64)
    cx = oracle_mod.codebook_encode(y[1200:1500], lo32, inv32).astype(np.int64)
    c, e = oracle_mod.forward(cx, cy)
    assert c == 0 and e <= 1499 and cy[e] == cx[-1]


# ---------------------------------------------------------------------------
# The paper's binary16 precision (Section 5.2): rounding routines pinned
# against numpy's float16 conversion and exact rational arithmetic; the
# binary16 DP against the int64 DP where every value is exact in binary16.

def test_round_f16_matches_numpy_float16(oracle_mod):
    rng = np.random.default_rng(21)
    v = rng.standard_normal(200_000) * np.exp(rng.uniform(-22, 12, 200_000))
    # exact midpoints between neighbouring binary16 values, both parities
    h = np.float16(rng.standard_normal(5000) * 100)
    nxt = np.nextafter(h, np.float16(np.inf))
    mids = (h.astype(np.float64) + nxt.astype(np.float64)) / 2
    special = np.array([65504.0, 65519.99, 65520.0, -65520.0, 2.0 ** -24, 2.0 ** -25, 3 * 2.0 ** -26, 0.0, -0.0])
    for arr in (v, mids, special):
        with np.errstate(over="ignore"):
            want = arr.astype(np.float16).astype(np.float64)
        got = oracle_mod.round_f16(arr)
        assert np.array_equal(got, want) and np.array_equal(np.signbit(got), np.signbit(want))


def _f16_nearest(fr):
    """The binary16 value nearest to the Fraction fr (ties to even), by exact
    comparison with the two neighbours that bracket it."""
    from fractions import Fraction
    lo = np.float16(float(fr))
    if Fraction(float(lo)) > fr:
        lo = np.nextafter(lo, np.float16(-np.inf))
    hi = np.nextafter(lo, np.float16(np.inf))
    dl, dh = fr - Fraction(float(lo)), Fraction(float(hi)) - fr
    if dl < dh:
        return float(lo)
    if dh < dl:
        return float(hi)
    return float(lo) if (lo.view(np.uint16) & 1) == 0 else float(hi)


def test_fma_f16_is_correctly_rounded(oracle_mod):
    from fractions import Fraction
    rng = np.random.default_rng(22)
    a = np.float16(rng.standard_normal(3000) * 30)
    c = np.float16(rng.standard_normal(3000) * 1000)
    c[:500] = np.float16(rng.standard_normal(500) * 1e-3)         # small addends
    # products that land exactly on midpoints once an addend is added
    a[500:800] = np.float16(rng.integers(1, 64, 300) * 0.5)
    c[500:800] = np.float16(0.25)
    got = oracle_mod.fma_f16(a, a, c)
    for k in range(len(a)):
        exact = Fraction(float(a[k])) * Fraction(float(a[k])) + Fraction(float(c[k]))
        assert got[k] == _f16_nearest(exact), (a[k], c[k], got[k])


def test_f16_dp_equals_int_dp_when_exact(oracle_mod):
    # small integer samples: every local cost and every D stays an integer
    # below 2048, exact in binary16, so the binary16 DP is the exact DP
    rng = np.random.default_rng(23)
    for _ in range(20):
        n, m = int(rng.integers(1, 12)), int(rng.integers(1, 40))
        x = rng.integers(-3, 4, n)
        y = rng.integers(-3, 4, m)
        c16, e16, row16 = oracle_mod.forward_f16(x.astype(np.float16), y.astype(np.float16), last_row=True)
        ci, ei = oracle_mod.forward(x.astype(np.int64), y.astype(np.int64))
        assert c16 == ci and e16 == ei and np.all(row16 < 2048)


def test_f16_dp_rounds_every_operation(oracle_mod):
    # one row and one column: D = fl16(d * d) with d = fl16(x - y); a case
    # where the subtraction itself rounds (1000 - 0.3 is not a binary16 value)
    x = np.array([1000.0], dtype=np.float16)
    y = np.array([0.3], dtype=np.float16)
    d = oracle_mod.round_f16(1000.0 - float(y[0]))
    c, e = oracle_mod.forward_f16(x, y)
    assert d != 1000.0 - float(y[0]) and c == oracle_mod.round_f16(d * d)[()] and e == 0
    # large costs overflow to +inf, as binary16 does
    c, e = oracle_mod.forward_f16(np.array([200.0] * 3, np.float16), np.array([-60.0], np.float16))
    assert c == np.inf and e == 0


def test_f16_dp_close_to_f64_on_paper_shaped_inputs(oracle_mod):
    # the binary16 cost of a z-normalised query against a z-normalised
    # reference stays within a few binary16 units of the FP64 cost of the
    # same (binary16) samples: each cell adds at most half a unit at its scale
    w = inputs.tiny(B=4, N=64, M=900, seed=24)
    for q in range(w.B):
        x = w.query(q).astype(np.float16)
        y = w.ref.astype(np.float16)
        c16, _ = oracle_mod.forward_f16(x, y)
        c64, _ = oracle_mod.forward(x.astype(np.float64), y.astype(np.float64))
        assert abs(c16 - c64) <= 64 * 2.0 ** -11 * max(c64, 1.0) * 2
    with pytest.raises(ValueError):
        oracle_mod.forward_f16(np.array([0.1]), np.array([0.2]))        # not binary16 values


# ---------------------------------------------------------------------------
# Early-INF pruning (Section 8): a cell whose samples differ by more than the
# gap costs +inf.  Pinned by brute force over whole paths (a path through a
# pruned cell costs +inf), the gap that prunes nothing, and monotonicity.

def brute_force_pruned(x, y, gap):
    """Minimum over whole warp paths of the path cost, +inf for a path that
    crosses a cell whose samples differ by more than gap (no recurrence)."""
    n, m = len(x), len(y)
    best = [math.inf] * m

    def extend(i, j, acc):
        if abs(x[i] - y[j]) > gap:
            return                                   # this path costs +inf
        acc = acc + (x[i] - y[j]) ** 2
        if i == n - 1 and acc < best[j]:
            best[j] = acc
        if i + 1 < n:
            extend(i + 1, j, acc)
        if j + 1 < m:
            extend(i, j + 1, acc)
        if i + 1 < n and j + 1 < m:
            extend(i + 1, j + 1, acc)

    for s in range(m):
        extend(0, s, 0)
    return best


@pytest.mark.parametrize("n,m", [(1, 4), (3, 3), (4, 5), (5, 4), (6, 6), (2, 7), (7, 2)])
def test_pruned_dp_equals_brute_force(oracle_mod, n, m):
    rng = np.random.default_rng(55 + 10 * n + m)
    for gap in (0, 1, 2, 3, 5, 100):
        for _ in range(3):
            x = [int(v) for v in rng.integers(-4, 5, size=n)]
            y = [int(v) for v in rng.integers(-4, 5, size=m)]
            bf = brute_force_pruned(x, y, gap)
            c, e = oracle_mod.forward_pruned(np.array(x), np.array(y), gap)
            if math.isinf(min(bf)):
                assert c == oracle_mod.PRUNED_INF and e == -1
            else:
                assert c == min(bf) and e == bf.index(min(bf))


def test_pruning_that_prunes_nothing_is_the_plain_dp(oracle_mod):
    w = inputs.paper_i8(B=3, N=60, M=700, seed=56)
    for q in range(w.B):
        x, y = w.query(q).astype(np.int64), w.ref.astype(np.int64)
        gap = int(np.abs(x[:, None] - y[None, :]).max())
        assert oracle_mod.forward_pruned(x, y, gap) == oracle_mod.forward(x, y)


def test_pruned_cost_never_falls_as_the_gap_shrinks(oracle_mod):
    w = inputs.paper_i8(B=2, N=80, M=900, seed=57)
    for q in range(w.B):
        x, y = w.query(q).astype(np.int64), w.ref.astype(np.int64)
        costs = [oracle_mod.forward_pruned(x, y, g)[0] for g in (200, 40, 20, 10, 5, 2, 0)]
        assert all(a <= b for a, b in zip(costs, costs[1:]))
