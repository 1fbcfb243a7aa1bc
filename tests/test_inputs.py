"""The seeded workload generator: shapes, determinism and the input recipe."""
import numpy as np

from paper_2403_06931_gb300 import inputs


def test_deterministic_and_seed_sensitive():
    a = inputs.tiny(seed=5)
    b = inputs.tiny(seed=5)
    c = inputs.tiny(seed=6)
    assert np.array_equal(a.ref, b.ref) and np.array_equal(a.queries, b.queries)
    assert not np.array_equal(a.ref, c.ref)


def test_znorm_population_statistics():
    rng = inputs.rng_for(1)
    z = inputs.znorm(3.0 + 2.0 * rng.standard_normal(1001))
    assert abs(z.mean()) < 1e-12
    assert abs(np.sqrt(np.mean(z * z)) - 1.0) < 1e-12
    assert np.array_equal(inputs.znorm(np.full(7, 4.0)), np.zeros(7))


def test_quantize_i8_rounding_and_clamp():
    z = np.array([0.0, 0.0625, 0.1875, -0.0625, 100.0, -100.0, 1.0])
    assert inputs.quantize_i8(z).tolist() == [0, 0, 2, 0, 127, -127, 8]


def test_shapes_of_the_named_workloads():
    s = inputs.small_fp32()
    assert s.queries.shape == (8, 128) and s.ref.shape == (4096,) and s.ref.dtype == np.float32
    assert (s.planted >= 0).all() and s.cells == 8 * 128 * 4096
    g = inputs.grad_subset()
    assert g.queries.shape == (8, 64) and g.ref.shape == (512,)
    r = inputs.ragged_fp32(B=50, M=20_000)
    assert r.offsets[0] == 0 and r.offsets[-1] == r.queries.shape[0]
    assert r.lengths.min() >= 200 and r.lengths.max() <= 4000
    assert np.array_equal(np.diff(r.offsets), r.lengths)
    p = inputs.paper_fp32(B=20, N=100, M=5000)
    assert (p.planted < 0).sum() == 2
    q = inputs.paper_i8(B=20, N=100, M=5000)
    assert q.ref.dtype == np.int8 and q.queries.dtype == np.int8
    assert q.queries.min() >= -127


def test_planted_queries_follow_the_recipe():
    """Cuts are ref[o:o+n] + N(0, 0.1^2), then z-normalised on their own."""
    w = inputs.paper_fp32(B=10, N=100, M=3000)
    planted = w.planted >= 0
    assert planted.sum() == 9
    for q in range(w.B):
        x = w.query(q).astype(np.float64)
        assert abs(x.mean()) < 1e-5 and abs(x.std() - 1.0) < 1e-5
    # a planted query is an affine image of its cut up to the noise: its
    # correlation with the cut is high, a decoy's is not
    for q in np.nonzero(planted)[0]:
        cut = w.ref[w.planted[q]:w.planted[q] + 100].astype(np.float64)
        r = np.corrcoef(cut, w.query(q))[0, 1]
        assert r > 0.5
