"""The seeded input recipes (the synthetic stand-ins for the paper's random
coefficient fields, Sec. 4): shapes, ranges, distributions and determinism,
as the generators' docstrings state them."""
import numpy as np

import workloads as W


def test_pixel_layout_and_seeding():
    assert W.pixel_shape((7, 5)) == (6, 8)
    assert W.pixel_shape((3, 4, 5)) == (6, 5, 4)
    a1 = W.log_uniform_pixels((31, 17), 1e-3, 1e3, seed=9)
    a2 = W.log_uniform_pixels((31, 17), 1e-3, 1e3, seed=9)
    a3 = W.log_uniform_pixels((31, 17), 1e-3, 1e3, seed=10)
    assert a1.shape == (18, 32) and np.array_equal(a1, a2) and not np.array_equal(a1, a3)


def test_log_uniform_field_covers_its_decades_evenly():
    a = W.log_uniform_pixels((255, 255), 1e-4, 1e4, seed=1)
    e = np.log10(a)
    assert e.min() >= -4 and e.max() <= 4
    assert abs(e.mean()) < 0.05 and abs(e.std() - 8 / np.sqrt(12)) < 0.05   # U[-4, 4]
    hist, _ = np.histogram(e, bins=8, range=(-4, 4))
    assert hist.min() > 0.9 * hist.mean()


def test_benchmark_problems_match_their_recipes():
    p0 = W.config_problem(0)
    assert p0.ns == (127, 127) and p0.n == 16129 and (p0.leaf, p0.tol, p0.b) == (8, 1e-3, 0.0)
    assert p0.f.shape == (16129,) and np.log10(p0.a).min() >= -2 and np.log10(p0.a).max() <= 2
    p1 = W.config_problem(1)
    assert p1.ns == (1023, 1023) and p1.n == 1046529 and (p1.leaf, p1.tol) == (16, 1e-3)
    p2 = W.config_problem(2)
    assert p2.ns == (63, 63, 63) and p2.n == 250047 and p2.b == 1e-2 and p2.a.shape == (64, 64, 64)
    f = p1.f
    assert abs(f.mean()) < 5e-3 and abs(f.std() - 1) < 5e-3                  # N(0, 1)


def test_batched_recipe():
    sides = W.batched_sides()
    assert len(sides) == 64 and min(sides) >= 127 and max(sides) <= 511
    assert sides == W.batched_sides()
    ps = W.batched_problems(3, 32)
    for s, p in zip(sides, ps):
        assert p.ns == (s, s) and p.f.shape == (32, s * s) and (p.leaf, p.tol) == (8, 1e-3)
        e = np.log10(p.a)
        assert e.min() >= -3 and e.max() <= 3


def test_bump_field_and_inverse_problem():
    ns = (63, 63)
    g = W.gaussian_bump_log_field(ns, seed=4)
    assert g.shape == W.pixel_shape(ns)
    # 20 bumps of height 3 with random signs: bounded by 20 * 3, smooth, both signs present
    assert np.abs(g).max() <= 60 and g.max() > 0 > g.min()
    assert np.abs(np.diff(g, axis=1)).max() < 3.0
    log_star, f = W.inverse_problem(ns)
    assert log_star.shape == W.pixel_shape(ns) and np.all(f == 1.0) and f.shape == (63 * 63,)


def test_paper_field_is_a_median_split_of_two_values():
    a = W.paper_quantized_field((127, 127), seed=3)
    vals, counts = np.unique(a, return_counts=True)
    assert list(vals) == [1e-2, 1e2]
    assert abs(counts[0] - counts[1]) <= 0.01 * a.size       # the median splits it in half
    # smoothing over 4h makes neighbours agree far more often than independent pixels would
    same = np.mean(a[:, 1:] == a[:, :-1])
    assert same > 0.8
