"""Pins of the oracle's iPALM update and VarNet constraint projection (CPU only).

The projection is checked against its defining optimality condition (the variational
inequality of a projection onto a closed convex set), not against a retyped formula; the
iteration against the closed-form constrained minimiser of a strongly convex quadratic and
against a plain projected gradient step where the inertia is zero (the first update)."""
import numpy as np
import pytest

from oracle import ipalm


def _rand_filters(rng, shape=(5, 11, 11), scale=1.0):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) * scale


def _feasible(rng, shape=(5, 11, 11)):
    k = _rand_filters(rng, shape)
    k -= k.mean(axis=(-2, -1), keepdims=True)
    n = np.sqrt(np.sum(np.abs(k) ** 2, axis=(-2, -1), keepdims=True))
    return k / n * rng.uniform(0.0, 1.0, size=n.shape)


@pytest.mark.parametrize("scale", [0.01, 0.1, 3.0])
def test_projection_is_feasible_idempotent_and_optimal(scale):
    rng = np.random.default_rng(1)
    v = _rand_filters(rng, scale=scale) + 0.5 * scale  # a nonzero mean too
    p = ipalm.project_filter(v)
    assert np.abs(p.mean(axis=(-2, -1))).max() <= 1e-14
    assert np.sqrt(np.sum(np.abs(p) ** 2, axis=(-2, -1))).max() <= 1 + 1e-12
    np.testing.assert_allclose(ipalm.project_filter(p), p, atol=1e-14)
    # variational inequality: Re<v - P v, w - P v> <= 0 for every feasible w
    for _ in range(50):
        w = _feasible(rng)
        ip = np.real(np.sum(np.conj(v - p) * (w - p), axis=(-2, -1)))
        assert ip.max() <= 1e-10
    # a feasible point is its own projection
    w = _feasible(rng)
    np.testing.assert_allclose(ipalm.project_filter(w), w, atol=1e-14)


def test_projection_brute_force_on_a_two_tap_filter():
    """For a 1x2 filter the feasible set is {(a, -a): 2|a|^2 <= 1}: the nearest point is
    found by a grid search over a in the complex disc."""
    rng = np.random.default_rng(2)
    for _ in range(5):
        v = _rand_filters(rng, (1, 1, 2), 1.5)
        p = ipalm.project_filter(v)
        R = 1 / np.sqrt(2)
        r = np.linspace(-R, R, 801)
        A = r[:, None] + 1j * r[None, :]
        A = np.concatenate([A[np.abs(A) <= R], R * np.exp(2j * np.pi * np.arange(40000) / 40000)])
        d = np.abs(v[0, 0, 0] - A) ** 2 + np.abs(v[0, 0, 1] + A) ** 2
        best = A[np.argmin(d)]
        assert abs(p[0, 0, 0] - best) <= 2e-3 and abs(p[0, 0, 1] + best) <= 2e-3


def test_lambda_clamped_and_rbf_free():
    f, r, l = ipalm.project(np.zeros((2, 3, 3)), np.array([[-5.0, 7.0]]), np.array([-0.3, 0.2]))
    np.testing.assert_array_equal(r, [[-5.0, 7.0]])
    np.testing.assert_array_equal(l, [0.0, 0.2])


def test_inertia_sequence():
    assert ipalm.inertia(1) == 0.0
    assert ipalm.inertia(2) == 0.25
    assert ipalm.inertia(3) == 0.4
    with pytest.raises(ValueError):
        ipalm.inertia(0)


def test_converges_to_constrained_minimiser_of_a_quadratic():
    """min 1/2 ||x - c||^2 over the constraint set has the minimiser P(c) (the definition of
    the projection); iPALM with step 0.5 reaches it."""
    rng = np.random.default_rng(3)
    c = (_rand_filters(rng, (4, 5, 5)) + 0.3, rng.standard_normal((4, 31)), np.array([-1.0, 2.0]))
    x0 = (np.zeros((4, 5, 5), complex), np.zeros((4, 31)), np.ones(2))
    grad = lambda z: tuple(np.asarray(zi) - ci for zi, ci in zip(z, c))
    x, _ = ipalm.run(x0, grad, (0.5, 0.5, 0.5), 200)
    want = ipalm.project(*c)
    for a, b in zip(x, want):
        np.testing.assert_allclose(a, b, atol=1e-10)


def test_first_update_is_projected_gradient_and_inertial_points():
    rng = np.random.default_rng(4)
    c = (_rand_filters(rng, (2, 3, 3)), rng.standard_normal((2, 31)), np.array([0.5]))
    grad = lambda z: tuple(2.0 * (np.asarray(zi) - ci) for zi, ci in zip(z, c))
    x0 = (np.zeros((2, 3, 3), complex), np.zeros((2, 31)), np.zeros(1))
    tau = (0.1, 0.2, 0.3)
    x, zs = ipalm.run(x0, grad, tau, 3)
    # update 1 (alpha = 0) is a projected gradient step from x^0
    for a, b in zip(zs[0], x0):
        np.testing.assert_array_equal(a, b)
    x1 = ipalm.step(x0, grad(x0), tau)
    # update 2 takes its gradient at x^1 + (1/4)(x^1 - x^0), update 3 at x^2 + (2/5)(x^2 - x^1)
    for a, b, cc in zip(zs[1], x1, x0):
        np.testing.assert_allclose(a, b + 0.25 * (b - cc), atol=1e-15)
    x2 = ipalm.step(zs[1], grad(zs[1]), tau)
    for a, b, cc in zip(zs[2], x2, x1):
        np.testing.assert_allclose(a, b + 0.4 * (b - cc), atol=1e-15)
    for a, b in zip(x, ipalm.step(zs[2], grad(zs[2]), tau)):
        np.testing.assert_array_equal(a, b)
