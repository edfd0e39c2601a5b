"""CPU checks of the learned preconditioner's host-side decisions (no GPU): the
iteration count read off an error history, the parabola refinement of the label
search, and the fallback gate (the model is used only if it lowers the median
iteration count on validation systems)."""
import math

import numpy as np
import pytest


@pytest.fixture(scope="module")
def learned():
    from paper_2503_22863_b300 import build
    build.build()
    from paper_2503_22863_b300 import learned as m
    return m


def test_iterations_to(learned):
    eh = [1e-1, 1e-4, 2e-9, 1e-9, 1e-12]
    assert learned.iterations_to(eh, 1e-9) == 4      # first iterate at or below tol, 1-based
    assert learned.iterations_to(eh, 1e-3) == 2
    assert learned.iterations_to(eh, 1e-13) is None
    assert learned.iterations_to([], 1e-9) is None


def test_vertex_exact_on_a_parabola(learned):
    # y = 3 (x - 0.1)^2 + 2 through the grid points -1/4, 0, 1/4
    xs = (-0.25, 0.0, 0.25)
    for c in (0.1, -0.2, 0.0, 0.249):
        ys = [3.0 * (x - c) ** 2 + 2.0 for x in xs]
        assert math.isclose(learned._vertex(xs, ys), c, rel_tol=0, abs_tol=1e-12)


def test_vertex_clamped_and_degenerate(learned):
    xs = (0.0, 0.25, 0.5)
    # vertex beyond the bracket is clamped to its end
    ys = [(x - 0.9) ** 2 for x in xs]
    assert learned._vertex(xs, ys) == 0.5
    # flat or concave: the middle point
    assert learned._vertex(xs, [1.0, 1.0, 1.0]) == 0.25
    assert learned._vertex(xs, [1.0, 2.0, 1.0]) == 0.25


class _FakeSystem:
    """Records which scaling was asked for; no device work."""

    def __init__(self, name):
        self.name = name
        self.calls = []

    def column_features(self):
        return ("features", self.name)

    def learned_scaling(self, m, clamp=None):
        self.calls.append((m, clamp))
        return ("learned", self.name) if m is not None else ("colnorm", self.name)


class _FakeModel:
    def predict(self, feats):
        return ("m", feats[1])


class _FakeProbe:
    def __init__(self, n_colnorm, n_learned):
        self.n_colnorm, self.n_learned = n_colnorm, n_learned

    def iterations(self, d):
        assert d[0] == "learned"   # validation always scores the learned scaling
        return self.n_learned


def _pairs(colnorm, learned_):
    return [(_FakeSystem(i), _FakeProbe(c, l)) for i, (c, l) in enumerate(zip(colnorm, learned_))]


def test_gate_keeps_a_model_that_lowers_the_median(learned):
    pre = learned.LearnedPreconditioner(_FakeModel(), clamp=2.0)
    v = pre.validate(_pairs([60, 58, 61], [55, 59, 57]))     # medians 57 < 60
    assert pre.enabled and v["enabled"]
    S = _FakeSystem("s")
    assert pre.scaling(S) == ("learned", "s")
    assert S.calls == [(("m", "s"), 2.0)]


def test_gate_falls_back_when_not_better(learned):
    for lrn in ([60, 58, 61], [61, 59, 62]):                  # equal, worse medians
        pre = learned.LearnedPreconditioner(_FakeModel())
        v = pre.validate(_pairs([60, 58, 61], lrn))
        assert not pre.enabled and not v["enabled"]
        S = _FakeSystem("s")
        assert pre.scaling(S) == ("colnorm", "s")
        assert S.calls == [(None, None)]


def test_a_disabled_model_stays_disabled(learned):
    pre = learned.LearnedPreconditioner(_FakeModel(), enabled=False)
    pre.validate(_pairs([60, 58, 61], [40, 40, 40]))
    assert not pre.enabled
    assert learned.LearnedPreconditioner(None).scaling(_FakeSystem("t")) == ("colnorm", "t")
