"""The oracle's exact gradient (autograd through the FP64 definition) against
central differences of its own loss, with the discrete structure frozen."""
import numpy as np
import pytest

import scenes
from oracle import pipeline as pl


def _check(sc, picks, tol=1e-6):
    res = pl.loss_and_grads(sc)
    for which, idx in picks:
        an = res["d" + which].reshape(-1)[idx]
        fd = pl.finite_difference(sc, which, idx, res["plans"])
        scale = max(abs(fd), 1e-3 * np.abs(res["d" + which]).max(), 1e-12)
        assert abs(an - fd) <= tol * scale + 1e-13, (which, idx, an, fd)


def _picks(sc, rng, n=6):
    out = []
    for which, arr in (("key", sc.key), ("tau", sc.tau), ("color", sc.color)):
        m = arr.size
        for i in rng.choice(m, min(n, m), replace=False):
            out.append((which, int(i)))
    return out


def test_open_stroke_gradients():
    sc = scenes.small_open(21, n_curves=2, size=32)
    _check(sc, _picks(sc, np.random.default_rng(0)))


def test_open_stroke_production_thresholds():
    sc = scenes.small_open(22, n_curves=2, size=32).with_raster(**scenes.RASTER_DEFAULTS)
    _check(sc, _picks(sc, np.random.default_rng(1)), tol=1e-5)


def test_closed_stroke_gradients():
    sc = scenes.small_closed(23, n_curves=2, size=32, filled=False, degrees=(2, 3, 5))
    _check(sc, _picks(sc, np.random.default_rng(2)))


def test_filled_gradients():
    sc = scenes.small_closed(24, n_curves=2, size=32, filled=True, h=2.0)
    _check(sc, _picks(sc, np.random.default_rng(3)))


def test_multi_scene_gradients():
    sc = scenes.small_closed(25, n_curves=2, size=24, filled=True, h=2.0, n_scenes=2)
    _check(sc, _picks(sc, np.random.default_rng(4), n=4))
