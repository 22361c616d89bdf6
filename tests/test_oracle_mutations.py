"""Mistakes planted in the oracle (on the CPU, by monkeypatching) must fail
the pins: each pin set is shown to be sensitive to a plausible error."""
import numpy as np
import pytest

from oracle import affine, derivs, engine, rng
from tests import test_oracle_affine as ta
from tests import test_oracle_derivs as td
from tests import test_oracle_engine as te


def fails(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_splitmix64_published_values():
    # Steele, Lea, Flood (2014); outputs of the reference implementation
    assert [rng.splitmix64(0, k) for k in range(3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                        0x06C45D188009454F]
    assert [rng.splitmix64(1234567, k) for k in range(2)] == [6457827717110365317, 3203168211198807973]


def test_off_by_one_falling_factorial_is_caught(monkeypatch):
    monkeypatch.setattr(derivs, "falling", lambda a, k: int(np.prod([a - i + (i > 0) for i in range(k)])))
    fails(td.test_single_monomial_closed_form, 3, 2, 1)
    fails(ta.test_worked_example_sec5)


def test_wrong_third_derivatives_are_caught(monkeypatch):
    real = derivs.third_tensor
    monkeypatch.setattr(derivs, "third_tensor", lambda e, c, x: 0.5 * real(e, c, x))
    # (a constant factor on T keeps affine covariance, so the closed form is the pin)
    fails(ta.test_plane_curve_closed_form)


def test_dropped_regularisation_is_caught(monkeypatch):
    real = affine.affine_normal_ad
    monkeypatch.setattr(affine, "affine_normal_ad", lambda e, c, x, r=1e-6, **kw: real(e, c, x, r=0.0, **kw))
    fails(ta.test_worked_example_sec5)


def test_non_orthonormal_frame_is_caught(monkeypatch):
    real = affine.qr_frame
    monkeypatch.setattr(affine, "qr_frame", lambda e: 1.5 * real(e))
    fails(ta.test_worked_example_sec5)


def test_wrong_monomial_order_is_caught(monkeypatch):
    monkeypatch.setattr(engine, "canonical_order", lambda ex: np.lexsort([ex[:, j] for j in range(ex.shape[1])][::-1]))
    fails(te.test_monolist_order_matches_paper)


def test_wrong_alignment_is_caught(monkeypatch):
    def bad_align(a, b):
        ids, ca, cb = real(a, b)
        return ids, ca, (cb + 1) % len(ids)
    real = engine.align
    monkeypatch.setattr(engine, "align", bad_align)
    fails(te.test_mixed_variable_alignment_sec32)
