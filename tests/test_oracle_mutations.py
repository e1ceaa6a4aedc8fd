"""The pins catch plausible mistakes: each case plants one error in the oracle
(on the CPU, through monkeypatch) and checks that a pin test then fails."""
import math

import numpy as np
import pytest

import oracle
import synth
import test_oracle_field as field_pins
import test_oracle_pins as pins


@pytest.fixture(scope="module")
def sp4():
    return synth.diamond_system(2, "sp4", 6.0, 6.0)


def _expect_failure(fn, *args):
    with pytest.raises(AssertionError):
        fn(*args)


def test_wrong_taylor_sign_is_caught(monkeypatch, sp4):
    orig = oracle.taylor_em

    def bad(T, dt, terms, pat_u):  # (+i dt) instead of (-i dt)
        return orig(T, -dt, terms, pat_u)

    monkeypatch.setattr(oracle, "taylor_em", bad)
    _expect_failure(pins.test_step_matches_eigenpair_closed_form, sp4, "em")


def test_dropped_taylor_term_is_caught(monkeypatch, sp4):
    orig = oracle.taylor_em

    def bad(T, dt, terms, pat_u):  # five terms instead of six
        return orig(T, dt, terms - 1, pat_u)

    monkeypatch.setattr(oracle, "taylor_em", bad)
    _expect_failure(pins.test_step_matches_eigenpair_closed_form, sp4, "em")


def test_missing_dagger_in_sandwich_is_caught(monkeypatch, sp4):
    def bad(U, K, pat_m):  # K' = M U instead of M U^dagger
        M = oracle.spgemm(U, K, pat_m)
        Kn = oracle.zeros(K.bsize, K.pat)
        oracle.spgemm(M, U, K.pat, b_dag=False, upper_only=True, out=Kn)
        return Kn, oracle.mirror_upper(Kn)

    monkeypatch.setattr(oracle, "sandwich", bad)
    _expect_failure(pins.test_step_matches_eigenpair_closed_form, sp4, "cn")


def test_transposed_operand_in_product_is_caught(monkeypatch):
    orig = oracle.spgemm

    def bad(A, B, pat_c, a_dag=False, b_dag=False, **kw):  # op(B) transposed by mistake
        return orig(A, B, pat_c, a_dag=a_dag, b_dag=not b_dag, **kw)

    monkeypatch.setattr(oracle, "spgemm", bad)
    _expect_failure(pins.test_spgemm_matches_masked_dense, False, False)


def test_wrong_cn_sign_is_caught(monkeypatch, sp4):
    orig = oracle.axpy

    def bad(alpha, X, Y):  # S - i dt/2 H where S + i dt/2 H is meant (and vice versa)
        if isinstance(alpha, complex) and alpha.real == 0.0:
            alpha = -alpha
        return orig(alpha, X, Y)

    monkeypatch.setattr(oracle, "axpy", bad)
    _expect_failure(pins.test_step_matches_eigenpair_closed_form, sp4, "cn")


def test_wrong_field_sign_is_caught(monkeypatch):
    def bad(H0, D, E):  # H0 + E D instead of H0 - E D
        return oracle.axpy(+E, D, H0)

    monkeypatch.setattr(oracle, "hamiltonian", bad)
    _expect_failure(field_pins.test_pulse_approaches_kick)


def test_wrong_midpoint_is_caught(monkeypatch):
    orig = oracle.field_value

    def bad(field, t):  # field sampled a step late
        return orig(field, t + 0.01)

    monkeypatch.setattr(oracle, "field_value", bad)
    _expect_failure(field_pins.test_pulse_approaches_kick)


def test_wrong_hotelling_update_is_caught(monkeypatch, tiny_spd13):
    orig = oracle.identity

    def bad(bsize, pat, scale=1.0):  # X(I - SX) instead of X(2I - SX)
        return orig(bsize, pat, 1.0 if scale == 2.0 else scale)

    monkeypatch.setattr(oracle, "identity", bad)
    _expect_failure(pins.test_hotelling_matches_lu_inverse, tiny_spd13)


def test_pattern_without_minimum_image_is_caught(monkeypatch, sp4):
    orig = oracle.pattern

    def bad(pos, cell, r):  # plain distance: periodic images ignored
        return orig(pos, None, r)

    monkeypatch.setattr(oracle, "pattern", bad)
    _expect_failure(pins.test_pattern_matches_explicit_images, sp4, 6.0)
