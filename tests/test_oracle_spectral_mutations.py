"""The pins of the spectral oracles catch plausible mistakes: each mistake is
planted in the oracle (on the CPU, by replacing one of its functions) and at
least one pin must then fail."""
import numpy as np
import pytest

from oracle import fourier, legendre

import test_oracle_fourier as tf
import test_oracle_legendre as tl


def _fourier_pins():
    yield lambda: tf.test_matches_the_direct_sum(40)
    yield lambda: tf.test_matches_the_direct_sum(1280)
    yield tf.test_pure_tones
    yield tf.test_parseval_and_shift


def _legendre_pins():
    yield tl.test_closed_forms
    yield tl.test_against_scipy_lpmv
    yield tl.test_parity_and_orthonormality_under_quadrature
    yield tl.test_layout
    yield lambda: tl.test_recovers_the_generator_coefficients(64, 32, 21)


def _caught(pins):
    for pin in pins:
        try:
            pin()
        except AssertionError:
            return True
    return False


def test_unmutated_oracles_pass_every_pin():
    assert not _caught(_fourier_pins())
    assert not _caught(_legendre_pins())


_rfft, _dft = fourier.rfft_lon, fourier.dft_direct


@pytest.mark.parametrize("name,mutants", [
    ("no 1/N", {"rfft_lon": lambda x, K: tuple(v * np.shape(x)[-1] for v in _rfft(x, K))}),
    ("conjugated, in both statements", {"rfft_lon": lambda x, K: (_rfft(x, K)[0], -_rfft(x, K)[1]),
                                        "dft_direct": lambda x, K: (_dft(x, K)[0], -_dft(x, K)[1])}),
    ("wavenumbers shifted by one", {"rfft_lon": lambda x, K: tuple(np.roll(v, 1, axis=-1) for v in _rfft(x, K))}),
])
def test_fourier_mistakes_are_caught(monkeypatch, name, mutants):
    for attr, fn in mutants.items():
        monkeypatch.setattr(fourier, attr, fn)
    assert _caught(_fourier_pins()), name


_pbar, _nodes, _offset = legendre.pbar_m, legendre.gauss_nodes, legendre.offset


def _scale_from(l0, f):
    def pbar(m, T, mu):
        P = _pbar(m, T, mu).copy()
        P[max(0, l0 - m):] *= f
        return P
    return pbar


@pytest.mark.parametrize("name,attr,fn", [
    ("no Condon-Shortley phase", "pbar_m", lambda m, T, mu: _pbar(m, T, mu) * (-1.0) ** m),
    ("a recurrence coefficient off from l = 2", "pbar_m", _scale_from(2, 1.0 + 1e-6)),
    ("normalised to 2 instead of 1", "pbar_m", lambda m, T, mu: _pbar(m, T, mu) * np.sqrt(2.0)),
    ("weights not symmetric", "gauss_nodes", lambda n: (_nodes(n)[0], _nodes(n)[1] * (1 + 1e-3 * _nodes(n)[0]))),
    ("nodes south to north", "gauss_nodes", lambda n: (_nodes(n)[0][::-1].copy(), _nodes(n)[1][::-1].copy())),
    ("layout off by one order", "offset", lambda m, T: _offset(m, T) + (1 if m else 0)),
])
def test_legendre_mistakes_are_caught(monkeypatch, name, attr, fn):
    monkeypatch.setattr(legendre, attr, fn)
    assert _caught(_legendre_pins()), name
