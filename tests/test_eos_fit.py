"""The fourth-order Birch-Murnaghan fit of the EOS sweep
(paper_1611_00731_gb300/eos.py), pinned on the CPU by the closed-form
third-order Birch-Murnaghan curve, which the quartic fit contains exactly."""
import numpy as np
import pytest

from paper_1611_00731_gb300 import eos


def _bm3(V, E0, V0, B0, B0p):
    x = (V0 / V) ** (2.0 / 3.0) - 1.0
    return E0 + 9.0 * V0 * B0 / 16.0 * (x ** 3 * B0p + x ** 2 * (6.0 - 4.0 * (V0 / V) ** (2.0 / 3.0)))


def test_fit_recovers_third_order_birch_murnaghan_parameters():
    E0, V0, B0, B0p = -7.83, 112.3, 0.0125, 3.6
    V = V0 * np.linspace(0.94, 1.06, 11) ** 3
    fit = eos.birch_murnaghan4_fit(V, _bm3(V, E0, V0, B0, B0p))
    assert abs(fit["V0"] - V0) < 1e-8 * V0
    assert abs(fit["E0"] - E0) < 1e-12 * abs(E0)
    assert abs(fit["B0"] - B0) < 1e-7 * B0
    assert abs(fit["B0p"] - B0p) < 1e-5 * B0p
    assert fit["rms"] < 1e-13


def test_fit_needs_five_samples_and_a_minimum():
    V = np.linspace(100.0, 120.0, 4)
    with pytest.raises(ValueError):
        eos.birch_murnaghan4_fit(V, -1.0 / V)
    V = np.linspace(100.0, 120.0, 7)
    with pytest.raises(ValueError):
        eos.birch_murnaghan4_fit(V, -V)          # monotonic: no minimum
