"""Pins of the oracle's delta kernels and Heaviside profile against closed forms
and the values the paper prints (Section 2.2 Eq. (cherby), Section 3.2
Eqs. (new_hea), (new_hea2))."""
import json
import os

import numpy as np
import pytest

GOLD = os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")


@pytest.mark.parametrize("kernel", [0, 1])
def test_partition_of_unity_and_parity_halves(O, kernel):
    # Section 2.2: the kernel sums to one over the grid points; both kernels
    # also split it evenly between even and odd points (1/2 each).
    for r in np.linspace(0.0, 1.0, 37, endpoint=False):
        k = np.arange(-3, 5)
        w = O.phi(k - r, kernel)
        assert abs(w.sum() - 1.0) < 1e-15
        assert abs(w[k % 2 == 0].sum() - 0.5) < 1e-15
        assert abs(w[k % 2 == 1].sum() - 0.5) < 1e-15


def test_cosine_first_moment_closed_form(O):
    # The paper's cosine kernel does NOT have a zero first moment.  Summing
    # (k - r) phi(k - r) over the four support points in closed form gives
    # (2 - 4r + 2 sin(pi r/2) - 2 cos(pi r/2)) / 4.
    for r in np.linspace(0.0, 1.0, 41, endpoint=False):
        k = np.arange(-3, 5)
        m1 = ((k - r) * O.phi(k - r, 0)).sum()
        ref = 0.25 * (2 - 4 * r + 2 * np.sin(np.pi * r / 2) - 2 * np.cos(np.pi * r / 2))
        assert abs(m1 - ref) < 1e-15
    rr = np.linspace(0, 1, 2001)
    ref = 0.25 * (2 - 4 * rr + 2 * np.sin(np.pi * rr / 2) - 2 * np.cos(np.pi * rr / 2))
    assert 0.0210 < np.abs(ref).max() < 0.0212


def test_peskin_first_moment_and_square_sum(O):
    # Peskin (2002) 4-point kernel: zero first moment and sum phi^2 = 3/8.
    for r in np.linspace(0.0, 1.0, 41, endpoint=False):
        k = np.arange(-3, 5)
        w = O.phi(k - r, 1)
        assert abs(((k - r) * w).sum()) < 1e-15
        assert abs((w * w).sum() - 0.375) < 1e-15


def test_kernel_support_and_symmetry(O):
    r = np.linspace(-3, 3, 601)
    for kernel in (0, 1):
        w = O.phi(r, kernel)
        assert np.all(w[np.abs(r) >= 2] == 0.0)
        assert np.allclose(w, O.phi(-r, kernel), atol=0, rtol=0)
        assert np.all(w >= 0)


def test_heaviside_profile_is_integral_of_kernel(O):
    # Eq. (new_hea): H(r) = integral_{-2}^{r} phi; check H' = phi by central
    # differences and H(r) + H(-r) = 1.
    r = np.linspace(-1.99, 1.99, 399)
    e = 1e-5
    dH = (O.heaviside_profile(r + e) - O.heaviside_profile(r - e)) / (2 * e)
    assert np.abs(dH - O.phi(r, 0)).max() < 1e-9
    assert np.abs(O.heaviside_profile(r) + O.heaviside_profile(-r) - 1).max() < 1e-15
    assert O.heaviside_profile([-2.0])[0] == 0.0 and O.heaviside_profile([2.0])[0] == 1.0


def test_heaviside_region_values_match_paper(O):
    gold = json.load(open(GOLD))["heaviside_regions"]
    vals = O.heaviside_profile(np.arange(-2, 3, dtype=float))
    printed = gold["values"]
    # regions I, III, IV, V as printed (3 digits)
    for k in (0, 2, 3, 4):
        assert abs(vals[k] - printed[k]) < 5e-4
    # region II: the printed 0.409 is a misprint of 1 - 0.909 = 0.0908
    assert abs(vals[1] - (1.0 - printed[3])) < 5e-4
    assert abs(vals[1] - printed[1]) > 0.3
