"""The synthetic workloads against the observation tables the paper prints (Tab. 1, Tab. 2),
stored as text in tests/golden/paper_tables.txt with their citation.

Tab. 2's field (3600^2 pixels over 2 x 2 degrees) fixes the MeerKAT-like preset's 2" pixels and
the 3600^2 side measurement; its two bands lie inside the preset's 8 channels. Tab. 1 fixes the
Cygnus A image shapes (square pixels over a 0.025 x 0.05 degree field at every band).
"""
import math
import os

import numpy as np
import pytest

from paper_2406_09144_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_tables.txt")
DEG = math.pi / 180.0


def _rows(tag):
    out = []
    with open(GOLDEN) as f:
        for line in f:
            parts = line.split()
            if parts and parts[0] == tag:
                out.append([float(x) for x in parts[1:]])
    return np.array(out)


def test_tables_parse():
    t1, t2 = _rows("tab1"), _rows("tab2")
    assert t1.shape == (4, 6) and t2.shape == (2, 8)
    # Tab. 1: 2052, 4811, 8427, 13360 MHz; the two lowest bands share their row count within 4
    assert list(t1[:, 0]) == [2052, 4811, 8427, 13360]
    assert abs(t1[0, 1] - t1[1, 1]) == 4
    # Tab. 2: both bands have the same rows and field
    assert t2[0, 2] == t2[1, 2] == 4598424


def test_tab1_pixels_are_square():
    for f, nrow, nx, ny, fx, fy in _rows("tab1"):
        assert math.isclose(fx / nx, fy / ny, rel_tol=1e-12), (f, nx, ny)


def test_tab2_field_fixes_the_meerkat_like_pixel_size():
    t2 = _rows("tab2")
    nx, fov = t2[0, 4], t2[0, 6]
    pix = fov * DEG / nx  # 2 degrees over 3600 pixels = 2 arcsec
    obs = synth.observation("meerkat1", hours=0.1)  # the preset's geometry; few rows
    assert math.isclose(obs.pixsize, pix, rel_tol=1e-12)
    side = synth.observation("meerkat1", hours=0.1, npix=3600)
    assert (side.nx, side.ny) == (int(t2[0, 4]), int(t2[0, 5]))
    assert math.isclose(side.nx * side.pixsize / DEG, fov, rel_tol=1e-12)


def test_tab2_bands_lie_inside_the_meerkat_like_channels():
    obs = synth.observation("meerkat1", hours=0.1)
    full = synth.observation("meerkat", hours=0.1)
    width = float(np.diff(full.freqs).min())
    lo = (full.freqs.min() - width / 2) / 1e6
    hi = (full.freqs.max() + width / 2) / 1e6
    for flo, fhi, *_ in _rows("tab2"):
        assert lo <= flo < fhi <= hi, (flo, fhi, lo, hi)
    assert obs.freqs[0] == full.freqs[-1]  # the single-channel preset is the top channel


@pytest.mark.parametrize("name", ["vla", "meerkat"])
def test_presets_keep_square_pixels_and_power_of_two_sides(name):
    obs = synth.observation(name, hours=0.1)
    assert obs.nx == obs.ny and obs.nx & (obs.nx - 1) == 0
