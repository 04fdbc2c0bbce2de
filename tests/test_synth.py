"""The seeded synthetic workloads (the inputs both the CUDA path and the oracle take).

Row counts follow from the arrays and tracks (baselines x time steps), the bands and pixel
sizes from the presets, and the tracks from Earth-rotation synthesis, under which every
baseline keeps its length |(u, v, w)| while the sky turns.
"""
import numpy as np
import pytest

from paper_2406_09144_gb300 import synth


@pytest.mark.parametrize("name,nant,hours,step,nrow", [
    ("small", 27, 4.0, 10.0, 505_440),
    ("vla", 27, 8.0, 2.0, 5_054_400),
    ("meerkat", 64, 8.0, 8.0, 7_257_600),
])
def test_rows_are_baselines_times_time_steps(name, nant, hours, step, nrow):
    obs = synth.observation(name)
    nbl = nant * (nant - 1) // 2
    assert obs.uvw.shape == (nrow, 3)
    assert nrow == nbl * int(round(hours * 3600 / step))
    assert obs.weights.shape == (nrow, len(obs.freqs))


def test_meerkat_like_band_and_visibility_count():
    obs = synth.observation("meerkat")
    assert np.allclose(obs.freqs, 909.5e6 + 107e6 * np.arange(8))
    assert obs.nvis == 58_060_800 and obs.per_channel_sky and obs.wterm
    assert np.isclose(obs.pixsize, 2.0 * synth.ARCSEC)
    # longest baseline about 8 km (antennas out to 4 km radius)
    assert 6e3 < np.hypot(obs.uvw[:, 0], obs.uvw[:, 1]).max() < 8.5e3


@pytest.mark.parametrize("name,nant", [("vla", 27), ("meerkat", 64)])
def test_earth_rotation_keeps_each_baseline_length(name, nant):
    obs = synth.observation(name, hours=1.0)
    nbl = nant * (nant - 1) // 2
    uvw = obs.uvw.reshape(-1, nbl, 3)  # time-major, baseline-minor
    length = np.linalg.norm(uvw, axis=2)
    assert np.allclose(length, length[0][None, :], rtol=1e-9, atol=1e-6)
    # the projection itself changes: the tracks are not static
    assert np.abs(uvw[-1, :, :2] - uvw[0, :, :2]).max() > 1.0


def test_small_preset_is_coplanar_and_others_are_not():
    assert np.all(synth.observation("small").uvw[:, 2] == 0.0)
    assert np.abs(synth.observation("vla", hours=0.5).uvw[:, 2]).max() > 0.0


@pytest.mark.parametrize("name", ["vla", "meerkat"])
def test_per_baseline_noise_levels(name):
    obs = synth.observation(name, hours=0.5)
    sig = obs.sigma
    assert np.all(sig >= 0.8e-2 * (1 - 1e-12)) and np.all(sig <= 1.2e-2 * (1 + 1e-12))
    assert np.allclose(obs.weights, 1.0 / sig ** 2)
    assert sig.std() > 0  # the weight path is exercised


def test_generators_are_seeded():
    a = synth.observation("vla", hours=0.2)
    b = synth.observation("vla", hours=0.2)
    assert np.array_equal(a.uvw, b.uvw) and np.array_equal(a.weights, b.weights)
    s1 = synth.random_skies(2, 64, 64, seed=3)
    s2 = synth.random_skies(2, 64, 64, seed=3)
    assert np.array_equal(s1, s2) and np.all(s1 >= 0) and s1.max() > 0
