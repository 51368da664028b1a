"""The seeded input generators: shapes and structure they promise (they hold
none of the method's arithmetic)."""
import numpy as np

from oracle import state_dim
from paper_1610_08035_gb300 import synth


def test_co2_shaped_series_has_the_stated_shape():
    """The CO2-shaped generator: 2195 weekly points in years, standardised,
    with the b = 16 model's seven parameters and the annual period to start."""
    s = synth.co2_shaped()
    assert len(s.t) == len(s.y) == 2195
    assert np.allclose(np.diff(s.t), 1.0 / 52.1775, rtol=0, atol=1e-12)
    assert abs(s.y.mean()) < 1e-12 and abs(s.y.std() - 1.0) < 1e-12
    assert state_dim(s.spec) == 16 and len(s.theta) == 7 and s.theta[4] == 1.0
    # the annual cycle dominates the detrended series' spectrum
    yd = s.y - np.polyval(np.polyfit(s.t, s.y, 2), s.t)
    f = np.fft.rfftfreq(len(yd), d=1.0 / 52.1775)
    peak = f[1 + np.argmax(np.abs(np.fft.rfft(yd))[1:])]
    assert abs(peak - 1.0) < 0.05
