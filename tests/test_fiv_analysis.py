"""The tip-oscillation analysis of the flow-induced-vibration run (Section
4.1: amplitude and frequency of the flag tip's transverse motion) on signals
whose amplitude and frequency are known."""
import numpy as np
import pytest

import bench


@pytest.mark.parametrize("f,A,mean", [(1.88, 0.086, 0.0), (0.5, 1.0, 0.3), (3.1, 0.01, -0.02)])
def test_sine(f, A, mean):
    t = np.arange(0.0, 20.0, 0.009)
    y = mean + A * np.sin(2 * np.pi * f * t + 0.4)
    amp, freq, cycles = bench._tip_oscillation(t, y, 10.0)
    assert freq == pytest.approx(f, rel=1e-3)
    assert amp == pytest.approx(A, rel=5e-3)
    assert cycles >= int(10.0 * f) - 1


def test_growing_signal_and_short_records():
    t = np.arange(0.0, 20.0, 0.005)
    y = (0.1 + 0.04 * t) * np.sin(2 * np.pi * 1.6 * t)
    a_late, f_late, _ = bench._tip_oscillation(t, y, 16.0)
    a_mid, _, _ = bench._tip_oscillation(t, y, 10.0)
    assert f_late == pytest.approx(1.6, rel=2e-3)
    assert a_mid < a_late < 0.1 + 0.04 * 20.0
    # fewer than three upward crossings: no estimate
    assert bench._tip_oscillation(t, y, 19.5)[:2] == (None, None)


def test_empty_and_short_windows():
    assert bench._tip_oscillation([], [], 0.0) == (None, None, 0)
    assert bench._tip_oscillation([0.1, 0.2], [0.0, 1.0], 5.0) == (None, None, 0)
