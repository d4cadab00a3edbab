"""The denoising study's trends on a small cloud (the shape of Sec. 3.3): a
radius a few times the noise reduces the deviation from the exact surface; a
radius far below the point spacing loses most points as outliers."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_denoising_trends():
    from paper_2401_03365_gb300 import build, denoise_study
    build.build()
    rows = denoise_study.run(n=50_000, surfaces=("sphere",), sigmas=(0.005,), radii=(0.003, 0.04))
    small, good = rows
    assert small["removed_frac"] > 0.5
    assert good["removed_frac"] < 0.01
    assert good["after"]["mean"] < 0.5 * good["before"]["mean"]
