"""Argument checks of the memetic loop that stop before any simulation (no GPU)."""
import pytest

from paper_2502_11129_b300 import evolve as E


def test_relative_targets_refuse_morphology_screening():
    with pytest.raises(ValueError, match="screen_morph"):
        E.memetic(n_morph=4, n_ctrl=2, gens=1, steps=10, surrogate=True, relative=True, screen_morph=2)
