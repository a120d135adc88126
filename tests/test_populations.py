"""The seeded input generators: structure, determinism and the stated recipe."""

import numpy as np

from paper_2606_15622_gb300 import populations as P


def _check_structure(pop):
    assert pop.offsets[0] == 0 and pop.offsets[-1] == pop.n_particles
    assert np.all(np.diff(pop.offsets) >= 0)
    assert pop.v64.shape == (3, pop.n_particles) and pop.v64.flags.c_contiguous
    assert pop.tau.shape == (pop.n_cells,) and np.all(pop.tau > 0)
    assert np.isfinite(pop.v64).all()


def test_couette_recipe():
    pop = P.couette()
    _check_structure(pop)
    assert pop.n_cells == 400 and np.all(pop.counts == 100)
    assert pop.meta["theta"].min() >= 0.8 and pop.meta["theta"].max() <= 1.2
    np.testing.assert_array_equal(pop.v64, P.couette().v64)
    assert not np.array_equal(pop.v64, P.couette(seed=5).v64)


def test_cavity_recipe(cavity_pop):
    pop = cavity_pop
    _check_structure(pop)
    assert pop.n_cells == 128 * 128
    assert pop.counts.min() >= 8 and pop.counts.max() <= 400
    assert 0.7e6 < pop.n_particles < 0.9e6
    th = pop.meta["theta"]
    assert th.max() / th.min() > 2.5
    frac = pop.meta["bimodal"].mean()
    assert 0.08 < frac < 0.12


def test_training_cells_structure():
    pop = P.training_cells(2000, seed=5)
    _check_structure(pop)
    assert np.all(pop.counts[:1000] == 100)
    assert pop.counts[1000:].min() >= 8 and pop.counts[1000:].max() <= 400
    np.testing.assert_array_equal(pop.v64, P.training_cells(2000, seed=5).v64)
