"""The seeded input generators (CPU): each is deterministic for its seed and produces the
fields its docstring promises (ranges, sums, positions), since tests, smoke and the bench
all draw their inputs from them."""
import numpy as np
import pytest

from paper_1306_6445_gb300 import inputs as I
from paper_1306_6445_gb300 import sweep


def test_droplet_and_layers():
    rho = I.droplet_density(101, 81, 20.0, 0.3, 0.02)
    assert rho.shape == (81, 101)
    assert rho[40, 50] == pytest.approx(0.3, rel=1e-8)           # centre ((nx-1)/2, (ny-1)/2)
    assert rho[0, 0] == pytest.approx(0.02, rel=1e-8)
    assert np.allclose(rho, rho[::-1, ::-1])                       # symmetric about the centre
    lay = I.layer_density(64, 40, 10.0, 0.3, 0.02)
    assert lay[0, 0] == pytest.approx(0.3, rel=1e-6) and lay[-1, 0] == pytest.approx(0.02, rel=1e-6)
    slab = I.layer_density(64, 40, 10.0, 0.3, 0.02, y_offset=15.0, two_sided=True)
    assert slab[20, 5] == pytest.approx(0.3, rel=1e-3)             # inside the slab
    assert slab[2, 5] == pytest.approx(0.02, rel=1e-3) and slab[38, 5] == pytest.approx(0.02, rel=1e-3)
    wav = I.layer_density(64, 40, 10.0, 0.3, 0.02, amplitude=3.0, wavenumber=2)
    assert np.allclose(wav[:, 0], wav[:, 32])                      # period nx / k


def test_shear_wave():
    rho, ux, uy = I.shear_wave(16, 32, 1e-3)
    assert np.all(rho == 1.0) and np.all(uy == 0.0)
    assert ux[8, 3] == pytest.approx(1e-3) and ux[0, 5] == 0.0     # sin(2 pi y / ny)


def test_random_fields_are_seeded_and_well_formed():
    a = I.smooth_random_density(np.random.default_rng(3), 40, 30, 0.05, 0.25)
    b = I.smooth_random_density(np.random.default_rng(3), 40, 30, 0.05, 0.25)
    assert np.array_equal(a, b)
    assert a.min() == pytest.approx(0.05) and a.max() == pytest.approx(0.25)
    f = I.random_populations(np.random.default_rng(4), a)
    assert f.shape == (9, 30, 40) and np.all(f > 0)
    assert np.allclose(f.sum(axis=0), a, rtol=1e-13)
    ux, uy = I.random_velocity(np.random.default_rng(5), (3, 4), 0.02)
    assert np.all(np.abs(ux) <= 0.02) and np.all(np.abs(uy) <= 0.02)


def test_batch_draws_and_training_points():
    d = I.batch_draws(200, seed=7)
    assert d == I.batch_draws(200, seed=7) and d != I.batch_draws(200, seed=8)
    assert all(e["side"] in range(64, 513, 32) for e in d)
    for key, lo, hi in (("t_over_tc", 0.65, 0.95), ("kappa", 0.0, 0.95), ("tau_v", 0.6, 1.2)):
        v = np.array([e[key] for e in d])
        assert v.min() >= lo and v.max() <= hi
    r = np.array([e["radius"] / e["side"] for e in d])
    assert r.min() >= 0.15 and r.max() <= 0.35
    p = sweep.training_points(50, seed=7)
    assert p.shape == (50, 3)
    assert np.array_equal(p[:, 0], [e["t_over_tc"] for e in I.batch_draws(50, seed=7)])


def test_mlp_generators():
    w = I.mlp_init(seed=2)
    assert w.dtype == np.float32 and w.size == 64 * 3 + 64 + 64 * 64 + 64 + 3 * 64 + 3
    assert np.array_equal(w, I.mlp_init(seed=2))
    # Glorot bound of the first layer, zero biases
    assert np.abs(w[:192]).max() <= np.sqrt(6.0 / (3 + 64))
    assert np.all(w[192:256] == 0)
    x, y = I.mlp_random_data(100, seed=3)
    assert x.shape == y.shape == (100, 3) and np.all(y > 0)
    assert x[:, 0].min() >= 0.65 and x[:, 0].max() <= 0.95
