"""The seeded input recipe both sides consume: reproducible per seed,
independent across seeds and streams, with the stated distributions
(E = exp(sigma g), g ~ N(0, 1); b ~ U[-1, 1]; Gaussian or Rademacher probes;
training sigma ~ U[0.5, 2]) and the parameter layout's size."""
import numpy as np

from paper_2412_07127_gb300 import inputs as I


def test_reproducible_and_seed_dependent():
    assert np.array_equal(I.material_field(12, 3), I.material_field(12, 3))
    assert not np.array_equal(I.material_field(12, 3), I.material_field(12, 4))
    assert np.array_equal(I.rhs(500, 3), I.rhs(500, 3))
    assert not np.array_equal(I.rhs(500, 3), I.rhs(500, 4))
    assert np.array_equal(I.probes(4, 300, 3), I.probes(4, 300, 3))


def test_material_field_is_lognormal_with_the_stated_sigma():
    N = 60
    for sigma in (0.5, 1.0, 2.0):
        lg = np.log(I.material_field(N, 9, sigma))
        assert lg.shape == (N ** 3,)
        # 216,000 draws: mean and standard deviation of g within 5 standard errors
        se = sigma / np.sqrt(lg.size)
        assert abs(lg.mean()) < 5 * se
        assert abs(lg.std() - sigma) < 5 * sigma / np.sqrt(2 * lg.size)
    # the same g for every sigma: the fields of one seed differ by a power
    assert np.allclose(np.log(I.material_field(N, 9, 2.0)), 2.0 * np.log(I.material_field(N, 9, 1.0)))


def test_rhs_and_probes_distributions():
    b = I.rhs(200000, 5)
    assert b.min() >= -1.0 and b.max() < 1.0
    assert abs(b.mean()) < 5 * np.sqrt(1 / 3 / b.size) and abs(b.var() - 1 / 3) < 0.01
    z = I.probes(8, 50000, 5)
    assert z.dtype == np.float32 and z.shape == (8, 50000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.02
    r = I.probes(8, 50000, 5, kind="rademacher")
    assert set(np.unique(r)) == {-1.0, 1.0}
    # streams of one seed are independent draws (b and z do not coincide)
    assert abs(np.corrcoef(I.rhs(1000, 5), I.probes(1, 1000, 5)[0])[0, 1]) < 0.15


def test_training_sigma_range_and_parameter_count():
    s = [I.training_sigma(k) for k in range(2000)]
    assert min(s) >= 0.5 and max(s) < 2.0 and abs(np.mean(s) - 1.25) < 0.03
    total = sum(int(np.prod(sh)) for _, sh in I.param_slices().values())
    assert total == I.N_PARAMS == 3504
    offs = sorted((off, int(np.prod(sh))) for off, sh in I.param_slices().values())
    assert all(o1 + n1 == o2 for (o1, n1), (o2, _) in zip(offs, offs[1:]))  # contiguous, no overlap
