"""The seeded input generator: published RNG vectors and the properties of the synthetic fields."""
import numpy as np

from paper_2009_02171_gb300.inputs import benchmark_B0, cell_centres, initial_state, normals, splitmix64


def test_splitmix64_reference_outputs():
    # SplitMix64 with seed 0 (Steele, Lea, Flood 2014; the reference C code's first outputs)
    assert [int(v) for v in splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_normals_are_standard():
    z = normals(1, 200000)
    assert abs(z.mean()) < 0.01 and abs(z.std() - 1) < 0.01


def test_initial_state_is_seeded_and_bc_exact():
    a, b = initial_state(6, 5, 3), initial_state(6, 5, 3)
    assert all(np.array_equal(a[k], b[k]) for k in a)
    c = initial_state(6, 5, 4)
    assert not np.array_equal(a['u'], c['u'])
    # B0 of eqn:initial: tangential part vanishes and r^2 B_r is flat at both walls
    for rw in (7 / 13, 20 / 13):
        rng = np.random.default_rng(0)
        v = rng.standard_normal((3, 50))
        v /= np.linalg.norm(v, axis=0)
        B = benchmark_B0(*(rw * v))
        Bt = B - (B * v).sum(0) * v
        assert abs(Bt).max() < 1e-12
        h = 1e-6
        f = lambda rr: rr ** 2 * (benchmark_B0(*(rr * v)) * v).sum(0)
        assert abs((f(rw + h) - f(rw - h)) / (2 * h)).max() < 1e-6
