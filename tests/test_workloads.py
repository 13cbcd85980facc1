"""The seeded input generators: SplitMix64 (Steele, Lea & Flood 2014) gives
the published reference outputs, the derived uniform and normal draws have
the right ranges and moments, and every workload is a deterministic function
of its seed."""
import numpy as np

import workloads as W


def test_splitmix64_reference_outputs():
    # the generator's published reference sequence for seed 0
    assert [int(v) for v in W.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_splitmix64_vectorised_equals_sequential():
    m = (1 << 64) - 1

    def seq(seed, n):
        x, out = seed, []
        for _ in range(n):
            x = (x + 0x9E3779B97F4A7C15) & m
            z = ((x ^ (x >> 30)) * 0xBF58476D1CE4E5B9) & m
            z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
            out.append(z ^ (z >> 31))
        return out

    for seed in (1, 3, 4, 7, 2 ** 63 + 5):
        assert [int(v) for v in W.splitmix64(seed, 50)] == seq(seed, 50)


def test_uniform_and_normal_draws():
    u = W.uniform01(1, 200_000)
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 3e-3 and abs(u.var() - 1 / 12) < 2e-3
    z = W.normals(2, 200_000)
    assert abs(z.mean()) < 1e-2 and abs(z.var() - 1.0) < 1e-2
    assert abs(np.mean(z ** 4) - 3.0) < 0.05                       # Gaussian kurtosis
    assert np.array_equal(W.normals(3, 10, skip=5), W.normals(3, 10, skip=5))


def test_workloads_are_deterministic():
    a, b = W.ladder_6lvl(n_cells=256, n_steps=10), W.ladder_6lvl(n_cells=256, n_steps=10)
    assert np.array_equal(a.qms[0].h0, b.qms[0].h0) and np.array_equal(a.qms[0].mu, b.qms[0].mu)
    c = W.ladder_6lvl(n_cells=256, n_steps=10, seed=4)
    assert not np.array_equal(a.qms[0].mu, c.qms[0].mu)
    j1, j2 = W.sit_2lvl_jitter(n_cells=4096, n_steps=10), W.sit_2lvl_jitter(n_cells=4096, n_steps=10)
    assert np.array_equal(j1.jitter, j2.jitter)
    assert np.abs(j1.jitter - 1.0).max() <= 0.01                  # +-1 % factors
    q1, q2 = W.qcl_tzenov(n_cells=512, n_steps=10), W.qcl_tzenov(n_cells=512, n_steps=10)
    assert np.array_equal(q1.e_init, q2.e_init)
    s1, s2 = W.batch_mixed(n_sims=16), W.batch_mixed(n_sims=16)
    assert [(p.n_cells, p.n_steps, p.qms[0].n_levels) for p in s1] == [(p.n_cells, p.n_steps, p.qms[0].n_levels)
                                                                      for p in s2]
