"""The seeded input generators shared by the oracle and the CUDA path: shapes,
value ranges and the structure each recipe promises (CPU only)."""
import numpy as np

from paper_2007_05239_gb300 import workloads


def test_block_model_structure_and_densities():
    sizes, p_in, p_out = [60, 40], [0.7, 0.5], [0.3, 0.5]
    Ws, truth = workloads.block_model_layers(sizes, p_in, p_out, seed=3)
    n = sum(sizes)
    assert truth.shape == (n,) and (np.bincount(truth) == sizes).all()
    same = truth[:, None] == truth[None, :]
    off = ~np.eye(n, dtype=bool)
    for W, pi, po in zip(Ws, p_in, p_out):
        assert W.shape == (n, n) and np.array_equal(W, W.T)
        assert np.all(np.diag(W) == 0) and set(np.unique(W)) <= {0.0, 1.0}
        # edge densities within 4 standard deviations of the requested probabilities
        for mask, p in ((same & off, pi), (~same, po)):
            m = mask.sum()
            assert abs(W[mask].mean() - p) <= 4 * np.sqrt(p * (1 - p) / m)
    # seeded: the same seed gives the same graphs, another seed different ones
    again, _ = workloads.block_model_layers(sizes, p_in, p_out, seed=3)
    other, _ = workloads.block_model_layers(sizes, p_in, p_out, seed=4)
    assert all(np.array_equal(a, b) for a, b in zip(Ws, again))
    assert not np.array_equal(Ws[0], other[0])


def test_known_labels_fraction_and_every_class():
    truth = np.repeat(np.arange(5), [400, 300, 200, 90, 10])
    lab = workloads.known_labels(truth, 0.04, seed=7)
    known = lab >= 0
    assert (lab[known] == truth[known]).all()
    assert set(lab[known]) == set(range(5))                 # at least one per class
    assert round(0.04 * len(truth)) <= known.sum() <= round(0.04 * len(truth)) + 5


def test_uniform_generators_stay_in_their_domains():
    X = workloads.uniform_cube(5000, 3, half=0.25, seed=1)
    assert X.shape == (5000, 3) and np.abs(X).max() <= 0.25
    B = workloads.uniform_ball(5000, 2, radius=1.0, seed=9)
    assert B.shape == (5000, 2) and np.linalg.norm(B, axis=1).max() <= 1.0 + 1e-12
    # uniform in the disc: the fraction inside radius 1/2 is close to 1/4
    assert abs(np.mean(np.linalg.norm(B, axis=1) <= 0.5) - 0.25) <= 0.03
