"""Pins for the oracle's k-nearest-neighbour search (Sec. 4.6, Sec. 4.7) -- CPU only.

* A hand-made 1-D example whose neighbour lists and distances are written out.
* Ties (duplicate points, symmetric points) go to the smaller index.
* Brute force on a tiny set by an independent route: the full distance matrix
  from numpy broadcasting, ordered by a lexicographic sort on (distance, index).
* Distances are invariant under translations and rotations, so the lists are.
"""
import numpy as np

from oracle.knn import knn


def test_hand_example_on_a_line():
    # points 0, 1, 3, 6, 10 on a line
    P = np.array([[0.0], [1.0], [3.0], [6.0], [10.0]])
    idx, d2 = knn(P, P, 2, exclude_self=True)
    np.testing.assert_array_equal(idx, [[1, 2], [0, 2], [1, 0], [2, 4], [3, 2]])
    np.testing.assert_array_equal(d2, [[1, 9], [1, 4], [4, 9], [9, 16], [16, 49]])
    # a separate query set: 2.5 is nearest to 3, then 1
    idx, d2 = knn(np.array([[2.5], [8.0]]), P, 3)
    np.testing.assert_array_equal(idx, [[2, 1, 0], [3, 4, 2]])
    np.testing.assert_array_equal(d2, [[0.25, 2.25, 6.25], [4, 4, 25]])


def test_ties_go_to_the_smaller_index():
    P = np.array([[0.0, 0.0], [1.0, 0.0], [-1.0, 0.0], [0.0, 1.0], [1.0, 0.0]])
    idx, d2 = knn(P[:1], P, 4, exclude_self=False)
    # 0 itself, then the three points at distance 1 in index order (1, 2, 3)
    np.testing.assert_array_equal(idx, [[0, 1, 2, 3]])
    idx, _ = knn(P, P, 1, exclude_self=True)
    assert idx[1, 0] == 4 and idx[4, 0] == 1       # duplicates are each other's nearest


def test_brute_force_by_broadcasting():
    rng = np.random.default_rng(3)
    P = rng.standard_normal((60, 5))
    Q = rng.standard_normal((9, 5))
    for A, exclude, k in ((P, True, 7), (Q, False, 11)):
        D = ((A[:, None, :] - P[None, :, :]) ** 2).sum(-1)
        idx, d2 = knn(A, P, k, exclude_self=exclude)
        for q in range(A.shape[0]):
            cand = np.arange(P.shape[0])
            dq = D[q]
            if exclude:
                keep = cand != q
                cand, dq = cand[keep], dq[keep]
            order = np.lexsort((cand, dq))[:k]
            np.testing.assert_array_equal(idx[q], cand[order])
            np.testing.assert_allclose(d2[q], dq[order], rtol=1e-12)


def test_rigid_motions_keep_the_lists():
    rng = np.random.default_rng(4)
    P = rng.standard_normal((80, 6))
    Rq, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    a, _ = knn(P, P, 10, exclude_self=True)
    b, _ = knn(P @ Rq + 3.0, P @ Rq + 3.0, 10, exclude_self=True)
    np.testing.assert_array_equal(a, b)
