"""The PCO work count the benchmark reports (the paper's update count U_m,
Sec. II C and App. B) equals the loop trip counts of the paper's algorithms
as the oracle's vector sets (Alg. 1) and compositions (Alg. 3) enumerate
them.  CPU only."""
import numpy as np
import pytest

import bench
from oracle import basis as B
from oracle import mps as M


def trip_count(bl, br, d, Q=None):
    """Updates of every PCO, counted entry by entry from the oracle's vector
    sets with the kappa-match condition of Alg. 2."""
    bp = B.single_mode_basis(d)
    spaces = ([(0, bl, q) for q in range(bl.ne)] + [(1, bp, 0)]
              + [(2, br, q) for q in range(br.ne)])
    dims = (bl.D, d, br.D)
    U = 0
    for z1 in range(len(spaces)):
        for z2 in range(z1, len(spaces)):
            if Q is not None and Q[z1, z2] == 0:
                continue
            ax1, b1, q1 = spaces[z1]
            ax2, b2, q2 = spaces[z2]
            v1 = B.vector_set(b1, q1)
            if z1 == z2:                                  # Alg. 5: even kappa
                rest = np.prod([dims[i] for i in range(3) if i != ax1])
                U += int((v1.vord % 2 == 0).sum()) * rest
            elif ax1 != ax2:                              # Alg. 2: equal kappa
                v2 = B.vector_set(b2, q2)
                third = [i for i in range(3) if i not in (ax1, ax2)][0]
                for k in np.unique(v1.vord):
                    U += int((v1.vord == k).sum()) * int((v2.vord == k).sum()) * dims[third]
            else:                                         # Algs. 3-4
                comp = B.compose(v1, B.vector_set(b2, q2))
                rest = np.prod([dims[i] for i in range(3) if i != ax1])
                U += comp.vord.size * rest
    return U


@pytest.mark.parametrize("seed,nl,nr,d,chil,chir", [
    (0, 2, 3, 4, 12, 15), (1, 0, 2, 5, 1, 20), (2, 3, 0, 3, 25, 1), (3, 4, 4, 6, 70, 90),
    (4, 1, 1, 8, 33, 47)])
def test_pco_update_count_equals_algorithm_trip_counts(seed, nl, nr, d, chil, chir):
    r = np.random.default_rng(seed)
    bl = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nl))[::-1], chil) if nl else M.vacuum_basis()
    br = B.kept_basis(np.sort(r.uniform(0.05, 0.4, nr))[::-1], chir) if nr else M.vacuum_basis()
    assert bench.pco_update_count(bl.occ, br.occ, d) == trip_count(bl, br, d)
    n = nl + 1 + nr
    Q = r.standard_normal((n, n))
    Q = Q + Q.T
    Q[0, n - 1] = Q[n - 1, 0] = 0.0
    Q[n // 2, n // 2] = 0.0
    assert bench.pco_update_count(bl.occ, br.occ, d, Q) == trip_count(bl, br, d, Q)
