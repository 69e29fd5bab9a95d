"""FP64 CPU oracle for the Gaussian-state -> MPS method of arXiv:2512.10643.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-correct
restatement of what the paper defines.  Only the test-suite, the smoke check
and the CPU-baseline leg of the benchmark may import it; the product library
(``paper_2512_10643_gb300``) never does, and the two share no code.  Library
primitives (numpy eigh/inv/det/matmul, sort) serve as steps; nothing is
blocked, fused or reordered beyond what the paper states.

Modules
  gaussian : covariance <-> paired form, Williamson, Bogoliubov (U,V),
             regularised Q_L, iterative GSVD chain           (Sec. II A-B, App. A)
  basis    : kept subspace, truncation error, vector sets    (Sec. II C, App. B Alg. 1, 3)
  pco      : projected-creation-operator tensor build        (Sec. II C, App. B Alg. 2, 4, 5)
  mps      : full build, environments/normalisation, amplitudes, sampling,
             fidelity
  hafnian  : brute-force hafnian amplitudes (exact reference for tiny cases)
  filtration: mixed -> pure decomposition of a lossy covariance (Sec. III, App. C)

Every public function is pinned by a check that does not reuse its own code
path (closed forms, brute-force hafnians, dense inner products and matrix
exponentials, identities of App. A); a function without such a pin would say
"parity unpinned" in its docstring, and none does.  ``gaussian.williamson_sqrt``
is a second valid FP64 route to the Williamson form, kept to measure how far
the MPS of a given covariance matrix is determined in FP64 at all.
"""
from . import gaussian, basis, pco, mps, hafnian, filtration  # noqa: F401
from .mps import build_mps, amplitudes, sample, environments, fidelity, normalise  # noqa: F401
