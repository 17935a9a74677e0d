"""Plain FP64 CPU oracle for the volumetric Fourier-transform reconstruction.

TEST INFRASTRUCTURE ONLY.  This package is the slow, obviously-correct
restatement of Section III-A/III-B/III-C/III-E of Alexiadis et al. (IEEE TCSVT 2017,
arXiv 1712.03084) against which the CUDA path is checked.  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / reference leg
of ``bench.py`` may import it.  The product path (the C-ABI library and its
Python binding) never imports, calls or links anything here, and this
package never imports the product path.

Every function works in float64 on float32 inputs promoted to float64 and
cites the passage of the paper it follows.  Readings of points where the
paper is silent are named constants (``oracle.conventions``).

Modules
  raw        points, normals, confidences from depth maps           (Sec. III-A)
  fft        own mixed-radix Stockham FFT + brute-force DFT        (Sec. III-B)
  splat      weighted Gaussian splat eq.(1)(2), simple splat        (Sec. III-B)
  spectral   integration filter jw/|w|^2, inverse transform         (Sec. III-B)
  level      iso-level L = mean of A at the input samples           (Sec. III-B)
  mc_table   marching-cubes case table generated from a face rule   (Sec. III-B, [35])
  mc         marching cubes (classes, vertices, normals, triangles) (Sec. III-B)
  texture    per-vertex visibility, weights, UVs, blended colour    (Sec. III-C)
  render     depth / colour-per-vertex / multitexture rendering     (Sec. III-C, III-E)
  evaluate   VRE, 2D Hausdorff, CP-RMSE, WMS3IM                     (Sec. III-E, eq. (3)-(7))
  pipeline   the whole per-frame path in the paper's order

Parity status: every function is pinned by ``tests/test_oracle_*.py``
(closed forms, brute force, invariants); none is "parity unpinned" except
the paper-level vertex-count sanity range, which has no dataset to pin to.
"""

# submodules are imported explicitly by their users (e.g. ``from oracle import fft``)
