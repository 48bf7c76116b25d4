"""Plain, slow, FP64 CPU oracle for sketched FOM / sketched GMRES (Guettel &
Schweitzer, "Randomized sketching for Krylov approximations of large-scale
matrix functions").

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The product path (the C ABI in ``include/skf.h`` and its Python
binding) never calls it, and it shares no code with the CUDA path: the only
common inputs come from the ``workloads`` package (seeded operators and
right-hand sides, no method arithmetic).

Modules
  sketch      the sparse-sign and SRHT embeddings S (Sec. 1, eq. (1.1)), from
              their definitions, via SplitMix64 (Steele, Lea & Flood 2014)
  quadrature  Stieltjes quadrature rules (Sec. 4.1) for z^-alpha, log(1+z)/z, 1/z
  arnoldi     k-truncated modified Gram-Schmidt Arnoldi with on-the-fly
              sketches (Algorithm 2, Sec. 2.2)
  sketched    whitening QR, sFOM closed form (sFOM'''), sFOM by quadrature
              (eq. (sFOM)), sGMRES by adaptive quadrature (eq. (sGMRES), Sec. 4.1)
  exact       reference values of f(A)b (dense Schur-based or shifted sparse solves)

Every function is pinned by ``tests/test_oracle_*.py`` against closed forms,
special cases and invariants stated in the paper.  Functions without such a
pin are marked "parity unpinned" in their docstring.
"""
