"""Plain, slow CPU oracle of fast spectral clustering (Macgregor, NeurIPS 2023).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may use it.  It shares no code with
the CUDA library (no kernels, headers, helpers or constants); the only common
dependency is the seeded input generator package ``workloads``.

Floating point is float64 throughout, except where the method turns floating
point into an integer decision (k-means++ sampling, Lloyd's argmin): there the
oracle takes the decision in the precision the CUDA kernels use (float32
squared distances in a fixed operation order), so the two sides can be compared
decision by decision.

Modules
-------
rng       Philox4x64-10 (Salmon et al., SC'11) and Box-Muller Gaussians.
spectral  degree, Laplacians, signless Laplacian M (Sec. 2), PowerMethod
          (Algorithm 1), the embedding of Algorithm 2, dense spectra.
eig       cyclic Jacobi eigensolver for small symmetric matrices.
kmeans    k-means cost (Sec. 2.2), k-means++ seeding and Lloyd iterations.
metrics   ARI, NMI, misclassified volume (Theorem 3.2), Frobenius cost form.
cluster   Algorithm 2 end to end.
filter    Chebyshev polynomial filters p(M), graph features, the filter MLP
          in float64 with hand-written backward pass.

Pinned functions and their pins are listed in ``tests/test_oracle_*.py``.
Parity unpinned: ``filter.mlp_*`` against the paper (the learned filter is not
in the paper; its gradients are pinned by finite differences only).
"""
