"""Plain FP64 CPU oracle for the Cholesky-factorised Sigma(2) propagator.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` may import this package.  The
GPU library never calls it and shares no code with it; the two meet only in
the seeded inputs drawn by ``workloads``.

Modules (each function cites the part of the paper it restates):

* ``eri``    -- product densities and s-Gaussian electron-repulsion
                integrals (Sec. II.A, Eq. integral), Boys F0.
* ``cd``     -- threshold-delta diagonal-pivoted Cholesky decomposition of
                the ERI supermatrix in the Gram-Schmidt form of Sec. II.A
                (Eq. gs_coulomb and the normalisation n_K, Eq. CD), full and
                atomic (one-centre) pivot sets.
* ``ao2mo``  -- AO->MO transform of the Cholesky vectors (Eq. transformation)
                and MO integrals from factors (Eq. aomo).
* ``sigma2`` -- diagonal second-order self-energy and its energy derivative
                (Eq. SE, Eq. ps); spin-orbital and MP2 (Eq. MP2) forms used as
                independent pins.
* ``qp``     -- Newton quasiparticle solve (Eq. qpapp, Eq. iter, Eq. ps, Eq. NR).
* ``grad``   -- implicit derivative of a converged quasiparticle energy.

Every floating-point step is IEEE binary64.  Functions are written for
clarity, not speed: library primitives (matmul, erf, eigh) serve as steps but
nothing is blocked, fused or reordered beyond the definitions.
"""
