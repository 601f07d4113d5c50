"""FP64 CPU oracle for the Galactic-Binary likelihood hot path (test infrastructure).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and
the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it. The
product path (``paper_2405_04690_gb300``) never imports, links or calls anything here,
and this package imports nothing from the product path. The two share no code, no
constants and no tables; each writes its own from the paper.

Contents (each function cites the passage of arXiv:2405.04690 it follows):

* ``constants``  -- physical constants and the observation grid (Sec. III, Eq. psd).
* ``orbits``     -- analytic equal-arm constellation (the paper cites it but gives no
                    model: first-order-in-eccentricity heliocentric orbits).
* ``psd``        -- Eq. psd with S_pm/S_op, and the Galactic foreground (Sec. III.A).
* ``waveform``   -- GB TDI A/E band by the fast/slow decomposition (App. F, Sec. II.A),
                    plus the brute-force time-domain response used to pin it.
* ``likelihood`` -- Eq. inner, Eq. like, Eq. addsource, Eq. swapsource.
* ``residual``   -- fixed-point residual add/subtract (bit-exact inverse).
* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al. 2011).
* ``mcmc``       -- Eq. rj-acceptance, Eq. temp-orig / temp-final, Alg. 1 and Alg. 2.

Everything is float64 numpy; loops are plain Python where the paper's algorithm is
sequential. Nothing here is blocked, fused or reordered beyond the definitions.
"""
