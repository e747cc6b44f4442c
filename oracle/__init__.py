"""Plain, slow, FP64 CPU oracle for the SCH particle-filter hot path.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import or run this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline``
/ ``--impl reference`` legs of ``bench.py`` use it.  It shares no code with the
CUDA library under ``paper_2402_06927_gb300/``; the only inputs both sides
receive are the seeded arrays of the separate ``workloads`` module.

Contents (paper: Cotter, Crisan, Singh, "Data assimilation for the stochastic
Camassa-Holm equation using particle filtering", arXiv 2402.06927):

* ``rng``     Philox4x64-10 counter-based generator (Salmon et al., SC'11) and
              the Box-Muller normal transform; keyed draws for every random
              choice of the method.
* ``model``   P1 finite elements on the periodic mesh, the Helmholtz relation
              between u and m (Eq. sde1, first line), SALT mode noise (Sec. 2),
              the implicit-midpoint step (Eq. fde1) solved by a linearly-implicit
              Picard iteration, and an independent Gauss-quadrature residual.
* ``filter``  likelihood (Eq. loglikeq), ESS (Eq. ess), adaptive tempering
              (Sec. 3.1.2), systematic resampling (Sec. 3.1.1), PCN jittering
              (Sec. 3.1.2), the discrete Girsanov weight (Eq. girsanov DG approx)
              and the EMRE / RB / RES diagnostics (Sec. 4.1.1).
* ``nudge``   the nudging cost and its gradient by the forward tangent-linear
              model, and the optimisation schedules of Sec. 3.1.3.
* ``convnet`` the FP64 reference of the learned drift proposal network.

Parity pins live in ``tests/test_oracle_*.py``.  Functions that no pin fixes
say "parity unpinned" in their docstring.
"""
