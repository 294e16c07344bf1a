"""FP64 CPU oracle for the reconstruction hot path of Modi, Feng & Seljak (2018).

TEST INFRASTRUCTURE ONLY. This package is a plain, slow, obviously correct
restatement of what the method computes, written from the paper in numpy and
scipy at float64. It exists to check the CUDA path. Only the test suite,
``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The product path never calls it and never
falls back to it.

It shares no code with the CUDA library: no kernels, headers, tables, constant
generators or pre/post-processing. Both sides receive the same seeded random
draws from ``paper_1805_02247_gb300.synth`` (which holds none of the method's
arithmetic) and compute everything else independently.

Modules
-------
cosmo   background expansion, linear growth D(a), BBKS power spectrum, sigma8
pm      mesh conventions, linear field, Zel'dovich ICs, CIC paint/readout,
        PM force, kick-drift-kick stepping and the hand-written adjoint
nn      the 81-50-30-1 network of Sec. 2.1 on the 27-point stencil of Sec. 2.2
loss    the loss of Eq. (loss) (Sec. 5.1) and its gradient w.r.t. s(k)
lbfgs   the L-BFGS step of Sec. 5.2 (two-loop recursion, Armijo backtracking)
anneal  the stages of the annealed reconstruction (Sec. 5.2-5.3)
twopt   the binned two-point statistics of Sec. 4.3

Parity status: every function here is pinned by a ``-m "not gpu"`` test
(closed forms, invariants, brute force, finite differences, and the values the
paper prints, kept under tests/golden/) except the whole annealed
reconstruction outcome, which the paper cannot fix on synthetic data; the
annealing driver itself (stage order, stop rule, line search) is pinned on
hand-solvable objectives.
"""
