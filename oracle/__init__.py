"""CPU FP64 oracle for the tetrahedral-stencil FFT homogenization solver.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, calls or
executes this package: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may use it.  It shares no code with the CUDA
path; the only common module is ``synth`` (seeded inputs, no solver
arithmetic).

Modules
-------
``tetra``   Algorithm 1 (displacement form) literally in q-space, in the
            paper's own Fourier convention, plus the strain form (Algorithm 2),
            the symbols ``D(q)``, the Green function ``Omega(q)`` and the
            strain Green operators (Sections 2.2-2.6).
``dense``   A brute-force real-space solve of the same discrete equilibrium on
            tiny grids: the energy of Eqs. (Elast_energy_k, Elast_energy) is
            assembled as a dense quadratic form from the real-space difference
            operators of Eqs. (DA1-DA2) and minimised with a pseudo-inverse.

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
(closed forms, invariants, the paper's identities, brute force, library
FFTs).  The iteration counts the paper prints are context only.
"""
