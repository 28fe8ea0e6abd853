"""Reference oracle for phaseless finite-temperature AFQMC of the 3D uniform
electron gas (Lee, Morales, Malone, arXiv:2012.12228).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, complex128 CPU
restatement of the method, written from the paper, that exists to check the
CUDA library.  Only the test-suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
The product path (``paper_2012_12228_gb300``) never imports it and shares no
code, tables or constants with it; the only module both sides use is
``synthetic_inputs`` (seeded random numbers and workload sizes, none of the
method's arithmetic).

Modules
-------
ueg      model setup: basis, momentum transfers, v(Q), HS couplings, the
         one-body correction of the sum-of-squares form, FE trial, mu_T.
ed       exact diagonalisation of the grand-canonical ensemble (M <= 7).
afqmc    walker propagation: force bias, V(x), Taylor exp, B chain, QRCP
         stabilisation, stable Green's function, phaseless / free-projection
         weights, energy and particle-number estimators.
population  comb population control between slices (the method the paper
         names in its Computational Details), with the draw passed in.

Every function cites the section / equation of the paper it follows.  Where
the paper is silent, garbled or self-contradictory the reading taken is
stated in the docstring (the same readings are listed in the design notes).
Parity of the phaseless energies at the large workloads is unpinned beyond
the internal invariants that the tests check (see ``afqmc``).
"""
