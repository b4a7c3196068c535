"""CPU oracle for TTN / ML-MCTDH projector-splitting time evolution.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
its Python binding) imports or calls this package; only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` do.

Everything here is plain complex128 NumPy/SciPy: per-term sum-of-product
environments with no term grouping, mode products through ``tensordot``,
textbook Householder QR, Lanczos/Arnoldi with full re-orthogonalisation and a
dense small exponential, and the recursive projector-splitting step.  Each
function names the paper passage it follows.

Pinned against (tests/test_oracle_*.py): brute-force dense effective
Hamiltonians and environments built from explicit single-particle and
single-hole basis vectors, exact state-vector propagation (full bond
dimension is exact), norm and energy conservation, second-order convergence,
closed-form dynamics (free spin, free oscillator, independent-boson
decoherence), LAPACK QR, dense matrix exponentials, and for the HEOM
generator a hierarchy assembled element by element from the free-pole HEOM
equation with exact trace conservation and the pure-dephasing closed form.
"""
