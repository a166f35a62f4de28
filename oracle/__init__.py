"""FP64 CPU oracle for the phaseless-AFQMC hot path (TEST INFRASTRUCTURE ONLY).

This package is the slow, plain reference that the CUDA library is checked
against.  Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg
of ``bench.py`` may import it; the product path never calls it and shares no
code with it (the only common dependency is the seeded input generator
``synthetic_inputs``, which holds none of the method's arithmetic).

Modules
-------
philox  Philox4x32-10 counter-based generator (Salmon et al., SC'11) and the
        Box-Muller normal transform with its own log / sin / cos, so that the
        auxiliary fields x of Eq. 8 are reproducible bit for bit.
afqmc   the method: set-up (Eqs. 3-6, the mean-field shift of Eq. 12), overlap
        and Green's function, force bias (Eq. 12), the propagator B(x - xbar)
        of Eqs. 8 and 10, the hybrid / phaseless weights (Eqs. 11, 13-16), the
        mixed local energy (Eq. 9), QR stabilisation and comb population
        control, and free projection (Section "Free projection AFQMC").
fci     brute-force Fock-space operators for tiny systems; used only to pin
        the oracle (overlaps, Green's functions, force bias, local energy and
        the propagator against exact many-body quantities).

Every function cites the passage it follows.  Pins: see tests/test_oracle_*.py.
Parity status: every function listed above is pinned; the physical-scale
results on the synthetic workloads are "parity unpinned" beyond agreement with
this oracle, because the paper prints no numbers for them.
"""
