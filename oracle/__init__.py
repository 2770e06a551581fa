"""Oracle for the higher-order time-evolution MPO method of arXiv:2302.14181.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import, call, link or
execute this package: only the tests, ``__graft_entry__.smoke()`` and the CPU
legs of ``bench.py`` (``cpu_baseline`` and ``--impl reference``) use it. It shares no code with the CUDA library.

Plain, slow, fp64-complex CPU code, written from the paper:

* ``oracle.mpo``   -- powers of the Hamiltonian MPO (Sec. 2.5) and Algorithms 1-4
                      (Secs. 3-6) giving the order-N MPO W^(N)(tau), densified per site.
* ``oracle.fit``   -- single-site variational fit of W|psi> back to bond dimension D
                      (Sec. 2.2, Table 1 "(i)DMRG" row; benchmark set-up of Sec. 8.2),
                      Householder QR, local expectation values, overlaps.
* ``oracle.dense`` -- dense references for small chains: H from the finite-state
                      expansion of Sec. 2.3, the dense MPO, exp(tau H) by eigh.

Parity pins (tests/test_oracle_*.py) tie each function to what the paper and the
mathematics fix; see the header of each module for what is pinned.
"""
