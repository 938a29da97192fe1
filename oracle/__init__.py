"""CPU oracle for the two-site gate path (TEST INFRASTRUCTURE).

A plain, slow, obviously correct complex128 restatement of the paper's method:
Householder QR with column pivoting stopped at chi_max pivots (oracle/src,
Sec. III-B.2), MPS gate application, SWAP routing, centre moves, amplitudes
and the norm fidelity (oracle/mps.py, Sec. III-C and III-E), and a
brute-force statevector (oracle/statevector.py) that checks the oracle itself.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this package.  The GPU library shares no code with it.
"""
