"""FP64 CPU oracle of the stable parareal-like method (Nguyen & Tsai, arXiv 1905.00473).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
execute this package: only the tests, the smoke check and the CPU-baseline leg
of the benchmark do.  It shares no code with the CUDA path.

Every function is a plain, slow, readable restatement of the paper's
definitions in float64 (numpy), each citing the section, equation or
algorithm it follows:

* ``fine``      -- the fine/coarse time stepper (Sec. 3.1): periodic
                   2nd-order central Laplacian and velocity Verlet; F over
                   all slices of one iteration.
* ``energy``    -- the gradient approximations nabla_h, the discrete wave
                   energy (Sec. 3.1, eq. discrete-wave-energy) and the error
                   measures of Sec. 6.
* ``transfer``  -- restriction R, Fourier interpolation I, the energy maps
                   Lambda and Lambda^dagger (grad2func, Alg. 2).
* ``procrustes``-- the orthogonal Procrustes corrector and UpdateSVD (Alg. 1).
* ``parareal``  -- the proposed method (Alg. 3), its Omega = 1 and plain
                   parareal variants and the serial fine reference.

Parity pins (tests/test_oracle_*.py) tie these to closed forms, invariants
and the paper's printed numbers: exact discrete plane waves, the exactly
conserved modified energy of velocity Verlet, time reversibility, Fourier
symbols of nabla_h and of Lambda^dagger Lambda, R I = 1, brute-force
Procrustes optimality, incremental = batch SVD, finite termination of the
iteration after N sweeps, and both columns of the Sec. 6.4 table.
"""
