"""CPU oracle for the MBT array solve -- TEST INFRASTRUCTURE ONLY.

Plain, slow, complex128 numpy/scipy code that states what the solver must
compute, used to check the CUDA library.  Only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import it; the library never
does, and nothing here imports the library.

What it computes (the method reaches the plain solution of Eq. 15, Z I = V, Sec.
III-A: the preconditioned normal equations have the same solution):

* dense.py     -- assemble the dense Z from the unique offset blocks (Eq. 1,
                  Sec. II-A) and solve by LAPACK LU.
* mbt.py       -- the MBT product by its definition (direct sum over
                  offsets), Z^H, the diagonal blocks of Z^H Z (Eq. 37), and
                  the circulant-embedded transformed blocks (Eqs. 3, 7, 11).
* ports.py     -- active impedance (Eqs. 16-17), passive port impedance
                  (Eq. 18) and active reflection coefficient (Eq. 19).
* iterative.py -- for sizes whose dense Z does not fit in memory: restarted
                  GMRES on the ORIGINAL system Z I = V with a block-Jacobi
                  preconditioner and the direct offset-sum product (no FFT,
                  so no algorithm in common with the CUDA path).
* predictors.py -- the error predictors of Sec. II-E: xi (Eq. 20), the
                  border bound (Eq. 23), xi_Z (Eqs. 24-25), the column
                  coupling C_n (Eqs. 28-30), S <-> Z (Eq. 31) and xi_S
                  (Eq. 36).

Pins (tests/test_oracle_*.py): brute-force inversion, exact reciprocity and
Toeplitz invariants of the assembly, per-entry recomputation from the
lattice geometry, closed forms for 1x1 and two-element arrays, the Hermitian
commutation theorem (Eq. 6) and circulant-embedding identity (Eq. 3), equal
spectra of the two preconditioned forms (Sec. III-A), agreement of the two
active-impedance routes, dense-vs-iterative agreement, and for the
predictors: the 1x1 reflection coefficient and uncoupled / matched special
cases of S <-> Z, Fourier coefficients of exp(a e^{j psi}) (a^n / n!), exact
recovery of trigonometric polynomials, the theta substitution, hand-counted
border sets, and the border bound holding when a lattice grows.
Parity is pinned for every function here; none is "parity unpinned".
"""
from . import dense, mbt, ports, iterative, predictors  # noqa: F401
