"""Plain FP64 CPU oracle for the preconditioned orbital minimization method.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
leg use it.  It shares no code with the CUDA path (no kernels, headers, tables or
constant generators); both sides receive the same seeded inputs from `workloads`.

Each function states the passage of the paper (Lu & Yang, "Preconditioning orbital
minimization method for planewave discretization", arXiv:1603.09724) it follows.  The
code is deliberately slow and direct: dense matrices, explicit DFT matrices, numpy
linear algebra, pocketfft only where an FFT of a grid function is the definition.

Modules
  hamiltonian  pseudospectral H (Sec. 4 Test 1, eq. ex1mat), dense and FFT forms
  omm          E_omm (eq. omm), gradient (Sec. 2.1), Hessian, quartic line search,
               preconditioned nonlinear CG (Algorithm 1)
  poles        pole expansion of the Fermi projector (Sec. 3.1, eq. dFOP)
  sparsify     sparsifying preconditioner (Sec. 3.2, eqs. GLu, QG, P)
  gmres        restarted right-preconditioned GMRES (Sec. 3.1 eq. lst, Sec. 4 params)
  precond      the preconditioner P = sum_j w_j (H - z_j)^-1 applied to a block
  gtpa         Fourier-diagonal comparison preconditioners (Sec. 2.2, eqs. Lap, TPA,
               gTPA) and their scale tau (Sec. 4)
  metrics      principal angles, d(X, X0) (Sec. 4), condition number (Sec. 2.3)

Parity status: every function here is pinned by a -m "not gpu" test against a closed
form, an invariant, a brute-force evaluation or a textbook special case; see
tests/test_oracle_*.py.  Nothing is "parity unpinned".
"""
