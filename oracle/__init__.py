"""Plain FP64 CPU reference of the SLIM boundary-element system (test infrastructure only).

This package is the oracle the CUDA path is checked against. It is slow and written for a
reader: every function follows one passage of the paper (cited by section and equation) or,
where the paper defers to another work, the reading of it that the project adopted. It shares
no code with the CUDA library; only the seeded input generator
(`paper_2108_03991_gb300.synth`) feeds both.

Only the test-suite, the smoke check and the benchmark's CPU-baseline leg may import it. The
product path never does.

Modules
  rwg        mesh -> RWG basis / pulse basis data (Sec. II)
  quad       triangle quadrature rules and closed-form potential integrals
  operators  Galerkin matrices L^A, L^Phi, I_x, F, D, L_k, K_k and the SLIM system
             (Sec. II-A/B/C, Eqs. AEFIEsys, MFIEinZin, EFIEeqYeq, AEFIEoutJ, Cdef)
  aim        adaptive integral method L = L_NR + W H P (Sec. III-A item 1, Eq. AIM_L)
  gmres      restarted GMRES (Sec. III-E)
  farfield   radiated far field, monostatic RCS and the Mie series (Sec. IV-A validation)
  ports      delta-gap port excitation and port currents
  sched      LPT (Alg. 1) and modified Part_Schedule (Alg. 2)
  blockops   block-diagonal GEMV (Sec. II-C, block diagonal Z and Y_eq)
  precond    block-diagonal preconditioner (the fallback of the constraint preconditioner)
  constraint the constraint preconditioner (near-field system, sparse LU)
  highk      large-|k_i| integrals of the lossy conductors (Sec. II-B)
  convnet    the learned correction's conv net
  sparse_internal  sparse internal operator at high frequency (Sec. III-A)
  sibc       surface-impedance boundary condition (the comparison model of Sec. I)
  ground     a PEC ground plane under the background, by images (Table I's bottom layer)
  layered    Green's functions of Table I's stratified backgrounds (same-layer, Toeplitz +
             Hankel in z) and the grid step inside a layer

Parity pins: every function is pinned in tests/test_oracle_*.py against closed forms,
exactness on polynomials, brute force on tiny inputs, invariants or the Mie series. No function
is "parity unpinned".
"""
