"""FP64 CPU oracle for the ISDF-xTC kernel build -- TEST INFRASTRUCTURE.

A plain, slow, step-by-step restatement of the paper's method used only to
check the CUDA library.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path; its one compiled part (the order-exact
pivot loop, ``pivots.c``) is built by ``oracle/build_oracle.py``.

Modules and the passages they follow:
  orbitals  -- phi_p(r_g) and grad phi_p(r_g)            (Alg. 2 step 2)
  jastrow   -- u, grad_1 u of the Boys-Handy correlator  (Eqs. bh-scaled, bh-u)
  pivots    -- weighted pivoted Cholesky + fusion        (Alg. 1, Sec. II.D)
  fit       -- least-squares ISDF fit, xi and xi~        (Eq. isdf-rho)
  wbuild    -- u^(1),c and u^(3) kernels                 (Eqs. K1-isdf, K3-isdf)
  xtc       -- G_nu, calG, D^(1), D^(4), X^(2), X^(3)    (Sec. III.B)
  energies  -- K, Delta U four-index forms and energies  (Eqs. K-recombine-final,
                                                          xtc-deltah, xtc-const)
  adjoint   -- dL/dtheta of the kernels                  (not in the paper)
  mlp       -- learned interpolation-point proposer      (not in the paper)
"""
