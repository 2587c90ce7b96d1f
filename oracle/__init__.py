"""Plain, slow CPU FP64 oracle of Adaptive-Multilevel BDDC (Sousedik, Sistek, Mandel).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or
link this package: only `tests/`, `__graft_entry__.smoke()` and the
`cpu_baseline` / `--impl reference` legs of `bench.py` use it.  It shares no
code with the CUDA path; both sides consume the seeded inputs of
`amb_inputs` and nothing else.

Modules
  fe        Q1 finite elements on a uniform hexahedral grid (Sec. 2)
  levels    substructuring of one level: interface, faces/edges/corners,
            local matrices, constraints, weights, Schur complements and the
            coarse basis (Sec. 2, Sec. 4 eq. def-Wtilde-dual, Sec. 5 eq.
            local_saddle_point_problem and the coarse-matrix identity)
  pair      the pairwise generalized eigenproblems and adaptive rows
            (Sec. 4 eq. eig-matrix, eq. d-def, Prop. 1; Sec. 7.2)
  solver    set-up (Algorithm 3), the Multilevel BDDC preconditioner
            (Algorithm 1), PCG with the Lanczos condition estimate (Sec. 8)
  gradient  adjoint gradient of a quantity of interest w.r.t. log-coefficients

Parity status of each function is stated in its docstring ("pinned by ..."
or "parity unpinned").
"""
