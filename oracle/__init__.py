"""Plain FP64 CPU oracle for the DFPT Hubbard-parameter path (arXiv:2203.15684).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` may import it.  The CUDA library never calls it, shares
no code with it, and the product fails loudly when its extension is missing instead of falling
back to this package.

The oracle follows the paper's definitions step by step in the paper's order, with numpy's FFT,
matmul and LAPACK eigensolvers as the only library primitives:

  model.py        cell, G-spheres, FFT-grid maps, closed-form form factors          (Sec. 2.2, 2.3)
  xc.py           LDA (Slater exchange + Perdew-Zunger 1981 correlation), V_xc, f_xc
  hamiltonian.py  H.psi through the grid, the same operator as a dense matrix
  groundstate.py  fixed-occupation SCF, occupation matrices (Eq. occ_matrix_0)
  response.py     self-consistent q-specific Sternheimer solve (Eqs. LRKSeq_lp, vpert,
                  proj_v, proj_c, occ_matrix_response_lp_2), modified Broyden mixing
  hubbard.py      q-sum with phases (Eq. occ_matrix_response_lp_1), chi0/chi, U and V
                  (Eqs. chi, U_def, V_def)
  sos.py          bare response by sum over states from full diagonalisation (pin)
  fd.py           finite-difference response of SCF occupations (pin)

Every function is pinned by a ``-m "not gpu"`` test (tests/test_oracle_*.py) against closed
forms, brute force, or an independent route to the same number; none is "parity unpinned".
"""
