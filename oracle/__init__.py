"""FP64 CPU oracle for the two-site DMRG effective-Hamiltonian path.

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
numpy (float64) statement of what the GPU library computes, written from the
ITensor paper (arXiv:2007.14822). Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it. The product path (the
CUDA library and its Python binding) never imports, links or calls anything
here, and nothing here imports the product.

Modules
  blocksparse  QN indices, flux rule, block-sparse tensors, labelled
               contraction over shared labels (paper Sec. 3, 4, 6, 8, 9.1-9.4)
  models       site operators and finite-state MPOs (Heisenberg Eq. (1) of
               Sec. 7.1, plus TFIM, J1-J2 chain/cylinder, Hubbard)
  dmrg         H_eff application, environment update, two-site theta,
               Lanczos, truncated SVD, two-site DMRG sweeps (Sec. 5, 7.2)
  ed           exact diagonalisation from operator terms (pins only)

Every function states the passage it follows. Where the paper is silent the
reading used is stated in the docstring. Parity of each function is pinned
by the ``-m "not gpu"`` tests in ``tests/test_oracle_*.py``.
"""
