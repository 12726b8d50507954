"""CPU oracle for the sparse spectral method (Gross & Iwen, arXiv 2302.00752).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 restatement of
the paper's definitions, used to check the CUDA library.  Only the test suite,
the smoke check and the benchmark's CPU-baseline leg may import it; the
library itself never does, and the two share no code (they share only the
seeded draws in ``workloads.py``).

Modules and the parts of the paper they follow:

  lattice   rank-1 lattices, the reconstructing property, the random-lattice
            size rule (Section "Previous results on SFTs", Definition of
            Lambda(z, M); Lemma RandomRank1Lattice) and a component-by-component
            search (named in Section "Improvements with randomized lattices").
  sft       lattice sampling and coefficient recovery by the plain DFT of the
            samples (Fourier coefficient definition, Section 2; Theorem
            SFTRecovery in known-support form).
  stamp     stamping sets S^N by breadth-first Minkowski sums (eq. StampSet,
            Proposition SolutionSupport) and the cardinality bounds of
            Lemma StampSetCardinality / Lemma StampSizeUpperBound.
  galerkin  the Galerkin operator written out as an explicit sparse matrix
            (eq. GF, eq. FiniteGalerkinOperator) and the exact convolution that
            manufactures f from u.
  solve     Jacobi-preconditioned CG, dense LU and the tridiagonal chain solve
            for the one-term problem (Algorithm 1, last step; the diagonal
            rearrangement in the proof of Proposition SolutionSupport).
  adr       the advection-diffusion-reaction operator of Remark ADR (union
            step set, explicit matrix, exact convolution, direct solve, proxy).

Parity status of every function is stated in its module header.
"""
