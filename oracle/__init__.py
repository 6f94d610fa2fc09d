"""FP64 CPU oracle of graph-neural-ansatz variational Monte Carlo (arXiv:2011.12453).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow restatement of what the
method computes, written from the paper's definitions in numpy float64.  Only the
tests, the smoke check and the CPU-baseline leg of the benchmark may import it; the
library's product path never does, and this package shares no code with the CUDA
sources (it does not import them, nor they it).

Modules and the passages they follow:

* ``gcn``        -- the GCN wavefunction: Eq. (gcn) and the embedding/readout
                    description of the GNA section; the two-unit complex head follows
                    the two-head suggestion of the conclusion.
* ``heisenberg`` -- the local energy E_x = sum_x' H_xx' Psi_x'/Psi_x of the scaling
                    section (Heisenberg bond form), the S_z-sector Hamiltonian, exact
                    diagonalisation and the variational energy E_v(w).
* ``sampler``    -- MCMC sampling of P ~ |Psi|^2 (scaling section) with
                    pair-exchange Metropolis moves, driven by Philox4x64-10
                    (Salmon et al., SC'11) restated from its published definition.
* ``isgo``       -- the importance-reweighted gradient of Eq. (isgo), with the
                    hand-derived reverse-mode derivative of log Psi.
* ``stats``      -- integrated autocorrelation time with automatic windowing.

Parity pins for every function are in ``tests/test_oracle_*.py``.  Parity unpinned:
none of the functions here; the trained-parameter energies of the large systems have
no closed form and are compared against this oracle only.
"""
