"""GB300-native two-range pseudopotential lattice Boltzmann for binary
mixtures with tunable viscosity ratio (Fei et al., arXiv:1806.06943).

The compute path is the CUDA library ``liblb.so`` built from ``csrc/``; the
Python layer in ``lb.py`` only marshals arguments to its C-ABI.  Importing this
package does not load the library; ``paper_1806_06943_gb300.lb`` does, and it
raises if the library has not been built.
"""

__all__ = ["lb", "workloads"]
