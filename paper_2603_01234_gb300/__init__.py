"""GB300-native (sm_103a) NEP evaluator for NEP-CG / NEP-AACG (arXiv 2603.01234).

The evaluation (cell list, neighbour lists, descriptors, network, forces, virials,
velocity-Verlet) runs in the CUDA library built from csrc/ and is reached through
the C ABI in include/nep.h; `binding` marshals arguments to it.  `inputs` holds
the seeded synthetic configurations.  Importing the package loads nothing; the
library is loaded on first use and its absence is an error.
"""
__all__ = ["binding", "inputs", "build"]
