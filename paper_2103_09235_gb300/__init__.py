"""GB300-native folded-stencil library (temporal computation folding, Li et al.).

Importing the package loads nothing compiled.  ``binding`` loads the CUDA
library and fails loudly when it has not been built; ``synth`` draws seeded
inputs.
"""

__all__ = ["binding", "synth"]
