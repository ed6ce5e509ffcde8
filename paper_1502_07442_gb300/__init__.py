"""GB300-native multi-species TreePM force (arXiv:1502.07442, "ngravs").

The compute path is the C-ABI CUDA library ``libngravs.so`` built from
``csrc/``; ``binding`` marshals torch tensors into it. Importing the package
does not load the library; the first call does, and fails loudly when the
library is missing.
"""
__all__ = ["inputs", "binding"]
