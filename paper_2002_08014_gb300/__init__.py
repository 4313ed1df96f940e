"""GB300-native LocalPower: the data-parallel hot path of "Communication-Efficient
Distributed SVD via Local Power Iterations" (Li, Wang, Chen & Zhang, ICML 2021)
as a CUDA library for sm_103a with a C ABI (include/localpower.h).

``binding`` marshals arguments to that library; ``build`` compiles it in-tree.
Importing the package loads nothing: the library is loaded on first use, and a
missing or unbuildable library is an error (there is no CPU path).
"""
__all__ = ["binding", "build"]
