"""GB300-native batched 1D-TDSE engine (length-gauge Crank-Nicolson, arXiv:2507.04115 Sec. 3.1, 4.2).

The compute path is the C-ABI library ``libtdse.so`` (hand-written CUDA for sm_103a); this
package holds its Python binding (``tdse``) and the seeded input generators (``inputs``).
Importing the package does not load the library; ``tdse.load()`` does, and fails loudly if
the library has not been built.
"""
