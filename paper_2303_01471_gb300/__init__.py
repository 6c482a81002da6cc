"""GB300-native simulator of Quantum Hamiltonian Descent (arXiv 2303.01471).

The product is libqhd.so (C ABI in include/qhd.h, CUDA kernels for sm_103a);
`paper_2303_01471_gb300.qhd` is its thin Python binding.  Importing this
package loads nothing; `qhd.load()` builds/loads the library.
"""
__all__ = ["qhd", "build"]
