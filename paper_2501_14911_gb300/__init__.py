"""GB300 (sm_103a) block-Toeplitz Bayesian inversion: Python binding of libbti.

The compute path is the CUDA library ``libbti.so`` built from ``csrc/``; this
package only marshals arguments to its C ABI.  The library is loaded on first
use, so importing the package (or its ``synthetic`` input generator) works on a
machine without a GPU; any call into the library then fails loudly if the
shared object is missing.
"""
