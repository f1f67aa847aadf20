"""GB300-native spectral Differentiable Poisson Surface Reconstruction (DPSR),
the layer of Shape As Points (arXiv 2106.03452, Sec. 3.1), forward and
backward, behind the C-ABI library libdpsr.

The compute path runs only in the hand-written CUDA kernels of libdpsr; this
package marshals arguments. Importing it does not load the library; the first
call that needs it does, and fails loudly when it is missing.
"""
__all__ = ["synth"]
