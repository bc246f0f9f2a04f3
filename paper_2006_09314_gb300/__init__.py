"""GB300-native solver for the control equation of the tensor method for
optimal control constrained by a fractional 3D elliptic operator with
separable variable coefficients (arXiv 2006.09314).

The compute path is the CUDA library libtensorctl.so (include/tensorctl.h);
`tensorctl` is its thin Python binding and `inputs` the seeded problem
generator.
"""
