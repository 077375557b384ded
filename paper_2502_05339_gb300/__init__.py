"""GB300-native DMD / DMDc hot path (fit by randomized SVD, batched exponential
integration, hand-written adjoint) behind the C ABI of libdmd.

Submodules: `dmd` (the binding of libdmd), `synth` (seeded input generators),
`build_lib` (in-tree nvcc build).
"""
