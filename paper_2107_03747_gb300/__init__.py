"""GB300-native twisted Wilson flow (arXiv:2107.03747, Sec. 3.1): CUDA kernels behind a C ABI.

``binding`` loads ``libtgf.so`` (built by ``build.build()``) and exposes the C entry points with
the same names; ``inputs`` holds the seeded synthetic input generators.
"""
