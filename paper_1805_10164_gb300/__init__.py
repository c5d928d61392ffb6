"""GB300-native Monte Carlo NEGF walk library (Musland, Bergli, Flage-Larsen,
arXiv:1805.10164): RGF transition tables, persistent Philox random walks over Buttiker-probe
sites and the lead-current tally, as CUDA kernels for sm_103a behind the C ABI of
include/negf.h.

Submodules: ``negf`` (ctypes binding, C entry point names), ``build`` (nvcc build of
libnegf.so), ``inputs`` (seeded synthetic wires), ``session`` (convenience wrapper).
Importing the package loads nothing; ``negf.load()`` loads the library and fails loudly if it
has not been built.
"""
__all__ = ["negf", "build", "inputs"]
