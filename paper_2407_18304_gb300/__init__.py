"""GB300 implicit multigroup matter-radiation source-term update.

``rhd`` is the Python binding of the C ABI (include/rhd.h) of the CUDA
library; ``synth`` draws seeded synthetic cell states; ``build`` compiles the
library in-tree for sm_103a.
"""
from . import build, rhd, synth  # noqa: F401
