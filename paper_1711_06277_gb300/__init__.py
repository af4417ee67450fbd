"""GB300-native adaptive ray tracing of point sources through a uniform grid
(Kim, Kim, Ostriker & Skinner 2017, Sec. 2): a CUDA library behind a C ABI
(``include/art.h``) and a thin Python binding.

Importing the package does not load the CUDA library; ``paper_1711_06277_gb300.art``
does, and fails loudly if it cannot be built or loaded.
"""

__all__ = ["art", "synth", "build"]
