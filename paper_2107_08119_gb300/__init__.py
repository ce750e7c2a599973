"""GB300-native hot path of neuroevolution potentials (NEP, arXiv 2107.08119).

The compute path is the CUDA library ``libnep.so`` (sm_103a) behind the C ABI
declared in ``include/nep.h``; :mod:`.nep` is its Python binding.  Importing
the package itself loads nothing, so the seeded input generators in
:mod:`.inputs` stay usable without a GPU.
"""
__all__ = ["inputs", "nep", "build"]
