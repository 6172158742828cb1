"""GB300-native Mixture Graph: build, forward TF propagation, box-histogram
queries by footprint assembly and reverse weight push, and ray-sample lookup.

The compute path is the C-ABI library ``_build/libmg.so`` (declared in
``include/mg.h``); ``paper_2009_02702_gb300.mg`` is its thin Python binding.
Importing the package does not load the library; the first call into the
binding does, and fails loudly if it is missing.
"""
__all__ = ["mg", "synth", "build"]
