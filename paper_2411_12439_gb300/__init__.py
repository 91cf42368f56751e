"""GB300 library for stable locally consistent grammars (arXiv 2411.12439).

BuildGram, MergeGrams and exp(S) run in hand-written CUDA kernels for sm_103a
behind the C ABI of ``include/lcg.h``; this package is its Python binding.
"""
from .lcg import Context, Grammar, LCGError, PPGrammar, load, library_path  # noqa: F401

__all__ = ["Context", "Grammar", "LCGError", "PPGrammar", "load", "library_path"]
