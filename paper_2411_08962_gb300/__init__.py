"""GB300-native nuclear two-point correlators (plane-wave sink, block algorithm).

The hot path lives in the CUDA library `libwick.so` (sources in `csrc/`, C ABI
in `include/wick.h`); `wick` is its thin Python binding and `operators` builds
the integer operator weight tables the ABI takes.  `synth` generates seeded
synthetic propagators.  Nothing here falls back to CPU arithmetic: loading the
binding without the compiled library raises.
"""
__all__ = ["synth", "operators", "wick"]
