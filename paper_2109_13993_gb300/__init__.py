"""GB300-native DirectLiNGAM causal-ordering library (ParaLiNGAM's hot path).

The computation lives in the CUDA library built from csrc/ (C ABI in
include/lingam.h); `lingam` is its Python binding and `synth` the seeded
synthetic-data generator.
"""
from . import synth  # noqa: F401
