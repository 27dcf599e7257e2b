"""GB300-native Rosenbluth chain growth (Guo & Baulin, arxiv 1704.04381).

The compute path is librosen.so (hand-written CUDA for sm_103a behind the C
ABI in include/rosen.h); ``paper_1704_04381_gb300.rosen`` is its thin Python
binding and ``paper_1704_04381_gb300.build`` compiles it.
"""
__all__ = ["rosen", "build"]
