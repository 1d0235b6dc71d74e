"""GB300 (sm_103a) renderer for sparse factorized HRIRs (Luo, Zotkin & Duraiswami,
"Sparse Head-Related Impulse Response for Efficient Direct Convolution").

Modules
  hrir   ctypes binding of the C ABI (include/hrir.h); the CUDA library does all the work
  synth  seeded synthetic inputs (sources, directions, filters)
  build  compiles csrc/*.cu into _lib/libhrir.so for sm_103a
"""
__all__ = ["hrir", "synth", "build"]
