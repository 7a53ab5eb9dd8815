"""GB300-native functional-map hot path (DeepShapeMatchingKit, arXiv 2604.10377, Sec. 3.1).

Modules:
  api    -- flat-buffer batches, the C-ABI calls, and the autograd Function (needs torch)
  _lib   -- ctypes binding of libfmap.so (include/fmap.h)
  synth  -- seeded synthetic inputs (no functional-map arithmetic)
  build  -- nvcc build of libfmap.so for sm_103a
"""
