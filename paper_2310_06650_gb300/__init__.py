"""GB300-native QuasiGrad hot path: penalized AC-UC objective + gradient and projected Adam.

The compute lives in libqg.so (hand-written sm_103a CUDA behind the C ABI of
include/qg.h); `paper_2310_06650_gb300.qg` is its ctypes binding.
"""
__version__ = "0.1.0"
