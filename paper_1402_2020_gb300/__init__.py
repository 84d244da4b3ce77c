"""GB300-native Binary Stereo Matching (Zhang et al., Sec. 3): CUDA kernels behind a C ABI.

The compute path is ``libbsm.so`` (sm_103a). ``paper_1402_2020_gb300.bsm`` is its thin ctypes
binding; ``paper_1402_2020_gb300.synth`` draws seeded synthetic inputs.
"""
__all__ = ["bsm", "synth"]
