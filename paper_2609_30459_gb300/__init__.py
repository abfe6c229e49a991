"""GB300-native stereo visual frontend (VkVIO, arxiv 2609.30459).

The compute path is a C-ABI CUDA library (``libvio.so``, declared in
``include/vio.h``); :mod:`paper_2609_30459_gb300.vio` is its thin ctypes
binding. :mod:`paper_2609_30459_gb300.synth` makes seeded synthetic inputs.
"""
__all__ = ["vio", "synth"]
