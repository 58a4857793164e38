"""GB300-native exact warehouse pick routing.

Batched multi-source Bellman-Ford distance rows and exhaustive pick
sequence evaluation, as hand-written sm_103a CUDA behind a C ABI
(include/wroute.h).  `wroute` is the Python binding; `synth` draws
seeded synthetic layouts and orders.
"""
__all__ = ["wroute", "synth"]
