"""GPU (B300, sm_103a) evaluation of AC optimal power flow NLP callbacks.

``opf``    the binding of libopf (include/opf.h): models, patterns, bounds,
           and the fused FP64 evaluation kernels
``synth``  seeded synthetic grids and evaluation points
"""
__all__ = ["opf", "synth"]
