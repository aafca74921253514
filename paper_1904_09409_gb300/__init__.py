"""GB300-native funnel transform (Wei, Feng & Zheng, arXiv:1904.09409).

``funnel``  ctypes binding of libfunnel.so (include/funnel.h)
``synth``   seeded synthetic line images (pictures only)
``build``   in-tree nvcc build of libfunnel.so for sm_103a
"""
