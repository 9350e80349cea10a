"""GEEK on GB300: bucketing, SILK seeding and one-pass assignment.

The library is libgeek.so (C ABI in include/geek.h, CUDA kernels for
sm_103a); ``geek`` is its thin Python binding.  Importing the binding fails
loudly when the library has not been built: there is no CPU fallback.
"""
from .build_ext import build  # noqa: F401


def binding():
    from . import geek
    geek.lib()
    return geek
