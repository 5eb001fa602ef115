"""GB300-native forward model of disc-galaxy kinematics (Bekiaris et al. 2015).

The compute lives in libgbk.so (CUDA, sm_103a; C ABI in include/gbk.h).
``gbk`` is its Python binding, ``synth`` draws the seeded synthetic inputs.
"""
from . import synth  # noqa: F401

__all__ = ["gbk", "synth", "build"]
