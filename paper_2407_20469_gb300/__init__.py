"""GB300-native per-tile APIC reconstruction (WSI-APIC, arXiv 2407.20469).

The compute path is the C-ABI library ``libapic.so`` (hand-written CUDA for
sm_103a, declared in ``include/apic.h``); ``apic`` is its thin Python binding.
``synth`` holds the seeded synthetic-input recipes.
"""
from . import synth  # noqa: F401

__all__ = ["synth", "apic", "build"]
