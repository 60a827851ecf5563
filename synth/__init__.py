"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the benchmark.

This package only builds inputs (meshes, scenes, count-image sets, small geometric fixtures).
It contains none of the RICI method's arithmetic, so neither side of a parity comparison can
leak into the other through it.
"""
from . import meshes, scenes, images, fixtures  # noqa: F401
from .scenes import Scene, tiny_scene, clutter_scene, large_scene, scene_batch  # noqa: F401
