"""Seeded synthetic snapshot streams shared by the oracle tests and the device tests.

This package only draws inputs: it holds none of the online-DMD arithmetic, so the
oracle and the CUDA path stay independent while still being fed identical bytes.
"""
from .fields import PlantedModes, WakeField, RandomPlanted, wake_grid_shape

__all__ = ["PlantedModes", "WakeField", "RandomPlanted", "wake_grid_shape"]
