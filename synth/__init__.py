"""Seeded synthetic inputs shared by the oracle and the CUDA path.

This package only synthesises raw array data and workload descriptions.  It
holds none of the windowed beamspace MVDR arithmetic (no channeliser, no
beamspace transform, no window, covariance or solve), so that the oracle and
the CUDA path stay independent of each other.
"""
from .scene import (
    SceneConfig,
    Scene,
    config_by_name,
    all_configs,
    make_scene,
    pulse,
    reference_records,
    scaled_config,
)

__all__ = [
    "SceneConfig",
    "Scene",
    "config_by_name",
    "all_configs",
    "make_scene",
    "pulse",
    "reference_records",
    "scaled_config",
]
