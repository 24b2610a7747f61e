"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench."""
from .seismic import (Channel, Fault, Salt, VolumeSpec, make_volume, random_volume,  # noqa: F401
                      ricker, sample_points, small_spec, spec_for, volume)
