"""Seeded synthetic ptychography scans (inputs only).

This package draws the random quantities a reconstruction starts from: the
object, the probe modes, the scan positions and the recorded intensities.
It is shared by the FP64 oracle, the CUDA path, the tests and the benchmark,
and it holds none of the difference-map iteration itself.
"""
from .scan import (WORKLOADS, BATCH16, batch16_configs, Scan, make_scan, grf_object, gaussian_probe,
                   hg_probe_modes, raster_positions, simulate_intensities,
                   initial_guess, random_exit_waves,
                   random_exit_waves_device)

from . import warmstart

__all__ = ["warmstart", "WORKLOADS", "BATCH16", "batch16_configs", "Scan", "make_scan", "grf_object", "gaussian_probe",
           "hg_probe_modes", "raster_positions", "simulate_intensities",
           "initial_guess", "random_exit_waves",
           "random_exit_waves_device"]
