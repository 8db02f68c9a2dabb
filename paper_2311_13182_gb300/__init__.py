"""GB300-native shooting-and-bouncing-rays FMCW radar simulator (arxiv 2311.13182 hot path).

The compute path is libsbr (hand-written sm_103a CUDA behind the C ABI in
``include/sbr.h``); this package builds it in-tree and marshals torch device
memory and streams into it.  Importing the package does not build anything;
``build.build()`` does, and ``_lib.load()`` raises if the library is missing.
"""
from . import build
from ._lib import SbrError, load
from .pipeline import Forward, PipelinedForward
from .sim import (PHASE_FP64, PHASE_NAIVE, PHASE_SPLIT, SYNTH_MOVING, Adjacency, PathBuffers, PcState, Scene, adam_step,
                  cfar_struct, chamfer, grid_struct, image_loss, laplacian, pointcloud, pointcloud_bwd, power_map,
                  radar_struct, synth_ws_bytes, synthesize, synthesize_bwd, trace, trace_bwd)

__all__ = ["build", "load", "SbrError", "Forward", "PipelinedForward", "Scene", "PathBuffers", "PcState", "Adjacency", "trace", "synthesize",
           "synthesize_bwd", "pointcloud", "pointcloud_bwd", "power_map", "image_loss", "trace_bwd", "chamfer", "laplacian", "adam_step",
           "synth_ws_bytes", "radar_struct", "grid_struct", "cfar_struct", "PHASE_SPLIT", "PHASE_FP64",
           "PHASE_NAIVE", "SYNTH_MOVING"]
