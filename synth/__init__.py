"""Seeded synthetic inputs (meshes, query points, nodal fields) for the findpts
hot path.

This package only *generates inputs*. It performs none of the point-location
or interpolation arithmetic: node positions are placed by closed-form maps of
a tensor-product reference grid, query points are random draws or copies of
mesh nodes with random offsets, fields are closed-form functions sampled at the
nodes. Both the CUDA path and the CPU oracle consume what it produces; neither
shares any other code.
"""
from .meshes import *  # noqa: F401,F403
