"""Seeded synthetic inputs shared by the CUDA path and the CPU oracle.

This package holds no arithmetic of the method itself: it only writes down
meshes of the unit cube, subdomain partitions, viscosity fields and load
functions, all from fixed seeds.  Both the library tests and the oracle read
the same arrays from here.
"""
from .mesh import cube_mesh, octa_mesh, cvt_mesh, box_partition, greedy_partition, element_vertex_average
from .fields import (manufactured_u, manufactured_f, sinker_centres,
                     sinker_viscosity, sinker_load)
from .configs import make_config, CONFIGS

__all__ = ["cube_mesh", "octa_mesh", "cvt_mesh", "box_partition", "greedy_partition",
           "element_vertex_average", "manufactured_u", "manufactured_f",
           "sinker_centres", "sinker_viscosity", "sinker_load",
           "make_config", "CONFIGS"]
