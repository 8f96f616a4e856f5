"""Seeded synthetic inputs for the non-isothermal single-phase flow problem.

This package only draws random fields and lays out wells and physical
constants. It holds none of the discretisation, linear algebra or
preconditioning arithmetic; both the CUDA path and the CPU oracle consume
what it produces.
"""
from .fields import gaussian_random_field, iid_log_normal, channelised, layered
from .recipes import make_problem, RECIPE_SHAPES, default_fluid, bennison_oil, scaling_case

__all__ = [
    "gaussian_random_field", "iid_log_normal", "channelised", "layered",
    "make_problem", "RECIPE_SHAPES", "default_fluid", "bennison_oil", "scaling_case",
]
