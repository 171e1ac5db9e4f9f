"""FP64 CPU oracle of the volumetric curvilinear lattice Boltzmann method.

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and the
CPU-baseline leg of bench.py. The product package never imports it.
"""
from .vlbo import (OracleSim, cell_geometry, collide, equilibrium, lattice, load,  # noqa: F401
                   position, set_threads)
