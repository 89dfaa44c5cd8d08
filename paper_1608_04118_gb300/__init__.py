"""GB300 (sm_103a) implementation of the three-distribution MRT lattice
Boltzmann step for porous convection under local thermal non-equilibrium
(Liu & He, arXiv:1608.04118).

``ltne`` binds the C ABI of ``libltne.so`` (include/ltne.h); ``workloads``
holds the seeded synthetic inputs; ``build`` compiles the CUDA library.
"""
__all__ = ["ltne", "workloads", "build"]
