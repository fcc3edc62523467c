"""GB300-native entropic (KBC) D3Q27 lattice Boltzmann step with Grad
moving-wall boundaries and momentum-exchange coupling (arXiv 1608.04658).

The compute path is liblbm.so (CUDA, sm_103a) behind the C ABI in
include/lbm.h; this package is its Python binding.
"""
from .builder import build  # noqa: F401
from .binding import (  # noqa: F401
    BODY_AIRFOIL, BODY_MESH, BODY_NONE, BODY_PLANES, BODY_SPHERE, FACE_EQ, FACE_OUTFLOW, FACE_PERIODIC, FACE_WALL,
    GAMMA_ANALYTIC, GAMMA_EXACT, GAMMA_LBGK, STORAGES, AdjointSpec, BodyState, Geometry, Lattice, LbmError, Params,
    Refinement, airfoil, declared_symbols, fine_nu, lib, make_params, planes, sphere, swimmer,
)
from .autograd import KinematicsObjective, kinematics_objective  # noqa: F401,E402
