"""GB300-native SBP-SAT solver for the 2-D anisotropic elastic wave equation on curvilinear
multiblock grids (Almquist & Dunham).  The compute path is the CUDA library ``libsbp.so``
(built in-tree for sm_103a by ``build.build()``); ``binding.Solver`` marshals arguments."""
from .binding import Batch, Solver, SbpError, lib, header_functions  # noqa: F401
