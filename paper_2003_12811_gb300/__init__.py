"""GB300-native SBP-SAT solver for the 2-D anisotropic elastic wave equation on curvilinear
multiblock grids (Almquist & Dunham), with the 3-D operator on one curvilinear block.  The
compute path is the CUDA library ``libsbp.so`` (built in-tree for sm_103a by ``build.build()``);
``binding.Solver`` and ``binding.Solver3D`` marshal arguments."""
from .binding import Batch, Solver, Solver3D, SbpError, lib, header_functions  # noqa: F401
