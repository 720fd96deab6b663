"""dbnet: GB300 (sm_103a) kernels for the hot path of the Digital Brain
(conductance LIF networks with delayed spike delivery, the Balloon-Windkessel
BOLD readout, and the diffusion ensemble Kalman filter of HMDA), behind the C
ABI in include/dbnet.h.  ``dbnet`` is the ctypes binding; ``_build`` compiles
the library in place."""
from . import dbnet  # noqa: F401
from .dbnet import Network  # noqa: F401
