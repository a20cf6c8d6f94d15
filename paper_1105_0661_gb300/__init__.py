"""GB300-native LOFAR station-to-beam library (Mol & Romein, "The LOFAR Beam Former").

The compute path is the CUDA library built from csrc/ (sm_103a); `lbf` is its Python binding.
"""

from .lbf import Batch, LbfError, Plan, load_library  # noqa: F401
