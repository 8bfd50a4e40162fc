"""GB300 (sm_103a) state-vector simulator for the computation defined in QCLAB
(Keip, Camps, Van Beeumen, arXiv:2503.03016).

All simulation work runs in the CUDA library behind include/qc.h; this package is
its Python binding (argument marshalling) plus a torch-facing convenience layer.
"""
from ._binding import *  # noqa: F401,F403
from ._binding import lib, QCError, Circuit, Hamiltonian  # noqa: F401
from .state import State  # noqa: F401
from .autograd import AdjointExpectation  # noqa: F401,E402
from .simulate import simulate, reduced_statevector, counts  # noqa: F401,E402
from .qasm import to_qasm, from_qasm, GateOp  # noqa: F401,E402
