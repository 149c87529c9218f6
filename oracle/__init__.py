"""FP64 CPU oracle for quantum-circuit amplitudes <x| C |0...0>.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this package: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference leg use it.  It shares no code with the CUDA
executor; it reads circuits only through the plain gate-list data produced by
``circuits``.

The contraction order never changes the value of a tensor network (the
separator hierarchy of the Thm. 1 proof, and the greedy leaves of the
"Numerical implementation" section, only change its cost), so the oracle is
the plain definition of the amplitude, computed four independent ways:

* :mod:`oracle.statevector` -- explicit time evolution of the state vector
  (the "explicit time evolution" baseline of the Thm. 2 discussion), which
  also gives c = <0| U^dagger P U |0> and marginal probabilities by their
  definitions;
* :mod:`oracle.sidewise` -- naive-order (left-to-right, "side-wise")
  contraction of the circuit's tensor network;
* :mod:`oracle.stabilizer` -- exact Clifford amplitudes in the CH form
  (Bravyi, Browne, Calpin, Campbell, Gosset, Howard, Quantum 3, 181 (2019));
* :mod:`oracle.iqp` -- closed forms for IQP circuits H D H (a Walsh-Hadamard
  transform, and a column transfer-matrix sum).

Every function returns complex128 amplitudes ``out[b, j]`` for bitstrings
``bits[b]`` with the open qubits ``open_qubits`` ranging over all values: bit
``i`` of ``j`` is the value of ``open_qubits[i]`` (ascending qubit order).
"""
from .statevector import statevector, statevector_amplitudes, statevector_expectation, statevector_marginal
from .sidewise import sidewise_amplitudes
from .stabilizer import CHForm, stabilizer_amplitudes
from .iqp import iqp_wht_amplitudes, iqp_transfer_amplitudes
from .common import expand_open, rel_error

__all__ = [
    "statevector", "statevector_amplitudes", "statevector_expectation", "statevector_marginal",
    "sidewise_amplitudes", "CHForm",
    "stabilizer_amplitudes", "iqp_wht_amplitudes", "iqp_transfer_amplitudes",
    "expand_open", "rel_error",
]
