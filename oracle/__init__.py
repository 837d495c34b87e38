"""FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library under
``paper_2207_00933_gb300`` never does: it shares no code, headers, tables or
helpers with this package, and it fails loudly when its CUDA extension is
missing rather than falling back here.

Pins (tests/test_oracle_pins.py): full-circuit statevector brute force on
small circuits (Eq. 1 end to end), the zero-cut identity, total probability
1, children bins summing to their parent, all-merged = 1, every contraction
order equal to the bin-by-bin Eq. 1 sum, and the worked cost numbers of
Section 6.2-6.3.
"""
from .reconstruct import (ACTIVE, MERGED, ZOOM0, ZOOM1, D, W, Graph, attribute,
                          attribute_literal, merge, reconstruct, reconstruct_bruteforce,
                          reconstruct_pairwise, subcircuit_tensors, top_bins, total_probability)
from .plan import (greedy_slicing, naive_multiplications, roles_for_recursion, sliced_sizes,
                   states_assignment, step_multiplications, tensor_floats)
