"""Seeded synthetic inputs shared by the tests, the smoke check and the
benchmark.  Circuits, the QPU stand-in (statevector simulation of every
subcircuit variant) and the workload recipes live here; none of the
reconstruction's arithmetic does."""
from .circuits import Block, CutCircuit, chain_grid_circuit, chain_line_circuit, random_block_circuit
from .qpu import full_circuit_probs, random_variant_probs, subcircuit_variant_probs
