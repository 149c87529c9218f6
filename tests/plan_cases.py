"""Workloads of the GPU tests whose plans must have a given structure (a
tensor-core step, sliced or grouped labels).  The GPU tests use them, and
tests/test_plan_structure.py checks the structure on the host, so that a
planner change cannot silently turn a GPU test into one that no longer
exercises what it names.  Data only."""

# 20 qubits, 16 bitstrings, 2 open legs: a node on the tcgen05 tensor cores
TC_CASE = dict(shape=(4, 5, 10, 2), open=[0, 3], batch=16)

# one sliced label runs grouped (as a batch index up to the root) beside serial ones
GROUPED_CASE = dict(shape=(4, 5, 10, 2), batch=4, cap=13480, max_group_log2=6)

# memory caps of the slicing tests on the 4 x 5 depth-10 circuit (open legs 0, 7, two bitstrings)
SLICING_CAPS = [(1 << 16, 0), (1 << 15, 3), (1 << 14, 6)]
PARTIAL_CASE = dict(open=[1], batch=2, cap=1 << 16, max_group_log2=0)

# the 6 x 6 depth-16 reduction of the 8 x 8 depth-16 workload: cap that slices it
RAND6X6_D16_CAP = 256 << 20

# the 8 x 8 depth-16 workload at full size
RAND8X8_D16_CAP = 180 * 10**9
