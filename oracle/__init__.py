"""CPU oracle of the NIRC hot path -- test infrastructure only.

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never uses it.
"""
