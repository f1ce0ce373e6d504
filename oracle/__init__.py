"""Serial FP64 CPU oracle of the p-multigrid compact gas-kinetic scheme.

Test infrastructure only (tests, smoke check, CPU baseline of the bench);
the product library never imports it.  See ``oracle.oracle``.
"""
