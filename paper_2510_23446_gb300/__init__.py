"""GB300 tree-cotree IETI-DP eddy-current solver.

``ieti`` is a thin ctypes binding of the C ABI in ``include/ieti.h`` (argument
marshalling only: all setup and solve work runs in ``libieti.so``).  Importing it
loads the in-tree library and fails loudly when it has not been built.
"""
