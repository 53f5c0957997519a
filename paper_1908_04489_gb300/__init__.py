"""GB300-native coordinate-descent sweep of the generic UCP solver.

The compute path lives in the CUDA library ``libucp.so`` (C ABI declared in
``include/ucp.h``); :mod:`paper_1908_04489_gb300.binding` marshals arguments
to it.  Importing this package does not load the library; the binding loads
it on first use and raises if it is missing.
"""
