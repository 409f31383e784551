"""B300-native delayed geometric-network simulator (Buibas & Silva, arXiv:0908.3934).

``paper_0908_3934_b300.geonet``  ctypes binding of the C-ABI library ``libgeonet.so``
``paper_0908_3934_b300.netgen``  seeded synthetic network generators

Importing the package loads nothing; the binding loads the CUDA library on first use
and raises if it is missing.
"""
