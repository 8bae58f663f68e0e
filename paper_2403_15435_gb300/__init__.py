"""GB300-native GeoFlood wave-propagation hot path (arXiv 2403.15435).

The compute path lives in the CUDA C-ABI library built from ``csrc/``; the
Python binding in :mod:`paper_2403_15435_gb300.geoflood` only marshals
arguments.  ``inputs`` builds seeded synthetic workloads.  Importing the
package loads nothing; the binding loads the shared library on first use and
raises if it is missing.
"""
