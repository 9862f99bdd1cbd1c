"""GB300-native 2D Serre-Green-Naghdi hot path (spectral RHS + GMRES + RK4).

The CUDA library ``libsgn.so`` is loaded lazily by :mod:`.sgn` on first use;
importing this package loads nothing.
"""
