"""GB300-native real-time TD-DFTB density-matrix propagator (C-ABI library + thin binding)."""
