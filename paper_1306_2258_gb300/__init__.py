"""GB300-native direct Debye summation for small-angle scattering profiles."""
