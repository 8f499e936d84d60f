"""GB300-native binned FFT kernel density estimation with unconstrained bandwidth."""
