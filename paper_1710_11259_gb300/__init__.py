"""GB300-native spectral Poisson ADI solver (Fortunato & Townsend, arXiv 1710.11259)."""
