"""GB300-native Fourier-Galerkin Boltzmann-Nordheim collision operator (Mouton & Rey, arXiv:2110.13735)."""
