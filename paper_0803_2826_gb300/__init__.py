"""GB300-native fluctuating D3Q19 lattice Boltzmann with point-particle coupling."""
