"""GB300-native two-component pseudopotential D3Q19 lattice Boltzmann step."""
