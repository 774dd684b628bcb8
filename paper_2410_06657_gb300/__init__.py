"""GB300-native phase-field lattice Boltzmann step for electrofreezing."""
