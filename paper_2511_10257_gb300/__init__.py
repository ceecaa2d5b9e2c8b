"""GB300-native enthalpy lattice Boltzmann flux solver (LBFS) time step."""
