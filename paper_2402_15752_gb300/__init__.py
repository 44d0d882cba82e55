"""GB300-native phase-field lattice Boltzmann with interfacial mass/heat transfer."""
