"""GB300-native circuit-coupled electrostatic PIC with ion-induced SEE."""
