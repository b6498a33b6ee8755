"""GB300-native OCD soft-output detection for massive MU-MIMO-OFDM."""
