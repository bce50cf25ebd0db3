"""GB300-native exact reverse k-MIPS (Simpfer) library."""
