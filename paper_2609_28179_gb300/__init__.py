"""GB300-native batched small-matrix linear algebra (GLASS hot path)."""
