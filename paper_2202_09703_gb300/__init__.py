"""GB300-native multi-layer collimated-beam MBIR (hot path: A, A^T and the MAP step)."""
