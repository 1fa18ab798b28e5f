"""GB300-native generalized vec trick (GVT) pairwise-kernel library."""
