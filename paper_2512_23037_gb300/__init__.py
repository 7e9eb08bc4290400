"""GB300-native generalized-stabilizer shot simulator (arxiv 2512.23037 hot path)."""
