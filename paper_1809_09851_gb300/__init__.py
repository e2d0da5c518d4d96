"""GB300-native Euler building blocks (FDBB hot path), placeholder."""
