"""GB300-native critical-point probability fields (arXiv 2407.18015)."""
