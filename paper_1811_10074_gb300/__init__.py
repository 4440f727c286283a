"""GB300-native sliding window sums and minimizers (arXiv 1811.10074)."""
