"""GB300-native LSH top-k multidimensional motif search (MOMENTI, arXiv 2502.14446)."""
