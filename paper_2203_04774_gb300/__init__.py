"""GB300-native triangle listing with a given vertex ordering (arXiv:2203.04774)."""
