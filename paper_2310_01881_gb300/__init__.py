"""GB300-native Adaptive Multi-NeRF rendering hot path (arXiv 2310.01881)."""
