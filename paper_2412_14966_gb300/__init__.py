"""GB300-native primary-vertex finding and fitting (arXiv:2412.14966, Sec. 3)."""
