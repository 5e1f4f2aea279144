"""GB300-native TRAPHIC transport sweep with recombination radiation (arXiv:1311.0182)."""
