"""GB300-native per-event matrix elements for the MG5aMC workflow (arXiv:2106.12631)."""
